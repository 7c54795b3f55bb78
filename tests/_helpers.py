"""Shared test helpers (no method arithmetic: packing, comparisons, bands)."""
import numpy as np


def pack(ijk):
    ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
    return (ijk[:, 0] | (ijk[:, 1] << 10) | (ijk[:, 2] << 20)).astype(np.int64)


def unpack(codes):
    c = np.asarray(codes, dtype=np.int64) & 0xFFFFFFFF
    return np.stack([c & 1023, (c >> 10) & 1023, (c >> 20) & 1023], axis=1)


def band_codes(levels, isos, band, L):
    """Finest-level descendants are excused when an ancestor-or-self's oracle bound endpoint lies
    within `band` of an iso-value.  Returns, per level, the set of codes of such cells."""
    isos = np.asarray(isos, dtype=np.float64)
    out = []
    for lv in levels:
        near = np.zeros(lv["ijk"].shape[0], dtype=bool)
        for c in isos:
            near |= (np.abs(lv["lower"] - c) <= band) | (np.abs(lv["upper"] - c) <= band)
        out.append(set(pack(lv["ijk"][near]).tolist()))
    return out


def excused(code, band_sets, L):
    ijk = unpack([code])[0]
    for l, s in enumerate(band_sets):
        a = ijk >> (L - l)
        if int(pack(a[None])[0]) in s:
            return True
    return False


def to_np(t):
    return t.detach().cpu().numpy()
