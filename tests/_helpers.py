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


def near_maps(levels, near_bits):
    """Per level of an oracle extraction, {code: bits} of its bounded cells with a non-zero near-iso
    bit set (tests/_rounding_model.near_iso_bits)."""
    out = []
    for lv, b in zip(levels, near_bits):
        sel = b != 0
        out.append(dict(zip(pack(lv["ijk"][sel]).tolist(), b[sel].tolist())))
    return out


def ancestor_bits(code, maps, L):
    """OR of the near-iso bits of the ancestors-or-self of a level-L cell."""
    ijk = unpack([code])[0]
    u = 0
    for l, m in enumerate(maps):
        if m:
            u |= m.get(int(pack((ijk >> (L - l))[None])[0]), 0)
    return u


def compare_active_pairs(o_map, g_map, maps, L):
    """(cell, iso) pairs of two active sets {code: mask}: returns (pairs in either set, differing
    pairs, pairs the band excuses, differing pairs the band does not excuse)."""
    n_pairs = n_diff = n_exc = 0
    bad = []
    for code in set(o_map) | set(g_map):
        o, g = o_map.get(code, 0), g_map.get(code, 0)
        u = o | g
        n_pairs += bin(u).count("1")
        anc = ancestor_bits(code, maps, L) if u else 0
        n_exc += bin(u & anc).count("1")
        d = o ^ g
        n_diff += bin(d).count("1")
        if d & ~anc:
            bad.append((code, o, g))
    return n_pairs, n_diff, n_exc, bad
