"""ctypes binding of the C interface in include/isx.h: argument marshalling only.

Device memory and streams come from PyTorch (tensors' data pointers, torch.cuda streams); every
step of the computation runs in the library's CUDA kernels.  There is no fallback: if the
library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "libisx.so"

ISX_MAX_ISO = 32
ISX_MAX_LEVEL = 10
ISX_MC_MAX_TRI = 5

SOUND, CLT, RAUA, RAFIXED = 0, 1, 2, 3
FP32, BF16 = 0, 1
ACTS = {"relu": 0, "elu": 1, "sine": 2}
MODES = {"sound": SOUND, "clt": CLT, "raua": RAUA, "rafixed": RAFIXED}
PRECS = {"fp32": FP32, "bf16": BF16}

STATUS = {0: "ISX_OK", 1: "ISX_ERR_ARG", 2: "ISX_ERR_CUDA", 3: "ISX_ERR_CAPACITY", 4: "ISX_ERR_TIMEOUT",
          5: "ISX_ERR_UNSUPPORTED", 6: "ISX_ERR_NOMEM"}


class IsxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class KernelStats(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double)]


class InrDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("dims", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
                ("activation", C.c_int)]


class TuneEntry(C.Structure):
    _fields_ = [("key", C.c_char_p), ("choice", C.c_char_p), ("variant", C.c_int), ("n_variants", C.c_int),
                ("ms_best", C.c_float), ("ms_first", C.c_float)]


class ExtractParams(C.Structure):
    _fields_ = [("max_level", C.c_int), ("n_iso", C.c_int), ("iso", C.c_float * ISX_MAX_ISO),
                ("mode", C.c_int), ("k", C.c_float), ("prec", C.c_int), ("inflate", C.c_int),
                ("bound_stop_level", C.c_int), ("proposer", C.c_void_p), ("proposer_level", C.c_int),
                ("tau_lo", C.c_float), ("tau_hi", C.c_float), ("eval_prec", C.c_int), ("kd_tree", C.c_int),
                ("record", C.c_void_p)]


class LevelRecord(C.Structure):
    _fields_ = [("d_code", C.c_void_p), ("d_mask", C.c_void_p), ("d_center", C.c_void_p), ("d_spread", C.c_void_p),
                ("cap", C.c_int64), ("level_off", C.c_int64 * (ISX_MAX_LEVEL + 2))]


class Mesh(C.Structure):
    _fields_ = [("d_active_code", C.c_void_p), ("d_active_mask", C.c_void_p), ("active_cap", C.c_int64),
                ("d_tri_vert", C.c_void_p), ("d_tri_edge", C.c_void_p), ("d_tri_iso", C.c_void_p),
                ("d_tri_cell", C.c_void_p), ("tri_cap", C.c_int64),
                ("n_active", C.c_int64), ("n_tris", C.c_int64), ("n_points", C.c_int64),
                ("cells_bounded", C.c_int64 * (ISX_MAX_LEVEL + 1)),
                ("cells_kept", C.c_int64 * (ISX_MAX_LEVEL + 1)),
                ("ms_acp", C.c_float), ("ms_inr", C.c_float), ("ms_mc", C.c_float), ("ms_total", C.c_float),
                ("cells_visited", C.c_int64 * (ISX_MAX_LEVEL + 1))]


_lib = None


def load(path: Path | None = None):
    """Load the shared library (building nothing); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise FileNotFoundError(f"{p} is missing: run __graft_entry__.build() (or python -m "
                                f"paper_2402_13861_gb300.build) first")
    lib = C.CDLL(str(p))
    vp, i64, f32p = C.c_void_p, C.c_int64, C.POINTER(C.c_float)
    lib.isx_create_inr.argtypes = [C.POINTER(InrDesc), C.POINTER(vp)]
    lib.isx_destroy_inr.argtypes = [vp]
    lib.isx_bound_cells.argtypes = [vp, vp, vp, i64, C.c_int, C.c_int, C.c_int, vp, vp, vp]
    lib.isx_eval_points.argtypes = [vp, vp, i64, C.c_int, vp, vp]
    lib.isx_bound_cells_noalloc.argtypes = [vp, vp, vp, i64, C.c_int, C.c_int, vp, vp, vp]
    lib.isx_bound_cells_noalloc.restype = C.c_int
    lib.isx_extract_isosurface.argtypes = [vp, C.POINTER(ExtractParams), C.POINTER(Mesh), vp]
    lib.isx_extract_dense.argtypes = [vp, C.POINTER(ExtractParams), C.POINTER(Mesh), vp]
    lib.isx_mc_table.argtypes = [C.POINTER(C.c_int8), C.POINTER(C.c_int8)]
    lib.isx_last_error.restype = C.c_char_p
    lib.isx_last_error.argtypes = []
    lib.isx_version.restype = C.c_int
    lib.isx_profile_enable.argtypes = [C.c_int]
    lib.isx_profile_enable.restype = None
    lib.isx_profile_reset.argtypes = []
    lib.isx_profile_reset.restype = None
    lib.isx_profile_read.argtypes = [C.POINTER(KernelStats), C.c_int]
    lib.isx_profile_read.restype = C.c_int
    lib.isx_tune_read.argtypes = [C.POINTER(TuneEntry), C.c_int]
    lib.isx_tune_read.restype = C.c_int
    lib.isx_tune_reset.argtypes = []
    lib.isx_tune_reset.restype = None
    lib.isx_batch_create.argtypes = [C.POINTER(vp), C.POINTER(ExtractParams), C.c_int, C.c_int, C.POINTER(vp)]
    lib.isx_batch_run.argtypes = [vp, C.POINTER(Mesh), vp]
    lib.isx_batch_destroy.argtypes = [vp]
    lib.isx_proposer_create.argtypes = [f32p, f32p, f32p, C.POINTER(vp)]
    lib.isx_proposer_destroy.argtypes = [vp]
    lib.isx_proposer_get_params.argtypes = [vp, f32p]
    lib.isx_proposer_predict.argtypes = [vp, vp, i64, vp, vp]
    lib.isx_proposer_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    lib.isx_proposer_train_step.argtypes = [vp, vp, vp, i64, C.c_float, vp, vp]
    lib.isx_check_bounded_wait.argtypes = [i64, vp]
    for name in ("isx_create_inr", "isx_destroy_inr", "isx_bound_cells", "isx_eval_points",
                 "isx_extract_isosurface", "isx_extract_dense", "isx_mc_table", "isx_proposer_create",
                 "isx_proposer_destroy", "isx_proposer_get_params", "isx_proposer_predict", "isx_proposer_grad",
                 "isx_proposer_train_step", "isx_batch_create", "isx_batch_run", "isx_batch_destroy",
                 "isx_check_bounded_wait"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise IsxError(status, load().isx_last_error().decode())


def mc_table():
    """The library's marching-cubes table: (ntri[256] int8, tris[256, 5, 3] int8)."""
    lib = load()
    ntri = np.zeros(256, dtype=np.int8)
    tris = np.zeros(256 * ISX_MC_MAX_TRI * 3, dtype=np.int8)
    _check(lib.isx_mc_table(ntri.ctypes.data_as(C.POINTER(C.c_int8)), tris.ctypes.data_as(C.POINTER(C.c_int8))))
    return ntri, tris.reshape(256, ISX_MC_MAX_TRI, 3)


def profile_enable(on=True):
    load().isx_profile_enable(int(bool(on)))


def profile_reset():
    load().isx_profile_reset()


def profile_read():
    """{kernel name: dict(launches, ms, flops, bytes)} accumulated since the last reset."""
    arr = (KernelStats * 64)()
    n = load().isx_profile_read(arr, 64)
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, flops=arr[i].flops,
                                       bytes=arr[i].bytes) for i in range(n)}


def tune_read():
    """{key: dict(choice, variant, n_variants, ms_best, ms_first)} of the autotuner's cached choices."""
    arr = (TuneEntry * 256)()
    n = min(load().isx_tune_read(arr, 256), 256)
    return {arr[i].key.decode(): dict(choice=arr[i].choice.decode(), variant=arr[i].variant,
                                      n_variants=arr[i].n_variants, ms_best=arr[i].ms_best, ms_first=arr[i].ms_first)
            for i in range(n)}


def tune_reset():
    load().isx_tune_reset()


def check_bounded_wait(limit_ns, stream=None):
    """Status of the library's bounded-wait self-check (isx_check_bounded_wait): 4 (ISX_ERR_TIMEOUT)
    when the wait on a never-completed mbarrier expired as designed."""
    return int(load().isx_check_bounded_wait(int(limit_ns), _stream_ptr(stream)))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class Inr:
    """An INR resident on the current CUDA device (wraps isx_inr)."""

    def __init__(self, layers, act="relu"):
        """``layers``: (W, b) pairs, W of shape (out, in); ``act``: "relu", "elu" or "sine" (a SIREN's
        omega_0 folded into W and b)."""
        lib = load()
        self.act = act
        self.layers = [(np.ascontiguousarray(W, dtype=np.float32), np.ascontiguousarray(b, dtype=np.float32))
                       for W, b in layers]
        dims = [self.layers[0][0].shape[1]] + [W.shape[0] for W, _ in self.layers]
        self.dims = dims
        n = len(self.layers)
        c_dims = (C.c_int * (n + 1))(*dims)
        Wp = (C.POINTER(C.c_float) * n)(*[W.ctypes.data_as(C.POINTER(C.c_float)) for W, _ in self.layers])
        bp = (C.POINTER(C.c_float) * n)(*[b.ctypes.data_as(C.POINTER(C.c_float)) for _, b in self.layers])
        desc = InrDesc(n, c_dims, Wp, bp, ACTS[act])
        h = C.c_void_p()
        _check(lib.isx_create_inr(C.byref(desc), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().isx_destroy_inr(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def bound_cells(self, lo, hi, mode="sound", prec="fp32", inflate=False, center=None, spread=None, stream=None):
        """Bounds of the INR over the boxes [lo, hi] (isx_bound_cells).  lo, hi: float32 CUDA tensors
        (n, 3).  Returns (center, spread) CUDA tensors (n,): (x0, r) for sound / rafixed, (mu, sigma)
        for clt / raua."""
        import torch
        n = lo.shape[0]
        assert lo.is_cuda and lo.dtype == torch.float32 and lo.is_contiguous() and hi.is_contiguous()
        if center is None:
            center = torch.empty(n, dtype=torch.float32, device=lo.device)
        if spread is None:
            spread = torch.empty(n, dtype=torch.float32, device=lo.device)
        _check(load().isx_bound_cells(self._h, _ptr(lo), _ptr(hi), n, MODES[mode], PRECS[prec], int(bool(inflate)),
                                      _ptr(center), _ptr(spread), _stream_ptr(stream)))
        return center, spread

    def eval_points(self, xyz, prec="fp32", out=None, stream=None):
        """The MLP at float32 CUDA points (n, 3) (isx_eval_points): prec "fp32" (CUDA cores) or "bf16"
        (tensor cores with two-term bf16 operands, float32-class)."""
        import torch
        n = xyz.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=xyz.device)
        _check(load().isx_eval_points(self._h, _ptr(xyz), n, PRECS[prec], _ptr(out), _stream_ptr(stream)))
        return out

    @staticmethod
    def params(max_level, isos, mode="sound", k=3.0, prec="fp32", inflate=False, bound_stop_level=-1,
               proposer=None, proposer_level=1, tau_lo=0.0, tau_hi=1.0, eval_prec="fp32", kd_tree=False):
        p = ExtractParams()
        p.max_level = max_level
        isos = list(np.atleast_1d(np.asarray(isos, dtype=np.float32)))
        p.n_iso = len(isos)
        for q, c in enumerate(isos):
            p.iso[q] = float(c)
        p.mode = MODES[mode]
        p.k = float(k)
        p.prec = PRECS[prec]
        p.inflate = int(bool(inflate))
        p.bound_stop_level = bound_stop_level
        p.proposer = proposer.handle if proposer is not None else None
        p.proposer_level = int(proposer_level)
        p.tau_lo = float(tau_lo)
        p.tau_hi = float(tau_hi)
        p.eval_prec = PRECS[eval_prec]
        p.kd_tree = int(bool(kd_tree))
        return p

    def extract(self, max_level, isos, mode="sound", k=3.0, prec="fp32", inflate=False, bound_stop_level=-1,
                active_cap=1 << 16, tri_cap=1 << 18, dense=False, stream=None, buffers=None, proposer=None,
                proposer_level=1, tau_lo=0.0, tau_hi=1.0, eval_prec="fp32", kd_tree=False, record=False,
                record_cap=1 << 22):
        """Hierarchical (or, with dense=True, dense) extraction (isx_extract_isosurface /
        isx_extract_dense).  mode: "sound", "clt", "raua" or "rafixed"; prec / eval_prec: "fp32" or
        "bf16" (bounds and corner values on the tensor cores); kd_tree: Algorithm 1's k-d tree
        instead of the octree; bound_stop_level: bound down to that level, keep every descendant of
        the survivors; proposer (a Proposer) with proposer_level, tau_lo, tau_hi: the learned gate;
        record: also return the level loop's record (isx_level_record) as ``levels``, one dict per
        level of the visited cells' codes, inherited masks, centres and spreads.
        Grows the output buffers and retries once if a capacity is exceeded.  Returns a dict of
        tensors (codes, masks, tri_vert, tri_edge, tri_iso, tri_cell) and counters (n_active,
        n_tris, cells_bounded / cells_kept / cells_visited per level, phase times in ms).  With
        dense=True, codes / masks are the cells with triangles and the isos they have triangles for."""
        import torch
        p = self.params(max_level, isos, mode, k, prec, inflate, bound_stop_level, proposer, proposer_level,
                        tau_lo, tau_hi, eval_prec, kd_tree)
        fn = load().isx_extract_dense if dense else load().isx_extract_isosurface
        dev = torch.device("cuda", torch.cuda.current_device())
        bufs = buffers if buffers is not None else {}
        for attempt in range(3):
            if bufs.get("active_cap", -1) < active_cap:
                bufs["code"] = torch.empty(max(active_cap, 1), dtype=torch.int32, device=dev)
                bufs["mask"] = torch.empty(max(active_cap, 1), dtype=torch.int32, device=dev)
                bufs["active_cap"] = active_cap
            if bufs.get("tri_cap", -1) < tri_cap:
                bufs["vert"] = torch.empty((max(tri_cap, 1), 3, 3), dtype=torch.float32, device=dev)
                bufs["edge"] = torch.empty((max(tri_cap, 1), 3), dtype=torch.int64, device=dev)
                bufs["iso"] = torch.empty(max(tri_cap, 1), dtype=torch.int32, device=dev)
                bufs["cell"] = torch.empty(max(tri_cap, 1), dtype=torch.int32, device=dev)
                bufs["tri_cap"] = tri_cap
            m = Mesh()
            m.d_active_code = bufs["code"].data_ptr()
            m.d_active_mask = bufs["mask"].data_ptr()
            m.active_cap = bufs["active_cap"]
            m.d_tri_vert = bufs["vert"].data_ptr()
            m.d_tri_edge = bufs["edge"].data_ptr()
            m.d_tri_iso = bufs["iso"].data_ptr()
            m.d_tri_cell = bufs["cell"].data_ptr()
            m.tri_cap = bufs["tri_cap"]
            rec = None
            if record:
                if bufs.get("record_cap", -1) < record_cap:
                    bufs["r_code"] = torch.empty(max(record_cap, 1), dtype=torch.int32, device=dev)
                    bufs["r_mask"] = torch.empty(max(record_cap, 1), dtype=torch.int32, device=dev)
                    bufs["r_center"] = torch.empty(max(record_cap, 1), dtype=torch.float32, device=dev)
                    bufs["r_spread"] = torch.empty(max(record_cap, 1), dtype=torch.float32, device=dev)
                    bufs["record_cap"] = record_cap
                rec = LevelRecord()
                rec.d_code, rec.d_mask = bufs["r_code"].data_ptr(), bufs["r_mask"].data_ptr()
                rec.d_center, rec.d_spread = bufs["r_center"].data_ptr(), bufs["r_spread"].data_ptr()
                rec.cap = bufs["record_cap"]
                p.record = C.cast(C.pointer(rec), C.c_void_p)
            st = fn(self._h, C.byref(p), C.byref(m), _stream_ptr(stream))
            short = dense and st == 0 and int(m.n_active) > bufs["active_cap"]
            if (st == 3 or short) and attempt < 2:
                active_cap = max(active_cap, int(m.n_active))
                tri_cap = max(tri_cap, int(m.n_tris))
                if rec is not None:
                    record_cap = max(record_cap, int(rec.level_off[max_level + 1]))
                continue
            _check(st)
            break
        na, nt = int(m.n_active), int(m.n_tris)
        levels = None
        if rec is not None:
            off = list(rec.level_off)
            levels = [dict(codes=bufs["r_code"][off[l]:off[l + 1]], masks=bufs["r_mask"][off[l]:off[l + 1]],
                           centre=bufs["r_center"][off[l]:off[l + 1]], spread=bufs["r_spread"][off[l]:off[l + 1]])
                      for l in range(max_level + 1)]
        return dict(
            levels=levels,
            codes=bufs["code"][:na], masks=bufs["mask"][:na],
            tri_vert=bufs["vert"][:nt], tri_edge=bufs["edge"][:nt], tri_iso=bufs["iso"][:nt], tri_cell=bufs["cell"][:nt],
            n_active=na, n_tris=nt, n_points=int(m.n_points),
            cells_bounded=list(m.cells_bounded)[:max_level + 1], cells_kept=list(m.cells_kept)[:max_level + 1],
            cells_visited=list(m.cells_visited)[:max_level + 1],
            ms_acp=m.ms_acp, ms_inr=m.ms_inr, ms_mc=m.ms_mc, ms_total=m.ms_total, buffers=bufs)


PROPOSER_NPARAM = 8961


class Proposer:
    """The cell-subdivision proposer on the current CUDA device (wraps isx_proposer).

    ``params``: packed float32 vector of ISX_PROPOSER_NPARAM values (W1[64][8] b1 W2[64][64] b2
    W3[64][64] b3 W4[1][64] b4); ``mean`` / ``std``: the 8 feature standardisation constants."""

    def __init__(self, params, mean, std):
        lib = load()
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        assert params.size == PROPOSER_NPARAM
        self.mean = np.ascontiguousarray(mean, dtype=np.float32).reshape(8)
        self.std = np.ascontiguousarray(std, dtype=np.float32).reshape(8)
        h = C.c_void_p()
        f32p = C.POINTER(C.c_float)
        _check(lib.isx_proposer_create(params.ctypes.data_as(f32p), self.mean.ctypes.data_as(f32p),
                                       self.std.ctypes.data_as(f32p), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().isx_proposer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(PROPOSER_NPARAM, dtype=np.float32)
        _check(load().isx_proposer_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def predict(self, feat, out=None, stream=None):
        """Logits of feature rows (float32 CUDA tensor [n, 8])."""
        import torch
        n = feat.shape[0]
        assert feat.is_cuda and feat.dtype == torch.float32 and feat.is_contiguous()
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=feat.device)
        _check(load().isx_proposer_predict(self._h, _ptr(feat), n, _ptr(out), _stream_ptr(stream)))
        return out

    def grad(self, feat, label, stream=None):
        """(gradient [NPARAM], mean BCE) of labelled rows, without updating the parameters."""
        import torch
        g = torch.empty(PROPOSER_NPARAM, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        _check(load().isx_proposer_grad(self._h, _ptr(feat), _ptr(label), feat.shape[0], _ptr(g), _ptr(loss),
                                        _stream_ptr(stream)))
        return g, loss

    def train_step(self, feat, label, lr, loss=None, stream=None):
        """One Adam step on a labelled mini-batch; ``loss`` (CUDA float32 [1]) receives its loss."""
        _check(load().isx_proposer_train_step(self._h, _ptr(feat), _ptr(label), feat.shape[0], float(lr),
                                              _ptr(loss), _stream_ptr(stream)))


class Batch:
    """Many extractions in flight together (wraps isx_batch): every entry runs isx_extract_isosurface
    on one of ``workers`` host threads, each with its own CUDA stream.  ``nets``: Inr objects;
    ``params``: one dict of Inr.params keyword arguments per entry (max_level, isos, mode, k, prec, ...)."""

    def __init__(self, nets, params, workers=8):
        lib = load()
        self.nets = list(nets)
        self.params = [Inr.params(**p) for p in params]
        self.max_levels = [p["max_level"] for p in params]
        n = len(self.nets)
        hs = (C.c_void_p * n)(*[net.handle for net in self.nets])
        ps = (ExtractParams * n)(*self.params)
        h = C.c_void_p()
        _check(lib.isx_batch_create(hs, ps, n, int(workers), C.byref(h)))
        self._h = h
        self._bufs = [dict() for _ in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            load().isx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, active_cap=1 << 16, tri_cap=1 << 18, stream=None):
        """Runs every entry; grows the per-entry output buffers and reruns on a capacity error."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        n = len(self.nets)
        caps = [[active_cap, tri_cap] for _ in range(n)]
        for attempt in range(3):
            meshes = (Mesh * n)()
            for i, b in enumerate(self._bufs):
                ac, tc = caps[i]
                if b.get("active_cap", -1) < ac:
                    b["code"] = torch.empty(max(ac, 1), dtype=torch.int32, device=dev)
                    b["mask"] = torch.empty(max(ac, 1), dtype=torch.int32, device=dev)
                    b["active_cap"] = ac
                if b.get("tri_cap", -1) < tc:
                    b["vert"] = torch.empty((max(tc, 1), 3, 3), dtype=torch.float32, device=dev)
                    b["edge"] = torch.empty((max(tc, 1), 3), dtype=torch.int64, device=dev)
                    b["iso"] = torch.empty(max(tc, 1), dtype=torch.int32, device=dev)
                    b["cell"] = torch.empty(max(tc, 1), dtype=torch.int32, device=dev)
                    b["tri_cap"] = tc
                m = meshes[i]
                m.d_active_code, m.d_active_mask, m.active_cap = b["code"].data_ptr(), b["mask"].data_ptr(), b["active_cap"]
                m.d_tri_vert, m.d_tri_edge = b["vert"].data_ptr(), b["edge"].data_ptr()
                m.d_tri_iso, m.d_tri_cell, m.tri_cap = b["iso"].data_ptr(), b["cell"].data_ptr(), b["tri_cap"]
            st = load().isx_batch_run(self._h, meshes, _stream_ptr(stream))
            if st == 3 and attempt < 2:
                for i in range(n):
                    caps[i] = [max(caps[i][0], int(meshes[i].n_active)), max(caps[i][1], int(meshes[i].n_tris))]
                continue
            _check(st)
            break
        out = []
        for i, b in enumerate(self._bufs):
            m = meshes[i]
            na, nt = int(m.n_active), int(m.n_tris)
            out.append(dict(codes=b["code"][:na], masks=b["mask"][:na], tri_vert=b["vert"][:nt],
                            tri_edge=b["edge"][:nt], tri_iso=b["iso"][:nt], tri_cell=b["cell"][:nt], n_active=na,
                            n_tris=nt, n_points=int(m.n_points), ms_acp=m.ms_acp, ms_inr=m.ms_inr, ms_mc=m.ms_mc,
                            ms_total=m.ms_total, cells_bounded=list(m.cells_bounded)[:self.max_levels[i] + 1]))
        return out
