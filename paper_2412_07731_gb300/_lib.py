"""ctypes binding of the C ABI in include/ahlp.h (argument marshalling only).

Every computation happens inside ``libahlp.so``; this module only converts a
block LP description into the C structs, passes pointers through and turns
status codes into exceptions.  It refuses to run without the compiled library:
there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libahlp.so")

AHLP_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "DIM_MISMATCH", -3: "UNSUPPORTED", -4: "NOT_SPD",
          -5: "REFINE_FAIL", -6: "MAX_ITER", -7: "INFEASIBLE_OR_UNBOUNDED", -8: "CUDA",
          -9: "OOM", -10: "TIMEOUT", -11: "STOPPED"}
PREC_FP64, PREC_MIXED = 0, 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class CSC(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("colptr", _ip), ("rowidx", _ip),
                ("val", _dp)]


class Desc(C.Structure):
    _fields_ = [("N", C.c_int32), ("n0", C.c_int32), ("mg", C.c_int32), ("c0", _dp),
                ("A", C.POINTER(CSC)), ("W", C.POINTER(CSC)), ("b", C.POINTER(_dp)),
                ("c", C.POINTER(_dp)), ("l", _ip), ("FL", C.POINTER(CSC)),
                ("FR", C.POINTER(CSC)), ("F0", C.POINTER(CSC)), ("blink", C.POINTER(_dp)),
                ("Fg", C.POINTER(CSC)), ("Fg0", C.POINTER(CSC)), ("bg", _dp),
                ("lb", C.POINTER(_dp)), ("ub", C.POINTER(_dp)), ("lb0", _dp), ("ub0", _dp),
                ("mD", _ip), ("D", C.POINTER(CSC)), ("C", C.POINTER(CSC)),
                ("dlo", C.POINTER(_dp)), ("dhi", C.POINTER(_dp)),
                ("lG", _ip), ("GL", C.POINTER(CSC)), ("GR", C.POINTER(CSC)),
                ("G0", C.POINTER(CSC)), ("glo", C.POINTER(_dp)), ("ghi", C.POINTER(_dp)),
                ("mgG", C.c_int32), ("Gg", C.POINTER(CSC)), ("Gg0", C.POINTER(CSC)),
                ("gglo", _dp), ("gghi", _dp)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("eta", C.c_double), ("delta", C.c_double), ("rho", C.c_double),
                ("refine_max", C.c_int32), ("refine_tol", C.c_double),
                ("pivot_tol", C.c_double), ("verbose", C.c_int32),
                ("max_correctors", C.c_int32), ("fp32_cond_max", C.c_double),
                ("ipm_refine_tol", C.c_double), ("correctors_by_cost", C.c_int32),
                ("fp32_update", C.c_int32), ("ff_update", C.c_int32),
                ("schur_chain", C.c_int32), ("profile_kernels", C.c_int32),
                ("iter_cb", C.c_void_p),
                ("iter_cb_ctx", C.c_void_p), ("pivot_mode", C.c_int32),
                ("tile_sparse", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("pobj", C.c_double),
                ("dobj", C.c_double), ("rel_gap", C.c_double), ("pinf", C.c_double),
                ("dinf", C.c_double), ("mu", C.c_double), ("ms_total", C.c_double),
                ("ms_factor", C.c_double), ("ms_solve", C.c_double),
                ("refine_steps", C.c_int32), ("tiny_pivots", C.c_int32),
                ("kkt_residual", C.c_double), ("escalations", C.c_int32),
                ("fp64_switch_iter", C.c_int32), ("factors_fp32", C.c_int32),
                ("factors_fp64", C.c_int32), ("correctors", C.c_int32),
                ("ms_block_fp32", C.c_double), ("ms_block_fp64", C.c_double),
                ("factors_ff", C.c_int32), ("ms_block_ff", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(C.Structure):
    _fields_ = [("refine_steps", C.c_int32), ("rel_residual", C.c_double)]


EXPORTS = ["ahlp_default_options", "ahlp_status_string", "arrowhead_lp_create",
           "arrowhead_lp_destroy", "ahlp_last_error", "arrowhead_lp_sizes",
           "arrowhead_lp_set_stream", "arrowhead_lp_set_options", "kkt_factor", "kkt_solve",
           "kkt_adjoint_solve", "ipm_solve", "kkt_schur_dense", "kkt_stage_times",
           "ahlp_launch_count", "kkt_residual_noalloc", "kkt_block_factor_dense",
           "ahlp_transfer_bytes", "arrowhead_lp_set_cb", "kkt_factor_kernel_times",
           "arrowhead_lp_recover", "arrowhead_lp_original_size", "arrowhead_lp_autotune",
           "kkt_update_jobs", "ahlp_tile_sparse_jobs"]


def kkt_block_factor_dense(prob, block: int):
    """Block ``block``'s partially factored augmented matrix (lower, dense)."""
    a = C.c_int32(0)
    probe = np.zeros(1)
    prob._lib.kkt_block_factor_dense(prob._h, block, C.c_void_p(probe.ctypes.data), 0, C.byref(a))
    if a.value <= 0:
        prob._check(prob._lib.kkt_block_factor_dense(prob._h, block,
                                                     C.c_void_p(probe.ctypes.data), 0, None))
    out = np.zeros((a.value, a.value), order="F")
    prob._check(prob._lib.kkt_block_factor_dense(prob._h, block, C.c_void_p(out.ctypes.data),
                                                 max(a.value, 1), C.byref(a)))
    return out


def launch_count() -> int:
    """Kernels launched by libahlp.so in this process so far."""
    return int(load().ahlp_launch_count())


def batch_layout(lps):
    """For a batch of LPs: per LP, the index arrays (ix, iy) that place its own
    global vectors -- x = [x_1..x_N, x_0], y = [y_1..y_N, y_links, y_g] -- in
    the direct sum's vectors: x = [blocks of every LP, x_0 of every LP],
    y = [block rows of every LP, link rows of every LP, global rows of every
    LP].  combined[ix] = own_x, own_x = combined[ix]."""
    nxb = [int(sum(A.shape[1] for A in q.A)) for q in lps]
    nyb = [int(sum(A.shape[0] for A in q.A)) for q in lps]
    nl = [int(sum(int(v) for v in q.l)) for q in lps]
    xb0 = np.concatenate([[0], np.cumsum(nxb)]).astype(np.int64)
    x00 = xb0[-1] + np.concatenate([[0], np.cumsum([q.n0 for q in lps])]).astype(np.int64)
    yb0 = np.concatenate([[0], np.cumsum(nyb)]).astype(np.int64)
    yl0 = yb0[-1] + np.concatenate([[0], np.cumsum(nl)]).astype(np.int64)
    yg0 = yl0[-1] + np.concatenate([[0], np.cumsum([q.mg for q in lps])]).astype(np.int64)
    out = []
    for k, q in enumerate(lps):
        ix = np.concatenate([np.arange(xb0[k], xb0[k + 1]), np.arange(x00[k], x00[k + 1])])
        iy = np.concatenate([np.arange(yb0[k], yb0[k + 1]), np.arange(yl0[k], yl0[k + 1]),
                             np.arange(yg0[k], yg0[k + 1])])
        out.append((ix, iy))
    return out


def set_cb(prob, c=None, b=None):
    """Replace the objective c ([n]) and/or right-hand side b ([m]) of the
    handle; host (numpy) or device (torch) vectors, None keeps the current."""
    keep = _Keep()
    prob._stream_for(c, b)
    prob._check(prob._lib.arrowhead_lp_set_cb(prob._h, _vec_ptr(c, keep, prob.n, "c"),
                                              _vec_ptr(b, keep, prob.m, "b")))


def autotune(prob, x=None, z=None):
    """Choose the faster trailing-update kernels (FP32 and float-float block
    factors) for this handle at (x, z) (default x = z = 1); the choice goes
    into the handle's options.  Returns the six candidates' block-factor times
    (ms) and the chosen fp32_update and ff_update."""
    keep = _Keep()
    prob._stream_for(x, z)
    ms = (C.c_double * 6)()
    prob._check(prob._lib.arrowhead_lp_autotune(
        prob._h, _vec_ptr(x, keep, prob.n, "x") if x is not None else None,
        _vec_ptr(z, keep, prob.n, "z") if z is not None else None, ms))
    # mirror the handle's new choice in the Python-side copy of its options
    prob.options.fp32_update = (3 if ms[4] <= min(ms[0], ms[1]) else
                                2 if ms[0] <= ms[1] else 1)
    prob.options.ff_update = 3 if ms[5] <= min(ms[2], ms[3]) else 2 if ms[2] <= ms[3] else 1
    return {"fp32_tensor_ms": ms[0], "fp32_pipe_ms": ms[1], "ff_tensor_ms": ms[2],
            "ff_pipe_ms": ms[3], "fp32_tensor_persistent_ms": ms[4],
            "ff_tensor_persistent_ms": ms[5],
            "fp32_update": prob.options.fp32_update, "ff_update": prob.options.ff_update}


def recover(prob, x):
    """(x_orig, obj_offset): the original variables of an LP given with bounds
    or inequality rows, from a point x of the equality form the handle works
    on; the original objective is c'x + obj_offset."""
    keep = _Keep()
    n = C.c_int64(0)
    prob._check(prob._lib.arrowhead_lp_original_size(prob._h, C.byref(n)))
    out = _out_like(x, n.value)
    off = C.c_double(0.0)
    prob._check(prob._lib.arrowhead_lp_recover(prob._h, _vec_ptr(x, keep, prob.n, "x"),
                                               _vec_ptr(out, keep, n.value, "x_orig"),
                                               C.byref(off)))
    return out, off.value


def kkt_factor_kernel_times(prob):
    """Device ms and launch groups of the last factor's diagonal tiles, panels
    and trailing updates (option profile_kernels)."""
    ms = (C.c_double * 3)()
    n = (C.c_int64 * 3)()
    prob._check(prob._lib.kkt_factor_kernel_times(prob._h, ms, n))
    return {"diag_ms": ms[0], "panel_ms": ms[1], "update_ms": ms[2],
            "diag_launches": n[0], "panel_launches": n[1], "update_launches": n[2]}


def kkt_update_jobs(prob) -> tuple[int, int]:
    """(kept, dense) tile jobs of one factor's tensor-core trailing updates."""
    kept, dense = C.c_int64(0), C.c_int64(0)
    prob._check(prob._lib.kkt_update_jobs(prob._h, C.byref(kept), C.byref(dense)))
    return kept.value, dense.value


def tile_sparse_jobs(T, Tp, nz=None):
    """The tile-sparse job table (host only, no device): T, Tp per block and
    nz (list of per-block T x T tile patterns, or None for dense blocks).
    Returns (jobs as an int32 array of (block, I0, J, has_i1) rows, step
    offsets, dense job count)."""
    T = np.ascontiguousarray(T, dtype=np.int32)
    Tp = np.ascontiguousarray(Tp, dtype=np.int32)
    nblk = len(T)
    pat = None
    if nz is not None:
        pat = np.ascontiguousarray(np.concatenate(
            [np.asarray(z, dtype=np.uint8).reshape(-1) for z in nz]) if nblk else
            np.zeros(0, np.uint8))
    lib = load()
    kept, dense = C.c_int64(0), C.c_int64(0)
    maxtp = int(Tp.max()) if nblk else 0
    off = np.zeros(maxtp + 1, dtype=np.int64)
    ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    st = lib.ahlp_tile_sparse_jobs(nblk, ptr(T), ptr(Tp), ptr(pat), None, ptr(off), 0,
                                   C.byref(kept), C.byref(dense))
    if st != AHLP_OK:
        raise AHLPError(st, "ahlp_tile_sparse_jobs: invalid sizes")
    jobs = np.zeros((kept.value, 4), dtype=np.int32)
    st = lib.ahlp_tile_sparse_jobs(nblk, ptr(T), ptr(Tp), ptr(pat), ptr(jobs), ptr(off),
                                   kept.value, C.byref(kept), C.byref(dense))
    if st != AHLP_OK:
        raise AHLPError(st, "ahlp_tile_sparse_jobs failed")
    return jobs, off, dense.value


def transfer_bytes(prob) -> tuple[int, int]:
    """(host->device, device->host) bytes copied by this handle since create."""
    h2d, d2h = C.c_int64(0), C.c_int64(0)
    prob._check(prob._lib.ahlp_transfer_bytes(prob._h, C.byref(h2d), C.byref(d2h)))
    return int(h2d.value), int(d2h.value)

_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Load libahlp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} not found: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(p)
    vp = C.c_void_p
    L.ahlp_default_options.argtypes = [C.POINTER(Options)]
    L.ahlp_default_options.restype = None
    L.ahlp_status_string.argtypes = [C.c_int]
    L.ahlp_status_string.restype = C.c_char_p
    L.arrowhead_lp_create.argtypes = [C.POINTER(Desc), C.c_int32, C.POINTER(Options),
                                      C.POINTER(vp)]
    L.arrowhead_lp_create.restype = C.c_int
    L.arrowhead_lp_destroy.argtypes = [vp]
    L.arrowhead_lp_destroy.restype = None
    L.ahlp_last_error.argtypes = [vp]
    L.ahlp_last_error.restype = C.c_char_p
    L.arrowhead_lp_sizes.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.arrowhead_lp_set_stream.argtypes = [vp, vp]
    L.arrowhead_lp_set_options.argtypes = [vp, C.POINTER(Options)]
    L.kkt_factor.argtypes = [vp, vp, vp, C.c_double, C.c_double]
    L.kkt_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(SolveInfo)]
    L.kkt_adjoint_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(SolveInfo)]
    L.ipm_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(Result)]
    L.kkt_schur_dense.argtypes = [vp, vp, C.c_int64]
    L.kkt_stage_times.argtypes = [vp, _dp]
    L.ahlp_launch_count.argtypes = []
    L.ahlp_launch_count.restype = C.c_int64
    L.kkt_residual_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.kkt_residual_noalloc.restype = C.c_int
    L.kkt_block_factor_dense.argtypes = [vp, C.c_int32, vp, C.c_int64, C.POINTER(C.c_int32)]
    L.kkt_block_factor_dense.restype = C.c_int
    L.ahlp_tile_sparse_jobs.argtypes = [C.c_int32, vp, vp, vp, vp, vp, C.c_int64,
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.ahlp_tile_sparse_jobs.restype = C.c_int
    L.kkt_update_jobs.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.kkt_update_jobs.restype = C.c_int
    L.ahlp_transfer_bytes.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.ahlp_transfer_bytes.restype = C.c_int
    L.arrowhead_lp_autotune.argtypes = [vp, vp, vp, _dp]
    L.arrowhead_lp_autotune.restype = C.c_int
    L.arrowhead_lp_recover.argtypes = [vp, vp, vp, _dp]
    L.arrowhead_lp_recover.restype = C.c_int
    L.arrowhead_lp_original_size.argtypes = [vp, C.POINTER(C.c_int64)]
    L.arrowhead_lp_original_size.restype = C.c_int
    L.kkt_factor_kernel_times.argtypes = [vp, _dp, C.POINTER(C.c_int64)]
    L.kkt_factor_kernel_times.restype = C.c_int
    L.arrowhead_lp_set_cb.argtypes = [vp, vp, vp]
    L.arrowhead_lp_set_cb.restype = C.c_int
    for name in ("arrowhead_lp_sizes", "arrowhead_lp_set_stream", "arrowhead_lp_set_options",
                 "kkt_factor", "kkt_solve", "kkt_adjoint_solve", "ipm_solve", "kkt_schur_dense",
                 "kkt_stage_times"):
        getattr(L, name).restype = C.c_int
    if path is None:
        _lib = L
    return L


class AHLPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_options(**kw) -> Options:
    o = Options()
    load().ahlp_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class _Keep:
    """Holds every buffer handed to C for the lifetime of one call."""

    def __init__(self):
        self.refs = []

    def f64(self, a):
        a = _f64(a)
        self.refs.append(a)
        return a.ctypes.data_as(_dp)

    def i32(self, a):
        a = _i32(a)
        self.refs.append(a)
        return a.ctypes.data_as(_ip)

    def csc(self, M, shape):
        s = CSC()
        if M is None:
            s.m, s.n = shape
            return s
        M = M.tocsc()
        s.m, s.n = M.shape
        s.colptr = self.i32(M.indptr)
        s.rowidx = self.i32(M.indices)
        s.val = self.f64(M.data)
        return s

    def csc_array(self, mats, shapes):
        arr = (CSC * max(len(mats), 1))()
        for k, (M, sh) in enumerate(zip(mats, shapes)):
            arr[k] = self.csc(M, sh)
        self.refs.append(arr)
        return arr

    def ptr_array(self, vecs):
        arr = (_dp * max(len(vecs), 1))()
        for k, v in enumerate(vecs):
            arr[k] = self.f64(v)
        self.refs.append(arr)
        return arr


def make_desc(lp, keep: _Keep) -> Desc:
    """Block LP (instances.BlockLP or anything with the same fields) -> Desc."""
    d = Desc()
    N, n0, mg = lp.N, lp.n0, lp.mg
    d.N, d.n0, d.mg = N, n0, mg
    ms = [a.shape[0] for a in lp.A]
    ns = [a.shape[1] for a in lp.A]
    l = [int(v) for v in lp.l]
    d.c0 = keep.f64(lp.c0 if n0 else np.zeros(1))
    d.A = keep.csc_array(lp.A, [a.shape for a in lp.A])
    d.W = keep.csc_array(lp.W, [(m, n0) for m in ms])
    d.b = keep.ptr_array(lp.b)
    d.c = keep.ptr_array(lp.c)
    d.l = keep.i32(l if l else [0])
    d.FL = keep.csc_array(lp.FL, [(l[j], ns[j]) for j in range(N - 1)])
    d.FR = keep.csc_array(lp.FR, [(l[j], ns[j + 1]) for j in range(N - 1)])
    d.F0 = keep.csc_array(lp.F0, [(l[j], n0) for j in range(N - 1)])
    d.blink = keep.ptr_array([v if len(v) else np.zeros(1) for v in lp.blink])
    d.Fg = keep.csc_array(lp.Fg, [(mg, n) for n in ns])
    fg0 = (CSC * 1)()
    fg0[0] = keep.csc(lp.Fg0, (mg, n0))
    keep.refs.append(fg0)
    d.Fg0 = fg0
    d.bg = keep.f64(lp.bg if mg else np.zeros(1))
    # the full statement of Sec. 3.2: bounds and inequality rows (optional)
    g = lambda name: getattr(lp, name, None)  # noqa: E731
    if g("lb") is not None:
        d.lb = keep.ptr_array(lp.lb)
    if g("ub") is not None:
        d.ub = keep.ptr_array(lp.ub)
    if g("lb0") is not None and n0:
        d.lb0 = keep.f64(lp.lb0)
    if g("ub0") is not None and n0:
        d.ub0 = keep.f64(lp.ub0)
    if g("D") is not None:
        mD = [int(M.shape[0]) for M in lp.D]
        d.mD = keep.i32(mD)
        d.D = keep.csc_array(lp.D, [(mD[i], ns[i]) for i in range(N)])
        d.C = keep.csc_array(lp.C if g("C") is not None else [None] * N,
                             [(mD[i], n0) for i in range(N)])
        d.dlo = keep.ptr_array([v if len(v) else np.zeros(1) for v in lp.dlo])
        d.dhi = keep.ptr_array([v if len(v) else np.zeros(1) for v in lp.dhi])
    if g("GL") is not None and N > 1:
        lG = [int(M.shape[0]) for M in lp.GL]
        d.lG = keep.i32(lG)
        d.GL = keep.csc_array(lp.GL, [(lG[j], ns[j]) for j in range(N - 1)])
        d.GR = keep.csc_array(lp.GR, [(lG[j], ns[j + 1]) for j in range(N - 1)])
        d.G0 = keep.csc_array(lp.G0 if g("G0") is not None else [None] * (N - 1),
                              [(lG[j], n0) for j in range(N - 1)])
        d.glo = keep.ptr_array([v if len(v) else np.zeros(1) for v in lp.glo])
        d.ghi = keep.ptr_array([v if len(v) else np.zeros(1) for v in lp.ghi])
    if g("Gg") is not None and g("gglo") is not None and len(lp.gglo):
        mgG = len(lp.gglo)
        d.mgG = mgG
        d.Gg = keep.csc_array(lp.Gg, [(mgG, nn) for nn in ns])
        gg0 = (CSC * 1)()
        gg0[0] = keep.csc(g("Gg0"), (mgG, n0))
        keep.refs.append(gg0)
        d.Gg0 = gg0
        d.gglo = keep.f64(lp.gglo)
        d.gghi = keep.f64(lp.gghi)
    return d


def _vec_ptr(v, keep: _Keep, n: int, name: str):
    """Pointer of a host (numpy) or device (torch) vector of length n."""
    if v is None:
        return None
    if hasattr(v, "data_ptr"):          # torch tensor, host or device
        if v.dtype.__str__() != "torch.float64" or v.numel() != n or not v.is_contiguous():
            raise ValueError(f"{name}: need a contiguous float64 tensor of length {n}")
        keep.refs.append(v)
        return C.c_void_p(v.data_ptr())
    a = _f64(v)
    if a.shape != (n,):
        raise ValueError(f"{name}: expected length {n}, got {a.shape}")
    keep.refs.append(a)
    return C.c_void_p(a.ctypes.data)


def _out_like(template, n):
    if template is not None and hasattr(template, "data_ptr"):
        import torch
        return torch.empty(n, dtype=torch.float64, device=template.device)
    return np.empty(n)


class Problem:
    """Owner of one ``ahlp_problem`` handle."""

    def __init__(self, handle, lib, n, m):
        self._h = handle
        self._lib = lib
        self.n, self.m = n, m
        # bumped by every call through this binding that replaces the handle's
        # factor (kkt_factor, ipm_solve), so a caller holding on to a factor
        # (the autograd backward) can tell whether it is still the current one
        self.factor_gen = 0

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            self._lib.arrowhead_lp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != AHLP_OK:
            raise AHLPError(st, self._lib.ahlp_last_error(self._h).decode())

    def _stream_for(self, *vs):
        for v in vs:
            if v is not None and hasattr(v, "is_cuda") and v.is_cuda:
                import torch
                self._lib.arrowhead_lp_set_stream(
                    self._h, C.c_void_p(torch.cuda.current_stream(v.device).cuda_stream))
                return


def arrowhead_lp_create(lp, options: Options | None = None, batch: int | None = None) -> Problem:
    """Handle for one LP, or for a batch (a list of LPs, solved as their direct
    sum; see batch_layout for the ordering of its vectors)."""
    L = load()
    keep = _Keep()
    lps = list(lp) if isinstance(lp, (list, tuple)) else [lp]
    if batch is None:
        batch = len(lps)
    lps = [lps[min(k, len(lps) - 1)] for k in range(batch)]
    descs = (Desc * batch)()
    for k in range(batch):
        descs[k] = make_desc(lps[k], keep)
    h = C.c_void_p()
    st = L.arrowhead_lp_create(descs, batch, C.byref(options) if options is not None else None,
                               C.byref(h))
    if st != AHLP_OK:
        raise AHLPError(st, L.ahlp_last_error(None).decode())
    n, m = C.c_int64(), C.c_int64()
    L.arrowhead_lp_sizes(h, C.byref(n), C.byref(m))
    prob = Problem(h, L, n.value, m.value)
    prob.schur_dim = sum(int(sum(int(v) for v in q.l)) + q.n0 + q.mg for q in lps)
    prob.batch = batch
    prob.options = Options.from_buffer_copy(options) if options is not None else default_options()
    return prob


def set_options(prob: Problem, options: Options):
    prob._check(prob._lib.arrowhead_lp_set_options(prob._h, C.byref(options)))
    prob.options = Options.from_buffer_copy(options)


def kkt_factor(prob: Problem, x, z, delta: float = -1.0, rho: float = -1.0):
    keep = _Keep()
    prob._stream_for(x, z)
    prob.factor_gen += 1
    prob._check(prob._lib.kkt_factor(prob._h, _vec_ptr(x, keep, prob.n, "x"),
                                     _vec_ptr(z, keep, prob.n, "z"), delta, rho))


def _solve(fn, prob, a, b, c, out):
    keep = _Keep()
    prob._stream_for(a, b, c)
    if out is None:
        out = (_out_like(a, prob.n), _out_like(a, prob.m), _out_like(a, prob.n))
    info = SolveInfo()
    st = fn(prob._h, _vec_ptr(a, keep, prob.n, "arg1"), _vec_ptr(b, keep, prob.m, "arg2"),
            _vec_ptr(c, keep, prob.n, "arg3"), _vec_ptr(out[0], keep, prob.n, "out1"),
            _vec_ptr(out[1], keep, prob.m, "out2"), _vec_ptr(out[2], keep, prob.n, "out3"),
            C.byref(info))
    prob._check(st)
    return out, {"refine_steps": info.refine_steps, "rel_residual": info.rel_residual}


def kkt_solve(prob: Problem, r_d, r_p, r_c, out=None):
    """(dx, dy, dz), info for J d = (r_d, r_p, r_c) at the factored point."""
    return _solve(prob._lib.kkt_solve, prob, r_d, r_p, r_c, out)


def kkt_adjoint_solve(prob: Problem, g_x, g_y, g_z, out=None):
    """(lam_x, lam_y, lam_z), info for J' lam = (g_x, g_y, g_z)."""
    return _solve(prob._lib.kkt_adjoint_solve, prob, g_x, g_y, g_z, out)


def ipm_solve(prob: Problem, x0=None, y0=None, z0=None, out=None, check: bool = True):
    """Run the IPM; returns (x, y, z), result dict."""
    keep = _Keep()
    prob._stream_for(x0, y0, z0, *(out or ()))
    if out is None:
        out = (np.empty(prob.n), np.empty(prob.m), np.empty(prob.n))
    res = Result()
    prob.factor_gen += 1
    st = prob._lib.ipm_solve(prob._h, _vec_ptr(x0, keep, prob.n, "x0"),
                             _vec_ptr(y0, keep, prob.m, "y0"), _vec_ptr(z0, keep, prob.n, "z0"),
                             _vec_ptr(out[0], keep, prob.n, "x"),
                             _vec_ptr(out[1], keep, prob.m, "y"),
                             _vec_ptr(out[2], keep, prob.n, "z"), C.byref(res))
    r = res.as_dict()
    r["status_name"] = STATUS.get(st, st)
    if check and st not in (AHLP_OK,):
        raise AHLPError(st, prob._lib.ahlp_last_error(prob._h).decode())
    return out, r


def kkt_schur_dense(prob: Problem) -> np.ndarray:
    nS = _schur_dim(prob)
    S = np.zeros((nS, nS), order="F")
    prob._check(prob._lib.kkt_schur_dense(prob._h, C.c_void_p(S.ctypes.data), max(nS, 1)))
    return S


def _schur_dim(prob):
    return prob.schur_dim


def kkt_stage_times(prob: Problem):
    out = (C.c_double * 4)()
    prob._check(prob._lib.kkt_stage_times(prob._h, out))
    return {"form_ms": out[0], "block_factor_ms": out[1], "schur_ms": out[2],
            "last_solve_ms": out[3]}


def kkt_residual_noalloc(prob: Problem, r_d, r_p, r_c, dx, dy, dz, out):
    """Relative Newton residual of (dx, dy, dz) for (r_d, r_p, r_c), written
    into the one-element float64 CUDA tensor ``out`` without any device
    allocation (for callers that cannot allocate at that point).  Every
    argument must be a CUDA tensor."""
    keep = _Keep()
    prob._stream_for(r_d, out)
    st = prob._lib.kkt_residual_noalloc(
        prob._h, _vec_ptr(r_d, keep, prob.n, "r_d"), _vec_ptr(r_p, keep, prob.m, "r_p"),
        _vec_ptr(r_c, keep, prob.n, "r_c"), _vec_ptr(dx, keep, prob.n, "dx"),
        _vec_ptr(dy, keep, prob.m, "dy"), _vec_ptr(dz, keep, prob.n, "dz"),
        _vec_ptr(out, keep, 1, "out"))
    prob._check(st)
    return out
