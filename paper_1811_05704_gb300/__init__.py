"""Thin Python binding of the GB300 smoothed-aggregation AMG library.

Every function here marshals arguments to the C ABI of include/amg.h (same
names) and checks the returned status; all computation happens in the CUDA
library libamg_gb300.so.  PyTorch supplies device memory and streams.  There is
no CPU fallback: importing this package fails if the compiled library is
missing (build it with ``python paper_1811_05704_gb300/build.py`` or
``__graft_entry__.build()``).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libamg_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"the CUDA library {LIB_PATH} is not built; run `python paper_1811_05704_gb300/build.py`")

_lib = C.CDLL(LIB_PATH)

# ----------------------------------------------------------------- constants
AMG_OK, AMG_ERR_INVALID_ARG, AMG_ERR_OOM, AMG_ERR_CUDA = 0, 1, 2, 3
AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN, AMG_ERR_COARSENING_STALLED, AMG_ERR_TOO_LARGE = 4, 5, 6, 7
AMG_SMOOTHER_JACOBI, AMG_SMOOTHER_SPAI0 = 0, 1
AMG_SOLVER_CG, AMG_SOLVER_BICGSTAB = 0, 1
AMG_PRECISION_FP64, AMG_PRECISION_FP32, AMG_PRECISION_BF16 = 0, 1, 2
AMG_MAX_LEVELS = 32
KERNEL_CLASSES = ["spmv_dot", "krylov_update", "presmooth_l0", "restrict_l0", "prolong_l0",
                  "postsmooth_l0", "vcycle_coarser", "coarse_solve", "other"]
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED",
                5: "BREAKDOWN", 6: "COARSENING_STALLED", 7: "TOO_LARGE"}


class amg_params(C.Structure):
    _fields_ = [
        ("strength_eps", C.c_double),
        ("strength_halving", C.c_int),
        ("smoother", C.c_int),
        ("jacobi_omega", C.c_double),
        ("npre", C.c_int),
        ("npost", C.c_int),
        ("coarse_enough", C.c_int),
        ("max_levels", C.c_int),
        ("max_coarse_dense", C.c_int),
        ("solver", C.c_int),
        ("precision", C.c_int),
        ("use_graph", C.c_int),
        ("use_stream", C.c_int),
        ("use_pdl", C.c_int),
        ("use_tail", C.c_int),
        ("device_setup", C.c_int),
        ("fused_restriction", C.c_int),
    ]


class amg_csr(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("row_ptr", C.c_void_p),
        ("col", C.c_void_p),
        ("val", C.c_void_p),
        ("on_device", C.c_int),
    ]


_VP, _I, _D, _I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
_sigs = {
    "amg_params_default": [C.POINTER(amg_params)],
    "amg_setup": [C.POINTER(amg_csr), C.POINTER(amg_params), _VP, C.POINTER(_VP)],
    "amg_solve": [_VP, _VP, _VP, _D, _I, C.POINTER(_I), C.POINTER(_D)],
    "amg_solve_host": [_VP, _VP, _VP, _D, _I, C.POINTER(_I), C.POINTER(_D)],
    "amg_free": [_VP],
    "amg_hierarchy_info": [_VP, C.POINTER(_I), _VP, _VP, _VP],
    "amg_get_level_matrix": [_VP, _I, _I, _VP, _VP, _VP],
    "amg_get_aggregates": [_VP, _I, _VP],
    "amg_get_smoother_diag": [_VP, _I, _VP],
    "amg_apply_precond": [_VP, _VP, _VP],
    "amg_level_spmv": [_VP, _I, _I, _VP, _VP],
    "amg_spmv_dot": [C.POINTER(amg_csr), _VP, _VP, _VP, _VP],
    "amg_spmv_dot_noalloc": [C.POINTER(amg_csr), _VP, _VP, _VP, _VP],
    "amg_solve_profile": [_VP, _VP, _VP, _D, _I, C.POINTER(_I), C.POINTER(_D), _VP, _VP],
    "amg_last_launch_count": [_VP, C.POINTER(_I64)],
    "amg_hierarchy_bytes": [_VP, C.POINTER(_D)],
    "amg_fused_restriction_nnz": [_VP, _I, C.POINTER(_I64)],
    "amg_batch_bytes": [_VP, _VP],
    "amg_server_solve_bytes": [_VP, C.POINTER(_D)],
    "amg_last_solve_mode": [_VP, C.POINTER(_I), C.POINTER(_I)],
    "amg_check_wait_limit": [C.POINTER(_D)],
    "amg_batch_setup": [_I, _VP, C.POINTER(amg_params), _VP, C.POINTER(_VP)],
    "amg_batch_solve": [_VP, _VP, _VP, _D, _I, _VP, _VP, _VP],
    "amg_batch_tune": [_VP, _VP, _VP, _D, _I, C.POINTER(_I), C.POINTER(_I)],
    "amg_batch_info": [_VP, C.POINTER(_I64), _VP, _VP],
    "amg_batch_free": [_VP],
    "amg_server_create": [_VP, C.POINTER(amg_params), C.POINTER(_VP)],
    "amg_server_submit": [_VP, _I64, C.POINTER(amg_csr), _VP, _I64, C.POINTER(amg_params), _D, _I,
                          C.POINTER(_I64)],
    "amg_server_wait": [_VP, _I64, _VP, C.POINTER(_I), C.POINTER(_D), C.POINTER(_D), C.POINTER(_D)],
    "amg_server_stats": [_VP, C.POINTER(_I64), C.POINTER(_I), C.POINTER(_I64), C.POINTER(_I64),
                         C.POINTER(_I64)],
    "amg_server_destroy": [_VP],
}
for _name, _args in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.amg_last_error.restype = C.c_char_p
_lib.amg_last_error.argtypes = []

EXPORTED = sorted(list(_sigs) + ["amg_last_error"])


class AmgError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.amg_last_error().decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st, where, allow=()):
    if st != AMG_OK and st not in allow:
        raise AmgError(st, where)
    return st


def _ptr(t):
    """Raw pointer of a torch tensor or numpy array (contiguous)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------ C-ABI names
def amg_last_error() -> str:
    return _lib.amg_last_error().decode()


def amg_params_default(**overrides) -> amg_params:
    p = amg_params()
    _check(_lib.amg_params_default(C.byref(p)), "amg_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def make_csr(n, row_ptr, col, val):
    """amg_csr over host numpy arrays (int32, int32, float64) or CUDA tensors."""
    on_device = not isinstance(val, np.ndarray)
    return amg_csr(n=n, nnz=int(len(col) if isinstance(col, np.ndarray) else col.numel()),
                   row_ptr=_ptr(row_ptr), col=_ptr(col), val=_ptr(val), on_device=int(on_device))


def amg_setup(csr: amg_csr, params: amg_params = None, stream=None):
    h = C.c_void_p()
    p = C.byref(params) if params is not None else None
    _check(_lib.amg_setup(C.byref(csr), p, _stream(stream), C.byref(h)), "amg_setup")
    return h


def amg_free(h):
    _check(_lib.amg_free(h), "amg_free")


def amg_solve(h, f, x, rtol=1e-8, maxiter=500, raise_on=()):
    """Solve on device tensors f, x (x: initial guess in, solution out).

    Returns (status, iterations, true relative residual).  NOT_CONVERGED and
    BREAKDOWN are returned, not raised, unless listed in raise_on."""
    it, rr = C.c_int(), C.c_double()
    st = _lib.amg_solve(h, _ptr(f), _ptr(x), rtol, maxiter, C.byref(it), C.byref(rr))
    allow = tuple(s for s in (AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN) if s not in raise_on)
    _check(st, "amg_solve", allow)
    return st, it.value, rr.value


def amg_solve_host(h, f_host, x_host, rtol=1e-8, maxiter=500):
    it, rr = C.c_int(), C.c_double()
    st = _lib.amg_solve_host(h, _ptr(f_host), _ptr(x_host), rtol, maxiter, C.byref(it), C.byref(rr))
    _check(st, "amg_solve_host", (AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN))
    return st, it.value, rr.value


def amg_solve_profile(h, f, x, rtol=1e-8, maxiter=500):
    """Returns (status, iterations, relres, {class: ms}, {class: launches})."""
    it, rr = C.c_int(), C.c_double()
    ms = (C.c_double * len(KERNEL_CLASSES))()
    ln = (C.c_int * len(KERNEL_CLASSES))()
    st = _lib.amg_solve_profile(h, _ptr(f), _ptr(x), rtol, maxiter, C.byref(it), C.byref(rr),
                                C.cast(ms, C.c_void_p), C.cast(ln, C.c_void_p))
    _check(st, "amg_solve_profile", (AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN))
    return (st, it.value, rr.value, dict(zip(KERNEL_CLASSES, list(ms))),
            dict(zip(KERNEL_CLASSES, list(ln))))


def amg_check_wait_limit():
    """Run the bounded-wait check (see include/amg.h); returns (status, seconds).
    The expected status is AMG_ERR_CUDA."""
    sec = C.c_double()
    st = _lib.amg_check_wait_limit(C.byref(sec))
    return st, sec.value


def amg_last_launch_count(h) -> int:
    v = C.c_int64()
    _check(_lib.amg_last_launch_count(h, C.byref(v)), "amg_last_launch_count")
    return v.value


def amg_last_solve_mode(h):
    """(graph attempts, host-launched attempts) of the last solve."""
    g, hst = C.c_int(), C.c_int()
    _check(_lib.amg_last_solve_mode(h, C.byref(g), C.byref(hst)), "amg_last_solve_mode")
    return g.value, hst.value


def amg_hierarchy_info(h):
    lv = C.c_int()
    rows = np.zeros(AMG_MAX_LEVELS, np.int64)
    nnz = np.zeros(AMG_MAX_LEVELS, np.int64)
    nnzp = np.zeros(AMG_MAX_LEVELS, np.int64)
    _check(_lib.amg_hierarchy_info(h, C.byref(lv), rows.ctypes.data, nnz.ctypes.data,
                                   nnzp.ctypes.data), "amg_hierarchy_info")
    L = lv.value
    return dict(levels=L, rows=rows[:L].tolist(), nnz=nnz[:L].tolist(), nnz_p=nnzp[:L].tolist())


def amg_fused_restriction_nnz(h, level) -> int:
    v = C.c_int64()
    _check(_lib.amg_fused_restriction_nnz(h, level, C.byref(v)), "amg_fused_restriction_nnz")
    return v.value


def amg_get_level_matrix(h, level, which):
    """which in {'A','P','R','M'} -> (row_ptr int32, col int32, val float64, shape)."""
    info = amg_hierarchy_info(h)
    w = {"A": 0, "P": 1, "R": 2, "M": 3}[which]
    n = info["rows"][level]
    nc = info["rows"][level + 1] if level + 1 < info["levels"] else 0
    nrows = nc if which in ("R", "M") else n
    ncols = nc if which == "P" else n
    nnz = {"A": lambda: info["nnz"][level], "P": lambda: info["nnz_p"][level],
           "R": lambda: info["nnz_p"][level], "M": lambda: amg_fused_restriction_nnz(h, level)}[which]()
    ptr = np.zeros(nrows + 1, np.int32)
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float64)
    _check(_lib.amg_get_level_matrix(h, level, w, ptr.ctypes.data, col.ctypes.data, val.ctypes.data),
           "amg_get_level_matrix")
    return ptr, col[:nnz], val[:nnz], (nrows, ncols)


def amg_get_aggregates(h, level):
    n = amg_hierarchy_info(h)["rows"][level]
    agg = np.zeros(n, np.int32)
    _check(_lib.amg_get_aggregates(h, level, agg.ctypes.data), "amg_get_aggregates")
    return agg


def amg_get_smoother_diag(h, level):
    n = amg_hierarchy_info(h)["rows"][level]
    d = np.zeros(n, np.float64)
    _check(_lib.amg_get_smoother_diag(h, level, d.ctypes.data), "amg_get_smoother_diag")
    return d


def amg_apply_precond(h, r, z):
    _check(_lib.amg_apply_precond(h, _ptr(r), _ptr(z)), "amg_apply_precond")


def amg_level_spmv(h, level, which, x, y):
    w = {"A": 0, "P": 1, "R": 2}[which]
    _check(_lib.amg_level_spmv(h, level, w, _ptr(x), _ptr(y)), "amg_level_spmv")


def amg_spmv_dot(csr: amg_csr, x, y, dot, stream=None):
    _check(_lib.amg_spmv_dot(C.byref(csr), _ptr(x), _ptr(y), _ptr(dot), _stream(stream)),
           "amg_spmv_dot")


def amg_spmv_dot_noalloc(csr: amg_csr, x, y, dot, stream=None):
    """amg_spmv_dot for callers that cannot allocate: scratch is a fixed static
    device array of the library (see include/amg.h for the size limit and the
    rule that overlapping calls race)."""
    _check(_lib.amg_spmv_dot_noalloc(C.byref(csr), _ptr(x), _ptr(y), _ptr(dot), _stream(stream)),
           "amg_spmv_dot_noalloc")


# ---------------------------------------------------------------- batched
def amg_batch_setup(systems, params: amg_params = None, stream=None):
    """systems: list of amg_csr (see make_csr).  Returns a batch handle."""
    arr = (amg_csr * len(systems))(*systems)
    h = C.c_void_p()
    p = C.byref(params) if params is not None else None
    _check(_lib.amg_batch_setup(len(systems), C.cast(arr, C.c_void_p), p, _stream(stream), C.byref(h)),
           "amg_batch_setup")
    return h


def amg_hierarchy_bytes(h) -> float:
    v = C.c_double()
    _check(_lib.amg_hierarchy_bytes(h, C.byref(v)), "amg_hierarchy_bytes")
    return v.value


def amg_batch_bytes(b, nsys):
    out = np.zeros(nsys, np.float64)
    _check(_lib.amg_batch_bytes(b, out.ctypes.data), "amg_batch_bytes")
    return out


def amg_server_solve_bytes(srv) -> float:
    v = C.c_double()
    _check(_lib.amg_server_solve_bytes(srv, C.byref(v)), "amg_server_solve_bytes")
    return v.value


def amg_batch_info(b, nsys):
    tot = C.c_int64()
    off = np.zeros(nsys + 1, np.int64)
    lev = np.zeros(nsys, np.int32)
    _check(_lib.amg_batch_info(b, C.byref(tot), off.ctypes.data, lev.ctypes.data), "amg_batch_info")
    return tot.value, off, lev


def amg_batch_solve(b, nsys, f, x, rtol=1e-8, maxiter=500):
    """Returns (status, iters[nsys], relres[nsys], status[nsys])."""
    it = np.zeros(nsys, np.int32)
    rr = np.zeros(nsys, np.float64)
    st = np.zeros(nsys, np.int32)
    s = _lib.amg_batch_solve(b, _ptr(f), _ptr(x), rtol, maxiter, it.ctypes.data, rr.ctypes.data,
                             st.ctypes.data)
    _check(s, "amg_batch_solve", (AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN, AMG_ERR_INVALID_ARG))
    return s, it, rr, st


def amg_batch_tune(b, f, x, rtol=1e-8, maxiter=500):
    t, c = C.c_int(), C.c_int()
    _check(_lib.amg_batch_tune(b, _ptr(f), _ptr(x), rtol, maxiter, C.byref(t), C.byref(c)), "amg_batch_tune")
    return t.value, c.value


def amg_batch_free(b):
    _check(_lib.amg_batch_free(b), "amg_batch_free")


# ---------------------------------------------------------------- serving
class amg_server_params(C.Structure):
    _fields_ = [
        ("slots", C.c_int),
        ("reserved0", C.c_int),
        ("hbm_budget", C.c_int64),
        ("reserved", C.c_int64 * 4),
    ]


def amg_server_create(slots=4, hbm_budget=0, params: amg_params = None):
    sp = amg_server_params(slots=slots, hbm_budget=hbm_budget)
    h = C.c_void_p()
    p = C.byref(params) if params is not None else None
    _check(_lib.amg_server_create(C.byref(sp), p, C.byref(h)), "amg_server_create")
    return h


def amg_server_submit(s, key, csr, f_host, params: amg_params = None, rtol=1e-8, maxiter=500):
    """csr: amg_csr over host arrays, or None to reuse key's resident
    hierarchy.  f_host: float64 numpy array (copied).  params: parameters of
    a hierarchy this request builds (None: the server's).  Returns the
    request id."""
    f = np.ascontiguousarray(f_host, dtype=np.float64)
    rid = C.c_int64()
    c = C.byref(csr) if csr is not None else None
    p = C.byref(params) if params is not None else None
    _check(_lib.amg_server_submit(s, key, c, f.ctypes.data, f.size, p, rtol, maxiter, C.byref(rid)),
           "amg_server_submit")
    return rid.value


def amg_server_wait(s, rid, n):
    """Returns (status, x, iters, relres, latency_s, queue_s); blocks until
    the request has finished (releases the GIL meanwhile)."""
    x = np.zeros(n, np.float64)
    it, rr, lat, q = C.c_int(), C.c_double(), C.c_double(), C.c_double()
    st = _lib.amg_server_wait(s, rid, x.ctypes.data, C.byref(it), C.byref(rr), C.byref(lat), C.byref(q))
    return st, x, it.value, rr.value, lat.value, q.value


def amg_server_stats(s):
    """Returns dict(completed, resident_count, resident_bytes, peak_bytes, evictions)."""
    c, rc, rb, pk, ev = C.c_int64(), C.c_int(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.amg_server_stats(s, C.byref(c), C.byref(rc), C.byref(rb), C.byref(pk), C.byref(ev)),
           "amg_server_stats")
    return dict(completed=c.value, resident_count=rc.value, resident_bytes=rb.value, peak_bytes=pk.value,
                evictions=ev.value)


def amg_server_destroy(s):
    _check(_lib.amg_server_destroy(s), "amg_server_destroy")


# ------------------------------------------------------------- convenience
class Solver:
    """Owns a handle: Solver(n, row_ptr, col, val, **params).solve(f, x)."""

    def __init__(self, n, row_ptr, col, val, stream=None, **params):
        self._keep = (row_ptr, col, val)
        self.params = amg_params_default(**params)
        self.handle = amg_setup(make_csr(n, row_ptr, col, val), self.params, stream)
        self.n = n

    def close(self):
        if getattr(self, "handle", None):
            amg_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, f, x, rtol=1e-8, maxiter=500):
        return amg_solve(self.handle, f, x, rtol, maxiter)

    def info(self):
        return amg_hierarchy_info(self.handle)
