"""Python access to the FP64 CPU oracle (oracle/amg_oracle.c).

TEST INFRASTRUCTURE ONLY: the correctness reference for the CUDA library.
Only tests/, the smoke check in __graft_entry__.py and bench.py's CPU-baseline
leg use it; the library in paper_1811_05704_gb300/ never imports it, and this
module never imports the library.

The C file is compiled with gcc (-O2 -ffp-contract=off) into
oracle/_build/liboracle.so on first use (or by ``build()``).
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, OOM, NOT_CONVERGED, BREAKDOWN, STALLED, TOO_LARGE = 0, 1, 2, 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile the oracle shared library if missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    """Mirror of ``oparams`` in amg_oracle.c."""
    _fields_ = [
        ("eps_strong", C.c_double),
        ("eps_halving", C.c_int),
        ("smoother", C.c_int),
        ("jacobi_omega", C.c_double),
        ("npre", C.c_int),
        ("npost", C.c_int),
        ("coarse_enough", C.c_int),
        ("max_levels", C.c_int),
        ("max_coarse_dense", C.c_int),
    ]


def default_params(**kw) -> Params:
    p = Params(eps_strong=0.08, eps_halving=1, smoother=0, jacobi_omega=0.72, npre=1, npost=1,
               coarse_enough=500, max_levels=25, max_coarse_dense=4096)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


_P = C.c_void_p
_I64 = C.c_int64
_DP = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_U8P = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_setup.restype = _P
            L.orc_setup.argtypes = [_I64, _I32P, _I32P, _DP, C.POINTER(Params), C.POINTER(C.c_int)]
            L.orc_free.argtypes = [_P]
            L.orc_levels.restype = C.c_int
            L.orc_levels.argtypes = [_P]
            L.orc_level_info.argtypes = [_P, C.c_int, _I64P]
            L.orc_get_matrix.argtypes = [_P, C.c_int, C.c_int, _I64P, _I32P, _DP]
            L.orc_get_level_vectors.argtypes = [_P, C.c_int, _P, _P, _P]
            L.orc_vcycle.argtypes = [_P, _DP, _DP, C.POINTER(Params)]
            for name in ("orc_cg", "orc_bicgstab"):
                f = getattr(L, name)
                f.restype = C.c_int
                f.argtypes = [_P, _DP, _DP, C.c_double, C.c_int, C.POINTER(Params),
                              C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.orc_aggregate.restype = _I64
            L.orc_aggregate.argtypes = [_I64, _I32P, _I32P, _DP, C.c_double, _I32P]
            L.orc_strength.argtypes = [_I64, _I32P, _I32P, _DP, C.c_double, _U8P]
            L.orc_spmv.argtypes = [_I64, _I64, _I32P, _I32P, _DP, _DP, _DP]
            L.orc_spgemm.restype = _P
            L.orc_spgemm.argtypes = [_I64, _I64, _I64, _I32P, _I32P, _DP, _I32P, _I32P, _DP]
            L.orc_csr_nnz.restype = _I64
            L.orc_csr_nnz.argtypes = [_P]
            L.orc_csr_export.argtypes = [_P, _I64P, _I32P, _DP]
            L.orc_csr_free.argtypes = [_P]
            L.orc_dense_solve.restype = C.c_int
            L.orc_dense_solve.argtypes = [_I64, _DP, _DP, _DP]
            L.orc_prolongation.restype = _P
            L.orc_prolongation.argtypes = [_I64, _I32P, _I32P, _DP, C.c_double, _I32P, _I64,
                                           C.POINTER(C.c_double)]
            L.orc_tentative_values.argtypes = [_I64, _I32P, _I64, _DP]
            L.orc_smoother_diag.argtypes = [_I64, _I32P, _I32P, _DP, C.POINTER(Params), _DP]
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _take_csr(handle, nrows):
    L = lib()
    if not handle:
        raise MemoryError("oracle allocation failed")
    nnz = L.orc_csr_nnz(handle)
    ptr = np.empty(nrows + 1, np.int64)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    L.orc_csr_export(handle, ptr, col, val)
    L.orc_csr_free(handle)
    return ptr, col, val


# ---------------------------------------------------------------- steps
def strength(A, eps):
    s = np.zeros(A.nnz, np.uint8)
    lib().orc_strength(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), eps, s)
    return s.astype(bool)


def aggregate(A, eps):
    agg = np.empty(A.n, np.int32)
    nagg = lib().orc_aggregate(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), eps, agg)
    return agg, int(nagg)


def prolongation(A, eps, agg, nagg):
    om = C.c_double()
    h = lib().orc_prolongation(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), eps, _i32(agg),
                               nagg, C.byref(om))
    return _take_csr(h, A.n), om.value


def spmv(nrows, ncols, ptr, col, val, x):
    y = np.empty(nrows)
    lib().orc_spmv(nrows, ncols, _i32(ptr), _i32(col), _f64(val), _f64(x), y)
    return y


def spgemm(n, k, m, a, b):
    """C = A B; a, b = (ptr, col, val) with int32 pointers. Returns (ptr64, col, val)."""
    h = lib().orc_spgemm(n, k, m, _i32(a[0]), _i32(a[1]), _f64(a[2]),
                         _i32(b[0]), _i32(b[1]), _f64(b[2]))
    return _take_csr(h, n)


def dense_solve(a, b):
    a = _f64(a)
    n = a.shape[0]
    x = np.empty(n)
    st = lib().orc_dense_solve(n, a, _f64(b), x)
    if st != OK:
        raise np.linalg.LinAlgError("singular")
    return x


def tentative_values(agg, nagg):
    t = np.empty(len(agg))
    lib().orc_tentative_values(len(agg), _i32(agg), nagg, t)
    return t


def smoother_diag(A, params=None):
    d = np.empty(A.n)
    p = params or default_params()
    lib().orc_smoother_diag(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), C.byref(p), d)
    return d


# ------------------------------------------------------------ hierarchy
class Hierarchy:
    """Oracle AMG hierarchy (Algorithm 1) with the V-cycle and Krylov solvers."""

    def __init__(self, A, params=None, **kw):
        self.params = params or default_params(**kw)
        st = C.c_int(0)
        self._A = A
        self._h = lib().orc_setup(A.n, _i32(A.row_ptr), _i32(A.col), _f64(A.val),
                                  C.byref(self.params), C.byref(st))
        self.status = st.value
        if not self._h:
            raise OracleError(st.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    @property
    def levels(self) -> int:
        return lib().orc_levels(self._h)

    def level_info(self, l):
        out = np.zeros(5, np.int64)
        lib().orc_level_info(self._h, l, out)
        return dict(n=int(out[0]), nnz=int(out[1]), ncoarse=int(out[2]), nnz_p=int(out[3]),
                    nnz_r=int(out[4]))

    def matrix(self, l, which):
        """which in {'A','P','R'} -> (ptr int64, col int32, val float64, shape)."""
        info = self.level_info(l)
        w = {"A": 0, "P": 1, "R": 2}[which]
        nrows = info["ncoarse"] if which == "R" else info["n"]
        ncols = info["ncoarse"] if which == "P" else info["n"]
        nnz = {"A": info["nnz"], "P": info["nnz_p"], "R": info["nnz_r"]}[which]
        ptr = np.empty(nrows + 1, np.int64)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        lib().orc_get_matrix(self._h, l, w, ptr, col, val)
        return ptr, col, val, (nrows, ncols)

    def dense(self, l, which):
        ptr, col, val, shape = self.matrix(l, which)
        d = np.zeros(shape)
        rows = np.repeat(np.arange(shape[0]), np.diff(ptr))
        d[rows, col] = val
        return d

    def aggregates(self, l):
        n = self.level_info(l)["n"]
        agg = np.empty(n, np.int32)
        lib().orc_get_level_vectors(self._h, l, agg.ctypes.data, None, None)
        return agg

    def smoother_diagonal(self, l):
        n = self.level_info(l)["n"]
        d = np.empty(n)
        lib().orc_get_level_vectors(self._h, l, None, d.ctypes.data, None)
        return d

    def omega_p(self, l):
        om = C.c_double()
        lib().orc_get_level_vectors(self._h, l, None, None, C.addressof(om))
        return om.value

    def vcycle(self, r):
        z = np.empty_like(_f64(r))
        lib().orc_vcycle(self._h, _f64(r), z, C.byref(self.params))
        return z

    def _krylov(self, fn, f, x0, rtol, maxiter):
        x = _f64(np.zeros(self._A.n) if x0 is None else np.array(x0, dtype=np.float64))
        it = C.c_int()
        rr = C.c_double()
        st = fn(self._h, _f64(f), x, rtol, maxiter, C.byref(self.params), C.byref(it), C.byref(rr))
        return x, int(it.value), float(rr.value), int(st)

    def cg(self, f, x0=None, rtol=1e-8, maxiter=500):
        """Returns (x, iterations, true relative residual, status)."""
        return self._krylov(lib().orc_cg, f, x0, rtol, maxiter)

    def bicgstab(self, f, x0=None, rtol=1e-8, maxiter=500):
        return self._krylov(lib().orc_bicgstab, f, x0, rtol, maxiter)


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle setup failed with status {status}")
        self.status = status
