"""amg_spmv_dot_noalloc: the product y = A x with x.y for callers that cannot
allocate device memory while they run.  Its scratch is a fixed static device
array of the library instead of a per-call cudaMallocAsync.  This file checks,
through the C ABI, that two calls in a row give what the allocating entry
point amg_spmv_dot gives (the same kernel and schedule, so the results must
agree within the tolerances the parity tests use), and that a matrix too large
for the static scratch is refused with a clear error.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test; it also passes alone in a fresh process.
"""
import importlib.util
import os

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U = 2.0 ** -53


@pytest.fixture(scope="module")
def amg():
    spec = importlib.util.spec_from_file_location(
        "_b", os.path.join(ROOT, "paper_1811_05704_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1811_05704_gb300 as m
    return m


def _row_bound(A, x):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return np.bincount(rows, weights=np.abs(A.val * x[A.col]), minlength=A.n)


def test_noalloc_matches_allocating_entry_point(amg):
    import torch
    dev = torch.device("cuda:0")
    cases = [gen.poisson3d(40), gen.varcoef3d(17, seed=3), gen.poisson2d_shift(9, 0.02)]
    for A in cases:
        rp, cl, vl = (torch.from_numpy(a).to(dev) for a in (A.row_ptr, A.col, A.val))
        csr = amg.make_csr(A.n, rp, cl, vl)
        xs = [torch.from_numpy(gen.uniform_pm1(s, 30, A.n)).to(dev) for s in (1, 2)]
        for x in xs:  # two calls in a row on the shared static scratch
            y_ref = torch.zeros(A.n, dtype=torch.float64, device=dev)
            d_ref = torch.zeros(1, dtype=torch.float64, device=dev)
            amg.amg_spmv_dot(csr, x, y_ref, d_ref)
            y = torch.full((A.n,), np.nan, dtype=torch.float64, device=dev)
            d = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
            amg.amg_spmv_dot_noalloc(csr, x, y, d)
            torch.cuda.synchronize()
            yn, yr, xn = y.cpu().numpy(), y_ref.cpu().numpy(), x.cpu().numpy()
            assert np.all(np.abs(yn - yr) <= 64 * U * _row_bound(A, xn))
            assert abs(d.item() - d_ref.item()) <= 1e-12 * np.abs(xn * yr).sum()
            # and the product itself is right
            rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
            y_np = np.bincount(rows, weights=A.val * xn[A.col], minlength=A.n)
            assert np.all(np.abs(yn - y_np) <= 64 * U * _row_bound(A, xn))


def test_noalloc_refuses_matrix_above_its_limit(amg):
    import torch
    dev = torch.device("cuda:0")
    n = (1 << 24) + 1  # 65,537 row blocks of 256 rows: one more than the static scratch holds
    rp = torch.arange(n + 1, dtype=torch.int32, device=dev)
    cl = torch.arange(n, dtype=torch.int32, device=dev)
    vl = torch.full((n,), 2.0, dtype=torch.float64, device=dev)
    x = torch.ones(n, dtype=torch.float64, device=dev)
    y = torch.zeros(n, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(amg.AmgError) as e:
        amg.amg_spmv_dot_noalloc(amg.make_csr(n, rp, cl, vl), x, y, d)
    assert e.value.status == amg.AMG_ERR_TOO_LARGE
    assert "65536" in str(e.value)
    # the allocating entry point handles the same matrix
    amg.amg_spmv_dot(amg.make_csr(n, rp, cl, vl), x, y, d)
    assert d.item() == 2.0 * n


def _cudart():
    """The CUDA runtime as a shared library (the toolkit's), for reading the
    device's default memory pool, from which amg_spmv_dot's stream-ordered
    scratch comes."""
    import ctypes
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.fail("no CUDA runtime shared library found")


# cudaMemPoolAttr values of the CUDA runtime API
_RESERVED_CURRENT, _USED_CURRENT, _USED_HIGH = 5, 7, 8


def test_noalloc_moves_no_pool_watermark(amg):
    """The reason for the entry point: it allocates nothing.  After a first
    (warm-up) call, the device's default memory pool -- where amg_spmv_dot's
    scratch comes from -- keeps its used-memory high watermark and its
    reserved size through two more calls; one amg_spmv_dot call then raises
    the watermark, which shows that the check sees an allocation."""
    import ctypes
    import torch
    dev = torch.device("cuda:0")
    rt = _cudart()
    A = gen.poisson3d(40)
    rp, cl, vl = (torch.from_numpy(a).to(dev) for a in (A.row_ptr, A.col, A.val))
    csr = amg.make_csr(A.n, rp, cl, vl)
    x = torch.from_numpy(gen.uniform_pm1(3, 30, A.n)).to(dev)
    y = torch.zeros(A.n, dtype=torch.float64, device=dev)
    d = torch.zeros(1, dtype=torch.float64, device=dev)
    amg.amg_spmv_dot_noalloc(csr, x, y, d)
    torch.cuda.synchronize()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), 0) == 0

    def attr(a):
        v = ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
        return v.value

    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, _USED_HIGH, ctypes.byref(zero)) == 0
    used0, reserved0 = attr(_USED_CURRENT), attr(_RESERVED_CURRENT)
    for _ in range(2):
        amg.amg_spmv_dot_noalloc(csr, x, y, d)
    torch.cuda.synchronize()
    assert attr(_USED_HIGH) <= used0
    assert attr(_RESERVED_CURRENT) == reserved0
    amg.amg_spmv_dot(csr, x, y, d)
    torch.cuda.synchronize()
    assert attr(_USED_HIGH) > used0
