"""Batched form: many independent systems in one persistent launch, each
against the FP64 oracle solved alone (same tolerances as the single-system
solves: true residual <= rtol, x within 1e-6 of the oracle's, iterations
within +-1 for the FP64 V-cycle, within +3 for the FP32 one)."""
import importlib.util
import os

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def amg():
    spec = importlib.util.spec_from_file_location(
        "_b", os.path.join(ROOT, "paper_1811_05704_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1811_05704_gb300 as m
    return m


def _systems(count, seed, lo=16, hi=40):
    sides, sigma = gen.batched_sides(count, seed, lo, hi)
    mats = [gen.poisson2d_shift(int(m), float(s)) for m, s in zip(sides, sigma)]
    rhs = [gen.uniform_pm1(seed, 1000 + k, A.n) for k, A in enumerate(mats)]
    return mats, rhs


def _oracle_solve(A, f, **kw):
    import oracle
    H = oracle.Hierarchy(A, **kw)
    return H.cg(f, rtol=1e-8, maxiter=300)


def _true_relres(A, x, f):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return np.linalg.norm(f - np.bincount(rows, weights=A.val * x[A.col], minlength=A.n)) / np.linalg.norm(f)


def _run(amg, mats, rhs, **params):
    import torch
    dev = torch.device("cuda:0")
    csrs = [amg.make_csr(A.n, A.row_ptr, A.col, A.val) for A in mats]
    b = amg.amg_batch_setup(csrs, amg.amg_params_default(**params))
    tot, off, lev = amg.amg_batch_info(b, len(mats))
    assert tot == sum(A.n for A in mats) and off[-1] == tot
    f = torch.from_numpy(np.concatenate(rhs)).to(dev)
    x = torch.zeros(tot, dtype=torch.float64, device=dev)
    st, it, rr, sst = amg.amg_batch_solve(b, len(mats), f, x, 1e-8, 300)
    return b, st, it, rr, sst, x.cpu().numpy(), off, lev


@pytest.mark.parametrize("precision,slack", [(0, 1), (1, 3)])
def test_batch_matches_oracle(amg, precision, slack):
    mats, rhs = _systems(40, seed=3)
    b, st, it, rr, sst, x, off, lev = _run(amg, mats, rhs, precision=precision, coarse_enough=100)
    assert st == 0 and (sst == 0).all()
    assert lev.max() >= 2 and lev.min() >= 1
    for k, A in enumerate(mats):
        xs = x[off[k]:off[k + 1]]
        xo, ito, rro, sto = _oracle_solve(A, rhs[k], coarse_enough=100)
        assert sto == 0 and rr[k] <= 1e-8 and _true_relres(A, xs, rhs[k]) <= 1e-8
        assert abs(rr[k] - _true_relres(A, xs, rhs[k])) <= 1e-12
        assert (it[k] - ito <= slack) and (ito - it[k] <= 1), (k, it[k], ito)
        assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    amg.amg_batch_free(b)


def test_batch_edge_systems_and_tuning(amg):
    import torch
    dev = torch.device("cuda:0")
    one = gen.Csr(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    small = gen.poisson2d_shift(12, 0.05)   # 144 rows: one level, M = A^-1
    mid = gen.poisson2d_shift(45, 0.01)     # several levels
    zero_rhs = gen.poisson2d_shift(20, 0.02)
    bad = gen.poisson2d_shift(18, 0.03)
    mats = [one, small, mid, zero_rhs, bad]
    rhs = [np.array([8.0]), gen.uniform_pm1(1, 1, small.n), gen.uniform_pm1(1, 2, mid.n),
           np.zeros(zero_rhs.n), gen.uniform_pm1(1, 3, bad.n)]
    rhs[4][5] = np.nan
    b, st, it, rr, sst, x, off, lev = _run(amg, mats, rhs, precision=1)
    assert st == amg.AMG_ERR_INVALID_ARG
    assert list(sst) == [0, 0, 0, 0, amg.AMG_ERR_INVALID_ARG]
    assert x[0] == 2.0 and it[0] == 1
    assert it[1] == 1 and lev[1] == 1
    assert it[3] == 0 and rr[3] == 0.0 and not x[off[3]:off[4]].any()
    assert rr[2] <= 1e-8
    # tuning picks a schedule; solving again with it gives the same answers up to rounding
    rhs[4][5] = 0.5
    f = torch.from_numpy(np.concatenate(rhs)).to(dev)
    xt = torch.zeros(off[-1], dtype=torch.float64, device=dev)
    threads, ctas = amg.amg_batch_tune(b, f, xt, 1e-8, 300)
    assert threads in (128, 256, 512, 1024) and ctas in (1, 2, 4)
    x2 = torch.zeros(off[-1], dtype=torch.float64, device=dev)
    st2, it2, rr2, sst2 = amg.amg_batch_solve(b, len(mats), f, x2, 1e-8, 300)
    assert st2 == 0 and (rr2 <= 1e-8).all()
    assert np.allclose(xt.cpu().numpy(), x2.cpu().numpy(), rtol=0, atol=1e-6 * np.abs(x2.cpu().numpy()).max())
    amg.amg_batch_free(b)


def test_batch_full_size_4096(amg):
    """The batched workload: 4096 2D Poisson systems with sides U{16..128},
    shifts U(0, 0.1), f ~ U(-1,1), FP32 V-cycle under FP64 CG."""
    import torch
    sides, sigma = gen.batched_sides(4096, 0)
    mats = [gen.poisson2d_shift(int(m), float(s)) for m, s in zip(sides, sigma)]
    rhs = [gen.uniform_pm1(0, 1000 + k, A.n) for k, A in enumerate(mats)]
    b, st, it, rr, sst, x, off, lev = _run(amg, mats, rhs, precision=1)
    assert st == 0 and (rr <= 1e-8).all()
    for k in np.random.default_rng(0).choice(4096, 6, replace=False):
        A = mats[k]
        xs = x[off[k]:off[k + 1]]
        assert _true_relres(A, xs, rhs[k]) <= 1e-8
        xo, ito, rro, sto = _oracle_solve(A, rhs[k])
        assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
        assert it[k] <= ito + 3
    amg.amg_batch_free(b)


def _model_bytes(info, precision):
    """Bytes of one CG iteration without the fused restriction operator (the
    model of amg_hierarchy_bytes, written out): e bytes per V-cycle nonzero,
    v per level-vector entry."""
    e, v = (12, 8) if precision == 0 else (8, 4)
    b, L = 0, info["levels"]
    for l in range(L - 1):
        n, z, zp, nc = info["rows"][l], info["nnz"][l], info["nnz_p"][l], info["rows"][l + 1]
        b += (e * z + 4 * n + 4 * v * n) + (e * zp + 4 * nc + v * n + v * nc)
        b += (e * zp + 4 * n + v * nc + 2 * v * n) + (e * z + 4 * n + 4 * v * n)
    nL = info["rows"][-1]
    n0, z0 = info["rows"][0], info["nnz"][0]
    return b + 8 * nL * nL + 2 * v * nL + 12 * z0 + 20 * n0 + 72 * n0


def test_iteration_bytes_agree_with_single_system(amg):
    """amg_batch_bytes gives each system the bytes per CG iteration of its
    hierarchy (the same hierarchy as the matrix set up alone), by the model
    written out on the hierarchy's sizes; the batched kernel does not use the
    fused restriction operator, so a single-system handle gives the same
    count, less the 8 bytes a row that its deferred x update saves, exactly
    when none of its levels uses one."""
    mats, rhs = _systems(6, 5, lo=20, hi=60)
    for precision in (0, 1):
        b, st, it, rr, sst, x, off, lev = _run(amg, mats, rhs, precision=precision)
        per = amg.amg_batch_bytes(b, len(mats))
        amg.amg_batch_free(b)
        for A, v in zip(mats, per):
            S = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=precision)
            info = S.info()
            want = _model_bytes(info, precision)
            assert abs(v - want) <= 1e-12 * want and v > 0
            if not any(amg.amg_fused_restriction_nnz(S.handle, l) for l in range(info["levels"])):
                # the single-system CG moves x += alpha p into the p update: 8 bytes a row less
                single = want - 8 * info["rows"][0]
                assert abs(amg.amg_hierarchy_bytes(S.handle) - single) <= 1e-12 * single
            S.close()
