"""The solve server (continuous batching over resident hierarchies).

A served request must give the same answer as the same request solved alone
(identical bits: every solve is deterministic and the hierarchy of a matrix
does not depend on what else runs), admission must respect the HBM budget
(evicting idle hierarchies, least recently used first), and a failing request
must fail alone."""
import importlib.util
import os
import threading

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RTOL = 1e-8


@pytest.fixture(scope="module")
def amg():
    spec = importlib.util.spec_from_file_location(
        "_b", os.path.join(ROOT, "paper_1811_05704_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1811_05704_gb300 as m
    return m


def _estimate(A):
    """The charge of a new matrix stated by the header (amg_server_params)."""
    return 72 * A.nnz + 64 * A.n + (8 << 20)


def _params(amg, q):
    """CG with damped Jacobi for the SPD requests; BiCGStab with SPAI-0 for
    the convection-diffusion ones (damped Jacobi stalls at high Peclet)."""
    if q.solver:
        return amg.amg_params_default(solver=amg.AMG_SOLVER_BICGSTAB, smoother=amg.AMG_SMOOTHER_SPAI0)
    return amg.amg_params_default()


def _true_relres(A, x, f):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return np.linalg.norm(f - np.bincount(rows, weights=A.val * x[A.col], minlength=A.n)) / np.linalg.norm(f)


def _alone(amg, reqs, seed):
    """Each request solved on its own handle (one per key), in order."""
    handles, mats, out = {}, {}, []
    for q in reqs:
        if q.key not in mats:
            mats[q.key] = q.matrix()
        A = mats[q.key]
        if q.key not in handles:
            handles[q.key] = amg.amg_setup(amg.make_csr(A.n, A.row_ptr, A.col, A.val), _params(amg, q))
        f = q.rhs(seed, A.n)
        x = np.zeros(A.n)
        st, it, rr = amg.amg_solve_host(handles[q.key], f, x, RTOL, 300)
        out.append((st, x, it, rr, amg.amg_hierarchy_bytes(handles[q.key]) * it))
    for h in handles.values():
        amg.amg_free(h)
    return mats, out


def _submit(amg, srv, q, mats, seed, with_matrix=True):
    A = mats[q.key]
    csr = amg.make_csr(A.n, A.row_ptr, A.col, A.val) if with_matrix else None
    return amg.amg_server_submit(srv, q.key, csr, q.rhs(seed, A.n), _params(amg, q), RTOL, 300)


def test_served_results_equal_alone(amg):
    seed = 5
    reqs = gen.serving_requests(28, seed, lo=8, hi=30)
    assert any(q.reuse for q in reqs) and any(q.solver for q in reqs)
    mats, alone = _alone(amg, reqs, seed)
    srv = amg.amg_server_create(slots=4)
    # reused keys are submitted without their matrix half of the time
    ids = [_submit(amg, srv, q, mats, seed, with_matrix=not (q.reuse and q.index % 2)) for q in reqs]
    for q, rid, (st0, x0, it0, rr0, _) in zip(reqs, ids, alone):
        st, x, it, rr, lat, qt = amg.amg_server_wait(srv, rid, mats[q.key].n)
        assert st == st0 == 0, (q, amg.amg_last_error())
        assert it == it0 and rr == rr0, q
        assert np.array_equal(x, x0), q
        assert 0.0 <= qt <= lat
    stats = amg.amg_server_stats(srv)
    assert stats["completed"] == len(reqs)
    assert stats["resident_count"] == len({q.key for q in reqs}) and stats["evictions"] == 0
    # the server's byte count is the sum of the same solves' counts alone
    want = sum(a[4] for a in alone)
    assert abs(amg.amg_server_solve_bytes(srv) - want) <= 1e-12 * want and want > 0
    amg.amg_server_destroy(srv)


def test_served_results_match_oracle(amg):
    import oracle
    seed = 9
    reqs = [q for q in gen.serving_requests(12, seed, lo=10, hi=22) if not q.reuse][:4]
    mats = {q.key: q.matrix() for q in reqs}
    srv = amg.amg_server_create(slots=3)
    ids = [_submit(amg, srv, q, mats, seed) for q in reqs]
    for q, rid in zip(reqs, ids):
        A = mats[q.key]
        f = q.rhs(seed, A.n)
        st, x, it, rr, _, _ = amg.amg_server_wait(srv, rid, A.n)
        H = oracle.Hierarchy(A, smoother=1 if q.solver else 0)
        xo, ito, rro, sto = (H.bicgstab if q.solver else H.cg)(f, rtol=RTOL, maxiter=300)
        assert st == 0 and sto == 0
        assert _true_relres(A, x, f) <= RTOL and abs(rr - _true_relres(A, x, f)) <= 1e-12
        assert abs(it - ito) <= 1, (q, it, ito)
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    amg.amg_server_destroy(srv)


def test_concurrent_submitters(amg):
    """Several host threads submit and wait at once; every result is the
    request's result alone."""
    seed = 11
    reqs = gen.serving_requests(24, seed, lo=8, hi=24)
    mats, alone = _alone(amg, reqs, seed)
    srv = amg.amg_server_create(slots=6)
    bad = []

    def client(part):
        for i in part:
            q = reqs[i]
            rid = _submit(amg, srv, q, mats, seed)
            st, x, it, rr, _, _ = amg.amg_server_wait(srv, rid, mats[q.key].n)
            if st != 0 or not np.array_equal(x, alone[i][1]) or it != alone[i][2]:
                bad.append(i)

    threads = [threading.Thread(target=client, args=(range(k, len(reqs), 4),)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not bad
    amg.amg_server_destroy(srv)


def test_admission_evicts_least_recently_used(amg):
    seed = 13
    A0, A1, A2 = gen.poisson3d(20), gen.varcoef3d(20, seed=4), gen.poisson3d(18)
    f = {k: gen.uniform_pm1(seed, k, A.n) for k, A in enumerate((A0, A1, A2))}
    # the bytes a resident 20^3 hierarchy holds
    probe = amg.amg_server_create(slots=1)
    rid = amg.amg_server_submit(probe, 0, amg.make_csr(A0.n, A0.row_ptr, A0.col, A0.val), f[0])
    assert amg.amg_server_wait(probe, rid, A0.n)[0] == 0
    b0 = amg.amg_server_stats(probe)["resident_bytes"]
    amg.amg_server_destroy(probe)
    assert 0 < b0

    # room for one new hierarchy, not for a resident one beside it
    budget = max(_estimate(A0), _estimate(A1)) + b0 // 2
    assert budget < b0 + _estimate(A1)
    srv = amg.amg_server_create(slots=1, hbm_budget=budget)
    c = lambda A: amg.make_csr(A.n, A.row_ptr, A.col, A.val)  # noqa: E731
    ids = [amg.amg_server_submit(srv, 0, c(A0), f[0]),
           amg.amg_server_submit(srv, 1, c(A1), f[1]),   # evicts key 0
           amg.amg_server_submit(srv, 0, None, f[0]),    # key 0 is gone: fails
           amg.amg_server_submit(srv, 1, None, f[1])]    # key 1 is resident
    res = [amg.amg_server_wait(srv, i, A0.n) for i in ids]
    assert [r[0] for r in res] == [0, 0, amg.AMG_ERR_INVALID_ARG, 0]
    assert np.array_equal(res[1][1], res[3][1]) and res[1][2] == res[3][2]
    st = amg.amg_server_stats(srv)
    assert st["evictions"] == 1 and st["resident_count"] == 1 and st["peak_bytes"] <= budget
    amg.amg_server_destroy(srv)

    # a budget below every request: each runs alone, evicting the one before
    srv = amg.amg_server_create(slots=3, hbm_budget=1)
    ids = [(amg.amg_server_submit(srv, k, c(A), f[k]), A) for k, A in enumerate((A0, A1, A2))]
    for rid, A in ids:
        st, x, it, rr, _, _ = amg.amg_server_wait(srv, rid, A.n)
        assert st == 0 and rr <= RTOL
    st = amg.amg_server_stats(srv)
    assert st["evictions"] == 2 and st["resident_count"] == 1
    amg.amg_server_destroy(srv)


def test_failing_requests_fail_alone(amg):
    seed = 17
    A = gen.poisson3d(12)
    good = gen.uniform_pm1(seed, 1, A.n)
    nan_f = good.copy()
    nan_f[7] = np.nan
    bad_diag = gen.poisson3d(10)
    bad_diag.val[bad_diag.row_ptr[3]:bad_diag.row_ptr[4]] = 0.0  # row 3 has no usable diagonal
    c = lambda M: amg.make_csr(M.n, M.row_ptr, M.col, M.val)  # noqa: E731
    srv = amg.amg_server_create(slots=2)
    r_ok = amg.amg_server_submit(srv, 1, c(A), good)
    r_nan = amg.amg_server_submit(srv, 1, None, nan_f)
    r_diag = amg.amg_server_submit(srv, 2, c(bad_diag), gen.uniform_pm1(seed, 2, bad_diag.n))
    r_nokey = amg.amg_server_submit(srv, 99, None, good)
    r_len = amg.amg_server_submit(srv, 1, None, good[:100])
    r_prm = amg.amg_server_submit(srv, 4, c(A), good, amg.amg_params_default(npre=99))
    with pytest.raises(amg.AmgError):  # matrix and right-hand side sizes differ
        amg.amg_server_submit(srv, 3, c(A), good[:100])
    r_after = amg.amg_server_submit(srv, 1, None, good)
    st_ok = amg.amg_server_wait(srv, r_ok, A.n)
    assert st_ok[0] == 0
    assert amg.amg_server_wait(srv, r_nan, A.n)[0] == amg.AMG_ERR_INVALID_ARG
    assert amg.amg_server_wait(srv, r_diag, bad_diag.n)[0] == amg.AMG_ERR_INVALID_ARG
    assert amg.amg_last_error()
    assert amg.amg_server_wait(srv, r_nokey, A.n)[0] == amg.AMG_ERR_INVALID_ARG
    assert amg.amg_server_wait(srv, r_len, 100)[0] == amg.AMG_ERR_INVALID_ARG
    assert amg.amg_server_wait(srv, r_prm, A.n)[0] == amg.AMG_ERR_INVALID_ARG
    assert "npre" in amg.amg_last_error()
    st_after = amg.amg_server_wait(srv, r_after, A.n)
    assert st_after[0] == 0 and np.array_equal(st_after[1], st_ok[1])
    assert amg.amg_server_wait(srv, r_after, A.n)[0] == amg.AMG_ERR_INVALID_ARG  # already collected
    amg.amg_server_destroy(srv)
