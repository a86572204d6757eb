"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Tolerances (derived in the design notes):
  * aggregates, sparsity patterns of P, R and A_l: bit-exact;
  * values of P, R, A_l and the smoother diagonal: bit-exact (the host setup
    and the GPU Galerkin product evaluate every entry in the oracle's order
    without FMA contraction);
  * one SpMV row: |y - y_ref| <= 64 u sum_j |a_ij x_j| (u = 2^-53);
  * one V-cycle: ||z - z_ref|| <= 1e-10 ||z_ref||;
  * solves: true FP64 residual <= rtol = 1e-8, ||x - x_ref|| <= 1e-6 ||x_ref||,
    iterations within +-1 of the oracle's.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def amg():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("_b", os.path.join(root, "paper_1811_05704_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1811_05704_gb300 as m
    return m


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    assert torch.cuda.is_available()
    return torch, torch.device("cuda:0")


def orc_params(**kw):
    import oracle
    m = {"strength_eps": "eps_strong", "strength_halving": "eps_halving"}
    keep = {"eps_strong", "eps_halving", "smoother", "jacobi_omega", "npre", "npost",
            "coarse_enough", "max_levels", "max_coarse_dense"}
    p = {}
    for k, v in kw.items():
        k = m.get(k, k)
        if k in keep:
            p[k] = v
    return oracle.default_params(**p)


def both(amg, A, **kw):
    import oracle
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val, **kw)
    H = oracle.Hierarchy(A, params=orc_params(**kw))
    return S, H


CASES = {
    "poisson32": (lambda: gen.poisson3d(32), {}),
    "poisson17": (lambda: gen.poisson3d(17), {"coarse_enough": 60}),
    "varcoef20": (lambda: gen.varcoef3d(20, seed=1), {"coarse_enough": 100}),
    "convdiff18": (lambda: gen.convdiff3d(18, seed=2)[0], {"solver": 1, "coarse_enough": 100}),
    "poisson2d_101": (lambda: gen.poisson2d_shift(101, 0.05), {"coarse_enough": 100}),
    "spai0_varcoef": (lambda: gen.varcoef3d(16, seed=3), {"smoother": 1, "coarse_enough": 50}),
    "tail_varcoef20": (lambda: gen.varcoef3d(20, seed=1), {"coarse_enough": 40, "use_tail": 1}),
    # a dense row: Galerkin rows of 3,559 (block hash) and 7,896 (dense accumulator) columns
    "star40": (lambda: gen.poisson3d_star(40), {}),
}


def t(torch_dev, a):
    torch, dev = torch_dev
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def _random_nonsymmetric(n, seed, per_row=8):
    """A random sparse matrix with a dominant diagonal whose off-diagonal
    magnitudes straddle the strength threshold, so that the strength relation
    is asymmetric and all four aggregation passes have work."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        c = np.unique(np.concatenate([[i], rng.integers(max(0, i - 40), min(n, i + 40), per_row)]))
        v = -rng.uniform(0.0, 2.0, len(c)) * (rng.random(len(c)) < 0.9)
        v[c == i] = 10.0 + rng.uniform(0, 5)
        rows.append(np.full(len(c), i))
        cols.append(c)
        vals.append(v)
    col = np.concatenate(cols).astype(np.int32)
    ptr = np.zeros(n + 1, np.int32)
    np.cumsum([len(c) for c in cols], out=ptr[1:])
    return gen.Csr(n, ptr, col, np.concatenate(vals))


def _path(n):
    """1D Laplacian: the longest chain of ordered aggregation decisions."""
    i = np.arange(n)
    cols = [np.stack([i - 1, i, i + 1], 1)]
    c = cols[0].reshape(-1)
    v = np.tile([-1.0, 2.0, -1.0], n)
    keep = (c >= 0) & (c < n)
    ptr = np.zeros(n + 1, np.int32)
    np.cumsum(keep.reshape(n, 3).sum(1), out=ptr[1:])
    return gen.Csr(n, ptr, c[keep].astype(np.int32), v[keep])


def _aniso2d(m, eps=1e-3):
    """2D 5-point stencil with weak y couplings: strong x-lines only."""
    A = gen.poisson2d_shift(m, 0.0)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    val = A.val.copy()
    ydir = np.abs(A.col - rows) == m
    val[ydir] *= eps
    val[A.col == rows] = 2.0 + 2.0 * eps
    return gen.Csr(A.n, A.row_ptr, A.col, val)


# further hierarchies for the device set-up's ordered aggregation passes
SETUP_CASES = {
    "random_nonsym": (lambda: _random_nonsymmetric(6000, 3), {"solver": 1, "coarse_enough": 200}),
    "path20000": (lambda: _path(20000), {}),
    "aniso2d_150": (lambda: _aniso2d(150), {"coarse_enough": 200}),
}


@pytest.mark.parametrize("device_setup", [1, 0])
@pytest.mark.parametrize("case", sorted(CASES) + sorted(SETUP_CASES))
def test_hierarchy_bit_exact(amg, case, device_setup):
    """Every level's A, P, R, aggregates and smoother diagonal are identical
    to the oracle's, with the hierarchy built on the GPU (device_setup = 1,
    the default) and by the host set-up (device_setup = 0)."""
    make, kw = CASES[case] if case in CASES else SETUP_CASES[case]
    A = make()
    S, H = both(amg, A, device_setup=device_setup, **kw)
    info = S.info()
    assert info["levels"] == H.levels >= 2
    for l in range(H.levels):
        oi = H.level_info(l)
        assert info["rows"][l] == oi["n"] and info["nnz"][l] == oi["nnz"]
        ptr, col, val, _ = amg.amg_get_level_matrix(S.handle, l, "A")
        optr, ocol, oval, _ = H.matrix(l, "A")
        assert np.array_equal(ptr, optr) and np.array_equal(col, ocol)
        assert np.array_equal(val, oval), f"A_{l} values differ: {np.abs(val - oval).max()}"
        assert np.array_equal(amg.amg_get_smoother_diag(S.handle, l), H.smoother_diagonal(l))
        if l == H.levels - 1:
            continue
        assert np.array_equal(amg.amg_get_aggregates(S.handle, l), H.aggregates(l))
        for w in "PR":
            ptr, col, val, _ = amg.amg_get_level_matrix(S.handle, l, w)
            optr, ocol, oval, _ = H.matrix(l, w)
            assert np.array_equal(ptr, optr) and np.array_equal(col, ocol)
            assert np.array_equal(val, oval), f"{w}_{l} values differ"
    S.close()


@pytest.mark.parametrize("case", ["poisson32", "varcoef20", "convdiff18", "spai0_varcoef"])
def test_fused_restriction_operator(amg, case):
    """Where a level uses the fused restriction operator, M = R - R A D
    (D the smoother diagonal), entry by entry against scipy's sparse products of
    the level's own R, A and d, on the structural pattern of R A.  The finest
    level of the 7-point problems uses it."""
    make, kw = CASES[case]
    A = make()
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val, **kw)
    info = S.info()
    used = 0
    for l in range(info["levels"] - 1):
        if amg.amg_fused_restriction_nnz(S.handle, l) == 0:
            continue
        used += 1
        import scipy.sparse as sp
        mats = {}
        for w in "ARM":
            ptr, col, val, shape = amg.amg_get_level_matrix(S.handle, l, w)
            mats[w] = sp.csr_matrix((val, col, ptr), shape=shape)
            # structural pattern, stored zeros included
            mats[w + "s"] = sp.csr_matrix((np.ones(len(col)), col, ptr), shape=shape)
        dl = amg.amg_get_smoother_diag(S.handle, l)
        ref = mats["R"] - (mats["R"] @ mats["A"]) @ sp.diags(dl)
        diff = (mats["M"] - ref).tocsr()
        assert abs(diff).max() <= 1e-14 * abs(ref).max(), l
        pat = (mats["Rs"] @ mats["As"]).tocsr()
        pat.sort_indices()
        assert np.array_equal(pat.indptr, mats["Ms"].indptr), l
        assert np.array_equal(pat.indices, mats["Ms"].indices), l
    if case == "poisson32":
        assert amg.amg_fused_restriction_nnz(S.handle, 0) > 0
    S.close()


def _row_bound(ptr, col, val, x):
    rows = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    return np.bincount(rows, weights=np.abs(val * x[col]), minlength=len(ptr) - 1)


@pytest.mark.parametrize("case", ["poisson32", "varcoef20", "convdiff18", "star40"])
def test_level_spmv(amg, torch_dev, case):
    import oracle
    make, kw = CASES[case]
    A = make()
    S, H = both(amg, A, **kw)
    rng = np.random.default_rng(7)
    for l in range(H.levels):
        for w in ("A", "P", "R") if l < H.levels - 1 else ("A",):
            ptr, col, val, (nr, nc) = H.matrix(l, w)
            x = rng.uniform(-1, 1, nc)
            y = t(torch_dev, np.zeros(nr))
            amg.amg_level_spmv(S.handle, l, w, t(torch_dev, x), y)
            yo = oracle.spmv(nr, nc, ptr.astype(np.int32), col, val, x)
            bound = 64 * U * _row_bound(ptr, col, val, x)
            assert np.all(np.abs(y.cpu().numpy() - yo) <= bound), (l, w)
    S.close()


def _assert_vcycle_close(z, zo):
    """One V-cycle against the oracle's, entry by entry: every
    |z_i - zo_i| <= 1e-10 max_j |zo_j| (and the same bound for the 2-norm), so
    an error confined to a few entries cannot hide under a norm."""
    assert z.shape == zo.shape and np.all(np.isfinite(z))
    d = np.abs(z - zo)
    scale = np.abs(zo).max()
    worst = int(np.argmax(d))
    assert d[worst] <= 1e-10 * scale, (worst, d[worst] / scale)
    assert np.linalg.norm(z - zo) <= 1e-10 * np.linalg.norm(zo)


@pytest.mark.parametrize("case", sorted(CASES))
def test_vcycle(amg, torch_dev, case):
    make, kw = CASES[case]
    A = make()
    S, H = both(amg, A, **kw)
    r = gen.uniform_pm1(5, 20, A.n)
    z = t(torch_dev, np.zeros(A.n))
    amg.amg_apply_precond(S.handle, t(torch_dev, r), z)
    zo = H.vcycle(r)
    _assert_vcycle_close(z.cpu().numpy(), zo)
    S.close()


@pytest.mark.parametrize("npre,npost", [(2, 0), (0, 2), (2, 3)])
def test_vcycle_sweep_variants(amg, torch_dev, npre, npost):
    A = gen.varcoef3d(14, seed=4)
    S, H = both(amg, A, coarse_enough=40, npre=npre, npost=npost)
    r = gen.uniform_pm1(6, 20, A.n)
    z = t(torch_dev, np.zeros(A.n))
    amg.amg_apply_precond(S.handle, t(torch_dev, r), z)
    zo = H.vcycle(r)
    _assert_vcycle_close(z.cpu().numpy(), zo)
    S.close()


def _true_relres(A, x, f):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    Ax = np.bincount(rows, weights=A.val * x[A.col], minlength=A.n)
    return np.linalg.norm(f - Ax) / np.linalg.norm(f)


@pytest.mark.parametrize("case", sorted(CASES))
def test_solve_matches_oracle(amg, torch_dev, case):
    make, kw = CASES[case]
    A = make()
    S, H = both(amg, A, **kw)
    f, ustar = gen.rhs_from_solution(A, 11)
    x = t(torch_dev, np.zeros(A.n))
    st, it, rr = S.solve(t(torch_dev, f), x, rtol=1e-8, maxiter=300)
    xs = x.cpu().numpy()
    solve = H.bicgstab if kw.get("solver") == 1 else H.cg
    xo, ito, rro, sto = solve(f, rtol=1e-8, maxiter=300)
    assert st == 0 and sto == 0
    assert rr <= 1e-8 and _true_relres(A, xs, f) <= 1e-8
    assert abs(rr - _true_relres(A, xs, f)) <= 1e-12
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert amg.amg_last_launch_count(S.handle) > 0
    S.close()


@pytest.mark.parametrize("case", ["poisson32", "varcoef20", "convdiff18"])
def test_fused_restriction_on_and_off_match_oracle(amg, torch_dev, case):
    """The solve with the fused restriction operator (the default) and
    without it (fused_restriction = 0: pre-sweep, residual and restriction
    as separate steps) both meet the oracle's solve: true residual <= rtol,
    iterations +/- 1, x within 1e-6; and the two V-cycles agree entry by
    entry within the V-cycle bound."""
    make, kw = CASES[case]
    A = make()
    f, _ = gen.rhs_from_solution(A, 13)
    import oracle
    H = oracle.Hierarchy(A, params=orc_params(**kw))
    xo, ito, _, sto = (H.bicgstab if kw.get("solver") == 1 else H.cg)(f, rtol=1e-8, maxiter=300)
    r = gen.uniform_pm1(7, 20, A.n)
    zs = []
    for fused in (1, 0):
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val, fused_restriction=fused, **kw)
        used = any(amg.amg_fused_restriction_nnz(S.handle, l) for l in range(S.info()["levels"]))
        assert used if (fused and case == "poisson32") else (not used or fused)
        x = t(torch_dev, np.zeros(A.n))
        st, it, rr = S.solve(t(torch_dev, f), x, rtol=1e-8, maxiter=300)
        xs = x.cpu().numpy()
        assert st == 0 and sto == 0 and _true_relres(A, xs, f) <= 1e-8
        assert abs(it - ito) <= 1, (fused, it, ito)
        assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
        z = t(torch_dev, np.zeros(A.n))
        amg.amg_apply_precond(S.handle, t(torch_dev, r), z)
        zs.append(z.cpu().numpy())
        S.close()
    _assert_vcycle_close(zs[0], zs[1])


def test_graph_and_host_loop_agree_bitwise(amg, torch_dev):
    """The graph solve (device-side while loop) and the host-launched loop
    give identical iterates; amg_last_solve_mode shows that the first really
    ran as a graph (a silent fall-back to host launches fails here) and the
    second from the host."""
    A = gen.varcoef3d(18, seed=9)
    f, _ = gen.rhs_from_solution(A, 1)
    xs = []
    for use_graph in (1, 0):
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val, coarse_enough=80, use_graph=use_graph)
        assert amg.amg_last_solve_mode(S.handle) == (0, 0)
        x = t(torch_dev, np.zeros(A.n))
        st, it, rr = S.solve(t(torch_dev, f), x)
        g, hst = amg.amg_last_solve_mode(S.handle)
        if use_graph:
            assert g >= 1 and hst == 0, (g, hst)
        else:
            assert g == 0 and hst >= 1, (g, hst)
        xs.append((x.cpu().numpy(), it, rr))
        S.close()
    assert np.array_equal(xs[0][0], xs[1][0]) and xs[0][1:] == xs[1][1:]


def _shifted_poisson(m, sigma):
    """7-point Poisson minus sigma on the diagonal: symmetric, indefinite once
    sigma exceeds the smallest eigenvalue, so CG breaks down."""
    A = gen.poisson3d(m)
    val = A.val.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    val[rows == A.col] -= sigma
    return type(A)(A.n, A.row_ptr, A.col, val)


# (m, sigma): the check that fails (Saad Alg. 9.1 needs r.z > 0 and p.q > 0)
# and the iteration it fails in, found with the oracle's own recurrences
BREAKDOWN_CASES = [(10, 0.5), (10, 1.0), (12, 2.0), (14, 3.0)]  # r.z at 3, p.q at 1, p.q at 0, r.z at 0


@pytest.mark.parametrize("m,sigma", BREAKDOWN_CASES)
def test_cg_breakdown_matches_oracle(amg, torch_dev, m, sigma):
    """CG on an indefinite matrix stops with BREAKDOWN where the oracle does,
    with x as of the last completed update (the x update that is still
    pending when the loop stops is applied after it, or dropped when the
    breakdown is in p.q), in the graph and in the host loop."""
    import oracle
    A = _shifted_poisson(m, sigma)
    f, _ = gen.rhs_from_solution(A, 4)
    xo, ito, rro, sto = oracle.Hierarchy(A, coarse_enough=50).cg(f)
    assert sto == oracle.BREAKDOWN
    for use_graph in (1, 0):
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val, coarse_enough=50, use_graph=use_graph)
        x = t(torch_dev, np.zeros(A.n))
        st, it, rr = S.solve(t(torch_dev, f), x)
        S.close()
        assert (st, it) == (amg.AMG_ERR_BREAKDOWN, ito), (st, it, ito)
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) <= 1e-9 * max(np.linalg.norm(xo), 1e-300) or (ito == 0 and not xg.any())
        assert abs(rr - rro) <= 1e-9 * rro


def test_programmatic_dependent_launch_same_result(amg, torch_dev):
    """use_pdl = 1 (consecutive streaming kernels overlap their start with
    the predecessor's tail; off by default) changes only the scheduling:
    the solve gives the same iterates bit for bit as with it off, in the
    graph and from the host, on a hierarchy that uses the fused restriction
    operators and the long-row engine (a dense row)."""
    for A, kw in ((gen.varcoef3d(18, seed=9), {"coarse_enough": 80}), (gen.poisson3d_star(24), {})):
        f, _ = gen.rhs_from_solution(A, 2)
        out = []
        for pdl, graph in ((0, 1), (1, 1), (1, 0)):
            S = amg.Solver(A.n, A.row_ptr, A.col, A.val, use_pdl=pdl, use_graph=graph, **kw)
            x = t(torch_dev, np.zeros(A.n))
            st, it, rr = S.solve(t(torch_dev, f), x)
            assert st == 0
            out.append((it, x.cpu().numpy()))
            S.close()
        for it, xs in out[1:]:
            assert it == out[0][0] and np.array_equal(xs, out[0][1])


def test_unaligned_solution_vector(amg, torch_dev):
    """x at an 8-byte offset (a view into a larger tensor, odd length): the
    solve runs on the caller's vector as it is and gives the same iterates
    as with an aligned x."""
    torch, dev = torch_dev
    A = gen.poisson3d(33)
    f, _ = gen.rhs_from_solution(A, 2)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
    ft = t(torch_dev, f)
    xa = torch.zeros(A.n, dtype=torch.float64, device=dev)
    big = torch.zeros(A.n + 1, dtype=torch.float64, device=dev)
    xu = big[1:]
    assert xu.data_ptr() % 16 == 8
    sa, ia, ra = S.solve(ft, xa, rtol=1e-8, maxiter=200)
    su, iu, ru = S.solve(ft, xu, rtol=1e-8, maxiter=200)
    assert sa == su == 0 and ra <= 1e-8 and ru <= 1e-8 and ia == iu
    assert torch.equal(xa, xu)
    S.close()


def test_repeat_solves_deterministic_and_host_buffers(amg, torch_dev):
    A = gen.poisson3d(24)
    f, _ = gen.rhs_from_solution(A, 2)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
    ft = t(torch_dev, f)
    out = []
    for _ in range(3):
        x = t(torch_dev, np.zeros(A.n))
        out.append((S.solve(ft, x), x.cpu().numpy()))
    assert all(np.array_equal(out[0][1], o[1]) and out[0][0] == o[0] for o in out)
    xh = np.zeros(A.n)
    res = amg.amg_solve_host(S.handle, np.ascontiguousarray(f), xh)
    assert res == out[0][0] and np.array_equal(xh, out[0][1])
    S.close()


def test_profile_solve_same_result(amg, torch_dev):
    A = gen.poisson3d(20)
    f, _ = gen.rhs_from_solution(A, 3)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val, coarse_enough=100)
    x1 = t(torch_dev, np.zeros(A.n))
    r1 = S.solve(t(torch_dev, f), x1)
    x2 = t(torch_dev, np.zeros(A.n))
    st, it, rr, ms, ln = amg.amg_solve_profile(S.handle, t(torch_dev, f), x2)
    assert (st, it, rr) == r1 and np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    assert ln["spmv_dot"] == it and ln["postsmooth_l0"] == it and ms["spmv_dot"] > 0
    S.close()


def test_standalone_spmv_dot(amg, torch_dev):
    import oracle
    torch, dev = torch_dev
    for A in (gen.poisson3d(30), gen.varcoef3d(11, seed=2), gen.poisson2d_shift(7, 0.0)):
        x = gen.uniform_pm1(1, 21, A.n)
        rp, cl, vl = (torch.from_numpy(a).to(dev) for a in (A.row_ptr, A.col, A.val))
        csr = amg.make_csr(A.n, rp, cl, vl)
        y = t(torch_dev, np.zeros(A.n))
        d = t(torch_dev, np.zeros(1))
        amg.amg_spmv_dot(csr, t(torch_dev, x), y, d)
        yo = oracle.spmv(A.n, A.n, A.row_ptr, A.col, A.val, x)
        assert np.all(np.abs(y.cpu().numpy() - yo) <= 64 * U * _row_bound(A.row_ptr, A.col, A.val, x))
        do = float(x @ yo)
        assert abs(d.item() - do) <= 1e-12 * np.abs(x * yo).sum()
    # broken structure is refused, not read out of bounds
    A = gen.poisson3d(6)
    bad_ptr = A.row_ptr.copy()
    bad_ptr[5] = bad_ptr[7]
    bad_col = A.col.copy()
    bad_col[3] = A.n + 5
    for p_, c_ in ((bad_ptr, A.col), (A.row_ptr, bad_col)):
        rp, cl, vl = (torch.from_numpy(a).to(dev) for a in (p_, c_, A.val))
        y = t(torch_dev, np.zeros(A.n))
        d = t(torch_dev, np.zeros(1))
        with pytest.raises(amg.AmgError) as e:
            amg.amg_spmv_dot(amg.make_csr(A.n, rp, cl, vl), t(torch_dev, np.ones(A.n)), y, d)
        assert e.value.status == amg.AMG_ERR_INVALID_ARG


def test_edge_cases(amg, torch_dev):
    import oracle
    # 1 x 1
    S = amg.Solver(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    x = t(torch_dev, np.zeros(1))
    assert S.solve(t(torch_dev, [8.0]), x) == (0, 1, 0.0) and x.item() == 2.0
    S.close()
    # single level (n <= coarse_enough): M = A^-1, one iteration
    A = gen.poisson3d(7)
    f, _ = gen.rhs_from_solution(A, 4)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
    assert S.info()["levels"] == 1
    x = t(torch_dev, np.zeros(A.n))
    st, it, rr = S.solve(t(torch_dev, f), x)
    assert (st, it) == (0, 1) and rr <= 1e-12
    S.close()
    A = gen.poisson3d(12)
    f, _ = gen.rhs_from_solution(A, 5)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val, coarse_enough=50)
    # f = 0 -> x = 0
    x = t(torch_dev, np.ones(A.n))
    assert S.solve(t(torch_dev, np.zeros(A.n)), x) == (0, 0, 0.0) and not x.any().item()
    # maxiter = 0
    x = t(torch_dev, np.zeros(A.n))
    st, it, rr = S.solve(t(torch_dev, f), x, maxiter=0)
    assert (st, it, rr) == (amg.AMG_ERR_NOT_CONVERGED, 0, 1.0)
    # exact initial guess
    xs = np.linalg.solve(A.to_dense(), f)
    x = t(torch_dev, xs)
    st, it, rr = S.solve(t(torch_dev, f), x)
    assert st == 0 and it == 0
    S.close()
    # non-finite right-hand side or initial guess: refused, not iterated on
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val, coarse_enough=50)
    fn = f.copy()
    fn[7] = np.nan
    with pytest.raises(amg.AmgError) as e:
        S.solve(t(torch_dev, fn), t(torch_dev, np.zeros(A.n)))
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    x0 = np.zeros(A.n)
    x0[3] = np.inf
    with pytest.raises(amg.AmgError) as e:
        S.solve(t(torch_dev, f), t(torch_dev, x0))
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    # the handle stays usable
    x = t(torch_dev, np.zeros(A.n))
    assert S.solve(t(torch_dev, f), x)[0] == 0
    S.close()
    # invalid inputs
    bad = gen.poisson3d(4)
    col = bad.col.copy()
    col[1], col[2] = col[2], col[1]
    with pytest.raises(amg.AmgError) as e:
        amg.Solver(bad.n, bad.row_ptr, col, bad.val)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    val = bad.val.copy()
    val[bad.row_ptr[3] + 1] = 0.0  # diagonal of row 3 (one lower neighbour before it)
    with pytest.raises(amg.AmgError) as e:
        amg.Solver(bad.n, bad.row_ptr, bad.col, val)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    # aggregation stall on a large diagonal matrix
    n = 5000
    with pytest.raises(amg.AmgError) as e:
        amg.Solver(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    assert e.value.status == amg.AMG_ERR_COARSENING_STALLED
    with pytest.raises(amg.AmgError) as e:
        amg.Solver(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert e.value.status == amg.AMG_ERR_INVALID_ARG


# iterations the mixed-precision V-cycles may add to the oracle's FP64 count
MIXED_SLACK = {1: 3, 2: 6}


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_vcycle_reaches_fp64_tolerance(amg, torch_dev, precision):
    """FP32 V-cycle, and FP32 V-cycle with bfloat16-stored values, under FP64
    CG: the FP64 tolerance is still reached, x within 1e-6 of the oracle's."""
    import oracle
    for A, kw in ((gen.poisson3d(32), {}), (gen.varcoef3d(24, seed=6), {"coarse_enough": 100}),
                  (gen.varcoef3d(24, seed=6), {"coarse_enough": 40, "use_tail": 1}),
                  (gen.poisson3d_star(24), {})):
        f, _ = gen.rhs_from_solution(A, 8)
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=precision, **kw)
        x = t(torch_dev, np.zeros(A.n))
        st, it, rr = S.solve(t(torch_dev, f), x, rtol=1e-8, maxiter=300)
        xs = x.cpu().numpy()
        H = oracle.Hierarchy(A, params=orc_params(**kw))
        xo, ito, rro, sto = H.cg(f, rtol=1e-8, maxiter=300)
        assert st == 0 and rr <= 1e-8 and _true_relres(A, xs, f) <= 1e-8
        assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
        assert it <= ito + MIXED_SLACK[precision], (it, ito)
        S.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_vcycle_bicgstab(amg, torch_dev, precision):
    """BiCGStab with the float32 V-cycle (whose finest level reads the float32
    copies of p and s that the Krylov kernels write) on a nonsymmetric
    convection-diffusion system: the FP64 tolerance is reached, x within 1e-6
    of the FP64 oracle's BiCGStab solution."""
    import oracle
    A = gen.convdiff3d(18, seed=2)[0]
    kw = {"solver": 1, "smoother": 1, "coarse_enough": 100}
    f, _ = gen.rhs_from_solution(A, 9)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=precision, **kw)
    x = t(torch_dev, np.zeros(A.n))
    st, it, rr = S.solve(t(torch_dev, f), x, rtol=1e-8, maxiter=300)
    xs = x.cpu().numpy()
    H = oracle.Hierarchy(A, params=orc_params(**kw))
    xo, ito, rro, sto = H.bicgstab(f, rtol=1e-8, maxiter=300)
    assert sto == 0 and st == 0 and rr <= 1e-8 and _true_relres(A, xs, f) <= 1e-8
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert it <= ito + MIXED_SLACK[precision], (it, ito)
    # the host-driven launches take the same float32 copies: same result
    S2 = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=precision, use_graph=0, **kw)
    x2 = t(torch_dev, np.zeros(A.n))
    st2, it2, rr2 = S2.solve(t(torch_dev, f), x2, rtol=1e-8, maxiter=300)
    assert (st2, it2) == (st, it) and np.array_equal(x2.cpu().numpy(), xs)
    S.close()
    S2.close()


def test_full_size_poisson150(amg, torch_dev):
    """The 150^3 workload the benchmark times: hierarchy sizes and sampled
    rows against the oracle, the solve against the oracle's solve."""
    import oracle
    A = gen.poisson3d(150)
    f, ustar = gen.rhs_from_solution(A, 0)
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
    H = oracle.Hierarchy(A)
    info = S.info()
    assert info["levels"] == H.levels
    for l in range(H.levels):
        assert info["rows"][l] == H.level_info(l)["n"] and info["nnz"][l] == H.level_info(l)["nnz"]
    # aggregates of the finest level, bit-exact
    assert np.array_equal(amg.amg_get_aggregates(S.handle, 0), H.aggregates(0))
    # sampled rows of the finest-level product
    x = gen.uniform_pm1(3, 22, A.n)
    y = t(torch_dev, np.zeros(A.n))
    amg.amg_level_spmv(S.handle, 0, "A", t(torch_dev, x), y)
    yg = y.cpu().numpy()
    rows = np.random.default_rng(0).choice(A.n, 2000, replace=False)
    for i in rows:
        k = slice(A.row_ptr[i], A.row_ptr[i + 1])
        assert abs(yg[i] - np.dot(A.val[k], x[A.col[k]])) <= 64 * U * np.abs(A.val[k] * x[A.col[k]]).sum()
    xd = t(torch_dev, np.zeros(A.n))
    st, it, rr = S.solve(t(torch_dev, f), xd, rtol=1e-8, maxiter=200)
    xs = xd.cpu().numpy()
    xo, ito, rro, sto = H.cg(f, rtol=1e-8, maxiter=200)
    assert st == 0 and rr <= 1e-8 and _true_relres(A, xs, f) <= 1e-8
    assert abs(it - ito) <= 1
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert np.linalg.norm(xs - ustar) <= 1e-5 * np.linalg.norm(ustar)
    S.close()
    # the mixed-precision forms of the same solve
    for precision in (1, 2):
        S = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=precision)
        xd = t(torch_dev, np.zeros(A.n))
        st, it, rr = S.solve(t(torch_dev, f), xd, rtol=1e-8, maxiter=200)
        xs = xd.cpu().numpy()
        assert st == 0 and rr <= 1e-8 and _true_relres(A, xs, f) <= 1e-8
        assert it <= ito + MIXED_SLACK[precision], (precision, it, ito)
        assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
        S.close()


def _transpose(ptr, col, val, ncols):
    """CSR transpose (rows sorted by column, stable), plain numpy."""
    rows = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    order = np.argsort(col, kind="stable")
    tptr = np.zeros(ncols + 1, np.int64)
    np.cumsum(np.bincount(col, minlength=ncols), out=tptr[1:])
    return tptr.astype(np.int32), rows[order].astype(np.int32), val[order]


def _sha(*arrays):
    import hashlib
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _sampled_x_check(x, gold, idx, rel):
    """x against the oracle's solution on the stored sample: every sampled
    |x_i - xo_i| <= rel max|xo|, and the sample's root-mean-square difference,
    scaled to all n entries, <= rel ||xo||_2 (the relative 2-norm bound,
    estimated on the sample).  Returns that estimate of ||x - xo|| / ||xo||."""
    xo = np.array([float.fromhex(v) for v in gold["sample"]["x"]])
    d = np.abs(x[idx] - xo)
    est = np.sqrt(np.mean(d * d) * gold["n"]) / gold["x_norm2"]
    assert d.max() <= rel * gold["x_norm_inf"], (d.max(), gold["x_norm_inf"])
    assert est <= rel, est
    return float(est)


def test_full_size_varcoef200(amg, torch_dev):
    """The 200^3 variable-coefficient workload (coefficients over six decades,
    10% anisotropic cells; 8M unknowns, 55.76M nonzeros) against the FP64
    oracle's own run of it (tests/golden/varcoef200_oracle.json, written by
    tests/golden/make_varcoef200.py from oracle/ alone):
      - the hierarchy bit for bit: every level's rows, nonzeros, matrix A_l
        and aggregates (SHA-256 over the same arrays), and level 0's
        prolongation against the oracle's step;
      - the FP64 solve: true residual <= 1e-8, the oracle's iteration count
        +/- 1, x within 1e-6 of the oracle's x on the stored sample;
      - the FP32 V-cycle under FP64 CG: the same, with at most 3 extra
        iterations;
      - the bfloat16-stored V-cycle: residual and iterations (<= oracle + 6);
        its distance from the oracle's x is reported, not bounded at 1e-6
        (values rounded to 8 significant bits on a problem whose solution is
        itself only 1e-5 from u*)."""
    import json
    import os
    import oracle
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "varcoef200_oracle.json")))
    A = gen.varcoef3d(200, seed=0)
    assert (A.n, A.nnz) == (gold["n"], gold["nnz"]) == (8_000_000, 55_760_000)
    f, ustar = gen.rhs_from_solution(A, 0)
    idx = gen.sample_indices(A.n, 8192, 0)
    assert len(idx) == gold["sample"]["count"]
    S = amg.Solver(A.n, A.row_ptr, A.col, A.val)
    info = S.info()
    assert info["levels"] == len(gold["levels"])
    for l, g in enumerate(gold["levels"]):
        assert (info["rows"][l], info["nnz"][l]) == (g["rows"], g["nnz"]), l
        ptr, col, val, _ = amg.amg_get_level_matrix(S.handle, l, "A")
        assert _sha(ptr.astype(np.int32), col, val) == g["A_sha256"], l
        del ptr, col, val
        if "aggregates_sha256" in g:
            assert _sha(amg.amg_get_aggregates(S.handle, l)) == g["aggregates_sha256"], l
            assert info["nnz_p"][l] == g["nnz_p"], l
    # level 0's prolongation against the oracle's step on the finest matrix
    agg, nagg = oracle.aggregate(A, 0.08)
    (pp, pc, pv), _ = oracle.prolongation(A, 0.08, agg, nagg)
    gp, gc, gv, gshape = amg.amg_get_level_matrix(S.handle, 0, "P")
    assert gshape == (A.n, nagg)
    assert np.array_equal(gp, pp) and np.array_equal(gc, pc) and np.array_equal(gv, pv)
    del pp, pc, pv, gp, gc, gv, agg
    ito = gold["iterations"]
    measured = {}
    for prec in (0, 1, 2):
        if prec:
            S = amg.Solver(A.n, A.row_ptr, A.col, A.val, precision=prec)
        x = t(torch_dev, np.zeros(A.n))
        st, it, rr = S.solve(t(torch_dev, f), x, rtol=1e-8, maxiter=500)
        xs = x.cpu().numpy()
        assert st == 0 and rr <= 1e-8 and _true_relres(A, xs, f) <= 1e-8, (prec, st, it, rr)
        assert np.linalg.norm(xs - ustar) <= 1e-4 * np.linalg.norm(ustar)
        if prec == 0:
            assert abs(it - ito) <= 1, (it, ito)
        else:
            assert it <= ito + MIXED_SLACK[prec], (prec, it, ito)
        if prec < 2:
            err = _sampled_x_check(xs, gold, idx, 1e-6)
        else:
            xo = np.array([float.fromhex(v) for v in gold["sample"]["x"]])
            err = float(np.sqrt(np.mean((xs[idx] - xo) ** 2) * gold["n"]) / gold["x_norm2"])
        measured[("fp64", "fp32", "bf16")[prec]] = {"iterations": it, "oracle_iterations": ito,
                                                    "rel_err_vs_oracle_x": err}
        S.close()
    print("varcoef200 vs oracle:", measured)
