"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties one oracle function to a closed form, a hand-derived value, a
mathematical invariant, dense linear algebra (numpy) on a tiny input, or the
figure the paper prints (Sec. 4.1).  Chosen so that a dropped term, a wrong
sign, a wrong index or a transposed operand in the oracle fails at least one.
"""
import json
import os

import numpy as np
import pytest

import gen
from gen import Csr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_from_dense(d):
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    ptr = [0]
    col, val = [], []
    for i in range(n):
        for j in range(n):
            if d[i, j] != 0.0 or i == j:
                col.append(j)
                val.append(d[i, j])
        ptr.append(len(col))
    return Csr(n, np.array(ptr, np.int32), np.array(col, np.int32), np.array(val))


def laplace1d(n, diag=2.0):
    return csr_from_dense(diag * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))


def dense_from(ptr, col, val, shape):
    d = np.zeros(shape)
    rows = np.repeat(np.arange(shape[0]), np.diff(ptr))
    d[rows, col] = val
    return d


# ------------------------------------------------------------------ inputs
def test_paper_poisson150_size():
    """Sec. 4.1: 150^3 Poisson has 3,375,000 unknowns and 23,490,000 nonzeros."""
    g = json.load(open(os.path.join(GOLDEN, "paper_poisson150.json")))
    A = gen.poisson3d(g["grid_side"])
    assert A.n == g["unknowns"]
    assert A.nnz == g["nonzeros"]
    assert gen.poisson3d_nnz(150) == g["nonzeros"]


def test_generators_structure():
    A = gen.poisson3d(5)
    d = A.to_dense()
    assert np.array_equal(d, d.T)
    assert np.all(np.diff(A.col[A.row_ptr[0]:A.row_ptr[1]]) > 0)
    B = gen.varcoef3d(5, seed=3)
    db = B.to_dense()
    assert np.allclose(db, db.T, rtol=0, atol=1e-12 * np.abs(db).max())
    assert np.linalg.eigvalsh(db).min() > 0
    C, v, pe = gen.convdiff3d(5, seed=3)
    dc = C.to_dense()
    assert not np.allclose(dc, dc.T)
    assert abs(np.linalg.norm(v) - 1.0) < 1e-14 and 1.0 <= pe <= 100.0
    # row sums of interior rows vanish (diffusion + upwinding conserve)
    assert np.abs(dc.sum(1)).min() < 1e-12
    S = gen.poisson3d_star(5, w=0.5)
    ds = S.to_dense()
    assert np.array_equal(ds, ds.T) and np.linalg.eigvalsh(ds).min() > 0
    assert np.count_nonzero(ds[0]) == S.n and all(np.all(np.diff(S.col[S.row_ptr[i]:S.row_ptr[i + 1]]) > 0)
                                                   for i in range(S.n))
    # the star adds a graph Laplacian: row sums equal poisson3d's
    assert np.allclose(ds.sum(1), d.sum(1))


# ---------------------------------------------------------------- strength
def test_strength_poisson_all_strong(oracle_lib):
    A = gen.poisson3d(4)
    s = oracle_lib.strength(A, 0.08)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    offdiag = A.col != rows
    # 1 > 0.0064 * 36: every neighbour is strong, the diagonal never is
    assert s[offdiag].all() and not s[~offdiag].any()


def test_strength_threshold_is_strict_and_squared(oracle_lib):
    A = csr_from_dense([[1.0, -0.5], [-0.5, 1.0]])
    # a_ij^2 = 0.25 = eps^2 |a_ii a_jj| at eps = 0.5: not strong (strict)
    assert not oracle_lib.strength(A, 0.5).any()
    assert oracle_lib.strength(A, 0.49).sum() == 2
    # diagonal scaling: a_ii a_jj = 4 -> threshold eps^2 * 4
    B = csr_from_dense([[2.0, 0.5], [0.5, 2.0]])
    assert oracle_lib.strength(B, 0.249).sum() == 2
    assert not oracle_lib.strength(B, 0.25).any()


def test_strength_anisotropic_keeps_x_lines(oracle_lib):
    m = 6
    n = m * m
    d = np.zeros((n, n))
    for j in range(m):
        for i in range(m):
            r = i + m * j
            d[r, r] = 2.0 + 2.0e-3
            if i > 0:
                d[r, r - 1] = -1.0
            if i < m - 1:
                d[r, r + 1] = -1.0
            if j > 0:
                d[r, r - m] = -1e-3
            if j < m - 1:
                d[r, r + m] = -1e-3
    A = csr_from_dense(d)
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    ys = np.arange(n) // m
    for a in range(nagg):
        assert len(set(ys[agg == a])) == 1, "aggregate crosses a weak (y) connection"


# -------------------------------------------------------------- aggregation
@pytest.mark.parametrize("n,expected", [
    # pass 1 on a path graph: roots 0, 3, 6, 9 ...; hand-derived
    (4, [0, 0, 1, 1]),
    (5, [0, 0, 1, 1, 1]),
    (6, [0, 0, 1, 1, 1, 1]),       # node 5 joins via pass 2
    (10, [0, 0, 1, 1, 1, 2, 2, 2, 3, 3]),
    (11, [0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3]),
])
def test_aggregation_path_graph(oracle_lib, n, expected):
    agg, nagg = oracle_lib.aggregate(laplace1d(n), 0.08)
    assert agg.tolist() == expected
    assert nagg == max(expected) + 1


def test_aggregation_grid_3x3(oracle_lib):
    # 5-point 3x3 grid, node = i + 3j.  Pass 1: root 0 takes {0,1,3}; nodes
    # 2, 4 have aggregated neighbours; root 5 takes {2,4,5,8}; 6, 7 skip.
    # Pass 2: 6 -> neighbour 3 (agg 0); 7 -> neighbours 4, 8 (agg 1).
    A = gen.poisson2d_shift(3, 0.0)
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    assert agg.tolist() == [0, 0, 1, 0, 1, 1, 0, 1, 1]
    assert nagg == 2


def _tie_matrix(a43):
    # edges 0-2, 1-3, 2-4, 3-4; pass 1 makes {0,2} and {1,3}; node 4 is left
    d = 4.0 * np.eye(5)
    for i, j, w in [(0, 2, 1.0), (1, 3, 1.0), (2, 4, 1.0), (3, 4, a43)]:
        d[i, j] = d[j, i] = -w
    return csr_from_dense(d)


def test_aggregation_pass2_tie_goes_to_smallest_neighbour(oracle_lib):
    agg, nagg = oracle_lib.aggregate(_tie_matrix(1.0), 0.08)
    assert agg.tolist() == [0, 1, 0, 1, 0] and nagg == 2


def test_aggregation_pass2_takes_strongest(oracle_lib):
    agg, _ = oracle_lib.aggregate(_tie_matrix(2.0), 0.08)
    assert agg.tolist() == [0, 1, 0, 1, 1]


def test_aggregation_isolated_node_is_singleton_first(oracle_lib):
    d = 2.0 * np.eye(5)
    d[0, 1] = d[1, 0] = -1.0
    d[3, 4] = d[4, 3] = -1.0
    agg, nagg = oracle_lib.aggregate(csr_from_dense(d), 0.08)
    assert agg.tolist() == [1, 1, 0, 2, 2] and nagg == 3


@pytest.mark.parametrize("maker", [
    lambda: gen.poisson3d(7),
    lambda: gen.varcoef3d(7, seed=1),
    lambda: gen.convdiff3d(7, seed=2)[0],
    lambda: gen.poisson2d_shift(13, 0.05),
])
def test_aggregates_partition_and_connected(oracle_lib, maker):
    A = maker()
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    assert agg.min() == 0 and agg.max() == nagg - 1
    assert len(np.unique(agg)) == nagg  # every id used, every node exactly once
    # each aggregate is connected in the graph of strong connections
    s = oracle_lib.strength(A, 0.08)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    adj = {}
    for r, c in zip(rows[s], A.col[s]):
        adj.setdefault(int(r), set()).add(int(c))
        adj.setdefault(int(c), set()).add(int(r))
    for a in range(nagg):
        members = set(np.nonzero(agg == a)[0].tolist())
        start = next(iter(members))
        seen, stack = {start}, [start]
        while stack:
            u = stack.pop()
            for w in adj.get(u, ()):
                if w in members and w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert seen == members


# ------------------------------------------------------------- prolongation
def test_tentative_orthonormal_columns(oracle_lib):
    A = gen.poisson3d(6)
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    t = oracle_lib.tentative_values(agg, nagg)
    Pt = np.zeros((A.n, nagg))
    Pt[np.arange(A.n), agg] = t
    assert np.allclose(Pt.T @ Pt, np.eye(nagg), rtol=0, atol=1e-15)
    assert (t > 0).all()


def test_prolongation_damping_poisson(oracle_lib):
    # Gershgorin on 7-point Poisson: interior rows give (6 + 6)/6 = 2 -> 4/3 / 2
    A = gen.poisson3d(5)
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    _, omega = oracle_lib.prolongation(A, 0.08, agg, nagg)
    assert omega == (4.0 / 3.0) / 2.0


def test_prolongation_preserves_constant_on_interior(oracle_lib):
    # A 1 = 0 on rows away from the boundary, so (I - w D^-1 A) keeps the
    # constant there: P s = 1 with s_J = sqrt(|J|).  Holds with lumping too
    # (lumping keeps row sums), so use the anisotropic problem as well.
    for A in (gen.poisson3d(7), gen.poisson2d_shift(9, 0.0)):
        agg, nagg = oracle_lib.aggregate(A, 0.08)
        (ptr, col, val), _ = oracle_lib.prolongation(A, 0.08, agg, nagg)
        P = dense_from(ptr, col, val, (A.n, nagg))
        s = np.sqrt(np.bincount(agg, minlength=nagg).astype(float))
        Ps = P @ s
        rowsum = A.to_dense().sum(1)
        interior = np.abs(rowsum) < 1e-14
        assert interior.sum() > 0
        assert np.allclose(Ps[interior], 1.0, rtol=0, atol=1e-13)
        # and P differs from P_t (the smoothing really happened)
        Pt = np.zeros_like(P)
        Pt[np.arange(A.n), agg] = oracle_lib.tentative_values(agg, nagg)
        assert np.abs(P - Pt).max() > 0.05


def test_prolongation_lumping_anisotropic(oracle_lib):
    # x-coupling -1 strong, y-coupling -e weak (e = 1e-3).  Lumped diagonal
    # aF = a_ii - (sum of weak) = (2 + 2e) + (number of y-neighbours) e.  The
    # Gershgorin ratio (aF + sum of strong |a_ij|)/aF is largest where aF is
    # smallest with two x-neighbours: rows on the y-boundary, aF = 2 + 3e, so
    # rho = (4 + 3e)/(2 + 3e) and omega = 4/3 / rho (derived by hand).
    m, e = 6, 1e-3
    n = m * m
    d = np.zeros((n, n))
    for j in range(m):
        for i in range(m):
            r = i + m * j
            d[r, r] = 2.0 + 2.0 * e
            for di, dj, w in [(-1, 0, 1.0), (1, 0, 1.0), (0, -1, e), (0, 1, e)]:
                ii, jj = i + di, j + dj
                if 0 <= ii < m and 0 <= jj < m:
                    d[r, ii + m * jj] = -w
    A = csr_from_dense(d)
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    _, omega = oracle_lib.prolongation(A, 0.08, agg, nagg)
    aF = 2.0 + 3.0 * e
    assert abs(omega - (4.0 / 3.0) / ((aF + 2.0) / aF)) < 1e-15


def test_prolongation_reduces_column_energy(oracle_lib):
    # (I - w D^-1 A) with 0 < w lambda_max(D^-1 A) < 2 is an A-norm contraction:
    # each smoothed column has lower energy than its tentative column.  A sign
    # error in the smoothing step raises the energy instead.
    A = gen.poisson3d(6)
    Ad = A.to_dense()
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    (ptr, col, val), _ = oracle_lib.prolongation(A, 0.08, agg, nagg)
    P = dense_from(ptr, col, val, (A.n, nagg))
    Pt = np.zeros_like(P)
    Pt[np.arange(A.n), agg] = oracle_lib.tentative_values(agg, nagg)
    e_s = np.einsum("ij,ik,kj->j", P, Ad, P)
    e_t = np.einsum("ij,ik,kj->j", Pt, Ad, Pt)
    assert (e_s < e_t).all()


def test_prolongation_pattern_is_structural_union(oracle_lib):
    A = gen.poisson3d(5)
    agg, nagg = oracle_lib.aggregate(A, 0.08)
    (ptr, col, val), _ = oracle_lib.prolongation(A, 0.08, agg, nagg)
    Pt = np.zeros((A.n, nagg), bool)
    Pt[np.arange(A.n), agg] = True
    pattern = (A.to_dense() != 0).astype(int) @ Pt.astype(int) > 0
    got = np.zeros_like(pattern)
    got[np.repeat(np.arange(A.n), np.diff(ptr)), col] = True
    assert np.array_equal(got, pattern | Pt)


# ----------------------------------------------------------------- smoothers
def test_jacobi_diagonal(oracle_lib):
    A = gen.varcoef3d(4, seed=5)
    d = oracle_lib.smoother_diag(A, oracle_lib.default_params(smoother=0))
    assert np.allclose(d * np.diag(A.to_dense()), 0.72, rtol=1e-15)


def test_spai0_is_frobenius_optimal(oracle_lib):
    A = gen.convdiff3d(4, seed=5)[0]
    Ad = A.to_dense()
    d = oracle_lib.smoother_diag(A, oracle_lib.default_params(smoother=1))

    def rowres(i, di):
        r = -di * Ad[i]
        r[i] += 1.0
        return r @ r

    for i in range(0, A.n, 7):
        f0 = rowres(i, d[i])
        for h in (1e-3, -1e-3):
            assert f0 < rowres(i, d[i] * (1 + h))
    # a diagonal matrix is inverted exactly
    D = csr_from_dense(np.diag([2.0, 4.0, 0.5]))
    assert np.allclose(oracle_lib.smoother_diag(D, oracle_lib.default_params(smoother=1)),
                       [0.5, 0.25, 2.0], rtol=1e-15)


# ------------------------------------------------------------ R, RAP, solver
def _hier(A, **kw):
    import oracle
    return oracle.Hierarchy(A, **kw)


def test_restriction_is_transpose(oracle_lib):
    H = _hier(gen.poisson3d(10), coarse_enough=50)
    assert H.levels >= 3
    for l in range(H.levels - 1):
        assert np.array_equal(H.dense(l, "R"), H.dense(l, "P").T)


@pytest.mark.parametrize("maker", [
    lambda: gen.poisson3d(8),
    lambda: gen.varcoef3d(8, seed=4),
    lambda: gen.convdiff3d(8, seed=4)[0],
    lambda: gen.poisson3d_star(8),
])
def test_galerkin_equals_dense_triple_product(oracle_lib, maker):
    A = maker()
    H = _hier(A, coarse_enough=20)
    assert H.levels >= 3
    for l in range(H.levels - 1):
        Ad, Pd, Rd = H.dense(l, "A"), H.dense(l, "P"), H.dense(l, "R")
        Ac = H.dense(l + 1, "A")
        ref = Rd @ Ad @ Pd
        assert np.abs(Ac - ref).max() <= 1e-13 * np.abs(ref).max()
        # structural pattern (numerical zeros kept)
        pat = ((Rd != 0).astype(int) @ (Ad != 0).astype(int) @ (Pd != 0).astype(int)) > 0
        ptr, col, _, shape = H.matrix(l + 1, "A")
        got = np.zeros(shape, bool)
        got[np.repeat(np.arange(shape[0]), np.diff(ptr)), col] = True
        assert np.array_equal(got, pat)


def test_spgemm_standalone_matches_dense(oracle_lib):
    rng = np.random.default_rng(0)
    a = (rng.random((30, 20)) < 0.2) * rng.standard_normal((30, 20))
    b = (rng.random((20, 25)) < 0.2) * rng.standard_normal((20, 25))

    def to_csr(d):
        ptr, col, val = [0], [], []
        for row in d:
            nz = np.nonzero(row)[0]
            col += nz.tolist()
            val += row[nz].tolist()
            ptr.append(len(col))
        return np.array(ptr, np.int32), np.array(col, np.int32), np.array(val)

    ptr, col, val = oracle_lib.spgemm(30, 20, 25, to_csr(a), to_csr(b))
    assert np.allclose(dense_from(ptr, col, val, (30, 25)), a @ b, rtol=0, atol=1e-14)
    for i in range(30):
        assert np.all(np.diff(col[ptr[i]:ptr[i + 1]]) > 0)


def _level_csr(H, l):
    ptr, col, val, shape = H.matrix(l, "A")
    return Csr(shape[0], ptr.astype(np.int32), col, val)


def test_strength_schedule_halves_per_level(oracle_lib):
    """The strength threshold of level l is eps_0 * 0.5^l (the schedule of the
    smoothed aggregation that Sec. 3 cites, Vanek, Mandel and Brezina 1996),
    and a constant eps_0 with the halving switched off.  Each level's
    aggregates inside the hierarchy must equal the standalone aggregation of
    that level's matrix at the scheduled threshold.  The problem is chosen so
    that on levels 1 and 2 the thresholds eps/2, eps and 2 eps give three
    different aggregations: skipping the halving, applying it twice per level
    or starting it one level early each fails."""
    A = gen.varcoef3d(10, seed=0)
    H = _hier(A, coarse_enough=20)
    assert H.levels >= 4
    for l in (1, 2, 3):
        eps = 0.08 * 0.5 ** l
        Al = _level_csr(H, l)
        got = H.aggregates(l)
        want, nagg = oracle_lib.aggregate(Al, eps)
        assert np.array_equal(got, want), l
        assert H.level_info(l + 1)["n"] == nagg
        if l < 3:
            for wrong in (2 * eps, 0.5 * eps):
                assert not np.array_equal(got, oracle_lib.aggregate(Al, wrong)[0]), (l, wrong)
    # the finest level always uses eps_0
    assert np.array_equal(H.aggregates(0), oracle_lib.aggregate(A, 0.08)[0])
    # constant threshold with the halving off: level 1 aggregates at eps_0;
    # level 2 then keeps more than 95% of its rows at eps_0 (the stall rule
    # makes it the coarsest), where the halved threshold would coarsen on
    H0 = _hier(A, coarse_enough=20, eps_halving=0)
    A1 = _level_csr(H0, 1)
    got = H0.aggregates(1)
    assert np.array_equal(got, oracle_lib.aggregate(A1, 0.08)[0])
    assert not np.array_equal(got, oracle_lib.aggregate(A1, 0.04)[0])
    A2 = _level_csr(H0, 2)
    assert H0.levels == 3
    assert oracle_lib.aggregate(A2, 0.08)[1] >= 0.95 * A2.n
    assert oracle_lib.aggregate(A2, 0.04)[1] < 0.95 * A2.n


def test_coarse_levels_symmetric(oracle_lib):
    H = _hier(gen.varcoef3d(12, seed=2), coarse_enough=30)
    assert H.levels >= 3
    for l in range(1, H.levels):
        ptr, col, val, shape = H.matrix(l, "A")
        d = dense_from(ptr, col, val, shape)
        assert np.array_equal(d != 0, (d != 0).T) or np.array_equal(
            np.abs(d) > 0, np.abs(d.T) > 0)
        assert np.abs(d - d.T).max() <= 1e-14 * np.abs(d).max()


def test_dense_solver_with_pivoting(oracle_lib):
    a = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    b = np.array([1.0, 2.0, 3.0])
    assert np.allclose(oracle_lib.dense_solve(a, b), np.linalg.solve(a, b), rtol=1e-14)
    rng = np.random.default_rng(1)
    m = rng.standard_normal((60, 60)) + 8 * np.eye(60)
    v = rng.standard_normal(60)
    assert np.allclose(oracle_lib.dense_solve(m, v), np.linalg.solve(m, v), rtol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        oracle_lib.dense_solve(np.zeros((2, 2)), np.ones(2))


# ---------------------------------------------------------------- V-cycle
def _vcycle_operator(H, n):
    return np.stack([H.vcycle(e) for e in np.eye(n)], axis=1)


@pytest.mark.parametrize("npre,npost,smoother", [(1, 1, 0), (2, 0, 0), (0, 2, 1), (1, 2, 1)])
def test_vcycle_closed_form(oracle_lib, npre, npost, smoother):
    # I - M_l A_l = S^npost (I - P_l M_{l+1} R_l A_l) S^npre, S = I - D_l A_l,
    # M_{L-1} = A_{L-1}^{-1}: the multilevel error propagation of Algorithm 2
    # with zero initial guess, evaluated with dense matrices.
    A = gen.varcoef3d(8, seed=7)
    H = _hier(A, coarse_enough=25, npre=npre, npost=npost, smoother=smoother)
    L = H.levels
    assert L >= 3
    M = np.linalg.inv(H.dense(L - 1, "A"))
    for l in range(L - 2, -1, -1):
        Al, Pl, Rl = H.dense(l, "A"), H.dense(l, "P"), H.dense(l, "R")
        S = np.eye(Al.shape[0]) - np.diag(H.smoother_diagonal(l)) @ Al
        E = (np.linalg.matrix_power(S, npost) @ (np.eye(Al.shape[0]) - Pl @ M @ Rl @ Al)
             @ np.linalg.matrix_power(S, npre))
        M = (np.eye(Al.shape[0]) - E) @ np.linalg.inv(Al)
    Mo = _vcycle_operator(H, A.n)
    assert np.abs(Mo - M).max() <= 1e-11 * np.abs(M).max()


def test_vcycle_symmetric_for_symmetric_smoothing(oracle_lib):
    A = gen.poisson3d(7)
    H = _hier(A, coarse_enough=30)
    M = _vcycle_operator(H, A.n)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


# ----------------------------------------------------------------- Krylov
def test_single_level_cg_is_one_iteration(oracle_lib):
    A = gen.poisson3d(6)       # 216 <= 500 rows: M = A^-1
    f, _ = gen.rhs_from_solution(A, 1)
    H = _hier(A)
    assert H.levels == 1
    x, it, rr, st = H.cg(f, rtol=1e-10)
    assert (it, st) == (1, 0)
    assert np.allclose(x, np.linalg.solve(A.to_dense(), f), rtol=1e-12, atol=1e-12)
    x, it, rr, st = H.bicgstab(f, rtol=1e-10)   # half step: alpha = 1, s = 0
    assert (it, st) == (1, 0)


def test_cg_iterates_are_krylov_optimal(oracle_lib):
    # CG with SPD M minimises ||x - x*||_A over span{z0, (MA) z0, ...}: compare
    # x_k (maxiter = k) with the Galerkin projection onto that space.
    A = gen.varcoef3d(6, seed=9)
    Ad = A.to_dense()
    H = _hier(A, coarse_enough=20)
    assert H.levels >= 2
    M = _vcycle_operator(H, A.n)
    f, _ = gen.rhs_from_solution(A, 3)
    xs = np.linalg.solve(Ad, f)
    prev = np.inf
    for k in range(1, 6):
        x, it, rr, st = H.cg(f, rtol=1e-30, maxiter=k)
        assert it == k and st == 4
        K = [M @ f]
        for _ in range(k - 1):
            K.append(M @ (Ad @ K[-1]))
        V, _ = np.linalg.qr(np.stack(K, axis=1))
        V, _ = np.linalg.qr(V)
        y = np.linalg.solve(V.T @ Ad @ V, V.T @ f)
        xk = V @ y
        assert np.linalg.norm(x - xk) <= 1e-8 * np.linalg.norm(xk)
        err = np.sqrt((x - xs) @ Ad @ (x - xs))
        assert err < prev
        prev = err
        # the reported residual is the true one
        assert abs(rr - np.linalg.norm(f - Ad @ x) / np.linalg.norm(f)) <= 1e-12


def test_cg_recovers_solution_32cubed(oracle_lib):
    A = gen.poisson3d(32)
    f, ustar = gen.rhs_from_solution(A, 0)
    H = _hier(A)
    x, it, rr, st = H.cg(f, rtol=1e-8)
    assert st == 0 and rr <= 1e-8
    assert np.linalg.norm(x - ustar) / np.linalg.norm(ustar) <= 1e-5
    assert 5 <= it <= 30


def test_bicgstab_nonsymmetric_matches_dense_solve(oracle_lib):
    A, _, _ = gen.convdiff3d(9, seed=11)
    f, ustar = gen.rhs_from_solution(A, 4)
    H = _hier(A, coarse_enough=40)
    assert H.levels >= 2
    x, it, rr, st = H.bicgstab(f, rtol=1e-10)
    assert st == 0 and rr <= 1e-10
    xs = np.linalg.solve(A.to_dense(), f)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert abs(rr - np.linalg.norm(f - A.to_dense() @ x) / np.linalg.norm(f)) <= 1e-14
    # CG on the same hierarchy with SPAI-0 also converges for SPD variants
    B = gen.varcoef3d(9, seed=11)
    g, _ = gen.rhs_from_solution(B, 4)
    HB = _hier(B, coarse_enough=40, smoother=1)
    x, it, rr, st = HB.bicgstab(g, rtol=1e-10)
    assert st == 0 and rr <= 1e-10


def test_krylov_edge_cases(oracle_lib):
    import oracle
    A = gen.poisson3d(9)
    H = _hier(A, coarse_enough=50)
    # f = 0: x = 0, no iterations
    x, it, rr, st = H.cg(np.zeros(A.n), x0=np.ones(A.n))
    assert (it, rr, st) == (0, 0.0, 0) and not x.any()
    # maxiter = 0: not converged, true residual reported
    f, _ = gen.rhs_from_solution(A, 2)
    x, it, rr, st = H.cg(f, maxiter=0)
    assert (it, st) == (0, oracle.NOT_CONVERGED) and rr == 1.0
    x, it, rr, st = H.bicgstab(f, maxiter=1, rtol=1e-12)
    assert (it, st) == (1, oracle.NOT_CONVERGED)
    # exact initial guess: nothing to do
    xs = np.linalg.solve(A.to_dense(), f)
    x, it, rr, st = H.cg(f, x0=xs, rtol=1e-8)
    assert it == 0 and st == 0


def test_setup_edge_cases(oracle_lib):
    import oracle
    # 1 x 1 system
    H = _hier(csr_from_dense([[3.0]]))
    x, it, rr, st = H.cg(np.array([6.0]))
    assert (it, st) == (1, 0) and x[0] == 2.0
    # zero diagonal: invalid
    with pytest.raises(oracle.OracleError) as e:
        _hier(csr_from_dense([[0.0, 1.0], [1.0, 2.0]]))
    assert e.value.status == oracle.INVALID
    # aggregation stall on a diagonal matrix: small -> one dense level, big -> error
    n = 1000
    D = Csr(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    H = _hier(D)
    assert H.levels == 1
    n = 5000
    D = Csr(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    with pytest.raises(oracle.OracleError) as e:
        _hier(D)
    assert e.value.status == oracle.STALLED


def test_setup_is_deterministic(oracle_lib):
    A = gen.varcoef3d(10, seed=3)
    H1, H2 = _hier(A, coarse_enough=40), _hier(A, coarse_enough=40)
    assert H1.levels == H2.levels
    for l in range(H1.levels):
        for w in "APR" if l < H1.levels - 1 else "A":
            a, b = H1.matrix(l, w), H2.matrix(l, w)
            assert all(np.array_equal(u, v) for u, v in zip(a[:3], b[:3]))


def test_bicgstab_first_step_conditions(oracle_lib):
    # One full BiCGStab step from x0 = 0 (r^ = f): alpha is fixed by the BiCG
    # condition r^.s = 0 with s = (I - alpha A M) f; omega minimises
    # ||s - omega t|| with t = A M s, i.e. the new residual is orthogonal to t.
    A, _, _ = gen.convdiff3d(7, seed=6)
    Ad = A.to_dense()
    H = _hier(A, coarse_enough=40)
    M = _vcycle_operator(H, A.n)
    f, _ = gen.rhs_from_solution(A, 5)
    x1, it, rr, st = H.bicgstab(f, rtol=1e-30, maxiter=1)
    assert it == 1
    AMf = Ad @ (M @ f)
    alpha = (f @ f) / (f @ AMf)
    s = f - alpha * AMf
    assert abs(f @ s) <= 1e-12 * np.linalg.norm(f) * np.linalg.norm(s)
    t = Ad @ (M @ s)
    r1 = f - Ad @ x1
    assert abs(r1 @ t) <= 1e-10 * np.linalg.norm(r1) * np.linalg.norm(t)
    assert np.linalg.norm(r1) < np.linalg.norm(s)
    omega = (t @ s) / (t @ t)
    assert np.linalg.norm(x1 - (alpha * (M @ f) + omega * (M @ s))) <= 1e-10 * np.linalg.norm(x1)
