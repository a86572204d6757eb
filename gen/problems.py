"""Model problems (sparse matrices in CSR) and right-hand sides.

All matrices are square CSR with int32 row pointers and column indices (sorted
ascending within each row, no duplicates) and float64 values.  Unknowns of a
d-dimensional grid with side m are the interior nodes, numbered
lexicographically: i + m*(j + m*k).  Homogeneous Dirichlet neighbours are
eliminated (their columns are dropped), so a 7-point 3D stencil on m^3 nodes
has 7*m^3 - 6*m^2 nonzeros: 23,490,000 for m = 150, the figure Sec. 4.1 of the
paper gives for its Poisson benchmark.  Mesh-size scaling (1/h^2) is omitted:
it multiplies A by a constant and does not change x for f = A u*.

Stream numbers used with ``gen.rng``: 1 cell coefficients, 2 anisotropy mask,
3 velocity / Peclet number, 4 diagonal shift, 10 solution vector u*, 11 direct
right-hand sides.
"""
from dataclasses import dataclass

import numpy as np

from .rng import uniform01

STREAM_COEF = 1
STREAM_ANISO = 2
STREAM_VEL = 3
STREAM_SHIFT = 4
STREAM_USTAR = 10
STREAM_RHS = 11
STREAM_KIND = 20
STREAM_REUSE = 21
STREAM_PICK = 22
STREAM_ARRIVAL = 23
STREAM_SAMPLE = 30
STREAM_REQ_RHS = 100000  # + request index
SERVE_VARCOEF_RANGE = (-2.0, 2.0)  # log10 of the cell coefficients of served SPD requests


@dataclass
class Csr:
    n: int
    row_ptr: np.ndarray  # int32, n+1
    col: np.ndarray      # int32, nnz
    val: np.ndarray      # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def poisson3d_nnz(m: int) -> int:
    """nnz of the 7-point stencil with eliminated Dirichlet neighbours."""
    return 7 * m ** 3 - 6 * m ** 2


def _assemble(n: int, offsets, cols_list, vals_list, mask_list) -> Csr:
    """Pack per-row neighbour slots (already in ascending column order) into CSR."""
    cols = np.stack(cols_list, axis=1)
    vals = np.stack(vals_list, axis=1)
    mask = np.stack(mask_list, axis=1)
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("problem too large for int32 row pointers")
    col = cols[mask].astype(np.int32)
    val = vals[mask].astype(np.float64)
    return Csr(n, row_ptr.astype(np.int32), col, val)


def _grid3(m: int):
    idx = np.arange(m ** 3, dtype=np.int64)
    i = idx % m
    j = (idx // m) % m
    k = idx // (m * m)
    return idx, i, j, k


def poisson3d(m: int) -> Csr:
    """7-point -Laplacian on an m^3 interior grid: diagonal 6, -1 per in-grid neighbour."""
    n = m ** 3
    idx, i, j, k = _grid3(m)
    offs = [-m * m, -m, -1, 0, 1, m, m * m]
    masks = [k > 0, j > 0, i > 0, np.ones(n, bool), i < m - 1, j < m - 1, k < m - 1]
    cols = [idx + o for o in offs]
    vals = [np.full(n, -1.0) if o != 0 else np.full(n, 6.0) for o in offs]
    return _assemble(n, offs, cols, vals, masks)


def poisson3d_star(m: int, w: float = 1.0) -> Csr:
    """poisson3d(m) plus a star: node 0 coupled to every other node with weight
    w (graph-Laplacian entries: -w off the diagonal, +w on node j's diagonal,
    (n-1) w on node 0's).  SPD, with one dense row and column, so the coarse
    operators carry a row as wide as the coarse level (an edge case of the
    Galerkin product)."""
    P = poisson3d(m)
    n = P.n
    rows = np.repeat(np.arange(n), np.diff(P.row_ptr))
    cols = P.col.astype(np.int64)
    vals = P.val.copy()
    vals[(rows == cols) & (rows > 0)] += w
    vals[(rows == 0) & (cols == 0)] += (n - 1) * w
    # the star's off-diagonal entries not already present in the stencil
    have0 = set(cols[rows == 0].tolist())
    extra = np.array([j for j in range(1, n) if j not in have0], dtype=np.int64)
    vals[(rows == 0) & (cols > 0)] += -w
    vals[(cols == 0) & (rows > 0)] += -w
    r = np.concatenate([rows, np.zeros(len(extra), np.int64), extra])
    c = np.concatenate([cols, extra, np.zeros(len(extra), np.int64)])
    v = np.concatenate([vals, np.full(len(extra), -w), np.full(len(extra), -w)])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=row_ptr[1:])
    return Csr(n, row_ptr.astype(np.int32), c.astype(np.int32), v)


def poisson2d_shift(m: int, sigma: float) -> Csr:
    """5-point -Laplacian on an m^2 interior grid with diagonal 4 + sigma."""
    n = m * m
    idx = np.arange(n, dtype=np.int64)
    i = idx % m
    j = idx // m
    offs = [-m, -1, 0, 1, m]
    masks = [j > 0, i > 0, np.ones(n, bool), i < m - 1, j < m - 1]
    cols = [idx + o for o in offs]
    vals = [np.full(n, -1.0) if o != 0 else np.full(n, 4.0 + sigma) for o in offs]
    return _assemble(n, offs, cols, vals, masks)


# Transcendental functions of numpy and libm may round differently on
# different machines (vectorised implementations, contracted multiply-adds),
# which would make the same seed give different matrices on the x86 build host
# and the Arm GPU host.  The generators therefore use only +, -, *, / and
# sqrt, which IEEE 754 rounds the same everywhere.
_LN10 = 2.302585092994046       # ln 10
_LN2 = 0.6931471805599453        # ln 2


def _exp_small(y: np.ndarray) -> np.ndarray:
    """exp(y) for 0 <= y < 2.5, from basic operations only: exp(y / 32) by a
    degree-12 Taylor polynomial (Horner; truncation error below 1e-22
    relative), squared five times."""
    z = np.asarray(y, dtype=np.float64) / 32.0
    p = np.ones_like(z)
    for k in range(12, 0, -1):
        p = 1.0 + p * z / k
    for _ in range(5):
        p = p * p
    return p


def _ln_det(x: float) -> float:
    """ln(x) for x > 0 from basic operations: x = 2^e m with m in [1, 2)
    (exact), ln m = 2 atanh((m - 1)/(m + 1)) by its series (|y| <= 1/3,
    30 terms)."""
    m, e = np.frexp(np.float64(x))  # x = m 2^e, m in [0.5, 1)
    m, e = m * 2.0, e - 1
    y = (m - 1.0) / (m + 1.0)
    y2 = y * y
    acc = 0.0
    for k in range(29, -1, -1):
        acc = 1.0 / (2 * k + 1) + y2 * acc
    return float(e * _LN2 + 2.0 * y * acc)


def exp10_det(x: np.ndarray) -> np.ndarray:
    """10^x for x in [-3, 3], the same bits on every machine: 10^floor(x)
    (a table of the double constants 1e-3 .. 1e3) times exp(frac(x) ln 10)."""
    x = np.asarray(x, dtype=np.float64)
    e = np.floor(x)
    table = np.array([1e-3, 1e-2, 1e-1, 1.0, 1e1, 1e2, 1e3])
    return table[(e + 3).astype(np.int64)] * _exp_small((x - e) * _LN10)


def varcoef3d(m: int, seed: int, log10_range=(-3.0, 3.0), aniso_frac=0.1, aniso_z=0.01) -> Csr:
    """Cell-centred finite-volume diffusion with per-cell coefficient.

    k_c = 10^U(lo, hi) per cell; on a Bernoulli(aniso_frac) subset of cells the
    z-direction coefficient is aniso_z * k_c (anisotropy 1:1:aniso_z).  The face
    coefficient between cells a and b in direction d is the harmonic mean
    2 k_a k_b / (k_a + k_b) of their d-coefficients; a boundary face carries
    2 k_c (Dirichlet value at the face, half a cell away).  Off-diagonals are
    minus the face coefficients, the diagonal is the sum of all six faces.
    """
    n = m ** 3
    idx, i, j, k = _grid3(m)
    lo, hi = log10_range
    if not (-3.0 <= lo <= hi <= 3.0):
        raise ValueError("log10_range must lie within [-3, 3]")
    kc = exp10_det(lo + (hi - lo) * uniform01(seed, STREAM_COEF, n))
    aniso = uniform01(seed, STREAM_ANISO, n) < aniso_frac
    kd = [kc, kc, np.where(aniso, aniso_z * kc, kc)]  # x, y, z coefficients

    def face(d, nb):
        a = kd[d]
        b = kd[d][np.clip(nb, 0, n - 1)]
        return 2.0 * a * b / (a + b)

    # neighbours in ascending column order: z-, y-, x-, diag, x+, y+, z+
    spec = [(2, -m * m, k > 0), (1, -m, j > 0), (0, -1, i > 0),
            None, (0, 1, i < m - 1), (1, m, j < m - 1), (2, m * m, k < m - 1)]
    cols, vals, masks = [], [], []
    diag = np.zeros(n)
    for s in spec:
        if s is None:
            cols.append(idx)
            vals.append(None)
            masks.append(np.ones(n, bool))
            continue
        d, o, inside = s
        nb = idx + o
        f = np.where(inside, face(d, nb), 2.0 * kd[d])
        diag += f
        cols.append(nb)
        vals.append(-f)
        masks.append(inside)
    vals[3] = diag
    return _assemble(n, None, cols, vals, masks)


def convdiff3d(m: int, seed: int, pe_range=(1.0, 100.0)):
    """Upwind convection-diffusion: 7-point diffusion plus first-order upwinding.

    Velocity v is a seeded unit vector (uniform on the sphere, by Marsaglia's
    rejection method: (x1, x2) uniform in the unit disc, v = (2 x1 sqrt(1-s),
    2 x2 sqrt(1-s), 1 - 2 s) with s = x1^2 + x2^2), the cell Peclet
    number Pe ~ U(pe_range).  For each axis d with c_d = Pe*|v_d|, c_d is added
    to the diagonal and -c_d to the coefficient of the upwind neighbour (the one
    at -sign(v_d)); an upwind neighbour outside the grid is eliminated like the
    Dirichlet neighbours.  The result is a nonsymmetric M-matrix.
    Returns (Csr, v, Pe).
    """
    n = m ** 3
    idx, i, j, k = _grid3(m)
    u = uniform01(seed, STREAM_VEL, 64)
    for q in range(0, 62, 2):
        x1, x2 = 2.0 * u[q] - 1.0, 2.0 * u[q + 1] - 1.0
        s2 = x1 * x1 + x2 * x2
        if 0.0 < s2 < 1.0:
            break
    r = 2.0 * np.sqrt(1.0 - s2)
    v = np.array([x1 * r, x2 * r, 1.0 - 2.0 * s2])
    pe = pe_range[0] + (pe_range[1] - pe_range[0]) * u[63]
    c = pe * np.abs(v)
    offs = [-m * m, -m, -1, 0, 1, m, m * m]
    axis = [2, 1, 0, None, 0, 1, 2]
    masks = [k > 0, j > 0, i > 0, np.ones(n, bool), i < m - 1, j < m - 1, k < m - 1]
    cols = [idx + o for o in offs]
    vals = []
    for o, d in zip(offs, axis):
        if d is None:
            vals.append(np.full(n, 6.0 + c.sum()))
            continue
        upwind = (o < 0) == (v[d] > 0)  # o<0 is the minus neighbour
        vals.append(np.full(n, -1.0 - (c[d] if upwind else 0.0)))
    return _assemble(n, offs, cols, vals, masks), v, pe


def uniform_pm1(seed: int, stream: int, count: int) -> np.ndarray:
    """U(-1, 1) doubles: 2u - 1 with 53-bit u."""
    return 2.0 * uniform01(seed, stream, count) - 1.0


def rhs_from_solution(A: Csr, seed: int):
    """Seeded u* ~ U(-1,1) and f = A u* (input construction; returns (f, u*))."""
    ustar = uniform_pm1(seed, STREAM_USTAR, A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    f = np.bincount(rows, weights=A.val * ustar[A.col], minlength=A.n)
    return f, ustar


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    """Up to `count` distinct indices in [0, n), sorted, drawn uniformly from the
    seeded stream (which entries of a large vector a test compares)."""
    u = uniform01(seed, STREAM_SAMPLE, count)
    return np.unique(np.minimum((u * n).astype(np.int64), n - 1))


def batched_sides(count: int, seed: int, lo: int = 16, hi: int = 128):
    """Per-system grid sides n ~ U{lo..hi} and shifts sigma ~ U(0, 0.1)."""
    u = uniform01(seed, STREAM_COEF, count)
    sides = lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)
    sigma = 0.1 * uniform01(seed, STREAM_SHIFT, count)
    return sides, sigma


def serving_sides(count: int, seed: int, lo: int = 20, hi: int = 160):
    """Per-request grid sides, log-uniform on [lo, hi] (so unknowns log-uniform too)."""
    u = uniform01(seed, STREAM_COEF, count)
    span = _ln_det(hi / lo)
    if not (0.0 <= span < 2.5):
        raise ValueError("serving sides need 1 <= hi / lo < 12")
    return np.rint(lo * _exp_small(span * u)).astype(np.int64)


@dataclass
class ServeRequest:
    """One request of a served stream: the key of its matrix, the matrix's
    kind ('poisson' or 'varcoef' with coefficients 10^U(-2,2): SPD, solved by CG; 'convdiff':
    nonsymmetric, solved by BiCGStab), its grid side, whether the key was seen
    before (a new right-hand side for a resident matrix), the seed of its
    right-hand side and its arrival time in seconds."""
    index: int
    key: int
    kind: str
    side: int
    reuse: bool
    arrival: float

    @property
    def solver(self) -> int:
        return 1 if self.kind == "convdiff" else 0

    def matrix(self) -> "Csr":
        if self.kind == "poisson":
            return poisson3d(self.side)
        if self.kind == "varcoef":
            return varcoef3d(self.side, seed=self.key, log10_range=SERVE_VARCOEF_RANGE)
        return convdiff3d(self.side, seed=self.key)[0]

    def rhs(self, seed: int, n: int) -> np.ndarray:
        return uniform_pm1(seed, STREAM_REQ_RHS + self.index, n)


def serving_requests(count: int, seed: int, lo: int = 20, hi: int = 160, rate: float = 0.0,
                     spd_frac: float = 0.7, reuse_frac: float = 0.2):
    """A seeded stream of solve requests.  Each request reuses, with
    probability reuse_frac, the key (and so the matrix) of a uniformly chosen
    earlier request; otherwise it has a new key, a grid side log-uniform on
    [lo, hi], and is SPD with probability spd_frac (half 'poisson', half
    'varcoef') or 'convdiff'.  Arrivals form a Poisson process of the given
    rate (requests per second; 0: all at time 0)."""
    sides = serving_sides(count, seed, lo, hi)
    kind_u = uniform01(seed, STREAM_KIND, count)
    reuse_u = uniform01(seed, STREAM_REUSE, count)
    pick_u = uniform01(seed, STREAM_PICK, count)
    arr_u = uniform01(seed, STREAM_ARRIVAL, count)
    out = []
    t = 0.0
    for i in range(count):
        if rate > 0:
            t += -np.log1p(-arr_u[i]) / rate
        if i > 0 and reuse_u[i] < reuse_frac:
            src = out[min(int(pick_u[i] * i), i - 1)]
            out.append(ServeRequest(i, src.key, src.kind, src.side, True, float(t)))
            continue
        u = kind_u[i]
        kind = ("poisson" if u < spd_frac / 2 else "varcoef") if u < spd_frac else "convdiff"
        out.append(ServeRequest(i, i, kind, int(sides[i]), False, float(t)))
    return out
