"""Write tests/golden/varcoef200_oracle.json from the FP64 CPU oracle alone.

The 200^3 variable-coefficient workload (8,000,000 unknowns, 55,760,000
nonzeros; cell coefficients 10^U(-3,3), 10% of the cells with z-anisotropy
0.01, harmonic-mean faces; generator seed 0, f = A u* with u* seed 0, x0 = 0)
is too large for the oracle to solve inside a GPU test (its single-threaded
setup alone takes minutes), so this script runs it once and stores what the
GPU test compares against:

  - the hierarchy of Algorithm 1: rows and nonzeros of every level, and a
    SHA-256 of every level's matrix A_l (row pointers as int32, columns,
    float64 values) and of every level's aggregates, so that the GPU
    hierarchy can be checked bit for bit at full size;
  - the CG solve (Algorithm 2 as the preconditioner, rtol 1e-8): iterations,
    true relative residual, ||x||_2 and ||x||_inf;
  - x at 8192 seeded sample indices (gen.sample_indices(n, 8192, 0)), as
    exact hexadecimal floats.

Only gen/ (input construction) and oracle/ are used; nothing here touches the
CUDA library.  Run from the repository root:

    python tests/golden/make_varcoef200.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "varcoef200_oracle.json")
SIDE, SEED, NSAMPLE = 200, 0, 8192


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def main():
    t0 = time.time()
    A = gen.varcoef3d(SIDE, seed=SEED)
    f, _ = gen.rhs_from_solution(A, SEED)
    H = oracle.Hierarchy(A)
    setup_s = time.time() - t0
    levels = []
    for l in range(H.levels):
        info = H.level_info(l)
        ptr, col, val, _ = H.matrix(l, "A")
        lev = {"rows": info["n"], "nnz": info["nnz"],
               "A_sha256": sha(ptr.astype(np.int32), col, val)}
        if l < H.levels - 1:
            lev["aggregates_sha256"] = sha(H.aggregates(l).astype(np.int32))
            lev["nnz_p"] = info["nnz_p"]
        levels.append(lev)
    t1 = time.time()
    x, it, rr, st = H.cg(f, rtol=1e-8, maxiter=500)
    solve_s = time.time() - t1
    idx = gen.sample_indices(A.n, NSAMPLE, SEED)
    out = {
        "what": "FP64 oracle (oracle/amg_oracle.c) on the 200^3 variable-coefficient workload: "
                "Algorithm 1 hierarchy and the CG solve preconditioned by one V-cycle (Algorithm 2)",
        "workload": {"generator": "gen.varcoef3d(200, seed=0)", "rhs": "gen.rhs_from_solution(A, 0)",
                     "x0": 0, "rtol": 1e-8, "params": "oracle defaults (eps 0.08 halved per level, "
                     "Jacobi 0.72, 1/1 sweeps, coarse <= 500 rows, 25 levels at most)"},
        "written_by": "tests/golden/make_varcoef200.py",
        "n": int(A.n), "nnz": int(A.nnz),
        "levels": levels,
        "operator_complexity": sum(v["nnz"] for v in levels) / A.nnz,
        "status": int(st), "iterations": int(it), "relres": float(rr),
        "x_norm2": float(np.linalg.norm(x)), "x_norm_inf": float(np.abs(x).max()),
        "sample": {"indices": "gen.sample_indices(n, 8192, 0)", "count": int(len(idx)),
                   "x": [float(v).hex() for v in x[idx]]},
        "oracle_seconds": {"setup": round(setup_s, 1), "solve": round(solve_s, 1)},
    }
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(f"wrote {OUT}: {H.levels} levels, {it} iterations, relres {rr:.2e}, "
          f"setup {setup_s:.0f} s, solve {solve_s:.0f} s")


if __name__ == "__main__":
    main()
