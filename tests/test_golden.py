"""CPU checks of the stored oracle results under tests/golden/: the fixture
still describes the inputs the generators build today (so a change to a
generator cannot leave a GPU test comparing against a stale oracle run)."""
import hashlib
import json
import os

import numpy as np

import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_varcoef200_fixture_matches_generator():
    g = json.load(open(os.path.join(GOLDEN, "varcoef200_oracle.json")))
    A = gen.varcoef3d(200, seed=0)
    assert (A.n, A.nnz) == (g["n"], g["nnz"])
    lev0 = g["levels"][0]
    assert (lev0["rows"], lev0["nnz"]) == (A.n, A.nnz)
    h = hashlib.sha256()
    for a in (A.row_ptr.astype(np.int32), A.col.astype(np.int32), A.val.astype(np.float64)):
        h.update(np.ascontiguousarray(a).tobytes())
    assert h.hexdigest() == lev0["A_sha256"]
    assert len(gen.sample_indices(A.n, 8192, 0)) == g["sample"]["count"] == len(g["sample"]["x"])
    # the stored run converged, and its hierarchy obeys the stop rule
    assert g["status"] == 0 and g["relres"] <= 1e-8
    rows = [v["rows"] for v in g["levels"]]
    assert all(b < 0.95 * a for a, b in zip(rows, rows[1:]))
    assert len(rows) == 25 or rows[-1] <= 500
