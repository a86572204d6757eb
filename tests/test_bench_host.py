"""Host logic of bench.py that needs no GPU: the check that decides whether
the committed ncu counters still describe the kernels (the `traffic` of the
bench line), and the algorithmic byte model of the 150^3 iteration."""
import os
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _with_source(tmp_path, text):
    """A copy of the repository layout bench.py reads, with spmv.cu replaced."""
    d = tmp_path / "paper_1811_05704_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "spmv.cu").write_text(text)
    shutil.copytree(os.path.join(ROOT, "profiles"), tmp_path / "profiles")
    return str(tmp_path)


def test_code_digest_ignores_comments_only(tmp_path, monkeypatch):
    src = open(os.path.join(ROOT, "paper_1811_05704_gb300", "csrc", "spmv.cu")).read()
    base = bench.spmv_code_digest()
    # comment edits and blank lines keep the digest ...
    monkeypatch.setattr(bench, "ROOT", _with_source(tmp_path / "a", "// note\n\n" + src.replace(
        "namespace amg {", "namespace amg {  // the library's namespace", 1)))
    assert bench.spmv_code_digest() == base
    # ... a code edit changes it, and the committed counters are then not used
    monkeypatch.setattr(bench, "ROOT", _with_source(tmp_path / "b", src.replace(
        "constexpr int kGatherBatch = 4;", "constexpr int kGatherBatch = 8;", 1)))
    assert bench.spmv_code_digest() != base
    assert bench.committed_traffic("restrict_l0") is None


def test_committed_counters_match_the_current_kernels():
    """The dominant kernel's ncu summary was captured from the current code."""
    t = bench.committed_traffic("restrict_l0")
    assert t is not None and 3.5e8 < t < 4.5e8


def test_iteration_bytes_of_the_150_cube_hierarchy():
    """The byte model on the 150^3 hierarchy's sizes (levels, rows, nonzeros
    of A, P and the fused restriction operators, as the set-up reports them:
    M keeps the pattern of R A, exact cancellations included) reproduces the
    count the library gave on the GPU (1,934,160,756 bytes)."""
    info = {"levels": 5, "rows": [3375000, 401950, 24749, 1382, 107],
            "nnz": [23490000, 12675914, 1775911, 92474, 4209],
            "nnz_p": [12172814, 1787969, 103597, 5292, 0],
            "nnz_m": [29925203, 7870655, 597649, 27677, 0]}
    assert bench.bytes_per_iteration(info, 107) == 1934160756
