"""CPU checks of the C-ABI boundary: the library loads, exports every entry
point declared in include/amg.h, and its structs have the layout the Python
binding assumes.  No GPU work is launched."""
import ctypes
import os
import re
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amg.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:amg_status|const char \*)\s*(amg_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("_b", os.path.join(ROOT, "paper_1811_05704_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1811_05704_gb300 as amg
    return amg


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), f"{n} declared in amg.h but not exported"
    assert sorted(lib.EXPORTED) == names


def test_struct_layout_matches_header(lib):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "amg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(amg_params), sizeof(amg_csr),
         offsetof(amg_params, use_graph), offsetof(amg_csr, on_device), offsetof(amg_params, jacobi_omega),
         sizeof(amg_server_params), offsetof(amg_server_params, hbm_budget));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = list(map(int, out))
    assert got == [ctypes.sizeof(lib.amg_params), ctypes.sizeof(lib.amg_csr),
                   lib.amg_params.use_graph.offset, lib.amg_csr.on_device.offset,
                   lib.amg_params.jacobi_omega.offset, ctypes.sizeof(lib.amg_server_params),
                   lib.amg_server_params.hbm_budget.offset]


def test_params_default(lib):
    p = lib.amg_params_default()
    assert (p.strength_eps, p.strength_halving, p.smoother, p.jacobi_omega) == (0.08, 1, 0, 0.72)
    assert (p.npre, p.npost, p.coarse_enough, p.max_levels) == (1, 1, 500, 25)
    assert (p.max_coarse_dense, p.solver, p.precision, p.use_graph) == (4096, 0, 0, 1)
    assert (p.use_stream, p.use_pdl, p.use_tail, p.device_setup, p.fused_restriction) == (1, 0, 0, 1, 1)
    assert lib._lib.amg_params_default(None) == lib.AMG_ERR_INVALID_ARG


def test_null_arguments_are_rejected_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib._lib.amg_setup(None, None, None, ctypes.byref(h)) == lib.AMG_ERR_INVALID_ARG
    assert "null" in lib.amg_last_error()
    assert lib._lib.amg_solve(None, None, None, 1e-8, 10, None, None) == lib.AMG_ERR_INVALID_ARG
    assert lib._lib.amg_free(None) == lib.AMG_OK
    rid = ctypes.c_int64()
    f = (ctypes.c_double * 4)()
    assert lib._lib.amg_server_create(None, None, None) == lib.AMG_ERR_INVALID_ARG
    assert lib._lib.amg_server_submit(None, 0, None, f, 4, None, 1e-8, 10, ctypes.byref(rid)) == lib.AMG_ERR_INVALID_ARG
    assert lib._lib.amg_server_wait(None, 1, None, None, None, None, None) == lib.AMG_ERR_INVALID_ARG
    assert lib._lib.amg_server_stats(None, None, None, None, None, None) == lib.AMG_ERR_INVALID_ARG
    assert lib._lib.amg_server_destroy(None) == lib.AMG_OK
    # parameter checks run before any device work
    import numpy as np
    ptr, col, val = np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0])
    csr = lib.make_csr(1, ptr, col, val)
    for bad in (dict(precision=3), dict(precision=2, npre=2), dict(solver=7), dict(max_levels=0)):
        assert lib._lib.amg_setup(ctypes.byref(csr), ctypes.byref(lib.amg_params_default(**bad)), None,
                                  ctypes.byref(h)) == lib.AMG_ERR_INVALID_ARG, bad
    arr = (lib.amg_csr * 1)(csr)
    assert lib._lib.amg_batch_setup(1, ctypes.cast(arr, ctypes.c_void_p),
                                    ctypes.byref(lib.amg_params_default(precision=2)), None,
                                    ctypes.byref(h)) == lib.AMG_ERR_INVALID_ARG
    assert "FP64 and FP32" in lib.amg_last_error()


def test_package_fails_loudly_without_library(lib, tmp_path):
    pkg = tmp_path / "paper_1811_05704_gb300"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1811_05704_gb300", "__init__.py"), pkg / "__init__.py")
    code = "import paper_1811_05704_gb300"
    r = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0 and "ImportError" in r.stderr and "not built" in r.stderr


def test_library_does_not_reference_the_oracle():
    csrc = os.path.join(ROOT, "paper_1811_05704_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f"{f} mentions the oracle"
