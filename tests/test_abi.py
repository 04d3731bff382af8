"""CPU checks of the boundary: the CUDA library loads without a GPU, exports every entry point
that include/otm.h declares, and the Python structs match the C layout of the header."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_08772_gb300 import build
    if not build.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        build.build()
    import paper_2206_08772_gb300 as g
    return g.load()


def test_exports_every_declared_symbol(lib):
    import paper_2206_08772_gb300 as g
    names = g.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header(tmp_path):
    from paper_2206_08772_gb300 import _lib
    src = tmp_path / "probe.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "otm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(otm_params), sizeof(otm_material), sizeof(otm_problem),
         offsetof(otm_params, max_support), offsetof(otm_params, mat), offsetof(otm_params, wall_p),
         offsetof(otm_material, d5));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(v) for v in out]
    want = [C.sizeof(_lib.Params), C.sizeof(_lib.Material), C.sizeof(_lib.Problem),
            _lib.Params.max_support.offset, _lib.Params.mat.offset, _lib.Params.wall_p.offset,
            _lib.Material.d5.offset]
    assert got == want


def test_argument_errors_need_no_gpu(lib):
    """Entry points validate sizes before touching the device."""
    from paper_2206_08772_gb300 import _lib
    P = _lib.Params()
    nb = C.c_size_t(0)
    assert lib.otm_workspace_bytes(10, 10, C.byref(P), C.byref(nb)) == _lib.ERR_ARG
    P.h, P.beta, P.rs2, P.cell_size, P.dt = 1e-3, 0.8e6, 1.7e-5, 2.1e-3, 1e-8
    P.n_materials, P.max_support, P.max_newton = 1, 384, 50
    assert lib.otm_workspace_bytes(100, 300, C.byref(P), C.byref(nb)) == _lib.OK
    assert nb.value > 300 * 384 * 32
    P.max_support = 100         # not a multiple of 32
    assert lib.otm_workspace_bytes(100, 300, C.byref(P), C.byref(nb)) == _lib.ERR_ARG
