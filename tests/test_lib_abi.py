"""The C-ABI library builds for sm_103a, loads and exports every symbol include/md.h
declares (no compute call: this runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "md.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libmd():
    from paper_1507_07068_gb300 import build_lib
    try:
        build_lib.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    path = build_lib.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("md_init", "md_build_neighbors", "md_compute_forces", "md_step", "md_get_energy",
                     "md_get_forces", "md_get_indenter_load", "md_free", "md_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(libmd):
    for name in declared_functions():
        assert hasattr(libmd, name), name


def test_binding_covers_the_header():
    from paper_1507_07068_gb300 import md
    for name in declared_functions():
        assert hasattr(md, name), name
        assert name in md.EXPORTS


def test_version_and_error_without_gpu(libmd):
    libmd.md_version.restype = C.c_int
    assert libmd.md_version() == 7
    libmd.md_last_error.restype = C.c_char_p
    libmd.md_last_error.argtypes = [C.c_void_p]
    assert libmd.md_last_error(None) is not None


def test_bad_arguments_rejected_before_any_device_work(libmd):
    from paper_1507_07068_gb300 import md
    md._lib = None
    L = md.lib()
    h = C.c_void_p()
    opt = md.md_options()
    assert L.md_init(None, 1, C.byref(opt), None, C.byref(h)) == md.MD_ERR_ARG
    assert not h.value
    sysarr = (md.md_system * 1)()
    assert L.md_init(sysarr, 0, C.byref(opt), None, C.byref(h)) == md.MD_ERR_ARG
    p = md.make_params(md.load_params())
    opt.pot = C.pointer(p)
    opt.precision = 7
    assert L.md_init(sysarr, 1, C.byref(opt), None, C.byref(h)) == md.MD_ERR_ARG
    assert b"precision" in L.md_last_error(None)
    opt.precision = md.MD_MIXED
    opt.tpa = 3
    assert L.md_init(sysarr, 1, C.byref(opt), None, C.byref(h)) == md.MD_ERR_ARG
    opt.tpa = 0
    # an empty replica (no film atoms) is rejected, not run
    assert L.md_init(sysarr, 1, C.byref(opt), None, C.byref(h)) == md.MD_ERR_ARG
    assert b"n_cr >= 1" in L.md_last_error(None) and not h.value
    md.md_free(None)


def test_struct_layouts_match_header_sizes():
    """The ctypes mirrors of the C structs have the sizes a C compiler gives them."""
    import subprocess
    import tempfile
    from paper_1507_07068_gb300 import md
    prog = r'''
#include <stdio.h>
#include "md.h"
int main(void){printf("%zu %zu %zu %zu %zu\n", sizeof(md_params), sizeof(md_system), sizeof(md_options),
 sizeof(md_energy), sizeof(md_phase_times)); return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(t) for t in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert sizes == [C.sizeof(md.md_params), C.sizeof(md.md_system), C.sizeof(md.md_options),
                     C.sizeof(md.md_energy), C.sizeof(md.md_phase_times)]
