"""The C ABI library builds for sm_103a, loads, and exports every function
include/fastmap.h declares; the ctypes structs match the C layout (no GPU)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2505_04612_b300 import build as B
from paper_2505_04612_b300 import fastmap as F

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fastmap.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:fm_status|void|const char\s*\*)\s*(fm_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["fm_problem_create", "fm_problem_destroy", "fm_loss_grad", "fm_step", "fm_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fm_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
    # the binding wraps exactly the declared calls
    assert sorted(F._SIGNATURES) == declared_functions()


def test_struct_layout_matches_c():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "fastmap.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fm_problem_desc),
         offsetof(fm_problem_desc, inputs_on_device), offsetof(fm_problem_desc, cuda_stream),
         sizeof(fm_problem_info), sizeof(fm_adam_opts), sizeof(fm_solve_opts), offsetof(fm_solve_opts, eps),
         sizeof(fm_result), offsetof(fm_result, n_kept), sizeof(fm_kernel_time),
         offsetof(fm_problem_desc, scene_cam_off), offsetof(fm_problem_info, n_scenes),
         offsetof(fm_result, cam_valid), offsetof(fm_problem_info, n_cams_connected));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(F.fm_problem_desc), F.fm_problem_desc.inputs_on_device.offset,
                    F.fm_problem_desc.cuda_stream.offset, ctypes.sizeof(F.fm_problem_info),
                    ctypes.sizeof(F.fm_adam_opts), ctypes.sizeof(F.fm_solve_opts), F.fm_solve_opts.eps.offset,
                    ctypes.sizeof(F.fm_result), F.fm_result.n_kept.offset, ctypes.sizeof(F.fm_kernel_time),
                    F.fm_problem_desc.scene_cam_off.offset, F.fm_problem_info.n_scenes.offset,
                    F.fm_result.cam_valid.offset, F.fm_problem_info.n_cams_connected.offset]


def test_errors_without_problem_are_reported(lib):
    # argument validation happens before any device work
    d = F.fm_problem_desc()
    d.n_cams = 1
    h = ctypes.c_void_p()
    st = lib.fm_problem_create(ctypes.byref(d), ctypes.byref(h))
    assert st == F.FM_ERR_INVALID_ARG and h.value is None
    assert "n_cams" in F.fm_last_error(None)
    assert lib.fm_problem_create(None, ctypes.byref(h)) == F.FM_ERR_INVALID_ARG
    assert lib.fm_loss_grad(None, 0, None, None, None, 0) == F.FM_ERR_INVALID_ARG
    lib.fm_problem_destroy(None)   # no-op
