"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every entry point include/raywave.h declares, and the ctypes
structures have the C layout."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "raywave.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_15418_gb300 import build, _capi
    build.build()
    return _capi.load()


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("rw_create", "rw_destroy", "rw_generate_rays", "rw_doe_emit", "rw_forward",
              "rw_loss_eq3", "rw_backward", "rw_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_2605_15418_gb300 import _capi
    assert set(_capi.EXPORTS) == set(declared_functions())


def test_ctypes_layout_matches_header(tmp_path):
    from paper_2605_15418_gb300 import _capi as A
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "raywave.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu",'
                   'sizeof(rw_surface),sizeof(rw_doe),sizeof(rw_sensor),sizeof(rw_system),'
                   'sizeof(rw_job),sizeof(rw_rays),sizeof(rw_emitted),'
                   'offsetof(rw_system,doe),offsetof(rw_system,sensor));}')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    ref = [C.sizeof(A.rw_surface), C.sizeof(A.rw_doe), C.sizeof(A.rw_sensor),
           C.sizeof(A.rw_system), C.sizeof(A.rw_job), C.sizeof(A.rw_rays),
           C.sizeof(A.rw_emitted), A.rw_system.doe.offset, A.rw_system.sensor.offset]
    assert got == ref


def test_version_and_null_context_without_gpu(lib):
    assert b"sm_103a" in lib.rw_version()
    assert lib.rw_destroy(None) == 1          # RW_EINVAL
    assert lib.rw_forward(None, None, None, 0, None, None) == 1
    out = C.c_void_p()
    # no device here: creation is refused with RW_EINVAL, nothing crashes
    import torch
    if not torch.cuda.is_available():
        assert lib.rw_create(C.byref(out), 0, None) == 1
