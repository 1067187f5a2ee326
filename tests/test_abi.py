"""The C-ABI library builds for sm_103a, loads, and exports what include/osp.h
declares (no GPU needed: only symbol lookups and pure host calls)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1712_00595_gb300 import build as B
from paper_1712_00595_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "osp.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load_library()


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(osp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_binding_set():
    assert declared() == sorted(N.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (osp_[a-z0-9_]+)$", out, flags=re.M))
    for name in declared():
        assert name in exported, name
        assert getattr(lib, name)


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include "osp.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(osp_update), '
                    'sizeof(osp_batch_stats), sizeof(osp_options), offsetof(osp_batch_stats, ms_update));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    a, b, c, d = map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                         check=True).stdout.split())
    assert a == 12 == N.UPDATE_DTYPE.itemsize
    assert b == C.sizeof(N.osp_batch_stats)
    assert c == C.sizeof(N.osp_options)
    assert d == N.osp_batch_stats.ms_update.offset


def test_host_only_entry_points(lib):
    assert lib.osp_max_batch() == 16384
    assert lib.osp_status_string(-1) == b"OSP_EINVAL"
    assert lib.osp_status_string(0) == b"OSP_OK"
    opt = N.osp_options()
    lib.osp_default_options(C.byref(opt))
    assert opt.precision == N.OSP_PREC_FP32_ACC64 and opt.device == 0
    assert lib.osp_create(None, None) == N.OSP_EINVAL


def test_host_side_argument_checks(lib):
    # rejected before any CUDA call, so they run without a GPU
    assert lib.osp_selftest_wait(0, 7, 0) == N.OSP_EINVAL
    opt = N.osp_options()
    lib.osp_default_options(C.byref(opt))
    assert opt.seed_gather == 0
    opt.seed_gather = 5
    h = C.c_void_p()
    assert lib.osp_create(C.byref(h), C.byref(opt)) == N.OSP_EINVAL
    opt.seed_gather = 0
    opt.precision = 9
    assert lib.osp_create(C.byref(h), C.byref(opt)) == N.OSP_EINVAL
    opt.precision = N.OSP_PREC_FP32_ACC64
    opt.seed_group = 48  # not a multiple of 32 columns
    assert lib.osp_create(C.byref(h), C.byref(opt)) == N.OSP_EINVAL
    assert lib.osp_num_nodes(None) == -1 and lib.osp_device_bytes(None) == -1
