"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/psvd.h declares (no compute calls: CPU only)."""
import ctypes
import os
import re
import shutil

import pytest

from paper_2108_08845_gb300 import build, psvd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(psvd_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "psvd_incorporate_data" in names and len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"missing exports: {missing}"


def test_status_strings_without_gpu():
    assert psvd.status_string(psvd.PSVD_ERR_SHAPE) == "unsupported shape"
    assert psvd.status_string(12345) == "unknown status"


def test_new_entry_points_reject_bad_arguments_without_gpu():
    # every check below returns before any CUDA call
    lib = psvd.load()
    C = ctypes
    assert lib.psvd_update_adjoint(None, 0, None, 0, None, None, 0, 1, psvd.PSVD_F32, 1, None, 0,
                                   None, None, 0, None, None, 0, None, None, 0) == \
        psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_autotune(None, None, 0, 1, psvd.PSVD_F32, None) == psvd.PSVD_ERR_INVALID_ARG
    cfg = psvd.psvd_config(1024, 8, 16, 1.0, psvd.PSVD_PREC_FP32, 0, 10, 0, 0, None)
    g = C.c_void_p()
    assert lib.psvd_group_create(None, 4, C.byref(cfg)) == psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_group_create(C.byref(g), 0, C.byref(cfg)) == psvd.PSVD_ERR_INVALID_ARG
    assert g.value is None
    assert lib.psvd_group_initialize(None, None, 1024, 16, psvd.PSVD_F32) == psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_group_incorporate_data(None, None, 1024, 16, psvd.PSVD_F32) == \
        psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_group_member(None, 0) is None
    assert lib.psvd_group_status(None) == psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_group_stats(None, None, None) == psvd.PSVD_ERR_INVALID_ARG
    lib.psvd_group_destroy(None)  # a null group is ignored
    assert psvd.status_string(psvd.PSVD_WARN_DEGENERATE).startswith("warning: coincident")


def test_wait_budget_hook_checks_arguments_without_gpu():
    lib = psvd.load()
    assert lib.psvd_debug_set_wait_budget(2, 100) == psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_debug_set_wait_budget(1, -1) == psvd.PSVD_ERR_INVALID_ARG
    assert lib.psvd_debug_set_wait_budget(1, 0) == psvd.PSVD_OK
