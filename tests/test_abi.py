"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/qst.h declares (no compute calls here)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "qst.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qst_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["qst_plan_create", "qst_plan_destroy", "qst_forward", "qst_adjoint", "qst_evaluate_host",
                 "qst_plan_status", "qst_params_default", "qst_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2607_19577_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(str(lib_path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points_without_gpu():
    """Entry points that touch no device: defaults and status strings."""
    from paper_2607_19577_b300 import qst
    lib = qst.load()
    prm = qst._Params()
    lib.qst_params_default(ctypes.byref(prm))
    assert prm.eps == 1e-8 and prm.validate == 1 and prm.norm_settings == 0
    assert lib.qst_status_string(0) == b"ok"
    assert lib.qst_status_string(5) == b"device-side error"


def test_plan_create_rejects_bad_shapes_before_touching_the_device():
    from paper_2607_19577_b300 import qst
    lib = qst.load()
    h = ctypes.c_void_p()
    for n, M, K, nnz in [(0, 4, 2, 0), (4, 0, 2, 0), (4, 4, 0, 0), (4, 4, 2, -1), (3, 2, 1, 17)]:
        assert lib.qst_plan_create(ctypes.byref(h), n, M, K, nnz, None) == 1  # QST_ERR_INVALID_ARG
    # n = 21 is beyond this build's largest shape
    assert lib.qst_plan_create(ctypes.byref(h), 21, 4, 2, 0, None) == 2
