"""The C-ABI library loads on a machine without a GPU and exports every
function include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mdhp_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("mdhp_loglik_grad", "mdhp_fit_batch", "mdhp_plan_create", "mdhp_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2411_10258_gb300 import build, _lib

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the ctypes layer declares exactly the header's functions
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == declared_functions()


def test_struct_layouts_match_header():
    from paper_2411_10258_gb300 import _lib

    # mdhp_batch: 2 int32, int64, 5 pointers, 2 int32 -> 64 bytes on LP64
    assert ctypes.sizeof(_lib.MdhpBatch) == 64
    # mdhp_fit_opts: 4 int32, 7 float, int32, double -> 56 bytes
    assert ctypes.sizeof(_lib.MdhpFitOpts) == 56


def test_missing_library_fails_loudly(tmp_path):
    from paper_2411_10258_gb300 import _lib

    with pytest.raises(RuntimeError):
        _lib.load(str(tmp_path / "nope.so"))


def test_plan_setters_reject_bad_arguments_without_a_gpu():
    """The plan's tuning setters check their arguments on the host before any
    CUDA call: a NULL plan and out-of-range values return MDHP_E_ARG with a
    message, and the getters report -1 for a NULL plan."""
    from paper_2411_10258_gb300 import build, _lib

    lib = _lib.load(build.build())
    null = ctypes.c_void_p(None)
    assert lib.mdhp_plan_set_feature_store(null, 1) == _lib.E_ARG
    assert b"NULL" in lib.mdhp_last_error()
    assert lib.mdhp_plan_get_feature_store(null) == -1
    assert lib.mdhp_plan_set_pipeline(null, 2, 2) == _lib.E_ARG
    assert lib.mdhp_plan_set_split(null, 1, 256, 1) == _lib.E_ARG
    assert lib.mdhp_plan_set_wait_limit(null, 0) == _lib.E_ARG
    assert lib.mdhp_plan_last_launches(null) == -1
