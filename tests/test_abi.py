"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/hull3d.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hull3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hull3d_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1205_1171_gb300 import build

    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1205_1171_gb300 import hull3d

    assert sorted(hull3d.EXPORTS) == _declared()


def test_strerror_without_gpu(lib):
    lib.hull3d_strerror.restype = ctypes.c_char_p
    assert lib.hull3d_strerror(0) == b"ok"
    assert b"duplicate" in lib.hull3d_strerror(3)
    assert lib.hull3d_strerror(12345) == b"unknown error"


def test_plan_rejects_bad_arguments_without_touching_the_gpu(lib):
    plan = ctypes.c_void_p()
    lib.hull3d_plan.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    assert lib.hull3d_plan(ctypes.byref(plan), 0, 0, None) == 1
    assert lib.hull3d_plan(ctypes.byref(plan), (1 << 28) + 1, 0, None) == 1
    assert lib.hull3d_plan(None, 10, 0, None) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1205_1171_gb300 import hull3d

    monkeypatch.setattr(hull3d, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(hull3d, "_lib", None)
    with pytest.raises(RuntimeError):
        hull3d.load()
