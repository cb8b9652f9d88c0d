"""The device merge header (merge.cuh with predicates.cuh), compiled for the
host, against the oracle on the CPU: the merge loop the batch kernel and the
serial fallback run (form 0), the loop of the thread-per-merge level kernel
with its shared-memory candidate slice (form 1), and the compacted slot-table
form of the warp-per-merge kernel, driven level by level like the device
(tests/host/merge_header_check.cpp).
Faces must be identical on degenerate tiny sets, on sets crowded onto a few
x-values (every comparison through the equal-x tiers), and on seeded clouds of
every distribution.  This catches a regression in the merge or predicate
logic without a GPU; the GPU tests check the kernels themselves."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1205_1171_gb300 import inputs
from tests.test_oracle_hull import _tiny_sets

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    oracle.build()
    so = tmp_path_factory.mktemp("mhc") / "libmerge_header_check.so"
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", os.path.join(HERE, "host", "merge_header_check.cpp"),
                    "-o", str(so)], check=True, capture_output=True, text=True)
    return ctypes.CDLL(str(so))


def _hull(lib, pts, cmp_level, form=1):
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    n = len(pts)
    faces = np.zeros((max(2 * n, 2), 3), np.int32)
    nf = ctypes.c_int64(0)
    rc = lib.merge_header_hull(pts.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(n), ctypes.c_int(form),
                               ctypes.c_int(cmp_level), faces.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nf))
    assert rc == 0, rc
    return faces[: nf.value]


@pytest.mark.parametrize("form,cmp_level", [(0, 0), (1, 0), (1, 3)])
def test_tiny_degenerate_sets(lib, form, cmp_level):
    for pts in _tiny_sets(1500, 41):
        assert np.array_equal(_hull(lib, pts, cmp_level, form), oracle.hull(pts)), pts.tolist()


@pytest.mark.parametrize("form,cmp_level", [(0, 0), (1, 0), (1, 4)])
def test_sets_on_few_x_values(lib, form, cmp_level):
    rng = np.random.default_rng(5)
    for trial in range(40):
        n = int(rng.integers(8, 2500))
        xr = int(rng.integers(1, 40))
        yz = int(rng.choice([3, 50, 1 << 20]))
        p = np.stack([rng.integers(0, xr, n), rng.integers(-yz, yz, n), rng.integers(-yz, yz, n)], 1)
        p = np.unique(p, axis=0)
        p = p[rng.permutation(len(p))].astype(np.int32)
        if len(p) < 4:
            continue
        assert np.array_equal(_hull(lib, p, cmp_level, form), oracle.hull(p)), (trial, len(p), xr, yz)


@pytest.mark.parametrize("dist", inputs.DISTS)
def test_seeded_clouds(lib, dist):
    for n in (5, 17, 100, 1000, 4097, 20000):
        pts = inputs.cloud_seeded(dist, n, 300 + n)
        want = oracle.hull(pts)
        assert np.array_equal(_hull(lib, pts, 0, 0), want), (dist, n)
        assert np.array_equal(_hull(lib, pts, 0, 1), want), (dist, n)
        assert np.array_equal(_hull(lib, pts, 6, 1), want), (dist, n)
