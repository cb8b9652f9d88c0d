"""CPU oracle for the kinetic divide-and-conquer 3D hull (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never touches it, and it shares no code with that path: the C
source here is compiled on its own with the host compiler.

The algorithm is the one of White & Wortman, Sec. 2 (Chan's minimalist hull
recast as a kinetic 2D lower hull, merged by bridge tracking) with the act()
and time() figures of Sec. 3; degeneracies follow one fixed symbolic
perturbation (see the header of ``hull3d_oracle.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hull3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "invalid argument", 2: "coordinate out of range", 3: "duplicate point",
          4: "capacity", 5: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {ERRORS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no target flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_hull.argtypes = [P, i64, ctypes.c_int, P, i64, P]
            lib.oracle_sort_order.argtypes = [P, i64, P]
            lib.oracle_node_events.argtypes = [P, i64, i64, i64, ctypes.c_int, P, P, P, P, i64, P, P, P]
            lib.oracle_brute_faces.argtypes = [P, i64, P, i64, P]
            lib.oracle_delaunay.argtypes = [P, i64, P, i64, P]
            lib.oracle_turn_sign.argtypes = [P, P]
            lib.oracle_time_cmp.argtypes = [P, P]
            lib.oracle_orient3d_sign.argtypes = [P, P]
            for f in (lib.oracle_hull, lib.oracle_sort_order, lib.oracle_node_events, lib.oracle_brute_faces,
                      lib.oracle_turn_sign, lib.oracle_time_cmp, lib.oracle_orient3d_sign, lib.oracle_delaunay):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _pts(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz), dtype=np.int32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must be an (n, 3) array")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def hull(xyz, split: str = "half") -> np.ndarray:
    """Canonical face list (F x 3 int32) of the hull: outward-CCW triples of
    input indices, rotated min-first, sorted lexicographically."""
    lib = _load()
    a = _pts(xyz)
    n = a.shape[0]
    cap = max(2 * n - 4, 2)
    faces = np.zeros((cap, 3), dtype=np.int32)
    nf = ctypes.c_int64(0)
    rc = lib.oracle_hull(_ptr(a), n, 1 if split == "aligned" else 0, _ptr(faces), cap, ctypes.byref(nf))
    if rc:
        raise OracleError(rc, "hull")
    return faces[: nf.value].copy()


def delaunay(xy) -> np.ndarray:
    """Canonical triangle list (T x 3 int32) of the 2D Delaunay triangulation
    of the (n, 2) int32 points (|x|, |y| < 2^15) through the lifting map: the
    lower hull of (x, y, x^2 + y^2) by the method's lower pass, triangles
    counter-clockwise in the plane, rotated min-first, sorted."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(xy), dtype=np.int32)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("points must be an (n, 2) array")
    n = a.shape[0]
    cap = max(2 * n, 2)
    tris = np.zeros((cap, 3), dtype=np.int32)
    nt = ctypes.c_int64(0)
    rc = lib.oracle_delaunay(_ptr(a), n, _ptr(tris), cap, ctypes.byref(nt))
    if rc:
        raise OracleError(rc, "delaunay")
    return tris[: nt.value].copy()


def sort_order(xyz) -> np.ndarray:
    """Input index of each rank in the perturbed x-order (x, then z, then y)."""
    lib = _load()
    a = _pts(xyz)
    out = np.zeros(a.shape[0], dtype=np.int32)
    rc = lib.oracle_sort_order(_ptr(a), a.shape[0], _ptr(out))
    if rc:
        raise OracleError(rc, "sort")
    return out


def node_events(xyz, lo: int, hi: int, upper: bool = False):
    """Movie of the node holding sorted ranks [lo, hi) for one pass.

    Returns (w, a, b, ins, neg_hull): event points, their left/right
    neighbours at the event (ranks), insertion flags, and the node's
    t = -infinity hull as ranks."""
    lib = _load()
    a = _pts(xyz)
    m = hi - lo
    cap = max(2 * m, 1)
    w = np.zeros(cap, np.int32)
    aa = np.zeros(cap, np.int32)
    bb = np.zeros(cap, np.int32)
    ins = np.zeros(cap, np.int8)
    neg = np.zeros(m + 1, np.int32)
    nev = ctypes.c_int64(0)
    nneg = ctypes.c_int64(0)
    rc = lib.oracle_node_events(_ptr(a), a.shape[0], lo, hi, int(upper), _ptr(w), _ptr(aa), _ptr(bb), _ptr(ins),
                                cap, ctypes.byref(nev), _ptr(neg), ctypes.byref(nneg))
    if rc:
        raise OracleError(rc, "node events")
    k = nev.value
    return w[:k].copy(), aa[:k].copy(), bb[:k].copy(), ins[:k].astype(bool), neg[: nneg.value].copy()


def brute_faces(xyz) -> np.ndarray:
    """Perturbed O(n^4) brute-force face list (canonical), for tiny n."""
    lib = _load()
    a = _pts(xyz)
    n = a.shape[0]
    cap = max(n * (n - 1) * (n - 2) // 6 * 2, 2)
    faces = np.zeros((cap, 3), dtype=np.int32)
    nf = ctypes.c_int64(0)
    rc = lib.oracle_brute_faces(_ptr(a), n, _ptr(faces), cap, ctypes.byref(nf))
    if rc:
        raise OracleError(rc, "brute force")
    return faces[: nf.value].copy()


def turn_sign(pts, ids) -> int:
    lib = _load()
    return lib.oracle_turn_sign(_ptr(_pts(pts)), _ptr(np.ascontiguousarray(ids, dtype=np.int32)))


def time_cmp(pts, ids) -> int:
    """sign(t(T1) - t(T2)) for T1 = pts[0:3], T2 = pts[3:6] (perturbed times)."""
    lib = _load()
    return lib.oracle_time_cmp(_ptr(_pts(pts)), _ptr(np.ascontiguousarray(ids, dtype=np.int32)))


def orient3d_sign(pts, ids) -> int:
    lib = _load()
    return lib.oracle_orient3d_sign(_ptr(_pts(pts)), _ptr(np.ascontiguousarray(ids, dtype=np.int32)))
