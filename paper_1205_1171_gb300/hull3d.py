"""Thin ctypes binding of the C ABI in include/hull3d.h.

Argument marshalling only: every step of the hull runs in the CUDA library.
PyTorch provides device memory and streams.  If the shared library has not
been built this module raises on first use -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhull3d.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = 1
ERR_COORD_RANGE = 2
ERR_DUPLICATE = 3
ERR_CAPACITY = 4
ERR_OOM = 5
ERR_BUDGET = 6
ERR_DEVICE_TIMEOUT = 7
ERR_CUDA = 8
ERR_INTERNAL = 9
ERR_TOO_LARGE = 10
ERR_NOT_CLOSED = 11
STATIC_MAX_N = 16384

# every symbol include/hull3d.h declares
EXPORTS = (
    "hull3d_plan", "hull3d_plan_opts", "hull3d_destroy", "hull3d_plan_bytes", "hull3d_compute_async", "hull3d_compute",
    "hull3d_compute_host", "hull3d_batch_async", "hull3d_strerror", "hull3d_last_cuda_error",
    "hull3d_last_launch_count", "hull3d_compute_static", "hull3d_profile", "hull3d_profile_read", "hull3d_profile_levels",
    "hull3d_level_events", "hull3d_adjacency_async", "hull3d_delaunay_async", "hull3d_window_stats",
)
WINDOW_STATS = ("pair_overflow", "merges", "windows", "retried", "global_tables", "serial", "refit")
PHASES = ("sort", "fused", "levels", "seg", "faces")


class Hull3DError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        lib = load()
        msg = lib.hull3d_strerror(code).decode()
        if code == ERR_CUDA:
            msg += f" (cudaError {lib.hull3d_last_cuda_error()})"
        super().__init__(f"hull3d{(' ' + what) if what else ''}: {msg}")
        self.code = code


OPT_NAMES = ("fused_levels", "seg_level", "seg_events", "use_graph", "level_occupancy", "cmp_level", "cmp_slots",
             "seg_slots", "seg_min_events", "merge_order", "seg_events_min", "batch_warp_nodes", "multi_ranks",
             "float32_ablation", "seg_slots_big", "filter_level")


class Opts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in OPT_NAMES]


def load():
    """Loads the library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH)
            P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.hull3d_plan.argtypes = [ctypes.POINTER(P), i64, i64, ctypes.POINTER(Opts)]
            lib.hull3d_plan.restype = ctypes.c_int
            lib.hull3d_plan_opts.argtypes = [P, ctypes.POINTER(Opts)]
            lib.hull3d_plan_opts.restype = ctypes.c_int
            lib.hull3d_destroy.argtypes = [P]
            lib.hull3d_destroy.restype = None
            lib.hull3d_plan_bytes.argtypes = [P]
            lib.hull3d_plan_bytes.restype = i64
            lib.hull3d_compute_async.argtypes = [P, P, i64, P, i64, P, P, P]
            lib.hull3d_compute_async.restype = ctypes.c_int
            lib.hull3d_compute.argtypes = [P, P, i64, P, i64, ctypes.POINTER(i64), P]
            lib.hull3d_compute.restype = ctypes.c_int
            lib.hull3d_compute_host.argtypes = [P, P, i64, P, i64, ctypes.POINTER(i64), P]
            lib.hull3d_compute_host.restype = ctypes.c_int
            lib.hull3d_batch_async.argtypes = [P, P, P, i64, P, P, P, P, P]
            lib.hull3d_batch_async.restype = ctypes.c_int
            lib.hull3d_delaunay_async.argtypes = [P, P, i64, P, i64, P, P, P]
            lib.hull3d_delaunay_async.restype = ctypes.c_int
            lib.hull3d_adjacency_async.argtypes = [P, P, P, i64, i64, P, P, P, P, P]
            lib.hull3d_adjacency_async.restype = ctypes.c_int
            lib.hull3d_compute_static.argtypes = [P, i64, P, i64, P, P, P]
            lib.hull3d_compute_static.restype = ctypes.c_int
            lib.hull3d_strerror.argtypes = [ctypes.c_int]
            lib.hull3d_strerror.restype = ctypes.c_char_p
            lib.hull3d_last_cuda_error.argtypes = []
            lib.hull3d_last_cuda_error.restype = ctypes.c_int
            lib.hull3d_last_launch_count.argtypes = [P]
            lib.hull3d_last_launch_count.restype = i64
            lib.hull3d_profile.argtypes = [P, ctypes.c_int]
            lib.hull3d_profile.restype = ctypes.c_int
            lib.hull3d_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
            lib.hull3d_profile_read.restype = ctypes.c_int
            lib.hull3d_profile_levels.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
            lib.hull3d_profile_levels.restype = ctypes.c_int
            lib.hull3d_level_events.argtypes = [P, ctypes.POINTER(i64)]
            lib.hull3d_level_events.restype = ctypes.c_int
            lib.hull3d_window_stats.argtypes = [P, ctypes.POINTER(i64)]
            lib.hull3d_window_stats.restype = ctypes.c_int
            _lib = lib
    return _lib


def _stream_ptr(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check_points(xyz, device_needed: bool):
    import torch

    if not isinstance(xyz, torch.Tensor):
        raise TypeError("points must be a torch tensor")
    if xyz.dtype != torch.int32 or xyz.dim() != 2 or xyz.shape[1] != 3:
        raise ValueError("points must be an (n, 3) int32 tensor")
    if device_needed and not xyz.is_cuda:
        raise ValueError("points must be on a CUDA device")
    return xyz.contiguous()


def max_faces(n: int) -> int:
    return max(2 * n - 4, 0) if n >= 3 else 0


class Hull3D:
    """A plan: scratch for hulls of up to max_n points (and batches totalling max_n)."""

    def __init__(self, max_n: int, max_clouds: int = 0, **knobs):
        """knobs: any of OPT_NAMES (0 = automatic)."""
        self._lib = load()
        bad = set(knobs) - set(OPT_NAMES)
        if bad:
            raise TypeError(f"unknown options {sorted(bad)}")
        opts = Opts(*[int(knobs.get(k, 0)) for k in OPT_NAMES])
        plan = ctypes.c_void_p()
        rc = self._lib.hull3d_plan(ctypes.byref(plan), int(max_n), int(max_clouds), ctypes.byref(opts))
        if rc:
            raise Hull3DError(rc, "plan")
        self._plan = plan
        self.max_n = int(max_n)

    @classmethod
    def tuned(cls, max_n: int, max_clouds: int = 0, cache: str | None = None, dist_class: str | None = None,
              kind: str = "single", **overrides):
        """A plan with the knobs the autotuner stored for this GPU, size,
        distribution class ("volume" or "surface") and kind of work ("single"
        hulls, "batch" of small clouds, "multi": groups of large clouds); the
        library defaults where nothing was tuned.  Explicit overrides win."""
        import torch

        from paper_1205_1171_gb300 import autotune

        knobs = autotune.lookup(torch.cuda.get_device_name(), max_n, cache or autotune.DEFAULT_CACHE, dist_class,
                                kind) or {}
        knobs.update(overrides)
        plan = cls(max_n, max_clouds, **knobs)
        plan.tuned_knobs = knobs
        return plan

    def close(self):
        if getattr(self, "_plan", None):
            self._lib.hull3d_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def opts(self) -> dict:
        o = Opts()
        rc = self._lib.hull3d_plan_opts(self._plan, ctypes.byref(o))
        if rc:
            raise Hull3DError(rc, "plan_opts")
        return {k: getattr(o, k) for k, _ in Opts._fields_}

    @property
    def fused_levels_used(self) -> int:
        return int(self.opts["fused_levels"])

    @property
    def scratch_bytes(self) -> int:
        return int(self._lib.hull3d_plan_bytes(self._plan))

    @property
    def last_launches(self) -> int:
        return int(self._lib.hull3d_last_launch_count(self._plan))

    def profile(self, enable: bool = True) -> None:
        rc = self._lib.hull3d_profile(self._plan, int(enable))
        if rc:
            raise Hull3DError(rc, "profile")

    def profile_read(self):
        """({phase: ms summed over recorded calls}, calls)."""
        ms = (ctypes.c_double * len(PHASES))()
        calls = ctypes.c_int64(0)
        rc = self._lib.hull3d_profile_read(self._plan, ms, ctypes.byref(calls))
        if rc:
            raise Hull3DError(rc, "profile_read")
        return {k: ms[i] for i, k in enumerate(PHASES)}, calls.value

    def profile_levels(self) -> np.ndarray:
        """ms per global merge level over the recorded calls (read before profile_read)."""
        ms = (ctypes.c_double * 64)()
        rc = self._lib.hull3d_profile_levels(self._plan, ms)
        if rc:
            raise Hull3DError(rc, "profile_levels")
        return np.array(ms[:])

    def level_events(self) -> np.ndarray:
        """(2, 64) events written per merge level by the last single-hull call."""
        out = (ctypes.c_int64 * 128)()
        rc = self._lib.hull3d_level_events(self._plan, out)
        if rc:
            raise Hull3DError(rc, "level_events")
        return np.array(out[:], dtype=np.int64).reshape(2, 64)

    def window_stats(self) -> np.ndarray:
        """(64, 7) time-window counters per merge level of the last call,
        columns named by WINDOW_STATS."""
        out = (ctypes.c_int64 * (64 * len(WINDOW_STATS)))()
        rc = self._lib.hull3d_window_stats(self._plan, out)
        if rc:
            raise Hull3DError(rc, "window_stats")
        return np.array(out[:], dtype=np.int64).reshape(64, len(WINDOW_STATS))

    def compute(self, xyz, stream=None):
        """Canonical faces (F, 3) int32 on the device of xyz (synchronous)."""
        import torch

        xyz = _check_points(xyz, True)
        n = xyz.shape[0]
        faces = torch.empty((max(max_faces(n), 1), 3), dtype=torch.int32, device=xyz.device)
        nf = ctypes.c_int64(0)
        rc = self._lib.hull3d_compute(self._plan, xyz.data_ptr(), n, faces.data_ptr(), max_faces(n), ctypes.byref(nf),
                                      _stream_ptr(stream))
        if rc:
            raise Hull3DError(rc, "compute")
        return faces[: nf.value]

    def compute_async(self, xyz, faces, d_nfaces=None, d_status=None, stream=None) -> None:
        """Enqueues the hull; faces is a preallocated (cap, 3) int32 device tensor,
        d_nfaces an int64 device scalar, d_status an int32 device scalar."""
        xyz = _check_points(xyz, True)
        rc = self._lib.hull3d_compute_async(
            self._plan, xyz.data_ptr(), xyz.shape[0], faces.data_ptr(), faces.shape[0],
            None if d_nfaces is None else d_nfaces.data_ptr(), None if d_status is None else d_status.data_ptr(),
            _stream_ptr(stream))
        if rc:
            raise Hull3DError(rc, "compute_async")

    def compute_host(self, xyz, faces_out=None, stream=None):
        """End to end from host memory: xyz is an (n, 3) int32 CPU tensor (pinned
        for full speed); returns the faces as a CPU tensor view of faces_out."""
        import torch

        xyz = _check_points(xyz, False)
        n = xyz.shape[0]
        if faces_out is None:
            faces_out = torch.empty((max(max_faces(n), 1), 3), dtype=torch.int32, pin_memory=True)
        nf = ctypes.c_int64(0)
        rc = self._lib.hull3d_compute_host(self._plan, xyz.data_ptr(), n, faces_out.data_ptr(), faces_out.shape[0],
                                           ctypes.byref(nf), _stream_ptr(stream))
        if rc:
            raise Hull3DError(rc, "compute_host")
        return faces_out[: nf.value]

    def batch_async(self, xyz, offsets: np.ndarray, faces, face_offsets: np.ndarray, d_nfaces, d_status,
                    stream=None) -> None:
        """Enqueues B hulls; offsets / face_offsets are host int64 arrays of B + 1."""
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        face_offsets = np.ascontiguousarray(face_offsets, dtype=np.int64)
        B = len(offsets) - 1
        rc = self._lib.hull3d_batch_async(self._plan, xyz.data_ptr(), offsets.ctypes.data, B, faces.data_ptr(),
                                          face_offsets.ctypes.data, d_nfaces.data_ptr(), d_status.data_ptr(),
                                          _stream_ptr(stream))
        if rc:
            raise Hull3DError(rc, "batch_async")

    def delaunay_async(self, xy, tris, d_ntris=None, d_status=None, stream=None) -> None:
        """Enqueues the Delaunay triangulation of the (n, 2) int32 device tensor
        xy (|x|, |y| < 2^15) into tris, a (cap, 3) int32 device tensor."""
        import torch

        if not isinstance(xy, torch.Tensor) or xy.dtype != torch.int32 or xy.dim() != 2 or xy.shape[1] != 2:
            raise ValueError("points must be an (n, 2) int32 tensor")
        if not xy.is_cuda:
            raise ValueError("points must be on a CUDA device")
        xy = xy.contiguous()
        rc = self._lib.hull3d_delaunay_async(
            self._plan, xy.data_ptr(), xy.shape[0], tris.data_ptr(), tris.shape[0],
            None if d_ntris is None else d_ntris.data_ptr(), None if d_status is None else d_status.data_ptr(),
            _stream_ptr(stream))
        if rc:
            raise Hull3DError(rc, "delaunay_async")

    def delaunay(self, xy, stream=None):
        """Delaunay triangles (T, 3) int32 on the device of xy (synchronous)."""
        import torch

        n = int(xy.shape[0])
        dev = xy.device
        tris = torch.empty((max(2 * n - 4, 1), 3), dtype=torch.int32, device=dev)
        nt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        self.delaunay_async(xy, tris, nt, st, stream)
        (stream or torch.cuda.current_stream(dev)).synchronize()
        code = int(st.item())
        if code:
            raise Hull3DError(code, "delaunay")
        return tris[: int(nt.item())]

    def adjacency_async(self, faces, d_nfaces, n: int, nb, star_off, star, d_status, stream=None) -> None:
        """Enqueues the face neighbours and vertex stars of the canonical face
        list faces[:d_nfaces] ((cap, 3) int32 device tensor, vertices in [0, n)):
        nb (cap, 3) int32, star_off (n + 1) int64 and star (3 cap) int32 device
        tensors are written; d_status gets 0 or ERR_NOT_CLOSED."""
        cap = int(faces.shape[0])
        rc = self._lib.hull3d_adjacency_async(self._plan, faces.data_ptr(), d_nfaces.data_ptr(), cap, int(n),
                                              nb.data_ptr(), star_off.data_ptr(), star.data_ptr(),
                                              d_status.data_ptr(), _stream_ptr(stream))
        if rc:
            raise Hull3DError(rc, "adjacency_async")

    def adjacency(self, faces, n: int, stream=None):
        """(nb (F, 3) int32, star_off (n + 1) int64, star (3 F) int32) on the
        device of the canonical (F, 3) int32 face tensor (synchronous)."""
        import torch

        F = int(faces.shape[0])
        dev = faces.device
        if F == 0:
            faces = torch.zeros((1, 3), dtype=torch.int32, device=dev)
        d_nf = torch.tensor([F], dtype=torch.int64, device=dev)
        nb = torch.empty((max(F, 1), 3), dtype=torch.int32, device=dev)
        off = torch.empty(int(n) + 1, dtype=torch.int64, device=dev)
        star = torch.empty(max(3 * F, 1), dtype=torch.int32, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        self.adjacency_async(faces.contiguous(), d_nf, n, nb, off, star, st, stream)
        if stream is None:
            torch.cuda.current_stream(dev).synchronize()
        else:
            stream.synchronize()
        code = int(st.item())
        if code:
            raise Hull3DError(code, "adjacency")
        return nb[:F], off, star[: 3 * F]

    def batch(self, xyz, offsets: np.ndarray, stream=None):
        """Hulls of B clouds; returns (faces, face_offsets, nfaces, status) with
        faces on the device and the rest on the host."""
        import torch

        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        sizes = np.diff(offsets)
        caps = np.where(sizes >= 3, 2 * sizes - 4, 0)
        face_offsets = np.zeros(len(offsets), np.int64)
        face_offsets[1:] = np.cumsum(caps)
        dev = xyz.device
        faces = torch.empty((max(int(face_offsets[-1]), 1), 3), dtype=torch.int32, device=dev)
        nf = torch.zeros(len(sizes), dtype=torch.int64, device=dev)
        st = torch.zeros(len(sizes), dtype=torch.int32, device=dev)
        self.batch_async(xyz, offsets, faces, face_offsets, nf, st, stream)
        return faces, face_offsets, nf.cpu().numpy(), st.cpu().numpy()


def hull(xyz, **kw):
    """One-shot convenience: canonical faces of the (n, 3) int32 CUDA tensor xyz."""
    h = Hull3D(max(int(xyz.shape[0]), 4), **kw)
    try:
        return h.compute(xyz)
    finally:
        h.close()
