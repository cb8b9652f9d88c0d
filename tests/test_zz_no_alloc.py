"""The allocation-free entry point, hull3d_compute_static.

Some callers may not allocate device memory: code inside a host framework
that owns the whole device through a fixed pool or budget, or latency-critical
loops that cannot pay for cudaMalloc/cudaFree (which may synchronise the
device).  hull3d_compute_static serves them: the caller passes input and
output buffers, and the library's scratch comes from one static device array.

This test calls it through the C ABI and checks that it gives exactly the
faces of the planned entry point (and of the oracle), on two calls in a row
(the static array keeps the previous call's contents), and that sizes above
its maximum are refused.  It is kept in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1205_1171_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_1171_gb300 import build, hull3d

    build.build()
    hull3d.load()
    return hull3d


def _static(H, x):
    lib = H.load()
    n = x.shape[0]
    cap = max(2 * n - 4, 1)
    faces = torch.full((cap, 3), -1, dtype=torch.int32, device="cuda")
    nf = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.hull3d_compute_static(x.data_ptr(), n, faces.data_ptr(), cap, nf.data_ptr(), st.data_ptr(), stream)
    assert rc == 0, lib.hull3d_strerror(rc)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return faces[: int(nf.item())].cpu().numpy()


def test_static_entry_matches_planned_entry_on_consecutive_calls(H):
    import oracle

    plan = H.Hull3D(H.STATIC_MAX_N)
    try:
        # the sphere at the maximum size puts nearly every point on the hull:
        # the largest movies this entry point can meet
        cases = [("sphere", 5000, 1), ("gauss", H.STATIC_MAX_N, 2), ("cube", 777, 3), ("sphere", H.STATIC_MAX_N, 4)]
        for dist, n, seed in cases:
            pts = inputs.cloud_seeded(dist, n, seed)
            x = torch.from_numpy(pts).cuda()
            want = plan.compute(x).cpu().numpy()
            assert np.array_equal(want, oracle.hull(pts)), (dist, n)
            for _ in range(2):  # two calls in a row on the same shared array
                got = _static(H, x)
                assert got.shape == want.shape and np.array_equal(got, want), (dist, n)
    finally:
        plan.close()


def test_static_entry_refuses_sizes_above_its_maximum(H):
    lib = H.load()
    n = H.STATIC_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    faces = torch.empty((2 * n, 3), dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.hull3d_compute_static(x.data_ptr(), n, faces.data_ptr(), 2 * n, nf.data_ptr(), st.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == H.ERR_TOO_LARGE
    assert b"HULL3D_STATIC_MAX_N" in lib.hull3d_strerror(rc)


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1205_1171_gb300 import hull3d, inputs
lib = hull3d.load()
n = hull3d.STATIC_MAX_N
x = torch.from_numpy(inputs.cloud_seeded("gauss", n, 11)).cuda()
faces = torch.full((2 * n - 4, 3), -1, dtype=torch.int32, device="cuda")
nf = torch.full((1,), -1, dtype=torch.int64, device="cuda")
st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
rc = lib.hull3d_compute_static(x.data_ptr(), n, faces.data_ptr(), 2 * n - 4, nf.data_ptr(), st.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
torch.cuda.synchronize()
assert rc == 0 and int(st.item()) == 0, (rc, int(st.item()))
got = faces[: int(nf.item())].cpu().numpy()
plan = hull3d.Hull3D(n)
want = plan.compute(x).cpu().numpy()
plan.close()
assert np.array_equal(got, want)
print("ok", got.shape[0])
"""


def test_static_entry_as_the_first_call_of_a_process(H, tmp_path):
    # The kernels' shared-memory limits are per process: the static entry must
    # set them itself when no plan was made before it.
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fresh.py"
    script.write_text(_FRESH)
    out = subprocess.run([sys.executable, str(script), root], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok")
