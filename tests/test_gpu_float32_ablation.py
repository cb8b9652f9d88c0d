"""The float32 arithmetic ablation (hull3d_opts.float32_ablation on batch
calls: the paper's cl_float predicates in the batch kernel): it runs on every
size class, reports only well-formed results or an internal-error status, is
wrong on a degenerate lattice (the exact path's perturbation resolves it), and
leaves the exact kernel's faces equal to the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1205_1171_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_1171_gb300 import build, hull3d

    build.build()
    oracle.build()
    return hull3d


def test_float32_ablation_runs_and_the_exact_path_is_unchanged(H):
    xyz, off, _ = inputs.batch(400, inputs.seed_for(9))
    lattice = np.array([(x, y, z) for x in range(8) for y in range(8) for z in range(8)], np.int32) * (1 << 16)
    lattice -= 1 << 18
    xyz = np.concatenate([xyz, lattice]).astype(np.int32)
    off = np.append(off, off[-1] + len(lattice))
    B = len(off) - 1
    x = torch.from_numpy(xyz).cuda()
    exact = H.Hull3D(4096, max_clouds=B)
    f32 = H.Hull3D(4096, max_clouds=B, float32_ablation=1)
    try:
        fe, foff, ne, se = exact.batch(x, off)
        ff, foff2, nf, sf = f32.batch(x, off)
        fe, ff = fe.cpu().numpy(), ff.cpu().numpy()
        assert not se.any() and np.array_equal(foff, foff2)
        assert set(np.unique(sf).tolist()) <= {0, H.ERR_INTERNAL}
        wrong = 0
        for b in range(B):
            n = int(off[b + 1] - off[b])
            got = fe[foff[b]: foff[b] + ne[b]]
            assert np.array_equal(got, oracle.hull(xyz[off[b]: off[b + 1]])), b
            if sf[b] == 0:
                g = ff[foff[b]: foff[b] + nf[b]]
                assert g.size == 0 or (g.min() >= 0 and g.max() < n)
                wrong += int(nf[b] != ne[b] or not np.array_equal(g, got))
        # the lattice: collinear and coplanar everywhere; float ties are not the hull
        assert sf[B - 1] != 0 or nf[B - 1] != ne[B - 1] or not np.array_equal(
            ff[foff[B - 1]: foff[B - 1] + nf[B - 1]], fe[foff[B - 1]: foff[B - 1] + ne[B - 1]])
    finally:
        exact.close()
        f32.close()
