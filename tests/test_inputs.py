"""The seeded generators: distinct, in range, reproducible, right shapes."""
import numpy as np
import pytest

from paper_1205_1171_gb300 import inputs


@pytest.mark.parametrize("dist", inputs.DISTS)
def test_cloud_distinct_in_range_reproducible(dist):
    a = inputs.cloud_seeded(dist, 20000, 11)
    b = inputs.cloud_seeded(dist, 20000, 11)
    assert a.dtype == np.int32 and a.shape == (20000, 3)
    assert np.array_equal(a, b)
    assert a.min() >= inputs.LO and a.max() <= inputs.HI
    assert np.unique(a, axis=0).shape[0] == len(a)
    if dist == "ball":
        assert np.all((a.astype(np.int64) ** 2).sum(1) < (1 << 40))
    if dist == "sphere":
        r = np.sqrt((a.astype(np.float64) ** 2).sum(1))
        assert np.all(np.abs(r - inputs.HI) < 2.0)


def test_gauss_clips_onto_the_cube_faces():
    a = inputs.cloud_seeded("gauss", 1 << 20, 3)
    on_face = np.sum((a == inputs.HI) | (a == inputs.LO))
    assert 50 < on_face < 400  # ~ 2^20 * 6 * P(N(0,1) > 4) ~ 200


def test_batch_shapes():
    xyz, off, kinds = inputs.batch(64, 5)
    assert off[0] == 0 and off[-1] == len(xyz) and len(off) == 65
    sizes = np.diff(off)
    assert sizes.min() >= 16 and sizes.max() <= 4096
    assert set(kinds) <= set(inputs.DISTS)


def test_planar_sets_are_distinct_in_range_and_seeded():
    import numpy as np

    from paper_1205_1171_gb300 import inputs

    for kind in inputs.PLANAR:
        for n in (1, 3, 257, 4000):
            a = inputs.planar_seeded(kind, n, 17)
            assert a.shape == (n, 2) and a.dtype == np.int32
            assert np.abs(a).max() <= (1 << 15) - 1
            assert len(np.unique(a, axis=0)) == n
            assert np.array_equal(a, inputs.planar_seeded(kind, n, 17))
