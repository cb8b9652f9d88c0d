"""The autotuner's search and cache logic (CPU), and on the GPU that tuned
knobs never change the faces (against the default plan and the oracle)."""
import numpy as np
import pytest

import oracle

from paper_1205_1171_gb300 import autotune


def test_candidates_cover_the_knobs_and_are_unique():
    c = autotune.candidates(1 << 20)
    assert len(c) == len({tuple(sorted(k.items())) for k in c})
    for k in c:
        assert set(k) == set(autotune.KNOBS)
    # 0 = the library's automatic choice, always among the candidates
    assert {k["level_occupancy"] for k in c} == {0, 4}
    assert 0 in {k["cmp_level"] for k in c} and 0 in {k["seg_min_events"] for k in c}
    assert {k["seg_events"] for k in c} >= {256, 512, 1024}
    small = autotune.candidates(1000)
    assert all(k["cmp_level"] <= autotune.bucket(1000) + 1 for k in small)


def test_search_picks_the_fastest():
    space = [dict(a=i) for i in range(10)]
    best, ms, allr = autotune.search(space, lambda k: (k["a"] - 6) ** 2 + 1.0)
    assert best == {"a": 6} and ms == 1.0 and len(allr) == 10


def test_cache_roundtrip_and_bucket_fallback(tmp_path):
    path = str(tmp_path / "t.json")
    assert autotune.lookup("GPU", 1 << 20, path) is None
    cache = autotune.load(path)
    kn = dict(cmp_level=11, seg_level=10, seg_events=512, seg_min_events=512, level_occupancy=4)
    cache[autotune.key("GPU", 1 << 16)] = {"knobs": kn}
    autotune.save(cache, path)
    assert autotune.lookup("GPU", 1 << 16, path) == kn
    assert autotune.lookup("GPU", 1 << 18, path) == kn  # nearest tuned bucket below
    assert autotune.lookup("GPU", 1 << 10, path) is None
    assert autotune.lookup("OTHER", 1 << 16, path) is None


@pytest.mark.gpu
def test_tuning_never_changes_the_faces(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_1171_gb300 import build, hull3d, inputs

    build.build()
    path = str(tmp_path / "t.json")
    best = autotune.tune(1 << 12, reps=1, path=path, max_candidates=6)
    assert set(best) == set(autotune.KNOBS)
    p = hull3d.Hull3D.tuned(1 << 12, cache=path)
    ref = hull3d.Hull3D(1 << 12)
    try:
        for d in inputs.DISTS:
            pts = inputs.cloud_seeded(d, 4000, 3)
            x = torch.from_numpy(pts).cuda()
            got = p.compute(x).cpu().numpy()
            assert np.array_equal(got, ref.compute(x).cpu().numpy())
            assert np.array_equal(got, oracle.hull(pts)), d  # the tuned plan gives the oracle's faces
    finally:
        p.close()
        ref.close()
