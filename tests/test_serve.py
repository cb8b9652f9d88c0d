"""The serving loop: admission under a memory budget, continuous batching,
and (on the GPU) results identical alone, in the mix and to the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1205_1171_gb300 import inputs, serve


class FakeBackend:
    """Completes work after a fixed delay; records what ran together."""

    def __init__(self, delay=0.002, resident=1000, large_slots=2, large_max=1 << 20, large_rank_space=1 << 22):
        self.delay, self.res, self.large_max = delay, resident, large_max
        self.large_rank_space = large_rank_space
        self.large = [None] * large_slots
        self.batches = [None, None]
        self.log = []

    def resident_bytes(self):
        return self.res

    def free_large(self):
        return [i for i, s in enumerate(self.large) if s is None]

    def launch_large(self, slot, reqs):
        self.large[slot] = (time.perf_counter() + self.delay, reqs)
        self.log.append(("large", [r.rid for r in reqs]))

    def free_batch(self):
        return [i for i, s in enumerate(self.batches) if s is None]

    def launch_batch(self, slot, reqs):
        self.batches[slot] = (time.perf_counter() + self.delay, reqs)
        self.log.append(("batch", [r.rid for r in reqs]))

    def poll(self):
        out, now = [], time.perf_counter()
        for store in (self.large, self.batches):
            for i, s in enumerate(store):
                if s is not None and s[0] <= now:
                    for r in s[1]:
                        out.append((r, np.full((1, 3), r.rid, np.int32)))
                    store[i] = None
        return out

    def idle(self):
        return all(s is None for s in self.large + self.batches)


def test_every_request_completes_in_order_of_admission():
    fb = FakeBackend()
    with serve.HullServer(fb, budget_bytes=1 << 30, small_max=100) as srv:
        futs = [srv.submit(np.zeros((n, 3), np.int32)) for n in [5, 500, 7, 9, 2000, 3, 50]]
        res = [f.result(timeout=10) for f in futs]
    assert [int(r[0, 0]) for r in res] == list(range(7))
    kinds = {k for k, _ in fb.log}
    assert kinds == {"large", "batch"}
    st = srv.stats.summary()
    assert st["completed"] == 7 and st["rejected"] == 0


def test_requests_above_the_budget_are_rejected_and_inflight_bytes_respect_it():
    fb = FakeBackend(delay=0.01, resident=1000)
    budget = 1000 + 20 * serve.footprint(1000)
    with serve.HullServer(fb, budget_bytes=budget, small_max=4096) as srv:
        too_big = srv.submit(np.zeros((10 ** 6, 3), np.int32))
        futs = [srv.submit(np.zeros((1000, 3), np.int32)) for _ in range(100)]
        with pytest.raises(serve.ServeError) as e:
            too_big.result(timeout=10)
        assert e.value.code == serve.ERR_BUDGET
        for f in futs:
            f.result(timeout=30)
    assert srv.stats.max_inflight_bytes <= budget - 1000
    # the budget allows 20 requests at a time: they were batched in groups
    assert max(len(ids) for k, ids in fb.log if k == "batch") <= 20


def test_requests_arriving_during_a_batch_join_the_next_one():
    fb = FakeBackend(delay=0.05)
    with serve.HullServer(fb, budget_bytes=1 << 30, small_max=4096) as srv:
        first = [srv.submit(np.zeros((10, 3), np.int32)) for _ in range(3)]
        time.sleep(0.01)  # the first batch is running; these arrive meanwhile
        later = [srv.submit(np.zeros((10, 3), np.int32)) for _ in range(5)]
        for f in first + later:
            f.result(timeout=10)
    batches = [ids for k, ids in fb.log if k == "batch"]
    assert len(batches) >= 2 and sum(len(b) for b in batches) == 8


def test_large_requests_are_batched_within_the_rank_space():
    # rank space 2^16: blocks of 2^14 (9000 points) fit four to a batch
    fb = FakeBackend(delay=0.05, large_slots=1, large_rank_space=1 << 16)
    with serve.HullServer(fb, budget_bytes=1 << 30, small_max=4096) as srv:
        futs = [srv.submit(np.zeros((9000, 3), np.int32)) for _ in range(10)]
        for f in futs:
            f.result(timeout=10)
    larges = [ids for k, ids in fb.log if k == "large"]
    assert sum(len(b) for b in larges) == 10
    assert max(len(b) for b in larges) <= 4 and max(len(b) for b in larges) >= 2
    assert serve.rank_block(9000) == 1 << 14 and serve.rank_block(8192) == 8192 and serve.rank_block(1) == 1


def test_poisson_arrivals_have_the_requested_rate():
    t = serve.poisson_arrivals(20000.0, 1.0, np.random.default_rng(1))
    assert 19000 < len(t) < 21000 and np.all(np.diff(t) > 0) and t[-1] < 1.0


@pytest.mark.gpu
def test_results_identical_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_1171_gb300 import build, hull3d

    build.build()
    pool = serve.request_pool(48, 5, 2.0, 16.0)
    dup = inputs.cloud_seeded("ball", 100, 3).copy()
    dup[7] = dup[3]
    pool.append(dup)
    backend = serve.CudaBackend(batch_points=1 << 18, batch_clouds=256, large_slots=2, large_max=1 << 16,
                                large_rank_space=1 << 18, large_clouds=64)
    single = hull3d.Hull3D(1 << 16)
    try:
        with serve.HullServer(backend, budget_bytes=4 << 30) as srv:
            rng = np.random.default_rng(2)
            order = rng.integers(0, len(pool), size=300)
            futs = [srv.submit(pool[k]) for k in order]
            got = []
            for f in futs:
                try:
                    got.append(f.result(timeout=120))
                except Exception as e:  # noqa: BLE001
                    got.append(e)
        # the oracle's faces of every distinct cloud (None: the oracle rejects it)
        want_oracle = {}
        for k in set(order.tolist()):
            try:
                want_oracle[k] = oracle.hull(pool[k])
            except oracle.OracleError:
                want_oracle[k] = None
        for k, g in zip(order, got):
            x = torch.from_numpy(pool[k]).cuda()
            try:
                want = single.compute(x).cpu().numpy()
            except hull3d.Hull3DError as e:
                assert isinstance(g, hull3d.Hull3DError) and g.code == e.code
                assert want_oracle[k] is None, k  # the oracle rejects it too
                continue
            assert np.array_equal(g, want), (k, len(pool[k]))
            # served, alone and the definition (Sec. 2: one face per root event) agree
            assert want_oracle[k] is not None and np.array_equal(g, want_oracle[k]), (k, len(pool[k]))
        assert srv.stats.batches >= 1 and srv.stats.large >= 1
    finally:
        single.close()
