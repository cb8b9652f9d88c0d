"""The N-replica path of bench.py (one rank per GPU, no data exchange) on
world-size-2 gloo process groups on the CPU: the max-over-ranks timing, the
per-rank inputs, and the reference arm's rank handling."""
import argparse
import contextlib
import hashlib
import io
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        res = {"max": bench.max_over_ranks(10.0 * (rank + 1), dist, device="cpu")}
        clouds = bench.make_inputs(rank, 512, ("cube", "gauss"))
        mine = [hashlib.sha256(c.tobytes()).hexdigest() for c in clouds]
        every = [None] * world
        dist.all_gather_object(every, mine)
        res["digests"] = every
        buf = io.StringIO()
        if rank != 0:  # rank 0 would time the oracle for minutes; the others must do nothing
            args = argparse.Namespace(gpus=world, steps=1, warmup=3)
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args, rank, world)
        res["reference_stdout"] = buf.getvalue()
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_without_a_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None) == 3.5


def test_two_replicas_on_gloo(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    # both ranks time with the slowest rank's duration
    assert r[0]["max"] == r[1]["max"] == 20.0
    # each rank hulls its own clouds (weak scaling: no shared input, no exchange)
    assert r[0]["digests"] == r[1]["digests"]
    assert not set(r[0]["digests"][0]) & set(r[0]["digests"][1])
    # the reference arm runs on rank 0 only
    assert r[1]["reference_stdout"] == ""
