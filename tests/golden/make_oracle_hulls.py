"""Writes oracle_hulls.json: the oracle's face count and the SHA-256 of its
canonical face list (int32 little-endian rows (a, b, c)) for the full-size
single-hull workloads, so that GPU tests can check those sizes bit for bit
without rerunning the serial oracle (minutes per cloud at n = 2^24).

Every value is computed by oracle/ alone from the seeded synthetic clouds of
paper_1205_1171_gb300/inputs.py:
  cube and gauss at n = 2^24, seeds seed_for(30) and seed_for(31) (the clouds
  bench.py times in its main leg, rank 0);
  ball and sphere at n = 2^20, seed seed_for(2).
Run:  python tests/golden/make_oracle_hulls.py [name ...]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1205_1171_gb300 import inputs  # noqa: E402

CASES = {
    "cube_2e24": ("cube", 1 << 24, inputs.seed_for(30)),
    "gauss_2e24": ("gauss", 1 << 24, inputs.seed_for(31)),
    "ball_2e20": ("ball", 1 << 20, inputs.seed_for(2)),
    "sphere_2e20": ("sphere", 1 << 20, inputs.seed_for(2)),
}
OUT = os.path.join(HERE, "oracle_hulls.json")


def face_digest(faces: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(faces, dtype="<i4").tobytes()).hexdigest()


def main(names):
    oracle.build()
    for name in names:
        dist, n, seed = CASES[name]
        pts = inputs.cloud_seeded(dist, n, seed)
        t0 = time.time()
        faces = oracle.hull(pts)
        entry = {"dist": dist, "n": n, "seed": seed, "faces": int(faces.shape[0]), "sha256": face_digest(faces),
                 "oracle_seconds": round(time.time() - t0, 1)}
        print(name, entry, flush=True)
        # re-read just before writing: several cases may run as separate processes
        try:
            with open(OUT) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
        table[name] = entry
        tmp = f"{OUT}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, OUT)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
