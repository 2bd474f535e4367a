"""Write batch64_oracle.txt: the CPU oracle's exact cut of every pair of the
64-pair batch workload (uneven sizes w ~ U[160, 640], h ~ U[120, 480], depth
numbers ~ U[16, 64], layered scenes; ``synth.make_batch(64)``).

Calls only the oracle (cost volume + Boykov-Kolmogorov) and the seeded input
generator; nothing here touches the CUDA library.  One line per pair:
    index w h D sha256(L)[:16] sha256(R)[:16] flow sha256(labels)[:16]
labels as little-endian int32 [h][n_g], row-major.  It takes tens of minutes
on a few cores: run it once (``python tests/golden/make_batch64_oracle.py``)
and commit the output.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch64_oracle.txt")


def sha16(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]


def solve_one(k: int):
    import oracle
    from paper_1803_01516_gb300 import synth
    wl, L, R, _ = synth.make_batch(64)[k]
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1, "bk")
    X = ref["labels"].astype("<i4")
    return k, wl.w, wl.h, wl.D, sha16(L), sha16(R), ref["flow"], sha16(X)


def main():
    import oracle
    oracle.build()
    from paper_1803_01516_gb300 import synth
    batch = synth.make_batch(64)
    nodes = [(wl.w - 2 * (wl.D - 1)) * wl.h * (wl.D - 1) for wl, _, _, _ in batch]
    order = sorted(range(64), key=lambda k: -nodes[k])      # largest first
    workers = int(os.environ.get("WORKERS", os.cpu_count() or 1))
    rows = {}
    with mp.get_context("spawn").Pool(workers) as pool:
        for r in pool.imap_unordered(solve_one, order):
            rows[r[0]] = r
            print(f"pair {r[0]}: {nodes[r[0]]} nodes, flow {r[6]}", flush=True)
    with open(OUT, "w") as f:
        f.write("# The CPU oracle's exact cut of the 64-pair batch workload (synth.make_batch(64)),\n"
                "# written by make_batch64_oracle.py (oracle only).  Columns:\n"
                "# index w h D sha256(L)[:16] sha256(R)[:16] flow sha256(labels int32 [h][n_g])[:16]\n")
        for k in range(64):
            f.write(" ".join(str(x) for x in rows[k]) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
