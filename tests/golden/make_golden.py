"""Writes the stored expected values of the large K-truss workloads.

Every value here comes from the CPU oracle (``oracle.ktruss``, Alg. 1 bulk
peeling with the eager credit rule) run on inputs from ``graphgen``; nothing is
taken from the CUDA library.  The files hold digests (SHA-256 of the uint8 mask
and of the little-endian int32 supports, in input edge order) and the
per-round statistics, so that GPU tests can compare full outputs of graphs too
large to rerun the oracle on in a test.

    python tests/golden/make_golden.py rmat20 rmat20r      # config 2
    python tests/golden/make_golden.py rmat23c --K 3       # config 3, K=3
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

DEFAULT_K = {"rmat20": [3, 4, 8, 16], "rmat20r": [3, 4, 8, 16], "rmat23c": [3]}
DEFAULT_SEEDS = {"rmat20": [0, 1, 2], "rmat20r": [0, 1, 2], "rmat23c": [0]}


def sha(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()


def graph_digest(g) -> str:
    import numpy as np
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    return h.hexdigest()


def one(args):
    name, seed, K = args
    import numpy as np
    import graphgen as gg
    import oracle
    g = gg.cached_workload(name, seed)
    t0 = time.time()
    r = oracle.ktruss(g.row_ptr, g.col, K)
    dt = time.time() - t0
    return {
        "workload": name, "seed": seed, "K": K, "n": g.n, "m": g.m,
        "graph_sha256": graph_digest(g),
        "rounds": r.rounds, "removed_per_round": r.removed_per_round,
        "edges_out": int(r.mask.sum()), "triangles_out": int(r.triangles),
        "support_sum": int(r.support.astype(np.int64).sum()),
        "mask_sha256": sha(np.ascontiguousarray(r.mask, dtype=np.uint8)),
        "support_sha256": sha(np.ascontiguousarray(r.support, dtype="<i4")),
        "oracle_seconds": round(dt, 2),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--K", type=int, nargs="*")
    ap.add_argument("--seeds", type=int, nargs="*")
    ap.add_argument("--jobs", type=int, default=4)
    a = ap.parse_args()
    import graphgen as gg
    import oracle
    gg.build()
    oracle.build()
    for name in a.workloads:
        seeds = a.seeds if a.seeds else DEFAULT_SEEDS[name]
        for s in seeds:
            gg.cached_workload(name, s)  # generate once, before the pool
        ks = a.K if a.K else DEFAULT_K[name]
        jobs = [(name, s, K) for s in seeds for K in ks]
        path = os.path.join(HERE, f"{name}.json")
        old = []
        if os.path.exists(path):
            with open(path) as f:
                old = json.load(f)["cases"]
        with mp.get_context("spawn").Pool(min(a.jobs, len(jobs))) as pool:
            new = pool.map(one, jobs)
        keep = {(c["seed"], c["K"]): c for c in old}
        for c in new:
            keep[(c["seed"], c["K"])] = c
        cases = [keep[k] for k in sorted(keep)]
        with open(path, "w") as f:
            json.dump({"source": "oracle.ktruss (CPU), tests/golden/make_golden.py",
                       "cases": cases}, f, indent=1)
        print(f"wrote {path} ({len(cases)} cases)")


if __name__ == "__main__":
    main()
