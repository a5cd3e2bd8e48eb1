"""Writes the stored expected values of the large K-truss workloads.

Every value here comes from the CPU oracle (``oracle.ktruss``, Alg. 1 bulk
peeling with the eager credit rule) run on inputs from ``graphgen``; nothing is
taken from the CUDA library.  The files hold digests (SHA-256 of the uint8 mask
and of the little-endian int32 supports, in input edge order) and the
per-round statistics, so that GPU tests can compare full outputs of graphs too
large to rerun the oracle on in a test.

    python tests/golden/make_golden.py rmat20 rmat20r      # config 2
    python tests/golden/make_golden.py rmat23c --K 3       # config 3, K=3
    python tests/golden/make_golden.py batch --jobs 8      # config 4, 4096 graphs
    python tests/golden/make_golden.py serve --jobs 8      # config 5, 64 requests
    python tests/golden/make_golden.py decompose rmat20 rmat20r   # K = 3 .. K_max

decompose stores, per graph, the oracle's truss decomposition (per-edge
trussness by the second, independent algorithm, oracle.truss_decomposition):
its digest (little-endian int32 in input edge order), K_max and the number of
edges at each trussness.

The batching workload (graphgen.batch_config: 4096 graphs, 1e3..2e6 edges,
K per graph in 3..12, seed 0) is stored per graph (K, rounds, kept edges) and
as digests of digests: the SHA-256 of the concatenated hex SHA-256 digests of
every graph's mask (resp. little-endian int32 supports, resp. CSR), in batch
order.

The serving workload (graphgen.serve_config: 64 requests, 1e4..5e7 edges, K in
3..16, seed 0) is stored per request for every request the oracle can finish
in minutes: all G(n, m) requests and the R-MAT requests up to scale 20 (the
scale-21 and -22 ones would take hours at K up to 16).
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


def relabelled_slots(g):
    """(h, slot): h is g renumbered by ascending degree (graphgen's relabel,
    an isomorphic copy) and slot[e] the slot in h of g's edge e."""
    import numpy as np
    import graphgen as gg
    h = gg.from_edges(g.n, g.edges(), relabel=True)
    new = gg.relabel_map(g.n, g.row_ptr, g.col).astype(np.int64)
    a, b = new[g.rows().astype(np.int64)], new[g.col.astype(np.int64)]
    key = np.minimum(a, b) * g.n + np.maximum(a, b)
    hkey = h.rows().astype(np.int64) * g.n + h.col.astype(np.int64)
    slot = np.searchsorted(hkey, key)
    assert np.array_equal(hkey[slot], key)
    return h, slot


def one(args):
    name, seed, K = args[:3]
    relabel = len(args) > 3 and args[3]
    import numpy as np
    import graphgen as gg
    import oracle
    g = gg.cached_workload(name, seed)
    t0 = time.time()
    if relabel:
        # the K-truss, its supports and its rounds do not depend on how the
        # vertices are numbered: run the oracle on the degree-relabelled
        # isomorphic copy (shorter upper rows, less merge work) and read every
        # edge's outputs at its slot there
        h, slot = relabelled_slots(g)
        r = oracle.ktruss(h.row_ptr, h.col, K)
        r.mask = r.mask[slot]
        r.support = r.support[slot]
    else:
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


BATCH = {"graphs": 4096, "seed": 0, "m_lo": 1e3, "m_hi": 2e6, "k_lo": 3, "k_hi": 12}


def one_batch_graph(args):
    k, spec, K = args
    import numpy as np
    import graphgen as gg
    import oracle
    g = gg.from_spec(spec)
    t0 = time.time()
    r = oracle.ktruss(g.row_ptr, g.col, K)
    dt = time.time() - t0
    return {"index": k, "K": K, "m": g.m, "graph_sha256": graph_digest(g), "rounds": r.rounds,
            "edges_out": int(r.mask.sum()), "triangles_out": int(r.triangles),
            "support_sum": int(r.support.astype(np.int64).sum()),
            "mask_sha256": sha(np.ascontiguousarray(r.mask, dtype=np.uint8)),
            "support_sha256": sha(np.ascontiguousarray(r.support, dtype="<i4")),
            "seconds": dt}


def digest_of_digests(hexes) -> str:
    return hashlib.sha256("".join(hexes).encode("ascii")).hexdigest()


def make_batch(jobs: int):
    import graphgen as gg
    specs = gg.batch_specs(BATCH["graphs"], BATCH["seed"], BATCH["m_lo"], BATCH["m_hi"],
                           BATCH["k_lo"], BATCH["k_hi"])
    tasks = [(k, sp, K) for k, (sp, K) in enumerate(specs)]
    # largest graphs first, so that the pool ends evenly
    tasks.sort(key=lambda t: -(t[1][2] if t[1][0] == "er" else t[1][2] << t[1][1]))
    t0 = time.time()
    with mp.get_context("spawn").Pool(jobs) as pool:
        res = pool.map(one_batch_graph, tasks, chunksize=1)
    res.sort(key=lambda r: r["index"])
    out = dict(BATCH)
    out.update({
        "source": "oracle.ktruss (CPU) on every graph of graphgen.batch_config, "
                  "tests/golden/make_golden.py",
        "edges": sum(r["m"] for r in res),
        "graphs_sha256": digest_of_digests(r["graph_sha256"] for r in res),
        "mask_sha256": digest_of_digests(r["mask_sha256"] for r in res),
        "support_sha256": digest_of_digests(r["support_sha256"] for r in res),
        "edges_out_total": sum(r["edges_out"] for r in res),
        "support_sum_total": sum(r["support_sum"] for r in res),
        "triangles_out_total": sum(r["triangles_out"] for r in res),
        "oracle_cpu_seconds": round(sum(r["seconds"] for r in res), 1),
        "wall_seconds": round(time.time() - t0, 1),
        "K": [r["K"] for r in res],
        "rounds": [r["rounds"] for r in res],
        "edges_out": [r["edges_out"] for r in res],
    })
    path = os.path.join(HERE, "batch4096.json")
    with open(path, "w") as f:
        # one key per line; the per-graph lists stay on one line each
        f.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v, separators=(',', ':'))}"
                                   for k, v in out.items()) + "\n}\n")
    print(f"wrote {path} ({len(res)} graphs, {out['wall_seconds']} s)")


SERVE = {"requests": 64, "seed": 0, "m_lo": 1e4, "m_hi": 5e7, "k_lo": 3, "k_hi": 16,
         "rmat_max_scale": 20}


def make_serve(jobs: int):
    import graphgen as gg
    specs = gg.serve_specs(SERVE["requests"], SERVE["seed"], SERVE["m_lo"], SERVE["m_hi"],
                           SERVE["k_lo"], SERVE["k_hi"])
    tasks = [(k, sp, K) for k, (sp, K) in enumerate(specs)
             if sp[0] == "er" or sp[1] <= SERVE["rmat_max_scale"]]
    # R-MAT first (they take longest), larger first
    tasks.sort(key=lambda t: (t[1][0] == "er", -(t[1][2] if t[1][0] == "er" else 16 << t[1][1])))
    t0 = time.time()
    with mp.get_context("spawn").Pool(jobs) as pool:
        res = pool.map(one_batch_graph, tasks, chunksize=1)
    res.sort(key=lambda r: r["index"])
    for r in res:
        r["seconds"] = round(r["seconds"], 2)
    out = dict(SERVE)
    out.update({
        "source": "oracle.ktruss (CPU) on the requests of graphgen.serve_config listed here, "
                  "tests/golden/make_golden.py",
        "wall_seconds": round(time.time() - t0, 1),
        "cases": res,
    })
    path = os.path.join(HERE, "serve64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path} ({len(res)} requests, {out['wall_seconds']} s)")


def one_decomposition(args):
    name, seed = args
    import numpy as np
    import graphgen as gg
    import oracle
    g = gg.cached_workload(name, seed)
    t0 = time.time()
    tr = oracle.truss_decomposition(g.row_ptr, g.col)
    dt = time.time() - t0
    hist = np.bincount(tr, minlength=int(tr.max()) + 1 if g.m else 1)
    return {"workload": name, "seed": seed, "n": g.n, "m": g.m, "graph_sha256": graph_digest(g),
            "kmax": int(tr.max()) if g.m else 0,
            "trussness_sha256": sha(np.ascontiguousarray(tr, dtype="<i4")),
            "edges_per_trussness": {str(k): int(c) for k, c in enumerate(hist) if c},
            "oracle_seconds": round(dt, 1)}


def make_decompositions(names, jobs: int):
    import graphgen as gg
    for name in names:
        gg.cached_workload(name, 0)  # generate once, before the pool
    with mp.get_context("spawn").Pool(min(jobs, len(names))) as pool:
        res = pool.map(one_decomposition, [(name, 0) for name in names], chunksize=1)
    for r in res:
        path = os.path.join(HERE, f"{r['workload']}_trussness.json")
        with open(path, "w") as f:
            json.dump(dict(r, source="oracle.truss_decomposition (CPU), "
                                     "tests/golden/make_golden.py"), f, indent=1)
        print(f"wrote {path} ({r['oracle_seconds']} s)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--K", type=int, nargs="*")
    ap.add_argument("--seeds", type=int, nargs="*")
    ap.add_argument("--jobs", type=int, default=4)
    ap.add_argument("--relabel", action="store_true",
                    help="run the oracle on the degree-relabelled isomorphic copy of each graph "
                         "(same outputs in input edge order, less merge work)")
    a = ap.parse_args()
    import graphgen as gg
    import oracle
    gg.build()
    oracle.build()
    if a.workloads[0] == "decompose":
        make_decompositions(a.workloads[1:], a.jobs)
        return
    for name in a.workloads:
        if name == "batch":
            make_batch(a.jobs)
            continue
        if name == "serve":
            make_serve(a.jobs)
            continue
        seeds = a.seeds if a.seeds else DEFAULT_SEEDS[name]
        for s in seeds:
            gg.cached_workload(name, s)  # generate once, before the pool
        ks = a.K if a.K else DEFAULT_K[name]
        jobs = [(name, s, K, a.relabel) for s in seeds for K in ks]
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
