"""Seeded generators: deterministic, valid upper-triangular CSR, recipes as stated."""
import numpy as np
import pytest

import graphgen as gg
import oracle


def valid(g):
    return oracle.check_csr(g.row_ptr, g.col) == 0


def test_er_exact_edge_count_and_determinism():
    for s in range(3):
        a, b = gg.er(2000, 16000, s), gg.er(2000, 16000, s)
        assert a.m == 16000 and valid(a)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert not np.array_equal(gg.er(2000, 16000, 0).col, gg.er(2000, 16000, 1).col)


def test_rmat_valid_deterministic_and_skewed():
    a = gg.rmat(14, 16, 0)
    b = gg.rmat(14, 16, 0)
    assert valid(a) and np.array_equal(a.col, b.col) and a.n == 1 << 14
    assert a.m <= 16 << 14
    deg = np.diff(a.row_ptr) + np.bincount(a.col, minlength=a.n)
    # original ids: vertex 0 is the hub of an a=0.57 R-MAT
    assert deg.argmax() == 0 and deg.max() > 20 * deg.mean()


def test_rmat_relabel_is_degree_ascending_and_isomorphic():
    a = gg.rmat(12, 16, 3)
    r = gg.rmat(12, 16, 3, relabel=True)
    assert valid(r) and r.m == a.m
    deg = np.diff(r.row_ptr) + np.bincount(r.col, minlength=r.n)
    assert np.all(np.diff(deg) >= 0)
    da = np.sort(np.diff(a.row_ptr) + np.bincount(a.col, minlength=a.n))
    assert np.array_equal(np.sort(deg), da)


def test_planted_cliques_present():
    g = gg.rmat(12, 4, 1, n_cliques=4, clique_lo=10, clique_hi=40)
    tr = oracle.truss_decomposition(g.row_ptr, g.col)
    assert tr.max() >= 40
    assert (tr >= 40).sum() >= 40 * 39 // 2


def test_from_edges_merges_duplicates_and_drops_loops():
    g = gg.from_edges(5, [(1, 0), (0, 1), (2, 2), (4, 3), (3, 4), (0, 4)])
    assert g.m == 3 and valid(g)
    assert g.edges().tolist() == [[0, 1], [0, 4], [3, 4]]


def test_counter_rng_is_pure():
    k = gg.stream_key(2, 7, 0)
    assert gg.rand_u64(k, 5) == gg.rand_u64(k, 5)
    assert gg.rand_u64(k, 5) != gg.rand_u64(k, 6)
    # SplitMix64 reference value: output function applied to state 0 + golden gamma
    assert gg.rand_u64(0, 0) == 0xE220A8397B1DCDAF


def _digest(pairs):
    import hashlib
    h = hashlib.sha256()
    for g, K in pairs:
        h.update(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
        h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
        h.update(int(K).to_bytes(4, "little"))
    return h.hexdigest()


def test_batch_and_serve_workloads_are_deterministic_and_in_range():
    # the graphs are built on a thread pool: the result must not depend on it
    b1 = gg.batch_config(48, seed=3, m_lo=1e3, m_hi=3e4)
    b2 = gg.batch_config(48, seed=3, m_lo=1e3, m_hi=3e4)
    assert _digest(b1) == _digest(b2)
    for k, (g, K) in enumerate(b1):
        assert 3 <= K <= 12
        assert g.row_ptr[0] == 0 and g.row_ptr[-1] == g.m
        if k % 2 == 0:  # G(n, m): exactly the drawn size
            assert 1e3 <= g.m <= 3e4 + 1
    s1 = gg.serve_config(12, seed=4, m_lo=1e4, m_hi=1e5)
    s2 = gg.serve_config(12, seed=4, m_lo=1e4, m_hi=1e5)
    assert _digest(s1) == _digest(s2)
    assert all(3 <= K <= 16 for _, K in s1)
    assert _digest(gg.batch_config(48, seed=5, m_lo=1e3, m_hi=3e4)) != _digest(b1)


def test_batch_workload_reproduces_the_stored_oracle_record():
    """The full batching workload (4096 graphs, 1.2e9 edges) must still be the
    one the oracle digests in tests/golden/batch4096.json were taken on: same
    K per graph, edge count and graph digest.  The record must also be
    consistent in itself: support sum = 3 x triangles (every triangle credits
    its three edges), one entry per graph."""
    import hashlib
    import json
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096.json")
    with open(p) as f:
        c = json.load(f)
    G = c["graphs"]
    assert len(c["K"]) == len(c["rounds"]) == len(c["edges_out"]) == G
    assert c["support_sum_total"] == 3 * c["triangles_out_total"]
    assert sum(c["edges_out"]) == c["edges_out_total"]
    assert all(r >= 1 for r in c["rounds"])
    specs = gg.batch_specs(G, c["seed"], c["m_lo"], c["m_hi"], c["k_lo"], c["k_hi"])
    assert [K for _, K in specs] == c["K"]
    hexes = []
    edges = 0
    for g, _ in gg.batch_config(G, seed=c["seed"], m_lo=c["m_lo"], m_hi=c["m_hi"],
                                k_lo=c["k_lo"], k_hi=c["k_hi"]):
        edges += g.m
        assert c["edges_out"][len(hexes)] <= g.m
        hexes.append(hashlib.sha256(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes()
                                    + np.ascontiguousarray(g.col, dtype="<i4").tobytes())
                     .hexdigest())
    assert edges == c["edges"]
    assert hashlib.sha256("".join(hexes).encode("ascii")).hexdigest() == c["graphs_sha256"]


def test_serve_workload_reproduces_the_stored_oracle_record():
    """The requests of the serving workload that tests/golden/serve64.json
    holds oracle results for must still be generated as they were (K, edge
    count, graph digest); each record is consistent in itself (support sum =
    3 x triangles) and covers every G(n,m) request and every R-MAT request up
    to the recorded scale."""
    import hashlib
    import json
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "serve64.json")
    with open(p) as f:
        c = json.load(f)
    specs = gg.serve_specs(c["requests"], c["seed"], c["m_lo"], c["m_hi"], c["k_lo"], c["k_hi"])
    covered = [k for k, (sp, _) in enumerate(specs)
               if sp[0] == "er" or sp[1] <= c["rmat_max_scale"]]
    assert [x["index"] for x in c["cases"]] == covered
    for x in c["cases"]:
        assert x["support_sum"] == 3 * x["triangles_out"]
        assert 0 <= x["edges_out"] <= x["m"] and x["rounds"] >= 1
        sp, K = specs[x["index"]]
        assert K == x["K"]
        g = gg.from_spec(sp)
        assert g.m == x["m"]
        assert hashlib.sha256(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes()
                              + np.ascontiguousarray(g.col, dtype="<i4").tobytes()
                              ).hexdigest() == x["graph_sha256"]


@pytest.mark.parametrize("name", ["rmat20", "rmat20r"])
def test_rmat20_workloads_reproduce_the_stored_oracle_records(name):
    """The R-MAT scale-20 graphs (original ids and degree-relabelled, seed 0)
    must still be the ones the stored oracle digests and truss decompositions
    were taken on."""
    import hashlib
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with open(os.path.join(here, f"{name}.json")) as f:
        want = {c["graph_sha256"] for c in json.load(f)["cases"] if c["seed"] == 0}
    with open(os.path.join(here, f"{name}_trussness.json")) as f:
        want.add(json.load(f)["graph_sha256"])
    assert len(want) == 1
    g = gg.workload(name, 0)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    assert h.hexdigest() in want
