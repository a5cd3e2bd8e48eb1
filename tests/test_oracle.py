"""Pins of the CPU oracle to things other than itself (no GPU).

* brute force: Alg. 1 written literally with dense matrices, on every graph
  with n <= 6 and on 1000 seeded random graphs with n <= 40;
* closed forms: K_n, the book graph, stars and trees, the triangle strip
  (which fixes the round-count reading by hand), disjoint unions;
* invariants: sum(support) = 3 x triangles (node-iterator count), kept edges
  meet K-2, nesting of the (K+1)-truss in the K-truss, label invariance, K=3
  needs at most two rounds, planted cliques survive;
* a second algorithm: sequential truss decomposition (trussness >= K);
* a library: networkx.k_truss, when installed;
* mutation checks: plausible mistakes planted in a copy of the oracle's C
  source make at least one pin fail.
"""
import ctypes
import os
import subprocess
import tempfile
from itertools import combinations

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.brute import ktruss_dense


def run(g, K):
    return oracle.ktruss(g.row_ptr, g.col, K)


def agree_dense(g, K, res=None):
    r = res if res is not None else run(g, K)
    tri = []
    mb, sb, rb = ktruss_dense(g.n, g.row_ptr, g.col, K, tri_out=tri)
    return (np.array_equal(r.mask, mb) and np.array_equal(r.support.astype(np.int64), sb)
            and r.rounds == rb and r.triangles_per_round == tri)


# --------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_small_graphs_match_dense_alg1(n):
    for bits in range(1 << (n * (n - 1) // 2)):
        g = gg.from_bits(n, bits)
        for K in (2, 3, 4, 5, 6):
            assert agree_dense(g, K), (n, bits, K)


def test_exhaustive_n6_matches_dense_alg1():
    n = 6
    for bits in range(1 << 15):
        g = gg.from_bits(n, bits)
        for K in (3, 4):
            assert agree_dense(g, K), (bits, K)


def test_random_graphs_match_dense_alg1():
    for s in range(1000):
        n = 3 + s % 38
        p = (0.05, 0.15, 0.3, 0.5, 0.7, 0.9)[s % 6]
        g = gg.gnp_small(n, p, seed=s)
        for K in (2, 3, 4, 5, 7):
            assert agree_dense(g, K), (s, n, p, K)


# -------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", list(range(3, 26)))
def test_complete_graph_is_n_truss_with_support_n_minus_2(n):
    g = gg.complete(n)
    r = run(g, n)
    assert r.mask.all() and (r.support == n - 2).all()
    assert r.rounds == 1 and r.removed_per_round == [0]
    assert r.triangles == n * (n - 1) * (n - 2) // 6
    assert r.triangles_per_round == [r.triangles]
    r2 = run(g, n + 1)
    assert not r2.mask.any() and not r2.support.any()
    assert r2.rounds == 1 and r2.removed_per_round == [n * (n - 1) // 2]


@pytest.mark.parametrize("t", [1, 2, 3, 7, 70000])
def test_book_graph(t):
    g = gg.book(t)
    r = run(g, 3)
    assert r.mask.all() and r.rounds == 1
    slot01 = 0  # (0,1) is the first slot of row 0
    assert g.col[slot01] == 1
    assert r.support[slot01] == t
    others = np.ones(g.m, bool)
    others[slot01] = False
    assert (r.support[others] == 1).all()
    r4 = run(g, 4)
    assert not r4.mask.any()
    # t >= 2: the spine survives round 1 (support t >= 2) and dies in round 2
    assert r4.rounds == (1 if t == 1 else 2)
    assert r4.triangles_per_round == ([1] if t == 1 else [t, 0])


@pytest.mark.parametrize("leaves", [1, 5, 40])
def test_star_and_tree_have_empty_3truss(leaves):
    for g in (gg.star(leaves), gg.from_edges(leaves + 1, [(i, i + 1) for i in range(leaves)])):
        r = run(g, 3)
        assert not r.mask.any() and r.rounds == 1 and r.triangles == 0


@pytest.mark.parametrize("L", [4, 5, 9, 50])
def test_triangle_strip_round_count(L):
    g = gg.triangle_strip(L)
    r3 = run(g, 3)
    assert r3.mask.all() and r3.rounds == 1
    r4 = run(g, 4)
    # round 1 removes the diagonals and the two end edges, round 2 the rest
    diagonals = L - 2
    assert r4.rounds == 2
    assert r4.removed_per_round == [diagonals + 2, (L - 1) - 2]
    assert r4.triangles_per_round == [L - 2, 0]
    assert not r4.mask.any()


def test_empty_graph_zero_rounds():
    for n in (0, 1, 10):
        r = run(gg.empty(n), 3)
        assert r.rounds == 0 and r.mask.size == 0


def test_k2_keeps_every_edge_with_triangle_counts():
    g = gg.er(300, 3000, seed=5)
    r = run(g, 2)
    assert r.mask.all() and r.rounds == 1
    sup = oracle.edge_support(g.row_ptr, g.col, np.arange(g.m))
    assert np.array_equal(r.support, sup)


def test_disjoint_union_is_per_component():
    parts = [gg.complete(6), gg.triangle_strip(9), gg.er(60, 400, seed=3), gg.book(4)]
    u = gg.disjoint_union(*parts)
    for K in (3, 4, 5, 6):
        ru = run(u, K)
        off_e = 0
        for p in parts:
            rp_ = run(p, K)
            assert np.array_equal(ru.mask[off_e:off_e + p.m], rp_.mask)
            assert np.array_equal(ru.support[off_e:off_e + p.m], rp_.support)
            off_e += p.m


# ---------------------------------------------------------------- invariants

def er_seeds():
    return [gg.er(2000, 16000, seed=s) for s in range(10)]


def test_sum_support_equals_three_triangles():
    graphs = er_seeds() + [gg.rmat(12, 16, seed=s) for s in range(3)]
    for g in graphs:
        for K in (2, 3, 4, 5):
            r = run(g, K)
            t = oracle.triangles(g.row_ptr, g.col, r.mask)
            assert int(r.support.sum()) == 3 * t
            assert r.triangles == t


def test_kept_edges_meet_threshold_and_nesting():
    for g in er_seeds()[:4] + [gg.rmat(13, 16, seed=1)]:
        prev = None
        for K in range(2, 12):
            r = run(g, K)
            assert (r.support[r.mask == 1] >= K - 2).all()
            assert (r.support[r.mask == 0] == 0).all()
            if prev is not None:
                assert not np.any((r.mask == 1) & (prev == 0))
            prev = r.mask


def test_support_is_triangle_count_inside_the_truss():
    g = gg.rmat(12, 16, seed=2)
    for K in (3, 5, 8):
        r = run(g, K)
        q = np.flatnonzero(r.mask)
        sup = oracle.edge_support(g.row_ptr, g.col, q, keep=r.mask)
        assert np.array_equal(r.support[q], sup)


def test_k3_needs_at_most_two_rounds():
    for g in er_seeds()[:3] + [gg.rmat(12, 16, seed=s) for s in range(3)]:
        assert run(g, 3).rounds <= 2


def test_relabel_invariance():
    for g in [gg.rmat(11, 16, seed=0), gg.er(500, 4000, seed=1)]:
        rel_map = gg.relabel_map(g.n, g.row_ptr, g.col)
        e = g.edges()
        new_e = np.sort(rel_map[e], axis=1)
        h = gg.from_edges(g.n, new_e)
        key_h = h.edges()[:, 0] * g.n + h.edges()[:, 1]
        key_g = new_e[:, 0] * g.n + new_e[:, 1]
        idx = np.searchsorted(key_h, key_g)
        assert np.array_equal(key_h[idx], key_g)
        for K in (3, 4, 6):
            rg, rh = run(g, K), run(h, K)
            assert np.array_equal(rg.mask, rh.mask[idx])
            assert np.array_equal(rg.support, rh.support[idx])


def test_planted_cliques_survive_in_their_truss():
    g = gg.rmat(12, 8, seed=4, n_cliques=6, clique_lo=10, clique_hi=30)
    r = run(g, 30)
    assert r.mask.sum() >= 30 * 29 // 2
    assert (r.support[r.mask == 1] >= 28).all()


# --------------------------------------------------- second algorithm, library

def test_truss_decomposition_agrees_with_peeling():
    graphs = er_seeds() + [gg.rmat(12, 16, seed=s) for s in range(2)] + \
        [gg.rmat(12, 16, seed=0, relabel=True), gg.complete(12), gg.book(9)]
    for g in graphs:
        tr = oracle.truss_decomposition(g.row_ptr, g.col)
        kmax = int(tr.max()) if g.m else 2
        for K in range(2, kmax + 2):
            r = run(g, K)
            assert np.array_equal(r.mask, (tr >= K).astype(np.uint8)), K


def test_networkx_k_truss():
    nx = pytest.importorskip("networkx")
    # networkx's k_truss(G, k) keeps edges in >= k-2 triangles: check on K_5
    K5 = nx.complete_graph(5)
    assert nx.k_truss(K5, 5).number_of_edges() == 10
    assert nx.k_truss(K5, 6).number_of_edges() == 0
    for s in range(6):
        g = gg.gnp_small(60, 0.2, seed=100 + s)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(map(tuple, g.edges()))
        for K in (3, 4, 5, 6):
            H = nx.k_truss(G, K)
            want = {tuple(sorted(e)) for e in H.edges()}
            r = run(g, K)
            got = {tuple(e) for e in g.edges()[r.mask == 1]}
            assert got == want, (s, K)


def test_invalid_csr_rejected():
    bad = [
        (np.array([0, 1], np.int32), np.array([0], np.int32)),        # col == row
        (np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32)),  # repeated column
        (np.array([0, 1, 1], np.int32), np.array([5], np.int32)),     # col >= n
        (np.array([0, 2, 1, 2], np.int32), np.array([1, 2], np.int32)),  # decreasing row_ptr
        (np.array([1, 1], np.int32), np.zeros(0, np.int32)),          # row_ptr[0] != 0
    ]
    for rp, c in bad:
        assert oracle.check_csr(rp, c) == oracle.ERR_INVALID
        with pytest.raises(oracle.OracleError):
            oracle.ktruss(rp, c, 3)
    g = gg.complete(4)
    with pytest.raises(oracle.OracleError):
        oracle.ktruss(g.row_ptr, g.col, 1)


# ------------------------------------------------------------ mutation checks

MUTANTS = {
    "drop_kappa_credit": ("S[lslot[y]] += 1;", ""),
    "drop_row_i_credit": ("S[lslot[x]] += 1;", ""),
    "drop_owner_credit": ("S[p] += 1;", ""),
    "threshold_off_by_one": ("S[e] < (int64_t)K - 2", "S[e] <= (int64_t)K - 2"),
    "tail_skips_first": ("int64_t x = a + 1, xe", "int64_t x = a + 2, xe"),
    "merge_advances_wrong_list": ("} else if (cx < cy) {\n                        ++x;",
                                  "} else if (cx < cy) {\n                        ++y;"),
    "stop_after_first_round": ("if (removed == 0) break;", "break;"),
}


def _load_mutant(path):
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.oracle_ktruss.argtypes = [i32, i64, vp, vp, i32, vp, vp, vp, vp, i32, vp, vp]
    lib.oracle_ktruss.restype = ctypes.c_int
    return lib


def _mutant_run(lib, g, K):
    m = g.m
    mask = np.zeros(max(m, 1), np.uint8)
    sup = np.zeros(max(m, 1), np.int32)
    rounds = ctypes.c_int32(0)
    removed = np.zeros(256, np.int64)
    tris = np.zeros(256, np.int64)
    tri = ctypes.c_int64(0)
    rp = np.ascontiguousarray(g.row_ptr)
    col = np.ascontiguousarray(g.col)
    rc = lib.oracle_ktruss(g.n, m, rp.ctypes.data, col.ctypes.data if m else None, K,
                           mask.ctypes.data, sup.ctypes.data, ctypes.addressof(rounds),
                           removed.ctypes.data, 256, ctypes.addressof(tri), tris.ctypes.data)
    assert rc == 0
    return oracle.KtrussResult(mask[:m], sup[:m], rounds.value,
                               [int(x) for x in removed[:rounds.value]], tri.value,
                               [int(x) for x in tris[:rounds.value]])


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "mut.so")
        with open(c, "w") as f:
            f.write(src.replace(old, new, 1))
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, c])
        lib = _load_mutant(so)
        caught = False
        cases = [(gg.complete(7), 7), (gg.triangle_strip(9), 4), (gg.book(5), 3)]
        cases += [(gg.gnp_small(12 + s, 0.5, seed=s), K) for s in range(30) for K in (3, 4, 5)]
        for g, K in cases:
            if not agree_dense(g, K, _mutant_run(lib, g, K)):
                caught = True
                break
        assert caught, f"mutant {name} passed every pin"


# ------------------------------------------- closed forms of the checkers

@pytest.mark.parametrize("n", [3, 4, 7, 15])
def test_checkers_on_complete_graph(n):
    g = gg.complete(n)
    assert (oracle.truss_decomposition(g.row_ptr, g.col) == n).all()
    assert oracle.triangles(g.row_ptr, g.col) == n * (n - 1) * (n - 2) // 6
    assert (oracle.edge_support(g.row_ptr, g.col, np.arange(g.m)) == n - 2).all()


def test_checkers_on_book_star_strip():
    b = gg.book(6)
    assert (oracle.truss_decomposition(b.row_ptr, b.col) == 3).all()
    assert oracle.triangles(b.row_ptr, b.col) == 6
    s = gg.star(9)
    assert (oracle.truss_decomposition(s.row_ptr, s.col) == 2).all()
    assert oracle.triangles(s.row_ptr, s.col) == 0
    t = gg.triangle_strip(10)
    assert oracle.triangles(t.row_ptr, t.col) == 8
    assert (oracle.truss_decomposition(t.row_ptr, t.col) == 3).all()
    # a kept-edge mask removes exactly the triangles that lose an edge
    keep = np.ones(t.m, np.uint8)
    keep[0] = 0  # edge (0,1) is in one triangle
    assert oracle.triangles(t.row_ptr, t.col, keep) == 7


def test_tail_start_reading():
    """Reading of Alg. 3: its first update intersects the whole a12 with row
    kappa, the other two only the tail a12(j+1:).  Both give the same matches
    because row kappa holds only columns > kappa.  An oracle whose merge starts
    at the edge itself (not after it) must therefore agree exactly."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old = "int64_t x = a + 1, xe"
    assert old in src
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "variant.c")
        so = os.path.join(d, "variant.so")
        with open(c, "w") as f:
            f.write(src.replace(old, "int64_t x = lstart[i], xe", 1))
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, c])
        lib = _load_mutant(so)
        for s in range(40):
            g = gg.gnp_small(10 + s % 25, 0.45, seed=700 + s)
            for K in (2, 3, 4, 5):
                a, b = run(g, K), _mutant_run(lib, g, K)
                assert np.array_equal(a.mask, b.mask) and np.array_equal(a.support, b.support)
                assert a.rounds == b.rounds


@pytest.mark.parametrize("name", ["rmat20", "rmat20r", "rmat23c"])
def test_decomposition_agrees_with_peeling_on_rmat20(name):
    """At full size (R-MAT-20, original ids and relabelled; R-MAT-23 with
    planted cliques) the oracle's two algorithms agree: the stored Alg. 1
    results (every stored K) keep exactly the edges whose trussness, from the
    stored sequential-peeling decomposition, is at least K; both were taken on
    the same graph."""
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    p = os.path.join(here, f"{name}_trussness.json")
    if not os.path.exists(p):
        pytest.skip(f"no stored oracle decomposition for {name}")
    with open(p) as f:
        dec = json.load(f)
    with open(os.path.join(here, f"{name}.json")) as f:
        cases = [c for c in json.load(f)["cases"] if c["seed"] == dec["seed"]]
    assert cases and all(c["graph_sha256"] == dec["graph_sha256"] for c in cases)
    hist = {int(k): v for k, v in dec["edges_per_trussness"].items()}
    assert sum(hist.values()) == dec["m"] and max(hist) == dec["kmax"]
    for c in cases:
        assert c["edges_out"] == sum(v for t, v in hist.items() if t >= c["K"]), c["K"]


# ---------------------------------------------- multi-core CPU baseline (CPU-F)

def test_cpu_f_matches_oracle():
    """The paper's fine-grained CPU design (per-edge tasks with atomic
    supports on several threads, zero-terminated rows) gives the oracle's
    masks, supports and round counts."""
    graphs = er_seeds()[:3] + [gg.rmat(12, 16, seed=s) for s in range(2)] + \
        [gg.rmat(12, 16, seed=0, relabel=True), gg.complete(12), gg.book(30), gg.star(9),
         gg.triangle_strip(40), gg.empty(4)]
    for g in graphs:
        for K in (2, 3, 4, 6):
            a = run(g, K)
            for threads in (1, 4):
                b = oracle.cpu_f_ktruss(g.row_ptr, g.col, K, threads)
                assert np.array_equal(a.mask, b.mask) and np.array_equal(a.support, b.support)
                assert a.rounds == b.rounds


def test_golden_relabel_route_matches_direct():
    """tests/golden/make_golden.py --relabel runs the oracle on the
    degree-relabelled isomorphic copy of a graph and reads each edge's outputs
    at its slot there.  The K-truss is defined on the undirected graph (Sec. I),
    so masks, supports, rounds, per-round removals and triangles must equal a
    direct run on the loaded numbering, edge by edge in input order."""
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    for g in (gg.rmat(12, 16, 1), gg.er(2000, 16000, 2),
              gg.rmat(11, 8, seed=4, n_cliques=6, clique_lo=10, clique_hi=30)):
        h, slot = mg.relabelled_slots(g)
        assert sorted(slot.tolist()) == list(range(g.m))
        for K in (3, 4, 6):
            r0 = oracle.ktruss(g.row_ptr, g.col, K)
            r1 = oracle.ktruss(h.row_ptr, h.col, K)
            assert np.array_equal(r0.mask, r1.mask[slot]), K
            assert np.array_equal(r0.support, r1.support[slot]), K
            assert r0.rounds == r1.rounds and list(r0.removed_per_round) == list(r1.removed_per_round)
            assert r0.triangles == r1.triangles
