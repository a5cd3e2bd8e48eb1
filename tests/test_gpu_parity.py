"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

All arithmetic is integer, so masks, supports and per-round statistics must be
identical (tolerance 0).  Small and mid-size graphs are compared element by
element with a live oracle run; the full-size R-MAT workloads are compared
against stored oracle digests and, where no digest exists, on sampled edges
the oracle computes one at a time plus size-independent properties.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
KERNELS = [0, 1, 2, 3]  # balanced, thread-per-edge, coarse (thread-per-row), auto
UPDATES = [0, 1, 2]     # recompute every round, decremental update always, auto


@pytest.fixture(scope="module")
def kt():
    import torch
    import paper_2009_07929_gb300 as kt
    kt.lib()
    torch.cuda.init()
    return kt


def gpu_run(kt, g, K, kernel=0, host=False, update=None):
    import torch
    if host:
        h = kt.load(g.row_ptr, g.col)
    else:
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    h.set_kernel(kernel)
    if update is not None:
        h.set_update(update)
    if host:
        mask, sup = h.run_host(K)
    else:
        m_t, s_t = h.run(K)
        torch.cuda.current_stream().synchronize()
        mask, sup = m_t.cpu().numpy(), s_t.cpu().numpy()
    st = h.stats()
    h.close()
    return mask, sup, st


def assert_parity(kt, g, K, kernel=0, host=False, update=None):
    r = oracle.ktruss(g.row_ptr, g.col, K)
    mask, sup, st = gpu_run(kt, g, K, kernel, host, update)
    where = f"(K={K}, kernel={kernel}, update={update})"
    assert np.array_equal(mask, r.mask), f"mask differs {where}"
    assert np.array_equal(sup, r.support), f"support differs {where}"
    assert st.rounds == r.rounds, where
    assert st.removed_per_round == r.removed_per_round, where
    assert st.triangles_per_round == r.triangles_per_round, where
    assert st.triangles_out == r.triangles
    assert st.edges_out == int(r.mask.sum())
    # the first round always runs the support step; under UPDATE_NEVER every
    # round does, under UPDATE_ALWAYS every later round is an update
    assert len(st.updated_per_round) == st.rounds
    if st.rounds:
        assert st.updated_per_round[0] == 0
        assert st.support_launches == st.rounds - sum(st.updated_per_round)
    if update == 0:
        assert not any(st.updated_per_round)
    if update == 1:
        assert all(st.updated_per_round[1:])
    return r, st


# ---------------------------------------------- decremental support update
# Every mode must give the recomputation's results round by round.

@pytest.mark.parametrize("update", UPDATES)
@pytest.mark.parametrize("seed", range(10))
def test_er2000_update_modes(kt, seed, update):
    g = gg.workload("er2000", seed)
    for K in (3, 4, 5):
        assert_parity(kt, g, K, 3, update=update)


@pytest.mark.parametrize("update", UPDATES)
def test_update_modes_on_small_and_structured_graphs(kt, update):
    cases = [gg.empty(0), gg.empty(17), gg.from_edges(2, [(0, 1)]), gg.star(50),
             gg.triangle_strip(4), gg.triangle_strip(101), gg.complete(3), gg.complete(33),
             gg.book(7), gg.book(70000)]
    for g in cases:
        for K in (2, 3, 4, 5, 34):
            assert_parity(kt, g, K, 3, update=update)
    for s in range(60):
        g = gg.gnp_small(5 + s % 36, (0.1, 0.3, 0.6, 0.9)[s % 4], seed=2000 + s)
        for K in (3, 4, 6):
            assert_parity(kt, g, K, 3, update=update)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("update", [1, 2])
def test_update_modes_on_deep_cascades_and_long_rows(kt, update, kernel):
    for g, K, rounds in deep_cascade_graphs():
        assert_parity(kt, g, K, kernel, update=update)
    L = 20000
    edges = [(0, j) for j in range(1, L + 1)]
    edges += [(j, j + 1) for j in range(1, L)] + [(j, j + 7) for j in range(1, L - 7, 3)]
    g = gg.from_edges(L + 1, edges)
    for K in (3, 4, 5):
        assert_parity(kt, g, K, kernel, update=update)


@pytest.mark.parametrize("update", UPDATES)
def test_update_modes_on_rmat(kt, update):
    for scale, seed in ((12, 0), (14, 1), (16, 2)):
        g = gg.rmat(scale, 16, seed)
        for K in (3, 4, 7, 12):
            assert_parity(kt, g, K, 3, update=update)
    g = gg.rmat(14, 8, seed=3, n_cliques=8, clique_lo=20, clique_hi=60)
    for K in (5, 12, 30):
        assert_parity(kt, g, K, 3, update=update)


# ---------------------------------------------------------------- config 1

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("seed", range(10))
def test_er2000_all_seeds(kt, seed, kernel):
    g = gg.workload("er2000", seed)
    for K in (3, 4, 5):
        assert_parity(kt, g, K, kernel)


# --------------------------------------------------------------- edge cases

@pytest.mark.parametrize("kernel", KERNELS)
def test_degenerate_graphs(kt, kernel):
    cases = [gg.empty(0), gg.empty(1), gg.empty(17), gg.from_edges(2, [(0, 1)]), gg.star(50),
             gg.triangle_strip(4), gg.triangle_strip(101), gg.complete(3)]
    for g in cases:
        for K in (2, 3, 4, 5):
            assert_parity(kt, g, K, kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_complete_graphs(kt, kernel):
    for n in (4, 5, 17, 33, 64, 130):
        g = gg.complete(n)
        r, st = assert_parity(kt, g, n, kernel)
        assert st.rounds == 1 and r.mask.all()
        assert_parity(kt, g, n + 1, kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_book_graph_support_above_uint16(kt, kernel):
    g = gg.book(70000)
    r, _ = assert_parity(kt, g, 3, kernel)
    assert r.support[0] == 70000
    assert_parity(kt, g, 4, kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_row_longer_than_any_stage(kt, kernel):
    # vertex 0 adjacent to 1..L, plus a path and chords among its neighbours,
    # so row 0 is far longer than a shared-memory stage and carries triangles
    L = 20000
    edges = [(0, j) for j in range(1, L + 1)]
    edges += [(j, j + 1) for j in range(1, L)] + [(j, j + 7) for j in range(1, L - 7, 3)]
    g = gg.from_edges(L + 1, edges)
    for K in (3, 4, 5):
        assert_parity(kt, g, K, kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_random_small_graphs(kt, kernel):
    for s in range(60):
        g = gg.gnp_small(5 + s % 36, (0.1, 0.3, 0.6, 0.9)[s % 4], seed=1000 + s)
        for K in (2, 3, 4, 6):
            assert_parity(kt, g, K, kernel)


def deep_cascade_graphs(count=6):
    """Seeded search over small random graphs keeping those whose peeling runs
    the most bulk rounds (the oracle decides)."""
    best = []
    for s in range(400):
        g = gg.gnp_small(30, 0.25, seed=5000 + s)
        for K in (4, 5):
            r = oracle.ktruss(g.row_ptr, g.col, K)
            best.append((r.rounds, s, K))
    best.sort(reverse=True)
    return [(gg.gnp_small(30, 0.25, seed=5000 + s), K, rounds) for rounds, s, K in best[:count]]


@pytest.mark.parametrize("kernel", KERNELS)
def test_deep_cascades(kt, kernel):
    for g, K, rounds in deep_cascade_graphs():
        assert rounds >= 3
        assert_parity(kt, g, K, kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_small_rmat_with_long_rows(kt, kernel):
    for scale, seed in ((12, 0), (14, 1), (16, 2)):
        g = gg.rmat(scale, 16, seed)
        assert np.diff(g.row_ptr).max() > 4096 or scale < 16
        for K in (3, 4, 7, 12):
            assert_parity(kt, g, K, kernel)


def test_long_rows_at_slots_above_2_30(kt):
    """Disjoint copies of a graph whose hub row is longer than a shared-memory
    stage, enough of them that the last copies' rows sit at CSR slots above
    2^30: searches over slot positions must not wrap there.  Every copy must
    get the oracle's result for one copy."""
    import torch
    L = 20000
    edges = [(0, j) for j in range(1, L + 1)]
    edges += [(j, j + 1) for j in range(1, L)] + [(j, j + 7) for j in range(1, L - 7, 3)]
    base = gg.from_edges(L + 1, edges)
    copies = (1 << 30) // base.m + 64
    n, m = base.n * copies, base.m * copies
    assert m > (1 << 30) + 32 * base.m and n < (1 << 31)
    rp = np.empty(n + 1, np.int32)
    rp[:n] = (base.row_ptr[:-1][None, :] +
              (np.arange(copies, dtype=np.int32) * np.int32(base.m))[:, None]).ravel()
    rp[n] = m
    col = (base.col[None, :] + (np.arange(copies, dtype=np.int32) * np.int32(base.n))[:, None]).ravel()
    h = kt.load(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda())
    del rp, col
    h.set_kernel(0)  # balanced: long rows go through the piecewise path
    for K in (3, 4):
        r = oracle.ktruss(base.row_ptr, base.col, K)
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        mask = m_t.cpu().numpy().reshape(copies, base.m)
        sup = s_t.cpu().numpy().reshape(copies, base.m)
        del m_t, s_t
        assert (mask == r.mask[None, :]).all(), K
        assert (sup == r.support[None, :]).all(), K
        assert h.stats().rounds == r.rounds
    h.close()
    torch.cuda.empty_cache()


def test_rmat_with_cliques_kmax(kt):
    g = gg.rmat(14, 8, seed=3, n_cliques=8, clique_lo=20, clique_hi=60)
    tr = oracle.truss_decomposition(g.row_ptr, g.col)
    kmax = int(tr.max())
    for K in (3, kmax - 1, kmax, kmax + 1):
        assert_parity(kt, g, K)


def test_relabel_variant_same_truss(kt):
    g = gg.rmat(13, 16, 5)
    h = gg.rmat(13, 16, 5, relabel=True)
    rel = gg.relabel_map(g.n, g.row_ptr, g.col)
    new_e = np.sort(rel[g.edges()], axis=1)
    key_h = h.edges()[:, 0] * g.n + h.edges()[:, 1]
    idx = np.searchsorted(key_h, new_e[:, 0] * g.n + new_e[:, 1])
    for K in (3, 5, 9):
        mg, sg, _ = gpu_run(kt, g, K)
        mh, sh, _ = gpu_run(kt, h, K)
        assert np.array_equal(mg, mh[idx]) and np.array_equal(sg, sh[idx])


def test_host_kind_buffers_match_device_kind(kt):
    g = gg.rmat(14, 16, 7)
    for K in (3, 6):
        assert_parity(kt, g, K, host=True)


def test_several_K_on_one_handle(kt):
    import torch
    g = gg.rmat(14, 16, 8)
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    prev = None
    for K in (9, 3, 5, 3, 12):
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        r = oracle.ktruss(g.row_ptr, g.col, K)
        assert np.array_equal(m_t.cpu().numpy(), r.mask)
        assert np.array_equal(s_t.cpu().numpy(), r.support)
        assert h.stats().rounds == r.rounds
    h.close()


def test_support_optional(kt):
    import torch
    g = gg.er(2000, 16000, 3)
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    mask, sup = h.run(3, support=False)
    torch.cuda.synchronize()
    assert sup is None
    assert np.array_equal(mask.cpu().numpy(), oracle.ktruss(g.row_ptr, g.col, 3).mask)
    h.close()


# ------------------------------------------------ device block cache

def test_freed_blocks_are_reused_and_trimmed(kt):
    import torch
    g = gg.rmat(15, 16, 1)
    r = oracle.ktruss(g.row_ptr, g.col, 4)
    kt.trim_cache()
    torch.cuda.synchronize()
    for cycle in range(3):  # load-run-free cycles reuse the cached block
        h = kt.load(g.row_ptr, g.col)  # host arrays: no torch allocation
        mask, sup = h.run_host(4)
        assert np.array_equal(mask, r.mask) and np.array_equal(sup, r.support), cycle
        h.close()
    held = torch.cuda.mem_get_info()[0]
    kt.trim_cache()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] > held  # the cached blocks were freed


# ------------------------------------------------ tracing

def test_trace_prints_one_line_per_round():
    import subprocess
    import sys
    code = ("import graphgen as gg, paper_2009_07929_gb300 as kt\n"
            "g = gg.triangle_strip(60)\n"
            "h = kt.load(g.row_ptr, g.col)\n"
            "h.run_host(4)\n"
            "print(h.stats().rounds)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, KTRUSS_TRACE="1")
    p = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    rounds = int(p.stdout.strip().splitlines()[-1])
    lines = [l for l in p.stderr.splitlines() if l.startswith("[ktruss run] round ")]
    assert rounds == 2 and len(lines) == rounds
    assert "round 1 live 117 removed 60" in lines[0]


# ------------------------------------------------ autotuner

def test_autotune_picks_candidates_and_keeps_results(kt):
    import torch
    for g, K in ((gg.rmat(14, 16, 4), 4), (gg.er(20000, 300000, 2), 3)):
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        t = h.autotune(K, reps=1)
        assert t["light_merge"] in (0, 32, 64, 128, 256)
        assert t["small_edges"] in (1 << 15, 1 << 17, 1 << 19, 1 << 21)
        assert t["update_mode"] in (0, 1, 2) and t["trials"] >= 10 and t["ms"] > 0
        assert t["support_shape"] in (0, 1)
        r = oracle.ktruss(g.row_ptr, g.col, K)
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        assert np.array_equal(m_t.cpu().numpy(), r.mask)
        assert np.array_equal(s_t.cpu().numpy(), r.support)
        assert h.stats().rounds == r.rounds
        h.close()


@pytest.mark.parametrize("shape", [0, 1])
def test_support_shapes(kt, shape):
    """Both CTA shapes of the balanced support kernel (1024 threads with
    8192-slot stages; 512 threads, three per SM, with 2048-slot stages) give
    the oracle's results, on graphs whose staged rows are shorter than a
    stage, longer than a 2048-slot stage, and longer than an 8192-slot one."""
    import torch
    L = 20000
    edges = [(0, j) for j in range(1, L + 1)]
    edges += [(j, j + 1) for j in range(1, L)] + [(j, j + 7) for j in range(1, L - 7, 3)]
    cases = [(gg.rmat(12, 16, 0), (3, 4)), (gg.rmat(16, 16, 2), (3, 5)),
             (gg.rmat(14, 16, 1, relabel=True), (3, 4)), (gg.from_edges(L + 1, edges), (3, 4)),
             (gg.book(70000), (3,)), (gg.workload("er2000", 1), (3, 4)),
             (gg.rmat(14, 8, seed=3, n_cliques=8, clique_lo=20, clique_hi=60), (3, 20))]
    for g, Ks in cases:
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        h.set_kernel(0)
        h.set_support_shape(shape)
        for K in Ks:
            r = oracle.ktruss(g.row_ptr, g.col, K)
            m_t, s_t = h.run(K)
            torch.cuda.synchronize()
            st = h.stats()
            assert np.array_equal(m_t.cpu().numpy(), r.mask), (shape, K)
            assert np.array_equal(s_t.cpu().numpy(), r.support), (shape, K)
            assert st.rounds == r.rounds and st.triangles_per_round == r.triangles_per_round
        h.close()


@pytest.mark.parametrize("light", [0, 16, 256, 1024])
def test_light_merge_thresholds(kt, light):
    import torch
    for g, K in ((gg.rmat(13, 16, 6), 5), (gg.er(4000, 60000, 3), 3), (gg.book(300), 3)):
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        h.set_kernel(0)
        h.set_option(kt.OPT_LIGHT_MERGE, light)
        r = oracle.ktruss(g.row_ptr, g.col, K)
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        assert np.array_equal(m_t.cpu().numpy(), r.mask)
        assert np.array_equal(s_t.cpu().numpy(), r.support)
        h.close()


# ------------------------------------------------ truss decomposition

@pytest.mark.parametrize("kernel,update", [(k, None) for k in KERNELS] + [(3, u) for u in UPDATES])
def test_decomposition_matches_oracle(kt, kernel, update):
    import torch
    graphs = [gg.complete(9), gg.book(20), gg.star(10), gg.triangle_strip(30), gg.empty(5),
              gg.er(2000, 16000, 1), gg.rmat(12, 16, 0),
              gg.rmat(14, 8, seed=3, n_cliques=8, clique_lo=20, clique_hi=60)]
    for g in graphs:
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        h.set_kernel(kernel)
        if update is not None:
            h.set_update(update)
        tr, kmax = h.decompose()
        torch.cuda.synchronize()
        got = tr.cpu().numpy()
        want = oracle.truss_decomposition(g.row_ptr, g.col)
        assert np.array_equal(got, want)
        assert kmax == (int(want.max()) if g.m else 0)
        # the K-truss of ktruss_run is {e : trussness >= K}
        for K in {3, max(3, kmax), max(3, kmax + 1)}:
            m_t, _ = h.run(K)
            torch.cuda.synchronize()
            assert np.array_equal(m_t.cpu().numpy(), (got >= K).astype(np.uint8))
        h.close()


# ---------------------------------------------------------------- errors

def test_malformed_csr_rejected_on_device(kt):
    import torch
    bad = [
        (np.array([0, 1], np.int32), np.array([0], np.int32)),
        (np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32)),
        (np.array([0, 1, 1], np.int32), np.array([5], np.int32)),
        (np.array([0, 2, 1, 2], np.int32), np.array([1, 2], np.int32)),
        (np.array([1, 1], np.int32), np.zeros(1, np.int32)[:0]),
        (np.array([0, 0, 3], np.int32), np.array([1, 2, 3], np.int32)),
    ]
    for rp, c in bad:
        for dev in (False, True):
            a = torch.from_numpy(rp).cuda() if dev else rp
            b = torch.from_numpy(c).cuda() if dev else c
            with pytest.raises(kt.KtrussError) as ei:
                kt.load(a, b)
            assert ei.value.code == kt.EINVAL


def test_k_below_two_rejected(kt):
    import torch
    g = gg.complete(5)
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    with pytest.raises(kt.KtrussError) as ei:
        h.run(1)
    assert ei.value.code == kt.EINVAL
    h.close()


def test_injected_allocation_failure(kt, monkeypatch):
    g = gg.complete(6)
    for budget in ("0", "3", "12"):
        monkeypatch.setenv("KTRUSS_TEST_FAIL_ALLOC", budget)
        with pytest.raises(kt.KtrussError) as ei:
            kt.load(g.row_ptr, g.col)
        assert ei.value.code == kt.ENOMEM
    monkeypatch.delenv("KTRUSS_TEST_FAIL_ALLOC")
    assert_parity(kt, g, 6)


# -------------------------------------------- full-size workloads (digests)

def sha(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()


def golden_cases(name):
    p = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(p):
        return []
    with open(p) as f:
        return json.load(f)["cases"]


def graph_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("name", ["rmat20", "rmat20r", "rmat23c"])
def test_full_size_against_oracle_digests(kt, name):
    cases = golden_cases(name)
    if not cases:
        pytest.skip(f"no stored oracle digests for {name}")
    import torch
    by_seed = {}
    for c in cases:
        by_seed.setdefault(c["seed"], []).append(c)
    for seed, cs in sorted(by_seed.items()):
        g = gg.workload(name, seed)
        assert graph_digest(g) == cs[0]["graph_sha256"], "generator output changed"
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        # the default CTA shape of the support kernel for every case, and the
        # other shape for the first case of each graph
        for shape, c in [(None, c) for c in cs] + [(0, cs[0])]:
            if shape is not None:
                h.set_support_shape(shape)
            m_t, s_t = h.run(c["K"])
            torch.cuda.synchronize()
            st = h.stats()
            mask = m_t.cpu().numpy()
            sup = np.ascontiguousarray(s_t.cpu().numpy(), dtype="<i4")
            assert st.rounds == c["rounds"], c
            assert st.removed_per_round == c["removed_per_round"], c
            assert st.edges_out == c["edges_out"] and st.triangles_out == c["triangles_out"]
            assert int(sup.astype(np.int64).sum()) == c["support_sum"]
            assert sha(mask) == c["mask_sha256"] and sha(sup) == c["support_sha256"]
        h.close()


@pytest.mark.parametrize("name", ["rmat20", "rmat20r", "rmat23c"])
def test_full_size_decomposition_against_oracle(kt, name):
    """ktruss_decompose (K = 3, 4, ... up to K_max, each K from the previous
    truss) of the full R-MAT-20 graph, original ids and degree-relabelled, and
    of R-MAT-23 with planted cliques, against the oracle's truss decomposition
    by its second, independent algorithm (sequential peeling; stored by
    tests/golden/make_golden.py): every edge's trussness, hence the K-truss
    for every K at once."""
    p = os.path.join(GOLDEN, f"{name}_trussness.json")
    if not os.path.exists(p):
        pytest.skip(f"no stored oracle decomposition for {name}")
    with open(p) as f:
        c = json.load(f)
    import torch
    g = gg.cached_workload(name, c["seed"])
    assert graph_digest(g) == c["graph_sha256"], "generator output changed"
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    tr_t, kmax = h.decompose()
    torch.cuda.synchronize()
    tr = np.ascontiguousarray(tr_t.cpu().numpy(), dtype="<i4")
    h.close()
    assert kmax == c["kmax"]
    hist = np.bincount(tr)
    assert {str(k): int(v) for k, v in enumerate(hist) if v} == c["edges_per_trussness"]
    assert sha(tr) == c["trussness_sha256"]


def test_rmat23_cliques_k3_sampled_and_kmax_sweep(kt):
    """Config 3 at full size: K=3 checked on sampled edges against per-edge
    oracle supports (for K=3 the kept edges are exactly those in a triangle and
    keep their full-graph support); then a ladder of K up to the largest
    non-empty truss (from the decomposition) and one past it, checking
    size-independent properties at every K and sampled supports inside the
    truss for a few K."""
    import torch
    g = gg.cached_workload("rmat23c", 0)
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    tr_t, kmax_dec = h.decompose()
    torch.cuda.synchronize()
    tr = tr_t.cpu().numpy()
    # when the oracle's decomposition of this graph is stored, the trussness
    # every rung below is checked against is the oracle's, element by element
    p = os.path.join(GOLDEN, "rmat23c_trussness.json")
    if os.path.exists(p):
        with open(p) as f:
            dec = json.load(f)
        assert dec["graph_sha256"] == graph_digest(g)
        assert sha(np.ascontiguousarray(tr, dtype="<i4")) == dec["trussness_sha256"]
        assert kmax_dec == dec["kmax"]
    rng = np.random.default_rng(0)
    m_t, s_t = h.run(3)
    torch.cuda.synchronize()
    mask3, sup3 = m_t.cpu().numpy(), s_t.cpu().numpy()
    st = h.stats()
    assert st.rounds <= 2
    q = np.unique(np.concatenate([rng.integers(0, g.m, 4000), np.arange(2000),
                                  np.flatnonzero(np.diff(g.row_ptr) > 0)[:500]]))
    q = q[q < g.m]
    full = oracle.edge_support(g.row_ptr, g.col, q)
    assert np.array_equal(sup3[q], full)
    assert np.array_equal(mask3[q], (full >= 1).astype(np.uint8))
    assert int(sup3.astype(np.int64).sum()) == 3 * st.triangles_out
    assert np.array_equal(mask3, (tr >= 3).astype(np.uint8))
    # a 200-clique was planted, so the 200-truss is non-empty
    assert kmax_dec >= 200 and (tr == kmax_dec).any() and not (tr > kmax_dec).any()
    ladder = sorted({4, 5, 6, 8, 12, 20, 50, 100, 200, (200 + kmax_dec) // 2, kmax_dec,
                     kmax_dec + 1})
    prev = mask3
    for K in ladder:
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        mask, sup = m_t.cpu().numpy(), s_t.cpu().numpy()
        st = h.stats()
        if K > kmax_dec:
            assert not mask.any() and not sup.any()
            continue
        assert np.array_equal(mask, (tr >= K).astype(np.uint8))
        assert (sup[mask == 1] >= K - 2).all() and (sup[mask == 0] == 0).all()
        assert not np.any((mask == 1) & (prev == 0))
        assert int(sup.astype(np.int64).sum()) == 3 * st.triangles_out
        if K in (6, 100, 200, kmax_dec) or mask.sum() < 50000:
            kept = np.flatnonzero(mask)
            qs = kept if kept.size <= 3000 else rng.choice(kept, 3000, replace=False)
            assert np.array_equal(sup[qs], oracle.edge_support(g.row_ptr, g.col, qs, keep=mask))
        prev = mask
    h.close()


def test_host_work_count_equals_library_merge_work(kt):
    """The benchmark's host count of the merge work W (sum over edges of the
    tail length plus the row-kappa length, from the CSR alone) equals the merge
    work the library reports for the first support step: on the loaded
    numbering with KTRUSS_OPT_REORDER off, and on the degree-ordered relabel
    (the generators' relabel of the same edges) with it on."""
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    for g in (gg.rmat(14, 16, seed=0), gg.rmat(12, 16, seed=1, relabel=True),
              gg.workload("er2000", 0), gg.book(50)):
        r = gg.from_edges(g.n, g.edges(), relabel=True)
        for reorder, ref in ((False, g), (True, r)):
            h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
            h.set_kernel(0)
            h.set_reorder(reorder)
            h.run(3)
            torch.cuda.synchronize()
            st = h.stats()
            h.close()
            assert st.merge_work_per_round[0] == bench.support_work(ref.row_ptr, ref.col)["W"]


@pytest.mark.parametrize("kernel", [0, 1, 3])
def test_reorder_on_and_off_match_oracle(kt, kernel):
    """Runs from the degree-ordered relabel made at load (default) and from
    the loaded numbering give the oracle's masks, supports and per-round
    statistics in input edge order."""
    import torch
    cases = [gg.rmat(14, 16, 2), gg.rmat(12, 8, seed=4, n_cliques=6, clique_lo=10, clique_hi=30),
             gg.workload("er2000", 5), gg.book(300), gg.star(40), gg.complete(20), gg.empty(9),
             gg.triangle_strip(50), gg.from_edges(2, [(0, 1)])]
    for g in cases:
        for K in (3, 4, 7):
            r = oracle.ktruss(g.row_ptr, g.col, K)
            for reorder in (True, False):
                h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
                h.set_kernel(kernel)
                h.set_reorder(reorder)
                m_t, s_t = h.run(K)
                torch.cuda.synchronize()
                st = h.stats()
                tr, kmax = h.decompose()
                torch.cuda.synchronize()
                h.close()
                where = (K, reorder, kernel)
                assert np.array_equal(m_t.cpu().numpy(), r.mask), where
                assert np.array_equal(s_t.cpu().numpy(), r.support), where
                assert st.rounds == r.rounds and st.removed_per_round == r.removed_per_round
                assert st.triangles_per_round == r.triangles_per_round, where
                assert np.array_equal(tr.cpu().numpy(), oracle.truss_decomposition(g.row_ptr, g.col))


def test_relabel_rows_longer_than_on_chip_sort(kt):
    """The relabel at load sorts rows of up to 1024 columns on chip and the
    longer ones through one radix-sorted list.  Two planted cliques of 1100
    and 1300 vertices in an R-MAT graph leave 350 relabelled rows above that
    size: the runs from the relabel equal the oracle (K = 3 and K = 1100), and
    the complete graph K_1100 (rows up to 1099) gives its closed form: every
    edge in K_1100 - 2 = 1098 triangles, the whole graph the 1100-truss and
    none of it the 1101-truss."""
    import torch
    g = gg.rmat(12, 8, seed=3, n_cliques=2, clique_lo=1100, clique_hi=1300)
    for K in (3, 1100):
        r = oracle.ktruss(g.row_ptr, g.col, K)
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        st = h.stats()
        h.close()
        assert np.array_equal(m_t.cpu().numpy(), r.mask), K
        assert np.array_equal(s_t.cpu().numpy(), r.support), K
        assert st.rounds == r.rounds and st.removed_per_round == r.removed_per_round, K
    kn = gg.complete(1100)
    h = kt.load(torch.from_numpy(kn.row_ptr).cuda(), torch.from_numpy(kn.col).cuda())
    m_t, s_t = h.run(1100)
    torch.cuda.synchronize()
    assert bool((m_t == 1).all()) and bool((s_t == 1098).all())
    m_t, s_t = h.run(1101)
    torch.cuda.synchronize()
    assert bool((m_t == 0).all()) and bool((s_t == 0).all())
    h.close()


# ------------------------------------------------ device-driven round loop

def _run_loop(kt, g, K, loop, update):
    import torch
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    h.set_device_loop(loop)
    h.set_update(update)
    m_t, s_t = h.run(K)
    torch.cuda.synchronize()
    st = h.stats()
    out = (m_t.cpu().numpy(), s_t.cpu().numpy(), st)
    h.close()
    return out


@pytest.mark.parametrize("update", [1, 2])
def test_device_loop_rounds_match_oracle(kt, update):
    """Rounds whose supports come from the decremental update run in the
    device-driven loop (one CUDA graph launch with conditional nodes, no host
    synchronisation per round).  Masks, supports and every per-round statistic
    equal the oracle's, with the loop on and off."""
    cases = [(g, K) for g, K, _ in deep_cascade_graphs()]
    cases += [(gg.triangle_strip(101), 4), (gg.rmat(14, 16, 1), 4), (gg.rmat(14, 16, 1), 8),
              (gg.rmat(12, 8, seed=4, n_cliques=6, clique_lo=10, clique_hi=30), 12),
              (gg.workload("er2000", 3), 4)]
    for g, K in cases:
        r = oracle.ktruss(g.row_ptr, g.col, K)
        for loop in (True, False):
            mask, sup, st = _run_loop(kt, g, K, loop, update)
            where = f"(K={K}, loop={loop}, update={update})"
            assert np.array_equal(mask, r.mask), where
            assert np.array_equal(sup, r.support), where
            assert st.rounds == r.rounds, where
            assert st.removed_per_round == r.removed_per_round, where
            assert st.triangles_per_round == r.triangles_per_round, where
            assert st.triangles_out == r.triangles and st.edges_out == int(r.mask.sum())
            if not loop:
                assert st.device_loop_rounds == 0 and st.device_loop_launches == 0
            elif update == 1 and r.rounds >= 2:
                # round 1 runs the support step on the host; every later
                # round takes its supports from the update, on the device
                assert st.device_loop_rounds == r.rounds - 1, where
                assert st.device_loop_launches >= 1


@pytest.mark.parametrize("update", [1, 2])
def test_device_loop_decomposition(kt, update):
    """The K sweep in the device-driven loop (a round that removes nothing
    raises K on the same graph) gives the oracle's trussness and the host
    loop's per-round statistics."""
    import torch
    graphs = [gg.rmat(14, 8, seed=3, n_cliques=8, clique_lo=20, clique_hi=60),
              gg.triangle_strip(60), gg.er(2000, 16000, 1), gg.book(20), gg.complete(12),
              gg.rmat(13, 16, seed=5)]
    for g in graphs:
        want = oracle.truss_decomposition(g.row_ptr, g.col)
        stats = []
        for loop in (True, False):
            h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
            h.set_device_loop(loop)
            h.set_update(update)
            tr, kmax = h.decompose()
            torch.cuda.synchronize()
            assert np.array_equal(tr.cpu().numpy(), want)
            assert kmax == (int(want.max()) if g.m else 0)
            stats.append(h.stats())
            h.close()
        a, b = stats
        assert a.rounds == b.rounds
        assert a.removed_per_round == b.removed_per_round
        assert a.live_per_round == b.live_per_round
        assert a.triangles_per_round == b.triangles_per_round
        assert a.updated_per_round == b.updated_per_round
        assert b.device_loop_rounds == 0
