"""Batched peeling on the GPU: every graph of a batch, each with its own K,
must get exactly the outputs and round count of its own solo run (tolerance 0;
all arithmetic is integer).  The oracle checks small batches directly; larger
config-4-shaped batches are checked against solo GPU runs, themselves parity-
tested against the oracle elsewhere."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import paper_2009_07929_gb300 as kt
    kt.lib()
    return kt


def run_batch(kt, graphs, Ks, kernel=None, update=None, reorder=None):
    import torch
    vo, rp, col, eo = kt.concat_graphs(graphs)
    h = kt.load_batch(vertex_offsets=vo, row_ptr=torch.from_numpy(rp).cuda(),
                      col=torch.from_numpy(col).cuda())
    if kernel is not None:
        h.set_kernel(kernel)
    if update is not None:
        h.set_update(update)
    if reorder is not None:
        h.set_reorder(reorder)
    mask, sup, rounds = h.run_batch(Ks)
    torch.cuda.synchronize()
    mask, sup = mask.cpu().numpy(), sup.cpu().numpy()
    st = h.stats()
    h.close()
    return mask, sup, rounds, eo, st


def mixed_small_graphs():
    gs = [gg.complete(9), gg.book(30), gg.triangle_strip(40), gg.star(12), gg.empty(0),
          gg.empty(7), gg.complete(4), gg.rmat(11, 16, 3), gg.er(2000, 16000, 2),
          gg.rmat(12, 8, seed=5, n_cliques=4, clique_lo=12, clique_hi=30)]
    gs += [gg.gnp_small(10 + s, 0.4, seed=900 + s) for s in range(20)]
    Ks = [9, 3, 4, 3, 3, 5, 5, 4, 3, 12] + [2 + s % 6 for s in range(20)]
    return gs, Ks


@pytest.mark.parametrize("kernel,update", [(0, None), (1, None), (3, 0), (3, 1), (3, 2)])
def test_batch_equals_solo_oracle(kt, kernel, update):
    gs, Ks = mixed_small_graphs()
    mask, sup, rounds, eo, st = run_batch(kt, gs, Ks, kernel, update)
    for k, (g, K) in enumerate(zip(gs, Ks)):
        r = oracle.ktruss(g.row_ptr, g.col, K)
        assert np.array_equal(mask[eo[k]:eo[k + 1]], r.mask), k
        assert np.array_equal(sup[eo[k]:eo[k + 1]], r.support), k
        assert rounds[k] == r.rounds, k
    assert st.rounds == max(rounds)


@pytest.mark.parametrize("update", [0, 1, 2])
def test_batch_config_shape_equals_solo_gpu(kt, update):
    import torch
    batch = gg.batch_config(48, seed=1, m_lo=1e3, m_hi=6e4)
    gs = [b[0] for b in batch]
    Ks = [b[1] for b in batch]
    mask, sup, rounds, eo, _ = run_batch(kt, gs, Ks, update=update)
    for k, (g, K) in enumerate(batch):
        h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
        h.set_update(0)  # the solo reference recomputes every round (Alg. 1 as written)
        m_t, s_t = h.run(K)
        torch.cuda.synchronize()
        assert np.array_equal(mask[eo[k]:eo[k + 1]], m_t.cpu().numpy()), k
        assert np.array_equal(sup[eo[k]:eo[k + 1]], s_t.cpu().numpy()), k
        assert rounds[k] == h.stats().rounds, k
        h.close()
    # a few graphs against the oracle directly
    for k in (0, 1, 7, 30):
        g, K = batch[k]
        r = oracle.ktruss(g.row_ptr, g.col, K)
        assert np.array_equal(mask[eo[k]:eo[k + 1]], r.mask)
        assert np.array_equal(sup[eo[k]:eo[k + 1]], r.support)


def test_batch_handle_runs_single_K_and_decompose(kt):
    import torch
    gs, _ = mixed_small_graphs()
    vo, rp, col, eo = kt.concat_graphs(gs)
    h = kt.load_batch(vertex_offsets=vo, row_ptr=torch.from_numpy(rp).cuda(),
                      col=torch.from_numpy(col).cuda())
    m_t, s_t = h.run(4)
    tr_t, kmax = h.decompose()
    torch.cuda.synchronize()
    mask, sup, tr = m_t.cpu().numpy(), s_t.cpu().numpy(), tr_t.cpu().numpy()
    for k, g in enumerate(gs):
        r = oracle.ktruss(g.row_ptr, g.col, 4)
        assert np.array_equal(mask[eo[k]:eo[k + 1]], r.mask)
        assert np.array_equal(sup[eo[k]:eo[k + 1]], r.support)
        assert np.array_equal(tr[eo[k]:eo[k + 1]], oracle.truss_decomposition(g.row_ptr, g.col))
    h.close()


def test_batch_autotune(kt):
    import torch
    gs, Ks = mixed_small_graphs()
    vo, rp, col, eo = kt.concat_graphs(gs)
    h = kt.load_batch(vertex_offsets=vo, row_ptr=torch.from_numpy(rp).cuda(),
                      col=torch.from_numpy(col).cuda())
    t = h.autotune(Ks, reps=1)
    assert t["trials"] >= 10
    mask, sup, rounds = h.run_batch(Ks)
    torch.cuda.synchronize()
    mask, sup = mask.cpu().numpy(), sup.cpu().numpy()
    for k, (g, K) in enumerate(zip(gs, Ks)):
        r = oracle.ktruss(g.row_ptr, g.col, K)
        assert np.array_equal(mask[eo[k]:eo[k + 1]], r.mask), k
        assert np.array_equal(sup[eo[k]:eo[k + 1]], r.support), k
        assert rounds[k] == r.rounds, k
    h.close()


def test_batch_rejects_edges_across_graphs(kt):
    g = gg.from_edges(4, [(0, 1), (1, 2), (0, 2), (2, 3)])
    # vertices {0,1} and {2,3} declared as two graphs: edge (1,2) crosses
    with pytest.raises(kt.KtrussError) as ei:
        kt.load_batch(vertex_offsets=np.array([0, 2, 4], np.int32), row_ptr=g.row_ptr,
                      col=g.col)
    assert ei.value.code == kt.EINVAL
    with pytest.raises(kt.KtrussError):
        kt.load_batch(vertex_offsets=np.array([0, 3, 2], np.int32), row_ptr=g.row_ptr,
                      col=g.col)


def test_full_batching_workload_against_oracle_digests(kt):
    """The batching workload at full size (4096 graphs of 1e3..2e6 edges, 1.2e9
    edges in all, K per graph uniform in 3..12, seed 0), run as one batch with
    the default options, as the benchmark times it, then with the supports
    recomputed every round.  Every graph's mask, supports and round count are
    compared with the oracle's, stored as digests by tests/golden/make_golden.py
    (oracle.ktruss on each graph; nothing from the CUDA library)."""
    import hashlib
    import json
    import os

    import torch
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096.json")
    if not os.path.exists(p):
        pytest.skip("no stored oracle digests for the batching workload")
    with open(p) as f:
        c = json.load(f)

    def sha(b) -> str:
        return hashlib.sha256(b).hexdigest()

    def digest_of_digests(hexes) -> str:
        return sha("".join(hexes).encode("ascii"))

    batch = gg.batch_config(c["graphs"], seed=c["seed"], m_lo=c["m_lo"], m_hi=c["m_hi"],
                            k_lo=c["k_lo"], k_hi=c["k_hi"])
    graphs = [b[0] for b in batch]
    Ks = [int(b[1]) for b in batch]
    assert Ks == c["K"]
    assert digest_of_digests(
        sha(np.ascontiguousarray(g.row_ptr, dtype="<i4").tobytes()
            + np.ascontiguousarray(g.col, dtype="<i4").tobytes()) for g in graphs
    ) == c["graphs_sha256"], "generator output changed"
    vo, rp, col, eo = kt.concat_graphs(graphs)
    del batch, graphs
    assert int(eo[-1]) == c["edges"]
    h = kt.load_batch(vertex_offsets=vo, row_ptr=torch.from_numpy(rp).cuda(),
                      col=torch.from_numpy(col).cuda())
    del rp, col
    lo, hi = eo[:-1].tolist(), eo[1:].tolist()
    # the default options first (decremental update), then Alg. 1 as written
    # (supports recomputed every round) on the same handle
    for update in (None, 0):
        if update is not None:
            h.set_update(update)
        mask_t, sup_t, rounds = h.run_batch(Ks)
        torch.cuda.synchronize()
        st = h.stats()
        mask = mask_t.cpu().numpy()
        sup = np.ascontiguousarray(sup_t.cpu().numpy(), dtype="<i4")
        del mask_t, sup_t
        assert [int(r) for r in rounds] == c["rounds"], update
        assert st.rounds == max(c["rounds"]), update
        csum = np.concatenate([[0], np.cumsum(mask, dtype=np.int64)])
        assert (csum[eo[1:]] - csum[eo[:-1]]).tolist() == c["edges_out"], update
        assert int(sup.sum(dtype=np.int64)) == c["support_sum_total"], update
        assert digest_of_digests(sha(mask[a:b].tobytes())
                                 for a, b in zip(lo, hi)) == c["mask_sha256"], update
        assert digest_of_digests(sha(sup[a:b].tobytes())
                                 for a, b in zip(lo, hi)) == c["support_sha256"], update
    h.close()


@pytest.mark.parametrize("reorder", [True, False])
def test_batch_reorder_on_and_off(kt, reorder):
    """A batch run from the per-graph degree-ordered relabel made at load
    (default) and from the loaded numbering: every graph gets the oracle's
    mask, supports and round count."""
    gs, Ks = mixed_small_graphs()
    gs = gs + [gg.rmat(13, 16, 7), gg.rmat(12, 16, 8, relabel=True)]
    Ks = Ks + [5, 4]
    mask, sup, rounds, eo, _ = run_batch(kt, gs, Ks, reorder=reorder)
    for k, (g, K) in enumerate(zip(gs, Ks)):
        r = oracle.ktruss(g.row_ptr, g.col, K)
        assert np.array_equal(mask[eo[k]:eo[k + 1]], r.mask), k
        assert np.array_equal(sup[eo[k]:eo[k + 1]], r.support), k
        assert rounds[k] == r.rounds, k
