"""ktruss_support_noalloc, the entry point for callers that may not allocate.

Some callers cannot call cudaMalloc on their path (they run inside a memory
pool they do not own, or must not grow the device footprint after start-up).
For them the library computes a graph's edge supports with working memory
taken from a fixed array inside the library.  This test calls that entry
point through the C ABI, twice in a row on the same device, and checks each
result against the regular entry point (ktruss_run with K = 2, whose supports
are the full-graph triangle counts) and against the CPU oracle's K = 2 run.
All arithmetic is integer, so the tolerance is zero.  It lives in a file of its
own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def regular_supports(kt, torch, g):
    h = kt.load(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
    _, sup = h.run(2)
    torch.cuda.synchronize()
    out = sup.cpu().numpy().copy()
    tri = h.stats().triangles_out
    h.close()
    return out, tri


def noalloc_supports(kt, torch, g):
    L = kt.lib()
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    out = torch.full((g.m,), -7, dtype=torch.int32, device="cuda")
    tri = ctypes.c_int64(-1)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.ktruss_support_noalloc(g.n, g.m, rp.data_ptr(), col.data_ptr(), out.data_ptr(),
                                  ctypes.addressof(tri), stream)
    assert rc == 0, L.ktruss_strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy(), tri.value


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    import paper_2009_07929_gb300 as kt
    # the R-MAT scale-15 graph (2^19 samples) is close to the edge limit and has
    # rows longer than a stage; the last graph sits at both size limits
    # (n = m = 524288)
    graphs = [gg.rmat(14, 16, seed=21), gg.er(2000, 16000, seed=4), gg.rmat(15, 16, seed=8),
              gg.er(kt.NOALLOC_MAX_VERTICES, kt.NOALLOC_MAX_EDGES, seed=6)]
    ref = [oracle.ktruss(g.row_ptr, g.col, 2) for g in graphs]
    ref = ref + ref[::-1]
    # two calls in a row on the same device; the second sees the first's leftovers
    for g, r in zip(graphs + graphs[::-1], ref):
        want, want_tri = regular_supports(kt, torch, g)
        got, got_tri = noalloc_supports(kt, torch, g)
        assert np.array_equal(got, want)
        assert got_tri == want_tri
        assert np.array_equal(got, r.support) and got_tri == r.triangles


def test_noalloc_rejects_oversized_graphs():
    import torch
    import paper_2009_07929_gb300 as kt
    L = kt.lib()
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    too_many_v = kt.NOALLOC_MAX_VERTICES + 1
    assert L.ktruss_support_noalloc(too_many_v, 0, rp.data_ptr(), None, None, None,
                                    stream) == kt.EINVAL
    assert L.ktruss_support_noalloc(1, kt.NOALLOC_MAX_EDGES + 1, rp.data_ptr(), rp.data_ptr(),
                                    rp.data_ptr(), None, stream) == kt.EINVAL
