// C ABI and host runtime of libktruss: graph handles, the peel-round driver of
// Alg. 1 (support step, prune, compaction, convergence test) and statistics.
//
// One round on the caller's stream:
//   memset S = 0                      (Alg. 1 recomputes S from scratch)
//   support step                      (Alg. 3 edge tasks; balanced or per-edge kernel)
//   prune count + tile scan           (Step 2: keep iff S >= K-2)
//   4-byte read of the kept count     (the isUnchanged test, the only host sync)
//   if nothing was removed: finalize outputs of the survivors, stop
//   else compact survivors into the other CSR buffer (removed edges' outputs
//        are written here), continue while any edge is live.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ktruss.h"
#include "ktruss_internal.cuh"

namespace {

thread_local int g_last_cuda_error = 0;

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return KTRUSS_OK;
    g_last_cuda_error = int(e);
    cudaGetLastError();  // clear a non-sticky error
    if (e == cudaErrorMemoryAllocation) return KTRUSS_ENOMEM;
    return KTRUSS_ECUDA;
}

#define KT_CK(call)                                  \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return map_cuda(e_);  \
    } while (0)

// Allocation with an optional simulated failure, for the out-of-memory tests:
// KTRUSS_TEST_FAIL_ALLOC=N makes the (N+1)-th device allocation of a load fail.
struct Allocator {
    long budget = -1;
    std::vector<void *> owned;
    Allocator() {
        const char *v = std::getenv("KTRUSS_TEST_FAIL_ALLOC");
        if (v && *v) budget = std::atol(v);
    }
    cudaError_t alloc(void **p, size_t bytes) {
        *p = nullptr;
        if (budget == 0) return cudaErrorMemoryAllocation;
        if (budget > 0) --budget;
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    }
};

}  // namespace

struct ktruss_graph {
    int32_t n = 0;
    int64_t m = 0;
    int device = 0;
    // immutable loaded graph
    int32_t *rp0 = nullptr, *col0 = nullptr;
    // double-buffered live graph
    int32_t *rp[2] = {nullptr, nullptr}, *col[2] = {nullptr, nullptr}, *eid[2] = {nullptr, nullptr};
    int32_t *S = nullptr, *pos = nullptr;
    int32_t *tile_count = nullptr, *tile_off = nullptr;
    kt::RoundCounters *cnt = nullptr;       // device
    kt::RoundCounters *cnt_host = nullptr;  // pinned mirror
    uint8_t *d_mask = nullptr;              // device outputs for host-kind runs
    int32_t *d_sup = nullptr;
    kt::BalancedScratch bs;
    // batches (ktruss_load_batch): G graphs, vertex offsets, graph of each vertex
    int32_t G = 0;
    int32_t *vo = nullptr, *gid = nullptr, *thr = nullptr, *live_g = nullptr,
            *removed_g = nullptr, *rounds_g = nullptr;
    uint8_t *keep = nullptr, *done = nullptr;
    std::vector<void *> owned;
    std::atomic<int> busy{0};
    // options
    int support_kernel = KTRUSS_KERNEL_AUTO;
    int timing = 1;
    // events: [0] run start, [1] run end, then 5 per round
    std::vector<cudaEvent_t> events;
    // stats of the last run
    bool has_stats = false;
    ktruss_stats_t st{};
    std::vector<int64_t> removed, live, tris, merge;
    std::vector<float> ms_sup;
};

namespace {

struct BusyGuard {
    ktruss_graph *g;
    bool ok;
    explicit BusyGuard(ktruss_graph *gg) : g(gg) {
        int exp = 0;
        ok = g->busy.compare_exchange_strong(exp, 1);
    }
    ~BusyGuard() {
        if (ok) g->busy.store(0);
    }
};

void release(ktruss_graph *g) {
    if (!g) return;
    for (void *p : g->owned) cudaFree(p);
    kt::balanced_scratch_free(&g->bs);
    if (g->cnt_host) cudaFreeHost(g->cnt_host);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    delete g;
}

cudaError_t ensure_events(ktruss_graph *g, size_t count) {
    while (g->events.size() < count) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        g->events.push_back(e);
    }
    return cudaSuccess;
}

// Live graphs below this many edges use the one-thread-per-edge kernel under
// KTRUSS_KERNEL_AUTO: the balanced step's fixed cost (a dozen small kernels
// before the support kernel) dominates there.
constexpr int32_t kAutoSmallEdges = 1 << 17;

// One support step (Alg. 1 Step 1) on the live graph with the handle's kernel
// choice.  When ev is given (the balanced path), ev[1] is recorded between the
// balance kernels and the support kernel; otherwise ev[1] is recorded before
// the support kernel.
cudaError_t support_step(ktruss_graph *g, const kt::Live &cur, cudaStream_t s, int *launches,
                         cudaEvent_t *ev) {
    int k = g->support_kernel;
    if (k == KTRUSS_KERNEL_AUTO) k = cur.m < kAutoSmallEdges ? KTRUSS_KERNEL_EDGE : KTRUSS_KERNEL_BALANCED;
    if (k == KTRUSS_KERNEL_BALANCED) {
        int l = 0;
        cudaError_t e = kt::launch_support_balanced(cur, g->S, g->cnt, &g->bs, s, &l, ev);
        *launches += l;
        return e;
    }
    if (ev) {
        cudaError_t e = cudaEventRecord(ev[1], s);
        if (e != cudaSuccess) return e;
    }
    ++*launches;
    return k == KTRUSS_KERNEL_EDGE ? kt::launch_support_edge(cur, g->S, g->cnt, s)
                                   : kt::launch_support_coarse(cur, g->S, g->cnt, s);
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

}  // namespace

extern "C" {

const char *ktruss_strerror(int code) {
    switch (code) {
        case KTRUSS_OK: return "ok";
        case KTRUSS_EINVAL: return "invalid argument or malformed CSR";
        case KTRUSS_ENOMEM: return "out of memory";
        case KTRUSS_ECUDA: return "CUDA runtime error";
        case KTRUSS_ETIMEOUT: return "bounded device wait timed out";
        case KTRUSS_EBUSY: return "graph handle busy";
        default: return "unknown error";
    }
}

int ktruss_last_cuda_error(void) { return g_last_cuda_error; }

int ktruss_version(void) { return 100; }

static int load_impl(ktruss_graph **out, int32_t n, int64_t m, const int32_t *row_ptr,
                     const int32_t *col, int mem_kind, void *cuda_stream, int32_t G,
                     const int32_t *vertex_offsets) {
    if (!out) return KTRUSS_EINVAL;
    *out = nullptr;
    if (n < 0 || m < 0 || m >= (int64_t(1) << 31) || !row_ptr || (m > 0 && !col))
        return KTRUSS_EINVAL;
    if (mem_kind != KTRUSS_HOST && mem_kind != KTRUSS_DEVICE) return KTRUSS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    ktruss_graph *g = new (std::nothrow) ktruss_graph();
    if (!g) return KTRUSS_ENOMEM;
    g->n = n;
    g->m = m;
    Allocator al;
    int rc = KTRUSS_OK;
    auto A = [&](void **p, size_t bytes) -> bool {
        cudaError_t e = al.alloc(p, bytes);
        if (e != cudaSuccess) {
            rc = map_cuda(e);
            return false;
        }
        return true;
    };
    const size_t rpb = (size_t(n) + 1) * sizeof(int32_t);
    const size_t eb = size_t(m) * sizeof(int32_t);
    const int32_t tiles = kt::compact_tiles(int32_t(m));
    bool ok = A((void **)&g->rp0, rpb) && A((void **)&g->col0, eb) && A((void **)&g->rp[0], rpb) &&
              A((void **)&g->rp[1], rpb) && A((void **)&g->col[0], eb) &&
              A((void **)&g->col[1], eb) && A((void **)&g->eid[0], eb) &&
              A((void **)&g->eid[1], eb) && A((void **)&g->S, eb) &&
              A((void **)&g->pos, eb) && A((void **)&g->tile_count, (tiles + 1) * 4) &&
              A((void **)&g->tile_off, (tiles + 1) * 4) &&
              A((void **)&g->cnt, sizeof(kt::RoundCounters));
    if (ok && G > 0) {
        const size_t gb = (size_t(G) + 1) * 4;
        ok = A((void **)&g->vo, gb) && A((void **)&g->gid, (size_t(n) + 1) * 4) &&
             A((void **)&g->thr, gb) && A((void **)&g->live_g, gb) &&
             A((void **)&g->removed_g, gb) && A((void **)&g->rounds_g, gb) &&
             A((void **)&g->keep, size_t(m) + 1) && A((void **)&g->done, size_t(G) + 1);
        g->G = G;
    }
    g->owned = al.owned;
    if (!ok) {
        release(g);
        return rc;
    }
    if (al.budget == 0) {  // simulated failure of the scratch allocation
        release(g);
        return KTRUSS_ENOMEM;
    }
    cudaError_t e = kt::balanced_scratch_alloc(&g->bs, n, m);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->cnt_host, sizeof(kt::RoundCounters));
    if (e == cudaSuccess) e = cudaGetDevice(&g->device);
    const cudaMemcpyKind kind =
        mem_kind == KTRUSS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->rp0, row_ptr, rpb, kind, s);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->col0, col, eb, kind, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->cnt, 0, sizeof(kt::RoundCounters), s);
    if (e == cudaSuccess) e = kt::launch_validate(g->rp0, g->col0, n, m, &g->cnt->error, s);
    if (e == cudaSuccess && G > 0) {
        e = cudaMemcpyAsync(g->vo, vertex_offsets, (size_t(G) + 1) * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = kt::launch_graph_of_vertex(g->vo, G, n, g->gid, s);
        if (e == cudaSuccess) e = kt::launch_batch_validate(g->rp0, g->col0, n, g->gid,
                                                            &g->cnt->error, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->cnt_host, g->cnt, sizeof(kt::RoundCounters),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rc = map_cuda(e);
        release(g);
        return rc;
    }
    if (g->cnt_host->error != 0) {
        release(g);
        return KTRUSS_EINVAL;
    }
    *out = g;
    return KTRUSS_OK;
}

int ktruss_load_csr(ktruss_graph **out, int32_t n, int64_t m, const int32_t *row_ptr,
                    const int32_t *col, int mem_kind, void *cuda_stream) {
    return load_impl(out, n, m, row_ptr, col, mem_kind, cuda_stream, 0, nullptr);
}

int ktruss_load_batch(ktruss_graph **out, int32_t num_graphs, const int32_t *vertex_offsets,
                      int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                      int mem_kind, void *cuda_stream) {
    if (!out) return KTRUSS_EINVAL;
    *out = nullptr;
    if (num_graphs < 1 || !vertex_offsets) return KTRUSS_EINVAL;
    if (vertex_offsets[0] != 0 || vertex_offsets[num_graphs] != n) return KTRUSS_EINVAL;
    for (int32_t k = 0; k < num_graphs; ++k)
        if (vertex_offsets[k + 1] < vertex_offsets[k]) return KTRUSS_EINVAL;
    return load_impl(out, n, m, row_ptr, col, mem_kind, cuda_stream, num_graphs, vertex_offsets);
}

int ktruss_batch_size(const ktruss_graph *g, int32_t *num_graphs) {
    if (!g || !num_graphs) return KTRUSS_EINVAL;
    *num_graphs = g->G;
    return KTRUSS_OK;
}

int ktruss_run_batch(ktruss_graph *g, const int32_t *K, uint8_t *mask_out, int32_t *support_out,
                     int32_t *rounds_out, int mem_kind, void *cuda_stream) {
    if (!g || g->G < 1 || !K || (g->m > 0 && !mask_out)) return KTRUSS_EINVAL;
    if (mem_kind != KTRUSS_HOST && mem_kind != KTRUSS_DEVICE) return KTRUSS_EINVAL;
    const int32_t G = g->G;
    for (int32_t k = 0; k < G; ++k)
        if (K[k] < 2) return KTRUSS_EINVAL;
    BusyGuard guard(g);
    if (!guard.ok) return KTRUSS_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int32_t n = g->n;
    const int32_t m = int32_t(g->m);
    g->has_stats = false;
    g->removed.clear();
    g->live.clear();
    g->tris.clear();
    g->merge.clear();
    g->ms_sup.clear();
    uint8_t *mask_d = mask_out;
    int32_t *sup_d = support_out;
    if (mem_kind == KTRUSS_HOST && m > 0) {
        if (!g->d_mask) {
            Allocator al;
            KT_CK(al.alloc((void **)&g->d_mask, size_t(m)));
            g->owned.push_back(g->d_mask);
            KT_CK(al.alloc((void **)&g->d_sup, size_t(m) * 4));
            g->owned.push_back(g->d_sup);
        }
        mask_d = g->d_mask;
        sup_d = support_out ? g->d_sup : nullptr;
    }
    // per-graph thresholds K_g - 2 (the staging vector lives until the final
    // synchronisation below)
    std::vector<int32_t> thr(G);
    for (int32_t k = 0; k < G; ++k) thr[k] = K[k] - 2;
    KT_CK(cudaMemcpyAsync(g->thr, thr.data(), size_t(G) * 4, cudaMemcpyHostToDevice, s));
    KT_CK(cudaMemsetAsync(g->done, 0, size_t(G), s));
    KT_CK(cudaMemsetAsync(g->rounds_g, 0, size_t(G) * 4, s));
    const bool timing = g->timing != 0;
    if (timing) {
        KT_CK(ensure_events(g, 2));
        KT_CK(cudaEventRecord(g->events[0], s));
    }
    int launches = 0, support_launches = 0, rounds = 0;
    kt::Live cur{g->rp0, g->col0, nullptr, n, m};
    int buf = 0;
    while (cur.m > 0) {
        ++rounds;
        KT_CK(cudaMemsetAsync(g->S, 0, size_t(cur.m) * 4, s));
        KT_CK(cudaMemsetAsync(g->cnt, 0, sizeof(kt::RoundCounters), s));
        KT_CK(cudaMemsetAsync(g->live_g, 0, size_t(G) * 4, s));
        KT_CK(cudaMemsetAsync(g->removed_g, 0, size_t(G) * 4, s));
        KT_CK(support_step(g, cur, s, &launches, nullptr));
        ++support_launches;
        KT_CK(kt::launch_batch_prune(cur, g->S, g->gid, g->thr, g->keep, g->live_g, g->removed_g,
                                     g->done, g->rounds_g, G, g->tile_count, g->tile_off, g->cnt,
                                     s, &launches));
        const int nb = buf;
        KT_CK(kt::launch_batch_compact(cur, g->S, g->keep, g->done, g->gid, g->tile_off, g->cnt,
                                       g->pos, g->rp[nb], g->col[nb], g->eid[nb], mask_d, sup_d,
                                       s, &launches));
        KT_CK(cudaMemcpyAsync(g->cnt_host, g->cnt, sizeof(kt::RoundCounters),
                              cudaMemcpyDeviceToHost, s));
        KT_CK(cudaStreamSynchronize(s));
        const kt::RoundCounters c = *g->cnt_host;
        if (c.error) return (c.error & kt::kDevErrTimeout) ? KTRUSS_ETIMEOUT : KTRUSS_ECUDA;
        g->live.push_back(cur.m);
        g->tris.push_back(int64_t(c.triangles));
        g->merge.push_back(int64_t(c.merge_work));
        g->removed.push_back(int64_t(cur.m) - c.kept);
        g->ms_sup.push_back(0.f);
        cur = kt::Live{g->rp[nb], g->col[nb], g->eid[nb], n, c.kept};
        buf ^= 1;
    }
    if (timing) KT_CK(cudaEventRecord(g->events[1], s));
    if (mem_kind == KTRUSS_HOST && m > 0) {
        KT_CK(cudaMemcpyAsync(mask_out, mask_d, size_t(m), cudaMemcpyDeviceToHost, s));
        if (support_out)
            KT_CK(cudaMemcpyAsync(support_out, sup_d, size_t(m) * 4, cudaMemcpyDeviceToHost, s));
    }
    if (rounds_out)
        KT_CK(cudaMemcpyAsync(rounds_out, g->rounds_g, size_t(G) * 4, cudaMemcpyDeviceToHost, s));
    KT_CK(cudaStreamSynchronize(s));
    g->st = ktruss_stats_t{};
    g->st.rounds = rounds;
    g->st.edges_in = g->m;
    g->st.per_round_len = rounds;
    g->st.removed_per_round = g->removed.data();
    g->st.live_per_round = g->live.data();
    g->st.triangles_per_round = g->tris.data();
    g->st.ms_support_per_round = g->ms_sup.data();
    g->st.merge_work_per_round = g->merge.data();
    g->st.ms_total = timing ? elapsed(g->events[0], g->events[1]) : 0.f;
    g->st.support_launches = support_launches;
    g->st.kernel_launches = launches;
    g->has_stats = true;
    return KTRUSS_OK;
}

int ktruss_graph_size(const ktruss_graph *g, int32_t *n, int64_t *m) {
    if (!g || !n || !m) return KTRUSS_EINVAL;
    *n = g->n;
    *m = g->m;
    return KTRUSS_OK;
}

int ktruss_set_option(ktruss_graph *g, int32_t key, int64_t value) {
    if (!g) return KTRUSS_EINVAL;
    switch (key) {
        case KTRUSS_OPT_SUPPORT_KERNEL:
            if (value != KTRUSS_KERNEL_BALANCED && value != KTRUSS_KERNEL_EDGE &&
                value != KTRUSS_KERNEL_COARSE && value != KTRUSS_KERNEL_AUTO)
                return KTRUSS_EINVAL;
            g->support_kernel = int(value);
            return KTRUSS_OK;
        case KTRUSS_OPT_TIMING:
            if (value != 0 && value != 1) return KTRUSS_EINVAL;
            g->timing = int(value);
            return KTRUSS_OK;
        default:
            return KTRUSS_EINVAL;
    }
}

int ktruss_run(ktruss_graph *g, int32_t K, uint8_t *mask_out, int32_t *support_out, int mem_kind,
               void *cuda_stream) {
    if (!g || K < 2 || (g->m > 0 && !mask_out)) return KTRUSS_EINVAL;
    if (mem_kind != KTRUSS_HOST && mem_kind != KTRUSS_DEVICE) return KTRUSS_EINVAL;
    BusyGuard guard(g);
    if (!guard.ok) return KTRUSS_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int32_t n = g->n;
    const int32_t m = int32_t(g->m);
    const int32_t thr = K - 2;

    g->has_stats = false;
    g->removed.clear();
    g->live.clear();
    g->tris.clear();
    g->merge.clear();
    g->ms_sup.clear();

    uint8_t *mask_d = mask_out;
    int32_t *sup_d = support_out;
    if (mem_kind == KTRUSS_HOST && m > 0) {
        if (!g->d_mask) {
            Allocator al;
            KT_CK(al.alloc((void **)&g->d_mask, size_t(m)));
            g->owned.push_back(g->d_mask);
            KT_CK(al.alloc((void **)&g->d_sup, size_t(m) * 4));
            g->owned.push_back(g->d_sup);
        }
        mask_d = g->d_mask;
        sup_d = support_out ? g->d_sup : nullptr;
    }

    const bool timing = g->timing != 0;
    int launches = 0, support_launches = 0;
    if (timing) {
        KT_CK(ensure_events(g, 2));
        KT_CK(cudaEventRecord(g->events[0], s));
    }

    kt::Live cur{g->rp0, g->col0, nullptr, n, m};
    int buf = 0;
    int32_t rounds = 0;
    int64_t tri_final = 0;
    float ms_balance = 0.f, ms_support = 0.f, ms_prune = 0.f, ms_final = 0.f;
    std::vector<int> ev_base;
    while (cur.m > 0) {
        ++rounds;
        size_t base = 2 + size_t(rounds - 1) * 5;
        if (timing) {
            KT_CK(ensure_events(g, base + 5));
            ev_base.push_back(int(base));
        }
        KT_CK(cudaMemsetAsync(g->S, 0, size_t(cur.m) * 4, s));
        KT_CK(cudaMemsetAsync(g->cnt, 0, sizeof(kt::RoundCounters), s));
        if (timing) KT_CK(cudaEventRecord(g->events[base + 0], s));
        KT_CK(support_step(g, cur, s, &launches, timing ? &g->events[base + 0] : nullptr));
        ++support_launches;
        if (timing) KT_CK(cudaEventRecord(g->events[base + 2], s));
        KT_CK(kt::launch_prune_count(g->S, cur.m, thr, g->tile_count, g->tile_off, g->cnt, s,
                                     &launches));
        KT_CK(cudaMemcpyAsync(g->cnt_host, g->cnt, sizeof(kt::RoundCounters),
                              cudaMemcpyDeviceToHost, s));
        KT_CK(cudaStreamSynchronize(s));
        const kt::RoundCounters c = *g->cnt_host;
        if (c.error) return (c.error & kt::kDevErrTimeout) ? KTRUSS_ETIMEOUT : KTRUSS_ECUDA;
        const int32_t kept = c.kept;
        const int64_t removed = int64_t(cur.m) - kept;
        g->removed.push_back(removed);
        g->live.push_back(cur.m);
        g->tris.push_back(int64_t(c.triangles));
        g->merge.push_back(int64_t(c.merge_work));
        if (removed == 0) {
            if (timing) KT_CK(cudaEventRecord(g->events[base + 3], s));
            KT_CK(kt::launch_finalize(cur, g->S, mask_d, sup_d, s, &launches));
            if (timing) KT_CK(cudaEventRecord(g->events[base + 4], s));
            tri_final = int64_t(c.triangles);
            break;
        }
        if (timing) KT_CK(cudaEventRecord(g->events[base + 3], s));
        const int nb = buf;
        KT_CK(kt::launch_compact(cur, g->S, thr, g->tile_off, g->cnt, g->pos, g->rp[nb],
                                 g->col[nb], g->eid[nb], mask_d, sup_d, s, &launches));
        if (timing) KT_CK(cudaEventRecord(g->events[base + 4], s));
        cur = kt::Live{g->rp[nb], g->col[nb], g->eid[nb], n, kept};
        buf ^= 1;
        tri_final = 0;
    }
    if (timing) KT_CK(cudaEventRecord(g->events[1], s));
    if (mem_kind == KTRUSS_HOST && m > 0) {
        KT_CK(cudaMemcpyAsync(mask_out, mask_d, size_t(m), cudaMemcpyDeviceToHost, s));
        if (support_out)
            KT_CK(cudaMemcpyAsync(support_out, sup_d, size_t(m) * 4, cudaMemcpyDeviceToHost, s));
    }
    KT_CK(cudaStreamSynchronize(s));

    float ms_total = 0.f;
    if (timing) {
        ms_total = elapsed(g->events[0], g->events[1]);
        for (size_t r = 0; r < ev_base.size(); ++r) {
            const size_t b = size_t(ev_base[r]);
            const float bal = elapsed(g->events[b + 0], g->events[b + 1]);
            const float sup = elapsed(g->events[b + 1], g->events[b + 2]);
            const float pr = elapsed(g->events[b + 2], g->events[b + 3]);
            const float tail = elapsed(g->events[b + 3], g->events[b + 4]);
            ms_balance += bal;
            ms_support += sup;
            g->ms_sup.push_back(sup);
            if (r + 1 == ev_base.size() && g->removed.back() == 0) {
                ms_prune += pr;
                ms_final += tail;
            } else {
                ms_prune += pr + tail;
            }
        }
    } else {
        g->ms_sup.assign(size_t(rounds), 0.f);
    }
    int64_t edges_out = 0;
    if (rounds > 0 && g->removed.back() == 0) edges_out = g->live.back();
    g->st = ktruss_stats_t{};
    g->st.rounds = rounds;
    g->st.edges_in = g->m;
    g->st.edges_out = edges_out;
    g->st.triangles_out = tri_final;
    g->st.per_round_len = rounds;
    g->st.removed_per_round = g->removed.data();
    g->st.live_per_round = g->live.data();
    g->st.triangles_per_round = g->tris.data();
    g->st.ms_support_per_round = g->ms_sup.data();
    g->st.merge_work_per_round = g->merge.data();
    g->st.ms_total = ms_total;
    g->st.ms_support = ms_support;
    g->st.ms_balance = ms_balance;
    g->st.ms_prune_compact = ms_prune;
    g->st.ms_finalize = ms_final;
    g->st.support_launches = support_launches;
    g->st.kernel_launches = launches;
    g->has_stats = true;
    return KTRUSS_OK;
}

int ktruss_decompose(ktruss_graph *g, int32_t *trussness_out, int32_t *kmax_out, int mem_kind,
                     void *cuda_stream) {
    if (!g || (g->m > 0 && !trussness_out)) return KTRUSS_EINVAL;
    if (mem_kind != KTRUSS_HOST && mem_kind != KTRUSS_DEVICE) return KTRUSS_EINVAL;
    BusyGuard guard(g);
    if (!guard.ok) return KTRUSS_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int32_t n = g->n;
    const int32_t m = int32_t(g->m);
    g->has_stats = false;
    g->removed.clear();
    g->live.clear();
    g->tris.clear();
    g->merge.clear();
    g->ms_sup.clear();
    int32_t *tr_d = trussness_out;
    if (mem_kind == KTRUSS_HOST && m > 0) {
        if (!g->d_mask) {
            Allocator al;
            KT_CK(al.alloc((void **)&g->d_mask, size_t(m)));
            g->owned.push_back(g->d_mask);
            KT_CK(al.alloc((void **)&g->d_sup, size_t(m) * 4));
            g->owned.push_back(g->d_sup);
        }
        tr_d = g->d_sup;
    }
    const bool timing = g->timing != 0;
    if (timing) {
        KT_CK(ensure_events(g, 2));
        KT_CK(cudaEventRecord(g->events[0], s));
    }
    int launches = 0, support_launches = 0, rounds = 0;
    kt::Live cur{g->rp0, g->col0, nullptr, n, m};
    int buf = 0;
    int32_t K = 3;          // the whole graph is the 2-truss
    bool have_s = false;    // S holds the supports of the current live graph
    while (cur.m > 0) {
        if (!have_s) {
            ++rounds;
            KT_CK(cudaMemsetAsync(g->S, 0, size_t(cur.m) * 4, s));
            KT_CK(cudaMemsetAsync(g->cnt, 0, sizeof(kt::RoundCounters), s));
            KT_CK(support_step(g, cur, s, &launches, nullptr));
            ++support_launches;
        }
        KT_CK(kt::launch_prune_count(g->S, cur.m, K - 2, g->tile_count, g->tile_off, g->cnt, s,
                                     &launches));
        KT_CK(cudaMemcpyAsync(g->cnt_host, g->cnt, sizeof(kt::RoundCounters),
                              cudaMemcpyDeviceToHost, s));
        KT_CK(cudaStreamSynchronize(s));
        const kt::RoundCounters c = *g->cnt_host;
        if (c.error) return (c.error & kt::kDevErrTimeout) ? KTRUSS_ETIMEOUT : KTRUSS_ECUDA;
        const int32_t kept = c.kept;
        if (!have_s) {
            g->live.push_back(cur.m);
            g->tris.push_back(int64_t(c.triangles));
            g->merge.push_back(int64_t(c.merge_work));
            g->removed.push_back(int64_t(cur.m) - kept);
            g->ms_sup.push_back(0.f);
        } else if (!g->removed.empty()) {
            g->removed.back() += int64_t(cur.m) - kept;
        }
        if (kept == cur.m) {
            // cur is the (non-empty) K-truss: the (K+1)-truss lies inside it,
            // and its supports are already in S
            ++K;
            have_s = true;
            continue;
        }
        const int nb = buf;
        KT_CK(kt::launch_compact(cur, g->S, K - 2, g->tile_off, g->cnt, g->pos, g->rp[nb],
                                 g->col[nb], g->eid[nb], nullptr, nullptr, s, &launches, tr_d,
                                 K - 1));
        cur = kt::Live{g->rp[nb], g->col[nb], g->eid[nb], n, kept};
        buf ^= 1;
        have_s = false;
    }
    if (timing) KT_CK(cudaEventRecord(g->events[1], s));
    if (mem_kind == KTRUSS_HOST && m > 0)
        KT_CK(cudaMemcpyAsync(trussness_out, tr_d, size_t(m) * 4, cudaMemcpyDeviceToHost, s));
    KT_CK(cudaStreamSynchronize(s));
    if (kmax_out) *kmax_out = m == 0 ? 0 : K - 1;
    g->st = ktruss_stats_t{};
    g->st.rounds = rounds;
    g->st.edges_in = g->m;
    g->st.per_round_len = rounds;
    g->st.removed_per_round = g->removed.data();
    g->st.live_per_round = g->live.data();
    g->st.triangles_per_round = g->tris.data();
    g->st.ms_support_per_round = g->ms_sup.data();
    g->st.merge_work_per_round = g->merge.data();
    g->st.ms_total = timing ? elapsed(g->events[0], g->events[1]) : 0.f;
    g->st.support_launches = support_launches;
    g->st.kernel_launches = launches;
    g->has_stats = true;
    return KTRUSS_OK;
}

int ktruss_stats(const ktruss_graph *g, ktruss_stats_t *out) {
    if (!g || !out || !g->has_stats) return KTRUSS_EINVAL;
    *out = g->st;
    return KTRUSS_OK;
}

void ktruss_free(ktruss_graph *g) { release(g); }

}  // extern "C"
