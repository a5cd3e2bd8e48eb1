// K-truss request server: continuous batching of many K-truss queries.
//
// Requests (a graph in host memory and its K) are queued by
// ktruss_server_submit, which stages the graph on the device and validates
// it there while the budget has room (else it keeps a validated host copy
// until admission).  Each ktruss_server_step:
//   1. admits queued requests in arrival order while they fit: a free slot,
//      room in the live CSR (vertices, edges) and in the device budget for
//      the request's own input staging and output buffers (its HBM
//      footprint); an admitted request's graph is appended to the live CSR;
//   2. runs one peel round (supports of every active request, then each
//      request pruned with its own threshold) — the rounds of all active
//      requests are one batched computation on the device.  Each request
//      admitted in this step gets a support step over its own CSR; the older
//      requests keep the previous step's supports updated for the edges it
//      removed (decremental update, the default), except those whose own
//      rule chose a support step, which get one (masked) step over the older
//      part of the live CSR;
//   3. finishes the requests whose round removed nothing or removed every
//      live edge (their outputs are already in their device buffers), copies
//      their outputs to the caller's host buffers and returns their device
//      blocks to the cache.
// A request therefore goes through exactly the bulk rounds of its own
// ktruss_run, whatever else is in flight (the paper's Alg. 1 per request).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "ktruss.h"
#include "ktruss_internal.cuh"

namespace {

struct Request {
    int64_t ticket;
    int32_t n;
    int64_t m;
    int32_t K;
    std::unique_ptr<int32_t[]> rp, col;  // host copies (left uninitialised, then filled)
    uint8_t *mask_out;
    int32_t *support_out;
    // staged at submit: the input already on the device (row_ptr then col)
    // and the request's bytes already counted against the budget
    int32_t *din = nullptr;
    bool staged = false;
};

struct Slot {
    bool used = false;
    int64_t ticket = 0;
    int32_t n = 0;
    int64_t m = 0;
    size_t bytes = 0;
    uint8_t *host_mask = nullptr;
    int32_t *host_sup = nullptr;
    uint8_t *dmask = nullptr;
    int32_t *dsup = nullptr;
    int32_t *din = nullptr;  // staged input: row_ptr then col
    size_t din_bytes = 0;
    int32_t *dre = nullptr;  // degree-ordered relabel: row_ptr, col, input slot of each slot
    size_t dre_bytes = 0;
};

// Device bytes of a request's staged input (row_ptr then col).
size_t input_bytes(int32_t n, int64_t m) { return (size_t(n) + 1 + size_t(m)) * 4; }
// Device bytes of a request's degree-ordered relabel (row_ptr, col, slot map).
size_t relabel_bytes(int32_t n, int64_t m) { return (size_t(n) + 1 + 2 * size_t(m)) * 4; }

constexpr int32_t kAutoSmallEdges = 1 << 17;

int map_err(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KTRUSS_ENOMEM : KTRUSS_ECUDA;
}

#define SV_CK(call)                                \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return map_err(e_); \
    } while (0)

}  // namespace

struct ktruss_server {
    int32_t vcap = 0;
    int64_t ecap = 0;
    int32_t slots = 0;
    int64_t budget = 0, used = 0;
    cudaStream_t s = nullptr;
    int32_t *rp[2] = {}, *col[2] = {}, *eid[2] = {}, *gid[2] = {};
    int32_t *S = nullptr, *S2 = nullptr, *pos = nullptr, *vmap = nullptr;
    uint8_t *keep = nullptr, *fin = nullptr;
    int32_t *thr = nullptr, *kept_g = nullptr, *removed_g = nullptr, *rounds_g = nullptr;
    int32_t *verr = nullptr;       // device: validation error word of submit
    int32_t *verr_host = nullptr;  // pinned mirror
    uint8_t **mask_ptr = nullptr;
    int32_t **sup_ptr = nullptr;
    int32_t *etile_count = nullptr, *etile_off = nullptr, *vtile_count = nullptr,
            *vtile_off = nullptr;
    kt::RoundCounters *cnt = nullptr;       // [0] edges, [1] vertices, [2] update
    kt::RoundCounters *cnt_host = nullptr;  // pinned [3]
    uint8_t *fin_host = nullptr;            // pinned [slots]
    int32_t *rounds_host = nullptr;         // pinned [slots]
    void **ptr_host = nullptr;              // pinned [2 * slots] staging of slot pointers
    int32_t *thr_host = nullptr;            // pinned [slots]
    kt::BalancedScratch bs;
    kt::UpdateState ust;  // recomputed each step: vertex ids change between steps
    std::vector<void *> owned;
    int cur = 0;
    int32_t n_live = 0;
    int32_t m_live = 0;
    // per slot: upd_s = 1 when the slot's supports in S are current (carried
    // and updated from the last step, or computed at admission); listed_s /
    // kept_s: the round's listed and surviving edges of the slot
    uint8_t *upd_s = nullptr;
    int32_t *listed_s = nullptr, *kept_s = nullptr;
    bool any_valid = false;  // some live slot has upd_s = 1
    int32_t need_slots = 0;  // live slots with upd_s = 0
    int update_mode = KTRUSS_UPDATE_AUTO;
    int reorder = 1;  // KTRUSS_OPT_REORDER: requests are relabelled by degree at admission
    int64_t next_ticket = 1;
    std::deque<Request> queue;
    std::vector<Slot> slot;
    std::vector<int64_t> done_tickets;
    std::vector<int32_t> done_rounds;
    int64_t steps = 0;
};

namespace {

void server_release(ktruss_server *v) {
    if (!v) return;
    for (Slot &sl : v->slot) {
        if (sl.dmask) kt::cache_put(sl.dmask, size_t(sl.m));
        if (sl.dsup) kt::cache_put(sl.dsup, size_t(sl.m) * 4);
        if (sl.din) kt::cache_put(sl.din, sl.din_bytes);
        if (sl.dre) kt::cache_put(sl.dre, sl.dre_bytes);
    }
    for (Request &r : v->queue)
        if (r.din) kt::cache_put(r.din, input_bytes(r.n, r.m));
    if (v->verr_host) cudaFreeHost(v->verr_host);
    for (void *p : v->owned) cudaFree(p);
    kt::balanced_scratch_free(&v->bs);
    kt::balanced_side_destroy(&v->bs);
    if (v->cnt_host) cudaFreeHost(v->cnt_host);
    if (v->fin_host) cudaFreeHost(v->fin_host);
    if (v->rounds_host) cudaFreeHost(v->rounds_host);
    if (v->ptr_host) cudaFreeHost(v->ptr_host);
    if (v->thr_host) cudaFreeHost(v->thr_host);
    delete v;
}

// Runs body(lo, hi) on the parts of [0, count): one part per grain, at most
// one per hardware thread, all in the calling thread when there is one part.
template <typename F>
void parallel_ranges(int64_t count, int64_t grain, F body) {
    int64_t hw = int64_t(std::thread::hardware_concurrency());
    if (hw < 1) hw = 1;
    const int64_t parts = std::min<int64_t>(hw, std::max<int64_t>(1, count / grain));
    if (parts <= 1) {
        body(int64_t(0), count);
        return;
    }
    std::vector<std::thread> ts;
    ts.reserve(size_t(parts));
    for (int64_t k = 0; k < parts; ++k)
        ts.emplace_back(body, count * k / parts, count * (k + 1) / parts);
    for (std::thread &t : ts) t.join();
}

// The CSR contract of ktruss_load_csr, checked on the host (rows split over
// host threads for large requests).  Every row checks its own bounds before
// it reads its columns, so no part reads outside col whatever the input.
bool valid_csr(int32_t n, int64_t m, const int32_t *rp, const int32_t *col) {
    if (rp[0] != 0 || rp[n] != m) return false;
    std::atomic<bool> ok{true};
    parallel_ranges(int64_t(n), int64_t(1) << 16, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi && ok.load(std::memory_order_relaxed); ++i) {
            const int64_t b = rp[i], e = rp[i + 1];
            if (b < 0 || e < b || e > m) {
                ok = false;
                return;
            }
            for (int64_t p = b; p < e; ++p) {
                if (col[p] <= i || col[p] >= n || (p > b && col[p] <= col[p - 1])) {
                    ok = false;
                    return;
                }
            }
        }
    });
    return ok;
}

// dst[0..count) = src[0..count), split over host threads for large copies.
void parallel_copy(int32_t *dst, const int32_t *src, int64_t count) {
    parallel_ranges(count, int64_t(1) << 22, [&](int64_t lo, int64_t hi) {
        std::memcpy(dst + lo, src + lo, size_t(hi - lo) * sizeof(int32_t));
    });
}

// Device bytes a request holds while active besides the shared live CSR:
// staged input and its output buffers.
size_t request_bytes(int32_t n, int64_t m) {
    return (size_t(n) + 1 + size_t(m)) * 4 + size_t(m) * 5 + 768;
}

cudaError_t support_step(ktruss_server *v, const kt::Live &g, int32_t *S, int *launches) {
    if (g.m < kAutoSmallEdges) {
        ++*launches;
        return kt::launch_support_edge(g, S, v->cnt, v->s);
    }
    return kt::launch_support_balanced(g, S, v->cnt, &v->bs, v->s, launches, nullptr);
}

// A request admitted in the current step: its CSR as staged on the device
// (request-local vertex ids) and its first slot in the live CSR.
struct Fresh {
    const int32_t *rp, *col;
    int32_t n, m, nb, mb;
};

}  // namespace

extern "C" {

int ktruss_server_create(ktruss_server **out, int32_t max_vertices, int64_t max_edges,
                         int32_t max_requests, int64_t request_bytes_budget, void *cuda_stream) {
    if (!out) return KTRUSS_EINVAL;
    *out = nullptr;
    if (max_vertices < 1 || max_edges < 1 || max_edges >= (int64_t(1) << 31) || max_requests < 1 ||
        request_bytes_budget < 0)
        return KTRUSS_EINVAL;
    ktruss_server *v = new (std::nothrow) ktruss_server();
    if (!v) return KTRUSS_ENOMEM;
    v->vcap = max_vertices;
    v->ecap = max_edges;
    v->slots = max_requests;
    v->budget = request_bytes_budget;
    v->s = static_cast<cudaStream_t>(cuda_stream);
    v->slot.resize(size_t(max_requests));
    const size_t nb = (size_t(max_vertices) + 1) * 4, eb = size_t(max_edges) * 4;
    const size_t sb = size_t(max_requests) * 4;
    const int32_t et = kt::compact_tiles(int32_t(max_edges)) + 1;
    const int32_t vt = kt::compact_tiles(max_vertices) + 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) v->owned.push_back(*p);
    };
    for (int b = 0; b < 2; ++b) {
        A((void **)&v->rp[b], nb);
        A((void **)&v->col[b], eb);
        A((void **)&v->eid[b], eb);
        A((void **)&v->gid[b], nb);
    }
    A((void **)&v->S, eb);
    A((void **)&v->S2, eb);
    A((void **)&v->pos, eb);
    A((void **)&v->vmap, nb);
    A((void **)&v->ust.ldeg, nb);
    A((void **)&v->ust.flag, nb);
    A((void **)&v->ust.nz, 16);
    A((void **)&v->keep, size_t(max_edges));
    A((void **)&v->fin, size_t(max_requests));
    A((void **)&v->thr, sb);
    A((void **)&v->kept_g, sb);
    A((void **)&v->removed_g, sb);
    A((void **)&v->rounds_g, sb);
    A((void **)&v->upd_s, size_t(max_requests));
    A((void **)&v->listed_s, sb);
    A((void **)&v->kept_s, sb);
    A((void **)&v->mask_ptr, size_t(max_requests) * sizeof(void *));
    A((void **)&v->sup_ptr, size_t(max_requests) * sizeof(void *));
    A((void **)&v->etile_count, size_t(et) * 4);
    A((void **)&v->etile_off, size_t(et) * 4);
    A((void **)&v->vtile_count, size_t(vt) * 4);
    A((void **)&v->vtile_off, size_t(vt) * 4);
    A((void **)&v->cnt, 3 * sizeof(kt::RoundCounters));
    A((void **)&v->verr, 16);
    if (e == cudaSuccess) e = kt::balanced_scratch_alloc(&v->bs, max_vertices, max_edges);
    if (e == cudaSuccess) e = kt::balanced_side_create(&v->bs);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->cnt_host, 3 * sizeof(kt::RoundCounters));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->verr_host, 16);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->fin_host, size_t(max_requests));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->rounds_host, sb);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->ptr_host, 2 * size_t(max_requests) * sizeof(void *));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->thr_host, sb);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->rp[0], 0, 4, v->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->ust.flag, 0, nb, v->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->s);
    if (e != cudaSuccess) {
        const int rc = map_err(e);
        server_release(v);
        return rc;
    }
    *out = v;
    return KTRUSS_OK;
}

void ktruss_server_free(ktruss_server *srv) { server_release(srv); }

int ktruss_server_set_option(ktruss_server *srv, int32_t key, int64_t value) {
    if (!srv) return KTRUSS_EINVAL;
    if (key == KTRUSS_OPT_REORDER) {
        if (value != 0 && value != 1) return KTRUSS_EINVAL;
        srv->reorder = int(value);
        return KTRUSS_OK;
    }
    if (key != KTRUSS_OPT_UPDATE) return KTRUSS_EINVAL;
    if (value != KTRUSS_UPDATE_NEVER && value != KTRUSS_UPDATE_ALWAYS &&
        value != KTRUSS_UPDATE_AUTO)
        return KTRUSS_EINVAL;
    srv->update_mode = int(value);
    return KTRUSS_OK;
}

int ktruss_server_submit(ktruss_server *srv, int32_t n, int64_t m, const int32_t *row_ptr,
                         const int32_t *col, int32_t K, uint8_t *mask_out, int32_t *support_out,
                         int64_t *ticket_out) {
    if (!srv || n < 0 || m < 0 || K < 2 || !row_ptr || (m > 0 && (!col || !mask_out)))
        return KTRUSS_EINVAL;
    if (n > srv->vcap || m > srv->ecap ||
        int64_t(request_bytes(n, m)) > srv->budget)
        return KTRUSS_EINVAL;  // could never be admitted
    Request r;
    r.n = n;
    r.m = m;
    r.K = K;
    const size_t bytes = request_bytes(n, m);
    // Staged requests hold their budget while queued; staging only while no
    // host-copied request waits keeps every staged request ahead of every
    // host-copied one, so that admission in arrival order cannot stall on a
    // budget that queued requests behind it hold.
    if (m > 0 && srv->used + int64_t(bytes) <= srv->budget &&
        (srv->queue.empty() || srv->queue.back().staged)) {
        // room in the budget now: stage the input on the device straight from
        // the caller's arrays and validate it there (no host copy)
        void *p = nullptr;
        if (kt::cache_get(input_bytes(n, m), &p) == cudaSuccess) {
            cudaStream_t s = srv->s;
            int32_t *din = static_cast<int32_t *>(p);
            cudaError_t e = cudaMemcpyAsync(din, row_ptr, (size_t(n) + 1) * 4,
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(din + n + 1, col, size_t(m) * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(srv->verr, 0, 4, s);
            if (e == cudaSuccess) e = kt::launch_validate(din, din + n + 1, n, m, srv->verr, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(srv->verr_host, srv->verr, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess || *srv->verr_host != 0) {
                kt::cache_put(p, input_bytes(n, m));
                return e != cudaSuccess ? map_err(e) : KTRUSS_EINVAL;
            }
            r.din = din;
            r.staged = true;
            srv->used += int64_t(bytes);
        } else {
            cudaGetLastError();  // no memory to stage now: keep a host copy
        }
    }
    if (!r.staged) {
        if (!valid_csr(n, m, row_ptr, col)) return KTRUSS_EINVAL;
        r.rp.reset(new (std::nothrow) int32_t[size_t(n) + 1]);
        if (m > 0) r.col.reset(new (std::nothrow) int32_t[size_t(m)]);
        if (!r.rp || (m > 0 && !r.col)) return KTRUSS_ENOMEM;
        parallel_copy(r.rp.get(), row_ptr, int64_t(n) + 1);
        if (m > 0) parallel_copy(r.col.get(), col, m);
    }
    r.ticket = srv->next_ticket++;
    r.mask_out = mask_out;
    r.support_out = support_out;
    if (ticket_out) *ticket_out = r.ticket;
    srv->queue.push_back(std::move(r));
    return KTRUSS_OK;
}

int ktruss_server_step(ktruss_server *srv, int32_t *num_done) {
    if (!srv) return KTRUSS_EINVAL;
    if (num_done) *num_done = 0;
    cudaStream_t s = srv->s;
    int launches = 0;
    int32_t finished = 0;
    std::vector<Request> admitted;
    std::vector<Fresh> fresh;
    // ---- 1. admission, in arrival order
    while (!srv->queue.empty()) {
        Request &r = srv->queue.front();
        if (r.m == 0) {  // nothing to peel: 0 rounds, no output
            srv->done_tickets.push_back(r.ticket);
            srv->done_rounds.push_back(0);
            ++finished;
            srv->queue.pop_front();
            continue;
        }
        int32_t sid = -1;
        for (int32_t k = 0; k < srv->slots; ++k)
            if (!srv->slot[size_t(k)].used) {
                sid = k;
                break;
            }
        const size_t bytes = request_bytes(r.n, r.m);
        if (sid < 0 || int64_t(srv->n_live) + r.n > srv->vcap ||
            int64_t(srv->m_live) + r.m > srv->ecap ||
            (!r.staged && srv->used + int64_t(bytes) > srv->budget))
            break;
        Slot &sl = srv->slot[size_t(sid)];
        {
            // take every buffer first, so that a failure leaves the request queued as it was
            void *din = r.din, *dm = nullptr, *ds = nullptr, *dre = nullptr;
            const bool relabel = srv->reorder && r.m > 0;
            cudaError_t e = din ? cudaSuccess : kt::cache_get(input_bytes(r.n, r.m), &din);
            if (e == cudaSuccess) e = kt::cache_get(size_t(r.m), &dm);
            if (e == cudaSuccess && r.support_out) e = kt::cache_get(size_t(r.m) * 4, &ds);
            if (e == cudaSuccess && relabel) e = kt::cache_get(relabel_bytes(r.n, r.m), &dre);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (dm) kt::cache_put(dm, size_t(r.m));
                if (ds) kt::cache_put(ds, size_t(r.m) * 4);
                if (din && !r.staged) kt::cache_put(din, input_bytes(r.n, r.m));
                return map_err(e);
            }
            sl.din = static_cast<int32_t *>(din);
            sl.din_bytes = input_bytes(r.n, r.m);
            sl.dmask = static_cast<uint8_t *>(dm);
            sl.dsup = static_cast<int32_t *>(ds);
            sl.dre = static_cast<int32_t *>(dre);
            sl.dre_bytes = dre ? relabel_bytes(r.n, r.m) : 0;
            r.din = nullptr;
        }
        sl.used = true;
        sl.ticket = r.ticket;
        sl.n = r.n;
        sl.m = r.m;
        sl.bytes = bytes;
        sl.host_mask = r.mask_out;
        sl.host_sup = r.support_out;
        int32_t *drp = sl.din, *dcol = sl.din + r.n + 1;
        if (!r.staged) {
            srv->used += int64_t(bytes);
            SV_CK(cudaMemcpyAsync(drp, r.rp.get(), (size_t(r.n) + 1) * 4, cudaMemcpyHostToDevice,
                                  s));
            if (r.m > 0)
                SV_CK(cudaMemcpyAsync(dcol, r.col.get(), size_t(r.m) * 4, cudaMemcpyHostToDevice,
                                      s));
        }
        // the request's vertices numbered by ascending degree (as a loaded
        // graph's are), the balanced scratch serving as the sort's memory
        // (it is idle during admission); slots map back to input edges
        const int32_t *emap = nullptr;
        if (sl.dre) {
            int32_t *rpR = sl.dre, *colR = sl.dre + r.n + 1, *eidR = colR + r.m;
            SV_CK(kt::launch_reorder(drp, dcol, r.n, r.m, srv->bs.base, rpR, colR, eidR, s));
            drp = rpR;
            dcol = colR;
            emap = eidR;
        }
        SV_CK(kt::launch_server_append(drp, dcol, r.n, int32_t(r.m), srv->n_live, srv->m_live, sid,
                                       srv->rp[srv->cur], srv->col[srv->cur], srv->eid[srv->cur],
                                       srv->gid[srv->cur], s, emap));
        ++launches;
        srv->ptr_host[2 * sid] = sl.dmask;
        srv->ptr_host[2 * sid + 1] = sl.dsup;
        srv->thr_host[sid] = r.K - 2;
        SV_CK(cudaMemcpyAsync(srv->mask_ptr + sid, &srv->ptr_host[2 * sid], sizeof(void *),
                              cudaMemcpyHostToDevice, s));
        SV_CK(cudaMemcpyAsync(srv->sup_ptr + sid, &srv->ptr_host[2 * sid + 1], sizeof(void *),
                              cudaMemcpyHostToDevice, s));
        SV_CK(cudaMemcpyAsync(srv->thr + sid, &srv->thr_host[sid], 4, cudaMemcpyHostToDevice, s));
        SV_CK(cudaMemsetAsync(srv->rounds_g + sid, 0, 4, s));
        SV_CK(cudaMemsetAsync(srv->upd_s + sid, 1, 1, s));  // supports computed below
        fresh.push_back(Fresh{drp, dcol, r.n, int32_t(r.m), srv->n_live, srv->m_live});
        srv->n_live += r.n;
        srv->m_live += int32_t(r.m);
        admitted.push_back(std::move(r));
        srv->queue.pop_front();
    }
    kt::trace_phase(s, "server admission");
    const auto t_step = std::chrono::steady_clock::now();
    // ---- 2. one peel round over every active request
    if (srv->m_live > 0) {
        const int c = srv->cur, o = c ^ 1;
        const kt::Live g{srv->rp[c], srv->col[c], srv->eid[c], srv->n_live, srv->m_live};
        SV_CK(cudaMemsetAsync(srv->cnt, 0, 3 * sizeof(kt::RoundCounters), s));
        // The requests admitted now follow the older ones in the live CSR:
        // the older requests are the prefix [0, n_old) x [0, m_old), itself a
        // valid CSR (the first admitted vertex's row starts at m_old).
        const int32_t n_old = fresh.empty() ? g.n : fresh.front().nb;
        const int32_t m_old = fresh.empty() ? g.m : fresh.front().mb;
        // a support step per request admitted now, over its own CSR (its
        // supports land at its first slot) ...
        if (!fresh.empty()) {
            SV_CK(cudaMemsetAsync(srv->S + m_old, 0, size_t(g.m - m_old) * 4, s));
            for (const Fresh &f : fresh) {
                const kt::Live rg{f.rp, f.col, nullptr, f.n, f.m};
                SV_CK(support_step(srv, rg, srv->S + f.mb, &launches));
            }
        }
        // ... and one over the older requests: all of them when no supports
        // were carried, else those whose own rule chose a support step (the
        // tasks of every other slot skipped)
        if (m_old > 0) {
            const kt::Live prefix{g.rp, g.col, g.eid, n_old, m_old};
            if (!srv->any_valid) {
                SV_CK(cudaMemsetAsync(srv->S, 0, size_t(m_old) * 4, s));
                SV_CK(support_step(srv, prefix, srv->S, &launches));
            } else if (srv->need_slots > 0) {
                SV_CK(kt::launch_batch_zero(prefix, srv->gid[c], srv->upd_s, srv->S, s,
                                            &launches));
                kt::Live masked = prefix;
                masked.gid = srv->gid[c];
                masked.skip = srv->upd_s;
                SV_CK(support_step(srv, masked, srv->S, &launches));
            }
        }
        kt::trace_phase(s, "server support steps");
        SV_CK(cudaMemsetAsync(srv->kept_g, 0, size_t(srv->slots) * 4, s));
        SV_CK(cudaMemsetAsync(srv->removed_g, 0, size_t(srv->slots) * 4, s));
        const bool track = srv->update_mode != KTRUSS_UPDATE_NEVER;
        const kt::UpdateScratch us = kt::update_scratch(&srv->bs);
        if (track) {
            SV_CK(cudaMemsetAsync(srv->listed_s, 0, size_t(srv->slots) * 4, s));
            SV_CK(cudaMemsetAsync(srv->kept_s, 0, size_t(srv->slots) * 4, s));
        }
        SV_CK(kt::launch_server_prune(g, srv->S, srv->gid[c], srv->thr, srv->keep, srv->kept_g,
                                      srv->removed_g, s, &launches, track ? us.list : nullptr,
                                      &srv->cnt[0].removed_tri, track ? srv->listed_s : nullptr));
        // the round tail carries the supports of surviving edges into S2 when
        // the update may run; each slot then takes its own choice
        SV_CK(kt::launch_server_round_tail(
            g, srv->S, srv->keep, srv->kept_g, srv->removed_g, srv->fin, srv->rounds_g,
            srv->slots, srv->gid[c], srv->vmap, srv->vtile_count, srv->vtile_off, srv->cnt + 1,
            srv->etile_count, srv->etile_off, srv->cnt, srv->pos, srv->rp[o], srv->col[o],
            srv->eid[o], srv->gid[o], srv->mask_ptr, srv->sup_ptr, s, &launches,
            track ? srv->S2 : nullptr, track ? srv->kept_s : nullptr));
        kt::trace_phase(s, "server prune + round tail");
        const int32_t mode = srv->update_mode == KTRUSS_UPDATE_ALWAYS ? 1 : 2;
        if (track)
            SV_CK(kt::launch_server_decide(srv->slots, srv->kept_s, srv->listed_s, mode, srv->upd_s,
                                           srv->cnt + 2, s, &launches));
        SV_CK(cudaMemcpyAsync(srv->cnt_host, srv->cnt, 3 * sizeof(kt::RoundCounters),
                              cudaMemcpyDeviceToHost, s));
        SV_CK(cudaMemcpyAsync(srv->fin_host, srv->fin, size_t(srv->slots), cudaMemcpyDeviceToHost, s));
        SV_CK(cudaMemcpyAsync(srv->rounds_host, srv->rounds_g, size_t(srv->slots) * 4,
                              cudaMemcpyDeviceToHost, s));
        SV_CK(cudaStreamSynchronize(s));
        const kt::RoundCounters c0 = srv->cnt_host[0], c2 = srv->cnt_host[2];
        if (c0.error) return (c0.error & kt::kDevErrTimeout) ? KTRUSS_ETIMEOUT : KTRUSS_ECUDA;
        const int32_t nlist = c0.removed_tri;
        srv->any_valid = track && c2.kept > c2.removed_tri;
        srv->need_slots = track ? c2.removed_tri : 0;
        if (srv->any_valid && nlist > 0) {
            // the update of the updated slots runs on this step's graph and
            // subtracts into the carried supports through the position map
            kt::Live old = g;
            old.gid = srv->gid[c];
            srv->ust.ldeg_valid = false;
            SV_CK(kt::launch_support_update(old, srv->keep, us.list, nlist, srv->S,
                                            &srv->cnt[2].triangles, us, &srv->ust, s, &launches,
                                            srv->pos, srv->S2, srv->upd_s));
        }
        kt::trace_phase(s, "server update");
        if (kt::trace_on())
            std::fprintf(stderr,
                         "[ktruss server] step %lld admitted %d live %d -> %d edges, listed %d, "
                         "recomputed slots next %d, %s, %.3f ms to the round tail\n",
                         (long long)srv->steps, int(admitted.size()), int(g.m), int(c0.kept),
                         int(nlist), int(srv->need_slots),
                         srv->any_valid ? "update" : "support step next",
                         std::chrono::duration<double, std::milli>(
                             std::chrono::steady_clock::now() - t_step).count());
        srv->m_live = c0.kept;
        srv->n_live = srv->cnt_host[1].kept;
        srv->cur = o;
        if (track) std::swap(srv->S, srv->S2);
        ++srv->steps;
        // ---- 3. finished requests: outputs to the caller, memory back
        std::vector<int32_t> fin_slots;
        for (int32_t k = 0; k < srv->slots; ++k) {
            Slot &sl = srv->slot[size_t(k)];
            if (!sl.used || !srv->fin_host[k]) continue;
            const auto t_copy = std::chrono::steady_clock::now();
            SV_CK(cudaMemcpyAsync(sl.host_mask, sl.dmask, size_t(sl.m), cudaMemcpyDeviceToHost, s));
            if (sl.host_sup)
                SV_CK(cudaMemcpyAsync(sl.host_sup, sl.dsup, size_t(sl.m) * 4,
                                      cudaMemcpyDeviceToHost, s));
            if (kt::trace_phases()) {
                SV_CK(cudaStreamSynchronize(s));
                std::fprintf(stderr, "[ktruss server] outputs of slot %d: %d edges, %.3f ms\n",
                             int(k), int(sl.m),
                             std::chrono::duration<double, std::milli>(
                                 std::chrono::steady_clock::now() - t_copy).count());
            }
            fin_slots.push_back(k);
        }
        if (!fin_slots.empty()) SV_CK(cudaStreamSynchronize(s));
        kt::trace_phase(s, "server finished outputs");
        for (int32_t k : fin_slots) {
            Slot &sl = srv->slot[size_t(k)];
            srv->done_tickets.push_back(sl.ticket);
            srv->done_rounds.push_back(srv->rounds_host[k]);
            ++finished;
            kt::cache_put(sl.din, sl.din_bytes);
            if (sl.dre) kt::cache_put(sl.dre, sl.dre_bytes);
            kt::cache_put(sl.dmask, size_t(sl.m));
            if (sl.dsup) kt::cache_put(sl.dsup, size_t(sl.m) * 4);
            srv->used -= int64_t(sl.bytes);
            sl = Slot{};
        }
    } else {
        SV_CK(cudaStreamSynchronize(s));
    }
    if (num_done) *num_done = finished;
    return KTRUSS_OK;
}

int ktruss_server_take_done(ktruss_server *srv, int64_t *tickets, int32_t *rounds, int32_t max,
                            int32_t *count) {
    if (!srv || !count || max < 0 || (max > 0 && !tickets)) return KTRUSS_EINVAL;
    const int32_t k = int32_t(std::min<size_t>(size_t(max), srv->done_tickets.size()));
    for (int32_t i = 0; i < k; ++i) {
        tickets[i] = srv->done_tickets[size_t(i)];
        if (rounds) rounds[i] = srv->done_rounds[size_t(i)];
    }
    srv->done_tickets.erase(srv->done_tickets.begin(), srv->done_tickets.begin() + k);
    srv->done_rounds.erase(srv->done_rounds.begin(), srv->done_rounds.begin() + k);
    *count = k;
    return KTRUSS_OK;
}

int ktruss_server_status(const ktruss_server *srv, int32_t *queued, int32_t *active,
                         int64_t *live_edges) {
    if (!srv) return KTRUSS_EINVAL;
    if (queued) *queued = int32_t(srv->queue.size());
    if (active) {
        int32_t a = 0;
        for (const Slot &sl : srv->slot) a += sl.used ? 1 : 0;
        *active = a;
    }
    if (live_edges) *live_edges = srv->m_live;
    return KTRUSS_OK;
}

}  // extern "C"
