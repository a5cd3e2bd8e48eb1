// Batched peeling: many graphs, each with its own K, peeled together.
//
// A batch is one block-diagonal strictly upper-triangular CSR: graph g owns
// the vertices [vo[g], vo[g+1]) and every edge joins two vertices of one graph,
// so no triangle spans two graphs and the support step (Alg. 3) of the whole
// batch computes every graph's supports at once.  Pruning (Alg. 1 Step 2)
// uses the threshold K_g - 2 of the edge's graph.  Graphs converge at
// different rounds: a graph whose round removed nothing is finished, its live
// edges get their final outputs and leave the live set at that round's
// compaction, so later rounds only touch unfinished graphs.  Every graph goes
// through exactly the bulk rounds of its solo run.
#include "ktruss_internal.cuh"

namespace kt {
namespace {

constexpr int kWarpsPerTile = kCompactThreads / 32;
constexpr int kWarpSpan = kCompactTile / kWarpsPerTile;

// gid[v] = graph owning vertex v (largest g with vo[g] <= v).
__global__ void graph_of_vertex_kernel(const int32_t *__restrict__ vo, int32_t G, int32_t n,
                                       int32_t *__restrict__ gid) {
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t lo = 0, hi = G - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (vo[mid] <= v) lo = mid; else hi = mid - 1;
    }
    gid[v] = lo;
}

// Flags edges that join two graphs (the batch must be block diagonal).
__global__ void batch_validate_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                      int32_t n, const int32_t *__restrict__ gid,
                                      int32_t *__restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += warps) {
        const int32_t gi = gid[i];
        int32_t bad = 0;
        for (int32_t p = rp[i] + lane; p < rp[i + 1]; p += 32) bad |= gid[col[p]] != gi;
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, 16);
    }
}

// Per live edge: keep flag (support >= K_g - 2) and, per graph, whether this
// round kept some edge (kept_g) and removed some edge (removed_g): both are
// 0/1 flags set with a plain store after a read shows them unset.  Removed
// edges with S > 0 are appended to list (when given) at positions taken from
// *list_count (and, when listed_g is given, counted per graph); when ldeg is
// given, each removed edge (u, v) subtracts one from ldeg[v].
__global__ void __launch_bounds__(256)
batch_prune_kernel(const int32_t *__restrict__ S, const int32_t *__restrict__ col, int32_t m,
                   const int32_t *__restrict__ gid, const int32_t *__restrict__ thr,
                   uint8_t *__restrict__ keep, int32_t *kept_g, int32_t *removed_g,
                   int32_t *__restrict__ list, int32_t *list_count, int32_t *__restrict__ ldeg,
                   int32_t *__restrict__ listed_g) {
    const int lane = threadIdx.x & 31;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int32_t g = -1;
    bool k = false;
    int32_t sv = 0;
    if (e < m) {
        const int32_t v = col[e];
        g = gid[v];
        sv = S[e];
        k = sv >= thr[g];
        keep[e] = k;
        int32_t *f = k ? kept_g + g : removed_g + g;
        if (*f == 0) *f = 1;  // a stale 0 only repeats the store
        if (!k && ldeg) atomicSub(ldeg + v, 1);
    }
    if (list) {
        const uint32_t b = __ballot_sync(0xffffffffu, e < m && !k && sv > 0);
        if (b) {
            int32_t at = 0;
            if (lane == __ffs(b) - 1) at = atomicAdd(list_count, __popc(b));
            at = __shfl_sync(0xffffffffu, at, __ffs(b) - 1);
            if ((b >> lane) & 1u) list[at + __popc(b & ((1u << lane) - 1u))] = int32_t(e);
            if (listed_g) {
                const bool mine = (b >> lane) & 1u;
                const uint32_t peers = __match_any_sync(0xffffffffu, mine ? g : -1);
                if (mine && lane == __ffs(peers) - 1) atomicAdd(listed_g + g, __popc(peers));
            }
        }
    }
}

// Per graph: count the round for graphs that had live edges; a graph with
// live edges and no removal is finished.
__global__ void batch_done_kernel(int32_t G, const int32_t *__restrict__ kept_g,
                                  const int32_t *__restrict__ removed_g,
                                  uint8_t *__restrict__ done, int32_t *__restrict__ rounds_g) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= G) return;
    const int32_t g = int32_t(t);
    if (kept_g[g] || removed_g[g]) {
        rounds_g[g] += 1;
        done[g] = removed_g[g] == 0;
    }
}

// First pass of the per-graph rule: cnt->forced = graphs whose listed edges
// exceed a quarter of their survivors and number at least kRecomputeMinListed.
__global__ void batch_force_kernel(int32_t G, const int32_t *__restrict__ vo,
                                   const int32_t *__restrict__ rp_new,
                                   const int32_t *__restrict__ listed_g, RoundCounters *cnt) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= G) return;
    const int32_t g = int32_t(t);
    const int32_t kept = rp_new[vo[g + 1]] - rp_new[vo[g]];
    const int32_t listed = listed_g[g];
    if (kept > 0 && listed >= kRecomputeMinListed && int64_t(listed) * 4 > kept)
        atomicAdd(&cnt->forced, 1);
}

// Per graph after a round's compaction (rp_new: the new row pointers, graph g
// owns vertices [vo[g], vo[g+1])): its surviving edges, and whether its next
// supports come from the update of this round (upd_g = 1) or from a support
// step (0).  mode: 0 never update, 1 always, 2 the kRecomputeMinListed rule
// (cnt->forced: the graphs of batch_force_kernel).  Counts the graphs that stay live
// (cnt->kept) and those that need a support step (cnt->removed_tri).
__global__ void batch_decide_kernel(int32_t G, const int32_t *__restrict__ vo,
                                    const int32_t *__restrict__ rp_new,
                                    const int32_t *__restrict__ listed_g, int32_t mode,
                                    uint8_t *__restrict__ upd_g, RoundCounters *cnt) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= G) return;
    const int32_t g = int32_t(t);
    const int32_t kept = rp_new[vo[g + 1]] - rp_new[vo[g]];
    const int32_t listed = listed_g[g];
    const bool upd = kept > 0 && (mode == 1 || (mode == 2 && (int64_t(listed) * 4 <= kept ||
                                                             (listed < kRecomputeMinListed &&
                                                              cnt->forced == 0))));
    upd_g[g] = upd ? 1 : 0;
    if (kept > 0) {
        atomicAdd(&cnt->kept, 1);
        if (!upd) atomicAdd(&cnt->removed_tri, 1);
    }
}

// S[e] = 0 for the live edges of graphs whose next supports come from a
// support step (upd_g == 0).
__global__ void batch_zero_kernel(const int32_t *__restrict__ col, int32_t m,
                                  const int32_t *__restrict__ gid,
                                  const uint8_t *__restrict__ upd_g, int32_t *__restrict__ S) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride)
        if (!upd_g[gid[col[e]]]) S[e] = 0;
}

__device__ __forceinline__ bool stays(const uint8_t *keep, const uint8_t *done, const int32_t *gid,
                                      const int32_t *col, int64_t e) {
    return keep[e] && !done[gid[col[e]]];
}

__global__ void __launch_bounds__(kCompactThreads)
batch_count_kernel(const uint8_t *__restrict__ keep, const uint8_t *__restrict__ done,
                   const int32_t *__restrict__ gid, const int32_t *__restrict__ col, int32_t m,
                   int32_t *__restrict__ tile_count) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kCompactTile + int64_t(w) * kWarpSpan + lane;
    int32_t c = 0;
#pragma unroll 4
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t e = base + j * 32;
        c += (e < m && stays(keep, done, gid, col, e)) ? 1 : 0;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) warp_tot[w] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int k = 0; k < kWarpsPerTile; ++k) t += warp_tot[k];
        tile_count[blockIdx.x] = t;
    }
}

// Compaction of the edges that stay; edges that leave get their outputs: the
// kept edges of a finished graph mask 1 and their support, removed edges 0.
__global__ void __launch_bounds__(kCompactThreads)
batch_compact_kernel(const int32_t *__restrict__ col, const int32_t *__restrict__ eid,
                     const int32_t *__restrict__ S, const uint8_t *__restrict__ keep,
                     const uint8_t *__restrict__ done, const int32_t *__restrict__ gid, int32_t m,
                     const int32_t *__restrict__ tile_off, int32_t *__restrict__ pos,
                     int32_t *__restrict__ col_out, int32_t *__restrict__ eid_out,
                     uint8_t *__restrict__ mask_out, int32_t *__restrict__ support_out,
                     int32_t *__restrict__ S_out) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kCompactTile + int64_t(w) * kWarpSpan + lane;
    uint32_t ballots[kCompactItemsPerThread];
    int32_t c = 0;
#pragma unroll
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t e = base + j * 32;
        ballots[j] = __ballot_sync(0xffffffffu, e < m && stays(keep, done, gid, col, e));
        c += __popc(ballots[j]);
    }
    if (lane == 0) warp_tot[w] = c;
    __syncthreads();
    int32_t run = tile_off[blockIdx.x];
    for (int k = 0; k < w; ++k) run += warp_tot[k];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t e = base + j * 32;
        const int32_t p = run + __popc(ballots[j] & lt);
        if (e < m) {
            pos[e] = p;
            const int32_t id = eid ? eid[e] : int32_t(e);
            if ((ballots[j] >> lane) & 1u) {
                col_out[p] = col[e];
                eid_out[p] = id;
                if (S_out) S_out[p] = S[e];
            } else {
                const bool k = keep[e];
                mask_out[id] = k ? 1 : 0;
                if (support_out) support_out[id] = k ? S[e] : 0;
            }
        }
        run += __popc(ballots[j]);
    }
}

}  // namespace

cudaError_t launch_graph_of_vertex(const int32_t *vo, int32_t G, int32_t n, int32_t *gid,
                                   cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    graph_of_vertex_kernel<<<int((int64_t(n) + 255) / 256), 256, 0, s>>>(vo, G, n, gid);
    return cudaGetLastError();
}

cudaError_t launch_batch_validate(const int32_t *rp, const int32_t *col, int32_t n,
                                  const int32_t *gid, int32_t *err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (int64_t(n) * 32 + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    batch_validate_kernel<<<int(blocks), 256, 0, s>>>(rp, col, n, gid, err);
    return cudaGetLastError();
}

cudaError_t launch_batch_keep(const Live &g, const int32_t *S, const int32_t *gid,
                              const int32_t *thr, uint8_t *keep, int32_t *kept_g,
                              int32_t *removed_g, cudaStream_t s, int *launches, int32_t *list,
                              int32_t *list_count, int32_t *listed_g) {
    if (g.m == 0) return cudaSuccess;
    batch_prune_kernel<<<int((int64_t(g.m) + 255) / 256), 256, 0, s>>>(S, g.col, g.m, gid, thr, keep, kept_g,
                                                         removed_g, list, list_count, nullptr,
                                                         listed_g);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_batch_prune(const Live &g, const int32_t *S, const int32_t *gid,
                               const int32_t *thr, uint8_t *keep, int32_t *kept_g,
                               int32_t *removed_g, uint8_t *done, int32_t *rounds_g, int32_t G,
                               int32_t *tile_count, int32_t *tile_off, RoundCounters *cnt,
                               cudaStream_t s, int *launches, int32_t *list, int32_t *ldeg,
                               int32_t *listed_g) {
    if (list) {
        cudaError_t e = cudaMemsetAsync(&cnt->removed_tri, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    }
    batch_prune_kernel<<<int((int64_t(g.m) + 255) / 256), 256, 0, s>>>(S, g.col, g.m, gid, thr, keep, kept_g,
                                                         removed_g, list, &cnt->removed_tri, ldeg,
                                                         listed_g);
    batch_done_kernel<<<int((int64_t(G) + 255) / 256), 256, 0, s>>>(G, kept_g, removed_g, done, rounds_g);
    const int32_t tiles = compact_tiles(g.m);
    batch_count_kernel<<<tiles, kCompactThreads, 0, s>>>(keep, done, gid, g.col, g.m, tile_count);
    *launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // scan of the tile counts (the single-graph kernels' scan, which ignores S
    // when given tile counts directly)
    return launch_scan_tiles(tile_count, tiles, tile_off, cnt, s, launches);
}

cudaError_t launch_batch_decide(int32_t G, const int32_t *vo, const int32_t *rp_new,
                                const int32_t *listed_g, int32_t mode, uint8_t *upd_g,
                                RoundCounters *cnt, cudaStream_t s, int *launches) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(RoundCounters), s);
    if (e != cudaSuccess) return e;
    if (mode == 2) {
        batch_force_kernel<<<int((int64_t(G) + 255) / 256), 256, 0, s>>>(G, vo, rp_new, listed_g, cnt);
        ++*launches;
    }
    batch_decide_kernel<<<int((int64_t(G) + 255) / 256), 256, 0, s>>>(G, vo, rp_new, listed_g, mode, upd_g, cnt);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_batch_zero(const Live &g, const int32_t *gid, const uint8_t *upd_g, int32_t *S,
                              cudaStream_t s, int *launches) {
    if (g.m == 0) return cudaSuccess;
    int64_t blocks = (int64_t(g.m) + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    batch_zero_kernel<<<int(blocks), 256, 0, s>>>(g.col, g.m, gid, upd_g, S);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_batch_compact(const Live &in, const int32_t *S, const uint8_t *keep,
                                 const uint8_t *done, const int32_t *gid, const int32_t *tile_off,
                                 const RoundCounters *cnt, int32_t *pos, int32_t *rp_out,
                                 int32_t *col_out, int32_t *eid_out, uint8_t *mask_out,
                                 int32_t *support_out, cudaStream_t s, int *launches,
                                 int32_t *S_out) {
    const int32_t tiles = compact_tiles(in.m);
    if (tiles > 0) {
        batch_compact_kernel<<<tiles, kCompactThreads, 0, s>>>(
            in.col, in.eid, S, keep, done, gid, in.m, tile_off, pos, col_out, eid_out, mask_out,
            support_out, S_out);
        ++*launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_rowptr(in, pos, cnt, rp_out, s, launches);
}

}  // namespace kt
