// pruneEdges (Alg. 1 Step 2) and the per-round rewrite of the live CSR.
//
// The paper marks removed edges with zeros inside a zero-terminated CSR
// (Sec. III-D); here the surviving edges are instead compacted into a fresh,
// dense CSR every round, so that the next support step never walks over dead
// slots.  An edge leaves for good when it is removed, so its final outputs
// (mask 0, support 0) are written at that moment, at its input edge id.
//
// Tile geometry: a block of 256 threads owns kCompactTile = 4096 consecutive
// slots; warp w of the block owns slots [w*512, (w+1)*512) of the tile and
// walks them 32 at a time, so every global access is coalesced and the keep
// flags of a warp are exchanged with ballots.
#include "ktruss_internal.cuh"

namespace kt {
namespace {

constexpr int kWarpsPerTile = kCompactThreads / 32;
constexpr int kWarpSpan = kCompactTile / kWarpsPerTile;  // 512 slots per warp
static_assert(kWarpSpan == 32 * kCompactItemsPerThread, "tile geometry");

// Appends the lanes of `ballot` (this warp) to list at a position taken from
// *count with one atomic.
__device__ __forceinline__ void warp_append(uint32_t ballot, int lane, int32_t value,
                                            int32_t *__restrict__ list, int32_t *count) {
    if (!ballot) return;
    int32_t at = 0;
    if (lane == __ffs(ballot) - 1) at = atomicAdd(count, __popc(ballot));
    at = __shfl_sync(0xffffffffu, at, __ffs(ballot) - 1);
    if ((ballot >> lane) & 1u) list[at + __popc(ballot & ((1u << lane) - 1u))] = value;
}

// With a LoopCtl (device loop) the edge count, the threshold and whether the
// lower degrees are kept come from it; each block walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... (one tile per block in a host-sized launch).
__global__ void __launch_bounds__(kCompactThreads)
prune_count_kernel(const int32_t *__restrict__ S, int32_t m, int32_t thr,
                   int32_t *__restrict__ tile_count, uint8_t *__restrict__ keep,
                   int32_t *__restrict__ list, RoundCounters *cnt,
                   const int32_t *__restrict__ col, int32_t *__restrict__ ldeg,
                   const LoopCtl *lc) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    if (lc) {
        m = lc->m;
        thr = lc->thr;
        if (!lc->ldeg_valid) ldeg = nullptr;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t tiles = compact_tiles(m);
    for (int32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t base = int64_t(tile) * kCompactTile + int64_t(w) * kWarpSpan + lane;
        int32_t c = 0;
#pragma unroll 4
        for (int j = 0; j < kCompactItemsPerThread; ++j) {
            const int64_t e = base + j * 32;
            const int32_t sv = e < m ? __ldg(S + e) : 0;
            const bool k = e < m && sv >= thr;
            c += k ? 1 : 0;
            if (keep && e < m) keep[e] = k;
            if (ldeg && e < m && !k) atomicSub(ldeg + __ldg(col + e), 1);
            if (list)
                warp_append(__ballot_sync(0xffffffffu, e < m && !k && sv > 0), lane, int32_t(e),
                            list, &cnt->removed_tri);
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) warp_tot[w] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = 0;
            for (int k = 0; k < kWarpsPerTile; ++k) t += warp_tot[k];
            tile_count[tile] = t;
        }
        __syncthreads();
    }
}

// Exclusive scan of tile counts by one block; total -> cnt->kept.
__global__ void __launch_bounds__(1024)
scan_tiles_kernel(const int32_t *__restrict__ tile_count, int32_t tiles,
                  int32_t *__restrict__ tile_off, RoundCounters *cnt, const LoopCtl *lc) {
    __shared__ int32_t warp_sum[32];
    if (lc) tiles = compact_tiles(lc->m);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t per = (tiles + 1023) / 1024;
    const int32_t b = tid * per;
    const int32_t e = min(tiles, b + per);
    int32_t local = 0;
    for (int32_t k = b; k < e; ++k) local += tile_count[k];
    // block exclusive scan of `local`
    int32_t incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t v = warp_sum[lane];
        int32_t vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += u;
        }
        warp_sum[lane] = vi - v;  // exclusive
        if (lane == 31) cnt->kept = vi;
    }
    __syncthreads();
    int32_t run = warp_sum[w] + incl - local;
    for (int32_t k = b; k < e; ++k) {
        tile_off[k] = run;
        run += tile_count[k];
    }
}

// With a LoopCtl the kernel does nothing unless the round compacts; the edge
// count, the outputs of removed edges, their level and whether S is carried
// come from it.
__global__ void __launch_bounds__(kCompactThreads)
compact_kernel(const int32_t *__restrict__ col, const int32_t *__restrict__ eid,
               const int32_t *__restrict__ S, int32_t m, int32_t thr,
               const int32_t *__restrict__ tile_off, int32_t *__restrict__ pos,
               int32_t *__restrict__ col_out, int32_t *__restrict__ eid_out,
               uint8_t *__restrict__ mask_out, int32_t *__restrict__ support_out,
               int32_t *__restrict__ level_out, int32_t level, const uint8_t *__restrict__ keep_in,
               int32_t *__restrict__ S_out, const LoopCtl *lc) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    if (lc) {
        const int32_t a = lc->action;
        if (!(a & kActCompact)) return;
        m = lc->m;
        if (!(a & kActCarry)) S_out = nullptr;
        mask_out = lc->mask_out;
        support_out = lc->sup_out;
        level_out = lc->level_out;
        level = lc->level;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t tiles = compact_tiles(m);
    for (int32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t base = int64_t(tile) * kCompactTile + int64_t(w) * kWarpSpan + lane;
        uint32_t ballots[kCompactItemsPerThread];
        int32_t c = 0;
#pragma unroll
        for (int j = 0; j < kCompactItemsPerThread; ++j) {
            const int64_t e = base + j * 32;
            const bool keep = e < m && (keep_in ? keep_in[e] != 0 : __ldg(S + e) >= thr);
            ballots[j] = __ballot_sync(0xffffffffu, keep);
            c += __popc(ballots[j]);
        }
        if (lane == 0) warp_tot[w] = c;
        __syncthreads();
        int32_t run = tile_off[tile];
        for (int k = 0; k < w; ++k) run += warp_tot[k];
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int j = 0; j < kCompactItemsPerThread; ++j) {
            const int64_t e = base + j * 32;
            const int32_t p = run + __popc(ballots[j] & lt);
            if (e < m) {
                pos[e] = p;
                const int32_t id = eid ? __ldg(eid + e) : int32_t(e);
                if ((ballots[j] >> lane) & 1u) {
                    col_out[p] = __ldg(col + e);
                    eid_out[p] = id;
                    if (S_out) S_out[p] = S[e];
                } else {
                    if (mask_out) mask_out[id] = 0;
                    if (support_out) support_out[id] = 0;
                    if (level_out) level_out[id] = level;
                }
            }
            run += __popc(ballots[j]);
        }
        __syncthreads();  // warp_tot is rewritten by the next tile
    }
}

// With a LoopCtl: nothing unless the round compacts, edge count from it, and
// the threads loop over the rows.
__global__ void rowptr_kernel(const int32_t *__restrict__ rp_in, int32_t n, int32_t m,
                              const int32_t *__restrict__ pos, const RoundCounters *cnt,
                              int32_t *__restrict__ rp_out, const LoopCtl *lc) {
    if (lc) {
        if (!(lc->action & kActCompact)) return;
        m = lc->m;
    }
    const int32_t kept = cnt->kept;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t r = rp_in[i];
        rp_out[i] = r < m ? pos[r] : kept;
    }
}

__global__ void finalize_kernel(const int32_t *__restrict__ eid, const int32_t *__restrict__ S,
                                int32_t m, uint8_t *__restrict__ mask_out,
                                int32_t *__restrict__ support_out) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t id = eid ? eid[e] : int32_t(e);
    mask_out[id] = 1;
    if (support_out) support_out[id] = S[e];
}

}  // namespace

cudaError_t launch_prune_count(const int32_t *S, int32_t m, int32_t thr, int32_t *tile_count,
                               int32_t *tile_off, RoundCounters *cnt, cudaStream_t s,
                               int *launches, uint8_t *keep, int32_t *list, const int32_t *col,
                               int32_t *ldeg, const LoopCtl *lc) {
    // in the device loop m is the capacity: the grid is fixed, the kernels
    // read the live count (and the loop's end kernel resets removed_tri)
    const int32_t tiles = compact_tiles(m);
    if (list && !lc) {
        cudaError_t e = cudaMemsetAsync(&cnt->removed_tri, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    }
    if (tiles > 0) {
        const int32_t grid = lc ? (tiles < kLoopBlocks ? tiles : kLoopBlocks) : tiles;
        prune_count_kernel<<<grid, kCompactThreads, 0, s>>>(S, m, thr, tile_count, keep, list,
                                                            cnt, col, ldeg, lc);
        ++*launches;
    }
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tile_count, tiles, tile_off, cnt, lc);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_compact(const Live &in, const int32_t *S, int32_t thr, const int32_t *tile_off,
                           const RoundCounters *cnt, int32_t *pos, int32_t *rp_out,
                           int32_t *col_out, int32_t *eid_out, uint8_t *mask_out,
                           int32_t *support_out, cudaStream_t s, int *launches,
                           int32_t *level_out, int32_t level, const uint8_t *keep,
                           int32_t *S_out, const LoopCtl *lc) {
    const int32_t tiles = compact_tiles(in.m);
    if (tiles > 0) {
        const int32_t grid = lc ? (tiles < kLoopBlocks ? tiles : kLoopBlocks) : tiles;
        compact_kernel<<<grid, kCompactThreads, 0, s>>>(in.col, in.eid, S, in.m, thr, tile_off,
                                                        pos, col_out, eid_out, mask_out,
                                                        support_out, level_out, level, keep,
                                                        S_out, lc);
        ++*launches;
    }
    const int64_t rows = int64_t(in.n) + 1;
    int64_t rblocks = (rows + 255) / 256;
    if (lc && rblocks > kLoopBlocks) rblocks = kLoopBlocks;
    rowptr_kernel<<<int(rblocks), 256, 0, s>>>(in.rp, in.n, in.m, pos, cnt, rp_out, lc);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const int32_t *tile_count, int32_t tiles, int32_t *tile_off,
                              RoundCounters *cnt, cudaStream_t s, int *launches) {
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tile_count, tiles, tile_off, cnt, nullptr);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_rowptr(const Live &in, const int32_t *pos, const RoundCounters *cnt,
                          int32_t *rp_out, cudaStream_t s, int *launches) {
    const int64_t rows = int64_t(in.n) + 1;
    rowptr_kernel<<<int((rows + 255) / 256), 256, 0, s>>>(in.rp, in.n, in.m, pos, cnt, rp_out,
                                                           nullptr);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Live &g, const int32_t *S, uint8_t *mask_out,
                            int32_t *support_out, cudaStream_t s, int *launches) {
    if (g.m == 0) return cudaSuccess;
    finalize_kernel<<<int((int64_t(g.m) + 255) / 256), 256, 0, s>>>(g.eid, S, g.m, mask_out, support_out);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace kt
