// Device side of the K-truss request server (continuous batching).
//
// The server's live state is one strictly upper-triangular, block-diagonal
// CSR holding every active request's live graph: request slot s owns a
// contiguous range of vertices, gid[v] is the slot of vertex v, and eid[e] is
// the request-local index of live edge e.  Each step appends the requests
// admitted in it, runs one support step (Alg. 3) over all of them, prunes
// each with its own threshold (Alg. 1 Step 2) and rewrites the live CSR
// without the requests that finished, renumbering the surviving vertices so
// the live state stays dense.  Outputs of edges that leave go straight to the
// owning request's output buffers through per-slot device pointer tables.
#include "ktruss_internal.cuh"

namespace kt {
namespace {

constexpr int kWarpsPerTile = kCompactThreads / 32;
constexpr int kWarpSpan = kCompactTile / kWarpsPerTile;

// Appends a request's CSR (device copy of its input) at vertex base nb and
// edge base mb of the live CSR.
// emap (optional): request-local input edge of each slot of (rp_in, col_in)
// (the request's degree-ordered relabel); else slot e is input edge e.
__global__ void append_kernel(const int32_t *__restrict__ rp_in, const int32_t *__restrict__ col_in,
                              int32_t n, int32_t m, int32_t nb, int32_t mb, int32_t slot,
                              int32_t *__restrict__ rp, int32_t *__restrict__ col,
                              int32_t *__restrict__ eid, int32_t *__restrict__ gid,
                              const int32_t *__restrict__ emap) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = t; v <= n; v += stride) {
        rp[nb + v] = mb + rp_in[v];
        if (v < n) gid[nb + v] = slot;
    }
    for (int64_t e = t; e < m; e += stride) {
        col[mb + e] = nb + col_in[e];
        eid[mb + e] = emap ? emap[e] : int32_t(e);
    }
}

// Per slot (kept_g / removed_g: whether the round kept / removed some edge of
// the slot): the round counts for slots that had live edges; a slot whose
// round removed nothing, or removed every live edge, is finished.
__global__ void finish_kernel(int32_t slots, const int32_t *__restrict__ kept_g,
                              const int32_t *__restrict__ removed_g, uint8_t *__restrict__ fin,
                              int32_t *__restrict__ rounds_g) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= slots) return;
    const int32_t g = int32_t(t);
    if (kept_g[g] || removed_g[g]) {
        rounds_g[g] += 1;
        fin[g] = removed_g[g] == 0 || kept_g[g] == 0;
    } else {
        fin[g] = 0;
    }
}

// Tile counts of surviving vertices (their slot is not finished).
__global__ void __launch_bounds__(kCompactThreads)
vertex_count_kernel(const int32_t *__restrict__ gid, const uint8_t *__restrict__ fin, int32_t n,
                    int32_t *__restrict__ tile_count) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kCompactTile + int64_t(w) * kWarpSpan + lane;
    int32_t c = 0;
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t v = base + j * 32;
        c += (v < n && !fin[gid[v]]) ? 1 : 0;
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

// vmap[v] = new id of surviving vertex v (exclusive prefix of survivors).
__global__ void __launch_bounds__(kCompactThreads)
vertex_map_kernel(const int32_t *__restrict__ gid, const uint8_t *__restrict__ fin, int32_t n,
                  const int32_t *__restrict__ tile_off, int32_t *__restrict__ vmap) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kCompactTile + int64_t(w) * kWarpSpan + lane;
    uint32_t ballots[kCompactItemsPerThread];
    int32_t c = 0;
#pragma unroll
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t v = base + j * 32;
        ballots[j] = __ballot_sync(0xffffffffu, v < n && !fin[gid[v]]);
        c += __popc(ballots[j]);
    }
    if (lane == 0) warp_tot[w] = c;
    __syncthreads();
    int32_t run = tile_off[blockIdx.x];
    for (int k = 0; k < w; ++k) run += warp_tot[k];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t v = base + j * 32;
        if (v < n) vmap[v] = run + __popc(ballots[j] & lt);
        run += __popc(ballots[j]);
    }
}

__device__ __forceinline__ bool edge_stays(const uint8_t *keep, const uint8_t *fin,
                                           const int32_t *gid, const int32_t *col, int64_t e) {
    return keep[e] && !fin[gid[col[e]]];
}

__global__ void __launch_bounds__(kCompactThreads)
edge_count_kernel(const uint8_t *__restrict__ keep, const uint8_t *__restrict__ fin,
                  const int32_t *__restrict__ gid, const int32_t *__restrict__ col, int32_t m,
                  int32_t *__restrict__ tile_count) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kCompactTile + int64_t(w) * kWarpSpan + lane;
    int32_t c = 0;
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t e = base + j * 32;
        c += (e < m && edge_stays(keep, fin, gid, col, e)) ? 1 : 0;
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

// Compaction with vertex renumbering; leaving edges write their outputs into
// their request's buffers (mask 1 and the support for kept edges of a
// finished request, 0 for removed edges).
__global__ void __launch_bounds__(kCompactThreads)
edge_compact_kernel(const int32_t *__restrict__ col, const int32_t *__restrict__ eid,
                    const int32_t *__restrict__ S, const uint8_t *__restrict__ keep,
                    const uint8_t *__restrict__ fin, const int32_t *__restrict__ gid,
                    const int32_t *__restrict__ vmap, int32_t m,
                    const int32_t *__restrict__ tile_off, int32_t *__restrict__ pos,
                    int32_t *__restrict__ col_out, int32_t *__restrict__ eid_out,
                    uint8_t *const *__restrict__ mask_ptr, int32_t *const *__restrict__ sup_ptr,
                    int32_t *__restrict__ S_out) {
    __shared__ int32_t warp_tot[kWarpsPerTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kCompactTile + int64_t(w) * kWarpSpan + lane;
    uint32_t ballots[kCompactItemsPerThread];
    int32_t c = 0;
#pragma unroll
    for (int j = 0; j < kCompactItemsPerThread; ++j) {
        const int64_t e = base + j * 32;
        ballots[j] = __ballot_sync(0xffffffffu, e < m && edge_stays(keep, fin, gid, col, e));
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
            const int32_t c0 = col[e];
            if ((ballots[j] >> lane) & 1u) {
                col_out[p] = vmap[c0];
                eid_out[p] = eid[e];
                if (S_out) S_out[p] = S[e];
            } else {
                const int32_t g = gid[c0];
                const bool k = keep[e];
                mask_ptr[g][eid[e]] = k ? 1 : 0;
                int32_t *sp = sup_ptr[g];
                if (sp) sp[eid[e]] = k ? S[e] : 0;
            }
        }
        run += __popc(ballots[j]);
    }
}

// New row pointers and slot ids of the surviving vertices.  A slot's
// vertices are contiguous, so its surviving edges (kept_s, zero on entry,
// when given) are the new row pointer after its last vertex minus the one of
// its first: the two boundary vertices add them.
__global__ void vertex_rewrite_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ gid,
                                      const uint8_t *__restrict__ fin,
                                      const int32_t *__restrict__ vmap,
                                      const int32_t *__restrict__ pos, int32_t n, int32_t m,
                                      const RoundCounters *__restrict__ cnt,
                                      const int32_t *__restrict__ vtotal,
                                      int32_t *__restrict__ rp_out, int32_t *__restrict__ gid_out,
                                      int32_t *__restrict__ kept_s) {
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n && !fin[gid[v]]) {
        const int32_t g = gid[v];
        const int32_t r = rp[v];
        const int32_t nr = r < m ? pos[r] : cnt->kept;
        rp_out[vmap[v]] = nr;
        gid_out[vmap[v]] = g;
        if (kept_s) {
            if (v == 0 || gid[v - 1] != g) atomicSub(kept_s + g, nr);
            if (v == n - 1 || gid[v + 1] != g) {
                const int32_t r1 = rp[v + 1];
                atomicAdd(kept_s + g, r1 < m ? pos[r1] : cnt->kept);
            }
        }
    }
    if (v == 0) rp_out[*vtotal] = cnt->kept;
}

// Per slot: its first decision pass (batch_force_kernel).
__global__ void server_force_kernel(int32_t slots, const int32_t *__restrict__ kept_s,
                                    const int32_t *__restrict__ listed_s, RoundCounters *cnt) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= slots) return;
    const int32_t g = int32_t(t);
    const int32_t kept = kept_s[g], listed = listed_s[g];
    if (kept > 0 && listed >= kRecomputeMinListed && int64_t(listed) * 4 > kept)
        atomicAdd(&cnt->forced, 1);
}

// Per slot: update or support step next step (the rule of batch_decide_kernel
// on the slot's surviving and listed edges).
__global__ void server_decide_kernel(int32_t slots, const int32_t *__restrict__ kept_s,
                                     const int32_t *__restrict__ listed_s, int32_t mode,
                                     uint8_t *__restrict__ upd_s, RoundCounters *cnt) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= slots) return;
    const int32_t g = int32_t(t);
    const int32_t kept = kept_s[g];
    const int32_t listed = listed_s[g];
    const bool upd = kept > 0 && (mode == 1 || (mode == 2 && (int64_t(listed) * 4 <= kept ||
                                                             (listed < kRecomputeMinListed &&
                                                              cnt->forced == 0))));
    upd_s[g] = upd ? 1 : 0;
    if (kept > 0) {
        atomicAdd(&cnt->kept, 1);
        if (!upd) atomicAdd(&cnt->removed_tri, 1);
    }
}

}  // namespace

cudaError_t launch_server_append(const int32_t *rp_in, const int32_t *col_in, int32_t n, int32_t m,
                                 int32_t nb, int32_t mb, int32_t slot, int32_t *rp, int32_t *col,
                                 int32_t *eid, int32_t *gid, cudaStream_t s,
                                 const int32_t *emap) {
    const int64_t work = int64_t(n > m ? n : m) + 1;
    int64_t blocks = (work + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    append_kernel<<<int(blocks), 256, 0, s>>>(rp_in, col_in, n, m, nb, mb, slot, rp, col, eid, gid,
                                               emap);
    return cudaGetLastError();
}

cudaError_t launch_server_round_tail(const Live &cur, const int32_t *S, const uint8_t *keep,
                                     const int32_t *kept_g, const int32_t *removed_g,
                                     uint8_t *fin, int32_t *rounds_g, int32_t slots,
                                     const int32_t *gid, int32_t *vmap, int32_t *vtile_count,
                                     int32_t *vtile_off, RoundCounters *vcnt, int32_t *etile_count,
                                     int32_t *etile_off, RoundCounters *cnt, int32_t *pos,
                                     int32_t *rp_out, int32_t *col_out, int32_t *eid_out,
                                     int32_t *gid_out, uint8_t *const *mask_ptr,
                                     int32_t *const *sup_ptr, cudaStream_t s, int *launches,
                                     int32_t *S_out, int32_t *kept_s) {
    finish_kernel<<<int((int64_t(slots) + 255) / 256), 256, 0, s>>>(slots, kept_g, removed_g, fin, rounds_g);
    const int32_t vt = compact_tiles(cur.n);
    if (vt > 0) vertex_count_kernel<<<vt, kCompactThreads, 0, s>>>(gid, fin, cur.n, vtile_count);
    cudaError_t e = launch_scan_tiles(vtile_count, vt, vtile_off, vcnt, s, launches);
    if (e != cudaSuccess) return e;
    if (vt > 0) vertex_map_kernel<<<vt, kCompactThreads, 0, s>>>(gid, fin, cur.n, vtile_off, vmap);
    const int32_t et = compact_tiles(cur.m);
    if (et > 0)
        edge_count_kernel<<<et, kCompactThreads, 0, s>>>(keep, fin, gid, cur.col, cur.m,
                                                         etile_count);
    e = launch_scan_tiles(etile_count, et, etile_off, cnt, s, launches);
    if (e != cudaSuccess) return e;
    if (et > 0)
        edge_compact_kernel<<<et, kCompactThreads, 0, s>>>(cur.col, cur.eid, S, keep, fin, gid,
                                                           vmap, cur.m, etile_off, pos, col_out,
                                                           eid_out, mask_ptr, sup_ptr, S_out);
    vertex_rewrite_kernel<<<int((int64_t(cur.n) + 256) / 256), 256, 0, s>>>(
        cur.rp, gid, fin, vmap, pos, cur.n, cur.m, cnt, &vcnt->kept, rp_out, gid_out, kept_s);
    *launches += 6;
    return cudaGetLastError();
}

cudaError_t launch_server_prune(const Live &cur, const int32_t *S, const int32_t *gid,
                                const int32_t *thr, uint8_t *keep, int32_t *kept_g,
                                int32_t *removed_g, cudaStream_t s, int *launches, int32_t *list,
                                int32_t *list_count, int32_t *listed_s) {
    return launch_batch_keep(cur, S, gid, thr, keep, kept_g, removed_g, s, launches, list,
                             list_count, listed_s);
}

cudaError_t launch_server_decide(int32_t slots, const int32_t *kept_s, const int32_t *listed_s,
                                 int32_t mode, uint8_t *upd_s, RoundCounters *cnt, cudaStream_t s,
                                 int *launches) {
    if (mode == 2) {
        server_force_kernel<<<int((int64_t(slots) + 255) / 256), 256, 0, s>>>(slots, kept_s, listed_s, cnt);
        ++*launches;
    }
    server_decide_kernel<<<int((int64_t(slots) + 255) / 256), 256, 0, s>>>(slots, kept_s, listed_s, mode, upd_s,
                                                             cnt);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace kt
