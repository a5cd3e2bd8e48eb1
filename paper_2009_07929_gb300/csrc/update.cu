// Decremental support update between peel rounds.
//
// Alg. 1 recomputes S of the whole live graph in every round.  The supports of
// the next round are also fixed by this round's: after a round removes the
// edge set R from the live graph G, the support of a surviving edge e in
// G \ R is its support in G minus the triangles of G that contain e and at
// least one edge of R.  Only the triangles touching R change anything, and a
// removed edge with support 0 touches none.  This file computes that
// difference exactly (integer arithmetic), so the supports, the masks and the
// round-by-round removals are those of the recomputation.
//
// Every triangle {x, y, w} of G that contains a removed edge is handled once,
// by its removed edge with the smallest slot:
//   1. per removed edge p = (x, y) with S[p] > 0: its row x and the endpoint z
//      of smaller degree (the caller's lower degrees of the live graph, kept
//      current across rounds), flagged; each flagged vertex then gets a
//      compact index, so that nothing below is sized by the vertex count;
//   2. lower-neighbour lists of G for the flagged vertices only: the u < v
//      with (u, v) in G and the slot of (u, v) (a count, a scan and a scatter
//      over the edges; the order inside a list does not matter);
//   3. one warp per removed edge: it walks the full neighbourhood (upper row
//      and lower list) of z and, for each neighbour w, looks up the edge
//      between w and the other endpoint o by binary search in the upper row of
//      min(o, w).  A found edge closes a triangle; the triangle is credited
//      here unless one of its other two edges is removed and has a smaller
//      slot, and the credit subtracts one from each of its kept edges.  The
//      walk stops after S[p] triangles: S[p] is exactly the number of
//      triangles of G on p.
#include "ktruss_internal.cuh"

namespace kt {
namespace {

constexpr int kThreads = 256;
constexpr int kSlotsPerThread = 16;

// Row of slot e: the largest row whose first slot is <= e.
__device__ __forceinline__ int32_t row_of(const int32_t *__restrict__ rp, int32_t n, int32_t e) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (__ldg(rp + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First slot in the sorted row segment col[lo, hi) whose column is >= b
// (hi if there is none).
__device__ __forceinline__ int32_t lower_bound(const int32_t *__restrict__ col, int32_t lo,
                                               int32_t hi, int32_t b) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(col + mid) < b) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ldeg[v] = number of kept edges (u, v), u < v, of the live graph (its lower
// degree once the removed edges are gone; keep == nullptr keeps every edge).
__global__ void __launch_bounds__(kThreads)
lower_degree_kernel(const int32_t *__restrict__ col, const uint8_t *__restrict__ keep, int32_t m,
                    int32_t *__restrict__ ldeg) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride)
        if (!keep || keep[e]) atomicAdd(ldeg + __ldg(col + e), 1);
}

// Device loop: true when this round runs no update; otherwise the list length
// and the live edge count come from the loop's control block.
__device__ __forceinline__ bool loop_skip(const LoopCtl *lc, int32_t &nlist, int32_t &m) {
    if (!lc) return false;
    if (!(lc->action & kActUpdate)) return true;
    nlist = lc->nlist;
    m = lc->m;
    return false;
}

// Device loop: zeroes the per-list counters [0, nlist + 1) and the claimed
// vertex count before an update.
__global__ void __launch_bounds__(kThreads)
update_zero_kernel(const LoopCtl *lc, int32_t *__restrict__ lcnt, int32_t *__restrict__ lfill,
                   int32_t *__restrict__ nz) {
    int32_t nlist = 0, m = 0;
    if (loop_skip(lc, nlist, m)) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k <= nlist; k += stride) {
        lcnt[k] = 0;
        lfill[k] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *nz = 0;
}

// Per listed edge p = (x, y): its row x and the endpoint z of smaller degree
// (upper row length + lower degree), whose neighbourhood the update walks;
// flags z.  lx[k] = x, with bit 31 set when z = y; lx[k] = -1 when the edge's
// graph is not updated (upd_g given and upd_g[graph] == 0).
__global__ void __launch_bounds__(kThreads)
pick_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
            const int32_t *__restrict__ ldeg, const int32_t *__restrict__ list, int32_t nlist,
            int32_t *__restrict__ flag, int32_t *__restrict__ lx, const int32_t *__restrict__ gid,
            const uint8_t *__restrict__ upd_g, const LoopCtl *lc) {
    int32_t m_ = 0;
    if (loop_skip(lc, nlist, m_)) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nlist; k += stride) {
        const int32_t p = __ldg(list + k);
        const int32_t y = __ldg(col + p);
        if (upd_g && !upd_g[gid[y]]) {
            lx[k] = -1;
            continue;
        }
        const int32_t x = row_of(rp, n, p);
        const int32_t dx = __ldg(rp + x + 1) - __ldg(rp + x) + __ldg(ldeg + x);
        const int32_t dy = __ldg(rp + y + 1) - __ldg(rp + y) + __ldg(ldeg + y);
        const bool walk_y = dy < dx;
        flag[walk_y ? y : x] = 1;
        lx[k] = x | (walk_y ? int32_t(0x80000000u) : 0);
    }
}

// flag[v]: 0 = not flagged, 1 = flagged by pick_kernel, c + 2 = flagged with
// compact index c.  Each flagged vertex of the list is claimed once: it gets
// the next index and zlist[c] = v.
__global__ void __launch_bounds__(kThreads)
claim_kernel(const int32_t *__restrict__ col, const int32_t *__restrict__ list,
             const int32_t *__restrict__ lx, int32_t nlist, int32_t *__restrict__ flag,
             int32_t *__restrict__ zlist, int32_t *__restrict__ nz, const LoopCtl *lc) {
    int32_t m_ = 0;
    if (loop_skip(lc, nlist, m_)) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nlist; k += stride) {
        const int32_t xw = __ldg(lx + k);
        if (xw == -1) continue;
        const int32_t z = xw < 0 ? __ldg(col + __ldg(list + k)) : xw;
        if (atomicCAS(flag + z, 1, 0x7fffffff) == 1) {
            const int32_t c = atomicAdd(nz, 1);
            zlist[c] = z;
            flag[z] = c + 2;
        }
    }
}

// flag[zlist[c]] = 0 for every claimed vertex (c < *nz).
__global__ void __launch_bounds__(kThreads)
unflag_kernel(const int32_t *__restrict__ zlist, const int32_t *__restrict__ nz, int32_t cap,
              int32_t *__restrict__ flag, const LoopCtl *lc) {
    int32_t m_ = 0;
    if (loop_skip(lc, cap, m_)) return;
    const int32_t count = *nz;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < count && c < cap;
         c += stride)
        flag[zlist[c]] = 0;
}

// lcnt[c] += number of edges (u, v) of the live graph, for v with compact index c.
__global__ void __launch_bounds__(kThreads)
lower_count_kernel(const int32_t *__restrict__ col, int32_t m, const int32_t *__restrict__ flag,
                   int32_t *__restrict__ lcnt, const LoopCtl *lc) {
    int32_t nl_ = 0;
    if (loop_skip(lc, nl_, m)) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t f = flag[__ldg(col + e)];
        if (f >= 2) atomicAdd(lcnt + (f - 2), 1);
    }
}

// Scatters (u, slot) of every edge (u, v) with v flagged into the lower list
// of v.  A thread visits kSlotsPerThread consecutive slots, finding the row of
// the first by binary search and following rows from there.
__global__ void __launch_bounds__(kThreads)
lower_fill_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                  int32_t m, const int32_t *__restrict__ flag, const int32_t *__restrict__ lrp,
                  int32_t *__restrict__ lfill, int32_t *__restrict__ lsrc,
                  int32_t *__restrict__ lslot, const LoopCtl *lc) {
    int32_t nl_ = 0;
    if (loop_skip(lc, nl_, m)) return;
    const int64_t span = int64_t(gridDim.x) * kThreads * kSlotsPerThread;
    for (int64_t e0 = (int64_t(blockIdx.x) * kThreads + threadIdx.x) * kSlotsPerThread; e0 < m;
         e0 += span) {
        const int64_t e1 = e0 + kSlotsPerThread < m ? e0 + kSlotsPerThread : m;
        int32_t u = -1, uend = 0;
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t f = flag[__ldg(col + e)];
            if (f < 2) continue;
            if (u < 0 || e >= uend) {
                u = row_of(rp, n, int32_t(e));
                uend = __ldg(rp + u + 1);
            }
            const int32_t at = __ldg(lrp + (f - 2)) + atomicAdd(lfill + (f - 2), 1);
            lsrc[at] = u;
            lslot[at] = int32_t(e);
        }
    }
}

__global__ void __launch_bounds__(kThreads)
update_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
              const int32_t *__restrict__ flag, const int32_t *__restrict__ lrp,
              const int32_t *__restrict__ lsrc,
              const int32_t *__restrict__ lslot, const uint8_t *__restrict__ keep,
              const int32_t *__restrict__ list, const int32_t *__restrict__ lx, int32_t nlist,
              const int32_t *__restrict__ S, int32_t *__restrict__ S_dec,
              const int32_t *__restrict__ pos, unsigned long long *__restrict__ destroyed,
              const LoopCtl *lc) {
    int32_t m_ = 0;
    if (loop_skip(lc, nlist, m_)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    unsigned long long mine = 0;
    for (int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; k < nlist;
         k += warps) {
        const int32_t xw = __ldg(lx + k);
        if (xw == -1) continue;  // graph not updated (warp-uniform: one edge per warp)
        const int32_t p = __ldg(list + k);
        const int32_t x = xw & 0x7fffffff;
        const bool walk_y = xw < 0;
        const int32_t y = __ldg(col + p);
        const int32_t z = walk_y ? y : x, o = walk_y ? x : y;
        const int32_t zu0 = __ldg(rp + z), zu1 = __ldg(rp + z + 1);
        const int32_t zc = flag[z] - 2;  // compact index of the walked endpoint
        const int32_t zl0 = __ldg(lrp + zc), zl1 = __ldg(lrp + zc + 1);
        const int32_t nu = zu1 - zu0;
        const int32_t total = nu + (zl1 - zl0);
        const int32_t need = __ldg(S + p);
        int32_t found = 0;
        for (int32_t b = 0; b < total && found < need; b += 32) {
            const int32_t i = b + lane;
            bool hit = false;
            if (i < total) {
                int32_t w, qz;
                if (i < nu) {
                    qz = zu0 + i;
                    w = __ldg(col + qz);
                } else {
                    const int32_t t = zl0 + (i - nu);
                    w = __ldg(lsrc + t);
                    qz = __ldg(lslot + t);
                }
                if (w != o) {
                    const int32_t a = w < o ? w : o, c = w < o ? o : w;
                    const int32_t lo = __ldg(rp + a), hi = __ldg(rp + a + 1);
                    const int32_t qo = lower_bound(col, lo, hi, c);
                    if (qo < hi && __ldg(col + qo) == c) {
                        hit = true;
                        const bool rz = keep[qz] == 0, ro = keep[qo] == 0;
                        if (!((rz && qz < p) || (ro && qo < p))) {
                            if (!rz) atomicSub(S_dec + (pos ? pos[qz] : qz), 1);
                            if (!ro) atomicSub(S_dec + (pos ? pos[qo] : qo), 1);
                            ++mine;
                        }
                    }
                }
            }
            found += __popc(__ballot_sync(0xffffffffu, hit));
        }
    }
    for (int d = 16; d > 0; d >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, d);
    if (lane == 0 && mine) atomicAdd(destroyed, mine);
}

}  // namespace

cudaError_t launch_lower_degree(const Live &g, UpdateState *st, cudaStream_t s, int *launches) {
    cudaError_t e = cudaMemsetAsync(st->ldeg, 0, (size_t(g.n) + 1) * 4, s);
    if (e != cudaSuccess) return e;
    if (g.m > 0) {
        const int64_t blocks = (int64_t(g.m) + kThreads - 1) / kThreads;
        lower_degree_kernel<<<int(blocks < 152 * 16 ? blocks : 152 * 16), kThreads, 0, s>>>(
            g.col, nullptr, g.m, st->ldeg);
        ++*launches;
    }
    st->ldeg_valid = true;
    return cudaGetLastError();
}

cudaError_t launch_support_update(const Live &g, const uint8_t *keep, const int32_t *list,
                                  int32_t nlist, int32_t *S, unsigned long long *destroyed,
                                  const UpdateScratch &u, UpdateState *st, cudaStream_t s,
                                  int *launches, const int32_t *pos, int32_t *S_out,
                                  const uint8_t *upd_g, const LoopCtl *lc) {
    // in the device loop nlist and g.m are capacities (fixed grids): the
    // kernels read the round's values from lc and skip rounds without update
    if (nlist <= 0 || g.m == 0) return cudaSuccess;
    const int64_t rows = int64_t(g.n) + 1;
    auto grid = [lc](int64_t work, int64_t cap) {
        if (lc && cap > kLoopBlocks) cap = kLoopBlocks;
        return int((work + kThreads - 1) / kThreads < cap ? (work + kThreads - 1) / kThreads : cap);
    };
    cudaError_t e = cudaSuccess;
    if (!st->ldeg_valid) {
        if (lc) return cudaErrorInvalidValue;  // the loop starts with valid lower degrees
        // lower degrees after this round's removals; prune keeps them current
        // from here on by subtracting the edges it removes
        e = cudaMemsetAsync(st->ldeg, 0, size_t(rows) * 4, s);
        if (e != cudaSuccess) return e;
        lower_degree_kernel<<<grid(g.m, 152 * 16), kThreads, 0, s>>>(g.col, keep, g.m, st->ldeg);
        ++*launches;
        st->ldeg_valid = true;
    }
    // per-list arrays: at most nlist flagged vertices (st->flag is all zero
    // between calls; the claimed entries are reset at the end)
    const int64_t zcap = int64_t(nlist) + 1;
    if (lc) {
        update_zero_kernel<<<grid(zcap, 152 * 16), kThreads, 0, s>>>(lc, u.lcnt, u.lfill, st->nz);
        ++*launches;
    } else {
        e = cudaMemsetAsync(st->nz, 0, 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(u.lcnt, 0, size_t(zcap) * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(u.lfill, 0, size_t(zcap) * 4, s);
        if (e != cudaSuccess) return e;
    }
    pick_kernel<<<grid(nlist, 152 * 16), kThreads, 0, s>>>(g.rp, g.col, g.n, st->ldeg, list, nlist,
                                                            st->flag, u.lx, g.gid, upd_g, lc);
    claim_kernel<<<grid(nlist, 152 * 16), kThreads, 0, s>>>(g.col, list, u.lx, nlist, st->flag,
                                                             u.zlist, st->nz, lc);
    lower_count_kernel<<<grid(g.m, 152 * 16), kThreads, 0, s>>>(g.col, g.m, st->flag, u.lcnt, lc);
    *launches += 3;
    e = launch_scan_i32(u.lcnt, u.lrp, zcap, u, s, launches, lc);
    if (e != cudaSuccess) return e;
    int64_t fblocks =
        (int64_t(g.m) + int64_t(kThreads) * kSlotsPerThread - 1) / (int64_t(kThreads) * kSlotsPerThread);
    if (lc && fblocks > kLoopBlocks) fblocks = kLoopBlocks;
    lower_fill_kernel<<<int(fblocks), kThreads, 0, s>>>(g.rp, g.col, g.n, g.m, st->flag, u.lrp,
                                                        u.lfill, u.lsrc, u.lslot, lc);
    update_kernel<<<grid(int64_t(nlist) * 32, 152 * 32), kThreads, 0, s>>>(
        g.rp, g.col, st->flag, u.lrp, u.lsrc, u.lslot, keep, list, u.lx, nlist, S,
        pos ? S_out : S, pos, destroyed, lc);
    unflag_kernel<<<grid(nlist, 152 * 16), kThreads, 0, s>>>(u.zlist, st->nz, nlist, st->flag, lc);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace kt
