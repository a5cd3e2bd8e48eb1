// Balanced support step (Alg. 3 edge tasks, made ultra-fine-grained).
//
// The paper schedules one thread per edge task (Sec. III-B/C) and leaves the
// splitting of a task's row of A22 across workers to future work, because the
// per-task work depends on the length of row kappa (Sec. III-B, last
// paragraph).  Here that split is done:
//
//  * work estimate: task (i, kappa) at slot e probes every element of row
//    kappa, so its work is d+(kappa) items (0 when the tail of row i after e is
//    empty).  An int64 exclusive scan of the items gives a global item space.
//  * partition: the item space is cut into equal chunks; a chunk is a range of
//    (edge, offset in row kappa) pairs, so one long row kappa is cut across
//    many CTAs.
//  * intersection: a CTA stages the rows i of its chunk (whole rows, up to
//    kStageCap slots) into a shared-memory hash table keyed by (row, column)
//    holding each slot; then one warp per edge streams row kappa with coalesced
//    loads, probes each column w in the table of row i, and on a hit credits
//    (i,kappa) and (i,w) in shared memory and (kappa,w) with a global atomic.
//    Staged credits are flushed once per stage.  Every element of row kappa is
//    greater than kappa, so a hit in row i is always in the tail after e,
//    exactly the intersection a12(j+1:) o A(kappa,:) of Alg. 3.
//  * rows longer than a stage are handled by a second kernel that stages them
//    in pieces of kPieceCap slots (in column order) and walks, per edge, a
//    cursor through row kappa that advances piece by piece, so each element of
//    row kappa is still read once.
//
// All credits are integer additions, so the result is independent of the
// order in which CTAs run.
#include <cstdint>

#include "ktruss_internal.cuh"

namespace kt {
namespace {

// ----------------------------------------------------------- configuration
constexpr int kShortThreads = 256;
constexpr int kStageCap = 2048;             // staged slots per stage (short rows)
constexpr int kStageTable = 2 * kStageCap;  // hash entries (load factor <= 1/2)
constexpr int kStageRows = 512;             // rows per stage
constexpr long long kChunkMin = 16384;      // items per chunk (minimum)
constexpr int kMaxChunks = 1 << 22;         // chunk table capacity

constexpr int kLongThreads = 512;
constexpr int kPieceCap = 4096;  // staged slots per piece (long rows)
constexpr int kPieceTable = 2 * kPieceCap;
constexpr int kEdgeBlock = 1024;  // edges of a long row per task

constexpr int kWorkThreads = 256;
constexpr int kWorkPerThread = 16;
constexpr int kWorkTile = kWorkThreads * kWorkPerThread;

constexpr int32_t kEmpty = -1;

// sched[] layout
constexpr int kSchedChunkNext = 0;
constexpr int kSchedTasks = 1;
constexpr int kSchedTaskNext = 2;
constexpr int kSchedNChunks = 3;
constexpr int kSchedWords = 8;

struct ChunkPlan {
    long long chunk;  // items per chunk
    long long total;  // total items
};

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

// Largest row index i with rp[i] <= e (e < m).
__device__ __forceinline__ int32_t row_of_slot(const int32_t *__restrict__ rp, int32_t n,
                                               int32_t e) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(rp + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Largest e in [0, m-1] with wp[e] <= item.
__device__ __forceinline__ int32_t edge_of_item(const long long *__restrict__ wp, int32_t m,
                                                long long item) {
    int32_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(wp + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Hash of (row, column) to a bucket of 4 entries.
__device__ __forceinline__ uint32_t bucket_of(int32_t row, int32_t w, uint32_t bucket_mask) {
    uint32_t h = uint32_t(w) * 0x9E3779B1u + uint32_t(row) * 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 13;
    return h & bucket_mask;
}

__device__ __forceinline__ void table_insert(int32_t *keys, uint16_t *slots, uint32_t bucket_mask,
                                             int32_t row, int32_t w, int32_t s) {
    uint32_t b = bucket_of(row, w, bucket_mask);
    for (;;) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (atomicCAS(keys + 4 * b + j, kEmpty, w) == kEmpty) {
                slots[4 * b + j] = uint16_t(s);
                return;
            }
        }
        b = (b + 1) & bucket_mask;
    }
}

// Local slot of column w within the staged slots [lo, hi) of `row`, or -1.
__device__ __forceinline__ int32_t table_find(const int32_t *keys, const uint16_t *slots,
                                              uint32_t bucket_mask, int32_t row, int32_t w,
                                              int32_t lo, int32_t hi) {
    uint32_t b = bucket_of(row, w, bucket_mask);
    for (;;) {
        const int4 k = reinterpret_cast<const int4 *>(keys)[b];
        if (k.x == w) {
            const int32_t s = slots[4 * b + 0];
            if (s >= lo && s < hi) return s;
        }
        if (k.y == w) {
            const int32_t s = slots[4 * b + 1];
            if (s >= lo && s < hi) return s;
        }
        if (k.z == w) {
            const int32_t s = slots[4 * b + 2];
            if (s >= lo && s < hi) return s;
        }
        if (k.w == w) {
            const int32_t s = slots[4 * b + 3];
            if (s >= lo && s < hi) return s;
        }
        if (k.x == kEmpty || k.y == kEmpty || k.z == kEmpty || k.w == kEmpty) return -1;
        b = (b + 1) & bucket_mask;
    }
}

__device__ __forceinline__ int table_size_for(int32_t len) {
    int t = 64;
    while (t < 2 * len) t <<= 1;
    return t;
}

// ---------------------------------------------------------- work estimate
// w(e) = d+(col[e]) for edges of rows no longer than kStageCap whose tail is
// non-empty, else 0 (long rows get their own task list).  Writes w into wp[e]
// and the tile total into tile_sum[blockIdx.x].
__global__ void __launch_bounds__(kWorkThreads)
work_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n, int32_t m,
            long long *__restrict__ wp, long long *__restrict__ tile_sum,
            unsigned long long *__restrict__ merge_work) {
    __shared__ long long warp_part[kWorkThreads / 32];
    __shared__ long long warp_merge[kWorkThreads / 32];
    const int64_t e0 = (int64_t(blockIdx.x) * kWorkThreads + threadIdx.x) * kWorkPerThread;
    long long local = 0, merge = 0;
    if (e0 < m) {
        int32_t row = row_of_slot(rp, n, int32_t(e0));
        int32_t rbeg = __ldg(rp + row);
        int32_t rend = __ldg(rp + row + 1);
        const int64_t e1 = min(int64_t(m), e0 + kWorkPerThread);
        for (int64_t e = e0; e < e1; ++e) {
            while (rend <= e) {
                ++row;
                rbeg = rend;
                rend = __ldg(rp + row + 1);
            }
            const int32_t k = __ldg(col + e);
            const long long dk = __ldg(rp + k + 1) - __ldg(rp + k);
            const long long w = (rend - rbeg <= kStageCap && e + 1 < rend) ? dk : 0;
            merge += dk + (rend - e - 1);
            wp[e] = w;
            local += w;
        }
    }
    local = warp_sum_ll(local);
    merge = warp_sum_ll(merge);
    if ((threadIdx.x & 31) == 0) {
        warp_part[threadIdx.x >> 5] = local;
        warp_merge[threadIdx.x >> 5] = merge;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0, mw = 0;
        for (int k = 0; k < kWorkThreads / 32; ++k) {
            t += warp_part[k];
            mw += warp_merge[k];
        }
        tile_sum[blockIdx.x] = t;
        if (mw) atomicAdd(merge_work, (unsigned long long)mw);
    }
}

// Exclusive scan of tile sums by one block; the total goes to *total.
__global__ void __launch_bounds__(1024)
scan_tile_sums_kernel(const long long *__restrict__ tile_sum, int32_t tiles,
                      long long *__restrict__ tile_off, long long *__restrict__ total) {
    __shared__ long long wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t per = (tiles + 1023) / 1024;
    const int32_t b = tid * per;
    const int32_t e = min(tiles, b + per);
    long long local = 0;
    for (int32_t k = b; k < e; ++k) local += tile_sum[k];
    long long incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const long long v = wsum[lane];
        long long vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += u;
        }
        wsum[lane] = vi - v;
        if (lane == 31) *total = vi;
    }
    __syncthreads();
    long long run = wsum[w] + incl - local;
    for (int32_t k = b; k < e; ++k) {
        tile_off[k] = run;
        run += tile_sum[k];
    }
}

// In-place conversion of wp[0..m) from per-edge work to the exclusive prefix;
// wp[m] = total.
__global__ void __launch_bounds__(kWorkThreads)
prefix_kernel(long long *__restrict__ wp, int32_t m, const long long *__restrict__ tile_off,
              const long long *__restrict__ total) {
    __shared__ long long wsum[kWorkThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t e0 = (int64_t(blockIdx.x) * kWorkThreads + tid) * kWorkPerThread;
    long long v[kWorkPerThread];
    long long local = 0;
#pragma unroll
    for (int j = 0; j < kWorkPerThread; ++j) {
        const int64_t e = e0 + j;
        v[j] = e < m ? wp[e] : 0;
        local += v[j];
    }
    long long incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    long long before = tile_off[blockIdx.x];
    for (int k = 0; k < w; ++k) before += wsum[k];
    long long run = before + incl - local;
#pragma unroll
    for (int j = 0; j < kWorkPerThread; ++j) {
        const int64_t e = e0 + j;
        if (e < m) wp[e] = run;
        run += v[j];
    }
    if (blockIdx.x == 0 && tid == 0) wp[m] = *total;
}

// Chunk plan: chunk size so that the chunk count fits the table.
__global__ void plan_kernel(const long long *__restrict__ total, ChunkPlan *plan,
                            int32_t *__restrict__ sched) {
    const long long t = *total;
    long long c = kChunkMin;
    const long long need = (t + kMaxChunks - 1) / kMaxChunks;
    if (need > c) c = need;
    plan->chunk = c;
    plan->total = t;
    sched[kSchedNChunks] = int32_t((t + c - 1) / c);
}

// Chunk boundaries: bound[c] = (edge, row) holding item c * chunk, for
// c in [0, nchunks]; the last boundary is clamped to edge m-1.
__global__ void partition_kernel(const long long *__restrict__ wp, const int32_t *__restrict__ rp,
                                 int32_t n, int32_t m, const ChunkPlan *__restrict__ plan,
                                 const int32_t *__restrict__ sched, int2 *__restrict__ bound) {
    const int32_t nchunks = sched[kSchedNChunks];
    const long long chunk = plan->chunk, total = plan->total;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c <= nchunks;
         c += int64_t(gridDim.x) * blockDim.x) {
        long long item = c * chunk;
        if (item > total) item = total;
        const int32_t e = edge_of_item(wp, m, item);
        bound[c] = make_int2(e, row_of_slot(rp, n, e));
    }
}

// Long-row task list: every row longer than kStageCap whose edges have a
// non-empty tail contributes ceil((len-1)/kEdgeBlock) tasks (row, block).
__global__ void long_tasks_kernel(const int32_t *__restrict__ rp, int32_t n,
                                  int32_t *__restrict__ sched, int2 *__restrict__ tasks,
                                  int32_t cap) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t len = rp[r + 1] - rp[r];
    if (len <= kStageCap) return;
    const int32_t nb = (len - 1 + kEdgeBlock - 1) / kEdgeBlock;
    const int32_t at = atomicAdd(sched + kSchedTasks, nb);
    for (int32_t b = 0; b < nb && at + b < cap; ++b) tasks[at + b] = make_int2(int32_t(r), b);
}

// --------------------------------------------------- short-row support kernel
struct ShortSmem {
    int32_t keys[kStageTable];
    uint16_t slots[kStageTable];
    int32_t cnt[kStageCap];
    int32_t rpl[kStageRows + 1];
    int32_t ctl[8];
};

__global__ void __launch_bounds__(kShortThreads, 6)
support_short_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                     int32_t m, const long long *__restrict__ wp, const ChunkPlan *__restrict__ plan,
                     const int2 *__restrict__ bound, int32_t *__restrict__ sched,
                     int32_t *__restrict__ S, unsigned long long *__restrict__ tri_out) {
    __shared__ __align__(16) ShortSmem sm;
    const int tid = threadIdx.x, lane = tid & 31;
    const int32_t nchunks = sched[kSchedNChunks];
    const long long chunk = plan->chunk, total = plan->total;
    unsigned long long tri = 0;
    for (;;) {
        if (tid == 0) sm.ctl[0] = atomicAdd(sched + kSchedChunkNext, 1);
        __syncthreads();
        const int32_t c = sm.ctl[0];
        __syncthreads();
        if (c >= nchunks) break;
        const long long iA = c * chunk;
        const long long iB = min(total, iA + chunk);
        const int2 b0 = bound[c], b1 = bound[c + 1];
        const int32_t ea = b0.x, eb = b1.x, rb = b1.y;
        int32_t r = b0.y;
        while (r <= rb) {
            // ---- form a stage: rows [r, r2], slots [s0, s1)
            if (tid == 0) {
                int32_t rr = r;
                while (rr <= rb && __ldg(rp + rr + 1) - __ldg(rp + rr) > kStageCap) ++rr;
                int32_t r2 = -1, s0 = 0;
                if (rr <= rb) {
                    s0 = max(__ldg(rp + rr), ea);
                    int32_t lo = rr, hi = min(rb, rr + kStageRows - 1);
                    while (lo < hi) {
                        const int32_t mid = (lo + hi + 1) >> 1;
                        if (__ldg(rp + mid + 1) - s0 <= kStageCap) lo = mid; else hi = mid - 1;
                    }
                    r2 = lo;
                }
                sm.ctl[1] = rr;
                sm.ctl[2] = r2;
                sm.ctl[3] = s0;
                sm.ctl[4] = 0;  // next edge
            }
            __syncthreads();
            const int32_t rs = sm.ctl[1], r2 = sm.ctl[2], s0 = sm.ctl[3];
            if (r2 < 0) break;
            const int32_t nrows = r2 - rs + 1;
            for (int k = tid; k <= nrows; k += kShortThreads) sm.rpl[k] = __ldg(rp + rs + k);
            __syncthreads();
            const int32_t s1 = sm.rpl[nrows];
            const int32_t slen = s1 - s0;
            const int tsize = table_size_for(slen);
            const uint32_t bmask = uint32_t(tsize / 4 - 1);
            for (int k = tid; k < tsize / 4; k += kShortThreads)
                reinterpret_cast<int4 *>(sm.keys)[k] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
            for (int k = tid; k < slen; k += kShortThreads) sm.cnt[k] = 0;
            __syncthreads();
            // ---- build the (row, column) -> slot table
            for (int k = tid; k < slen; k += kShortThreads) {
                const int32_t abs = s0 + k;
                int32_t lo = 0, hi = nrows - 1;
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (sm.rpl[mid] <= abs) lo = mid; else hi = mid - 1;
                }
                table_insert(sm.keys, sm.slots, bmask, rs + lo, __ldg(col + abs), k);
            }
            __syncthreads();
            // ---- warp per edge over the chunk's edges in this stage
            const int32_t eLo = max(ea, s0), eHi = min(eb + 1, s1);
            for (;;) {
                int32_t e = 0;
                if (lane == 0) e = eLo + atomicAdd(&sm.ctl[4], 1);
                e = __shfl_sync(0xffffffffu, e, 0);
                if (e >= eHi) break;
                const long long base = __ldg(wp + e);
                const long long ka = max(iA, base) - base;
                const long long kb = min(iB, __ldg(wp + e + 1)) - base;
                if (ka >= kb) continue;
                // row of e within the stage
                int32_t lo = 0, hi = nrows - 1;
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (sm.rpl[mid] <= e) lo = mid; else hi = mid - 1;
                }
                const int32_t i = rs + lo;
                const int32_t qlo = max(sm.rpl[lo], s0) - s0, qhi = sm.rpl[lo + 1] - s0;
                const int32_t kappa = __ldg(col + e);
                const int32_t rk = __ldg(rp + kappa);
                int32_t own = 0;
                for (long long k = ka + lane; k < kb; k += 32) {
                    const int32_t w = __ldg(col + rk + k);
                    const int32_t q = table_find(sm.keys, sm.slots, bmask, i, w, qlo, qhi);
                    if (q >= 0) {
                        atomicAdd(&sm.cnt[q], 1);
                        atomicAdd(S + rk + k, 1);
                        ++own;
                    }
                }
                own = __reduce_add_sync(0xffffffffu, own);
                if (lane == 0 && own) {
                    atomicAdd(&sm.cnt[e - s0], own);
                    tri += own;
                }
            }
            __syncthreads();
            // ---- flush staged credits
            for (int k = tid; k < slen; k += kShortThreads) {
                const int32_t v = sm.cnt[k];
                if (v) atomicAdd(S + s0 + k, v);
            }
            __syncthreads();
            r = r2 + 1;
        }
    }
    if (lane == 0 && tri) atomicAdd(tri_out, tri);
}

// ---------------------------------------------------- long-row support kernel
struct LongSmem {
    int32_t keys[kPieceTable];
    uint16_t slots[kPieceTable];
    int32_t cnt[kPieceCap];
    int32_t cur[kEdgeBlock];
    int32_t endk[kEdgeBlock];
    int32_t own[kEdgeBlock];
    int32_t ctl[8];
};

__global__ void __launch_bounds__(kLongThreads, 2)
support_long_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                    const int2 *__restrict__ tasks, int32_t task_cap, int32_t *__restrict__ sched,
                    int32_t *__restrict__ S, unsigned long long *__restrict__ tri_out) {
    extern __shared__ __align__(16) unsigned char long_raw[];
    LongSmem &sm = *reinterpret_cast<LongSmem *>(long_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const int32_t ntasks = min(sched[kSchedTasks], task_cap);
    unsigned long long tri = 0;
    for (;;) {
        if (tid == 0) sm.ctl[0] = atomicAdd(sched + kSchedTaskNext, 1);
        __syncthreads();
        const int32_t t = sm.ctl[0];
        __syncthreads();
        if (t >= ntasks) break;
        const int2 tk = tasks[t];
        const int32_t r = tk.x;
        const int32_t rs = __ldg(rp + r), re = __ldg(rp + r + 1);
        const int32_t eA = rs + tk.y * kEdgeBlock;
        const int32_t eB = min(eA + kEdgeBlock, re - 1);  // edges with a non-empty tail
        const int32_t ne = eB - eA;
        for (int j = tid; j < ne; j += kLongThreads) {
            const int32_t kappa = __ldg(col + eA + j);
            sm.cur[j] = __ldg(rp + kappa);
            sm.endk[j] = __ldg(rp + kappa + 1);
            sm.own[j] = 0;
        }
        const int32_t pfirst = (eA + 1 - rs) / kPieceCap;
        const int32_t npieces = (re - rs + kPieceCap - 1) / kPieceCap;
        for (int32_t p = pfirst; p < npieces; ++p) {
            const int32_t ps = rs + p * kPieceCap;
            const int32_t pe = min(ps + kPieceCap, re);
            const int32_t plen = pe - ps;
            const int32_t vhi = pe < re ? __ldg(col + pe) : 0x7fffffff;
            const int tsize = table_size_for(plen);
            const uint32_t bmask = uint32_t(tsize / 4 - 1);
            __syncthreads();  // previous piece fully consumed
            for (int k = tid; k < tsize / 4; k += kLongThreads)
                reinterpret_cast<int4 *>(sm.keys)[k] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
            for (int k = tid; k < plen; k += kLongThreads) sm.cnt[k] = 0;
            if (tid == 0) sm.ctl[1] = 0;
            __syncthreads();
            for (int k = tid; k < plen; k += kLongThreads)
                table_insert(sm.keys, sm.slots, bmask, r, __ldg(col + ps + k), k);
            __syncthreads();
            // edges whose tail reaches into this piece: eA + j + 1 < pe
            const int32_t jmax = min(ne, pe - 1 - eA);
            for (;;) {
                int32_t j = 0;
                if (lane == 0) j = atomicAdd(&sm.ctl[1], 1);
                j = __shfl_sync(0xffffffffu, j, 0);
                if (j >= jmax) break;
                int32_t k = sm.cur[j];
                const int32_t ke = sm.endk[j];
                int32_t own = 0;
                for (;;) {
                    const int32_t idx = k + lane;
                    const int32_t w = idx < ke ? __ldg(col + idx) : 0x7fffffff;
                    const bool in = w < vhi;
                    if (in) {
                        const int32_t q = table_find(sm.keys, sm.slots, bmask, r, w, 0, plen);
                        if (q >= 0) {
                            atomicAdd(&sm.cnt[q], 1);
                            atomicAdd(S + idx, 1);
                            ++own;
                        }
                    }
                    const int32_t nin = __popc(__ballot_sync(0xffffffffu, in));
                    k += nin;
                    if (nin < 32) break;
                }
                own = __reduce_add_sync(0xffffffffu, own);
                if (lane == 0) {
                    sm.cur[j] = k;
                    sm.own[j] += own;
                }
            }
            __syncthreads();
            for (int k = tid; k < plen; k += kLongThreads) {
                const int32_t v = sm.cnt[k];
                if (v) atomicAdd(S + ps + k, v);
            }
        }
        __syncthreads();
        for (int j = tid; j < ne; j += kLongThreads) {
            const int32_t v = sm.own[j];
            if (v) {
                atomicAdd(S + eA + j, v);
                tri += v;
            }
        }
        __syncthreads();
    }
    tri = warp_sum_ll((long long)tri);
    if (lane == 0 && tri) atomicAdd(tri_out, tri);
}

int g_short_blocks = 0, g_long_blocks = 0;

cudaError_t configure_once() {
    if (g_short_blocks > 0) return cudaSuccess;
    int dev = 0, sms = 0, occ_s = 0, occ_l = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(support_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(sizeof(LongSmem)));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, support_short_kernel,
                                                          kShortThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l, support_long_kernel,
                                                          kLongThreads, sizeof(LongSmem));
    if (e != cudaSuccess) return e;
    g_short_blocks = sms * (occ_s > 0 ? occ_s : 1);
    g_long_blocks = sms * (occ_l > 0 ? occ_l : 1);
    return cudaSuccess;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

int32_t task_capacity(int64_t m) {
    return int32_t(m / kEdgeBlock + m / kStageCap + 16);
}

}  // namespace

size_t balanced_scratch_bytes(int32_t n, int64_t m) {
    const int64_t tiles = (m + kWorkTile - 1) / kWorkTile + 1;
    return align_up(size_t(m + 1) * 8) + 2 * align_up(size_t(tiles) * 8) + align_up(16) +
           align_up(sizeof(ChunkPlan)) + align_up(size_t(kMaxChunks + 1) * 8) +
           align_up(size_t(task_capacity(m)) * 8) + align_up(kSchedWords * 4) + size_t(n) * 0;
}

cudaError_t balanced_scratch_alloc(BalancedScratch *bs, int32_t n, int64_t m) {
    const size_t bytes = balanced_scratch_bytes(n, m);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return e;
    bs->base = p;
    bs->cap_m = m;
    bs->cap_n = n;
    bs->cap_tasks = task_capacity(m);
    return cudaSuccess;
}

void balanced_scratch_free(BalancedScratch *bs) {
    if (bs->base) cudaFree(bs->base);
    bs->base = nullptr;
}

cudaError_t launch_support_balanced(const Live &g, int32_t *S, RoundCounters *cnt,
                                    BalancedScratch *bs, cudaStream_t s, int *launches,
                                    cudaEvent_t *ev) {
    if (g.m == 0) {
        if (ev) return cudaEventRecord(ev[1], s);
        return cudaSuccess;
    }
    cudaError_t e = configure_once();
    if (e != cudaSuccess) return e;
    const int64_t m = g.m;
    const int32_t tiles = int32_t((m + kWorkTile - 1) / kWorkTile);
    // carve the scratch
    char *p = static_cast<char *>(bs->base);
    long long *wp = reinterpret_cast<long long *>(p);
    p += align_up(size_t(bs->cap_m + 1) * 8);
    const int64_t cap_tiles = (bs->cap_m + kWorkTile - 1) / kWorkTile + 1;
    long long *tile_sum = reinterpret_cast<long long *>(p);
    p += align_up(size_t(cap_tiles) * 8);
    long long *tile_off = reinterpret_cast<long long *>(p);
    p += align_up(size_t(cap_tiles) * 8);
    long long *total = reinterpret_cast<long long *>(p);
    p += align_up(16);
    ChunkPlan *plan = reinterpret_cast<ChunkPlan *>(p);
    p += align_up(sizeof(ChunkPlan));
    int2 *bound = reinterpret_cast<int2 *>(p);
    p += align_up(size_t(kMaxChunks + 1) * 8);
    int2 *tasks = reinterpret_cast<int2 *>(p);
    p += align_up(size_t(bs->cap_tasks) * 8);
    int32_t *sched = reinterpret_cast<int32_t *>(p);

    e = cudaMemsetAsync(sched, 0, kSchedWords * 4, s);
    if (e != cudaSuccess) return e;
    work_kernel<<<tiles, kWorkThreads, 0, s>>>(g.rp, g.col, g.n, g.m, wp, tile_sum,
                                               &cnt->merge_work);
    scan_tile_sums_kernel<<<1, 1024, 0, s>>>(tile_sum, tiles, tile_off, total);
    prefix_kernel<<<tiles, kWorkThreads, 0, s>>>(wp, g.m, tile_off, total);
    plan_kernel<<<1, 1, 0, s>>>(total, plan, sched);
    partition_kernel<<<152 * 4, 256, 0, s>>>(wp, g.rp, g.n, g.m, plan, sched, bound);
    long_tasks_kernel<<<(g.n + 255) / 256, 256, 0, s>>>(g.rp, g.n, sched, tasks,
                                                          int32_t(bs->cap_tasks));
    *launches += 6;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) {
        e = cudaEventRecord(ev[1], s);
        if (e != cudaSuccess) return e;
    }
    support_short_kernel<<<g_short_blocks, kShortThreads, 0, s>>>(
        g.rp, g.col, g.n, g.m, wp, plan, bound, sched, S, &cnt->triangles);
    support_long_kernel<<<g_long_blocks, kLongThreads, sizeof(LongSmem), s>>>(
        g.rp, g.col, tasks, int32_t(bs->cap_tasks), sched, S, &cnt->triangles);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace kt
