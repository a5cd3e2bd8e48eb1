// Balanced support step (Alg. 3 edge tasks, made ultra-fine-grained).
//
// Task (i, kappa) at slot e intersects two sorted lists: the tail of row i
// after e (length t) and row kappa (length d).  Alg. 3 credits, for every
// common column w, the edges (i,kappa), (i,w) and (kappa,w).  The paper runs
// one thread per task and leaves splitting a task across workers to future
// work (Sec. III-B, last paragraph).  Here:
//
//  * classification: each task stages the LONGER of its two lists and probes
//    it with every element of the shorter one, so its work is min(t, d)
//    items.  When row kappa is the shorter list the staged row is row i (the
//    probe values all exceed kappa, so a hit in row i is always in the tail);
//    otherwise the staged row is row kappa and the probes are the tail of row
//    i.  In both cases a hit at probe position x and staged slot q credits
//    S[x] and S[q], and the task's own slot e gets one per hit.
//  * grouping: a counting sort of the tasks by staged row (per round) gives
//    segments (owner e, probe start, item count) grouped by staged row, and
//    an int64 exclusive scan of the item counts gives a global item space.
//  * partition: the item space is cut into equal chunks (a few per CTA); a
//    chunk is a range of (segment, offset) pairs, so long probe lists are cut
//    across CTAs.
//  * intersection: a persistent kernel takes chunks dynamically.  Consecutive
//    short staged rows (<= kCap slots in total) are loaded into one shared-
//    memory hash table (one region per row, column -> slot); the probes of a
//    batch of segments form one flat item space that the warps split evenly,
//    each lane mapping its item to its segment, so short and long segments
//    keep every lane busy.  A staged row longer than kCap is loaded piece by
//    piece (in column order); per piece each segment contributes the run of
//    its probes below the piece's last column, found by binary search, so
//    every probe is still read once.  Credits to staged slots are gathered in
//    shared memory and flushed once per stage or piece.
//
// Light tasks (t + d <= light) skip all of the above: one thread merges the
// two short lists (support_light_kernel), which costs less than giving them a
// segment.  Which tasks are light is decided by the same test in both kernels.
//
// All credits are integer additions, so the result does not depend on the
// order in which CTAs, warps or the counting sort place the work.
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "ktruss_internal.cuh"

namespace kt {
namespace {

// ----------------------------------------------------------- configuration
#ifndef KT_SUPPORT_UNROLL
#define KT_SUPPORT_UNROLL 5
#endif
constexpr int kStageRows = 256;         // staged rows per stage
constexpr int kUnroll = KT_SUPPORT_UNROLL;  // 32-item windows in flight per warp
#ifndef KT_SUPPORT_GRAIN
#define KT_SUPPORT_GRAIN 0
#endif
// Items a warp takes from a batch at a time; 0 = an even static split.
constexpr int kGrain = KT_SUPPORT_GRAIN;
constexpr long long kChunkMin = 65536;  // items per chunk (minimum)
constexpr int kChunksPerCta = 16;       // target chunks per resident CTA
constexpr int kMaxChunks = 1 << 17;     // chunk table capacity

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kEdgeThreads = 256;
constexpr int kEdgesPerThread = 16;
constexpr int kLightPerThread = 4;

// Tasks whose two lists hold at most `light` columns together are merged by
// one thread (support_light_kernel) instead of being staged and probed.
__device__ __forceinline__ bool light_task(int32_t t, int32_t d, int32_t light) {
    return t + d <= light;
}

constexpr int32_t kIntMax = 0x7fffffff;

// sched[] words
constexpr int kSchedChunkNext = 0;
constexpr int kSchedNChunks = 1;
constexpr int kSchedGiveUp = 2;  // first loop that gave up (code), then two values
constexpr int kSchedWords = 8;

// Checks that cannot trigger on consistent inputs: an insertion that finds its
// region full (regions are at most a quarter full) or a stage that takes no
// row.  The first one records where it gave up in sched[kSchedGiveUp..+2],
// sets the round's error bit and stops its loop.  The lookups need no such
// bound: at load factor <= 1/4 every walk meets a bucket with a free entry,
// which ends it (and a bound in the probe loop costs about 4 % of the step).
constexpr int32_t kGiveUpInsert = 1, kGiveUpStage = 4;
__device__ __noinline__ void give_up(int32_t *sched, int32_t *err, int32_t code, int32_t v1,
                                     int32_t v2) {
    if (atomicCAS(sched + kSchedGiveUp, 0, code) == 0) {
        sched[kSchedGiveUp + 1] = v1;
        sched[kSchedGiveUp + 2] = v2;
    }
    atomicOr(err, kDevErrInternal);
}

struct ChunkPlan {
    long long chunk;  // items per chunk
    long long total;  // total items
    int32_t nseg;     // segments
    int32_t nact;     // active staged rows
};

struct Pair {
    int32_t a, b;
};
__device__ __forceinline__ Pair operator+(Pair x, Pair y) { return Pair{x.a + y.a, x.b + y.b}; }

__device__ __forceinline__ long long shfl_up(long long v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ int32_t shfl_up(int32_t v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ Pair shfl_up(Pair v, int d) {
    return Pair{__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d)};
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

// Largest i in [lo, hi] with a[i] <= x (a non-decreasing, a[lo] <= x).
template <typename T>
__device__ __forceinline__ int32_t last_le(const T *__restrict__ a, int32_t lo, int32_t hi, T x) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (a[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Row walker for a thread that visits consecutive slots: keeps [rbeg, rend)
// of the current row and jumps over runs of empty rows by binary search.
struct RowWalk {
    int32_t row, rbeg, rend;
    __device__ __forceinline__ void start(const int32_t *__restrict__ rp, int32_t n, int32_t e) {
        row = last_le(rp, 0, n - 1, e);
        rbeg = __ldg(rp + row);
        rend = __ldg(rp + row + 1);
    }
    __device__ __forceinline__ void advance(const int32_t *__restrict__ rp, int32_t n, int32_t e) {
        if (rend > e) return;
        int32_t nr = row + 1;
        int32_t ne = __ldg(rp + nr + 1);
        if (ne <= e) {
            nr = last_le(rp, nr + 1, n - 1, e);
            ne = __ldg(rp + nr + 1);
        }
        row = nr;
        rbeg = __ldg(rp + nr);
        rend = ne;
    }
};

// ------------------------------------------------------------ hash table
// Every staged row gets its own power-of-two region of the shared table.  A
// bucket holds 4 entries: a 32-bit word of four 8-bit fingerprints (0 = free)
// and four 16-bit local slots; the staged columns themselves sit in a plain
// array (vals) indexed by local slot.  A probe loads one fingerprint word,
// compares its four bytes at once and reads a slot and a column only for a
// fingerprint match, so a miss costs a single 4-byte shared load.  Entries of
// a bucket fill in order, so a bucket whose last fingerprint is free ends a
// search.  A region has at least 2 buckets and at most one key per 4 entries.
constexpr uint32_t kHashMul = 0x9E3779B1u;  // Fibonacci hashing: top bits select the bucket
constexpr uint32_t kFpMul = 0x85EBCA6Bu;    // independent multiplier for the fingerprint

// log2 of the bucket count of the region of a row of length len.
__device__ __forceinline__ int region_lb(int32_t len) {
    int lb = 1;
    while ((1 << lb) < len) ++lb;
    return lb;
}

// Fingerprint in [1, 255] (never 0, which marks a free entry).
__device__ __forceinline__ uint32_t fingerprint(int32_t w) {
    return ((uint32_t(w) * kFpMul) >> 24) | 1u;
}

// Bit 7 of byte j is set exactly where byte j of word equals the fingerprint
// replicated in fp4: a byte of x = word ^ fp4 is zero iff neither its low 7
// bits (which would carry into bit 7 when 0x7F is added) nor its bit 7 is
// set.  The addition never carries across bytes, so no other byte is flagged;
// in particular a free entry (byte 0) never matches, since fingerprints are
// never 0.
__device__ __forceinline__ uint32_t match_bytes(uint32_t word, uint32_t fp4) {
    const uint32_t x = word ^ fp4;
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
}

__device__ __forceinline__ bool table_insert(uint32_t *fpw, uint16_t *slots, int32_t bbase, int lb,
                                             int32_t w, int32_t s) {
    const uint32_t bm = (1u << lb) - 1u;
    const uint32_t fp = fingerprint(w);
    uint32_t b = (uint32_t(w) * kHashMul) >> (32 - lb);
    for (uint32_t step = 0; step <= bm; ++step) {
        const int32_t at = bbase + int32_t(b);
        uint32_t old = fpw[at];
        while ((old >> 24) == 0) {  // bucket not full: take its first free entry
            const int j = old == 0 ? 0 : (old >> 16) ? 3 : (old >> 8) ? 2 : 1;
            const uint32_t prev = atomicCAS(fpw + at, old, old | (fp << (8 * j)));
            if (prev == old) {
                slots[4 * at + j] = uint16_t(s);
                return true;
            }
            old = prev;
        }
        b = (b + 1) & bm;
    }
    return false;  // region full: cannot happen at load factor <= 1/4
}

// Local slot of column w in the region starting at bucket bbase with
// 2^(32 - sh) buckets (sh: the bucket shift of the hash), or -1.
__device__ __forceinline__ int32_t table_find(const uint32_t *fpw, const uint16_t *slots,
                                              const int32_t *vals, int32_t bbase, int sh,
                                              int32_t w) {
    const uint32_t bm = 0xffffffffu >> sh;
    const uint32_t fp4 = fingerprint(w) * 0x01010101u;
    uint32_t b = (uint32_t(w) * kHashMul) >> sh;
    for (;;) {
        const int32_t at = bbase + int32_t(b);
        const uint32_t word = fpw[at];
        for (uint32_t mm = match_bytes(word, fp4); mm; mm &= mm - 1u) {
            const int32_t sl = slots[4 * at + ((__ffs(mm) - 1) >> 3)];
            if (vals[sl] == w) return sl;
        }
        if ((word >> 24) == 0) return -1;
        b = (b + 1) & bm;
    }
}

// ------------------------------------------------------- generic tile scan
// Exclusive scan in three kernels: per-tile totals, a one-block scan of the
// totals, and the per-tile rescan that stores the prefixes.  Blocks loop over
// tiles.  With a LoopCtl (the device loop's int32 scan of the update) the
// count is lc->nlist + 1 and nothing runs in rounds without update.
__device__ __forceinline__ bool scan_loop_count(const LoopCtl *lc, int64_t &count) {
    if (!lc) return true;
    if (!(lc->action & kActUpdate)) return false;
    count = int64_t(lc->nlist) + 1;
    return true;
}

template <typename V, typename Load>
__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(Load ld, int64_t count, V *__restrict__ tile_sum, const LoopCtl *lc) {
    __shared__ V part[kScanThreads / 32];
    if (!scan_loop_count(lc, count)) return;
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t i0 = tile * kScanTile + threadIdx.x;
        V s{};
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const int64_t i = i0 + int64_t(j) * kScanThreads;
            if (i < count) s = s + ld(i);
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const V u = shfl_up(s, d);
            if ((threadIdx.x & 31) >= d) s = s + u;
        }
        if ((threadIdx.x & 31) == 31) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            V t{};
            for (int k = 0; k < kScanThreads / 32; ++k) t = t + part[k];
            tile_sum[tile] = t;
        }
        __syncthreads();
    }
}

template <typename V>
__global__ void __launch_bounds__(1024)
scan_totals_kernel(const V *__restrict__ tile_sum, int32_t tiles, V *__restrict__ tile_off,
                   V *__restrict__ total, const LoopCtl *lc) {
    __shared__ V wsum[32];
    if (lc) {
        int64_t count = 0;
        if (!scan_loop_count(lc, count)) return;
        tiles = int32_t((count + kScanTile - 1) / kScanTile);
    }
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t per = (tiles + 1023) / 1024;
    const int32_t b = tid * per, e = min(tiles, b + per);
    V local{};
    for (int32_t k = b; k < e; ++k) local = local + tile_sum[k];
    V incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const V u = shfl_up(incl, d);
        if (lane >= d) incl = incl + u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        V vi = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const V u = shfl_up(vi, d);
            if (lane >= d) vi = vi + u;
        }
        wsum[lane] = vi;  // inclusive over warps
        if (lane == 31) *total = vi;
    }
    __syncthreads();
    V run = w > 0 ? wsum[w - 1] : V{};
    const V prev = shfl_up(incl, 1);
    if (lane > 0) run = run + prev;
    for (int32_t k = b; k < e; ++k) {
        tile_off[k] = run;
        run = run + tile_sum[k];
    }
}

template <typename V, typename Load, typename Store>
__global__ void __launch_bounds__(kScanThreads)
scan_apply_kernel(Load ld, Store st, int64_t count, const V *__restrict__ tile_off,
                  const LoopCtl *lc) {
    __shared__ V part[kScanThreads / 32];
    if (!scan_loop_count(lc, count)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // blocked arrangement: a thread owns kScanPer consecutive items
        const int64_t i0 = tile * kScanTile + int64_t(threadIdx.x) * kScanPer;
        V v[kScanPer];
        V s{};
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const int64_t i = i0 + j;
            v[j] = i < count ? ld(i) : V{};
            s = s + v[j];
        }
        V incl = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const V u = shfl_up(incl, d);
            if (lane >= d) incl = incl + u;
        }
        if (lane == 31) part[w] = incl;
        __syncthreads();
        V run = tile_off[tile];
        for (int k = 0; k < w; ++k) run = run + part[k];
        const V prev = shfl_up(incl, 1);
        if (lane > 0) run = run + prev;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const int64_t i = i0 + j;
            if (i < count) st(i, run);
            run = run + v[j];
        }
        __syncthreads();  // part is rewritten by the next tile
    }
}

// --------------------------------------------------------- balance kernels
// Largest r in [0, n - 1] with rp[r] <= v (rp non-decreasing, rp[0] = 0 <= v),
// found by the whole warp: every pass probes 32 evenly spaced rows and keeps
// the gap between the last probe at or below v and the first above it.  All
// lanes pass the same v and get the same row.
__device__ __forceinline__ int32_t warp_row_of(const int32_t *__restrict__ rp, int32_t n,
                                               int64_t v) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = int64_t(n) - 1;
    while (hi - lo >= 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t p = min(lo + int64_t(lane + 1) * step, hi);
        const int c = __popc(__ballot_sync(0xffffffffu, __ldg(rp + p) <= v));
        const int64_t nlo = c > 0 ? min(lo + int64_t(c) * step, hi) : lo;
        const int64_t nhi = c < 32 ? min(lo + int64_t(c + 1) * step, hi) - 1 : hi;
        lo = nlo;
        hi = nhi;
    }
    const int64_t p = lo + lane;
    const bool le = p <= hi && __ldg(rp + p) <= v;
    return int32_t(lo + __popc(__ballot_sync(0xffffffffu, le)) - 1);
}

// Per live edge: staged row, probe start and item count; per staged row: the
// number of segments; per round: the merge work sum(t + d).  A warp takes a
// window of kClassWin consecutive slots, lane l the slots l, l + 32, ... (so
// loads and stores are coalesced); the window's first row comes from a warp
// search, a lane's later rows from a forward galloping search.  Counts of
// equal staged rows within a warp are aggregated into one atomic.
constexpr int kClassWin = 32 * kEdgesPerThread;
__global__ void __launch_bounds__(kEdgeThreads)
classify_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                int32_t m, int32_t *__restrict__ ekey, int32_t *__restrict__ epst,
                int32_t *__restrict__ eitems, int32_t *__restrict__ rcount,
                unsigned long long *__restrict__ merge_work, const int32_t *__restrict__ gid,
                const uint8_t *__restrict__ skip, int32_t light) {
    __shared__ long long part[kEdgeThreads / 32];
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t(blockIdx.x) * (kEdgeThreads / 32) + (threadIdx.x >> 5)) *
                         kClassWin;
    long long merge = 0;
    if (base < m) {  // warp-uniform
        int32_t row = warp_row_of(rp, n, base);
        int32_t rend = __ldg(rp + row + 1);
#pragma unroll 1
        for (int j = 0; j < kEdgesPerThread; ++j) {
            const int64_t e = base + lane + 32 * j;
            int32_t key = -1;
            if (e < m) {
                if (rend <= e) {
                    // rows row+1 .. are at or below e: gallop to a bound above it
                    int64_t lo = row + 1, step = 1, hi = lo + 1;
                    while (hi <= n - 1 && __ldg(rp + hi) <= e) {
                        lo = hi;
                        step <<= 1;
                        hi = lo + step;
                    }
                    row = last_le(rp, int32_t(lo), int32_t(min(hi - 1, int64_t(n) - 1)),
                                  int32_t(e));
                    rend = __ldg(rp + row + 1);
                }
                const int32_t kappa = __ldg(col + e);
                const int32_t kb = __ldg(rp + kappa);
                const int32_t d = __ldg(rp + kappa + 1) - kb;
                const int32_t t = rend - int32_t(e) - 1;
                const bool skipped = skip && skip[gid[row]];
                if (!skipped) merge += (long long)t + d;
                const int32_t items = (skipped || light_task(t, d, light)) ? 0 : min(t, d);
                if (items > 0) {
                    const bool stage_kappa = t < d;
                    key = stage_kappa ? kappa : row;
                    epst[e] = stage_kappa ? int32_t(e) + 1 : kb;
                }
                ekey[e] = key;
                eitems[e] = items;
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(rcount + key, __popc(peers));
        }
    }
    merge = warp_sum_ll(merge);
    if (lane == 0) part[threadIdx.x >> 5] = merge;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < kEdgeThreads / 32; ++k) t += part[k];
        if (t) atomicAdd(merge_work, (unsigned long long)t);
    }
}

// Light tasks: a thread walks kLightPerThread consecutive slots and merges the
// tail of row i after each light task's slot with row kappa (Listing 1's
// two-pointer loop), crediting both matching slots and, once, its own slot.
__global__ void __launch_bounds__(kEdgeThreads)
support_light_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                     int32_t m, int32_t *__restrict__ S, unsigned long long *__restrict__ tri,
                     const int32_t *__restrict__ gid, const uint8_t *__restrict__ skip,
                     int32_t light) {
    const int64_t e0 = (int64_t(blockIdx.x) * kEdgeThreads + threadIdx.x) * kLightPerThread;
    int32_t found = 0;
    if (e0 < m) {
        RowWalk rw{0, 0, 0};
        rw.start(rp, n, int32_t(e0));
#pragma unroll 1
        for (int j = 0; j < kLightPerThread; ++j) {
            const int64_t e = e0 + j;
            if (e >= m) break;
            rw.advance(rp, n, int32_t(e));
            const int32_t kappa = __ldg(col + e);
            int32_t y = __ldg(rp + kappa);
            const int32_t ye = __ldg(rp + kappa + 1);
            int32_t x = int32_t(e) + 1;
            const int32_t xe = rw.rend;
            if (x >= xe || y >= ye || !light_task(xe - x, ye - y, light)) continue;
            if (skip && skip[gid[rw.row]]) continue;
            int32_t own = 0;
            while (x < xe && y < ye) {
                const int32_t a = __ldg(col + x), b = __ldg(col + y);
                if (a == b) {
                    atomicAdd(S + x, 1);
                    atomicAdd(S + y, 1);
                    ++own;
                    ++x;
                    ++y;
                } else if (a < b) {
                    ++x;
                } else {
                    ++y;
                }
            }
            if (own) atomicAdd(S + e, own);
            found += own;
        }
    }
    const int32_t tot = __reduce_add_sync(0xffffffffu, found);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(tri, (unsigned long long)tot);
}

struct RowCountLoad {
    const int32_t *rcount;
    __device__ Pair operator()(int64_t i) const {
        const int32_t c = rcount[i];
        return Pair{c, c > 0 ? 1 : 0};
    }
};
struct RowCountStore {
    int32_t *rstart, *arank;
    __device__ void operator()(int64_t i, Pair v) const {
        rstart[i] = v.a;
        arank[i] = v.b;
    }
};

// Active staged rows (rows with at least one segment), in row order, and
// their first segment position; aseg[nact] = number of segments.
__global__ void active_rows_kernel(const int32_t *__restrict__ rcount,
                                   const int32_t *__restrict__ rstart,
                                   const int32_t *__restrict__ arank, const Pair *__restrict__ tot,
                                   int32_t n, int32_t *__restrict__ arow,
                                   int32_t *__restrict__ aseg) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r < n && rcount[r] > 0) {
        arow[arank[r]] = int32_t(r);
        aseg[arank[r]] = rstart[r];
    }
    if (r == 0) aseg[tot->b] = tot->a;
}

// Counting-sort scatter of the segments by staged row (consumes rcount).  A
// segment is one 16-byte record (owner slot, probe start, item count,
// active-row rank of its staged row), so its scatter is one random write.
__global__ void scatter_kernel(const int32_t *__restrict__ ekey, const int32_t *__restrict__ epst,
                               const int32_t *__restrict__ eitems, int32_t m,
                               const int32_t *__restrict__ rstart,
                               const int32_t *__restrict__ arank, int32_t *__restrict__ rcount,
                               int4 *__restrict__ srec) {
    const int lane = threadIdx.x & 31;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int32_t key = e < m ? ekey[e] : -1;
    const uint32_t peers = __match_any_sync(0xffffffffu, key);
    if (key < 0) return;
    const int leader = __ffs(peers) - 1;
    int32_t old = 0;
    if (lane == leader) old = atomicSub(rcount + key, __popc(peers));
    old = __shfl_sync(peers, old, leader);
    const int32_t pos = rstart[key] + old - 1 - __popc(peers & ((1u << lane) - 1u));
    srec[pos] = make_int4(int32_t(e), epst[e], eitems[e], arank[key]);
}

struct ItemLoad {
    const int4 *srec;
    const Pair *tot;
    __device__ long long operator()(int64_t i) const { return i < tot->a ? srec[i].z : 0; }
};
struct ItemStore {
    long long *wp;
    __device__ void operator()(int64_t i, long long v) const { wp[i] = v; }
};

// Chunk size: about kChunksPerCta chunks per resident CTA, at least kChunkMin
// items, at most kMaxChunks chunks.
__global__ void plan_kernel(const long long *__restrict__ total, const Pair *__restrict__ tot,
                            long long *__restrict__ wp, ChunkPlan *plan,
                            int32_t *__restrict__ sched, int32_t resident_ctas) {
    const long long t = *total;
    const long long want = (long long)resident_ctas * kChunksPerCta;
    long long c = (t + want - 1) / want;
    if (c < kChunkMin) c = kChunkMin;
    long long nch = (t + c - 1) / c;
    if (nch > kMaxChunks) {
        c = (t + kMaxChunks - 1) / kMaxChunks;
        nch = (t + c - 1) / c;
    }
    plan->chunk = c;
    plan->total = t;
    plan->nseg = tot->a;
    plan->nact = tot->b;
    wp[tot->a] = t;
    sched[kSchedNChunks] = int32_t(nch);
}

// bound[c] = (segment holding item c*chunk, active row holding that segment).
__global__ void partition_kernel(const long long *__restrict__ wp, const int32_t *__restrict__ aseg,
                                 const ChunkPlan *__restrict__ plan,
                                 const int32_t *__restrict__ sched, int2 *__restrict__ bound) {
    const int32_t nch = sched[kSchedNChunks];
    const long long chunk = plan->chunk, total = plan->total;
    const int32_t nseg = plan->nseg, nact = plan->nact;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c <= nch;
         c += int64_t(gridDim.x) * blockDim.x) {
        if (nseg == 0) {
            bound[c] = make_int2(0, 0);
            continue;
        }
        long long item = c * chunk;
        if (item > total) item = total;
        const int32_t p = last_le(wp, 0, nseg - 1, item);
        bound[c] = make_int2(p, last_le(aseg, 0, nact - 1, p));
    }
}

// ------------------------------------------------------------ support kernel
// Two CTA shapes of the support kernel (support_shape.cuh), chosen per handle
// (KTRUSS_OPT_SUPPORT_SHAPE, picked by the autotuner):
//   shape 0: 1024-thread CTAs, one per SM, stages and pieces of 8192 slots
//   shape 1: 512-thread CTAs, three per SM (48 warps resident instead of 32),
//            stages and pieces of 2048 slots
namespace shape0 {
constexpr int kThreads = 1024, kCap = 8192, kMinCtas = 1;
#include "support_shape.cuh"
}  // namespace shape0
namespace shape1 {
constexpr int kThreads = 512, kCap = 2048, kMinCtas = 3;
#include "support_shape.cuh"
}  // namespace shape1

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

struct Carve {
    // seg, pst, sitems and sact are consecutive: the support step uses their
    // memory as one array of 16-byte segment records (srec), the update as
    // four int32 arrays
    int32_t *ekey, *epst, *eitems, *seg, *pst, *sitems, *sact;
    int4 *srec;
    long long *wp;
    int32_t *rcount, *rstart, *arank, *arow, *aseg;
    Pair *rtile_sum, *rtile_off, *rtot;
    long long *itile_sum, *itile_off, *itot;
    ChunkPlan *plan;
    int2 *bound;
    int32_t *sched;
};

// Lays the scratch out in one allocation; with base == nullptr only sizes it.
size_t carve(void *base, int32_t n, int64_t m, Carve *c) {
    char *p = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    const int64_t mt = (m + kScanTile - 1) / kScanTile + 1;
    const int64_t nt = (int64_t(n) + 1 + kScanTile - 1) / kScanTile + 1;
    c->ekey = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->epst = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->eitems = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->seg = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->pst = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->sitems = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->sact = reinterpret_cast<int32_t *>(take(size_t(m + 1) * 4));
    c->srec = reinterpret_cast<int4 *>(c->seg);
    c->wp = reinterpret_cast<long long *>(take(size_t(m + 2) * 8));
    c->rcount = reinterpret_cast<int32_t *>(take(size_t(n + 1) * 4));
    c->rstart = reinterpret_cast<int32_t *>(take(size_t(n + 1) * 4));
    c->arank = reinterpret_cast<int32_t *>(take(size_t(n + 1) * 4));
    c->arow = reinterpret_cast<int32_t *>(take(size_t(n + 1) * 4));
    c->aseg = reinterpret_cast<int32_t *>(take(size_t(n + 2) * 4));
    c->rtile_sum = reinterpret_cast<Pair *>(take(size_t(nt) * sizeof(Pair)));
    c->rtile_off = reinterpret_cast<Pair *>(take(size_t(nt) * sizeof(Pair)));
    c->rtot = reinterpret_cast<Pair *>(take(sizeof(Pair)));
    c->itile_sum = reinterpret_cast<long long *>(take(size_t(mt) * 8));
    c->itile_off = reinterpret_cast<long long *>(take(size_t(mt) * 8));
    c->itot = reinterpret_cast<long long *>(take(8));
    c->plan = reinterpret_cast<ChunkPlan *>(take(sizeof(ChunkPlan)));
    c->bound = reinterpret_cast<int2 *>(take(size_t(kMaxChunks + 2) * 8));
    c->sched = reinterpret_cast<int32_t *>(take(kSchedWords * 4));
    return off;
}

struct I32Load {
    const int32_t *a;
    __device__ __forceinline__ int32_t operator()(int64_t i) const { return a[i]; }
};
struct I32Store {
    int32_t *out;
    __device__ __forceinline__ void operator()(int64_t i, int32_t v) const { out[i] = v; }
};

}  // namespace

UpdateScratch update_scratch(const BalancedScratch *bs) {
    Carve c;
    carve(bs->base, bs->cap_n, bs->cap_m, &c);
    return UpdateScratch{c.ekey,
                         c.epst,
                         c.eitems,
                         c.seg,
                         c.pst,
                         c.sitems,
                         reinterpret_cast<int32_t *>(c.wp),
                         c.sact,
                         reinterpret_cast<int32_t *>(c.itile_sum),
                         reinterpret_cast<int32_t *>(c.itile_off),
                         reinterpret_cast<int32_t *>(c.itot)};
}

cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t count,
                            const UpdateScratch &u, cudaStream_t s, int *launches,
                            const LoopCtl *lc) {
    if (count <= 0) return cudaSuccess;
    int32_t tiles = int32_t((count + kScanTile - 1) / kScanTile);
    const int32_t grid = lc && tiles > kLoopBlocks ? kLoopBlocks : tiles;
    I32Load ld{in};
    I32Store st{out};
    scan_reduce_kernel<int32_t, I32Load><<<grid, kScanThreads, 0, s>>>(ld, count, u.scan_sum, lc);
    scan_totals_kernel<int32_t><<<1, 1024, 0, s>>>(u.scan_sum, tiles, u.scan_off, u.scan_tot, lc);
    scan_apply_kernel<int32_t, I32Load, I32Store>
        <<<grid, kScanThreads, 0, s>>>(ld, st, count, u.scan_off, lc);
    *launches += 3;
    return cudaGetLastError();
}

size_t balanced_scratch_bytes(int32_t n, int64_t m) {
    Carve c;
    return carve(nullptr, n, m, &c);
}

cudaError_t balanced_scratch_alloc(BalancedScratch *bs, int32_t n, int64_t m) {
    void *p = nullptr;
    // large enough to also serve as the degree-ordered relabel's working
    // memory for any graph within the capacity (the server relabels requests)
    const size_t a = balanced_scratch_bytes(n, m), b = reorder_scratch_bytes(n, m);
    cudaError_t e = cudaMalloc(&p, a > b ? a : b);
    if (e != cudaSuccess) return e;
    bs->base = p;
    bs->cap_m = m;
    bs->cap_n = n;
    return cudaSuccess;
}

cudaError_t balanced_side_create(BalancedScratch *bs) {
    cudaError_t e = cudaStreamCreateWithFlags(&bs->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->join, cudaEventDisableTiming);
    if (e != cudaSuccess) balanced_side_destroy(bs);
    return e;
}

void balanced_side_destroy(BalancedScratch *bs) {
    if (bs->fork) cudaEventDestroy(bs->fork);
    if (bs->join) cudaEventDestroy(bs->join);
    if (bs->side) cudaStreamDestroy(bs->side);
    bs->side = nullptr;
    bs->fork = bs->join = nullptr;
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
    const int shape = bs->shape == 0 ? 0 : 1;
    int blocks = 0;
    cudaError_t e = shape == 0 ? shape0::configure_support(&blocks)
                               : shape1::configure_support(&blocks);
    if (e != cudaSuccess) return e;
    Carve c;
    carve(bs->base, bs->cap_n, bs->cap_m, &c);
    const int32_t n = g.n, m = g.m;
    // light tasks first: on the side stream they overlap the balancing
    // kernels below (S is zero on entry in stream order, so the fork is safe)
    const bool side = bs->side && bs->light > 0;
    if (bs->light > 0) {
        cudaStream_t ls = s;
        if (side) {
            e = cudaEventRecord(bs->fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(bs->side, bs->fork, 0);
            if (e != cudaSuccess) return e;
            ls = bs->side;
        }
        const int64_t lblocks = (int64_t(m) + int64_t(kEdgeThreads) * kLightPerThread - 1) /
                                (int64_t(kEdgeThreads) * kLightPerThread);
        support_light_kernel<<<int(lblocks), kEdgeThreads, 0, ls>>>(
            g.rp, g.col, n, m, S, &cnt->triangles, g.gid, g.skip, bs->light);
        *launches += 1;
        if (side) {
            e = cudaEventRecord(bs->join, bs->side);
            if (e != cudaSuccess) return e;
        }
    }
    e = cudaMemsetAsync(c.rcount, 0, size_t(n + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.sched, 0, kSchedWords * 4, s);
    if (e != cudaSuccess) return e;
    const int eblocks = int((int64_t(m) + kEdgeThreads * kEdgesPerThread - 1) /
                            (kEdgeThreads * kEdgesPerThread));
    classify_kernel<<<eblocks, kEdgeThreads, 0, s>>>(g.rp, g.col, n, m, c.ekey, c.epst, c.eitems,
                                                     c.rcount, &cnt->merge_work, g.gid, g.skip,
                                                     bs->light);
    trace_phase(s, "classify");
    // row scan: segment starts and active-row ranks (row n has count 0, so the
    // entries at n are the totals)
    const int64_t rows = int64_t(n) + 1;
    const int32_t rtiles = int32_t((rows + kScanTile - 1) / kScanTile);
    RowCountLoad rl{c.rcount};
    RowCountStore rs{c.rstart, c.arank};
    scan_reduce_kernel<Pair, RowCountLoad><<<rtiles, kScanThreads, 0, s>>>(rl, rows, c.rtile_sum,
                                                                       nullptr);
    scan_totals_kernel<Pair><<<1, 1024, 0, s>>>(c.rtile_sum, rtiles, c.rtile_off, c.rtot, nullptr);
    scan_apply_kernel<Pair, RowCountLoad, RowCountStore>
        <<<rtiles, kScanThreads, 0, s>>>(rl, rs, rows, c.rtile_off, nullptr);
    active_rows_kernel<<<int((rows + 255) / 256), 256, 0, s>>>(c.rcount, c.rstart, c.arank,
                                                               c.rtot, n, c.arow, c.aseg);
    trace_phase(s, "row scan + active rows");
    scatter_kernel<<<int((int64_t(m) + 255) / 256), 256, 0, s>>>(c.ekey, c.epst, c.eitems, m, c.rstart,
                                                   c.arank, c.rcount, c.srec);
    trace_phase(s, "scatter");
    // item scan over the segments (at most m of them; entries past nseg are 0)
    const int32_t itiles = int32_t((int64_t(m) + kScanTile - 1) / kScanTile);
    ItemLoad il{c.srec, c.rtot};
    ItemStore is{c.wp};
    scan_reduce_kernel<long long, ItemLoad><<<itiles, kScanThreads, 0, s>>>(il, m, c.itile_sum,
                                                                          nullptr);
    scan_totals_kernel<long long><<<1, 1024, 0, s>>>(c.itile_sum, itiles, c.itile_off, c.itot,
                                                     nullptr);
    scan_apply_kernel<long long, ItemLoad, ItemStore>
        <<<itiles, kScanThreads, 0, s>>>(il, is, m, c.itile_off, nullptr);
    trace_phase(s, "item scan");
    plan_kernel<<<1, 1, 0, s>>>(c.itot, c.rtot, c.wp, c.plan, c.sched, blocks);
    partition_kernel<<<64, 256, 0, s>>>(c.wp, c.aseg, c.plan, c.sched, c.bound);
    trace_phase(s, "plan + partition");
    if (trace_phases()) {
        ChunkPlan hp{};
        int32_t hs[kSchedWords] = {};
        if (cudaMemcpy(&hp, c.plan, sizeof(hp), cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaMemcpy(hs, c.sched, sizeof(hs), cudaMemcpyDeviceToHost) == cudaSuccess)
            std::fprintf(stderr, "[ktruss phase] plan: items %lld chunk %lld chunks %d segments %d "
                         "active rows %d (n %d m %d)\n", hp.total, hp.chunk, hs[kSchedNChunks],
                         hp.nseg, hp.nact, n, m);
    }
    *launches += 12;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) {
        e = cudaEventRecord(ev[1], s);
        if (e != cudaSuccess) return e;
    }
    if (shape == 0) {
        shape0::SupportArgs A{g.rp, g.col, c.srec, c.wp, c.arow, c.aseg, c.plan,
                              c.bound, c.sched, S, &cnt->triangles, &cnt->error};
        shape0::support_kernel<<<blocks, shape0::kThreads, sizeof(shape0::SupportSmem), s>>>(A);
    } else {
        shape1::SupportArgs A{g.rp, g.col, c.srec, c.wp, c.arow, c.aseg, c.plan,
                              c.bound, c.sched, S, &cnt->triangles, &cnt->error};
        shape1::support_kernel<<<blocks, shape1::kThreads, sizeof(shape1::SupportSmem), s>>>(A);
    }
    if (side) {
        e = cudaStreamWaitEvent(s, bs->join, 0);
        if (e != cudaSuccess) return e;
    }
    trace_phase(s, "support_kernel");
    if (trace_phases()) {
        int32_t hs[kSchedWords] = {};
        if (cudaMemcpy(hs, c.sched, sizeof(hs), cudaMemcpyDeviceToHost) == cudaSuccess &&
            hs[kSchedGiveUp] != 0)
            std::fprintf(stderr, "[ktruss phase] support_kernel gave up: code %d values %d %d\n",
                         hs[kSchedGiveUp], hs[kSchedGiveUp + 1], hs[kSchedGiveUp + 2]);
    }
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace kt
