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
//    memory hash table keyed by (row, column) -> slot; warps take segments
//    dynamically, stream the probe list with coalesced loads and probe the
//    table.  A staged row longer than kCap is loaded piece by piece (in column
//    order); each segment keeps a cursor that advances through its probe list
//    piece by piece, so every probe is still read once.  Credits to staged
//    slots are gathered in shared memory and flushed once per stage or piece.
//
// All credits are integer additions, so the result does not depend on the
// order in which CTAs, warps or the counting sort place the work.
#include <cstdint>

#include "ktruss_internal.cuh"

namespace kt {
namespace {

// ----------------------------------------------------------- configuration
constexpr int kThreads = 512;           // threads per support CTA
constexpr int kCap = 4096;              // staged slots per stage or piece
constexpr int kTable = 2 * kCap;        // hash entries (load factor <= 1/2)
constexpr int kStageRows = 256;         // staged rows per stage
constexpr int kSegBatch = 512;          // segments per long-row batch
constexpr long long kChunkMin = 65536;  // items per chunk (minimum)
constexpr int kChunksPerCta = 16;       // target chunks per resident CTA
constexpr int kMaxChunks = 1 << 17;     // chunk table capacity

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kEdgeThreads = 256;
constexpr int kEdgesPerThread = 16;

constexpr int32_t kEmpty = -1;
constexpr int32_t kIntMax = 0x7fffffff;

// sched[] words
constexpr int kSchedChunkNext = 0;
constexpr int kSchedNChunks = 1;
constexpr int kSchedWords = 8;

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
// Buckets of 4 int32 keys (one 16-byte shared load per probe), a parallel
// array of 16-bit local slots, load factor <= 1/2.  key_row disambiguates
// equal columns of different staged rows.
__device__ __forceinline__ uint32_t bucket_of(int32_t key_row, int32_t w, uint32_t mask) {
    uint32_t h = uint32_t(w) * 0x9E3779B1u + uint32_t(key_row) * 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 13;
    return h & mask;
}

__device__ __forceinline__ void table_insert(int32_t *keys, uint16_t *slots, uint32_t mask,
                                             int32_t key_row, int32_t w, int32_t s) {
    uint32_t b = bucket_of(key_row, w, mask);
    for (;;) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (atomicCAS(keys + 4 * b + j, kEmpty, w) == kEmpty) {
                slots[4 * b + j] = uint16_t(s);
                return;
            }
        }
        b = (b + 1) & mask;
    }
}

// Local slot of column w in the staged slots [lo, hi) of key_row, or -1.
__device__ __forceinline__ int32_t table_find(const int32_t *keys, const uint16_t *slots,
                                              uint32_t mask, int32_t key_row, int32_t w,
                                              int32_t lo, int32_t hi) {
    uint32_t b = bucket_of(key_row, w, mask);
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
        b = (b + 1) & mask;
    }
}

__device__ __forceinline__ int table_size_for(int32_t len) {
    int t = 64;
    while (t < 2 * len) t <<= 1;
    return t;
}

// ------------------------------------------------------- generic tile scan
// Exclusive scan in three kernels: per-tile totals, a one-block scan of the
// totals, and the per-tile rescan that stores the prefixes.
template <typename V, typename Load>
__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(Load ld, int64_t count, V *__restrict__ tile_sum) {
    __shared__ V part[kScanThreads / 32];
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + threadIdx.x;
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
        tile_sum[blockIdx.x] = t;
    }
}

template <typename V>
__global__ void __launch_bounds__(1024)
scan_totals_kernel(const V *__restrict__ tile_sum, int32_t tiles, V *__restrict__ tile_off,
                   V *__restrict__ total) {
    __shared__ V wsum[32];
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
scan_apply_kernel(Load ld, Store st, int64_t count, const V *__restrict__ tile_off) {
    __shared__ V part[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // blocked arrangement: a thread owns kScanPer consecutive items
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
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
    V run = tile_off[blockIdx.x];
    for (int k = 0; k < w; ++k) run = run + part[k];
    const V prev = shfl_up(incl, 1);
    if (lane > 0) run = run + prev;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        const int64_t i = i0 + j;
        if (i < count) st(i, run);
        run = run + v[j];
    }
}

// --------------------------------------------------------- balance kernels
// Per live edge: staged row, probe start and item count; per staged row: the
// number of segments; per round: the merge work sum(t + d).
__global__ void __launch_bounds__(kEdgeThreads)
classify_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                int32_t m, int32_t *__restrict__ ekey, int32_t *__restrict__ epst,
                int32_t *__restrict__ eitems, int32_t *__restrict__ rcount,
                unsigned long long *__restrict__ merge_work) {
    __shared__ long long part[kEdgeThreads / 32];
    const int64_t e0 = (int64_t(blockIdx.x) * kEdgeThreads + threadIdx.x) * kEdgesPerThread;
    long long merge = 0;
    if (e0 < m) {
        RowWalk rw;
        rw.start(rp, n, int32_t(e0));
        const int32_t e1 = int32_t(min(int64_t(m), e0 + kEdgesPerThread));
        for (int32_t e = int32_t(e0); e < e1; ++e) {
            rw.advance(rp, n, e);
            const int32_t kappa = __ldg(col + e);
            const int32_t kb = __ldg(rp + kappa);
            const int32_t d = __ldg(rp + kappa + 1) - kb;
            const int32_t t = rw.rend - e - 1;
            merge += (long long)t + d;
            const int32_t items = min(t, d);
            int32_t key = -1;
            if (items > 0) {
                const bool stage_kappa = t < d;
                key = stage_kappa ? kappa : rw.row;
                epst[e] = stage_kappa ? e + 1 : kb;
                atomicAdd(rcount + key, 1);
            }
            ekey[e] = key;
            eitems[e] = items;
        }
    }
    merge = warp_sum_ll(merge);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = merge;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < kEdgeThreads / 32; ++k) t += part[k];
        if (t) atomicAdd(merge_work, (unsigned long long)t);
    }
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

// Counting-sort scatter of the segments by staged row (consumes rcount).
__global__ void scatter_kernel(const int32_t *__restrict__ ekey, const int32_t *__restrict__ epst,
                               const int32_t *__restrict__ eitems, int32_t m,
                               const int32_t *__restrict__ rstart, int32_t *__restrict__ rcount,
                               int32_t *__restrict__ seg, int32_t *__restrict__ pst,
                               int32_t *__restrict__ sitems) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t key = ekey[e];
    if (key < 0) return;
    const int32_t pos = rstart[key] + atomicSub(rcount + key, 1) - 1;
    seg[pos] = int32_t(e);
    pst[pos] = epst[e];
    sitems[pos] = eitems[e];
}

struct ItemLoad {
    const int32_t *sitems;
    const Pair *tot;
    __device__ long long operator()(int64_t i) const { return i < tot->a ? sitems[i] : 0; }
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
struct StageDesc {
    int32_t gbase[kStageRows];     // global slot of each staged row's first element
    int32_t loc[kStageRows + 1];   // local slot offsets (prefix of row lengths)
    int32_t segb[kStageRows + 1];  // first segment position of each staged row
};
struct LongDesc {
    int32_t cur[kSegBatch];    // next probe position of each segment
    int32_t end[kSegBatch];    // end of the segment's probes in this chunk
    int32_t own[kSegBatch];    // hits counted for the segment's owner edge
    int32_t owner[kSegBatch];  // owner edge slot
};
struct SupportSmem {
    int32_t keys[kTable];
    uint16_t slots[kTable];
    int32_t cnt[kCap];
    union {
        StageDesc st;
        LongDesc lg;
    } u;
    int32_t ctl[32];
};

struct SupportArgs {
    const int32_t *rp, *col;
    const int32_t *seg, *pst;
    const long long *wp;
    const int32_t *arow, *aseg;
    const ChunkPlan *plan;
    const int2 *bound;
    int32_t *sched;
    int32_t *S;
    unsigned long long *tri;
};

// Probes the staged table with col[x], x in [x0, x1), lanes striding by 32
// (four loads in flight per lane); returns this lane's hits.
__device__ __forceinline__ int32_t probe_range(const SupportArgs &A, SupportSmem &sm,
                                               uint32_t mask, int32_t key_row, int32_t qlo,
                                               int32_t qhi, int32_t x0, int32_t x1, int lane) {
    int32_t own = 0;
    int32_t x = x0 + lane;
    for (; x + 96 < x1; x += 128) {
        const int32_t w0 = __ldg(A.col + x), w1 = __ldg(A.col + x + 32);
        const int32_t w2 = __ldg(A.col + x + 64), w3 = __ldg(A.col + x + 96);
        const int32_t q0 = table_find(sm.keys, sm.slots, mask, key_row, w0, qlo, qhi);
        const int32_t q1 = table_find(sm.keys, sm.slots, mask, key_row, w1, qlo, qhi);
        const int32_t q2 = table_find(sm.keys, sm.slots, mask, key_row, w2, qlo, qhi);
        const int32_t q3 = table_find(sm.keys, sm.slots, mask, key_row, w3, qlo, qhi);
        if (q0 >= 0) { atomicAdd(&sm.cnt[q0], 1); atomicAdd(A.S + x, 1); ++own; }
        if (q1 >= 0) { atomicAdd(&sm.cnt[q1], 1); atomicAdd(A.S + x + 32, 1); ++own; }
        if (q2 >= 0) { atomicAdd(&sm.cnt[q2], 1); atomicAdd(A.S + x + 64, 1); ++own; }
        if (q3 >= 0) { atomicAdd(&sm.cnt[q3], 1); atomicAdd(A.S + x + 96, 1); ++own; }
    }
    for (; x < x1; x += 32) {
        const int32_t w = __ldg(A.col + x);
        const int32_t q = table_find(sm.keys, sm.slots, mask, key_row, w, qlo, qhi);
        if (q >= 0) { atomicAdd(&sm.cnt[q], 1); atomicAdd(A.S + x, 1); ++own; }
    }
    return own;
}

__device__ __forceinline__ void clear_table(SupportSmem &sm, int tsize, int32_t len, int tid) {
    for (int k = tid; k < tsize / 4; k += kThreads)
        reinterpret_cast<int4 *>(sm.keys)[k] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
    for (int k = tid; k < len; k += kThreads) sm.cnt[k] = 0;
}

// The segments [s0, s1) of chunk [iA, iB) whose staged row (rbase, L) is
// longer than kCap: piece by piece, with a cursor per segment.
__device__ void long_row(const SupportArgs &A, SupportSmem &sm, int32_t rbase, int32_t L,
                         int32_t s0, int32_t s1, long long iA, long long iB,
                         unsigned long long &tri) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t npieces = (L + kCap - 1) / kCap;
    for (int32_t sb = s0; sb < s1; sb += kSegBatch) {
        const int32_t nb = min(kSegBatch, s1 - sb);
        int32_t minv = kIntMax;
        for (int j = tid; j < nb; j += kThreads) {
            const int32_t pos = sb + j;
            const long long base = __ldg(A.wp + pos);
            const int32_t ka = int32_t(max(iA, base) - base);
            const int32_t kb = int32_t(min(iB, __ldg(A.wp + pos + 1)) - base);
            const int32_t p0 = __ldg(A.pst + pos);
            sm.u.lg.cur[j] = p0 + ka;
            sm.u.lg.end[j] = p0 + max(ka, kb);
            sm.u.lg.own[j] = 0;
            sm.u.lg.owner[j] = __ldg(A.seg + pos);
            if (kb > ka) minv = min(minv, __ldg(A.col + p0 + ka));
        }
        minv = __reduce_min_sync(0xffffffffu, minv);
        if (lane == 0) sm.ctl[16 + warp] = minv;
        __syncthreads();
        if (tid == 0) {
            int32_t mv = kIntMax;
            for (int k = 0; k < kThreads / 32; ++k) mv = min(mv, sm.ctl[16 + k]);
            // the last piece starting at a column <= mv holds the smallest probe
            int32_t lo = 0, hi = npieces - 1;
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;
                if (__ldg(A.col + rbase + mid * kCap) <= mv) lo = mid; else hi = mid - 1;
            }
            sm.ctl[2] = mv == kIntMax ? npieces : lo;
        }
        __syncthreads();
        const int32_t pfirst = sm.ctl[2];
        for (int32_t p = pfirst; p < npieces; ++p) {
            const int32_t ps = rbase + p * kCap;
            const int32_t plen = min(kCap, L - p * kCap);
            const int32_t vhi = (p + 1 < npieces) ? __ldg(A.col + ps + plen) : kIntMax;
            const int tsize = table_size_for(plen);
            const uint32_t mask = uint32_t(tsize / 4 - 1);
            clear_table(sm, tsize, plen, tid);
            if (tid == 0) sm.ctl[1] = 0;
            __syncthreads();
            for (int k = tid; k < plen; k += kThreads)
                table_insert(sm.keys, sm.slots, mask, 0, __ldg(A.col + ps + k), k);
            __syncthreads();
            for (;;) {
                int32_t j = 0;
                if (lane == 0) j = atomicAdd(&sm.ctl[1], 1);
                j = __shfl_sync(0xffffffffu, j, 0);
                if (j >= nb) break;
                int32_t k = sm.u.lg.cur[j];
                const int32_t ke = sm.u.lg.end[j];
                if (k >= ke) continue;
                int32_t own = 0;
                for (;;) {
                    const int32_t x = k + lane;
                    const int32_t w = x < ke ? __ldg(A.col + x) : kIntMax;
                    const bool in = w < vhi;
                    if (in) {
                        const int32_t q = table_find(sm.keys, sm.slots, mask, 0, w, 0, plen);
                        if (q >= 0) {
                            atomicAdd(&sm.cnt[q], 1);
                            atomicAdd(A.S + x, 1);
                            ++own;
                        }
                    }
                    const int32_t nin = __popc(__ballot_sync(0xffffffffu, in));
                    k += nin;
                    if (nin < 32) break;
                }
                own = __reduce_add_sync(0xffffffffu, own);
                if (lane == 0) {
                    sm.u.lg.cur[j] = k;
                    sm.u.lg.own[j] += own;
                }
            }
            __syncthreads();
            for (int k = tid; k < plen; k += kThreads) {
                const int32_t v = sm.cnt[k];
                if (v) atomicAdd(A.S + ps + k, v);
            }
            int32_t left = 0;
            for (int j = tid; j < nb; j += kThreads) left |= sm.u.lg.cur[j] < sm.u.lg.end[j];
            if (!__syncthreads_or(left)) break;  // every cursor exhausted
        }
        __syncthreads();
        for (int j = tid; j < nb; j += kThreads) {
            const int32_t v = sm.u.lg.own[j];
            if (v) {
                atomicAdd(A.S + sm.u.lg.owner[j], v);
                tri += v;
            }
        }
        __syncthreads();
    }
}

// Forms a stage of consecutive short active rows starting at active row a
// (warp 0): rows a .. a+nr-1 with total length <= kCap and nr <= kStageRows.
__device__ void form_stage(const SupportArgs &A, SupportSmem &sm, int32_t a, int32_t ab) {
    const int lane = threadIdx.x & 31;
    int32_t acc = 0, nr = 0;
    for (;;) {
        const int32_t ai = a + nr + lane;
        int32_t len = -1, gb = 0, sgb = 0;
        if (ai <= ab && nr + lane < kStageRows) {
            const int32_t rr = __ldg(A.arow + ai);
            gb = __ldg(A.rp + rr);
            len = __ldg(A.rp + rr + 1) - gb;
            sgb = __ldg(A.aseg + ai);
            if (len > kCap) len = -1;
        }
        // inclusive prefix of lengths, saturating above kCap (ineligible rows
        // count as kCap + 1 so that every later lane fails too)
        int32_t incl = len < 0 ? kCap + 1 : len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl = min(incl + u, kCap + 1);
        }
        const bool ok = len >= 0 && acc + incl <= kCap;
        const uint32_t okm = __ballot_sync(0xffffffffu, ok);
        const int tk = okm == 0xffffffffu ? 32 : __ffs(~okm) - 1;  // ok is a lane prefix
        if (lane < tk) {
            sm.u.st.gbase[nr + lane] = gb;
            sm.u.st.loc[nr + lane] = acc + incl - len;
            sm.u.st.segb[nr + lane] = sgb;
        }
        if (tk > 0) acc += __shfl_sync(0xffffffffu, incl, tk - 1);
        nr += tk;
        if (tk < 32) break;
    }
    if (lane == 0) {
        sm.u.st.loc[nr] = acc;
        sm.u.st.segb[nr] = __ldg(A.aseg + a + nr);
        sm.ctl[3] = nr;
        sm.ctl[1] = 0;
    }
}

__global__ void __launch_bounds__(kThreads, 3)
support_kernel(SupportArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SupportSmem &sm = *reinterpret_cast<SupportSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t nch = A.sched[kSchedNChunks];
    const long long chunk = A.plan->chunk, total = A.plan->total;
    unsigned long long tri = 0;
    for (;;) {
        if (tid == 0) sm.ctl[0] = atomicAdd(A.sched + kSchedChunkNext, 1);
        __syncthreads();
        const int32_t c = sm.ctl[0];
        __syncthreads();
        if (c >= nch) break;
        const long long iA = c * chunk;
        const long long iB = min(total, iA + chunk);
        const int2 b0 = A.bound[c], b1 = A.bound[c + 1];
        const int32_t pa = b0.x, pb = b1.x;  // segment positions [pa, pb]
        const int32_t ab = b1.y;
        int32_t a = b0.y;
        while (a <= ab) {
            const int32_t r = __ldg(A.arow + a);
            const int32_t rbase = __ldg(A.rp + r);
            const int32_t L = __ldg(A.rp + r + 1) - rbase;
            if (L > kCap) {
                const int32_t s0 = max(pa, __ldg(A.aseg + a));
                const int32_t s1 = min(pb + 1, __ldg(A.aseg + a + 1));
                long_row(A, sm, rbase, L, s0, s1, iA, iB, tri);
                ++a;
                continue;
            }
            if (warp == 0) form_stage(A, sm, a, ab);
            __syncthreads();
            const int32_t nr = sm.ctl[3];
            const int32_t slen = sm.u.st.loc[nr];
            const int tsize = table_size_for(slen);
            const uint32_t mask = uint32_t(tsize / 4 - 1);
            clear_table(sm, tsize, slen, tid);
            __syncthreads();
            for (int k = tid; k < slen; k += kThreads) {
                const int32_t lr = last_le(sm.u.st.loc, 0, nr - 1, k);
                const int32_t g = sm.u.st.gbase[lr] + (k - sm.u.st.loc[lr]);
                table_insert(sm.keys, sm.slots, mask, lr, __ldg(A.col + g), k);
            }
            __syncthreads();
            const int32_t sLo = max(pa, sm.u.st.segb[0]);
            const int32_t sHi = min(pb + 1, sm.u.st.segb[nr]);
            for (;;) {
                int32_t pos = 0;
                if (lane == 0) pos = sLo + atomicAdd(&sm.ctl[1], 1);
                pos = __shfl_sync(0xffffffffu, pos, 0);
                if (pos >= sHi) break;
                const long long base = __ldg(A.wp + pos);
                const int32_t ka = int32_t(max(iA, base) - base);
                const int32_t kb = int32_t(min(iB, __ldg(A.wp + pos + 1)) - base);
                if (ka >= kb) continue;
                const int32_t lr = last_le(sm.u.st.segb, 0, nr - 1, pos);
                const int32_t p0 = __ldg(A.pst + pos);
                int32_t own = probe_range(A, sm, mask, lr, sm.u.st.loc[lr], sm.u.st.loc[lr + 1],
                                          p0 + ka, p0 + kb, lane);
                own = __reduce_add_sync(0xffffffffu, own);
                if (lane == 0 && own) {
                    atomicAdd(A.S + __ldg(A.seg + pos), own);
                    tri += own;
                }
            }
            __syncthreads();
            for (int k = tid; k < slen; k += kThreads) {
                const int32_t v = sm.cnt[k];
                if (v) {
                    const int32_t lr = last_le(sm.u.st.loc, 0, nr - 1, k);
                    atomicAdd(A.S + sm.u.st.gbase[lr] + (k - sm.u.st.loc[lr]), v);
                }
            }
            __syncthreads();
            a += nr;
        }
    }
    tri = warp_sum_ll((long long)tri);
    if (lane == 0 && tri) atomicAdd(A.tri, tri);
}

int g_support_blocks = 0;

cudaError_t configure_once() {
    if (g_support_blocks > 0) return cudaSuccess;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(support_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(sizeof(SupportSmem)));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, support_kernel, kThreads,
                                                          sizeof(SupportSmem));
    if (e != cudaSuccess) return e;
    g_support_blocks = sms * (occ > 0 ? occ : 1);
    return cudaSuccess;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

struct Carve {
    int32_t *ekey, *epst, *eitems, *seg, *pst, *sitems;
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

}  // namespace

size_t balanced_scratch_bytes(int32_t n, int64_t m) {
    Carve c;
    return carve(nullptr, n, m, &c);
}

cudaError_t balanced_scratch_alloc(BalancedScratch *bs, int32_t n, int64_t m) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, balanced_scratch_bytes(n, m));
    if (e != cudaSuccess) return e;
    bs->base = p;
    bs->cap_m = m;
    bs->cap_n = n;
    bs->cap_tasks = 0;
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
    Carve c;
    carve(bs->base, bs->cap_n, bs->cap_m, &c);
    const int32_t n = g.n, m = g.m;
    e = cudaMemsetAsync(c.rcount, 0, size_t(n + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.sched, 0, kSchedWords * 4, s);
    if (e != cudaSuccess) return e;
    const int eblocks = int((int64_t(m) + kEdgeThreads * kEdgesPerThread - 1) /
                            (kEdgeThreads * kEdgesPerThread));
    classify_kernel<<<eblocks, kEdgeThreads, 0, s>>>(g.rp, g.col, n, m, c.ekey, c.epst, c.eitems,
                                                     c.rcount, &cnt->merge_work);
    // row scan: segment starts and active-row ranks (row n has count 0, so the
    // entries at n are the totals)
    const int64_t rows = int64_t(n) + 1;
    const int32_t rtiles = int32_t((rows + kScanTile - 1) / kScanTile);
    RowCountLoad rl{c.rcount};
    RowCountStore rs{c.rstart, c.arank};
    scan_reduce_kernel<Pair, RowCountLoad><<<rtiles, kScanThreads, 0, s>>>(rl, rows, c.rtile_sum);
    scan_totals_kernel<Pair><<<1, 1024, 0, s>>>(c.rtile_sum, rtiles, c.rtile_off, c.rtot);
    scan_apply_kernel<Pair, RowCountLoad, RowCountStore>
        <<<rtiles, kScanThreads, 0, s>>>(rl, rs, rows, c.rtile_off);
    active_rows_kernel<<<int((rows + 255) / 256), 256, 0, s>>>(c.rcount, c.rstart, c.arank,
                                                               c.rtot, n, c.arow, c.aseg);
    scatter_kernel<<<(m + 255) / 256, 256, 0, s>>>(c.ekey, c.epst, c.eitems, m, c.rstart,
                                                   c.rcount, c.seg, c.pst, c.sitems);
    // item scan over the segments (at most m of them; entries past nseg are 0)
    const int32_t itiles = int32_t((int64_t(m) + kScanTile - 1) / kScanTile);
    ItemLoad il{c.sitems, c.rtot};
    ItemStore is{c.wp};
    scan_reduce_kernel<long long, ItemLoad><<<itiles, kScanThreads, 0, s>>>(il, m, c.itile_sum);
    scan_totals_kernel<long long><<<1, 1024, 0, s>>>(c.itile_sum, itiles, c.itile_off, c.itot);
    scan_apply_kernel<long long, ItemLoad, ItemStore>
        <<<itiles, kScanThreads, 0, s>>>(il, is, m, c.itile_off);
    plan_kernel<<<1, 1, 0, s>>>(c.itot, c.rtot, c.wp, c.plan, c.sched, g_support_blocks);
    partition_kernel<<<64, 256, 0, s>>>(c.wp, c.aseg, c.plan, c.sched, c.bound);
    *launches += 12;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) {
        e = cudaEventRecord(ev[1], s);
        if (e != cudaSuccess) return e;
    }
    SupportArgs A{g.rp, g.col, c.seg, c.pst, c.wp, c.arow, c.aseg, c.plan, c.bound, c.sched, S,
                  &cnt->triangles};
    support_kernel<<<g_support_blocks, kThreads, sizeof(SupportSmem), s>>>(A);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace kt
