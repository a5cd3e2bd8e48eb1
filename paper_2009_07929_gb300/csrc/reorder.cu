// Degree-ordered relabel of a loaded graph ("graph rebalancing via sorting",
// which the paper names as future work beside its fine-grained tasks).
//
// The K-truss does not depend on how the vertices are numbered, but the work
// of Alg. 3 does: the task of edge (i, kappa) intersects the part of row i
// after kappa with row kappa, so a hub with a small id owns a long upper row
// whose tails every one of its tasks walks.  Numbering the vertices by
// ascending degree (ties by old id) leaves every upper row holding only the
// neighbours of higher degree, so rows are short and tasks balanced (R-MAT
// scale 23 with planted cliques: longest upper row 1329 instead of ~2.4e5,
// 1.73e10 probes instead of 4.75e10).
//
// On the device, once per load:
//   1. deg[v] = number of edges on v;
//   2. vertices sorted stably by degree (radix sort of (deg, v)); rank r of v
//      in that order is its new id (ties keep the old order); in a batch the
//      sort key is (graph, degree), so that every graph keeps its vertex range;
//   3. every edge (u, v) at input slot e becomes (row, col) = (min, max) of
//      its new ids, counted into its row; row pointers are the exclusive scan
//      of the counts;
//   4. every edge is placed in its row through a per-row atomic cursor
//      (carrying e), then every row is sorted by column in on-chip memory:
//      rows of up to 32 by a bitonic network across the lanes of a warp, rows
//      of up to kRowCap by a bitonic sort in the warp's shared memory, and the
//      few longer rows, gathered into one list, by the radix sort below.  The
//      columns of a row are distinct, so the result does not depend on the
//      order in which the cursor placed them.  The carried slots map every
//      slot of the relabelled CSR back to its input edge, so outputs land in
//      input order.
//
// Radix sort (the vertex order, and the rows longer than kRowCap): least
// significant digit first, 8-bit digits, one pass = a per-tile digit
// histogram, an exclusive scan of the digit-major counts, and a stable
// scatter: a tile of 4096 elements is split over 8 warps in order, each warp
// walks its 512 elements 32 at a time and ranks equal digits with
// __match_any_sync, after the counts of the warps before it were added.
#include <cstdint>

#include "ktruss_internal.cuh"

namespace kt {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // elements per tile
constexpr int kWarpSpanSort = kSortTile / kSortWarps;     // 512 per warp
constexpr int kBins = 256;

constexpr int kScanT = 256;
constexpr int kScanPer = 16;
constexpr int kScanTileN = kScanT * kScanPer;

__device__ __forceinline__ uint32_t digit_of(uint32_t k, int shift) { return (k >> shift) & 0xFFu; }
__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) {
    return uint32_t(k >> shift) & 0xFFu;
}

// counts[d * tiles + t] = elements of tile t whose digit at `shift` is d.
template <typename K>
__global__ void __launch_bounds__(kSortThreads)
digit_hist_kernel(const K *__restrict__ keys, int64_t count, int shift, int32_t tiles,
                  int32_t *__restrict__ counts) {
    __shared__ int32_t h[kBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kSortTile;
    for (int j = 0; j < kSortPerThread; ++j) {
        const int64_t i = base + int64_t(j) * kSortThreads + threadIdx.x;
        if (i < count) atomicAdd(&h[digit_of(keys[i], shift)], 1);
    }
    __syncthreads();
    counts[int64_t(threadIdx.x) * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile to offsets[d * tiles + tile] + rank.
template <typename K>
__global__ void __launch_bounds__(kSortThreads)
digit_scatter_kernel(const K *__restrict__ keys, const int32_t *__restrict__ vals, int64_t count,
                     int shift, int32_t tiles, const int32_t *__restrict__ offsets,
                     K *__restrict__ keys_out, int32_t *__restrict__ vals_out) {
    __shared__ int32_t wh[kSortWarps][kBins];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kSortWarps * kBins; k += kSortThreads) (&wh[0][0])[k] = 0;
    __syncthreads();
    const int64_t wbase = int64_t(blockIdx.x) * kSortTile + int64_t(w) * kWarpSpanSort;
    const uint32_t lt = (1u << lane) - 1u;
    // per-warp digit counts, in element order
    for (int g = 0; g < kWarpSpanSort / 32; ++g) {
        const int64_t i = wbase + g * 32 + lane;
        const bool ok = i < count;
        const uint32_t d = ok ? digit_of(keys[i], shift) : kBins + lane;  // out of range: alone
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & lt) == 0) wh[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // start of each warp's share of each digit: the tile's offset plus the
    // counts of the warps before it
    {
        const int d = threadIdx.x;
        int32_t run = offsets[int64_t(d) * tiles + blockIdx.x];
        for (int k = 0; k < kSortWarps; ++k) {
            const int32_t c = wh[k][d];
            wh[k][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int g = 0; g < kWarpSpanSort / 32; ++g) {
        const int64_t i = wbase + g * 32 + lane;
        const bool ok = i < count;
        K key{};
        int32_t v = 0;
        if (ok) {
            key = keys[i];
            v = vals[i];
        }
        const uint32_t d = ok ? digit_of(key, shift) : kBins + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (ok) {
            const int32_t pos = wh[w][d] + __popc(peers & lt);
            keys_out[pos] = key;
            vals_out[pos] = v;
        }
        __syncwarp();
        if (ok && (peers & lt) == 0) wh[w][d] += __popc(peers);
        __syncwarp();
    }
}

// ---- exclusive int32 scan (three kernels; blocks loop over tiles)
__global__ void __launch_bounds__(kScanT)
scan32_reduce_kernel(const int32_t *__restrict__ in, int64_t count, int32_t *__restrict__ sums) {
    __shared__ int32_t part[kScanT / 32];
    const int64_t i0 = int64_t(blockIdx.x) * kScanTileN + threadIdx.x;
    int32_t s = 0;
    for (int j = 0; j < kScanPer; ++j) {
        const int64_t i = i0 + int64_t(j) * kScanT;
        if (i < count) s += in[i];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int k = 0; k < kScanT / 32; ++k) t += part[k];
        sums[blockIdx.x] = t;
    }
}

// offs[t] = sum of sums[0..t), one block (tiles is small: count / 4096).
__global__ void __launch_bounds__(1024)
scan32_totals_kernel(const int32_t *__restrict__ sums, int32_t tiles, int32_t *__restrict__ offs) {
    __shared__ int32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t per = (tiles + 1023) / 1024;
    const int32_t b = tid * per, e = min(tiles, b + per);
    int32_t local = 0;
    for (int32_t k = b; k < e; ++k) local += sums[k];
    int32_t incl = local;
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t v = ws[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        ws[lane] = v;
    }
    __syncthreads();
    int32_t run = (w > 0 ? ws[w - 1] : 0) + incl - local;
    for (int32_t k = b; k < e; ++k) {
        offs[k] = run;
        run += sums[k];
    }
}

__global__ void __launch_bounds__(kScanT)
scan32_apply_kernel(const int32_t *__restrict__ in, int64_t count, const int32_t *__restrict__ offs,
                    int32_t *__restrict__ out) {
    __shared__ int32_t part[kScanT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i0 = int64_t(blockIdx.x) * kScanTileN + int64_t(threadIdx.x) * kScanPer;
    int32_t v[kScanPer];
    int32_t s = 0;
    for (int j = 0; j < kScanPer; ++j) {
        const int64_t i = i0 + j;
        v[j] = i < count ? in[i] : 0;
        s += v[j];
    }
    int32_t incl = s;
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    int32_t run = offs[blockIdx.x];
    for (int k = 0; k < w; ++k) run += part[k];
    run += incl - s;
    for (int j = 0; j < kScanPer; ++j) {
        const int64_t i = i0 + j;
        if (i < count) out[i] = run;
        run += v[j];
    }
}

// ---- relabel kernels
__global__ void degree_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                              int32_t n, int64_t m, uint32_t *__restrict__ deg) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v < n; v += stride) atomicAdd(deg + v, uint32_t(rp[v + 1] - rp[v]));
    for (int64_t e = t0; e < m; e += stride) atomicAdd(deg + col[e], 1u);
}

// Batches: key[v] = (graph of v) << 32 | degree of v, so that sorting keeps
// every graph's vertices in its own contiguous range.
__global__ void graph_key_kernel(const int32_t *__restrict__ gid, const uint32_t *__restrict__ deg,
                                 int32_t n, uint64_t *__restrict__ key) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride)
        key[v] = (uint64_t(uint32_t(gid[v])) << 32) | deg[v];
}

__global__ void iota_kernel(int32_t *__restrict__ a, int64_t count) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
        a[i] = int32_t(i);
}

// newid[order[r]] = r; also the largest degree (for the caller's bit count is
// taken before the sort).
__global__ void rank_kernel(const int32_t *__restrict__ order, int32_t n,
                            int32_t *__restrict__ newid) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride)
        newid[order[r]] = int32_t(r);
}

__global__ void max_kernel(const uint32_t *__restrict__ a, int64_t count, uint32_t *__restrict__ mx) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    uint32_t v = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
        v = max(v, a[i]);
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicMax(mx, v);
}

// Largest i in [lo, hi] with a[i] <= x (a non-decreasing, a[lo] <= x).
__device__ __forceinline__ int32_t last_le32(const int32_t *__restrict__ a, int32_t lo,
                                             int32_t hi, int64_t x) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (a[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Largest r in [0, n - 1] with rp[r] <= v (rp[0] = 0 <= v), found by the
// whole warp: each pass probes 32 evenly spaced rows and keeps the gap between
// the last probe at or below v and the first above it.  All lanes pass the
// same v.
__device__ __forceinline__ int32_t warp_row_of(const int32_t *__restrict__ rp, int32_t n,
                                               int64_t v) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = int64_t(n) - 1;
    while (hi - lo >= 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t p = min(lo + int64_t(lane + 1) * step, hi);
        const int c = __popc(__ballot_sync(0xffffffffu, rp[p] <= v));
        const int64_t nlo = c > 0 ? min(lo + int64_t(c) * step, hi) : lo;
        const int64_t nhi = c < 32 ? min(lo + int64_t(c + 1) * step, hi) - 1 : hi;
        lo = nlo;
        hi = nhi;
    }
    const int64_t p = lo + lane;
    const bool le = p <= hi && rp[p] <= v;
    return int32_t(lo + __popc(__ballot_sync(0xffffffffu, le)) - 1);
}

// key[e] = (row << 32) | col of edge e in the new ids (row = the smaller end)
// and rowcnt[row] += 1.  A warp takes windows of kKeyWin consecutive slots,
// lane l the slots l, l + 32, ... (coalesced reads and writes); the window's
// first row comes from a warp search, a lane's later rows from a forward
// galloping search.
constexpr int kKeyWin = 256;
__global__ void __launch_bounds__(256)
edge_key_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                int64_t m, const int32_t *__restrict__ newid, uint64_t *__restrict__ key,
                int32_t *__restrict__ rowcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t base = gw * kKeyWin; base < m; base += nw * kKeyWin) {
        int32_t row = warp_row_of(rp, n, base);
        int32_t rend = rp[row + 1];
        int32_t a = newid[row];
        for (int j = 0; j < kKeyWin / 32; ++j) {
            const int64_t e = base + lane + 32 * j;
            if (e >= m) break;
            if (rend <= e) {
                // rows row+1 .. are at or below e: gallop to a bound above it
                int64_t lo = row + 1, step = 1, hi = lo + 1;
                while (hi <= n - 1 && rp[hi] <= e) {
                    lo = hi;
                    step <<= 1;
                    hi = lo + step;
                }
                row = last_le32(rp, int32_t(lo), int32_t(min(hi - 1, int64_t(n) - 1)), e);
                rend = rp[row + 1];
                a = newid[row];
            }
            const int32_t b = newid[col[e]];
            const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
            key[e] = (uint64_t(uint32_t(lo)) << 32) | uint32_t(hi);
            atomicAdd(rowcnt + lo, 1);
        }
    }
}

// Places edge e in its row: the next free slot of the row (cursor[row],
// starting at the row's first slot), with its column and input slot.
__global__ void edge_place_kernel(const uint64_t *__restrict__ key, int64_t m,
                                  int32_t *__restrict__ cursor, int32_t *__restrict__ col_out,
                                  int32_t *__restrict__ eid_out) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint64_t k = key[e];
        const int32_t pos = atomicAdd(cursor + int32_t(k >> 32), 1);
        col_out[pos] = int32_t(uint32_t(k));
        eid_out[pos] = int32_t(e);
    }
}

// Sorts every row of (col, eid) of length 2 .. kRowCap by column, in place.
// A warp reads the lengths of 32 consecutive rows and sorts them one after
// the other: a row of up to 32 in registers (one element per lane, a bitonic
// network over lane shuffles), a longer one in the warp's shared array (a
// bitonic sort over the next power of two, padded with the largest key).
// Elements are packed (column << 32 | input slot); columns of a row are
// distinct, so the packed order is the column order.
constexpr int kRowCap = 1024;
constexpr int kRowWarps = 4;
__global__ void __launch_bounds__(32 * kRowWarps)
row_sort_kernel(const int32_t *__restrict__ rp, int32_t n, int32_t *__restrict__ col,
                int32_t *__restrict__ eid) {
    __shared__ uint64_t sk[kRowWarps][kRowCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    uint64_t *a = sk[w];
    for (int64_t r0 = gw * 32; r0 < n; r0 += nw * 32) {
        const int64_t r = r0 + lane;
        int32_t b = 0, L = 0;
        if (r < n) {
            b = rp[r];
            L = rp[r + 1] - b;
        }
        unsigned todo = __ballot_sync(0xffffffffu, L >= 2 && L <= kRowCap);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int32_t rb = __shfl_sync(0xffffffffu, b, src);
            const int32_t rl = __shfl_sync(0xffffffffu, L, src);
            if (rl <= 32) {
                uint64_t v = ~0ull;
                if (lane < rl) v = (uint64_t(uint32_t(col[rb + lane])) << 32) | uint32_t(eid[rb + lane]);
#pragma unroll
                for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
                        const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                        v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
                    }
                }
                if (lane < rl) {
                    col[rb + lane] = int32_t(uint32_t(v >> 32));
                    eid[rb + lane] = int32_t(uint32_t(v));
                }
            } else {
                int P = 64;
                while (P < rl) P <<= 1;
                for (int i = lane; i < P; i += 32)
                    a[i] = i < rl ? (uint64_t(uint32_t(col[rb + i])) << 32) | uint32_t(eid[rb + i])
                                  : ~0ull;
                __syncwarp();
                for (int k = 2; k <= P; k <<= 1) {
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        for (int i = lane; i < (P >> 1); i += 32) {
                            const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                            const int hi = lo + j;
                            const uint64_t x = a[lo], y = a[hi];
                            if ((x > y) == ((lo & k) == 0)) {
                                a[lo] = y;
                                a[hi] = x;
                            }
                        }
                        __syncwarp();
                    }
                }
                for (int i = lane; i < rl; i += 32) {
                    const uint64_t v = a[i];
                    col[rb + i] = int32_t(uint32_t(v >> 32));
                    eid[rb + i] = int32_t(uint32_t(v));
                }
                __syncwarp();
            }
        }
    }
}

// lcount[r] = length of row r if it is longer than kRowCap, else 0 (r < n);
// lcount[n] = 0.
__global__ void long_count_kernel(const int32_t *__restrict__ rp, int32_t n,
                                  int32_t *__restrict__ lcount) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r <= n; r += stride) {
        const int32_t L = r < n ? rp[r + 1] - rp[r] : 0;
        lcount[r] = L > kRowCap ? L : 0;
    }
}

// The rows longer than kRowCap, in row order, as (row << 32 | col, input
// slot) at their offsets loff[row] of one list.
__global__ void long_gather_kernel(const int32_t *__restrict__ rp, int32_t n,
                                   const int32_t *__restrict__ loff,
                                   const int32_t *__restrict__ col,
                                   const int32_t *__restrict__ eid, uint64_t *__restrict__ key,
                                   int32_t *__restrict__ val) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int32_t b = rp[r], L = rp[r + 1] - b;
        if (L <= kRowCap) continue;
        const int32_t o = loff[r];
        for (int32_t i = 0; i < L; ++i) {
            key[o + i] = (uint64_t(uint32_t(r)) << 32) | uint32_t(col[b + i]);
            val[o + i] = eid[b + i];
        }
    }
}

// Writes the sorted list back: element i of row r goes to the row's slot
// i - loff[r] (rows keep their extents in the list, sorted by row first).
__global__ void long_scatter_kernel(const uint64_t *__restrict__ key,
                                    const int32_t *__restrict__ val, int64_t count,
                                    const int32_t *__restrict__ rp,
                                    const int32_t *__restrict__ loff, int32_t *__restrict__ col,
                                    int32_t *__restrict__ eid) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint64_t k = key[i];
        const int32_t r = int32_t(k >> 32);
        const int64_t dst = rp[r] + (i - loff[r]);
        col[dst] = int32_t(uint32_t(k));
        eid[dst] = val[i];
    }
}

int grid_for(int64_t work, int threads) {
    const int64_t b = (work + threads - 1) / threads;
    return int(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

// Carves the sort's scratch: ping-pong keys and values and the digit counts.
struct SortScratch {
    void *keys[2];
    int32_t *vals[2];
    int32_t *counts, *offsets, *tsum, *toff;
    uint32_t *mx;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// scan_min: the largest plain int32 scan the tile arrays must also serve.
size_t sort_layout(void *base, int64_t count, size_t key_bytes, int64_t scan_min,
                   SortScratch *s) {
    char *p = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *q = p ? p + off : nullptr;
        off += align256(bytes);
        return q;
    };
    const int64_t tiles = (count + kSortTile - 1) / kSortTile;
    const int64_t cells = tiles * kBins;
    const int64_t scanned = cells > scan_min ? cells : scan_min;
    const int64_t ctiles = (scanned + kScanTileN - 1) / kScanTileN;
    s->keys[0] = take(size_t(count) * key_bytes);
    s->keys[1] = take(size_t(count) * key_bytes);
    s->vals[0] = reinterpret_cast<int32_t *>(take(size_t(count) * 4));
    s->vals[1] = reinterpret_cast<int32_t *>(take(size_t(count) * 4));
    s->counts = reinterpret_cast<int32_t *>(take(size_t(cells) * 4 + 4));
    s->offsets = reinterpret_cast<int32_t *>(take(size_t(cells) * 4 + 4));
    s->tsum = reinterpret_cast<int32_t *>(take(size_t(ctiles) * 4 + 4));
    s->toff = reinterpret_cast<int32_t *>(take(size_t(ctiles) * 4 + 4));
    s->mx = reinterpret_cast<uint32_t *>(take(16));
    return off;
}

cudaError_t scan32(const int32_t *in, int64_t count, int32_t *out, int32_t *tsum, int32_t *toff,
                   cudaStream_t st) {
    const int32_t tiles = int32_t((count + kScanTileN - 1) / kScanTileN);
    if (tiles == 0) return cudaSuccess;
    scan32_reduce_kernel<<<tiles, kScanT, 0, st>>>(in, count, tsum);
    scan32_totals_kernel<<<1, 1024, 0, st>>>(tsum, tiles, toff);
    scan32_apply_kernel<<<tiles, kScanT, 0, st>>>(in, count, toff, out);
    return cudaGetLastError();
}

// Stable LSD radix sort of (keys, vals) by the digits at the given shifts,
// in place in buffer `cur` of the ping-pong pair; returns the buffer that
// holds the result.
template <typename K>
cudaError_t radix_sort(SortScratch &s, int64_t count, const int *shifts, int npass, int *cur,
                       cudaStream_t st) {
    const int32_t tiles = int32_t((count + kSortTile - 1) / kSortTile);
    const int64_t cells = int64_t(tiles) * kBins;
    for (int p = 0; p < npass; ++p) {
        const int a = *cur, b = a ^ 1;
        const K *kin = static_cast<const K *>(s.keys[a]);
        K *kout = static_cast<K *>(s.keys[b]);
        digit_hist_kernel<K><<<tiles, kSortThreads, 0, st>>>(kin, count, shifts[p], tiles,
                                                             s.counts);
        cudaError_t e = scan32(s.counts, cells, s.offsets, s.tsum, s.toff, st);
        if (e != cudaSuccess) return e;
        digit_scatter_kernel<K><<<tiles, kSortThreads, 0, st>>>(
            kin, s.vals[a], count, shifts[p], tiles, s.offsets, kout, s.vals[b]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *cur = b;
    }
    return cudaSuccess;
}

}  // namespace

size_t reorder_scratch_bytes(int32_t n, int64_t m) {
    SortScratch s;
    const size_t a = sort_layout(nullptr, m, 8, int64_t(n) + 1, &s);
    const size_t b = sort_layout(nullptr, n, 8, int64_t(n) + 1, &s);
    // degrees (n) beside the vertex sort, then new ids and row counts
    return (a > b + align256(size_t(n) * 4) ? a : b + align256(size_t(n) * 4)) +
           align256((size_t(n) + 1) * 4) * 2;
}

cudaError_t launch_reorder(const int32_t *rp, const int32_t *col, int32_t n, int64_t m,
                           void *scratch, int32_t *rp_out, int32_t *col_out, int32_t *eid_out,
                           cudaStream_t st, const int32_t *gid, int32_t num_graphs) {
    if (n == 0) return cudaMemsetAsync(rp_out, 0, 4, st);
    SortScratch es, vs;
    const size_t a_bytes = sort_layout(nullptr, m, 8, int64_t(n) + 1, &es);
    const size_t b_bytes = sort_layout(nullptr, n, 8, int64_t(n) + 1, &vs);
    const size_t vb_bytes = b_bytes + align256(size_t(n) * 4);
    const size_t sort_bytes = a_bytes > vb_bytes ? a_bytes : vb_bytes;
    char *base = static_cast<char *>(scratch);
    // new ids and row counts after the sorts' memory; the degrees after the
    // vertex sort's
    int32_t *newid = reinterpret_cast<int32_t *>(base + sort_bytes);
    int32_t *rowcnt = reinterpret_cast<int32_t *>(base + sort_bytes + align256((size_t(n) + 1) * 4));
    uint32_t *deg = reinterpret_cast<uint32_t *>(base + b_bytes);
    // 1-2: degrees, vertices sorted by degree (batches: by graph, then
    // degree), stably, so that ties keep their old order
    sort_layout(base, n, gid ? 8 : 4, int64_t(n) + 1, &vs);
    cudaError_t e = cudaMemsetAsync(deg, 0, size_t(n) * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(vs.mx, 0, 4, st);
    if (e != cudaSuccess) return e;
    degree_kernel<<<grid_for(m > n ? m : n, 256), 256, 0, st>>>(rp, col, n, m, deg);
    iota_kernel<<<grid_for(n, 256), 256, 0, st>>>(vs.vals[0], n);
    max_kernel<<<grid_for(n, 256), 256, 0, st>>>(deg, n, vs.mx);
    uint32_t maxdeg = 0;
    e = cudaMemcpyAsync(&maxdeg, vs.mx, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    int shifts[16];
    int np = 0;
    for (int sh = 0; sh < bits_for(maxdeg); sh += 8) shifts[np++] = sh;
    int cur = 0;
    if (gid) {
        graph_key_kernel<<<grid_for(n, 256), 256, 0, st>>>(gid, deg, n,
                                                           static_cast<uint64_t *>(vs.keys[0]));
        const int gb = bits_for(uint64_t(num_graphs > 0 ? num_graphs - 1 : 0));
        for (int sh = 0; sh < gb; sh += 8) shifts[np++] = 32 + sh;
        e = radix_sort<uint64_t>(vs, n, shifts, np, &cur, st);
    } else {
        e = cudaMemcpyAsync(vs.keys[0], deg, size_t(n) * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = radix_sort<uint32_t>(vs, n, shifts, np, &cur, st);
    }
    if (e != cudaSuccess) return e;
    rank_kernel<<<grid_for(n, 256), 256, 0, st>>>(vs.vals[cur], n, newid);
    // 3: every edge keyed by (new row, new col) and counted into its new row
    e = cudaGetLastError();
    if (e != cudaSuccess || m == 0) {
        if (e == cudaSuccess) e = cudaMemsetAsync(rp_out, 0, (size_t(n) + 1) * 4, st);
        return e;
    }
    sort_layout(base, m, 8, int64_t(n) + 1, &es);
    uint64_t *ekey = static_cast<uint64_t *>(es.keys[0]);
    e = cudaMemsetAsync(rowcnt, 0, (size_t(n) + 1) * 4, st);
    if (e != cudaSuccess) return e;
    edge_key_kernel<<<grid_for((m + kKeyWin - 1) / kKeyWin * 32, 256), 256, 0, st>>>(
        rp, col, n, m, newid, ekey, rowcnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // rp_out = exclusive scan of the row counts (n + 1 entries, the last is 0)
    e = scan32(rowcnt, int64_t(n) + 1, rp_out, es.tsum, es.toff, st);
    if (e != cudaSuccess) return e;
    // 4: place every edge in its row (rowcnt turns into the per-row cursor),
    // then sort the rows
    e = cudaMemcpyAsync(rowcnt, rp_out, size_t(n) * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    edge_place_kernel<<<grid_for(m, 256), 256, 0, st>>>(ekey, m, rowcnt, col_out, eid_out);
    row_sort_kernel<<<grid_for((int64_t(n) + 31) / 32 * 32, 32 * kRowWarps), 32 * kRowWarps, 0,
                      st>>>(rp_out, n, col_out, eid_out);
    // rows longer than kRowCap: one list (offsets loff in the cursor's memory,
    // counts in the new ids' memory, both free now), sorted by (row, col)
    int32_t *lcount = newid, *loff = rowcnt;
    long_count_kernel<<<grid_for(int64_t(n) + 1, 256), 256, 0, st>>>(rp_out, n, lcount);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan32(lcount, int64_t(n) + 1, loff, es.tsum, es.toff, st);
    int32_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, loff + n, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || total == 0) return e;
    long_gather_kernel<<<grid_for(n, 256), 256, 0, st>>>(rp_out, n, loff, col_out, eid_out,
                                                        static_cast<uint64_t *>(es.keys[0]),
                                                        es.vals[0]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int vb = bits_for(uint64_t(n - 1));
    np = 0;
    for (int sh = 0; sh < vb; sh += 8) shifts[np++] = sh;        // column
    for (int sh = 0; sh < vb; sh += 8) shifts[np++] = 32 + sh;   // row
    cur = 0;
    e = radix_sort<uint64_t>(es, total, shifts, np, &cur, st);
    if (e != cudaSuccess) return e;
    long_scatter_kernel<<<grid_for(total, 256), 256, 0, st>>>(
        static_cast<const uint64_t *>(es.keys[cur]), es.vals[cur], total, rp_out, loff, col_out,
        eid_out);
    return cudaGetLastError();
}

}  // namespace kt
