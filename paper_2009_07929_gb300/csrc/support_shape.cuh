// The support kernel and its block-level building blocks, written for one
// CTA shape.  support_balanced.cu includes this file once per shape, inside a
// namespace that defines kThreads (threads per CTA), kCap (staged slots per
// stage or piece) and kMinCtas (CTAs resident per SM the kernel is compiled
// for); everything here depends on those three.  Not a standalone header.

constexpr int kTable = 4 * kCap;        // hash entries (load factor <= 1/4)
constexpr int kWarps = kThreads / 32;
constexpr int kBatch = kThreads;        // segments per batch (one per thread)
constexpr int kLong = 6 * kBatch / 4;   // segments per batch of a long row

// ------------------------------------------------------------ support kernel
// Shared memory of one support CTA.
struct SupportSmem {
    uint32_t fpw[kTable / 4];         // fingerprint word of each bucket
    uint16_t slots[kTable];           // local staged slot of each entry
    int32_t vals[kCap];               // staged columns by local slot
    int32_t cnt[kCap];                // credits to staged slots
    int32_t gbase[kStageRows];        // stage: global slot of each row's first element
    int32_t loc[kStageRows + 1];      // stage: local slot offsets of the rows
    int32_t segb[kStageRows + 1];     // stage: first segment position of each row
    int32_t tbase[kStageRows + 1];    // stage: first bucket of each row's region
    int32_t tlb[kStageRows];          // stage: log2 bucket count of each row's region
    union {
        struct {                      // stages of short rows
            int32_t owner[kBatch];    // batch: owner edge slot of segment j
            int32_t hit[kBatch];      // batch: hits credited to segment j's owner
            int32_t rstart[kBatch + 1];  // runs: batch-local item offset of run r
            int32_t rdel[kBatch];     // runs: probe position of item i of run r is rdel[r] + i
            int32_t rreg[kBatch];     // runs: region probed (region_word)
            int32_t rseg[kBatch];     // runs: segment of run r
        } b;
        struct {                      // long rows: segment j of the current batch
            int32_t cur[kLong];       // next probe position
            int32_t end[kLong];       // end of its probes in the chunk
            int32_t nxt[kLong];       // column at cur (kIntMax when exhausted)
            int32_t hit[kLong];       // hits credited to its owner
        } l;
    };
    unsigned long long wtmp[64];
    int32_t ctl[64];
};
static_assert(sizeof(SupportSmem) <= 227 * 1024, "support CTA exceeds shared memory");

struct SupportArgs {
    const int32_t *rp, *col;
    const int4 *srec;  // segment records: owner slot, probe start, items, active-row rank
    const long long *wp;
    const int32_t *arow, *aseg;
    const ChunkPlan *plan;
    const int2 *bound;
    int32_t *sched;
    int32_t *S;
    unsigned long long *tri;
    int32_t *err;
};

// Exclusive block-wide prefix of v (kThreads threads); *total = sum.  wtmp is
// read after the second barrier, so the caller synchronises before reusing it.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long *wtmp,
                                                              unsigned long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) wtmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < kWarps ? wtmp[lane] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += u;
        }
        if (lane < kWarps) wtmp[32 + lane] = x;
    }
    __syncthreads();
    const unsigned long long before = warp > 0 ? wtmp[32 + warp - 1] : 0ull;
    total = wtmp[32 + kWarps - 1];
    return before + incl - v;
}

// Region word of a staged row: first bucket in the low 24 bits, the region's
// bucket shift (32 - log2 of its bucket count) above.
__device__ __forceinline__ int32_t region_word(int32_t bbase, int lb) {
    return bbase | ((32 - lb) << 24);
}

// Builds the run list from per-thread (len, pos, reg, seg) proposals: runs of
// positive length in thread order, each with its position offset and the
// region word of the staged row it probes.  Returns (runs, items) through the
// refs.  One scan serves both prefixes: the run flag in the high word, the
// length in the low word (a batch's items stay below 2^31, so no carry
// crosses).
__device__ __forceinline__ void build_runs(SupportSmem &sm, int32_t len, int32_t pos, int32_t reg,
                                           int32_t j, int32_t &nruns, int32_t &items) {
    const int32_t flag = len > 0 ? 1 : 0;
    unsigned long long tot;
    const unsigned long long pre =
        block_excl_scan((unsigned long long)flag << 32 | uint32_t(len > 0 ? len : 0), sm.wtmp, tot);
    const int32_t ridx = int32_t(pre >> 32), roff = int32_t(uint32_t(pre));
    nruns = int32_t(tot >> 32);
    items = int32_t(uint32_t(tot));
    if (flag) {
        sm.b.rstart[ridx] = roff;
        sm.b.rdel[ridx] = pos - roff;
        sm.b.rreg[ridx] = reg;
        sm.b.rseg[ridx] = j;
    }
    if (threadIdx.x == 0) {
        sm.b.rstart[nruns] = items;
        sm.ctl[4] = 0;
    }
    __syncthreads();
}

// Probes of the items [p, pe) of a batch's flat item space (p in run E).  The
// warp walks the range in windows of 32 consecutive items, kUnroll windows
// with their loads in flight at a time.  Each lane tracks the run of its own
// item (runs are consecutive in item space, so a lane only moves forward,
// crossing a run start when its item passes it) and keeps that run's probe
// offset and region in registers, so a window costs the same whether it lies
// inside one run or spans several.  Every hit adds one to the staged slot's
// shared counter, to S at the probe position and to its run owner's shared
// counter (a per-lane count carried across windows cost more registers than
// the shared atomic it saves).
__device__ __forceinline__ void probe_range(const SupportArgs &A, SupportSmem &sm, int32_t nruns,
                                            int32_t items, int32_t E, int32_t p, int32_t pe) {
    const int lane = threadIdx.x & 31;
    int32_t r = E, rnext = sm.b.rstart[E + 1];  // rstart[nruns] == items
    int32_t del = sm.b.rdel[E], reg = sm.b.rreg[E];
    for (; p < pe; p += 32 * kUnroll) {
        int32_t xv[kUnroll], gv[kUnroll], rv[kUnroll], wv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t item = p + 32 * u + lane;
            rv[u] = -1;
            xv[u] = 0;
            gv[u] = 0;
            if (item < pe) {
                if (rnext <= item) {
                    do {
                        ++r;
                        rnext = sm.b.rstart[r + 1];
                    } while (rnext <= item);
                    del = sm.b.rdel[r];
                    reg = sm.b.rreg[r];
                }
                rv[u] = r;
                xv[u] = del + item;
                gv[u] = reg;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) wv[u] = rv[u] >= 0 ? __ldg(A.col + xv[u]) : 0;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (rv[u] < 0) continue;
            const int32_t q = table_find(sm.fpw, sm.slots, sm.vals, gv[u] & 0xffffff, gv[u] >> 24,
                                         wv[u]);
            if (q >= 0) {
                atomicAdd(&sm.cnt[q], 1);
                atomicAdd(A.S + xv[u], 1);
                atomicAdd(&sm.b.hit[sm.b.rseg[rv[u]]], 1);
            }
        }
    }
}

// Probing of all runs of a batch: an even split of the items over the warps
// (kGrain == 0), or grains of kGrain items taken from a shared counter
// (sm.ctl[4], zero on entry) until the batch is exhausted.
__device__ __forceinline__ void probe_runs(const SupportArgs &A, SupportSmem &sm, int32_t nruns,
                                           int32_t items) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (kGrain == 0) {
        const int32_t per = ((items + kWarps - 1) / kWarps + 31) & ~31;
        const int32_t w0 = warp * per;
        const int32_t w1 = min(items, w0 + per);
        if (w0 < w1)
            probe_range(A, sm, nruns, items, last_le(sm.b.rstart, 0, nruns - 1, w0), w0, w1);
    } else {
        for (;;) {
            int32_t g = 0;
            if (lane == 0) g = atomicAdd(&sm.ctl[4], kGrain);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= items) break;
            const int32_t E = last_le(sm.b.rstart, 0, nruns - 1, g);
            probe_range(A, sm, nruns, items, E, g, min(items, g + kGrain));
        }
    }
}

__device__ __forceinline__ void clear_table(SupportSmem &sm, int32_t buckets, int32_t len, int tid) {
    for (int k = tid; k < buckets; k += kThreads) sm.fpw[k] = 0u;
    for (int k = tid; k < len; k += kThreads) sm.cnt[k] = 0;
}

// Adds the owner credits of a batch to S and to the triangle count.
__device__ __forceinline__ void flush_owners(const SupportArgs &A, SupportSmem &sm, int32_t nb,
                                             unsigned long long &tri) {
    const int j = threadIdx.x;
    if (j < nb) {
        const int32_t v = sm.b.hit[j];
        if (v) {
            atomicAdd(A.S + sm.b.owner[j], v);
            tri += v;
        }
    }
}

// Probes one column w of a window against the region (bb, lb) of the table;
// on a hit credits the staged slot (shared counter) and the probe position x
// (global) and returns true.
__device__ __forceinline__ bool probe_one(SupportSmem &sm, int32_t bb, uint32_t bm, int sh,
                                          int32_t w, int32_t *x) {
    const uint32_t fp4 = fingerprint(w) * 0x01010101u;
    uint32_t b = (uint32_t(w) * kHashMul) >> sh;
    for (;;) {
        const int32_t at = bb + int32_t(b);
        const uint32_t word = sm.fpw[at];
        for (uint32_t mm = match_bytes(word, fp4); mm; mm &= mm - 1u) {
            const int32_t sl = sm.slots[4 * at + ((__ffs(mm) - 1) >> 3)];
            if (sm.vals[sl] == w) {
                atomicAdd(&sm.cnt[sl], 1);
                atomicAdd(x, 1);
                return true;
            }
        }
        if ((word >> 24) == 0) return false;
        b = (b + 1) & bm;
    }
}

// Last piece (of kCap slots) of the row at rbase with npieces pieces whose
// first column is <= v (piece 0 if none is).
__device__ __forceinline__ int32_t piece_of(const int32_t *__restrict__ col, int32_t rbase,
                                            int32_t npieces, int32_t v) {
    int32_t lo = 0, hi = npieces - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (__ldg(col + rbase + mid * kCap) <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The segments [s0, s1) of chunk [iA, iB) whose staged row (rbase, L) is
// longer than kCap.  The row is staged piece by piece in column order, each
// piece once for up to kLong segments.  Every segment keeps a cursor (its next
// probe position and the column there); per piece, warps take the segments
// whose next probe lies below the piece's end column and stream their probes
// in windows of 32 until a probe reaches that column (the probes are sorted,
// so the probes of a piece are a prefix of what is left).  Pieces below every
// segment's next probe are skipped.
__device__ void long_row(const SupportArgs &A, SupportSmem &sm, int32_t rbase, int32_t L,
                         int32_t s0, int32_t s1, long long iA, long long iB,
                         unsigned long long &tri) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t npieces = (L + kCap - 1) / kCap;
    for (int32_t sb = s0; sb < s1; sb += kLong) {
        const int32_t nb = min(kLong, s1 - sb);
        int32_t mv = kIntMax;
        for (int32_t j = tid; j < nb; j += kThreads) {
            const int32_t pos = sb + j;
            const long long base = __ldg(A.wp + pos);
            const int32_t ka = int32_t(max(iA, base) - base);
            const int32_t kb = int32_t(min(iB, __ldg(A.wp + pos + 1)) - base);
            const int32_t p0 = __ldg(&A.srec[pos].y);
            sm.l.cur[j] = p0 + ka;
            sm.l.end[j] = p0 + max(ka, kb);
            sm.l.hit[j] = 0;
            const int32_t v = kb > ka ? __ldg(A.col + p0 + ka) : kIntMax;
            sm.l.nxt[j] = v;
            mv = min(mv, v);
        }
        mv = __reduce_min_sync(0xffffffffu, mv);
        if (lane == 0) sm.ctl[16 + warp] = mv;
        __syncthreads();
        if (tid == 0) {
            int32_t v = kIntMax;
            for (int k = 0; k < kWarps; ++k) v = min(v, sm.ctl[16 + k]);
            sm.ctl[2] = v;
        }
        __syncthreads();
        mv = sm.ctl[2];
        int32_t p = mv == kIntMax ? npieces : piece_of(A.col, rbase, npieces, mv);
        while (p < npieces) {
            const int32_t ps = rbase + p * kCap;
            const int32_t plen = min(kCap, L - p * kCap);
            const int32_t vhi = (p + 1 < npieces) ? __ldg(A.col + ps + plen) : kIntMax;
            const int lb = region_lb(plen);
            clear_table(sm, 1 << lb, plen, tid);
            if (tid == 0) {
                sm.ctl[5] = 0;        // next group of segments to take
                sm.ctl[6] = kIntMax;  // smallest next probe after this piece
            }
            __syncthreads();
            for (int q = tid; q < plen; q += kThreads) {
                const int32_t w = __ldg(A.col + ps + q);
                sm.vals[q] = w;
                if (!table_insert(sm.fpw, sm.slots, 0, lb, w, q))
                    give_up(A.sched, A.err, kGiveUpInsert, plen, lb);
            }
            __syncthreads();
            const uint32_t bm = (1u << lb) - 1u;
            const int sh = 32 - lb;
            // warps take one segment at a time, so that long runs spread
            int32_t low = kIntMax;  // smallest next probe this warp saw
            for (;;) {
                int32_t j = 0;
                if (lane == 0) j = atomicAdd(&sm.ctl[5], 1);
                j = __shfl_sync(0xffffffffu, j, 0);
                if (j >= nb) break;
                const int32_t nx = sm.l.nxt[j];
                if (nx >= vhi) {
                    low = min(low, nx);
                    continue;
                }
                int32_t x = sm.l.cur[j];
                const int32_t xe = sm.l.end[j];
                int32_t own = 0, nextv = kIntMax;
                for (;;) {
                    int32_t wv[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int32_t i = x + 32 * u + lane;
                        wv[u] = i < xe ? __ldg(A.col + i) : kIntMax;
                    }
                    int32_t tot = 0;
                    bool done = false;
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const bool valid = wv[u] < vhi;
                        if (valid && probe_one(sm, 0, bm, sh, wv[u], A.S + x + 32 * u + lane))
                            ++own;
                        const int nv = __popc(__ballot_sync(0xffffffffu, valid));
                        if (!done) {
                            tot += nv;
                            if (nv < 32) {
                                nextv = __shfl_sync(0xffffffffu, wv[u], nv & 31);
                                done = true;
                            }
                        }
                    }
                    x += tot;
                    if (done) break;
                }
                own = __reduce_add_sync(0xffffffffu, own);
                if (lane == 0) {
                    sm.l.cur[j] = x;
                    sm.l.nxt[j] = nextv;
                    sm.l.hit[j] += own;
                }
                low = min(low, nextv);
            }
            if (lane == 0 && low < kIntMax) atomicMin(&sm.ctl[6], low);
            __syncthreads();
            for (int q = tid; q < plen; q += kThreads) {
                const int32_t v = sm.cnt[q];
                if (v) atomicAdd(A.S + ps + q, v);
            }
            mv = sm.ctl[6];
            __syncthreads();  // the next piece clears the table and resets ctl[6]
            p = mv == kIntMax ? npieces : piece_of(A.col, rbase, npieces, mv);
        }
        // owner credits of the batch
        for (int32_t j = tid; j < nb; j += kThreads) {
            const int32_t v = sm.l.hit[j];
            if (v) {
                atomicAdd(A.S + __ldg(&A.srec[sb + j].x), v);
                tri += v;
            }
        }
        __syncthreads();  // the next batch rewrites the segment arrays
    }
}

// Forms a stage of consecutive short active rows starting at active row a
// (warp 0): rows a .. a+nr-1 with total length <= kCap, total region size
// <= kTable / 4 buckets and nr <= kStageRows.
__device__ void form_stage(const SupportArgs &A, SupportSmem &sm, int32_t a, int32_t ab) {
    const int lane = threadIdx.x & 31;
    constexpr int32_t kBuckets = kTable / 4;
    int32_t acc = 0, accb = 0, nr = 0;
    for (;;) {
        const int32_t ai = a + nr + lane;
        int32_t len = -1, gb = 0, sgb = 0, lb = 1;
        if (ai <= ab && nr + lane < kStageRows) {
            const int32_t rr = __ldg(A.arow + ai);
            gb = __ldg(A.rp + rr);
            len = __ldg(A.rp + rr + 1) - gb;
            sgb = __ldg(A.aseg + ai);
            if (len > kCap) len = -1;
            else lb = region_lb(len);
        }
        // inclusive prefixes of lengths and region sizes, saturating (an
        // ineligible row counts as too large, so every later lane fails too)
        int32_t incl = len < 0 ? kCap + 1 : len;
        int32_t inclb = len < 0 ? kBuckets + 1 : (1 << lb);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, incl, d);
            const int32_t ub = __shfl_up_sync(0xffffffffu, inclb, d);
            if (lane >= d) {
                incl = min(incl + u, kCap + 1);
                inclb = min(inclb + ub, kBuckets + 1);
            }
        }
        const bool ok = len >= 0 && acc + incl <= kCap && accb + inclb <= kBuckets;
        const uint32_t okm = __ballot_sync(0xffffffffu, ok);
        const int tk = okm == 0xffffffffu ? 32 : __ffs(~okm) - 1;  // ok is a lane prefix
        if (lane < tk) {
            sm.gbase[nr + lane] = gb;
            sm.loc[nr + lane] = acc + incl - len;
            sm.segb[nr + lane] = sgb;
            sm.tbase[nr + lane] = accb + inclb - (1 << lb);
            sm.tlb[nr + lane] = lb;
        }
        if (tk > 0) {
            acc += __shfl_sync(0xffffffffu, incl, tk - 1);
            accb += __shfl_sync(0xffffffffu, inclb, tk - 1);
        }
        nr += tk;
        if (tk < 32) break;
    }
    if (lane == 0) {
        sm.loc[nr] = acc;
        sm.tbase[nr] = accb;
        sm.segb[nr] = __ldg(A.aseg + a + nr);
        sm.ctl[3] = nr;
    }
}

__global__ void __launch_bounds__(kThreads, kMinCtas)
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
            // ------------------------------------- stage of short staged rows
            if (warp == 0) form_stage(A, sm, a, ab);
            __syncthreads();
            const int32_t nr = sm.ctl[3];
            const int32_t slen = sm.loc[nr];
            clear_table(sm, sm.tbase[nr], slen, tid);
            __syncthreads();
            for (int k = tid; k < slen; k += kThreads) {
                const int32_t lr = last_le(sm.loc, 0, nr - 1, k);
                const int32_t g = sm.gbase[lr] + (k - sm.loc[lr]);
                const int32_t w = __ldg(A.col + g);
                sm.vals[k] = w;
                if (!table_insert(sm.fpw, sm.slots, sm.tbase[lr], sm.tlb[lr], w, k))
                    give_up(A.sched, A.err, kGiveUpInsert, lr, sm.tlb[lr]);
            }
            __syncthreads();
            const int32_t sLo = max(pa, sm.segb[0]);
            const int32_t sHi = min(pb + 1, sm.segb[nr]);
            for (int32_t sb = sLo; sb < sHi; sb += kBatch) {
                const int32_t nb = min(kBatch, sHi - sb);
                int32_t len = 0, pos0 = 0, key = 0;
                if (tid < nb) {
                    const int32_t pos = sb + tid;
                    const long long base = __ldg(A.wp + pos);
                    const int32_t ka = int32_t(max(iA, base) - base);
                    const int32_t kb = int32_t(min(iB, __ldg(A.wp + pos + 1)) - base);
                    len = kb - ka;
                    const int4 rec = __ldg(A.srec + pos);
                    pos0 = rec.y + ka;
                    key = rec.w - a;
                    sm.b.owner[tid] = rec.x;
                    sm.b.hit[tid] = 0;
                }
                int32_t nruns, items;
                build_runs(sm, len, pos0, tid < nb ? region_word(sm.tbase[key], sm.tlb[key]) : 0,
                           tid, nruns, items);
                if (items > 0) probe_runs(A, sm, nruns, items);
                __syncthreads();
                // the next batch writes only this thread's owner/hit entries
                flush_owners(A, sm, nb, tri);
            }
            for (int k = tid; k < slen; k += kThreads) {
                const int32_t v = sm.cnt[k];
                if (v) {
                    const int32_t lr = last_le(sm.loc, 0, nr - 1, k);
                    atomicAdd(A.S + sm.gbase[lr] + (k - sm.loc[lr]), v);
                }
            }
            __syncthreads();
            if (nr == 0) {  // no row fits a stage: cannot happen for rows <= kCap
                if (tid == 0) give_up(A.sched, A.err, kGiveUpStage, a, L);
                break;
            }
            a += nr;
        }
    }
    tri = warp_sum_ll((long long)tri);
    if (lane == 0 && tri) atomicAdd(A.tri, tri);
}

// Resident support CTAs per device (SM count x CTAs per SM), set up once per
// device together with the kernel's shared-memory attribute, which is a
// per-device setting.  The first caller on a device does the set-up under a
// lock; later callers read the table without it.
constexpr int kMaxDevices = 64;
std::atomic<int> g_support_blocks[kMaxDevices];
std::mutex g_configure_mu;

cudaError_t configure_support(int *blocks) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int b = g_support_blocks[dev].load(std::memory_order_acquire);
    if (b > 0) {
        *blocks = b;
        return cudaSuccess;
    }
    std::lock_guard<std::mutex> lock(g_configure_mu);
    b = g_support_blocks[dev].load(std::memory_order_acquire);
    if (b == 0) {
        int sms = 0, occ = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(support_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(sizeof(SupportSmem)));
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, support_kernel, kThreads,
                                                              sizeof(SupportSmem));
        if (e != cudaSuccess) return e;
        b = sms * (occ > 0 ? occ : 1);
        g_support_blocks[dev].store(b, std::memory_order_release);
    }
    *blocks = b;
    return cudaSuccess;
}

