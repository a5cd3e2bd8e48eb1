// Internal interfaces of libktruss: kernel launchers shared by the C ABI
// runtime (capi.cu) and the kernel translation units.  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kt {

// Live graph of one peel round: strictly upper-triangular CSR plus, per slot,
// the input edge id it came from (eid == nullptr means the identity, which is
// the case before the first compaction).
struct Live {
    const int32_t *rp;   // [n+1]
    const int32_t *col;  // [m]
    const int32_t *eid;  // [m] or nullptr
    int32_t n;
    int32_t m;
    // Batches only (both null otherwise): gid[v] = graph of vertex v, and a
    // support step skips every task of a graph g with skip[g] != 0 (its
    // supports are current), leaving that graph's S untouched.
    const int32_t *gid = nullptr;
    const uint8_t *skip = nullptr;
};

// True when the task of an edge in row i belongs to a skipped graph.
__device__ __forceinline__ bool skipped_row(const Live &g, int32_t i) {
    return g.skip && g.skip[g.gid[i]];
}

// Device-side counters of one round, written by kernels, read once per round
// by the host through a pinned mirror.
struct RoundCounters {
    unsigned long long triangles;  // triangles found by the support step
    unsigned long long merge_work; // sum over live edges of tail + row-kappa lengths
    int32_t kept;                  // edges with support >= K-2
    int32_t error;                 // nonzero: a kernel detected an inconsistency
    int32_t removed_tri;           // removed edges with support > 0 (listed by prune)
    int32_t forced;                // per-graph decisions: graphs that need a support step
                                   // whatever the others do (first decision pass)
};

// Device error bits in RoundCounters::error during a run.
constexpr int32_t kDevErrTimeout = 1;   // a bounded wait gave up
constexpr int32_t kDevErrInternal = 2;  // an internal consistency check failed

constexpr int kWarp = 32;

// Default light-task threshold of the balanced support step (see
// BalancedScratch::light); chosen by a sweep on R-MAT and G(n,m) graphs.
constexpr int32_t kDefaultLight = 64;
constexpr int32_t kMaxLight = 1024;
// Default CTA shape of the support kernel (BalancedScratch::shape): the faster
// of the two on R-MAT-20 and on R-MAT-23 with planted cliques.
constexpr int32_t kDefaultShape = 1;
// Per-graph update rule of batches and the server: a graph's next supports
// come from the decremental update while its listed edges (removed, in some
// triangle) are at most a quarter of its surviving edges.  A graph above that
// with fewer than kRecomputeMinListed listed edges still takes the update
// when no graph needs a support step otherwise: a support step for a few
// small graphs classifies every live edge of the batch, which only pays off
// once some graph needs one anyway.
constexpr int32_t kRecomputeMinListed = 1 << 16;

// KTRUSS_TRACE=2 (or more): the launchers synchronise the stream after each
// phase and print its name and the time since the process loaded the library
// on stderr (a debugging aid; off by default).
bool trace_on();      // KTRUSS_TRACE >= 1
bool trace_phases();
void trace_phase(cudaStream_t s, const char *name);

// ---- device-driven round loop (loop.cu) ------------------------------------
// Control block of the device-driven round loop, in device memory.  The round
// kernels launched with a LoopCtl take the live edge count, the threshold and
// the round's decision from it instead of from their arguments (so their
// grids are fixed and they loop over the work), and skip their work when the
// decision does not call for it; the loop's decide and end kernels advance it.
constexpr int32_t kActUpdate = 1;   // the round updates S (decremental update)
constexpr int32_t kActCompact = 2;  // the round compacts the live graph into the other buffer
constexpr int32_t kActCarry = 4;    // the compaction carries S into the other buffer

// Why a device loop stopped (LoopCtl::status).
constexpr int32_t kLoopRunning = 0;
constexpr int32_t kLoopConverged = 1;    // a round removed nothing (fixed K): finalize
constexpr int32_t kLoopEmpty = 2;        // no edge is left
constexpr int32_t kLoopNeedSupport = 3;  // the next supports need a support step
constexpr int32_t kLoopCap = 4;          // record or iteration capacity reached

struct LoopCtl {
    // read by the round kernels
    int32_t m;           // live edges of the current graph
    int32_t thr;         // K - 2
    int32_t action;      // kAct* bits of the current round (decide kernel)
    int32_t nlist;       // listed edges of the round: removed with S > 0
    int32_t level;       // trussness written for edges removed now (K - 1)
    int32_t ldeg_valid;  // the update state's lower degrees are current
    uint8_t *mask_out;   // outputs of removed edges (may be null)
    int32_t *sup_out;
    int32_t *level_out;
    // loop state
    int32_t decompose;    // 1: K grows when a round removes nothing; 0: fixed K
    int32_t update_mode;  // KTRUSS_UPDATE_* value
    int32_t buf;          // CSR and S buffer holding the current graph (0 or 1)
    int32_t fresh;        // decompose: the current graph has not been pruned yet
    int32_t updated;      // the current graph's supports came from the update
    int32_t status;       // kLoop* value when the loop stopped
    int32_t rec, rec_cap; // round records written / capacity
    int32_t iters, iter_cap;  // loop iterations done / capacity
    long long tri;        // triangles of the current graph
};

// One round as the host records it (ktruss_stats): live edges, edges removed,
// whether the supports came from the update, triangles of the live graph.
struct LoopRecord {
    int32_t live;
    int32_t removed;
    int32_t upd;
    int32_t pad;
    long long tri;
};

// ---- device memory cache (memory.cu) ---------------------------------------
// cache_get: a block of at least `bytes` on the current device, reused from
// the cache (blocks of half to all of its size) or newly allocated; give it
// back with cache_put(p, bytes) using the same `bytes`.  cache_trim frees
// every cached block.
cudaError_t cache_get(size_t bytes, void **p);
void cache_put(void *p, size_t bytes);
void cache_trim();

// ---- validation (validate.cu) ----------------------------------------------
// Sets *err to a nonzero bit mask if (rp, col) violates the upper-triangular
// CSR contract.  *err must be zero on entry.
cudaError_t launch_validate(const int32_t *rp, const int32_t *col, int32_t n, int64_t m,
                            int32_t *err, cudaStream_t s);

// ---- support step (support_edge.cu, support_balanced.cu) -------------------
// S[0..m) must be zero on entry; adds every live edge's support into S and the
// number of triangles found into cnt->triangles.
cudaError_t launch_support_edge(const Live &g, int32_t *S, RoundCounters *cnt, cudaStream_t s);

// Coarse-grained support step (Alg. 2): one thread per row.
cudaError_t launch_support_coarse(const Live &g, int32_t *S, RoundCounters *cnt, cudaStream_t s);

// Scratch owned by the handle for the balanced support step, one block of
// balanced_scratch_bytes(n, m) carved into: per-edge classification and
// segment arrays, the int64 item prefix and the tile sums and offsets of its
// scans, per-row counts and active-row tables, the chunk plan, the chunk
// boundary table and the scheduler words.
struct BalancedScratch {
    void *base = nullptr;
    int64_t cap_m = 0;  // capacity in edges
    int32_t cap_n = 0;  // capacity in vertices
    // tasks whose two lists hold at most `light` columns together are merged
    // by one thread instead of being staged and probed (0 = none)
    int32_t light = kDefaultLight;
    // CTA shape of the support kernel: 0 = 1024 threads, one CTA per SM,
    // 8192-slot stages; 1 = 512 threads, three CTAs per SM, 2048-slot stages
    int32_t shape = kDefaultShape;
    // optional: a second stream and two events on which the light merge runs
    // alongside the balancing kernels (joined before the step returns)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
// Creates / destroys the side stream and events of a BalancedScratch.
cudaError_t balanced_side_create(BalancedScratch *bs);
void balanced_side_destroy(BalancedScratch *bs);

// Bytes of device scratch BalancedScratch needs for a graph of n vertices and
// m edges (used for allocation at load time).
size_t balanced_scratch_bytes(int32_t n, int64_t m);
// (also large enough for launch_reorder of any graph within n vertices and m edges)
cudaError_t balanced_scratch_alloc(BalancedScratch *bs, int32_t n, int64_t m);
void balanced_scratch_free(BalancedScratch *bs);

// Views of the balanced scratch used by the support update (which never runs
// at the same time as the balanced support step), all sized by the edge
// count m: lower-neighbour lists of the flagged vertices (lsrc, lslot; lcnt,
// lrp, lfill by compact vertex index), the list of removed edges that lie in
// triangles and per-entry data (list, lx), the flagged vertices (zlist), and
// the tile arrays of an int32 scan over up to m + 1 entries.
struct UpdateScratch {
    int32_t *lsrc, *lslot, *list, *lx, *zlist, *lcnt, *lrp, *lfill;
    int32_t *scan_sum, *scan_off, *scan_tot;
};

// State of the update that lives across rounds (owned by the caller): the
// lower degree of every vertex in the live graph (ldeg, n+1 ints; valid once
// ldeg_valid, after which prune subtracts the edges it removes), one flag
// word per vertex (n+1 ints, zero on entry and on return of every update)
// and a counter word (nz).
struct UpdateState {
    int32_t *ldeg = nullptr;
    int32_t *flag = nullptr;
    int32_t *nz = nullptr;
    bool ldeg_valid = false;
};
UpdateScratch update_scratch(const BalancedScratch *bs);
// out[i] = in[0] + ... + in[i-1] for i in [0, count) (int32, count <= cap_m + 1).
// With lc (device loop): count is the capacity, the scanned count is
// lc->nlist + 1 and nothing runs in rounds without update.
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int64_t count,
                            const UpdateScratch &u, cudaStream_t s, int *launches,
                            const LoopCtl *lc = nullptr);

// Balanced support step: work estimate + int64 scan + partition + staged
// warp-cooperative intersection.  Adds supports into S (zero on entry).
// Kernel launches issued are added to *launches.  When ev is given, ev[1] is
// recorded between the balance kernels and the support kernels.
cudaError_t launch_support_balanced(const Live &g, int32_t *S, RoundCounters *cnt,
                                    BalancedScratch *bs, cudaStream_t s, int *launches,
                                    cudaEvent_t *ev);

// ---- decremental support update (update.cu) --------------------------------
// S holds the exact supports of the live graph g and keep[] the decision of
// this round (0 = removed).  Subtracts from S[e] of every kept edge e the
// number of triangles of g that contain e and at least one removed edge, and
// adds the number of those triangles into *destroyed.  list[0..nlist) are the
// removed edges with S > 0 (removed edges with S = 0 lie in no triangle).
// Afterwards the kept edges' S are their supports in g minus the removed edges.
// st->ldeg is computed here the first time (st->ldeg_valid false).
// When pos is given (the slot map of a compaction that already ran, old slot
// -> new slot), the subtractions go to S_out[pos[q]] instead of S[q] (S is
// then only read).  When upd_g is given (batches: g.gid set), only listed
// edges of graphs with upd_g[graph] != 0 are processed.
cudaError_t launch_support_update(const Live &g, const uint8_t *keep, const int32_t *list,
                                  int32_t nlist, int32_t *S, unsigned long long *destroyed,
                                  const UpdateScratch &u, UpdateState *st, cudaStream_t s,
                                  int *launches, const int32_t *pos = nullptr,
                                  int32_t *S_out = nullptr, const uint8_t *upd_g = nullptr,
                                  const LoopCtl *lc = nullptr);

// ---- prune + compaction + finalize (compact.cu) ---------------------------
// Tile geometry of the compaction kernels.
constexpr int kCompactThreads = 256;
constexpr int kCompactItemsPerThread = 16;
constexpr int kCompactTile = kCompactThreads * kCompactItemsPerThread;

inline __host__ __device__ int32_t compact_tiles(int32_t m) {
    return int32_t((int64_t(m) + kCompactTile - 1) / kCompactTile);
}

// Grid of the round kernels inside the device loop: two waves of 8 blocks per
// SM, each block looping over its share of the tiles, slots or list entries
// (measured against one wave: the R-MAT-23 K sweep 2.65 -> 2.47 s; one block
// per SM doubles it).
constexpr int kLoopBlocks = 152 * 16;

// Counts edges with S >= thr per tile into tile_count[tiles], then scans the
// tile counts into tile_off[tiles] and writes the total into cnt->kept.  When
// keep is given, keep[e] = (S[e] >= thr); when list is given, the removed edges
// with S > 0 are appended to it and counted in cnt->removed_tri (reset here);
// when ldeg is given, every removed edge (u, v) subtracts one from ldeg[v].
cudaError_t launch_prune_count(const int32_t *S, int32_t m, int32_t thr, int32_t *tile_count,
                               int32_t *tile_off, RoundCounters *cnt, cudaStream_t s,
                               int *launches, uint8_t *keep = nullptr, int32_t *list = nullptr,
                               const int32_t *col = nullptr, int32_t *ldeg = nullptr,
                               const LoopCtl *lc = nullptr);

// Scatters kept edges (S >= thr) of `in` into (col_out, eid_out) in order,
// writes the exclusive kept-prefix of every slot into pos[m_in] (pos[m] =
// total), writes removed edges' final outputs (mask 0, support 0 at their
// input edge id) and builds rp_out[i] = pos[rp_in[i]] (cnt->kept for
// rp_in[i] == m).  mask_out / support_out may be null; when level_out is not
// null, removed edges also get level_out[id] = level (trussness).  When keep is
// given it decides which edges stay (instead of S >= thr); when S_out is given,
// kept edges carry their S into S_out at their new slot.
cudaError_t launch_compact(const Live &in, const int32_t *S, int32_t thr, const int32_t *tile_off,
                           const RoundCounters *cnt, int32_t *pos, int32_t *rp_out,
                           int32_t *col_out, int32_t *eid_out, uint8_t *mask_out,
                           int32_t *support_out, cudaStream_t s, int *launches,
                           int32_t *level_out = nullptr, int32_t level = 0,
                           const uint8_t *keep = nullptr, int32_t *S_out = nullptr,
                           const LoopCtl *lc = nullptr);

// Exclusive scan of tile counts by one block (total -> cnt->kept).
cudaError_t launch_scan_tiles(const int32_t *tile_count, int32_t tiles, int32_t *tile_off,
                              RoundCounters *cnt, cudaStream_t s, int *launches);

// rp_out[i] = pos[rp_in[i]] (cnt->kept where rp_in[i] == m).
cudaError_t launch_rowptr(const Live &in, const int32_t *pos, const RoundCounters *cnt,
                          int32_t *rp_out, cudaStream_t s, int *launches);

// ---- device-driven round loop (loop.cu) ------------------------------------
// The buffers of a handle that the loop's kernels are captured with: the two
// live CSR buffers and the two support buffers (buffer p holds a graph whose
// supports are S[p]; a round reads p and writes p ^ 1), the compaction and
// prune arrays, the round counters ([2]: the round's, the update's), the
// update's scratch and state, the control block and the round records.
struct LoopBuffers {
    int32_t n = 0, cap_m = 0;
    int32_t *rp[2] = {nullptr, nullptr}, *col[2] = {nullptr, nullptr},
            *eid[2] = {nullptr, nullptr}, *S[2] = {nullptr, nullptr};
    int32_t *pos = nullptr, *tile_count = nullptr, *tile_off = nullptr;
    uint8_t *keep = nullptr;
    RoundCounters *cnt = nullptr;
    UpdateScratch us{};
    const UpdateState *ust = nullptr;
    LoopCtl *lc = nullptr;
    LoopRecord *rec = nullptr;
};
// The instantiated loop graph of a handle (built on first use, on the device
// the handle lives on; launched with cudaGraphLaunch on the caller's stream).
struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
};
cudaError_t loop_graph_build(LoopGraph *lg, const LoopBuffers &b);
void loop_graph_destroy(LoopGraph *lg);

// st->ldeg = lower degree of every vertex in the live graph g (all its edges).
cudaError_t launch_lower_degree(const Live &g, UpdateState *st, cudaStream_t s, int *launches);

// ---- degree-ordered relabel (reorder.cu) -----------------------------------
// Bytes of working memory launch_reorder needs for a graph of n vertices and
// m edges.
size_t reorder_scratch_bytes(int32_t n, int64_t m);
// Numbers the vertices of the upper-triangular CSR (rp, col) by ascending
// degree (ties by old id) and writes the relabelled strictly upper-triangular
// CSR (rp_out[n+1], col_out[m], columns sorted) and, per slot, the input slot
// of its edge (eid_out[m]).  With gid (batches of num_graphs graphs with
// contiguous vertex ranges, gid[v] = graph of v) vertices are ordered by
// graph first, so every graph keeps its range.  scratch:
// reorder_scratch_bytes(n, m) bytes.
cudaError_t launch_reorder(const int32_t *rp, const int32_t *col, int32_t n, int64_t m,
                           void *scratch, int32_t *rp_out, int32_t *col_out, int32_t *eid_out,
                           cudaStream_t s, const int32_t *gid = nullptr, int32_t num_graphs = 0);

// ---- batches (batch.cu) -----------------------------------------------------
// gid[v] = graph of vertex v for vertex offsets vo[G+1].
cudaError_t launch_graph_of_vertex(const int32_t *vo, int32_t G, int32_t n, int32_t *gid,
                                   cudaStream_t s);
// Sets bit 16 of *err if an edge joins two graphs.
cudaError_t launch_batch_validate(const int32_t *rp, const int32_t *col, int32_t n,
                                  const int32_t *gid, int32_t *err, cudaStream_t s);
// Per-graph thresholds: keep flags, per-graph flags kept_g / removed_g (the
// round kept / removed some edge of the graph; zero on entry), finished flags
// and round counters, tile counts and their scan (edges that stay live ->
// cnt->kept).
// When list is given, removed edges with S > 0 are appended to it and counted
// in cnt->removed_tri (reset here); when ldeg is given, every removed edge
// (u, v) subtracts one from ldeg[v].
cudaError_t launch_batch_prune(const Live &g, const int32_t *S, const int32_t *gid,
                               const int32_t *thr, uint8_t *keep, int32_t *kept_g,
                               int32_t *removed_g, uint8_t *done, int32_t *rounds_g, int32_t G,
                               int32_t *tile_count, int32_t *tile_off, RoundCounters *cnt,
                               cudaStream_t s, int *launches, int32_t *list = nullptr,
                               int32_t *ldeg = nullptr, int32_t *listed_g = nullptr);
// After a round's compaction (rp_new), per graph: surviving edges and the
// choice of update (upd_g = 1) or support step for its next supports (mode:
// KTRUSS_UPDATE_* values); cnt (cleared here): kept = graphs that stay live,
// removed_tri = those that need a support step.
cudaError_t launch_batch_decide(int32_t G, const int32_t *vo, const int32_t *rp_new,
                                const int32_t *listed_g, int32_t mode, uint8_t *upd_g,
                                RoundCounters *cnt, cudaStream_t s, int *launches);
// S[e] = 0 for the live edges of graphs with upd_g == 0.
cudaError_t launch_batch_zero(const Live &g, const int32_t *gid, const uint8_t *upd_g, int32_t *S,
                              cudaStream_t s, int *launches);
// Keep flags (support >= threshold of the edge's graph) and the per-graph
// kept_g / removed_g flags (zero on entry) only.
cudaError_t launch_batch_keep(const Live &g, const int32_t *S, const int32_t *gid,
                              const int32_t *thr, uint8_t *keep, int32_t *kept_g,
                              int32_t *removed_g, cudaStream_t s, int *launches,
                              int32_t *list = nullptr, int32_t *list_count = nullptr,
                              int32_t *listed_g = nullptr);

// ---- request server (server_kernels.cu) --------------------------------------
// Appends a request's device CSR at vertex base nb / edge base mb of the live CSR
// (emap, when given: the request-local input edge of each slot).
cudaError_t launch_server_append(const int32_t *rp_in, const int32_t *col_in, int32_t n, int32_t m,
                                 int32_t nb, int32_t mb, int32_t slot, int32_t *rp, int32_t *col,
                                 int32_t *eid, int32_t *gid, cudaStream_t s,
                                 const int32_t *emap = nullptr);
// Keep flags and per-slot kept / removed flags (= launch_batch_keep); removed edges with
// S > 0 appended to list when given (count in *list_count, zero on entry) and
// counted per slot in listed_s when given.
cudaError_t launch_server_prune(const Live &cur, const int32_t *S, const int32_t *gid,
                                const int32_t *thr, uint8_t *keep, int32_t *kept_g,
                                int32_t *removed_g, cudaStream_t s, int *launches,
                                int32_t *list = nullptr, int32_t *list_count = nullptr,
                                int32_t *listed_s = nullptr);
// Per slot after a round tail (kept_s: the slot's surviving edges, as
// counted by the round tail): upd_s = 1 when its next supports come from the
// update (mode 0 never, 1 always, 2 the kRecomputeMinListed rule), cnt->kept =
// live slots, cnt->removed_tri = live slots that need a support step.
cudaError_t launch_server_decide(int32_t slots, const int32_t *kept_s, const int32_t *listed_s,
                                 int32_t mode, uint8_t *upd_s, RoundCounters *cnt, cudaStream_t s,
                                 int *launches);
// Finished slots, vertex renumbering (vcnt->kept = surviving vertices),
// edge compaction (cnt->kept = surviving edges) with outputs of leaving edges
// through the per-slot pointer tables, new row pointers and slot ids.  When
// given, S_out receives the S of the surviving edges in their new order and
// kept_s (zero on entry) each slot's surviving edges.
cudaError_t launch_server_round_tail(const Live &cur, const int32_t *S, const uint8_t *keep,
                                     const int32_t *kept_g, const int32_t *removed_g,
                                     uint8_t *fin, int32_t *rounds_g, int32_t slots,
                                     const int32_t *gid, int32_t *vmap, int32_t *vtile_count,
                                     int32_t *vtile_off, RoundCounters *vcnt, int32_t *etile_count,
                                     int32_t *etile_off, RoundCounters *cnt, int32_t *pos,
                                     int32_t *rp_out, int32_t *col_out, int32_t *eid_out,
                                     int32_t *gid_out, uint8_t *const *mask_ptr,
                                     int32_t *const *sup_ptr, cudaStream_t s, int *launches,
                                     int32_t *S_out = nullptr, int32_t *kept_s = nullptr);

// Compaction of the edges that stay live; outputs of the edges that leave.
// When S_out is given, edges that stay carry their S into S_out.
cudaError_t launch_batch_compact(const Live &in, const int32_t *S, const uint8_t *keep,
                                 const uint8_t *done, const int32_t *gid, const int32_t *tile_off,
                                 const RoundCounters *cnt, int32_t *pos, int32_t *rp_out,
                                 int32_t *col_out, int32_t *eid_out, uint8_t *mask_out,
                                 int32_t *support_out, cudaStream_t s, int *launches,
                                 int32_t *S_out = nullptr);

// Final outputs of the surviving edges: mask 1 and support S at their input id.
cudaError_t launch_finalize(const Live &g, const int32_t *S, uint8_t *mask_out,
                            int32_t *support_out, cudaStream_t s, int *launches);

}  // namespace kt
