/*
 * ktruss.h: C ABI of the GB300 (sm_103a) K-truss library, libktruss.so.
 *
 * Method: fine-grained Eager K-truss (M. Blanco, T. M. Low, K. Kim, "Exploration
 * of Fine-Grained Parallelism for Load Balancing Eager K-truss on GPU and CPU",
 * HPEC 2019).  The K-truss of an undirected graph is its largest subgraph in
 * which every edge lies in at least K-2 triangles of that subgraph (Sec. I).
 * It is reached by Alg. 1: compute the support of every live edge, remove every
 * edge whose support is below K-2, repeat until a round removes nothing.
 * Supports are computed per edge task (Alg. 3): edge (i, kappa) intersects the
 * part of row i after kappa with row kappa, and every common column w credits
 * the three edges (i,kappa), (i,w), (kappa,w) (the eager rule of Sec. II-B).
 *
 * Graph format (Sec. II-B, Sec. III-D): strictly upper-triangular CSR.
 *   row_ptr  int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col      int32[m],   row_ptr[i] <= p < row_ptr[i+1] => i < col[p] < n,
 *                        columns strictly increasing within a row
 * Edge e is CSR slot e; every per-edge output is indexed by that slot.
 * Limits: 0 <= n < 2^31, 0 <= m < 2^31.
 *
 * Memory kinds: KTRUSS_HOST means ordinary (pageable or pinned) host memory,
 * KTRUSS_DEVICE means device memory of the current CUDA device.  Device-side
 * work is issued on `cuda_stream` (a cudaStream_t; NULL = the legacy default
 * stream).  Every call returns after the work it issued has completed, so
 * outputs may be read, and inputs freed, as soon as it returns.
 *
 * Errors: every int-returning call returns KTRUSS_OK (0) or a negative code;
 * no C++ exception crosses this boundary.  ktruss_strerror() names a code, and
 * ktruss_last_cuda_error() gives the CUDA error behind the last KTRUSS_ECUDA
 * of the calling thread.
 *
 * Threads: a graph handle may be used by one call at a time; a call that finds
 * the handle in use returns KTRUSS_EBUSY.  Distinct handles are independent.
 */
#ifndef KTRUSS_H
#define KTRUSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KTRUSS_OK 0
#define KTRUSS_EINVAL (-1)   /* bad argument or malformed CSR */
#define KTRUSS_ENOMEM (-2)   /* device or host allocation failed */
#define KTRUSS_ECUDA (-3)    /* a CUDA runtime call failed */
#define KTRUSS_ETIMEOUT (-4) /* a bounded device wait gave up */
#define KTRUSS_EBUSY (-5)    /* handle in use by another call */

#define KTRUSS_HOST 0
#define KTRUSS_DEVICE 1

/* Support kernels selectable with KTRUSS_OPT_SUPPORT_KERNEL. */
#define KTRUSS_KERNEL_BALANCED 0 /* work-prefix balancer + staged warp intersection */
#define KTRUSS_KERNEL_EDGE 1     /* one thread per edge, two-pointer merge (Alg. 3 task as-is) */
#define KTRUSS_KERNEL_COARSE 2   /* one thread per row (coarse-grained Alg. 2), for comparison */
#define KTRUSS_KERNEL_AUTO 3     /* default: per round, EDGE below 131072 live edges, else BALANCED */

/*
 * How the supports of the rounds after the first are obtained, selectable
 * with KTRUSS_OPT_UPDATE.  Alg. 1 recomputes S of the whole live graph each
 * round.  The decremental update instead subtracts, from every surviving
 * edge's support, the triangles it loses with the removed edges (each triangle
 * that contains a removed edge is enumerated once).  Both give the same
 * supports, masks, removals and round counts; they differ only in time.
 */
#define KTRUSS_UPDATE_NEVER 0  /* recompute S every round (Alg. 1 as written) */
#define KTRUSS_UPDATE_ALWAYS 1 /* decremental update after every round that removes edges */
#define KTRUSS_UPDATE_AUTO 2   /* default: update when the removed edges that lie in
                                  triangles are few next to the surviving edges
                                  (at most one per four surviving edges), else
                                  recompute */

/* Option keys for ktruss_set_option. */
#define KTRUSS_OPT_SUPPORT_KERNEL 1 /* KTRUSS_KERNEL_* */
#define KTRUSS_OPT_TIMING 2         /* 1 = record per-phase CUDA events (default 1) */
#define KTRUSS_OPT_UPDATE 3         /* KTRUSS_UPDATE_* */
#define KTRUSS_OPT_LIGHT_MERGE 4    /* balanced step: tasks whose two lists (tail of row i,
                                       row kappa) hold at most this many columns together
                                       are merged by one thread instead of being staged
                                       and probed; 0..1024, default 64 */
#define KTRUSS_OPT_SMALL_EDGES 5    /* KTRUSS_KERNEL_AUTO: live graphs with fewer edges use
                                       the one-thread-per-edge kernel; >= 0, default
                                       131072 */
#define KTRUSS_OPT_SUPPORT_SHAPE 7  /* CTA shape of the balanced support kernel: 0 = 1024
                                       threads per CTA, one CTA per SM, stages of 8192 staged
                                       slots (32 warps resident); 1 (default) = 512 threads,
                                       three CTAs per SM, stages of 2048 slots (48 warps);
                                       results identical */
#define KTRUSS_OPT_REORDER 8        /* 1 (default): runs start from the handle's vertices
                                       renumbered by ascending degree (ties by old id; in a
                                       batch within each graph), made once at load on the
                                       device (graph rebalancing by sorting, the paper's
                                       future work, Sec. V); outputs stay in input edge
                                       order and are identical; 0: runs use the loaded
                                       numbering */
#define KTRUSS_OPT_DEVICE_LOOP 6    /* 1 (default): rounds whose supports come from the
                                       decremental update run in a device-driven loop (one
                                       CUDA graph launch, conditional nodes, no host
                                       synchronisation per round; results identical);
                                       0: every round is driven from the host */

typedef struct ktruss_graph ktruss_graph; /* opaque, library-owned */

/* Statistics of the last ktruss_run on a handle (Alg. 1 bookkeeping). */
typedef struct {
    int32_t rounds;            /* peel rounds (Alg. 1 iterations): supports evaluated on a live graph
                                  by the support step or the decremental update */
    int64_t edges_in;          /* m */
    int64_t edges_out;         /* edges in the K-truss */
    int64_t triangles_out;     /* triangles of the K-truss */
    int32_t per_round_len;     /* = rounds */
    const int64_t *removed_per_round;   /* [rounds] edges removed by each round */
    const int64_t *live_per_round;      /* [rounds] live edges entering each round */
    const int64_t *triangles_per_round; /* [rounds] triangles of the live graph of each round */
    const float *ms_support_per_round;  /* [rounds] support kernel time (timing on) */
    const int64_t *merge_work_per_round; /* [rounds] sum over live edges of the lengths of
                                            the two lists each edge task intersects (the
                                            tail of row i and row kappa); 0 with the
                                            thread-per-edge kernel */
    float ms_total;            /* whole run, device time on the stream (timing on) */
    float ms_support;          /* sum of support steps */
    float ms_balance;          /* sum of work-estimate / scan / partition steps */
    float ms_prune_compact;    /* sum of prune + compaction steps */
    float ms_finalize;         /* final scatter of outputs to input edge order */
    int32_t support_launches;  /* support-kernel launches issued */
    int32_t kernel_launches;   /* all kernels of this library issued by the run */
    const int32_t *updated_per_round; /* [rounds] 1 where the round's supports came from the
                                         decremental update of the previous round's (no
                                         support step ran: its time and merge work are 0) */
    float ms_update;           /* sum of decremental updates (timing on) */
    float ms_device_loop;      /* rounds run by the device-driven round loop (CUDA graph
                                  launches and the final scatter after one; timing on) */
    int32_t device_loop_launches; /* launches of the device-driven round loop */
    int32_t device_loop_rounds;   /* rounds it ran (included in rounds above) */
} ktruss_stats_t;

/*
 * Copies a strictly upper-triangular CSR graph into a new library-owned handle
 * on the current CUDA device (Sec. II-B input; Sec. III-D layout).
 *   out        receives the handle (set to NULL on error)
 *   n, m       vertex and edge counts
 *   row_ptr    int32[n+1], col int32[m], in memory of kind mem_kind
 *   cuda_stream stream for the copies and the validation kernel
 * The caller keeps ownership of row_ptr/col and may free them on return.
 * The whole CSR contract is validated on the device before the handle is
 * returned.  Returns KTRUSS_EINVAL for n < 0, m < 0, m >= 2^31, NULL arrays
 * (col may be NULL when m == 0), a bad mem_kind, row_ptr[0] != 0,
 * row_ptr[n] != m, a decreasing row_ptr, a column <= its row or >= n, or
 * columns not strictly increasing in a row; KTRUSS_ENOMEM, KTRUSS_ECUDA.
 */
int ktruss_load_csr(ktruss_graph **out, int32_t n, int64_t m, const int32_t *row_ptr,
                    const int32_t *col, int mem_kind, void *cuda_stream);

/*
 * Computes the K-truss of the loaded graph by Alg. 1 with fine-grained support
 * tasks (Alg. 3) and writes, per input edge slot e:
 *   mask_out[e]    = 1 if e is in the K-truss, else 0          (uint8[m])
 *   support_out[e] = number of triangles of the K-truss on e,
 *                    0 for removed edges                       (int32[m]; may be NULL)
 * Outputs are caller-owned, of kind mem_kind.  The loaded graph is not
 * modified, so several K may be run on one handle.  Rounds, removals and
 * timings are available from ktruss_stats until the next run or free.
 * K = 2 keeps every edge and returns triangle counts.
 * Returns KTRUSS_EINVAL for K < 2 or a NULL mask_out with m > 0,
 * KTRUSS_ENOMEM, KTRUSS_ECUDA, KTRUSS_ETIMEOUT, KTRUSS_EBUSY.
 */
int ktruss_run(ktruss_graph *g, int32_t K, uint8_t *mask_out, int32_t *support_out, int mem_kind,
               void *cuda_stream);

/*
 * Loads a batch of graphs to be peeled together (batched K-truss; the paper
 * peels one graph at a time).  The batch is one block-diagonal strictly
 * upper-triangular CSR over n vertices and m edges, in the format of
 * ktruss_load_csr with global vertex ids: graph k owns the vertices
 * [vertex_offsets[k], vertex_offsets[k+1]) and every edge must join two
 * vertices of the same graph.
 *   num_graphs       G >= 1
 *   vertex_offsets   int32[G+1] in HOST memory, vertex_offsets[0] = 0,
 *                    non-decreasing, vertex_offsets[G] = n (empty graphs allowed)
 *   n, m, row_ptr, col, mem_kind, cuda_stream: as for ktruss_load_csr
 * The handle also accepts ktruss_run (one K for all graphs), ktruss_decompose
 * and ktruss_stats.  Returns KTRUSS_EINVAL for bad offsets, a malformed CSR or
 * an edge joining two graphs; KTRUSS_ENOMEM, KTRUSS_ECUDA.
 */
int ktruss_load_batch(ktruss_graph **out, int32_t num_graphs, const int32_t *vertex_offsets,
                      int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                      int mem_kind, void *cuda_stream);

/* Number of graphs of a batch handle (0 for a handle from ktruss_load_csr). */
int ktruss_batch_size(const ktruss_graph *g, int32_t *num_graphs);

/*
 * K-truss of every graph of a batch, graph k with its own K[k] (host int32[G],
 * each >= 2).  All graphs are peeled in the same bulk rounds: each round runs
 * one support step over every unfinished graph, prunes each graph with its own
 * threshold K[k] - 2, and lets the graphs whose round removed nothing leave the
 * live set with their final outputs.  Every graph gets exactly the outputs and
 * the number of rounds of its own ktruss_run.
 *   mask_out, support_out  as for ktruss_run, indexed by batch edge slot
 *   rounds_out             host int32[G] (may be NULL): support steps of each
 *                          graph, as ktruss_stats reports for a single run
 * ktruss_stats reports the batch's rounds.  Returns KTRUSS_EINVAL for a
 * handle that is not a batch, a NULL K, a K[k] < 2 or a bad mem_kind;
 * KTRUSS_ENOMEM, KTRUSS_ECUDA, KTRUSS_ETIMEOUT, KTRUSS_EBUSY.
 */
int ktruss_run_batch(ktruss_graph *g, const int32_t *K, uint8_t *mask_out, int32_t *support_out,
                     int32_t *rounds_out, int mem_kind, void *cuda_stream);

/*
 * K-truss request server (continuous batching; the paper serves one graph at
 * a time).  Requests are graphs in host memory with their own K.  Each
 * ktruss_server_step admits queued requests in arrival order while they fit
 * (a free request slot, room for the graph in the live state, and the
 * request's own device bytes — staged input plus outputs, see
 * ktruss_server_submit — within the budget), runs one peel round of Alg. 1
 * over all active requests as one batched computation, and completes the
 * requests whose round removed nothing (or removed every live edge).  Each
 * request gets exactly the outputs and round count of its own ktruss_run.
 *
 * ktruss_server_create: capacities of the live state (max_vertices,
 * max_edges < 2^31: sums over active requests), max_requests active at once,
 * request_bytes_budget = device bytes for the requests' own buffers; work is
 * issued on cuda_stream.  KTRUSS_EINVAL for bad sizes; KTRUSS_ENOMEM,
 * KTRUSS_ECUDA.
 */
typedef struct ktruss_server ktruss_server;
int ktruss_server_create(ktruss_server **out, int32_t max_vertices, int64_t max_edges,
                         int32_t max_requests, int64_t request_bytes_budget, void *cuda_stream);

/*
 * Queues a request: strictly upper-triangular CSR (n, m, row_ptr, col) in
 * HOST memory (copied here; the caller may free it on return) and its K >= 2.
 * mask_out (uint8[m]) and support_out (int32[m] or NULL) are HOST buffers the
 * caller keeps valid until the request is reported done; they are written
 * when it completes.  The request's device bytes are 4(n+1+m) + 5m + 768.
 * While they fit in what the budget has left and no request waits as a host
 * copy, the graph is copied straight to a device block and validated there
 * (the call synchronises the server's stream), and the request holds its
 * budget from then on; otherwise it is validated and copied on host threads
 * and staged at admission.  *ticket_out (may be NULL) identifies it.
 * KTRUSS_EINVAL for bad arguments, a malformed CSR, or a graph that could
 * never fit the server's capacities; KTRUSS_ENOMEM, KTRUSS_ECUDA.
 */
int ktruss_server_submit(ktruss_server *srv, int32_t n, int64_t m, const int32_t *row_ptr,
                         const int32_t *col, int32_t K, uint8_t *mask_out, int32_t *support_out,
                         int64_t *ticket_out);

/* Admission + one peel round + completion (see above); returns after the
 * round's work and the completed requests' output copies have finished.
 * *num_done (may be NULL) = requests completed by this step. */
int ktruss_server_step(ktruss_server *srv, int32_t *num_done);

/* Drains up to max completed (ticket, rounds) pairs, oldest first. */
int ktruss_server_take_done(ktruss_server *srv, int64_t *tickets, int32_t *rounds, int32_t max,
                            int32_t *count);

/* Queued requests, active requests, live edges (each pointer may be NULL). */
int ktruss_server_status(const ktruss_server *srv, int32_t *queued, int32_t *active,
                         int64_t *live_edges);

/* Sets KTRUSS_OPT_UPDATE (KTRUSS_UPDATE_*) for the server's rounds: with the
 * update, a step takes the supports of requests already active from the
 * previous step's (updated for the edges it removed) and runs a support step
 * over its own CSR for each request it admits.  Each active request chooses
 * for itself: under AUTO it is recomputed (one support step over the live
 * CSR that skips every other request) when its removed edges that lie in
 * triangles exceed a quarter of its surviving edges and either number at
 * least 65536 or some other request is recomputed anyway.  Results do not
 * depend on it.  Also KTRUSS_OPT_REORDER (1, default: each request's vertices
 * are renumbered by ascending degree when it is admitted, on the device,
 * working in the server's own scratch; 0: appended in their own numbering;
 * results identical).  KTRUSS_EINVAL for another key or value. */
int ktruss_server_set_option(ktruss_server *srv, int32_t key, int64_t value);

/* Releases the server and every buffer it holds (NULL is a no-op). */
void ktruss_server_free(ktruss_server *srv);

/*
 * Truss decomposition of the loaded graph: trussness_out[e] = the largest K
 * such that edge e is in the K-truss (2 for an edge in no triangle), and
 * *kmax_out = the largest K whose K-truss is not empty (0 for a graph with no
 * edge).  Runs Alg. 1 for K = 3, 4, ... in turn, each K starting from the
 * (K-1)-truss, which contains it (the K-trusses are nested, Sec. I); an edge
 * removed while peeling for K gets trussness K-1.  Between two values of K the
 * supports of the converged truss are reused instead of recomputed.
 *   trussness_out int32[m], kind mem_kind (caller-owned); kmax_out host, may be NULL
 * ktruss_stats afterwards reports the support steps executed (rounds) with
 * their live edges and triangles; edges_out and triangles_out are 0.
 * Returns KTRUSS_EINVAL for a NULL output with m > 0 or a bad mem_kind;
 * KTRUSS_ENOMEM, KTRUSS_ECUDA, KTRUSS_ETIMEOUT, KTRUSS_EBUSY.
 */
int ktruss_decompose(ktruss_graph *g, int32_t *trussness_out, int32_t *kmax_out, int mem_kind,
                     void *cuda_stream);

/*
 * Copies the statistics of the last ktruss_run or ktruss_decompose into *out.  The per-round
 * arrays point into the handle and stay valid until the next run or free.
 * Returns KTRUSS_EINVAL for NULL arguments or a handle never run.
 */
int ktruss_stats(const ktruss_graph *g, ktruss_stats_t *out);

/* Sets a KTRUSS_OPT_* option on a handle.  KTRUSS_EINVAL for an unknown key
 * or value. */
int ktruss_set_option(ktruss_graph *g, int32_t key, int64_t value);

/* Settings chosen by ktruss_autotune. */
typedef struct {
    int32_t light_merge;  /* KTRUSS_OPT_LIGHT_MERGE */
    int64_t small_edges;  /* KTRUSS_OPT_SMALL_EDGES */
    int32_t update_mode;  /* KTRUSS_OPT_UPDATE */
    float ms;             /* device time of the best run (ms) */
    int32_t trials;       /* runs timed */
    int32_t support_shape; /* KTRUSS_OPT_SUPPORT_SHAPE */
} ktruss_tune_t;

/*
 * Autotuner: picks KTRUSS_OPT_SUPPORT_SHAPE (threads per CTA and staging
 * tile of the support kernel), KTRUSS_OPT_LIGHT_MERGE (merge or stage-and-
 * probe, by list length), KTRUSS_OPT_SMALL_EDGES (per-edge or balanced kernel,
 * by live size) and KTRUSS_OPT_UPDATE for this handle's graph by timing whole
 * runs on it:
 * ktruss_run with K[0] when num_K == 1, or ktruss_run_batch with K[0..G) when
 * the handle is a batch of G graphs and num_K == G.  Candidates are tried one
 * option at a time (coordinate descent from the current settings, a second
 * pass over the options when the first changed any), each run
 * reps times (best time counts); the best settings are left set on the
 * handle and copied to *out (may be NULL).  Results of the runs are discarded
 * (device buffers owned by the handle).  The support kernel choice
 * (KTRUSS_OPT_SUPPORT_KERNEL) is left as set.  Errors as ktruss_run /
 * ktruss_run_batch; KTRUSS_EINVAL for bad num_K or reps < 1.
 */
int ktruss_autotune(ktruss_graph *g, const int32_t *K, int32_t num_K, int32_t reps,
                    ktruss_tune_t *out, void *cuda_stream);

/* Vertex and edge counts of a loaded handle.  KTRUSS_EINVAL for NULL. */
int ktruss_graph_size(const ktruss_graph *g, int32_t *n, int64_t *m);

/* Releases a handle (NULL is a no-op).  Its device memory (one block per
 * load, plus one for host-kind outputs) goes to a per-process cache of at most
 * 16 GiB, reused by later loads that need between half and all of a cached
 * block; an allocation that fails empties the cache and retries. */
void ktruss_free(ktruss_graph *g);

/* Frees every device block held by the cache of ktruss_free.  Returns
 * KTRUSS_OK. */
int ktruss_trim_cache(void);

/* Static string naming a KTRUSS_* code. */
const char *ktruss_strerror(int code);

/* The cudaError_t behind the calling thread's last KTRUSS_ECUDA (0 if none). */
int ktruss_last_cuda_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int ktruss_version(void);

/*
 * Support of every edge of a graph that stays in the caller's device memory,
 * computed without allocating any memory.  The paper has no counterpart: this
 * entry point exists for callers that may not call cudaMalloc or any other
 * allocating routine on their path (code running inside someone else's memory
 * pool or arena, code that must not grow the device footprint after start-up,
 * embedded users with a fixed memory budget).
 *
 * Computes what the first support step of ktruss_run computes: support_out[e]
 * = number of triangles of the whole graph on edge e (so it equals the
 * support_out of ktruss_run with K = 2), plus the triangle count.
 *   n, m          vertex and edge count; at most 524288 each
 *   row_ptr, col  strictly upper-triangular CSR in DEVICE memory (caller-owned)
 *   support_out   int32[m] in DEVICE memory (caller-owned), overwritten
 *   triangles_out host int64, may be NULL
 *   cuda_stream   stream for all work; the call returns when it has finished
 * Working memory is one fixed 32 MiB device array inside the library, held by
 * every GPU that loads the library until the process exits.  All calls share
 * it and it keeps the last call's contents; calls whose work overlaps on the
 * GPU (other streams or host threads) race on it and must not be issued.  The
 * first call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  Every call
 * synchronises cuda_stream and reads counters back to the host before it
 * returns.
 * Returns KTRUSS_EINVAL for n or m out of range (including above 524288),
 * NULL pointers or a malformed CSR (checked on the device first);
 * KTRUSS_ECUDA for a failed CUDA call or a device-side consistency check of
 * the support kernel that gave up (the supports are then incomplete);
 * KTRUSS_ETIMEOUT if a bounded device wait gave up.
 */
int ktruss_support_noalloc(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                           int32_t *support_out, int64_t *triangles_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KTRUSS_H */
