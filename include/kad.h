/*
 * kad.h -- C ABI of the GB300 (sm_103a) KADABRA sampling library.
 *
 * KADABRA (Borassi & Natale) approximates betweenness centrality by adaptive
 * sampling; arXiv 1903.09422 (van der Grinten, Angriman, Meyerhenke, "Parallel
 * Adaptive Sampling with almost no Synchronization") parallelises its sampling
 * loop.  This library runs that loop on one GPU: every sample, the fold of
 * samples into the sampling state, and the stop check are CUDA kernels.
 *
 * Problem statement (Section 2.2-2.3): given an undirected graph G, eps and
 * delta, return b~(v) with |b~(v) - b(v)/(n(n-1))| <= eps for all v with
 * probability >= 1 - delta, where b(v) = sum over ordered pairs s != t != v of
 * sigma_st(v)/sigma_st.
 *
 * Conventions for every entry point:
 *   - Errors are returned as kad_status; the library never aborts or exits.
 *   - Pointers documented "host" are ordinary CPU memory; "device" pointers are
 *     CUDA global memory on the graph's device.  The caller keeps ownership of
 *     every array it passes; the library keeps none of them after returning.
 *   - A CUDA error poisons the graph handle (every later call on it returns
 *     KAD_ERR_CUDA); free it with kad_graph_free.
 *   - Calls that take a cudaStream_t enqueue their device work on that stream
 *     and return after synchronising it (the results are ready on return).
 *   - A graph handle must not be used by two host threads at once.
 */
#ifndef KAD_H
#define KAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *kad_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    KAD_OK = 0,
    KAD_ERR_INVALID_ARG = 1, /* argument out of range (eps, delta, n, NULL where required, ...) */
    KAD_ERR_BAD_CSR = 2,     /* CSR not symmetric / unsorted / self-loop / duplicate / out of range */
    KAD_ERR_OOM = 3,         /* device or host allocation failed; nothing leaked */
    KAD_ERR_CUDA = 4,        /* a CUDA call failed; the graph handle is poisoned */
    KAD_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    KAD_ERR_CANCELLED = 6,   /* the run was cancelled */
    KAD_ERR_INTERNAL = 7     /* a device-side consistency check failed (bug report material) */
} kad_status;

typedef struct kad_graph kad_graph; /* opaque; owns a device copy of the CSR */

/* Flags for kad_graph_create*. */
#define KAD_GRAPH_TRUSTED 1u  /* skip the O(m log d) symmetry validation of an undirected CSR */
#define KAD_GRAPH_DIRECTED 2u /* the CSR lists out-arcs of a directed graph (no symmetry required) */
#define KAD_GRAPH_TIGHT_VD 4u /* undirected: the double-sweep vertex-diameter bound (see below) */

/*
 * kad_graph_create -- copy a graph to the current CUDA device.
 *
 * Input (host): row_ptr[n+1] and col[row_ptr[n]], int32.  Undirected (default):
 * a symmetric CSR, every edge {u,v} appearing as arcs u->v and v->u.  With
 * KAD_GRAPH_DIRECTED: the out-arc rows of a directed graph (Section 5: KADABRA
 * also covers directed graphs).  Either way each row sorted strictly ascending,
 * no self-loops, no duplicates.  n >= 2.
 *
 * Graph set-up computes on the device (Section 2.3 preprocessing and
 * Appendix C.1): the connected components, and the vertex-diameter bound
 * VD = max over components of 2 ecc(v0) + 1, v0 = the component's vertex of
 * largest degree (smallest id on ties), by one multi-source BFS.  For a directed
 * graph: its in-arc rows (sorted; the t side of each sample searches along
 * them), the weak components, and VD = the heaviest chain of the strongly
 * connected components' DAG, a component S weighing min(|S|, ecc_in(r) +
 * ecc_out(r) + 1) with r its vertex of largest out- plus in-degree (smallest id
 * on ties) and the eccentricities taken within S.  A sample (s, t) with no
 * directed s-t path counts, with no increments.  With KAD_GRAPH_TIGHT_VD (an
 * undirected graph; ignored for a directed one) each component's bound becomes
 * 2 min(ecc(v0), ecc(m)) + 1, m the midpoint of a double sweep: a = the vertex
 * farthest from v0, b = the vertex farthest from a (smallest ids on ties), m =
 * the vertex with d(a,m) + d(m,b) = d(a,b) and d(a,m) = ceil(d(a,b)/2) nearest
 * v0 (then smallest id).  It is never above the default bound, costs four more
 * BFSs, and lowers omega when it crosses a power of two.
 * Errors: KAD_ERR_INVALID_ARG (n < 2, NULL pointer, m >= 2^31), KAD_ERR_BAD_CSR,
 * KAD_ERR_OOM, KAD_ERR_CUDA.  On error *out is NULL.
 */
kad_status kad_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col, uint32_t flags,
                            kad_stream_t stream, kad_graph **out);

/* Same, from device arrays (copied device-to-device; the caller keeps them). */
kad_status kad_graph_create_device(int32_t n, int64_t m, const int32_t *d_row_ptr, const int32_t *d_col,
                                   uint32_t flags, kad_stream_t stream, kad_graph **out);

/* Releases the graph.  Waits until the device is idle (as cudaFree does), then
   returns its arrays to the library's graph memory pool, which keeps them mapped
   for the next graph; its run workspace is kept for the next graph on the same
   device (see kad_trim).  NULL is a no-op. */
void kad_graph_free(kad_graph *g);

/* Frees the workspace kept from freed graphs and unmaps the free memory of the
 * graph pool.  kad_graph_free keeps the last freed graph's workspace (slot
 * scratch, epoch ring, per-vertex arrays: about 29 bytes x n x slots) for the
 * next graph created on the same device, one per device, and the graph pool
 * keeps freed CSR arrays and set-up scratch mapped, so that creating and freeing
 * graphs in a loop neither allocates nor clears them every time; both stay
 * until this call or the end of the process.  Not for use while other threads
 * run kad calls. */
void kad_trim(void);

/* Graph facts computed at creation: vertex and arc counts, VD bound, components. */
kad_status kad_graph_info(const kad_graph *g, int32_t *n, int64_t *m, int32_t *vd_bound, int32_t *components);

typedef struct {
    uint32_t epoch_size; /* N: samples per epoch; the stop check runs after each (App. C.2; default 1000) */
    uint32_t calib_div;  /* calibration length tau0 = N ceil(max(1, ceil(omega/calib_div))/N); default 100 */
    uint32_t ring_epochs;/* epochs of sample frames in flight at once (0 = automatic) */
    int32_t slots;       /* concurrent samples = resident sampling blocks (0 = automatic) */
    int32_t mcap;        /* meeting-set members kept in shared memory and ranked directly
                            (-1 = default 256, at most 256); larger sets are selected digit by
                            digit over the recorded members (up to mcap + 3840, the rest of
                            them in a per-slot global row), beyond that over the other side's
                            frontier.  0 forces the digit-wise path; results do not depend on it */
    int32_t block_threads; /* threads per sampling block: 128, 256, 512 or 1024 (0 = 512) */
    int32_t blocks_per_sm; /* resident sampling blocks per SM the kernel is built for: 128 threads 4|8,
                              256: 2|4, 512: 1|2, 1024: 1 (0 = 4, 2, 2, 1 respectively).  When both
                              are 0 the kernel is 256x4 on graphs of average degree at most 8
                              and 512x2 otherwise, or with KAD_RUN_AUTOTUNE the fastest of
                              512x2, 256x4, 256x2, 1024x1 and 128x8 on this graph */
    uint32_t flags;      /* KAD_RUN_* */
    uint32_t debug;      /* KAD_DEBUG_* (tests only; results do not depend on it) */
    uint32_t max_epochs; /* > 0: stop after this many epochs even if the stop rule does not hold
                            (a truncated run, for comparisons on large graphs); 0 = no limit */
    int32_t samples_per_block; /* > 0: the warp-per-sample kernel -- one block of 1024 threads per SM,
                                  this many of its 32 warps (at most 32) each computing its own
                                  samples, all of them expanding large rounds for each other through
                                  a job board in shared memory; 0 = the library's choice of kernel.
                                  block_threads / blocks_per_sm then do not apply */
    int32_t pair_cost;   /* the frontier-switch threshold: a round's pairwise test (|F_X| x |F_Y|
                            adjacency tests between the two frontiers before scanning X's rows) runs
                            when |F_X| x |F_Y| x pair_cost is below the arcs of F_X, those arcs are at
                            least 1024 and F_X fits one block's threads (one warp's in the
                            warp-per-sample kernel): the cost of one test counted in arc reads.
                            1..1048576; 0 = 8, or with KAD_RUN_AUTOTUNE the fastest of 4, 8 and 16
                            on this graph; KAD_ERR_INVALID_ARG outside.  Results do not depend on it */
} kad_options;

#define KAD_RUN_TIMING 1u      /* fill kad_result.t_* with CUDA-event times of each phase */
#define KAD_RUN_AUTOTUNE 2u    /* the graph's first run (block_threads, blocks_per_sm and samples_per_block
                                  all 0) times the same query, truncated after 4 epochs, twice under each
                                  candidate -- block per sample 512x2, 256x4, 256x2, 1024x1, 128x8, and
                                  warp per sample with 8 or 24 samples per block -- and keeps the fastest
                                  for the graph's later runs; then, when pair_cost is 0, it times the
                                  chosen variant the same way with pair_cost 4 and 16 and keeps the
                                  fastest of those and 8 (graphs under 16384 vertices keep the
                                  defaults).  Off by default: the degree rule picks the fastest on every
                                  configured workload, and tuning costs 18 truncated runs */
#define KAD_RUN_COMPLETION_ORDER 4u /* the non-deterministic mode of the epoch-based framework
                                  (Section 3.1; local-/shared-frame of Section 3.2): epoch k holds
                                  the samples that were the (kN+1)-th to (k+1)N-th to complete,
                                  instead of samples kN..(k+1)N-1, so no epoch waits for a slow
                                  sample drawn early.  Each check still sees a consistent state
                                  (the first (k+1)N completed samples, tau = (k+1)N); which samples
                                  those are depends on timing.  kad_run_order lists them. */
#define KAD_DEBUG_TRACE_SCAN 1u    /* trace-back always scans the current vertex's adjacency */
#define KAD_DEBUG_SMEM_BITMAP 2u /* keep the labelled-vertex bitmap in shared memory when it fits */
#define KAD_DEBUG_FULL_SCAN 4u   /* the meeting round always scans the expanding side's rows */
#define KAD_DEBUG_SERIAL_TRACE 8u /* one team traces both sides (no speculative t-side trace) */
#define KAD_DEBUG_NO_BITMAP 16u   /* read every neighbour's label directly (the default on graphs of
                                     average degree 8 or less) */
#define KAD_DEBUG_BITMAP 32u      /* filter label reads through the bitmap whatever the degree */
#define KAD_DEBUG_COARSE_BITMAP 64u /* one bitmap bit per 8 vertices (the default only when the slots'
                                       exact bitmaps would exceed 32 MB) */
#define KAD_DEBUG_NO_PROBE 256u  /* claim new vertices from a large round's first scan (no probe scan for
                                    the meeting first); results do not depend on it */
#define KAD_DEBUG_NO_MEXT 128u   /* record at most mcap meeting-set members (in shared memory);
                                    larger sets are re-collected from the other side's frontier */

/* Initialises *opt to the defaults above. */
void kad_options_default(kad_options *opt);

typedef struct {
    /* outputs the caller may request by setting the pointer before the call (NULL = not wanted) */
    double *bc;       /* host, n: b~(v) = counts[v]/tau, estimating b(v)/(n(n-1)) */
    uint32_t *counts; /* host, n: sum over the used samples of x_i(v) */
    uint32_t *c0;     /* host, n: calibration counts */
    double *ltab;     /* host, ltab_cap: L[c] = log(1/delta_v) for calibration count c, c = 0..tau0 */
    int64_t ltab_cap;
    /* scalars filled by the call */
    uint64_t tau;              /* samples used (= epochs * N) */
    uint64_t omega;            /* maximal number of samples (Section 2.3) */
    uint64_t calib_samples;    /* tau0 */
    uint64_t samples_computed; /* samples computed: calibration + adaptive, including speculative ones */
    uint64_t overflow_samples; /* used samples whose shortest-path count saturated at 2^64-1 */
    uint32_t epochs;           /* stop-check epochs used */
    int32_t vd_bound;
    int32_t sigma_overflow;    /* 1 if any used sample saturated */
    int32_t stopped_by_omega;  /* 1 if the run stopped because tau >= omega, 2 if by max_epochs */
    double tau_star;           /* calibration's bisection result */
    /* work of all samples computed (calibration and adaptive): frontier vertices
       expanded, arcs scanned, vertices labelled, arcs into the next level or
       meeting set, arcs read by the trace-back, path increments */
    uint64_t work[6];
    /* KAD_RUN_TIMING, milliseconds: t_total (CUDA events around the whole call's
       device work), t_calib (host wall time from the first launch until the
       calibration histogram arrived; sampling continues meanwhile), t_ads (events
       from the first sampling launch to the end), t_ads_kernel (events around the
       first sampling launch, which runs calibration and adaptive samples) */
    double t_total_ms, t_calib_ms, t_ads_ms, t_ads_kernel_ms;
    uint32_t ads_launches;     /* sampling-kernel launches */
    int32_t slots_used;        /* concurrent samples (resident sampling blocks) */
    uint32_t kernel_launches;  /* kernels this call launched (all phases) */
    int32_t block_threads_used, blocks_per_sm_used; /* sampling-kernel variant used */
    /* SM cycles the sampling blocks spent per stage of a sample, summed over
       blocks and samples: pair draw and set-up, BFS, meeting draw, trace-back
       and output, slot reset, epoch bookkeeping and close */
    uint64_t phase_cycles[6];
    /* KAD_RUN_TIMING, host milliseconds: t_host (the whole call), t_setup (from
       the call's entry until its first device work is enqueued), t_table (from the
       histogram's arrival until the L table is enqueued for upload: tau* and L) */
    double t_host_ms, t_setup_ms, t_table_ms;
    /* KAD_RUN_TIMING, the device's timeline of the sampling, milliseconds after
       its first sample started: calibration histogram published, first epoch
       closed, stop decided, last sampling block finished; and the sample indices
       (calibration + adaptive) handed out when the stop was decided */
    double t_dev_calib_ms, t_dev_first_close_ms, t_dev_stop_ms, t_dev_end_ms;
    uint64_t issued_at_stop;
    /* the warp-per-sample kernel's sampling contexts per block (0: the block-per-sample kernel ran) */
    int32_t samples_per_block_used;
    int32_t pair_cost_used;    /* the pairwise test's cost factor the sampling kernel ran with */
    /* of phase_cycles' BFS stage: cycles in expansion passes, and in round closes
       (the rest is pairwise tests and loading frontiers) */
    uint64_t bfs_split_cycles[2];
} kad_result;

/*
 * kad_run -- KADABRA on g: calibration, then adaptive sampling until the stop
 * rule holds (Algorithm 1 of Section 2.1 with KADABRA's sample() and
 * checkForStop of Section 2.3 and Appendix B, checked every N samples).
 *
 * Random numbers: sample i of phase d (0 = adaptive, 1 = calibration) draws from
 * Philox4x32-10 with key = seed and counter = (i, block, d), so the result depends
 * only on (g, eps, delta, seed, N, calib_div) -- never on the launch configuration
 * (the deterministic indexed-frame idea of Appendix D.2).
 * 0 < eps < 1, 0 < delta < 1.  Errors: KAD_ERR_INVALID_ARG, KAD_ERR_OOM,
 * KAD_ERR_CUDA, KAD_ERR_INTERNAL.  opt NULL = defaults.
 */
kad_status kad_run(kad_graph *g, double eps, double delta, uint64_t seed, kad_stream_t stream,
                   const kad_options *opt, kad_result *out);

/* As kad_run, but the per-vertex outputs go to device arrays (either may be NULL):
   d_bc[n] (double) and d_counts[n] (uint32).  out->bc/counts/c0/ltab are ignored. */
kad_status kad_run_device(kad_graph *g, double eps, double delta, uint64_t seed, kad_stream_t stream,
                          const kad_options *opt, double *d_bc, uint32_t *d_counts, kad_result *out);

/*
 * kad_sample_records -- the per-sample view used by parity tests: samples
 * [i0, i0+count) of phase `domain` (0 or 1), computed by the same sampling
 * kernel.  Host outputs (each count entries unless noted): s, t, D (= d(s,t), 0
 * if disconnected), sigma_st (saturating), overflow (0/1), paths[count * cap]
 * (the D-1 interior vertices in order of distance from s, then -1 padding),
 * work[6] (as kad_result.work).  cap >= max(VD-2, 1).
 */
kad_status kad_sample_records(kad_graph *g, uint64_t seed, uint32_t domain, uint64_t i0, int64_t count,
                              kad_stream_t stream, const kad_options *opt, int32_t *s, int32_t *t, int32_t *D,
                              uint64_t *sigma_st, int32_t *overflow, int32_t *paths, int32_t cap, uint64_t *work);

/*
 * kad_sample_records_noalloc -- kad_sample_records for callers that may not
 * allocate device memory.  The paper has no counterpart to this entry point.
 *
 * Some callers own all device memory through their own pool (a framework's
 * caching allocator, a serving process held to a fixed memory budget) and cannot
 * let a library call cudaMalloc or cudaFree: those calls can synchronise the
 * device, stall the caller's other streams, and take memory the pool does not
 * account for.  This entry point allocates nothing.  The caller passes the graph
 * and every output as device pointers; the sampling kernel's scratch (labels,
 * path counts and labelled lists of up to 64 concurrent sampling slots, a
 * control block, work counters) lives in one fixed 48 MiB device array in the
 * library, which every GPU that loads the library holds until the process exits.
 *
 * Inputs (device): d_row_ptr[n+1], d_col[m], a symmetric sorted CSR as for
 * kad_graph_create (not validated here); d_comp[n] component labels (any value
 * equal within a component) or NULL, in which case pairs in different
 * components are found disconnected by the search itself (same records).
 * Outputs (device, count entries each): d_s, d_t, d_D, d_sigma_st, d_overflow
 * (0/1), and d_paths[count * cap] (interior vertices in order of distance from
 * s, -1 padding), exactly as kad_sample_records.
 * Limits: n <= 1,436,032 (the scratch holds at least one slot; smaller graphs
 * get up to 64 slots), count <= 1,048,576 per call; larger values return
 * KAD_ERR_INVALID_ARG before any device work.  A path longer than cap returns
 * KAD_ERR_INVALID_ARG.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, a host-side query).  Every call shares the one array and leaves it as
 * it was at its end: the call clears what must start at zero, but calls whose
 * work overlaps on the GPU (different streams or host threads) race on it --
 * serialise them.  Returns after synchronising `stream`.
 */
kad_status kad_sample_records_noalloc(int32_t n, const int32_t *d_row_ptr, const int32_t *d_col,
                                      const int32_t *d_comp, uint64_t seed, uint32_t domain, uint64_t i0,
                                      int64_t count, kad_stream_t stream, int32_t *d_s, int32_t *d_t, int32_t *d_D,
                                      uint64_t *d_sigma_st, uint8_t *d_overflow, int32_t *d_paths, int32_t cap);

/* ------------------------------------------------------------------ sharding
 * A KADABRA run whose samples are split among `world` ranks, one GPU each: the
 * distributed reduction of sampling states that Section 6 (conclusions and
 * future work) names as the next step, with the fixed sample-to-epoch
 * assignment of the indexed-frame algorithm (Appendix D.2).
 *
 * The calibration range [0, tau0) and every epoch's range [kN, (k+1)N) are
 * split into `world` contiguous chunks in rank order (kad_shard_range); rank r
 * computes the samples of its chunks.  After each phase every rank contributes
 * its chunk's path rows and receives all ranks' rows through `allgather`, then
 * folds all of them into its own counts on the device (integer addition, so the
 * order does not matter) and evaluates the stop rule (Appendix B) on the same
 * state as every other rank: all ranks stop at the same epoch, with the same
 * counts, tau and L table as kad_run on one GPU, bit for bit.
 *
 * allgather(user, send, bytes, recv): a collective the caller provides (NCCL,
 * MPI, gloo, ...).  send: host, `bytes` bytes; recv: host, world * bytes,
 * receiving rank q's send at offset q * bytes.  Every rank calls it the same
 * number of times with the same `bytes`.  Return 0 on success; anything else
 * ends the run with KAD_ERR_CANCELLED.
 * Outputs as kad_run (host pointers in *out); work counters and samples_computed
 * are this rank's own.  KAD_RUN_COMPLETION_ORDER is rejected
 * (KAD_ERR_INVALID_ARG).  Blocking; device work on `stream`.
 */
typedef int (*kad_allgather_fn)(void *user, const void *send, size_t bytes, void *recv);
kad_status kad_run_sharded(kad_graph *g, double eps, double delta, uint64_t seed, int32_t rank, int32_t world,
                           kad_allgather_fn allgather, void *user, kad_stream_t stream, const kad_options *opt,
                           kad_result *out);

/* The chunk [*lo, *hi) of `count` items that rank `rank` of `world` takes:
 * contiguous, in rank order, sizes differing by at most one.  Host only. */
void kad_shard_range(int64_t count, int32_t rank, int32_t world, int64_t *lo, int64_t *hi);

/*
 * kad_run_order -- after a KAD_RUN_COMPLETION_ORDER run on g: idx_out[q] = the
 * adaptive sample index (phase 0 of the random stream) that took fold position q,
 * for q < count.  Positions [0, tau) are the samples the run counted, in epochs
 * of N; later positions completed after the stop was decided.  Valid until the
 * next run on g; count <= samples_computed - calib_samples (every completed
 * adaptive sample took a position).  idx_out is host memory.  Errors:
 * KAD_ERR_INVALID_ARG (no such run, or count out of range), KAD_ERR_CUDA.
 */
kad_status kad_run_order(kad_graph *g, uint64_t *idx_out, uint64_t count);

/*
 * kad_eval_fg -- the stop-check kernel's f and g (Appendix B) for n vertices on
 * the device: f[v] = f(counts[v]/tau, exp(-ltab[c0[v]]), omega, tau), same for g.
 * All arrays host; ltab has nclass entries; every c0[v] < nclass.
 */
kad_status kad_eval_fg(int32_t n, const uint32_t *counts, const uint32_t *c0, const double *ltab, int32_t nclass,
                       uint64_t tau, uint64_t omega, double *f, double *g);

/* ------------------------------------------------------------------ serving
 * A query server keeps many graphs resident and answers KADABRA queries on them
 * concurrently: `workers` host threads each run one query at a time on their own
 * CUDA stream, so queries overlap on the device.  A query starts with
 * `slots_per_query` sampling blocks, or by default with the device's resident
 * blocks divided by the number of queries running or waiting at that moment (at
 * most `workers`): alone it gets the whole device, under load a share of it.  A submitted query waits until a worker is free and its device-memory
 * footprint (slot scratch + epoch ring + per-vertex arrays) fits the budget next
 * to the queries in flight; a smaller query may start before a larger one that
 * is still waiting for memory (continuous batching).  A query's result does not
 * depend on what else is running: it equals kad_run's on the same graph.
 * The paper has no serving layer; this is the batched-query use of its method.
 */
typedef struct kad_server kad_server;

typedef struct {
    int32_t workers;         /* queries in flight at once (0 = 4) */
    int32_t slots_per_query; /* sampling blocks per query (0 = adaptive share of the resident blocks) */
    int64_t hbm_budget;      /* bytes the footprints of in-flight queries may add up to (0 = half of the
                                device memory free at creation); a query larger than the budget runs alone */
    int32_t block_threads;   /* sampling-kernel variant for every query (0 = 512 threads, 2 blocks/SM) */
    int32_t blocks_per_sm;
    int32_t policy;          /* which fitting queued query starts next: 0 = highest response ratio
                                (waited + expected) / expected, expected = the query's omega + tau0
                                samples times the graph's measured device time per sample (short
                                queries first, long ones aged in); 1 = arrival order */
} kad_server_options;

/* Starts the worker threads on the current CUDA device.  opt NULL = defaults. */
kad_status kad_server_create(const kad_server_options *opt, kad_server **out);

/* Copies a graph to the server's device (as kad_graph_create; host arrays); *gid names it. */
kad_status kad_server_add_graph(kad_server *s, int32_t n, const int32_t *row_ptr, const int32_t *col, uint32_t flags,
                                int32_t *gid);

/* Queues a query.  bc_out (host, n doubles, or NULL) receives b~ when the query
   completes and must stay valid until kad_wait returns for the ticket. */
kad_status kad_submit(kad_server *s, int32_t gid, double eps, double delta, uint64_t seed, double *bc_out,
                      uint64_t *ticket);

/* *done = 1 once the query has finished (successfully or not). */
kad_status kad_poll(kad_server *s, uint64_t ticket, int *done);

/* Waits up to timeout_ns (< 0 = no limit) for the query; on completion fills *out
   (its bc pointer is ignored; see kad_submit), the time it waited for a worker and
   its submit-to-finish latency in milliseconds (either may be NULL), releases the
   ticket and returns the query's status.  KAD_ERR_TIMEOUT if it has not finished. */
kad_status kad_wait(kad_server *s, uint64_t ticket, int64_t timeout_ns, kad_result *out, double *queue_ms,
                    double *latency_ms);

/* Stops the workers after their current queries (queued ones end KAD_ERR_CANCELLED)
   and releases every graph and buffer.  NULL is a no-op. */
void kad_server_free(kad_server *s);

/* Human-readable text of a status. Never NULL. */
const char *kad_status_string(kad_status s);

/* Library version, (major << 16) | minor. */
uint32_t kad_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KAD_H */
