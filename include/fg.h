/*
 * fg.h -- C ABI of the buffered fork-processing engine (sm_103a).
 *
 * The fork-processing pattern (FPP) launches many independent single-source
 * queries on one graph (Alg. 1; Def. 2.2). This library runs a batch of such
 * queries -- exact integer SSSP, BFS levels, or forward-push Personalized
 * PageRank -- in the buffered style of Alg. 2: the graph is split into
 * partitions (Def. 2.1), every query's pending operations <q, v, val>
 * (Def. 2.3) are kept in per-(partition, query) buffers, and all buffered
 * work on a partition is processed while that partition's data is on chip.
 *
 * Conventions for every call:
 *   - Vertex ids are the caller's original ids in [0, n).
 *   - Outputs are query-major: row i (n entries) belongs to src[i].
 *   - Unless opts->host_io is set, src and every output are DEVICE pointers
 *     owned by the caller, and the call is asynchronous on `stream` (a
 *     cudaStream_t, NULL = the legacy default stream). Results are valid
 *     after fg_sync(stream) returns FG_OK.
 *   - Errors that the host can detect (null or misaligned pointers, bad
 *     sizes, source ids out of range, negative weights) are returned at once
 *     and nothing is enqueued. Errors found on the device (watchdog timeout,
 *     distance overflow, CUDA faults) are returned by fg_sync.
 *   - fg_last_error() gives a message for the last failing call on the
 *     calling thread.
 *   - Batches on one graph are serialised in stream order by the library
 *     (each batch waits for the previous batch on the same graph), because
 *     they share the graph's device workspace.
 */
#ifndef FG_H
#define FG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FG_OK = 0,
    FG_ERR_INVALID_ARG = 1,   /* bad argument, detected on the host; nothing enqueued */
    FG_ERR_OOM = 2,           /* device or host allocation failed / HBM budget exceeded */
    FG_ERR_CUDA = 3,          /* a CUDA call failed (message in fg_last_error) */
    FG_ERR_TIMEOUT = 4,       /* device watchdog: max_rounds or a barrier wait limit was hit */
    FG_ERR_BIN_OVERFLOW = 5,  /* operation buffers could not hold the work (not raised: ops spill losslessly) */
    FG_ERR_OVERFLOW = 6,      /* an SSSP distance reached 2^32 - 1 (saturated) */
    FG_ERR_UNSUPPORTED = 7    /* size beyond the supported range (e.g. m >= 2^32) */
} fg_status;

typedef struct fg_graph fg_graph;

/* fg_graph_create flags */
#define FG_DEVICE_PTRS 0x1u   /* row_ptr, col, w are device pointers (the library copies them) */

/* partitioners (Def. 2.1: a division of V into |P| disjoint vertex sets) */
enum {
    FG_PART_AUTO = 0,    /* GROW when the id order has little locality, else RANGE */
    FG_PART_RANGE = 1,   /* contiguous id ranges [i*S, (i+1)*S): the paper's equal-vertex split */
    FG_PART_GROW = 2,    /* breadth-first region growing to S vertices (stand-in for METIS) */
    FG_PART_DEGREE = 3   /* vertices by out-degree, highest first (hubs share partitions) */
};

typedef struct {
    uint32_t struct_size;        /* sizeof(fg_graph_opts) */
    int32_t partition_method;    /* FG_PART_* */
    int32_t partition_vertices;  /* S, a power of two in [32, 4096]; 0 = from the on-chip budget */
} fg_graph_opts;

/* inter-partition scheduling (Sec. 5.2; the four schedulers of Tab. 4A) */
enum { FG_SCHED_FIFO = 0, FG_SCHED_PRIORITY = 1, FG_SCHED_MAXOPS = 2, FG_SCHED_RANDOM = 3 };
/* execution form */
enum { FG_MODE_BUFFERED = 0, FG_MODE_PLAIN = 1 };

typedef struct {
    uint32_t struct_size;   /* sizeof(fg_opts); fields past it keep their defaults */
    int32_t mode;           /* FG_MODE_BUFFERED (default); FG_MODE_PLAIN runs one query at a
                               time with ordinary whole-graph frontier kernels (the baseline) */
    int32_t sched;          /* FG_SCHED_FIFO (default, Sec. 5.2): every round processes every
                               non-empty buffer; FG_SCHED_PRIORITY ("Shortest"): a query's
                               buffers whose best value lies within sched_window of that
                               query's best pending value; FG_SCHED_MAXOPS: buffers holding at
                               least a quarter of the round's largest buffer's operations;
                               FG_SCHED_RANDOM: a seeded coin per (buffer, round). Buffers left
                               out carry their work to the next round, where they are always
                               taken (no starvation). SSSP/BFS with one query per warp; PPR
                               and the group engine run FIFO rounds (the group engine with its
                               own window, see group) */
    uint32_t sched_window;  /* window of FG_SCHED_PRIORITY (SSSP/BFS value units); 0 = 8 * delta */
    uint32_t delta;         /* yield heuristic 2 (Sec. 5.1): within one visit a query processes
                               values below (first value + delta); the rest stays buffered.
                               0 = no limit */
    uint32_t bucket;        /* in-visit near/far width: values are relaxed in windows of this
                               width (Delta-stepping order inside a partition). 0 = none */
    uint64_t yield_edges;   /* yield heuristic 1 (Sec. 5.1): arcs one query may scan in one
                               visit before yielding. 0 = no limit */
    uint32_t max_rounds;    /* watchdog: rounds before FG_ERR_TIMEOUT. 0 = 1,000,000 */
    uint32_t watchdog_ms;   /* watchdog: longest wait at a device-wide barrier. 0 = 30,000 */
    uint64_t emit_capacity; /* operations one round may buffer (20 B each). Visits stop once 3/4
                               of it is reserved; beyond it, work spills to per-partition pending
                               bitmaps (lossless). 0 = automatic: 128 per (partition, query)
                               buffer, clamped to [2^22, 2^29] */
    int32_t host_io;        /* 1: src and outputs are HOST pointers; the call copies them and
                               completes before returning (fg_sync still reports status).
                               2: the same, asynchronous: the results are in the host buffers
                               once fg_sync(stream) returns; until then the buffers must stay
                               valid and unread. Each graph stages two such batches in turn,
                               so one batch's copy to the host overlaps the next batch's
                               kernels when they run on different streams */
    int32_t query_batch;    /* queries per device launch; 0 = all (bounded by workspace) */
    int32_t threads_per_vertex; /* SSSP/BFS expansion: 1 = one lane per frontier vertex (graphs
                               with out-degree <= 8 only), 32 or 0 (default) = a warp shares
                               a batch of 32 frontier vertices' arcs evenly */
    int32_t group;          /* SSSP/BFS queries that share one partition visit lane by lane
                               (the query group): 8, 16, 32 or 64 = the group engine, whose state
                               keeps a group's values of one vertex in one line, so one access
                               and one read of the arcs serve the whole group (best where almost
                               every arc leaves its partition: power-law graphs); 1 = one query
                               per warp and visit (best on road-like graphs, whose partitions
                               keep most arcs inside). 0 (default) = automatic: when more than
                               half of the graph's arcs cross partitions, 64 for SSSP (32 with a
                               sched_window) and 32 for BFS (a smaller batch takes the smallest
                               group that holds it), else 1. PPR
                               always runs one query per warp. In the group engine, sched_window
                               (SSSP) bounds each round to values below the group's smallest
                               pending value plus the window (groups of 8 to 32 only: a group of
                               64 with a window is FG_ERR_UNSUPPORTED); delta, bucket,
                               yield_edges, emit_capacity and threads_per_vertex do not apply */
    int32_t group_order;    /* group engine: 0 (default) = the batch's queries are ordered before
                               they are cut into groups, so that a group's queries reach the same
                               vertices in the same rounds and share more of each partition
                               visit: by the number of arcs within two hops of their source,
                               largest first, or, on graphs whose partitions keep most arcs
                               inside, by source position (results still go to the caller's rows;
                               batches of more than 65,536 queries keep their order);
                               1 = groups follow the order of src */
    int32_t check_staging;  /* group engine self-test: 1 = after each shared-memory staging wait,
                               compare every staged row offset and pending mask with global
                               memory and report FG_ERR_CUDA (site: staged words differ) on a
                               mismatch; 0 (default) = off */
} fg_opts;

/* counters of the last completed batch on a graph (read by fg_stats after fg_sync) */
typedef struct {
    uint64_t rounds;        /* Alg. 2 loop iterations (sum over launches) */
    uint64_t visits;        /* (partition, query) buffers processed; group engine: (partition,
                               group) items and hub chunks */
    uint64_t edges;         /* arcs scanned by the relax/push kernels, counted per query (a
                               group engine arc counts once per lane it relaxes) */
    uint64_t ops;           /* operations buffered; group engine: target values lowered */
    uint64_t spills;        /* expansions deferred because the op arena was full */
    uint64_t yields;        /* visits that left work behind (yield or budget) */
    uint64_t launches;      /* kernels launched by the batch */
    uint64_t max_round_ops; /* most operations buffered in one round */
    uint64_t phase_ns[6];   /* device time per phase, summed over rounds, between device-wide
                               barriers: tile init, seeding, scan A, scan B (scheduling),
                               scatter into bins, intra-partition processing (the group engine
                               uses tile init, seeding, scan (in slot 2) and processing) */
    uint64_t arcs_read;     /* arcs read from the graph: per (arc, query) visit with one query
                               per warp, per (arc, group) with the group engine, where one read
                               serves every lane of the group */
    uint64_t group;         /* queries per group of the last launch (1 = one query per warp) */
} fg_stats_t;

typedef struct {
    int64_t n, m;
    int32_t partition_vertices;  /* S */
    int32_t num_partitions;      /* |P| */
    int32_t partition_method;    /* FG_PART_RANGE, FG_PART_GROW or FG_PART_DEGREE (after AUTO) */
    int32_t weighted;
    int64_t cut_arcs;            /* arcs whose endpoints lie in different partitions */
    int64_t device_bytes;        /* graph bytes resident on the device */
} fg_graph_info_t;

/* Fill *o with the defaults. */
void fg_default_opts(fg_opts *o);
void fg_default_graph_opts(fg_graph_opts *o);

/*
 * Build a device graph from CSR (Ligra-style storage, Sec. 3.1): row_ptr has
 * n + 1 entries (row_ptr[0] = 0, non-decreasing, row_ptr[n] = m), col has m
 * vertex ids in [0, n), w has m int32 weights >= 0 or is NULL (unit weights).
 * Undirected graphs store both arcs of every edge (Sec. 2.1). The caller's
 * arrays are copied; the caller keeps ownership. Requires 1 <= n < 2^31 and
 * m < 2^32. Partitions the vertices (Def. 2.1) and stores the graph
 * partition-major on the device. Synchronous. *out receives the handle.
 */
fg_status fg_graph_create(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                          const int32_t *w, uint32_t flags, fg_graph **out);

/* As fg_graph_create, with partitioning options (NULL = defaults). */
fg_status fg_graph_create_ex(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                             const int32_t *w, uint32_t flags, const fg_graph_opts *gopts,
                             fg_graph **out);

/* Release a graph and its workspace. Waits for its batches to finish. NULL is allowed. */
fg_status fg_graph_destroy(fg_graph *g);

/* Sizes and partition facts of a graph. */
fg_status fg_graph_info(const fg_graph *g, fg_graph_info_t *info);

/*
 * nq single-source shortest-path queries (Def. 2.3: an operation <q, v, l>
 * lowers v's path length to l when l is shorter). dist_out: uint32[nq * n],
 * exact distances; UINT32_MAX = unreachable. src: int32[nq] (duplicates are
 * allowed). Unweighted graphs use weight 1.
 */
fg_status fg_sssp_batch(fg_graph *g, const int32_t *src, int32_t nq, uint32_t *dist_out,
                        void *stream, const fg_opts *opts);

/* nq BFS queries: level_out uint32[nq * n], hop levels; UINT32_MAX = unreachable. */
fg_status fg_bfs_batch(fg_graph *g, const int32_t *src, int32_t nq, uint32_t *level_out,
                       void *stream, const fg_opts *opts);

/*
 * nq Personalized PageRank queries by forward push (non-lazy rule): a vertex
 * v with residual r(v) >= eps * max(deg(v), 1) moves alpha * r(v) into its
 * estimate and spreads (1 - alpha) * r(v) / deg(v) to each out-neighbour
 * (a dangling vertex returns (1 - alpha) * r(v) to the source); r(v) = 0.
 * Estimates are FP32 with compensated (Kahan) accumulation; residuals FP32.
 * p_out float[nq * n] (required), r_out float[nq * n] (may be NULL),
 * mass_out double[nq] (may be NULL): sum(p) + sum(r) per query in FP64.
 * Requires 0 < alpha < 1 and eps > 0.
 */
fg_status fg_ppr_batch(fg_graph *g, const int32_t *src, int32_t nq, float alpha, float eps,
                       float *p_out, float *r_out, double *mass_out, void *stream,
                       const fg_opts *opts);

/* Wait for the work enqueued on `stream`; return the first device-side error of its batches. */
fg_status fg_sync(void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *fg_last_error(void);

/* Counters of the last batch on g that fg_sync has completed. */
fg_status fg_stats(const fg_graph *g, fg_stats_t *out);

/*
 * Host-only partitioner, exposed for inspection: writes perm[i] = original id
 * of internal vertex i (partition j holds internal ids [j*S, (j+1)*S)).
 * Makes no CUDA call. method is FG_PART_RANGE, FG_PART_GROW or FG_PART_DEGREE.
 */
fg_status fg_partition_plan(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t method,
                            int32_t partition_vertices, int32_t *perm);

/* query kinds of the autotuner and the serving loop */
enum { FG_QUERY_SSSP = 0, FG_QUERY_BFS = 1, FG_QUERY_PPR = 2 };

/*
 * Autotuner. The paper tunes its scheduling and yield parameters by hand per
 * graph (Sec. 5, Tab. 4); here the host times candidate fg_opts for one query
 * kind (FG_QUERY_*, declared below) on a sample batch and writes the fastest
 * to *best: the default; for SSSP and BFS the query group (1, 16, 32 or 64; see
 * fg_opts.group); then, with one query per warp, FG_SCHED_PRIORITY windows from
 * wide to narrow -- multiples of the graph's mean arc weight for SSSP, levels
 * for BFS -- until one takes more than twice the best time, delta (yield
 * heuristic 2) of half and a quarter of the best window, and on graphs with
 * out-degree <= 8 lane-per-vertex expansion; with the group engine, SSSP
 * windows of 16 and 4 mean weights; last, for every kind with nq >= 64, half
 * the batch per launch (query_batch). PPR keeps FIFO scheduling. best->group
 * is never 0: the automatic choice is resolved. The partition size is a graph
 * property: compare graphs created with different partition_vertices. src: DEVICE int32[nq] (the sample; a few hundred sources is
 * typical). The tuner allocates nq * n * 4 B of output rows for the duration
 * of the call and runs each candidate once on `stream` (it synchronises).
 * report (nullable) receives the number of candidates and the default's and
 * the chosen schedule's batch times. The choice is cached in the graph per
 * (kind, batch size rounded up to a power of two): a later call with the same
 * key returns it without timing anything (report->candidates = 0).
 */
typedef struct {
    int32_t candidates;
    float best_ms;
    float default_ms;
} fg_tune_report;

fg_status fg_tune_opts(fg_graph *g, int32_t kind, const int32_t *src, int32_t nq, void *stream,
                       fg_opts *best, fg_tune_report *report);

/*
 * As fg_tune_opts, with the PPR parameters the caller will use (fg_tune_opts
 * times PPR candidates at alpha = 0.15, eps = 1e-6). For PPR the choice is
 * cached per (batch-size bucket, alpha, eps). alpha and eps are ignored for
 * SSSP and BFS. Requires 0 < alpha < 1 and eps > 0 for PPR.
 */
fg_status fg_tune_opts_ex(fg_graph *g, int32_t kind, const int32_t *src, int32_t nq, float alpha, float eps,
                          void *stream, fg_opts *best, fg_tune_report *report);

/*
 * Serving loop (continuous batching). Requests -- one SSSP, BFS or PPR query
 * from one source -- are submitted one at a time; fg_server_poll launches
 * the waiting requests of one kind as a batch on every free lane and reports
 * requests whose batch has completed. Each lane has its own stream, engine
 * workspace and output rows, and by default launches on 1/lanes of the GPU's
 * resident grid, so batches of different kinds and ages run on the device at
 * once. A lane is free again when every request of its batch has been
 * released. The server's device memory is fixed at creation: lanes *
 * max_batch output rows plus each lane's engine workspace, with max_batch
 * lowered if needed so that a full batch of every lane fits hbm_budget
 * (admission by HBM budget). Results are bit-identical to fg_sssp_batch /
 * fg_bfs_batch for the same source; PPR results meet the same bound as
 * fg_ppr_batch. The graph must outlive the server. Calls on one server are
 * serialised by the server's lock; fg_server_submit may be called from any
 * thread.
 *
 * Slot-level batching (continuous = 1): SSSP and BFS requests no longer wait
 * for a batch. Each of the two kinds has `slots` query lanes of the group
 * engine with their own state and result rows, and a mailbox in mapped host
 * memory. fg_server_poll writes a waiting request into a free slot; a running
 * launch admits it at its next round boundary, runs it alongside the queries
 * already in flight, and posts its completion as soon as that query has no
 * pending work left, whatever the other lanes are doing. A launch ends when
 * it holds no query and finds no new request; fg_server_poll starts one when a
 * slot holds a request. A slot is free again when its request is released.
 * The two slot lanes take half of hbm_budget (slots lowered to fit); PPR
 * requests still run in batches on the lanes, and the resident grid is
 * shared by lanes + 2 launches unless full_grid. The same results as batch
 * mode; batch_size reports the kind's slot count.
 */
typedef struct fg_server fg_server;

typedef struct {
    uint32_t struct_size;   /* sizeof(fg_server_opts) */
    int32_t lanes;          /* batches in flight at once, 1..64 (default 4) */
    int32_t max_batch;      /* requests per batch (default 256; lowered to fit hbm_budget) */
    int32_t full_grid;      /* 1: every batch launches on the whole resident grid; 0 (default): 1/lanes of it */
    float alpha, eps;       /* PPR parameters of every PPR request (default 0.15, 1e-6) */
    int64_t hbm_budget;     /* device bytes for all lanes' batches; 0 (default) = 60% of free memory */
    fg_opts opts[3];        /* engine options per kind (SSSP, BFS, PPR); struct_size 0 = defaults */
    int32_t continuous;     /* 1: slot-level batching of SSSP and BFS (below); 0 (default): batches on lanes */
    int32_t slots;          /* continuous: query slots per kind, a multiple of the group size (opts[0].group if
                               8, 16 or 32, else 32); default 128, lowered to fit half of hbm_budget */
} fg_server_opts;

typedef struct {
    int32_t kind;           /* FG_QUERY_* */
    int32_t source;         /* original vertex id */
    int32_t status;         /* -1 while pending or running, else the fg_status of its batch */
    int32_t batch_size;     /* requests in its batch */
    int64_t submit_ns, launch_ns, done_ns;  /* host steady clock; done = completion seen by fg_server_poll */
    const void *result;     /* DEVICE row, original order: uint32[n] (SSSP/BFS, UINT32_MAX = unreachable)
                               or float[n] PPR estimates; valid from completion until release */
    const float *residual;  /* DEVICE float[n] PPR residuals, else NULL */
    double mass;            /* PPR: sum(p) + sum(r) in FP64; else 0 */
} fg_request_info;

void fg_default_server_opts(fg_server_opts *o);
fg_status fg_server_create(fg_graph *g, const fg_server_opts *o, fg_server **out);
/* Waits for the lanes' work in flight, then frees everything (outstanding results become invalid). */
fg_status fg_server_destroy(fg_server *s);
/* Queues one request; *id identifies it until fg_server_release. Bad kind or source: FG_ERR_INVALID_ARG. */
fg_status fg_server_submit(fg_server *s, int32_t kind, int32_t source, uint64_t *id);
/*
 * Non-blocking progress step: collects completed batches, launches waiting
 * requests on free lanes, and writes up to cap completed request ids to done
 * (*n_done of them; the rest are reported by later polls). Returns the first
 * error of a batch seen in this call (its requests carry it in status).
 */
fg_status fg_server_poll(fg_server *s, uint64_t *done, int32_t cap, int32_t *n_done);
fg_status fg_server_info(fg_server *s, uint64_t id, fg_request_info *info);
/* Frees a completed request's result row; its lane is reused once its whole batch is released. */
fg_status fg_server_release(fg_server *s, uint64_t id);

/*
 * SSSP without any allocation. The paper has no counterpart: this is a
 * service for callers that must not allocate once running (device memory
 * fixed up front by another pool, or independent work on other streams that
 * must not be stalled by the device-wide synchronisation of cudaFree).
 *
 * Computes the same exact distances as fg_sssp_batch (dist_out uint32[nq * n],
 * original vertex order, UINT32_MAX = unreachable), one query after another
 * with the plain per-query kernel, on scratch compiled into the library: one
 * 16 MiB + 512 B array of device memory per device, so the graph may have at
 * most FG_NOALLOC_MAX_VERTICES vertices; a larger graph is rejected with
 * FG_ERR_UNSUPPORTED before anything is enqueued. src (int32[nq]) and
 * dist_out are DEVICE pointers owned by the caller, on the graph's device,
 * which must be the current device. The call makes no cudaMalloc, cudaFree or
 * host allocation, takes no fg_opts, and does not update fg_stats.
 *
 * Set-up: fg_graph_create, on the graph's device, places the scratch array in
 * device memory (with lazy module loading that happens when its address is
 * first looked up, with cudaGetSymbolAddress), loads the plain kernel and
 * sizes its cooperative grid. So the scratch is taken while the device's
 * memory is still free, and a later fg_sssp_batch_noalloc call adds no device
 * memory. If that set-up failed, the first call on the device retries it.
 * Each call clears the scratch's control block (a memset on `stream`) before
 * its first launch; nothing else needs to start at zero.
 *
 * The call is synchronous: it enqueues its work on `stream`, waits for the
 * stream, and returns device-side errors (source id out of range, distance
 * overflow, watchdog timeout) as its result. Host-detected errors (NULL or
 * misaligned pointers, nq <= 0, wrong current device, too many vertices) are
 * returned before anything is enqueued.
 *
 * All calls on one device share the one scratch array: two calls that
 * overlap in time on the same device (from two host threads) race, and their
 * results are undefined. The caller serialises them.
 */
#define FG_NOALLOC_MAX_VERTICES (1 << 20)
fg_status fg_sssp_batch_noalloc(const fg_graph *g, const int32_t *src, int32_t nq, uint32_t *dist_out,
                                void *stream);

/*
 * Sweep cuts over PPR vectors: the conductance step of the network community
 * profile (NCP) application, which runs PPRs from randomly chosen seed
 * vertices and keeps, for each cluster size, the best conductance found
 * (Sec. 1; Sec. 6.1 seeds 0.01% of the vertices).
 *
 * For each query q (row q of p, as fg_ppr_batch writes it: float[nq * n],
 * original vertex order) the vertices with p(v) > 0 are ordered by the FP32
 * key p(v) / max(d(v), 1), largest first, ties by smaller id; d = out-degree.
 * For each prefix S_k (k = 1 .. count) of the first `top` vertices:
 *   phi(S_k) = cut(S_k) / min(vol(S_k), vol(V) - vol(S_k))  (FP64; 1.0 when
 *   that minimum is 0), vol = sum of out-degrees (vol(V) = m), cut = arcs from
 *   S_k to the rest, computed as sum over v in S_k of d(v) - 2 * (arcs from v
 *   to vertices placed before v), exact for a graph stored with both arcs of
 *   every edge; on a directed graph the same formula is evaluated.
 *
 * Outputs (DEVICE pointers owned by the caller; any may be NULL, not all):
 *   order_out  int32[nq * top]: order_out[q * top + k] = the (k+1)-th vertex
 *              (original id); -1 past count
 *   phi_out    double[nq * top]: phi(S_{k+1}); NaN past count
 *   count_out  int32[nq]: min(top, number of vertices with p(v) > 0)
 *   ncp_out    double[top]: ncp_out[k] = min over this call's queries of
 *              phi(S_{k+1}), +inf where no query has k+1 vertices; with
 *              accumulate != 0 the minimum also takes the values already in
 *              ncp_out (profile over several calls).
 * Requires 1 <= top <= FG_NCP_MAX_TOP and nq >= 1; p 4-byte aligned, phi_out
 * and ncp_out 8-byte aligned; the graph's device must be current.
 *
 * Asynchronous on `stream`, with one exception: the first call on a graph
 * builds the graph's table of out-degrees by original id (4 * n bytes, freed
 * with the graph) and waits for it. Errors are detected on the host only.
 */
#define FG_NCP_MAX_TOP 4096
fg_status fg_ncp_sweep(fg_graph *g, const float *p, int32_t nq, int32_t top, int32_t *order_out,
                       double *phi_out, int32_t *count_out, double *ncp_out, int32_t accumulate, void *stream);

/*
 * Landmark labeling (LL): a batch of SSSP (or BFS) queries from landmark
 * vertices s_0 .. s_{K-1} gives every vertex a label of K distances, and a
 * pair of vertices is answered from their two labels alone (Sec. 1; Sec. 6.1
 * runs 1,024 SSSPs from randomly chosen landmarks).
 *
 * fg_ll_build_labels: label construction. dist: the batch's output,
 * uint32[K * n] query-major (row k = d(s_k, .), UINT32_MAX = unreachable);
 * labels: uint32[n * K] vertex-major, labels[v * K + k] = d(s_k, v). Both are
 * DEVICE pointers owned by the caller, 4-byte aligned, not overlapping. The
 * copy is asynchronous on `stream`; host-detected errors only.
 */
fg_status fg_ll_build_labels(const uint32_t *dist, int32_t K, int64_t n, uint32_t *labels, void *stream);

/*
 * fg_ll_query: distance estimates for Q vertex pairs. labels: uint32[n * K]
 * as above; pairs: int32[2 * Q] (u, v); est_out: uint64[Q],
 *   est_out[i] = min over k with labels[u][k], labels[v][k] both finite of
 *                labels[u][k] + labels[v][k]   (exact in 64 bits),
 * UINT64_MAX when no landmark reaches both, and for a pair with a vertex id
 * outside [0, n). On an undirected graph the estimate is an upper bound on
 * d(u, v), exact when some landmark lies on a shortest u-v path (in particular
 * when u or v is a landmark). DEVICE pointers owned by the caller (labels and
 * pairs 4-byte, est_out 8-byte aligned; K a multiple of 4 with 16-byte aligned
 * labels takes 16-byte loads). Q = 0 is a no-op. Asynchronous on `stream`.
 */
fg_status fg_ll_query(const uint32_t *labels, int64_t n, int32_t K, const int32_t *pairs, int64_t Q,
                      uint64_t *est_out, void *stream);

/*
 * Betweenness centrality from sampled sources (BC): one SSSP (weighted graph)
 * or BFS (unweighted graph) per sampled source, then the dependency
 * accumulation of Brandes (Sec. 1; Sec. 6.1 samples 100 sources).
 *
 * dist: the batch's exact rows, uint32[nq * n] in original vertex order, as
 * fg_sssp_batch (weighted = 1) or fg_bfs_batch (weighted = 0) wrote them for
 * the sources src (int32[nq]); an arc (u, w) of weight wt (1 when weighted = 0)
 * is on a shortest path from s when d_s(u) + wt = d_s(w). For every source:
 *   sigma_s(w) = number of shortest s-w paths (sigma_s(s) = 1),
 *   delta_s(u) = sum over u's tight out-arcs (u, w), in the order the graph
 *                lists them, of sigma_s(u) / sigma_s(w) * (1 + delta_s(w)),
 * each FP64 operation rounded as written. Then, for every vertex v,
 *   bc[v] = (accumulate ? bc[v] : 0) + sum over q in order, src[q] != v, of delta_{src[q]}(v).
 * Sampled BC is usually scaled by n / nq; that is left to the caller.
 *
 * Requirements: weighted = 1 needs a weighted graph with positive weights
 * (FG_ERR_UNSUPPORTED otherwise: a weight-0 arc would tie vertices at equal
 * distance); nq * n < 2^32 (split larger batches; scratch of about 32 * nq * n
 * bytes is kept with the graph). Graphs whose largest out-degree is at most 64
 * run one block per source, others one cooperative launch for the batch; the
 * results are the same. src, dist and bc (double[n]) are DEVICE pointers
 * owned by the caller. Each dist row must start at its source (d = 0 there):
 * otherwise FG_ERR_INVALID_ARG (detected on the device).
 *
 * info (host, nullable): waves = the longest shortest-path hop count over the
 * batch plus one; sigma_max = the largest path count; inexact = 1 when a path
 * count reached 2^53, beyond which FP64 sums of counts may round (the result
 * is then no longer independent of the order of the atomic additions).
 *
 * Synchronous: enqueues on `stream` (after the batch that wrote dist, if it
 * ran on the same stream), waits, and returns the device status.
 */
typedef struct {
    int32_t waves;
    int32_t inexact;
    double sigma_max;
} fg_bc_info_t;
fg_status fg_bc_accumulate(fg_graph *g, const int32_t *src, int32_t nq, const uint32_t *dist, int32_t weighted,
                           double *bc, int32_t accumulate, fg_bc_info_t *info, void *stream);

/*
 * Random-walk queries (RW, one of the framework's query types next to BFS,
 * SSSP, PPR and DFS; Sec. 3). Walk q starts at src[q] and takes `length`
 * steps: from vertex u it moves to the (r mod d(u))-th out-neighbour of u,
 * counting u's arcs in the order the graph was given, where r is output
 * number 2^32 * q + t + 1 (t = 0 .. length - 1 the step) of a SplitMix64
 * stream whose state starts at `seed` (Steele, Lea, Flood 2014: the state
 * advances by 0x9E3779B97F4A7C15 per output, which is mixed with shifts 30,
 * 27, 31 and multipliers 0xBF58476D1CE4E5B9, 0x94D049BB133111EB). A vertex
 * without out-arcs ends the walk.
 *
 * paths_out: int32[nq * (length + 1)] walk-major, paths_out[q * (length + 1) + t]
 * = the vertex after t steps (t = 0: src[q]), -1 once the walk has ended or
 * for a source id outside [0, n). src and paths_out are DEVICE pointers owned
 * by the caller. Asynchronous on `stream`; host-detected errors only.
 */
fg_status fg_rw_batch(const fg_graph *g, const int32_t *src, int32_t nq, int32_t length, uint64_t seed,
                      int32_t *paths_out, void *stream);

/*
 * Depth-first search queries (DFS, one of the framework's query types; Sec. 3):
 * query q is the recursive preorder from src[q], visiting out-neighbours in
 * the order the graph lists them. disc_out: uint32[nq * n], original vertex
 * order, disc_out[q * n + v] = the rank at which v is discovered (0 for the
 * source), UINT32_MAX = not reached. src and disc_out are DEVICE pointers
 * owned by the caller. Scratch of about 8.125 * nq * n bytes (12.125 * nq * n
 * on a relabelled graph) is kept with the graph. Synchronous: enqueues on `stream`,
 * waits, and returns FG_ERR_INVALID_ARG when a source id is outside [0, n)
 * (that query's row is left all UINT32_MAX).
 */
fg_status fg_dfs_batch(fg_graph *g, const int32_t *src, int32_t nq, uint32_t *disc_out, void *stream);

/*
 * Personalized PageRank with sparse per-query state, for local queries: the
 * push rule of fg_ppr_batch (same alpha, eps, dangling and compensation
 * rules; synchronous rounds), but each query keeps only the vertices it
 * touches, in an open-addressing table of `cap` slots (a power of two in
 * [64, 2^24]), so a batch needs about 24 * nq * cap bytes of scratch (from
 * the stream-ordered allocator) instead of 12 * nq * n.
 *
 * Outputs (DEVICE pointers owned by the caller): vert_out int32[nq * cap] and
 * p_out float[nq * cap] hold, in the first count_out[q] entries of row q, the
 * vertices with p(v) > 0 (original ids, in no particular order) and their
 * estimates; every other vertex has p(v) = 0. count_out[q] = -1 when the
 * query touched more than 3/4 of `cap` vertices (its row is then not valid:
 * retry with a larger cap or use fg_ppr_batch). mass_out double[nq]
 * (nullable) = sum(p) + sum(r) of the query in FP64.
 *
 * Requires 0 < alpha < 1 and eps > 0. Synchronous: enqueues on `stream`,
 * waits, returns FG_ERR_INVALID_ARG for a source id outside [0, n) (that
 * query's count is 0).
 */
fg_status fg_ppr_local_batch(const fg_graph *g, const int32_t *src, int32_t nq, float alpha, float eps, int32_t cap,
                             int32_t *vert_out, float *p_out, int32_t *count_out, double *mass_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FG_H */
