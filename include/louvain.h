/*
 * louvain.h — C ABI of the GB300 (sm_103a) Louvain community-detection engine.
 *
 * The engine runs the data-parallel hot path of the Louvain method as the
 * paper describes it (Sahu, "Enhancing Efficiency in Parallel Louvain
 * Algorithm for Community Detection", Section 3.2): the local-moving phase,
 * where every vertex moves to the neighbouring community of greatest
 * modularity gain, repeated while an iteration's total gain exceeds
 * `tolerance`; the aggregation phase, which collapses each community into a
 * super-vertex (inter-community edges merged with summed weights, intra-
 * community edges into a summed self-loop); passes of the two phases until the
 * pass gain is <= `pass_tolerance`; threshold scaling (tolerance 0.01 divided
 * by the decline factor 10 after every pass); synchronous (Jacobi) and
 * asynchronous (Gauss-Seidel) variants.  The result is the top level of the
 * dendrogram and its modularity.
 *
 * Modularity (Newman-Girvan, resolution 1; the paper states no formula) in
 * this CSR convention: an undirected edge {u,v}, u != v, is stored as (u,v) and
 * (v,u) with equal weight; a self-loop once.  K_i = row sum, M = sum K_i,
 * Sigma_c = sum of K_i over c, L_c = sum of entries inside c,
 * Q = (M sum L_c - sum Sigma_c^2) / M^2.  All gains and sums are exact
 * integers (128-bit where needed); Q is the correctly rounded quotient of the
 * exact numerator and M^2 as doubles.
 *
 * Conventions for every function below:
 *   - return 0 on success or a negative LOUVAIN_ERR_* code; the message of
 *     the last error of a context is louvain_last_error(ctx);
 *   - pointers whose kind is given by a `louvain_ptr_kind` argument are host
 *     or device (cuda:device of the context) memory of that kind;
 *   - the engine copies every input: the caller keeps ownership of its
 *     buffers and may free them once the call returns;
 *   - outputs go to caller-owned buffers of the stated length;
 *   - a context is not thread-safe; several contexts may share one device;
 *   - all device work is ordered on the context's stream; calls that return
 *     results synchronise that stream.
 */
#ifndef GB_LOUVAIN_H
#define GB_LOUVAIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ errors */
#define LOUVAIN_OK 0
#define LOUVAIN_ERR_INVALID_ARG (-1)   /* null pointer, negative size, bad option */
#define LOUVAIN_ERR_NOT_SYMMETRIC (-2) /* some (u,v,w) has no (v,u,w) */
#define LOUVAIN_ERR_BAD_CSR (-3)       /* offsets not monotone / col out of range / weight <= 0 */
#define LOUVAIN_ERR_OOM (-4)           /* device allocation failed */
#define LOUVAIN_ERR_CUDA (-5)          /* a CUDA runtime call or kernel failed */
#define LOUVAIN_ERR_TIMEOUT (-6)       /* a bounded device-side wait ran out */
#define LOUVAIN_ERR_STATE (-7)         /* e.g. run before load, result before run */
#define LOUVAIN_ERR_OVERFLOW (-8)      /* total weight M >= 2^62 or n >= 2^31 */
#define LOUVAIN_ERR_INTERNAL (-9)      /* a device-side consistency check failed */
#define LOUVAIN_ERR_CAPACITY (-10)     /* a size above a fixed capacity (louvain_modularity_static) */

/* Vertex capacity of louvain_modularity_static's fixed scratch. */
#define LOUVAIN_STATIC_MAX_VERTICES (1 << 20)

typedef enum { LOUVAIN_SYNC = 0, LOUVAIN_ASYNC = 1 } louvain_mode;
typedef enum { LOUVAIN_PTR_HOST = 0, LOUVAIN_PTR_DEVICE = 1 } louvain_ptr_kind;

/* Run options.  Defaults (louvain_default_options) are the paper's:
 * tolerance 0.01, decline factor 10, pass tolerance 0 (Section 3.2), with
 * 20 iterations per pass and 10 passes at most. */
typedef struct {
  int32_t mode;               /* louvain_mode */
  double tolerance;           /* an iteration ends the phase when its total gain 2S/M^2 <= tolerance */
  double tolerance_decline;   /* tolerance is divided by this after every pass (threshold scaling) */
  double pass_tolerance;      /* the run ends after a pass whose modularity gain is <= this */
  int32_t max_iterations;     /* local-moving iterations per pass (>= 1) */
  int32_t max_passes;         /* passes (>= 0, <= 64) */
  int32_t prune;              /* 1: after the first iteration of a pass, only vertices that moved or
                                 have a neighbour that moved in the previous iteration are visited */
  int32_t singleton_guard;    /* 1: a vertex alone in its community does not move to another
                                 single-vertex community of higher id (minimum-label rule, Grappolo;
                                 stops Jacobi updates from swapping pairs forever) */
  int32_t subrounds;          /* P >= 1: the vertices are split into P classes processed one after
                                 the other in each iteration; 1 = every vertex at once; 0 = automatic
                                 (synchronous 1; asynchronous, per graph: 32 for a graph of fewer than
                                 65,536 vertices, else 8 for a graph of fewer than 8 entries per vertex,
                                 else 16) */
  int32_t validate;           /* 1: louvain_load_csr checks symmetry and CSR form (costs a pass) */
  int32_t record_levels;      /* 1: keep each pass's membership and coarse CSR for louvain_get_level /
                                 louvain_get_coarse (copies them to host memory) */
  int32_t cuda_graphs;        /* 1: from the third iteration of a pass, replay that pass's iteration
                                 as one captured CUDA graph instead of individual launches (default 0:
                                 measured slower on the benchmark graphs) */
  int32_t reclass;            /* asynchronous mode with P > 1: 0 = classes id mod P; 1 = each
                                 iteration draws the classes anew, class = hash(id, pass, iteration)
                                 mod P (breaks the repeated same-class swaps of structured ids such
                                 as grids); 2 = hashed classes drawn once per pass; 3 = automatic
                                 (default; per graph: 2 for a graph of fewer than 65,536 vertices,
                                 else 1).  Synchronous classes are always id mod P.  Every graph of
                                 a batch gets the schedule it gets alone. */
  int32_t bucket_streams;     /* asynchronous mode: 1 (default) = every degree bucket (thread, warp,
                                 block and hub kernels) runs the iteration's classes in order on its
                                 own stream, without waiting for the other buckets' previous class
                                 (the streams' priorities rise with the bucket's degree range, so the
                                 blocks of high-degree vertices are scheduled first); 0 = a class
                                 starts when every bucket has finished the previous one.
                                 Synchronous classes always wait (Jacobi per class). */
  int32_t colour_classes;     /* 1: the classes of every pass are a greedy colouring of the pass graph
                                 instead of subrounds / reclass (Section 2's coarse-grained form: a set
                                 of vertices processed in parallel, as in the Grappolo heuristics the
                                 paper cites; here no two neighbours share a class).  Vertex priority
                                 lowbias32(local id XOR 0x9E3779B9 * (pass + 1)), higher first, ties to
                                 the lower id; in priority order each vertex takes the smallest class in
                                 0..62 that no preceding neighbour holds, else 63.  The pass has (largest
                                 class + 1) classes.  Synchronous: deterministic, equal to the oracle's
                                 colour-class mode.  0 (default): subrounds / reclass */
  int32_t stop_rule;          /* what an iteration's "total change in modularity" (Section 3.2) is:
                                 0 (default) = 2S/M^2, S the sum of the gains of its moves (exactly the
                                 change in sequential order); 1 = the exact change of the Q numerator over
                                 the iteration, recomputed from the membership after it (costs one scan of
                                 the pass graph per iteration), / M^2.  The two differ in synchronous
                                 order, where decisions taken together overlap */
  double reserved_d[4];
} louvain_options;

/* Per-run statistics. */
typedef struct {
  int32_t passes;             /* passes whose local-moving phase ran */
  int32_t iterations;         /* local-moving iterations over all passes */
  int64_t moves;              /* vertex moves over all iterations */
  int64_t lm_edges;           /* CSR entries scanned by local-moving (vertices visited x degree) */
  int64_t communities;        /* communities in the final membership */
  double q;                   /* final modularity */
  double lm_ms;               /* device time of local-moving kernels (CUDA events) */
  double agg_ms;              /* device time of renumbering + aggregation */
  double other_ms;            /* pass set-up, modularity, bucketing */
  double total_ms;            /* device time of louvain_run */
  int64_t lm_vertices;        /* vertices visited by local-moving */
  int64_t lm_bytes;           /* algorithmic bytes of local-moving: 8 + sizeof(weight) per scanned entry
                                 (column, weight, neighbour membership), 32 per visited vertex, 8 per
                                 distinct candidate community (its total) and 16 per move (two totals) */
  int64_t kernel_launches;    /* kernels the run launched */
  int64_t lm_candidates;      /* distinct candidate communities evaluated by local-moving */
  int64_t reserved[4];
} louvain_stats;

/* Per-pass record. */
typedef struct {
  int64_t n, nnz;             /* vertices and CSR entries of the pass graph */
  int64_t k;                  /* communities after the pass (its level's size) */
  int64_t moves;
  int32_t iterations;
  int32_t level_recorded;     /* louvain_get_level available for this pass */
  int32_t coarse_built;       /* aggregation ran after this pass (another pass followed) */
  int32_t pad;
  int64_t coarse_nnz;         /* entries of the coarse CSR built from this pass */
  int64_t n_before_hi;        /* exact Q numerator before the pass, as hi * 2^64 + lo */
  uint64_t n_before_lo;
  int64_t n_after_hi;         /* exact Q numerator after the pass's local-moving */
  uint64_t n_after_lo;
  double lm_ms, agg_ms;
} louvain_pass_info;

typedef struct louvain_ctx louvain_ctx;

/* Fill *opt with the defaults above. */
int louvain_default_options(louvain_options *opt);

/* Create a context on CUDA device `device` using CUDA stream `cuda_stream`
 * (a cudaStream_t; NULL = the context creates and owns a non-blocking
 * stream).  `opt` is copied; NULL = defaults. */
int louvain_create(louvain_ctx **out, const louvain_options *opt, int device, void *cuda_stream);

/* Replace the options of a context (takes effect at the next run). */
int louvain_set_options(louvain_ctx *ctx, const louvain_options *opt);

/* Load a graph: n vertices, nnz CSR entries; offsets[n+1] (int64, offsets[0] = 0,
 * non-decreasing, offsets[n] = nnz), cols[nnz] (int32 in [0,n)), weights[nnz]
 * (int32 > 0), all of kind `ptr_kind`.  The CSR must be symmetric as described
 * above (checked when opt.validate = 1).  Copies the graph to the device and
 * sizes the context's device memory for it; a previous graph and its results
 * are dropped.  Errors: INVALID_ARG, BAD_CSR, NOT_SYMMETRIC, OVERFLOW, OOM, CUDA. */
int louvain_load_csr(louvain_ctx *ctx, int64_t n, int64_t nnz, const int64_t *offsets, const int32_t *cols,
                     const int32_t *weights, int ptr_kind);

/* Load several independent graphs at once: graph g owns the vertices
 * [graph_offsets[g], graph_offsets[g+1]) of one CSR laid out as in
 * louvain_load_csr (block diagonal: no entry may join two graphs; checked).
 * graph_offsets[num_graphs + 1] has the kind `ptr_kind`.  louvain_run then runs
 * every graph as if alone — its own total weight M, its own iteration and
 * pass control — in shared launches; results are per graph
 * (louvain_batch_get_*, and louvain_get_membership with ids local to each
 * graph).  The paper runs one graph at a time; batching fills the GPU with
 * graphs that are each too small to fill it alone.
 * Errors: as louvain_load_csr. */
int louvain_load_batch(louvain_ctx *ctx, int64_t num_graphs, const int64_t *graph_offsets, int64_t n, int64_t nnz,
                       const int64_t *offsets, const int32_t *cols, const int32_t *weights, int ptr_kind);

/* Number of graphs loaded (1 after louvain_load_csr). */
int louvain_get_num_graphs(louvain_ctx *ctx, int64_t *num_graphs);

/* Load num_graphs graphs given as separate host CSRs (graph g: ns[g] vertices,
 * nnzs[g] entries, offsets[g], cols[g], weights[g] as in louvain_load_csr, ids
 * local to the graph): the same as louvain_load_batch of their block-diagonal
 * concatenation, without building it on the host (each graph is copied to its
 * place on the device, ids rebased there).  Errors as louvain_load_batch. */
int louvain_load_parts(louvain_ctx *ctx, int64_t num_graphs, const int64_t *ns, const int64_t *nnzs,
                       const int64_t *const *offsets, const int32_t *const *cols, const int32_t *const *weights);

/* Per graph g < num_graphs: modularity q[g]; exact numerator and M
 * (num_hi, num_lo, M may be NULL), host arrays of num_graphs entries. */
int louvain_batch_get_modularity(louvain_ctx *ctx, double *q, int64_t *num_hi, uint64_t *num_lo, int64_t *M);

/* Graph g: out[0] passes it took part in, out[1] iterations, out[2]
 * communities, out[3] moves. */
int louvain_batch_get_graph_info(louvain_ctx *ctx, int64_t g, int64_t out[4]);

/* Iterations of graph g (as louvain_get_iteration, 4 values each) into
 * out[4 * cap]; *count = how many there are. */
int louvain_batch_get_iterations(louvain_ctx *ctx, int64_t g, int64_t *out, int64_t cap, int64_t *count);

/* Vertex-to-kernel mapping of the local-moving phase.  thresholds[5] are the
 * largest degrees handled by, in order, a thread per vertex (register table,
 * at most 8), a warp with a 64-slot table (at most 32), a warp with a 256-slot
 * table (at most 128), a block with a 2048-slot table (at most 1024) and a
 * block with an 8192-slot table (at most 4096); larger degrees go to the hub
 * path (global tables).  They must increase.  Lowering one moves vertices to
 * a wider mapping whose table is emptier.  NULL restores the defaults (the
 * maxima).  The mapping never changes results: only which kernel computes
 * them.  Errors: INVALID_ARG. */
int louvain_set_mapping(louvain_ctx *ctx, const int32_t *thresholds);
int louvain_get_mapping(louvain_ctx *ctx, int32_t *thresholds);

/* Autotuner: times the first local-moving iteration of the loaded graph (or
 * batch) under candidate mappings (coordinate descent over the thresholds,
 * best of two trials each) and keeps the fastest for later runs.  Writes the
 * chosen thresholds[5] and the best trial's device time in ms (either may be
 * NULL).  Costs about a dozen iterations; the previous result is dropped (run
 * again).  Not in the paper: it picks the GPU mapping, not the method.
 * Errors: STATE (no graph), CUDA, INTERNAL. */
int louvain_autotune(louvain_ctx *ctx, int32_t *thresholds, double *ms);

/* Run the Louvain method on the loaded graph.  Errors: STATE (no graph), CUDA,
 * INTERNAL, TIMEOUT. */
int louvain_run(louvain_ctx *ctx);

/* Incremental re-run (the dynamic-graph setting the paper gives as motivation,
 * Section 1): run as louvain_run, but pass 0 starts from memb[n] (kind
 * `ptr_kind`, n = the loaded n) instead of singletons: community totals and
 * sizes are summed over its communities, the pass's "before" modularity is
 * memb's, and pass 0's level is kept even when no vertex moves.  With several
 * graphs loaded, memb holds global ids and each vertex's id must lie in its
 * own graph's vertex range.  Singletons give exactly louvain_run's result.
 * Errors: INVALID_ARG (wrong n, an id out of range: the graph stays loaded),
 * STATE, CUDA, INTERNAL. */
int louvain_run_from(louvain_ctx *ctx, const int32_t *memb, int64_t n, int ptr_kind);

/* Partition, then merge (one graph loaded): vertex u goes to part
 * floor(u * parts / n); every part's induced subgraph (the entries whose ends
 * share a part) runs on its own, all parts together as one batch in a second
 * context on the same device and stream; then the whole graph runs from the
 * parts' communities (louvain_run_from), whose pass 0 moves vertices across
 * part boundaries and whose later passes merge communities.  parts = 1 is
 * louvain_run.  *parts_ms (may be NULL) gets the parts' run time; statistics
 * and results are those of the whole-graph run.  Not in the paper (Section 2
 * reviews partition-based methods): the single-graph basis for spreading one
 * graph over several GPUs.  Errors: INVALID_ARG, STATE (no graph, or several
 * loaded), OOM, CUDA, INTERNAL. */
int louvain_run_partitioned(louvain_ctx *ctx, int64_t parts, double *parts_ms);

/* Top-level community of every input vertex into out[n] (kind `ptr_kind`);
 * community ids are dense in [0, k) by the renumbering rule (ascending old id
 * at every pass); with several graphs loaded, dense per graph.  n must equal
 * the loaded n. */
int louvain_get_membership(louvain_ctx *ctx, int32_t *out, int64_t n, int ptr_kind);

/* Modularity of the result (see the convention above); one graph loaded. */
int louvain_get_modularity(louvain_ctx *ctx, double *q);

/* Exact modularity of the result: Q = num / M^2 with num = num_hi * 2^64 + num_lo. */
int louvain_get_modularity_exact(louvain_ctx *ctx, int64_t *num_hi, uint64_t *num_lo, int64_t *M);

/* Modularity of an arbitrary membership memb[n] (kind `ptr_kind`, values in
 * [0, n)) of the loaded graph, computed on the device; exact numerator too
 * (num_hi / num_lo / M may be NULL). */
int louvain_modularity(louvain_ctx *ctx, const int32_t *memb, int64_t n, int ptr_kind, double *q, int64_t *num_hi,
                       uint64_t *num_lo, int64_t *M);

/* The paper has no counterpart to this entry point.  Exact modularity of
 * memb[n] for a graph given entirely in device memory (offsets[n+1], cols,
 * weights, memb: device pointers on the current device, in the CSR form that
 * louvain_load_csr takes), computed on `cuda_stream` (a cudaStream_t, NULL =
 * the default stream) without allocating any device memory: for callers that
 * must not allocate, such as code whose allocator already owns the device's
 * free memory, a service with a fixed memory plan, or a pipeline that cannot
 * take the device-wide synchronisation of cudaMalloc / cudaFree.  Its
 * scratch (degrees, community totals, sums) is a static device array of
 * 16 * LOUVAIN_STATIC_MAX_VERTICES + 256 bytes (16 MiB + 256 B) that every GPU
 * loading this library holds until the process exits.  The first call on a
 * device finds that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the array and each clears what it needs: calls that overlap on the
 * GPU race and must not be issued.  Outputs are host pointers; num_hi,
 * num_lo, M may be NULL.  The call synchronises `cuda_stream`.
 * Errors: CAPACITY (n > LOUVAIN_STATIC_MAX_VERTICES), INVALID_ARG (a null
 * pointer with n > 0, negative n, a membership outside [0, n)), BAD_CSR (a
 * row whose offsets are negative or decreasing, a column outside [0, n); the
 * kernels check both before they index with them), OVERFLOW (M >= 2^62),
 * CUDA.  The offsets must lie within the caller's cols / weights buffers
 * (offsets[n] <= their length): the call cannot see those lengths. */
int louvain_modularity_static(int64_t n, const int64_t *offsets, const int32_t *cols, const int32_t *weights,
                              const int32_t *memb, void *cuda_stream, double *q, int64_t *num_hi, uint64_t *num_lo,
                              int64_t *M);

int louvain_get_stats(louvain_ctx *ctx, louvain_stats *out);
int louvain_get_pass_info(louvain_ctx *ctx, int pass, louvain_pass_info *out);

/* Iteration t of the last run (all passes, in order): out[0] = pass,
 * out[1] = moves, out[2..3] = S (sum of the gains of the moves, as hi, lo). */
int louvain_get_iteration(louvain_ctx *ctx, int64_t t, int64_t out[4]);

/* Renumbered membership of pass `pass`'s graph (record_levels = 1), out[n] host. */
int louvain_get_level(louvain_ctx *ctx, int pass, int32_t *out, int64_t n);

/* Coarse CSR built after pass `pass` (record_levels = 1): off[k+1], col[nnz],
 * w[nnz] (int64), host.  Columns within a row are in no particular order. */
int louvain_get_coarse(louvain_ctx *ctx, int pass, int64_t *off, int64_t k, int32_t *col, int64_t *w,
                       int64_t nnz);

/* Device bytes the context holds (arena). */
int louvain_get_device_bytes(louvain_ctx *ctx, int64_t *bytes);

/* Device bytes a context's arena needs for a graph (or a batch) of n
 * vertices and nnz entries, without allocating anything. */
int louvain_arena_bytes(int64_t n, int64_t nnz, int64_t *bytes);

/* ------------------------------------------------------------ server
 * Requests (graphs) submitted at any time wait in arrival order.  Each worker
 * slot owns one context on its own stream, so slots' device work overlaps.
 * A free slot takes the oldest waiting request and every request behind it
 * while their CSR entries stay within batch_max_entries (and their count
 * within batch_max_graphs), and runs them as one batch (louvain_load_batch),
 * so each result equals the graph's result alone (synchronous: bit for bit).
 * Slot arenas stay resident between runs; admission keeps all slots' arenas
 * within hbm_budget_bytes: a slot that cannot grow waits for busy slots to
 * finish, takes back the arenas of idle slots, and a request that does not fit
 * even alone is answered with LOUVAIN_ERR_OOM.  Not in the paper (it runs one
 * graph at a time on the CPU); the server is how the engine serves many. */
typedef struct louvain_server louvain_server;
typedef struct {
  int32_t slots;              /* worker slots (contexts), default 2 */
  int32_t batch_max_graphs;   /* at most this many requests per run, default 1024 */
  int64_t batch_max_entries;  /* at most this many CSR entries per run, default 256 Mi; 0 = one request per run */
  int64_t hbm_budget_bytes;   /* device bytes all slots' arenas may hold; 0 = 90% of free memory at creation */
  int64_t borrow_inputs;      /* 0 (default): louvain_server_submit copies the graph (into a reused pinned
                                 host pool); 1: it keeps the caller's pointers, the caller keeps the arrays
                                 alive and unchanged until the request's result has been polled, and the
                                 worker slots copy them to the device themselves (no host copy on the
                                 submitting thread) */
  int64_t reserved[4];
} louvain_server_config;

typedef struct {
  int64_t request_id;
  int32_t status;             /* 0 or a LOUVAIN_ERR_* code */
  int32_t batch_size;         /* requests in the run that served it */
  int64_t n;                  /* vertices: the length of its membership */
  int64_t communities;
  double q;                   /* modularity; exact: (num_hi * 2^64 + num_lo) / M^2 */
  int64_t num_hi;
  uint64_t num_lo;
  int64_t M;
  double submit_s, start_s, done_s;   /* seconds since the server was created */
} louvain_server_result;

int louvain_server_default_config(louvain_server_config *cfg);
/* opt: the engine options every slot runs with (NULL = defaults). */
int louvain_server_create(louvain_server **out, const louvain_options *opt, const louvain_server_config *cfg,
                          int device);
/* Submit graph `request_id` (host CSR as in louvain_load_csr; copied, or
 * borrowed with borrow_inputs = 1). */
int louvain_server_submit(louvain_server *srv, int64_t request_id, int64_t n, int64_t nnz, const int64_t *offsets,
                          const int32_t *cols, const int32_t *weights);
/* Up to cap finished results into out (host); waits up to wait_ms for the
 * first if none is ready.  *count = results returned. */
int louvain_server_poll(louvain_server *srv, louvain_server_result *out, int64_t cap, int64_t *count, int32_t wait_ms);
/* Copy a finished request's membership (n entries) and forget it. */
int louvain_server_membership(louvain_server *srv, int64_t request_id, int32_t *out, int64_t n);
/* out: submitted, finished, runs, queued, reserved bytes, peak reserved, budget, slots. */
int louvain_server_stats(louvain_server *srv, int64_t out[8]);
/* Seconds spent, summed over all runs of all slots, in: assembling batches on
 * the host, loading them (copy to the device, validation), running them, and
 * fetching results (memberships, modularities). */
int louvain_server_timings(louvain_server *srv, double out[4]);
/* Finishes every queued request, then frees everything. */
void louvain_server_destroy(louvain_server *srv);

void louvain_destroy(louvain_ctx *ctx);
const char *louvain_last_error(const louvain_ctx *ctx);
const char *louvain_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GB_LOUVAIN_H */
