/*
 * jt.h -- C ABI of the GB300 junction-tree exact-inference library.
 *
 * The library answers the exact-inference query of a Bayesian network (BN):
 * given evidence e on some variables, P(e) and the posterior marginal
 * P(X_v | e) of every unobserved variable (Section 1 of "POSTER: Fast
 * Parallel Exact Inference on Bayesian Networks", the problem statement).
 * It follows the junction-tree route described there: the BN is compiled
 * once into a tree of cliques joined by separators, each with a potential
 * table (Section 1), and every query passes messages along the tree with
 * the three table operations of Section 2 -- marginalisation, extension and
 * reduction (evidence) -- plus Hugin separator division.  Cliques are
 * grouped into tree layers (Section 2, BFS traversal) and every table entry
 * of every clique is work for a whole batch of evidence cases at once, the
 * GPU counterpart of the paper's flattening of a layer's table entries into
 * one parallel task (Section 2, hybrid parallelism).  By default each pass
 * (collect, distribute) is one GPU launch that takes the work in layer
 * order and lets each case tile advance as soon as its own producers are
 * done; JT_SCHEDULE_LAYERS runs one launch per layer instead.
 *
 * Plans can be specialised at compile time: to an observed set that every
 * case observes (its dimensions sliced out of the tables) and to a query
 * set (barren variables removed); see jt_compile_opts.  Two comparators sit
 * beside the batched path for measurement: jt_infer_plain (per-case FP64
 * on the GPU, element-wise style) and jt_infer_cpu (the paper's own
 * layer-parallel design on the host cores).
 *
 * Conventions shared by every call:
 *   - Variables are numbered 0..n-1.  card[v] >= 2 is the number of states.
 *   - Parents are given in CSR form: the parents of v are
 *     parents[parent_ptr[v] .. parent_ptr[v+1]-1]; the graph must be acyclic.
 *   - cpt is all conditional probability tables concatenated in variable
 *     order.  The table of v has one row per joint configuration of its
 *     parents (mixed radix, the first listed parent varies slowest) and
 *     card[v] columns (the child's state varies fastest).  Entries must be
 *     >= 0 and every row must sum to 1 within 1e-6.
 *   - Evidence is int32 [n_cases][n]: the observed state of v, or -1.
 *   - Outputs: log_pe float64 [n_cases] (natural log of P(e));
 *     posteriors float64 [n_cases][sum(card)], the states of v at offsets
 *     sum(card[0..v-1]) ...; an observed variable gets a point mass (and a
 *     variable removed from a plan pruned to a query set gets NaN);
 *     case_status int32 [n_cases] (JT_CASE_*).
 *   - Every call returns a jt_status and never aborts.  The caller owns all
 *     buffers it passes; inputs are read during the call only.
 *   - Concurrency: calls on different plans are independent.  Calls on one
 *     plan from several host threads are serialised by the plan, but its
 *     batched calls share one set of per-batch device tables, so their
 *     device work must also be ordered: issue them on one stream (or order
 *     the streams) -- jt_infer and jt_profile synchronise before returning,
 *     jt_infer_device does not.  jt_infer_cpu only reads the plan.
 *     jt_plan_free must not overlap any call on the plan.  A server keeps
 *     its own per-batch tables for each batch in flight and serialises its
 *     calls internally.
 *   - Accuracy of the FP32 batched path against exact FP64 arithmetic:
 *     max abs posterior error <= 1e-5 and |d log P(e)| <= 1e-6*max(1,|log P(e)|)
 *     on the workloads this library is tested on.
 */
#ifndef JT_H
#define JT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JT_API __attribute__((visibility("default")))
#else
#define JT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jt_plan jt_plan;     /* opaque; owns all device memory of a compiled network */
typedef struct jt_server jt_server; /* opaque; continuous-batching request loop */

typedef enum {
  JT_OK = 0,
  JT_EINVAL = 1,    /* bad argument, CPT or evidence shape */
  JT_ECYCLE = 2,    /* the parent graph has a directed cycle */
  JT_ETOOBIG = 3,   /* a clique table exceeds max_clique_entries */
  JT_ENOMEM = 4,    /* device or host allocation failed / arena too small */
  JT_ECUDA = 5,     /* a CUDA call failed (see jt_last_error) */
  JT_ETIMEOUT = 6,  /* a bounded device wait expired */
  JT_EBUSY = 7,     /* serving: result not ready yet */
  JT_ENOTFOUND = 8  /* serving: unknown plan id or ticket */
} jt_status;

enum {
  JT_CASE_OK = 0,
  JT_CASE_ZERO_EVIDENCE = 1, /* P(e) = 0: log_pe = -inf, posteriors NaN */
  JT_CASE_BAD_EVIDENCE = 2,  /* a state outside [-1, card-1]: outputs NaN */
  JT_CASE_INCOMPLETE = 3     /* a bounded device wait of the pass expired:
                                outputs NaN (the call, or the next
                                synchronous one, returns JT_ETIMEOUT) */
};

enum {
  JT_ROOT_LARGEST = 0,   /* root = largest clique table (ties: lowest id) */
  JT_ROOT_MIN_HEIGHT = 1 /* root = clique of least eccentricity, i.e. fewest
                            layers (Section 2, root selection strategy);
                            ties: larger table, then lowest id */
};

/* Work order of a pass.  LAYERS: one launch per tree layer, every clique
 * of the layer for every case tile, each launch waiting for the previous
 * one (Section 2's layer-by-layer order).  DATAFLOW: one launch per pass;
 * case tiles are independent, so a clique's work on a tile starts as soon
 * as its own producers on that tile are done, and the small layers near the
 * root of one tile overlap the large layers of others.  A dataflow pass
 * holds every SM until it ends: when several plans share the GPU (a
 * server), LAYERS lets their short passes interleave and gives lower
 * latency. */
enum { JT_SCHEDULE_DATAFLOW = 0, JT_SCHEDULE_LAYERS = 1 };

/* Number of table-size buckets of the per-bucket work shape: bucket b holds
 * the tables with 2^b <= entries < 2^(b+1) (a clique for the collect pass,
 * a distribute task's source rows for the distribute pass). */
#define JT_SIZE_BUCKETS 32

typedef struct {
  int32_t root_rule;          /* JT_ROOT_* (default JT_ROOT_MIN_HEIGHT) */
  int32_t host_only;          /* 1: compile on the host only, allocate no
                                 device memory (inference calls then return
                                 JT_EINVAL); used to inspect a plan */
  int32_t cases_per_thread;   /* 1, 2, 4 or 8: each GPU thread carries this
                                 many evidence cases, a case tile is 32x that;
                                 0 = automatic (4; use 1 for small batches) */
  int32_t rows_per_cta;       /* table rows (entries) per thread block of a
                                 layer launch; 0 = automatic (per plan) */
  int64_t max_clique_entries; /* JT_ETOOBIG above this; 0 = 2^31 - 1 */
  int64_t arena_bytes;        /* device bytes for per-batch tables; the
                                 batch is processed in chunks that fit;
                                 0 = automatic (min(224 GiB, 70% of free)) */
  int32_t use_graphs;         /* 1 (default): replay the layer launches of a
                                 batch chunk as one captured CUDA graph */
  int32_t items_per_tile;     /* target warp work items per case tile and
                                 tree layer of the collect pass when
                                 rows_per_cta is 0: small values give long
                                 items, large values short ones;
                                 0 = automatic (192) */
  int32_t items_per_tile_distribute; /* the same for the distribute pass;
                                 0 = items_per_tile */
  int32_t schedule;           /* JT_SCHEDULE_*: how the work of a pass is
                                 ordered on the GPU (default dataflow) */
  int32_t wait_limit_us;      /* dataflow schedule: bound of a device wait
                                 for producers on the same tile; when it
                                 expires the call returns JT_ETIMEOUT;
                                 0 = automatic (2 s) */
  int32_t stall_clique;       /* testing only: 0 (default) = off; k > 0 makes
                                 the collect work of clique k-1 wait for one
                                 producer more than exists, so its waits
                                 expire (exercises JT_ETIMEOUT) */
  int32_t n_observed_set;     /* specialise the plan to an observed set: */
  const int32_t *observed_set;/* n_observed_set distinct variables that EVERY
                                 case run on the plan observes (their states
                                 vary from case to case).  Their dimensions
                                 are sliced out of every clique and separator
                                 table (each case reads its own slice of the
                                 base tables), which shrinks the tables by
                                 the product of those cardinalities; a case
                                 leaving one of them unobserved gets
                                 JT_CASE_BAD_EVIDENCE.  NULL / 0 = none.
                                 Read during jt_compile only.  Sliced plans
                                 support every call except jt_infer_plain. */
  int32_t rescale;            /* batched path: 1 (default) = every upward
                                 message is scaled by 2^-k, k the exponent of
                                 its largest entry for the case, before the
                                 parent absorbs it, and the k are added back
                                 into log P(e) (exact in binary floating
                                 point; keeps deep trees and strong evidence
                                 inside FP32's range); 0 = messages are used
                                 as computed, so a case whose messages
                                 underflow FP32 reports JT_CASE_ZERO_EVIDENCE
                                 or loses accuracy (for comparison with the
                                 unscaled definition).  The plain FP64 path
                                 never rescales. */
  int32_t n_query_set;        /* prune the plan to a query set: */
  const int32_t *query_set;   /* n_query_set distinct variables whose
                                 posteriors the plan must answer.  The plan
                                 keeps only these, the variables of
                                 observed_set, and their ancestors; every
                                 other variable is barren (no kept variable
                                 depends on it, so summing it out of its CPT
                                 gives exactly 1) and is removed from the
                                 network before the tree is built.  P(e) and
                                 the posteriors of every kept variable are
                                 unchanged; the posterior columns of removed
                                 variables are NaN; a case that observes a
                                 removed variable gets JT_CASE_BAD_EVIDENCE.
                                 Evidence and posterior rows keep the full
                                 network's layout.  NULL / 0 = none.  Read
                                 during jt_compile only.  Pruned plans
                                 support the batched calls (jt_infer,
                                 jt_infer_device, jt_infer_device_noalloc,
                                 jt_profile, jt_autotune), not
                                 jt_infer_plain, jt_infer_cpu or the server. */
  int32_t collect_rows_by_bucket[JT_SIZE_BUCKETS];
                              /* rows (table entries) per warp work item of
                                 the collect pass for the cliques of each
                                 size bucket (JT_SIZE_BUCKETS); 0 = the
                                 layer's automatic value (items_per_tile).
                                 Each value is rounded down to a power of two
                                 in [16, 4096].  Ignored when rows_per_cta is
                                 set.  jt_autotune fills these per bucket. */
  int32_t distribute_rows_by_bucket[JT_SIZE_BUCKETS];
                              /* the same for the distribute pass, bucketed
                                 by each task's source rows */
  int32_t fuse_distribute;    /* 1 (default): two marginalisations of the
                                 same clique table in the distribute pass
                                 (two child separators, or a separator and
                                 a posterior variable) share one read of
                                 the table when the second one's targets
                                 per block of common variables fit a warp's
                                 shared-memory sums; 0: every marginal reads
                                 the table on its own */
  int32_t recompute_psi;      /* 1: the collect pass stores no clique tables;
                                 the distribute pass recomputes every row it
                                 reads from the base table, the child
                                 messages and the evidence, in the collect
                                 pass's arithmetic order (so the values are
                                 the same bit for bit).  The per-batch
                                 tables then hold no clique tables (a case
                                 needs about 4*sum|S| + ... bytes instead of
                                 4*sum|C| more), so an arena admits several
                                 times more cases, and neither pass moves
                                 the clique tables through DRAM.  Fused
                                 distribute pairs are not used with it;
                                 ignored for plans specialised to an
                                 observed set.  0 (default): stored. */
  int32_t collect_prefetch;   /* 1: the collect pass requests the child
                                 message rows of each 32-row batch into L2
                                 when the batch starts, so the gathers of
                                 its row groups find them there (helps where
                                 the messages do not fit L2, costs
                                 instructions elsewhere); 0 (default): off.
                                 jt_autotune tries it per plan. */
} jt_compile_opts;

typedef struct {
  int32_t n_vars;               /* variables of an evidence row (the full network) */
  int32_t n_cliques;
  int32_t n_levels;             /* tree height + 1 */
  int32_t root;
  int64_t sum_clique_entries;   /* sum over cliques of |C| */
  int64_t max_clique_entries;
  int64_t sum_sep_entries;      /* sum over separators of |S| */
  int64_t sum_card;             /* length of one posterior row */
  int32_t tile_cases;           /* evidence cases per tile (32 * cases_per_thread) */
  int32_t chunk_cases;          /* cases per arena chunk (multiple of tile_cases) */
  int64_t arena_bytes;          /* bytes of the per-batch arena actually used */
  int64_t static_device_bytes;  /* base tables, index maps, work lists */
  int64_t collect_items;        /* thread blocks per tile, all collect layers */
  int64_t distribute_items;     /* thread blocks per tile, all distribute layers */
  double algorithmic_bytes_per_case; /* 8*sum|C| + 16*sum|S| + 4n + 8*sum(card) + 8 */
  int32_t kernels_per_chunk;    /* kernel launches of one batch chunk */
  int32_t sliced_vars;          /* size of the observed set sliced out (0: none) */
  int32_t separator_evidence_vars; /* variables whose evidence indicator is
                                 applied to an upward message (a separator
                                 smaller than every clique holding them)
                                 rather than evaluated per clique entry */
  int32_t pruned_vars;          /* barren variables removed (query_set) */
  int32_t budget_chunk_cases;   /* cases one arena chunk admits under the
                                   plan's arena budget (arena_bytes, or the
                                   automatic budget evaluated at this call);
                                   0 for host_only plans */
  int32_t collect_rows_by_bucket[JT_SIZE_BUCKETS];    /* rows per collect work
                                   item used for each size bucket (largest
                                   value in the bucket; 0 = no clique) */
  int32_t distribute_rows_by_bucket[JT_SIZE_BUCKETS]; /* the same for the
                                   distribute tasks */
  int64_t collect_entries_by_bucket[JT_SIZE_BUCKETS]; /* clique entries per
                                   case in each bucket (collect work) */
  int64_t distribute_entries_by_bucket[JT_SIZE_BUCKETS]; /* source rows per
                                   case of the distribute tasks in each
                                   bucket */
} jt_plan_info_t;

/* Fill opts with the defaults listed above. */
JT_API void jt_default_opts(jt_compile_opts *opts);

/*
 * Compile a network into a plan (host side; Section 1's secondary structure
 * and Section 2's layering): moralise, triangulate by min-fill elimination
 * (ties to the lowest variable id), keep the maximal elimination cliques,
 * join them by a maximum-weight spanning tree on the number of shared
 * variables, choose the root (opts->root_rule), group cliques into BFS
 * layers, order every clique's variables so that its separator towards the
 * parent is the outermost (slowest) block of its table, precompute the
 * index maps of every table operation, upload everything to the current
 * CUDA device.  All arrays are host pointers; they are copied.  opts may be
 * NULL for the defaults.  On success *out owns the plan; free it with
 * jt_plan_free.  Errors: JT_EINVAL (shapes, CPT rows), JT_ECYCLE,
 * JT_ETOOBIG, JT_ENOMEM, JT_ECUDA.
 */
JT_API jt_status jt_compile(int32_t n_vars, const int32_t *card, const int32_t *parent_ptr,
                     const int32_t *parents, const double *cpt, const jt_compile_opts *opts,
                     jt_plan **out);

/*
 * Batched FP32 inference with HOST buffers (Section 1's query for every case
 * of the batch).  Copies the evidence to the device, runs the collect and
 * distribute layers (FP32 tables, power-of-two rescaling, FP64 log P(e) and
 * posterior normalisation), and copies the results back; the call returns
 * after the results are in the caller's buffers.  cuda_stream is a
 * cudaStream_t or NULL for the plan's own stream.  Any n_cases >= 0.
 * Page-locked (pinned) caller buffers are copied directly and
 * asynchronously; pageable ones through the plan's pinned staging buffer.
 * Returns JT_ETIMEOUT if a bounded device wait expired (the dataflow
 * schedule's waits for producers, limit wait_limit_us); the condition is
 * then cleared.
 */
JT_API jt_status jt_infer(jt_plan *plan, int32_t n_cases, const int32_t *evidence, double *log_pe,
                   double *posteriors, int32_t *case_status, void *cuda_stream);

/*
 * Same as jt_infer with DEVICE buffers (all four pointers on the plan's
 * device).  Work is enqueued on cuda_stream (NULL = the plan's stream) and
 * the call returns without synchronising; the outputs are valid once the
 * stream has reached that point.  Evidence states outside [-1, card-1] give
 * JT_CASE_BAD_EVIDENCE for that case only.  An expired device wait marks
 * every case of the call JT_CASE_INCOMPLETE (outputs NaN); the condition
 * stays set (later device calls are marked the same) until a synchronous
 * call (jt_infer, jt_profile) returns JT_ETIMEOUT and clears it.
 */
JT_API jt_status jt_infer_device(jt_plan *plan, int32_t n_cases, const int32_t *d_evidence,
                          double *d_log_pe, double *d_posteriors, int32_t *d_case_status,
                          void *cuda_stream);

/*
 * Size of the fixed device array behind jt_infer_device_noalloc (64 MiB).
 */
#define JT_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * The paper has no counterpart to this call; it is a deployment variant of
 * jt_infer_device for callers that cannot allocate device memory while
 * serving -- a process whose device memory is owned by another allocator,
 * a latency-bound loop that cannot afford cudaMalloc/cudaFree (they
 * synchronise the whole device), or a deployment that forbids allocation
 * after start-up.  Same arguments and stream semantics as jt_infer_device,
 * and the same results bit for bit; it allocates nothing: the per-batch
 * tables live in one
 * fixed device array of JT_NOALLOC_SCRATCH_BYTES that the library defines
 * (every GPU that loads the library keeps it until the process exits).
 * The first call on a device looks up that array's device address, so make
 * the first call before any stream capture.  All calls, for every plan,
 * share the one array and leave their contents in it; calls whose work
 * overlaps on the GPU (different streams, threads or plans at once) race
 * and give wrong results -- serialise them.  A plan whose tables for one
 * case tile (jt_plan_info: tile_cases cases) exceed the array is refused
 * with JT_ENOMEM and a message from jt_last_error; larger batches are run
 * in chunks that fit.  One difference from jt_infer_device: every call
 * starts with the array's expired-wait flag cleared, so an expired device
 * wait marks the cases of that call only (JT_CASE_INCOMPLETE) and is not
 * carried into later calls (jt_infer_device keeps its flag set until a
 * synchronous call reports it).
 */
JT_API jt_status jt_infer_device_noalloc(jt_plan *plan, int32_t n_cases, const int32_t *d_evidence,
                                         double *d_log_pe, double *d_posteriors,
                                         int32_t *d_case_status, void *cuda_stream);

/*
 * The plain per-case FP64 GPU path (measurement comparator, element-wise
 * style of the prior GPU approach the paper compares against, Section 1 and
 * Section 3 "Elem."): the same plan, FP64 tables, one case at a time, one
 * kernel launch per table operation per tree edge, one thread per table
 * entry, mixed-radix indices by division, FP64 atomicAdd marginalisation,
 * no fusion, no graphs, no rescaling.  HOST buffers; synchronous.
 */
JT_API jt_status jt_infer_plain(jt_plan *plan, int32_t n_cases, const int32_t *evidence,
                         double *log_pe, double *posteriors, int32_t *case_status,
                         void *cuda_stream);

/*
 * Multi-core CPU comparator in the style of the paper's own design
 * (Section 2's hybrid inter- and intra-clique parallelism): on the HOST
 * cores, one case at a time, the tree walked layer by layer with cliques
 * and separators as the layers' nodes, every table entry of a layer one
 * task of a single parallel loop split statically over n_threads threads
 * (0 = the hardware's thread count), index mappings from each entry's
 * mixed-radix digits, FP64 tables without rescaling (P(e) below FP64's
 * range reports JT_CASE_ZERO_EVIDENCE).  For context measurements of that
 * design on the host; results do not depend on n_threads.  HOST buffers
 * laid out as for jt_infer; synchronous.  Runs on host_only plans too (it
 * needs no GPU); plans specialised to an observed set get JT_EINVAL.
 */
JT_API jt_status jt_infer_cpu(const jt_plan *plan, int32_t n_cases, const int32_t *evidence,
                              double *log_pe, double *posteriors, int32_t *case_status,
                              int32_t n_threads);

/*
 * Instrumented run of jt_infer_device (device buffers, same arguments) for
 * measurement: the pass launches (one per pass in the dataflow schedule,
 * one per layer in the layer schedule) are issued one by one (no graph)
 * with a CUDA event around each, on cuda_stream, and the call synchronises.
 * out[0] total ms of the collect launches, out[1] total ms of the
 * distribute launches, out[2] ms of the evidence and finalize launches,
 * out[3] number of collect launches, out[4] number of distribute launches,
 * out[5] the whole run's ms.  The results are written like jt_infer_device.
 */
JT_API jt_status jt_profile(jt_plan *plan, int32_t n_cases, const int32_t *d_evidence,
                            double *d_log_pe, double *d_posteriors, int32_t *d_case_status,
                            void *cuda_stream, double *out);

/*
 * Autotuner (no counterpart in the paper; it addresses the load imbalance
 * between threads that Section 2 attributes to tables of very different
 * sizes).  Times the collect and the distribute launches of n_cases cases
 * separately on the current device (jt_profile: one warm-up run, then the
 * best of two) in base's schedule, in three stages:
 *   1. per tile width (cases per thread 4 and 8, unless base fixes it) the
 *      work-item target of each pass over {96, 192, 384, 768, 1536} items
 *      per tile and layer; the fastest width and targets are kept;
 *   2. per table-size bucket (JT_SIZE_BUCKETS; the buckets holding at
 *      least 2 % of a pass's rows, largest first, at most eight) the rows
 *      of one warp work item -- hence the warps (threads) per table and
 *      the tile shape rows x cases -- over the powers of two 32 .. 4096,
 *      each pass keeping its own best value (coordinate descent; a change
 *      is kept when it is at least 1 % faster);
 *   3. the result with fuse_distribute, recompute_psi and collect_prefetch
 *      each turned the other way (each recompiled), the fastest kept if it
 *      is at least 1 % faster.
 * Between the candidates of stages 1 and 2 only the work lists are
 * rebuilt, not the plan.
 * Writes the result to *best (base fields kept; the bucket tables in
 * collect_rows_by_bucket / distribute_rows_by_bucket) and its pass time per
 * case in ns to *best_ns_per_case (may be NULL).  base may be NULL for the
 * defaults.  Allocates and frees its own device memory.
 */
JT_API jt_status jt_autotune(int32_t n_vars, const int32_t *card, const int32_t *parent_ptr,
                             const int32_t *parents, const double *cpt, const jt_compile_opts *base,
                             int32_t n_cases, jt_compile_opts *best, double *best_ns_per_case);

/*
 * Testing only (no counterpart in the paper): turn the stall compiled into
 * a plan by jt_compile_opts.stall_clique on (enabled = 1, the state after
 * jt_compile) or off (0), so that one plan can run a pass whose bounded
 * device waits expire and then a normal pass on the same per-batch tables.
 * It rewrites one producer count of the plan's device work description
 * and synchronises; it must not overlap a pass of the plan.  JT_EINVAL if
 * the plan was compiled without stall_clique or with host_only.
 */
JT_API jt_status jt_debug_stall(jt_plan *plan, int32_t enabled);

/* Sizes and layout of a compiled plan. */
JT_API jt_status jt_plan_info(const jt_plan *plan, jt_plan_info_t *out);

/*
 * Structure of clique c (for inspection and tests): its variables in table
 * layout order (upward separator first), its parent clique (-1 for the
 * root) and its depth.  vars must hold 64 entries; *n_vars receives the
 * count.
 */
JT_API jt_status jt_plan_clique(const jt_plan *plan, int32_t c, int32_t *n_vars, int32_t *vars,
                         int32_t *parent, int32_t *depth);

/* Release a plan and all of its device memory (NULL is ignored). */
JT_API void jt_plan_free(jt_plan *plan);

/* Static text for a status code. */
JT_API const char *jt_status_string(jt_status status);

/* Text of the last error on the calling thread ("" if none). */
JT_API const char *jt_last_error(void);

/*
 * Serving: a continuous-batching request loop (one host thread) over
 * resident plans.  Requests are single evidence cases; the loop coalesces
 * pending requests of the same plan into batches, admits a batch when its
 * per-batch tables fit the server's device pool (arena_bytes; 0 = 16 GiB),
 * keeps up to max_inflight batches in flight on separate CUDA streams so
 * that batches of different plans overlap on the device, and hands results
 * back by ticket.  A request's result does not depend on which other
 * requests share its batch (fixed per-case reduction order).
 * jt_server_create allocates the pool (one device allocation of
 * arena_bytes, JT_ENOMEM if it fails) and the streams; jt_server_add_plan
 * allocates the plan's pinned host and device staging buffers (outside the
 * pool); the request loop itself allocates nothing: a plan's batch slot is
 * a region of the pool, reused batch after batch, and idle slots of other
 * plans are evicted (least recently used first) when the pool is full.
 */
JT_API jt_status jt_server_create(int64_t arena_bytes, int32_t max_batch, int32_t max_inflight,
                           jt_server **out);
/* Register a plan (not copied; it must outlive the server). */
JT_API jt_status jt_server_add_plan(jt_server *srv, jt_plan *plan, int32_t *plan_id);
/*
 * Register a plan served with iteration-level batching (no counterpart in
 * the paper; the layer-by-layer order of Section 2 applied across
 * requests): the plan's tables for `tiles` case tiles (jt_plan_info
 * tile_cases cases each) are carved out of the server's pool now and stay
 * resident.  Each tile takes up to tile_cases pending requests and advances
 * one tree layer per tick -- collect layers from the deepest to the root,
 * then distribute layers from the root, then its log P(e) and posterior
 * kernels -- and one tick is two launches over every active tile, each at
 * its own layer.  A request arriving while other tiles are mid-pass starts
 * at the next tick, in a free tile, instead of waiting for a whole pass.
 * Up to eight ticks of a plan are enqueued ahead (phases advance on the
 * host), so ticks run back to back; they run on a stream of the
 * highest priority, so their blocks are dispatched ahead of the batch
 * slots' passes.  Results are the same bit for
 * bit as the batch-slot path's (same kernels per tile, fixed per-case
 * reduction order).  Allocates the plan's staging buffers and stream.
 * JT_ENOMEM when the tiles do not fit the free part of the pool.  The plan
 * must not be given a new work shape while the server holds it.
 */
JT_API jt_status jt_server_add_plan_rolling(jt_server *srv, jt_plan *plan, int32_t tiles, int32_t *plan_id);
/*
 * Queue one case.  evidence: int32 [n_vars of the plan]; query_vars: the
 * variables whose posteriors the caller wants (n_query entries, or NULL and
 * 0 for all).  Returns a ticket.
 */
JT_API jt_status jt_submit(jt_server *srv, int32_t plan_id, const int32_t *evidence,
                    const int32_t *query_vars, int32_t n_query, uint64_t *ticket);
/*
 * Fetch a result: JT_EBUSY while pending.  post receives the posteriors of
 * the queried variables concatenated in query order (all variables, in
 * layout of the plan's sum(card) row, when the query was NULL).  On JT_OK
 * the ticket is released.
 */
JT_API jt_status jt_poll(jt_server *srv, uint64_t ticket, double *log_pe, double *post,
                  int32_t *case_status);
/* Block until every submitted request has completed. */
JT_API jt_status jt_server_drain(jt_server *srv);
/*
 * Counters (out holds 9 entries): out[0] completed requests, out[1] batches
 * launched, out[2] largest batch, out[3] peak pool bytes in use, out[4] p50
 * latency (ns), out[5] p99 latency (ns), out[6] requests pending or in
 * flight, out[7] batch slots created (regions of the pool bound to a plan),
 * out[8] slots evicted to make room for another plan's.  Latency is
 * submit -> result ready on the host.
 */
JT_API jt_status jt_server_stats(jt_server *srv, int64_t *out);
/*
 * Counters of one plan (out holds 4 entries): out[0] completed requests,
 * out[1] batches launched, out[2] p50 latency (ns), out[3] p99 latency
 * (ns).  JT_ENOTFOUND for an unknown plan id.
 */
JT_API jt_status jt_server_plan_stats(jt_server *srv, int32_t plan_id, int64_t *out);
/*
 * Scheduling class of a batch-slot plan: high != 0 runs its batches on
 * streams of the highest priority, so when SMs free up the blocks of its
 * passes are dispatched before those of default-priority batches (a small
 * plan's short passes then need not wait behind a large plan's many
 * blocks).  Default 0; applies to batches launched after the call; results
 * do not depend on it.  Rolling plans always run at the highest priority.
 * JT_ENOTFOUND for an unknown plan id.  Serving has no counterpart in the
 * paper (Section 2 runs one query at a time).
 */
JT_API jt_status jt_server_set_priority(jt_server *srv, int32_t plan_id, int32_t high);
/*
 * Forget the latency samples collected so far (for every plan), e.g. after
 * a warm-up; the counters and the resident slots are kept.
 */
JT_API jt_status jt_server_reset_latency(jt_server *srv);
JT_API void jt_server_destroy(jt_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* JT_H */
