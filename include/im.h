/*
 * im.h -- C ABI of the GB300 (sm_103a) fused-sampling influence-maximization
 * library (INFuseR-MG hot path of Goktürk & Kaya, arXiv 2008.03095).
 *
 * Problem (Section 2.1): given an undirected graph G = (V, E), a seed-set size
 * K and R Monte-Carlo simulations under the independent-cascade model with a
 * uniform edge probability p, choose S (|S| = K) greedily to maximize the
 * estimated spread sigma(S).
 *
 * Sampling (Section 3.1, Eq. 1-2): edge {u,v} is live in simulation r iff
 *     (uint64)(X_r XOR h(u,v)) < T,   T = floor(p * 2^32)
 * where h(u,v) = MurmurHash3_x86_32 of the 8-byte key min(u,v) || max(u,v)
 * (little-endian uint32 halves, seed 0) and X_0..X_{R-1} are the first R
 * outputs of MT19937 seeded with rng_seed (the std::mt19937 sequence). No
 * sampled graph is ever stored: every arc is decided when it is read.
 *
 * Estimate: sigmaR(S) = sum over r of |vertices reachable from S in sample r|
 * (an integer; sigma = sigmaR / R). Seeds follow Algorithm 7: component labels
 * of every sample (Algorithm 5), memoized component sizes (Section 3.3), then
 * greedy/CELF selection of marginal gains summed over the R samples, ties
 * broken by the lowest vertex id. out_sigma_R[k] is sigmaR of the first k+1
 * seeds.
 *
 * Conventions
 *   - Every function returns IM_OK (0) or a negative IM_E* code; on error no
 *     output is written and im_last_error() describes the failure.
 *   - Vertex ids are int32 in [0, n). CSR: xadj[n+1], adj[2m], xadj[0] = 0,
 *     xadj non-decreasing, xadj[n] = 2m, every arc (u,v) has a reverse arc
 *     (v,u). Self-loops are accepted and ignored; duplicate arcs are accepted.
 *     Neighbour lists need not be sorted (unsorted lists are sorted once, on
 *     the host, at graph creation).
 *   - Limits: 1 <= n < 2^31, 2m < 2^31, 1 <= R <= 65536, n * R < 2^32,
 *     0 <= K <= n, 0 <= p <= 1 (NaN rejected).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the device the graph was created on.
 *   - Work is queued on the calling thread's stream (im_set_stream; default:
 *     the legacy default stream). Blocking calls synchronize that stream.
 *   - Graph handles are read-only after creation. Blocking calls on one graph
 *     from several threads are serialized internally; workspaces are not
 *     thread-safe (one workspace per concurrent query stream).
 */
#ifndef IM_GB300_IM_H
#define IM_GB300_IM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  IM_OK = 0,
  IM_EINVAL = -1,    /* invalid argument or malformed graph */
  IM_ENOMEM = -2,    /* device allocation failed; handles stay valid */
  IM_ECUDA = -3,     /* CUDA runtime error */
  IM_ETIMEOUT = -4,  /* a device loop exceeded its iteration budget */
  IM_EBUSY = -5,     /* resource in use */
  IM_EINTERNAL = -6  /* internal invariant violated */
};

typedef struct im_graph im_graph;         /* opaque, library-owned */
typedef struct im_workspace im_workspace; /* opaque, library-owned */

/* ---------------------------------------------------------------- graphs */

/* The influence graph G = (V, E) of the problem statement (Section 2.1),
 * undirected, held in the CSR form every algorithm of the paper reads
 * (Section 3.4, implementation details: xadj[v] is where v's neighbours
 * start in adj; every undirected edge appears as two arcs).
 * Validate a symmetric CSR (host arrays, see Conventions) and copy it to the
 * current device, where it stays resident until im_graph_destroy. The
 * library also derives the upper-triangle edge list {u < v} used by the
 * component kernel. Blocking. The caller keeps ownership of xadj/adj.
 * Errors: IM_EINVAL (bad CSR: ranges, ids, asymmetry), IM_ENOMEM, IM_ECUDA. */
int im_graph_create(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                    im_graph **out);

/* Same as im_graph_create, with a probability per edge instead of one uniform
 * p (the w_{u,v} of Algorithm 2 and Eq. 2, Section 4's weight settings):
 * w[2m] is a host array with one value per CSR arc, in [0, 1] (NaN
 * rejected), and both orientations of an edge carry the same value (for
 * duplicate arcs: the same multiset of values). Each weight becomes the
 * threshold code c = floor(w * 2^32) of Eq. 2, where the largest 32-bit code
 * means "always live" (so w >= 1 - 2^-32 is certain); the codes stay on the
 * device with the graph (4 bytes per arc and per edge). Queries use them
 * when called with IM_SAMPLE_EDGE_WEIGHTS; plain queries still take p.
 * Errors: as im_graph_create, and IM_EINVAL for out-of-range or asymmetric
 * weights. */
int im_graph_create_weighted(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                             const double *w, im_graph **out);

/* Release a graph of Section 2.1 and its device memory (its CSR copy, edge
 * list, weight codes and internal workspace). Workspaces, batches and
 * servers built on it must be destroyed first. Errors: IM_EINVAL (null). */
int im_graph_destroy(im_graph *g);

/* Number of vertices and undirected edges (m = len(adj) / 2). */
int im_graph_info(const im_graph *g, int32_t *n, int64_t *m);

/* ---------------------------------------------------------------- queries */

/* Select K seeds (Algorithm 7, INFuseR-MG): fused sampling + component labels
 * of all R samples, memoized sizes, first-seed gains mg_v = sum_r |C_r(v)|,
 * then exact CELF. out_seeds[K] and out_sigma_R[K] are host arrays owned by
 * the caller; out_sigma_R[k] = sigmaR({s_0..s_k}). Blocking.
 * Errors: IM_EINVAL (K, R, p out of range), IM_ENOMEM, IM_ECUDA, IM_ETIMEOUT. */
int im_select_seeds(const im_graph *g, int32_t K, int32_t R, double p, uint32_t rng_seed,
                    int32_t *out_seeds, uint64_t *out_sigma_R);

/* Spread of a given seed set (Algorithm 4 evaluated on the same fixed hash
 * samples, Eq. 2): *out_sigma_R = sum_r |union_{s in S} C_r(s)|. seeds is a
 * host array of num_seeds ids; duplicates count once. Blocking. */
int im_estimate_spread(const im_graph *g, const int32_t *seeds, int32_t num_seeds, int32_t R,
                       double p, uint32_t rng_seed, uint64_t *out_sigma_R);

/* Options of the _ex queries (bit flags):
 *   IM_SAMPLE_EDGE_WEIGHTS  sample edge {u,v} with the graph's own w(u,v)
 *                           (im_graph_create_weighted); p is ignored
 *   IM_SAMPLE_MIXED_HASH    live iff fmix32(X_r XOR h(u,v)) < T, fmix32 being
 *                           MurmurHash3's finalizer: with the plain XOR of
 *                           Eq. 2, edges whose hashes differ above T's
 *                           magnitude are never live in the same sample; the
 *                           mix makes co-sampling rates match independent
 *                           edges (a variant of this library, not the paper's
 *                           scheme; every lane is then tested for every edge)
 *   IM_ALGO_FUSED_SAMPLING  select only: the FusedSampling variant the paper
 *                           measures in Section 4 (Table 4): the same fused
 *                           hash sampling, but one simulation at a time and no
 *                           memoized labels -- the NewGreedy step runs R
 *                           single-simulation component passes, and every CELF
 *                           re-evaluation recomputes the spread of S + {u}
 *                           over the R samples one by one (Algorithm 3's
 *                           RandCas on the fixed samples). Same seeds and
 *                           sigma*R as the default path; a baseline of cost.
 * The options combine, except that IM_ALGO_FUSED_SAMPLING is blocking only. */
enum {
  IM_SAMPLE_EDGE_WEIGHTS = 1,
  IM_SAMPLE_MIXED_HASH = 2,
  IM_ALGO_FUSED_SAMPLING = 4
};

/* im_select_seeds / im_estimate_spread with options (flags above). */
int im_select_seeds_ex(const im_graph *g, int32_t K, int32_t R, double p, uint32_t rng_seed,
                       uint32_t flags, int32_t *out_seeds, uint64_t *out_sigma_R);
int im_estimate_spread_ex(const im_graph *g, const int32_t *seeds, int32_t num_seeds, int32_t R,
                          double p, uint32_t rng_seed, uint32_t flags, uint64_t *out_sigma_R);

/* Limits of im_estimate_spread_noalloc (the size of its static scratch). */
#define IM_NOALLOC_MAX_N 32768      /* vertices; also the largest num_seeds */
#define IM_NOALLOC_MAX_EDGES 524288 /* undirected edges m */
#define IM_NOALLOC_MAX_R 256        /* samples */

/* The same result as im_estimate_spread, computed without allocating any
 * device memory during the call. The paper has no counterpart: this is an
 * interface of this library, for callers that must not allocate, such as code
 * that runs while another allocator (a framework's caching pool) holds nearly
 * all free device memory, so that cudaMalloc would fail, or a latency-bound
 * loop in which cudaFree would synchronize the whole device.
 * All device scratch lives in one static region of the library's device code
 * (about 6.4 MiB, reserved when that code is loaded on a device), so inputs
 * are capped: g->n <= IM_NOALLOC_MAX_N, m <= IM_NOALLOC_MAX_EDGES,
 * R <= IM_NOALLOC_MAX_R, num_seeds <= IM_NOALLOC_MAX_N. Larger inputs return
 * IM_EINVAL before any device work.
 * The first call on a device looks the region up (which may load the
 * library's device code); make that first call before any stream capture.
 * Every call on a device uses the same region: calls that overlap in time, for
 * example from two host threads, race on it and return wrong results.
 * seeds is a host array of num_seeds ids (duplicates count once);
 * *out_sigma_R is written on the host. Runs on the thread's stream; blocking.
 * Errors: IM_EINVAL (limits, R, p, seed ids, null arguments), IM_ECUDA. */
int im_estimate_spread_noalloc(const im_graph *g, const int32_t *seeds, int32_t num_seeds,
                               int32_t R, double p, uint32_t rng_seed, uint64_t *out_sigma_R);

/* ---------------------------------------------------------------- async API */

/* Device scratch for queries with R <= R_max on graph g (about
 * n*R*4 + n*R/8 + 8n bytes). Owned by the library until destroyed. */
int im_workspace_create(const im_graph *g, int32_t R_max, im_workspace **out);
int im_workspace_destroy(im_workspace *ws);

/* Same as im_select_seeds, queued on the thread's stream without
 * synchronizing: d_seeds[K] (int32) and d_sigma_R[K] (uint64) are DEVICE
 * arrays owned by the caller. Device-side failures are recorded in the
 * workspace and reported by im_workspace_status. */
int im_select_seeds_async(const im_graph *g, im_workspace *ws, int32_t K, int32_t R, double p,
                          uint32_t rng_seed, int32_t *d_seeds, uint64_t *d_sigma_R);

/* Same as im_estimate_spread with DEVICE d_seeds[num_seeds] and DEVICE
 * d_sigma_R[1]; queued without synchronizing. Seed ids are checked on the
 * device (an out-of-range id sets IM_EINVAL in the workspace status). */
int im_estimate_spread_async(const im_graph *g, im_workspace *ws, const int32_t *d_seeds,
                             int32_t num_seeds, int32_t R, double p, uint32_t rng_seed,
                             uint64_t *d_sigma_R);

/* The async queries with options (IM_SAMPLE_* flags only). */
int im_select_seeds_ex_async(const im_graph *g, im_workspace *ws, int32_t K, int32_t R, double p,
                             uint32_t rng_seed, uint32_t flags, int32_t *d_seeds,
                             uint64_t *d_sigma_R);
int im_estimate_spread_ex_async(const im_graph *g, im_workspace *ws, const int32_t *d_seeds,
                                int32_t num_seeds, int32_t R, double p, uint32_t rng_seed,
                                uint32_t flags, uint64_t *d_sigma_R);

/* ---------------------------------------------------------------- batches
 * Many independent select queries -- each its own graph, K, R, p, options --
 * in ONE persistent kernel launch: the steps of Algorithm 7 (lane randoms,
 * label init, fused sample + union, size memo, first gains, lazy greedy) are
 * cut into work items (query, phase, tile) that the blocks of the launch take
 * in phase order from a device queue, waiting with an iteration budget for
 * the items they depend on. Every query's seeds and sigma*R are those of
 * im_select_seeds_ex on its own. The launch is an ordinary one (no
 * co-residency needed), so im_batch_run_async can be captured in a CUDA graph.
 * The tiling of each query's work (label slots, edges, size-memo tiles and
 * vertices per item) comes from the autotuner's cache for the query's size
 * class, or a default; im_batch_autotune fills the cache by timing.
 * All graphs of a batch are on one device; graphs must outlive the batch. */
typedef struct im_batch im_batch; /* opaque, library-owned */
typedef struct {
  int32_t graph;     /* index into the graphs array of im_batch_create */
  int32_t K;         /* 1 <= K <= n */
  int32_t R;         /* 1 <= R <= 16384 (a batch keeps the lane sort and pool on chip) */
  double p;          /* as im_select_seeds (ignored with IM_SAMPLE_EDGE_WEIGHTS) */
  uint32_t rng_seed;
  uint32_t flags;    /* IM_SAMPLE_* */
} im_batch_query;

/* Validate the queries and allocate every query's tables in one device
 * arena (n*R*4 + n*R/8 + 9n bytes and a few KB per query); host arrays are
 * copied. Errors: IM_EINVAL, IM_ENOMEM (the arena does not fit). */
int im_batch_create(const im_graph *const *graphs, int32_t num_graphs,
                    const im_batch_query *queries, int32_t count, im_batch **out);
int im_batch_destroy(im_batch *b);

/* Queue one run of all queries on the thread's stream: four small resets
 * and one persistent launch of one 1024-thread block per SM. A query's large
 * bound refreshes are cut into chunks that blocks without other work claim,
 * so the largest lazy greedies do not run on one SM alone. Runs may repeat;
 * each overwrites the results. */
int im_batch_run_async(im_batch *b);

/* Synchronize the thread's stream and copy the results to host arrays:
 * out_seeds / out_sigma_R hold sum(K) entries, query i's K values at offset
 * K_0 + ... + K_{i-1}; out_status (may be NULL) gets each query's device
 * status (IM_OK, IM_ETIMEOUT, IM_EINTERNAL). Returns the first non-OK status. */
int im_batch_results(im_batch *b, int32_t *out_seeds, uint64_t *out_sigma_R, int32_t *out_status);

/* Work counters of one query of the last run (IM_STAT_* layout). */
int im_batch_query_stats(im_batch *b, int32_t query, int64_t *out);

enum {
  IM_BATCH_INFO_QUERIES = 0,
  IM_BATCH_INFO_ITEMS = 1,        /* work items of one run */
  IM_BATCH_INFO_DEVICE_BYTES = 2, /* arena size */
  IM_BATCH_INFO_TOTAL_K = 3,
  IM_BATCH_INFO_LEVELS = 4,       /* histogram of tiling levels: 4 bits per level 0..4 */
  IM_BATCH_INFO_SCHEDULE = 5,     /* queries per schedule group (1: query by query; all: phase
                                     by phase) */
  IM_BATCH_INFO_COUNT = 6
};
int im_batch_info(const im_batch *b, int64_t *out);

/* SM cycles of the last run, summed over blocks: out[0..5] waiting for
 * dependencies and out[6..11] working, for the phases lanes, init, union,
 * compress, gains, lazy greedy; out[12] refresh chunks done for other
 * queries' lazy greedies. 13 int64 values. */
int im_batch_phase_cycles(im_batch *b, int64_t *out);

/* Autotune: for each size class (floor(log2(n*R)), R, flags) of the batch,
 * time up to four of its largest queries as a batch of their own at each of
 * five tiling granularities (trials timed runs each, after a warm-up) and keep
 * the fastest in a process-wide cache; then time b's item orders (queries,
 * largest first, in groups of 1, 2, 4, 8, 16, 32, 64 or all, each group phase
 * by phase) and keep the fastest for b.
 * Later batches of the same classes use the cache. The cache can be saved to
 * and loaded from a text file. */
int im_batch_autotune(im_batch *b, int32_t trials);
int im_autotune_cache_save(const char *path);
int im_autotune_cache_load(const char *path);
int im_autotune_cache_clear(void);

/* ---------------------------------------------------------------- serving
 * A serving loop over a resident pool of graphs: influence queries arrive at
 * any time (any thread) and a scheduler thread of the library admits them in
 * arrival order as soon as one of `slots` CUDA streams is free and the
 * query's workspace fits the memory budget (workspaces are pooled per graph
 * and reused; idle ones are freed least recently used first when a new one
 * would exceed the budget). Queries that arrive while others are on the GPU
 * are admitted into the running mix and their kernels overlap on the device
 * (continuous batching, not a queue in front of one query at a time). Each
 * query runs exactly the kernels of its blocking call, so its result is the
 * same alone and in the mix. This is an interface of this library; the paper
 * has none (it runs one query at a time). */
typedef struct im_server im_server; /* opaque, library-owned */
enum { IM_REQUEST_SELECT = 0, IM_REQUEST_SPREAD = 1 };
typedef struct {
  int32_t kind;          /* IM_REQUEST_SELECT or IM_REQUEST_SPREAD */
  int32_t graph;         /* index into the server's graphs */
  int32_t K;             /* select: seeds to choose (1..n); spread: seeds given (0..n) */
  int32_t R;
  double p;
  uint32_t rng_seed;
  uint32_t flags;        /* IM_SAMPLE_* */
  const int32_t *seeds;  /* spread: K host ids, copied at submission */
} im_request;

/* graphs: num_graphs handles on one device, which must outlive the server.
 * slots: queries on the GPU at once (1..256); memory_budget: bytes of device
 * memory the pooled workspaces may take. Starts the scheduler thread. */
int im_server_create(const im_graph *const *graphs, int32_t num_graphs, int32_t slots,
                     int64_t memory_budget, im_server **out);

/* Queue a query; *ticket identifies it. Thread-safe. Errors: IM_EINVAL (bad
 * query), IM_ENOMEM (its workspace alone exceeds the budget), IM_EBUSY
 * (server shutting down). */
int im_server_submit(im_server *s, const im_request *r, uint64_t *ticket);

/* Wait up to timeout_us (0: just poll, < 0: until done) for a query. Done:
 * select writes out_seeds[K] and out_sigma_R[K] (cumulative), spread writes
 * out_sigma_R[0]; out_times (may be NULL) gets the seconds since server
 * creation at submission, admission and completion; the ticket is released
 * and the query's own status returned. Not done: IM_EBUSY, ticket kept. */
int im_server_wait(im_server *s, uint64_t ticket, int64_t timeout_us, int32_t *out_seeds,
                   uint64_t *out_sigma_R, double *out_times);

enum {
  IM_SERVER_STAT_SUBMITTED = 0,
  IM_SERVER_STAT_ADMITTED = 1,
  IM_SERVER_STAT_COMPLETED = 2,
  IM_SERVER_STAT_IN_FLIGHT = 3,
  IM_SERVER_STAT_IN_FLIGHT_PEAK = 4,
  IM_SERVER_STAT_QUEUED = 5,
  IM_SERVER_STAT_QUEUE_PEAK = 6,
  IM_SERVER_STAT_WS_CREATED = 7,
  IM_SERVER_STAT_WS_EVICTED = 8,
  IM_SERVER_STAT_POOL_BYTES = 9,
  IM_SERVER_STAT_POOL_BYTES_PEAK = 10,
  IM_SERVER_STAT_BUDGET = 11,
  IM_SERVER_STAT_COUNT = 12
};
int im_server_stats(im_server *s, int64_t *out);

/* Finish every queued and running query, then free the server. */
int im_server_destroy(im_server *s);

/* Synchronize the thread's stream and return (then clear) the first device
 * status recorded in ws since the last call: IM_OK, IM_EINVAL, IM_ETIMEOUT or
 * IM_EINTERNAL. */
int im_workspace_status(im_workspace *ws);

/* Work counters accumulated by the device since the last call (synchronizes
 * the thread's stream, then clears them): */
enum {
  IM_STAT_CELF_ROUNDS = 0,       /* pool evaluation rounds of the lazy greedy */
  IM_STAT_CELF_EVALUATIONS = 1,  /* exact marginal-gain evaluations */
  IM_STAT_CELF_EXTRACTIONS = 2,  /* candidate prefixes extracted from the bounds */
  IM_STAT_SPREAD_LEVELS = 3,     /* BFS levels of the spread estimates */
  IM_STAT_CELF_CYC_EXTRACT = 4,  /* SM clock cycles of the CELF block in prefix extraction */
  IM_STAT_CELF_CYC_EVAL = 5,     /* ... in exact gain evaluation */
  IM_STAT_CELF_CYC_COMMIT = 6,   /* ... in commits and pool updates */
  IM_STAT_CELF_CYC_MERGE = 7,    /* ... in merging survivors back */
  IM_STAT_CELF_REFRESHES = 8,    /* grid-wide recomputations of all exact gains */
  IM_STAT_CELF_CYC_COMMITS = 9,  /* ... in the commit loop (picks, pool updates) */
  IM_STAT_CELF_CYC_COVER = 10,   /* ... marking committed components covered */
  IM_STAT_CELF_REFRESHED = 11,   /* vertices re-evaluated by the refreshes */
  IM_STAT_CELF_CYC_REFRESH = 12, /* batched lazy greedy: SM cycles in bound refreshes (a batch
                                    query's IM_STAT_CELF_CYC_EVAL holds its whole item) */
  IM_STAT_CHECK_CODE = 13,       /* first failed internal invariant check (0 = none) */
  IM_STAT_CHECK_V0 = 14,         /* ... and two values describing it */
  IM_STAT_CHECK_V1 = 15,
  IM_STAT_SPREAD_COMPONENTS = 16, /* spread estimates finished from the samples' components
                                     (a BFS frontier passed n/16 vertices, on a table larger
                                     than L2 with n R < 112 m) */
  IM_STAT_MEMO_ACCUMULATORS = 17, /* size memos run with per-warp root-count accumulators (a
                                     sampled component held more than 4.5% of the vertices) */
  IM_STAT_MEMO_LIVE = 18,         /* ... of those, walking only the listed non-root slots (fewer
                                     than 15% of the sampled slots were non-roots) */
  IM_NUM_STATS = 19
};
/* out: host array of IM_NUM_STATS int64 values. */
int im_workspace_stats(im_workspace *ws, int64_t *out);

/* ---------------------------------------------------------------- misc */

/* Thread-local description of the last failure of this thread (valid until
 * the thread's next library call). Never NULL. */
const char *im_last_error(void);

/* Set the calling thread's CUDA stream (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream); NULL selects the legacy default
 * stream. */
int im_set_stream(void *cuda_stream);

/* Host-only helper: the sampling threshold T = floor(p * 2^32) of Eq. 2 for
 * p in [0, 1]; returns IM_EINVAL for p outside [0, 1] or NaN. */
int im_sampling_threshold(double p, uint64_t *out_T);

/* ---------------------------------------------------------------- profiling
 * Optional per-phase timing of the calling thread's queries: when enabled,
 * every kernel the library launches is bracketed by CUDA events recorded on
 * the same stream. Phases: */
enum {
  IM_PHASE_PREP = 0,         /* X_r draw, lane order, label-table init */
  IM_PHASE_UNION = 1,        /* fused hash-sample + component hooking */
  IM_PHASE_COMPRESS = 2,     /* root pointers + size memo */
  IM_PHASE_GAINS = 3,        /* first-seed gains mg_v */
  IM_PHASE_CELF = 4,         /* on-device lazy greedy */
  IM_PHASE_SPREAD_PREP = 5,  /* X_r draw and lane order for the spread */
  IM_PHASE_SPREAD = 6,       /* bit-parallel multi-source BFS */
  IM_PHASE_SPREAD_CC = 7,    /* the spread's hand-over to components, last kernel: the
                                slots whose root is marked, counted */
  IM_PHASE_SPREAD_UNION = 8, /* ... its union (the select path's kernel) */
  IM_PHASE_SPREAD_MARK = 9,  /* ... the seeds' roots marked in every sample; the three are
                                queued behind the BFS where a hand-over can pay and return
                                at once unless the BFS handed over */
  IM_NUM_PHASES = 10
};

/* on != 0 starts recording (and clears earlier records); 0 stops. */
int im_profile_enable(int on);

/* Synchronize the recorded events and return, per phase, the summed kernel
 * time in milliseconds and the number of launches since the last enable or
 * read (host arrays of IM_NUM_PHASES entries, either may be NULL); clears the
 * records. */
int im_profile_read(double *total_ms, int64_t *launches);

/* Number of kernels this library has launched in this process (all threads). */
uint64_t im_kernel_launches(void);

/* ---------------------------------------------------------------- test hooks
 * Test-only exports used to compare intermediate tables with the oracle. All
 * outputs are host arrays owned by the caller; all calls are blocking. */

/* Component labels of all R samples in the paper's layout: out[v*R + r] is
 * the minimum vertex id of v's component in sample r (Algorithm 5 fixpoint). */
int im_debug_labels(const im_graph *g, int32_t R, double p, uint32_t rng_seed,
                    int32_t *out_labels);

/* Labels and size memo of selected simulations only (for full-size graphs
 * whose whole table is too large to copy): lanes[k] in [0, R) are simulation
 * indices; out_labels[v*num_lanes + k] is the label of v in simulation
 * lanes[k] and out_sizes[v*num_lanes + k] the size of the component rooted at
 * v there (0 if v is not a root). Host arrays of n*num_lanes entries. */
int im_debug_tables_lanes(const im_graph *g, int32_t R, double p, uint32_t rng_seed,
                          const int32_t *lanes, int32_t num_lanes, int32_t *out_labels,
                          uint32_t *out_sizes);

/* Labels and sizes (layouts of im_debug_labels / im_debug_sizes) under the
 * sampling options (IM_SAMPLE_* flags); either output may be NULL. */
int im_debug_tables_ex(const im_graph *g, int32_t R, double p, uint32_t rng_seed, uint32_t flags,
                       int32_t *out_labels, uint32_t *out_sizes);

/* First-seed marginal gains of the NewGreedy step (Algorithm 5, final loop):
 * out_mg[v] = sum_r |C_r(v)|, the n values the lazy greedy starts from, as
 * the device computed them (host array of n uint64 values). */
int im_debug_first_gains(const im_graph *g, int32_t R, double p, uint32_t rng_seed,
                         uint64_t *out_mg);

/* Size memo (Section 3.3): out[l*R + r] = #{v : label of v in sample r is l},
 * zero where l is not a component label of sample r. */
int im_debug_sizes(const im_graph *g, int32_t R, double p, uint32_t rng_seed,
                   uint32_t *out_sizes);

/* The per-simulation random values X_0..X_{R-1} as drawn on the device. */
int im_debug_lane_randoms(int32_t R, uint32_t rng_seed, uint32_t *out_X);

/* Edge hashes h(u[i], v[i]) (Eq. 1) computed by the device hash routine. */
int im_debug_edge_hash(const int32_t *u, const int32_t *v, int64_t count, uint32_t *out_h);

/* Seed selection with an explicit live mask instead of the hash sampler:
 * mask[a*R + r] != 0 iff CSR arc a is live in sample r (both orientations of
 * an edge must agree). out_labels[n*R] / out_sizes[n*R] may be NULL. Used to
 * feed the worked example of Figures 3-4 and brute-force enumerations. */
int im_debug_select_seeds_masked(const im_graph *g, int32_t K, int32_t R, const uint8_t *mask,
                                 int32_t *out_seeds, uint64_t *out_sigma_R,
                                 int32_t *out_labels, uint32_t *out_sizes);

/* Spread with an explicit live mask (same layout as above). */
int im_debug_estimate_spread_masked(const im_graph *g, const int32_t *seeds, int32_t num_seeds,
                                    int32_t R, const uint8_t *mask, uint64_t *out_sigma_R);

/* Test-only, process-wide overrides of launch shapes, loop budgets and
 * allocation outcomes, so that tests can drive the paths a healthy run never
 * takes. value 0 restores the library's own choice. Keys: */
enum {
  IM_OVR_CELF_CLUSTER = 0,     /* lazy-greedy launch: -1 = plain cooperative launch without a
                                  cluster attribute; c in {1, 2, 4, 8} = clusters of c blocks */
  IM_OVR_CELF_ROUND_CAP = 1,   /* budget of lazy-greedy rounds (exceeded: IM_ETIMEOUT) */
  IM_OVR_UF_CAP = 2,           /* budget of each union-find walk (exceeded: IM_ETIMEOUT) */
  IM_OVR_SPREAD_LEVEL_CAP = 3, /* budget of spread BFS levels (exceeded: IM_ETIMEOUT) */
  IM_OVR_FAIL_ALLOC = 4,       /* the value-th device allocation from now fails as if the
                                  device were out of memory (1 = the next one); one shot */
  IM_OVR_CELF_REFRESH_AFTER = 5, /* lazy greedy: exact evaluations without a commit before all
                                    gains are recomputed (any value keeps the result exact) */
  IM_OVR_BATCH_GROUP = 6,        /* batches planned from now: queries per schedule group */
  IM_OVR_CELF_EXT_REFRESH = 7,   /* lazy greedy's bulk refresh as a launch of its own: 1 always,
                                    2 never (0: above 2^20 vertices) */
  IM_NUM_OVERRIDES = 8
};
/* Errors: IM_EINVAL (unknown key, or a value outside the key's range). */
int im_debug_override(int32_t key, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* IM_GB300_IM_H */
