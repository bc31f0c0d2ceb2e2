/*
 * pg.h -- C ABI of a single-GPU (GB300, sm_103a) library that builds and
 * searches proximity graphs with the construction framework of
 * "Revisiting the Index Construction of Proximity Graph-Based Approximate
 * Nearest Neighbor Search" (arXiv 2410.01231).
 *
 * Problem (Section 2): a dataset D of n points in R^d, row-major float32
 * [n][d]; k-ANN search returns the k points with smallest distance to a
 * query.  Symbols follow the paper: K = k0 (out-degree of the initial
 * KNNG), L = pool width of the candidate search, R = the out-degree bound
 * M of the pruned graph, alpha = the angle of alpha-pruning.
 *
 * Distances.  s(x, y) is the squared L2 distance (PG_METRIC_L2SQ), or for
 * unit-norm rows the squared chord s = max(0, 2 - 2<x,y>) (PG_METRIC_COSINE
 * and PG_METRIC_IP: on the unit sphere both rank like -<x,y>; rows are not
 * normalised by the library).  Every list is ordered by the pair
 * (s, id) ascending; ids are int32 (n < 2^31); unused slots hold id -1.
 *
 * Exactness.  Kernels decide every comparison in FP32 and re-decide in
 * FP64, with the sequential coordinate-order sum of the CPU reference,
 * every decision whose FP32 margin is inside a rigorous rounding bound, so
 * pruned lists equal those of an FP64 evaluation of the same rule.
 *
 * Memory and streams.  Unless a parameter says "host", every pointer is a
 * DEVICE pointer owned by the caller; the library never frees caller
 * memory.  All work is queued on the stream given to pg_ctx_create; calls
 * that return host-side results (stats, counts, indexes) synchronise that
 * stream.  Scratch memory is taken from the stream-ordered allocator and
 * counted against the context's HBM budget.
 *
 * Errors.  Every entry point returns a pg_status.  Invalid arguments are
 * reported before any work is queued.  Kernels that meet an invalid input
 * (an id outside [-1, n)) skip it and record it in a device error word,
 * which the next synchronising call (or pg_ctx_sync) turns into
 * PG_ERR_DEVICE_CHECK.  pg_last_error() gives a one-line message.  No
 * exception crosses this boundary.
 *
 * Threads.  A context is used by one thread at a time.  Searches of one
 * index (pg_search, pg_search_host) may run concurrently from several
 * threads on different contexts, as the serving loop's workers do; builds,
 * pruning and insertion set per-kernel launch attributes and are not made
 * safe against each other across threads.  An index is not modified while
 * it is searched: insertion and growth need exclusive use (the serving
 * loop orders them).
 */
#ifndef PG_H
#define PG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PG_OK = 0,
    PG_ERR_INVALID_ARG = 1, /* argument outside its documented range     */
    PG_ERR_OOM = 2,         /* device allocation failed                   */
    PG_ERR_CUDA = 3,        /* a CUDA runtime call failed                 */
    PG_ERR_TIMEOUT = 4,     /* a bounded device wait ran out              */
    PG_ERR_CAPACITY = 5,    /* input larger than a documented capacity    */
    PG_ERR_BUDGET = 6,      /* scratch would exceed the context HBM budget */
    PG_ERR_INTERNAL = 7,    /* invariant broken inside the library         */
    PG_ERR_DEVICE_CHECK = 8, /* a kernel met an invalid id (skipped)       */
    PG_ERR_IO = 9            /* a file could not be opened, read or written */
} pg_status;

typedef enum { PG_METRIC_L2SQ = 0, PG_METRIC_COSINE = 1, PG_METRIC_IP = 2 } pg_metric;

/* PG_PREC_FP32: distances in FP32 (FP64 recheck near margins).
 * PG_PREC_BF16_SCREEN: distance tiles / gathers from a BF16 copy of D with
 * FP32 accumulation; decisions inside the BF16 error bound are redone in
 * FP32 and then FP64, so results equal the FP32 form's.
 * PG_PREC_FP8_SCREEN: queries only (pg_search, pg_search_host, serving):
 * the base-layer beam search ranks by distances from an FP8 E4M3 copy of
 * the index's points (one FP32 scale per row, the row's largest magnitude
 * mapped to 448; squared L2 to the decoded row, or the chord from its dot
 * product with the query), then the final pool is re-measured in FP32 and
 * its k best returned:
 * returned distances are FP32, membership is approximate (recall).  Every
 * other entry point refuses it with PG_ERR_INVALID_ARG. */
typedef enum {
    PG_PREC_FP32 = 0,
    PG_PREC_BF16_SCREEN = 1,
    PG_PREC_FP8_SCREEN = 2
} pg_precision;

typedef struct pg_ctx pg_ctx;
typedef struct pg_index pg_index;

/* Counters of one pruning call (host struct filled on return). */
typedef struct {
    int64_t rows;               /* points pruned                              */
    int64_t candidates;         /* distinct candidates after de-duplication   */
    int64_t scanned;            /* candidates visited before the R-stop       */
    int64_t occlusion_tests;    /* (v, w) pairs evaluated                     */
    int64_t fp64_rechecks;      /* decisions re-made in FP64                   */
    int64_t fp64_flips;         /* ... whose FP64 outcome differed from FP32's */
    int64_t edges;              /* kept edges (sum of out-degrees)            */
    int64_t long_rows;          /* rows handled by the long-row kernel        */
    int64_t near_ties;          /* decisions with relative margin < 1e-5 (counted
                                   only when pg_ctx_set_tie_count is on)        */
} pg_prune_stats;

/* Parameters of the graph builds (pg_default_params fills the defaults). */
typedef struct {
    pg_metric metric;
    pg_precision precision;
    int32_t K;               /* k0: degree of the exact initial KNNG (Alg. 6)   */
    int32_t L;               /* pool width of the k-CNA search (Alg. 5); ef    */
    int32_t R;               /* degree bound M of the RNG graph / NSWG layer 0     */
    int32_t M;               /* NSWG upper-layer degree bound and level base       */
    double alpha_deg;        /* alpha of the OptKCNA refinements (Section 4.1)     */
    double alpha_final_deg;  /* alpha of the final refinement; 60 = RNG pruning    */
    int32_t iters;           /* I: OptKCNA iterations (Alg. 6; paper default 2)     */
    int32_t connect_final;   /* RNG build: connectivity step after the final prune  */
    int32_t route_layers;    /* RNG build: add NSWG upper layers for query routing  */
    uint64_t seed;           /* level draw (SplitMix64, seed XOR id)                */
    int32_t reuse_pruning;   /* K2P (Section 5.4): a refinement whose angle is >= the
                                previous one's tests a candidate the previous pass kept
                                only against new members (same lists, fewer tests) */
    double quality_target;   /* > 0: quality examination (Section 5.2) ends the OptKCNA
                                loop of Algorithm 6 once the sampled k-CNA recall
                                reaches it; `iters` is then the most iterations run.
                                0: exactly `iters` iterations                        */
    double quality_eps;      /* epsilon of Theorem 3 (sample size n_s), default 0.6   */
    int32_t quality_k;       /* k of the recall r(u) (first k entries of C(u));
                                0 = K                                                */
    int32_t connect_replace; /* connectivity steps use edge replacement when every
                                reached node is full (pg_connect_replace); 0: such a
                                build fails with PG_ERR_CAPACITY                    */
    int32_t knn_descent_iters; /* initial KNNG: -1 the exact kNN tiles; >= 0 the
                                approximate graph of pg_knn_descent with that many
                                iterations from a random draw (seed), K <= 64  */
} pg_build_params;

/* Defaults: L2SQ, FP32, K=64, L=200, R=32, M=16, alpha 66/60, I=2,
 * connect_final=1, route_layers=1, seed=0, reuse_pruning=1,
 * quality_target=0 (fixed I), quality_eps=0.6, quality_k=0 (K),
 * connect_replace=1, knn_descent_iters=-1.  params must not be NULL. */
void pg_default_params(pg_build_params *params);

/* ---------------------------------------------------------------- context */

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  hbm_budget_bytes
 * caps the scratch the library may hold at once (0 = no cap).  *out
 * receives the context; destroy it with pg_ctx_destroy. */
pg_status pg_ctx_create(void *cuda_stream, size_t hbm_budget_bytes, pg_ctx **out);
void pg_ctx_destroy(pg_ctx *ctx);
/* Message of the last non-OK status returned on this context ("" if none).
 * The pointer stays valid until the next call on the context. */
const char *pg_last_error(const pg_ctx *ctx);
/* Synchronise the context stream; PG_ERR_DEVICE_CHECK if a kernel recorded
 * an invalid input since the previous synchronisation. */
pg_status pg_ctx_sync(pg_ctx *ctx);
/* Number of kernels this context has launched so far (host counter). */
int64_t pg_ctx_launches(const pg_ctx *ctx);

/* CUDA-event timing of the library's main kernels (off by default).
 * Enabling (or disabling) resets the totals.  Names: "knn" (distance tiles
 * + top-K), "prune", "union", "connect", "search" (beam search, including
 * k-CNA acquisition), "medoid".  *total_ms / *launches (host) receive the
 * summed device time and launch count since the last reset; the query
 * synchronises the stream. */
pg_status pg_ctx_set_timing(pg_ctx *ctx, int enable);
pg_status pg_ctx_kernel_time(pg_ctx *ctx, const char *name, double *total_ms, int64_t *launches);
/* Algorithmic work of the timed launches of `name` since the last reset:
 * "knn" counts 2*d flops per (query row, point) pair. */
pg_status pg_ctx_kernel_work(pg_ctx *ctx, const char *name, double *work);

/* Cumulative counters of this context.  Host side: "connect_edges" (edges
 * added by connectivity steps), "connect_full_rounds" (connectivity rounds
 * that needed a scan over all points), "connect_conflicts".  Device side
 * (reading one synchronises the stream; reset by pg_ctx_set_timing and by
 * pg_prune with host_stats): "search_expansions" and "search_evaluations"
 * (nodes expanded / distances evaluated by every beam search, Algorithm 1),
 * "prune_rows", "prune_candidates", "prune_scanned" (candidates visited by
 * the Algorithm 3 scan), "prune_occlusion_tests", and the algorithmic bytes
 * "search_bytes" (one data row per evaluation + one adjacency row per
 * expansion) and "prune_bytes" (one data row + 8 bytes per examined
 * candidate + the point's own row); a data row is 4d bytes, or d bytes
 * when the screened form gathers byte rows; "prune_edges" (kept edges),
 * "prune_fp64_rechecks" and "prune_fp64_flips" (decisions re-made in FP64,
 * and those whose FP64 outcome differed from the plain FP32 one), and
 * "prune_near_ties" (see pg_ctx_set_tie_count); "knn_fp64_rechecks" (kNN
 * entries re-ordered by FP64 distance) and "knn_fallback_rows" (rows of
 * the screened kNN that the certificate could not accept and the FP32
 * tiles computed). */
pg_status pg_ctx_counter(pg_ctx *ctx, const char *name, int64_t *value);

/* Launch-configuration autotuning (off by default; not in the paper).  The
 * persistent pruning and beam-search kernels give the same results under any
 * grid; with tuning on, the first pruning or search call for a key (kernel,
 * width d, degree / pool width, row form) on a device times each candidate
 * configuration on that call's own input (CUDA events; CTAs per SM, and the
 * search's visited-table size) and keeps the fastest in a process-wide
 * table that later calls use.  Search calls of fewer than 4096 queries are
 * not tuned. */
pg_status pg_ctx_set_autotune(pg_ctx *ctx, int enable);
/* The tuning table as text, one line per key ("label -> choice (config:ms
 * ...)"), written to buf (host, cap bytes, NUL-terminated, may be NULL);
 * returns the bytes the whole text needs. */
int64_t pg_autotune_report(char *buf, int64_t cap);

/* Tie accounting of the pruning kernels (off by default): when on, every
 * decision of the occlusion test (Section 4.1: s(u,w) < s(u,v),
 * s(v,w) < s(u,v) and the angle clause) whose relative margin is below
 * 1e-5 is counted in "prune_near_ties".  Margins: |a - b| / max(a, b) for a
 * distance comparison, |(s_uw + s_vw - s_uv) - 2 cos(alpha) sqrt(s_uw s_vw)|
 * / (s_uw + s_vw + s_uv) for the angle clause, from the FP32 distances.
 * Such decisions are still decided exactly (integer arithmetic or the FP64
 * recheck); the count states how many of them the tie budget covers. */
pg_status pg_ctx_set_tie_count(pg_ctx *ctx, int enable);

/* ------------------------------------------------------------------ steps */

/* Exact K nearest neighbours of every point (the KNNG G_k0 of the
 * initialization phase, Section 3.1 and Algorithm 6, computed by
 * brute force).  For every u the K smallest (s(u,v), v) with v != u.
 * ids [n][K], dist [n][K] (FP32 value of s); rows with fewer than K other
 * points are padded with -1 / +inf.  1 <= K <= 256, d % 4 == 0.
 * PG_PREC_BF16_SCREEN runs the distance tiles on the tensor cores
 * (tcgen05, BF16 inputs, FP32 accumulation).  When the BF16 copy of D and
 * every partial sum are exact (integer rows with |x| <= 256 whose squared
 * distances stay below 2^24, L2) the result equals the FP32 form's.  For
 * other rows the rows are centred (L2) and split into BF16 hi + lo parts;
 * the tiles contract [hi|hi|lo] with [hi|lo|hi] and keep each row's
 * Ks = min(120, max(2K, K + 8)) nearest, which are re-measured in FP32 with
 * FP64 re-ordering of near ties; a row is accepted only when a rigorous
 * bound on the screen's error shows that no point outside its shortlist can
 * come nearer than its K-th, and every other row is recomputed by the FP32
 * tiles ("knn_fallback_rows"), so the lists and distances equal the FP32
 * form's.  K beyond the tile kernels' limit, or PG_PREC_FP32, runs the
 * FP32 tiles (exact lists, FP64 fix-up of near ties).  Distances are the
 * FP64 values rounded to FP32 where a row was re-measured. */
pg_status pg_build_knn(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                       int32_t K, pg_precision precision, int32_t *ids, float *dist);

/* Approximate KNNG by 2-hop refinement, the KGraph (NN-descent) iteration
 * of the initialization phase (Section 3.1) as Exp. 12 describes it: each
 * point starts from K ids (init, DEVICE [n][K]: any order, repeats, -1 and
 * the point itself allowed and dropped; NULL: drawn by the library, id
 * j of point u = high 64 bits of SplitMix64(seed XOR (u K + j)) times n);
 * every iteration every point u takes the K best by (s(u, .), id) of its
 * neighbours and their neighbours, u excluded (all points read the previous
 * iteration's lists).  Pairs whose both entries were already there in the
 * previous iteration are not compared again (they cannot enter), which does
 * not change the result.  Out: ids / dist [n][K] as pg_build_knn (FP32
 * distances; orders decided on FP32 values, exact for rows whose FP32
 * distances are exact).  1 <= K <= 64, 0 <= iters <= 64.  host_updates
 * (host, may be NULL) [iters]: entries that entered a list per iteration. */
pg_status pg_knn_descent(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                         int32_t K, int32_t iters, const int32_t *init, uint64_t seed,
                         int32_t *ids, float *dist, int64_t *host_updates);

/* Exact k nearest points of D for external queries Q [nq][d] (ground
 * truth for recall).  Same output layout and precision rules as
 * pg_build_knn. */
pg_status pg_knn_query(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                       const float *Q, int64_t nq, int32_t k, pg_precision precision,
                       int32_t *ids, float *dist);

/* alpha-pruning of every candidate row (Section 4.1 definition, scanned
 * as in Prune, Algorithm 3).  Row u holds cand_ids[cand_off[u] ..
 * cand_off[u+1]-1] (cand_off has n+1 entries, non-decreasing); entries -1,
 * u itself and repeated ids are ignored.  The candidates are ordered by
 * (s(u,v), v); v is kept unless an already kept w has s(u,w) < s(u,v),
 * s(v,w) < s(u,v) and angle(u,w,v) > alpha; the scan stops at R kept.
 * alpha_deg = 60 is RNG pruning (the angle clause is then implied).
 * Output nbr [n][R] in keep order (-1 padded), deg [n].  R in [1, 64];
 * rows longer than 16384 candidates return PG_ERR_CAPACITY.
 * PG_PREC_BF16_SCREEN gathers byte rows when the rows are exact bytes (same
 * lists as FP32); PG_PREC_FP8_SCREEN is refused.  host_stats
 * (host pointer, may be NULL) receives counters and makes the call
 * synchronous. */
pg_status pg_prune(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                   const int64_t *cand_off, const int32_t *cand_ids, int32_t R,
                   double alpha_deg, pg_precision precision, int32_t *nbr, int32_t *deg,
                   pg_prune_stats *host_stats);

/* pg_prune with the K2P reuse of Section 5.4: prev_nbr [n][prev_R] /
 * prev_deg [n] (DEVICE) are the lists that an earlier pruning of the same
 * points kept, with an angle no larger than alpha_deg (the build passes the
 * previous refinement's lists).  A candidate v found in prev_nbr's row of u
 * was then tested against every member of that row that precedes it and was
 * not occluded; the occlusion test of a pair depends only on u, v and w (a
 * larger angle occludes less) and the scan order only on s(u, .), so v is
 * tested only against kept members that are not in the previous row.  The
 * lists equal pg_prune's; only "occlusion_tests" drops.  The caller
 * guarantees the premise: lists that are not such an earlier pruning give
 * other lists.  Other arguments and errors as pg_prune. */
pg_status pg_prune_k2p(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                       const int64_t *cand_off, const int32_t *cand_ids, const int32_t *prev_nbr,
                       const int32_t *prev_deg, int32_t prev_R, int32_t R, double alpha_deg,
                       pg_precision precision, int32_t *nbr, int32_t *deg,
                       pg_prune_stats *host_stats);

/* Largest n accepted by pg_prune_noalloc. */
#define PG_PRUNE_NOALLOC_MAX_N (1 << 20)

/* pg_prune for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a deployment variant of the same pruning step
 * (same rule, same output as pg_prune), for code that may not call
 * cudaMalloc or anything that allocates -- for instance under an allocator
 * or runtime that owns every device allocation, or in a process whose
 * memory footprint must stay fixed after start-up.  It needs no context: it
 * takes the stream (a cudaStream_t; NULL = the legacy default stream) and
 * uses the current device.  All scratch comes from one fixed device array
 * inside the library (about 4.2 MB; every GPU that loads the library holds
 * it until the process exits), so n may not exceed PG_PRUNE_NOALLOC_MAX_N
 * (larger n: PG_ERR_CAPACITY, before any work).  The first call on a device
 * looks up that array's device address with the device current.  Every call
 * shares the one array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The call is synchronous: it synchronises the stream twice and copies the
 * data facts and the error word to host memory, so it must not be made on a
 * stream that is being captured into a CUDA graph.  Errors:
 * PG_ERR_INVALID_ARG / PG_ERR_CAPACITY for bad arguments, PG_ERR_CUDA for a
 * failed CUDA call, PG_ERR_DEVICE_CHECK for a candidate id outside [-1, n). */
pg_status pg_prune_noalloc(void *cuda_stream, const float *D, int64_t n, int32_t d,
                           pg_metric metric, const int64_t *cand_off, const int32_t *cand_ids,
                           int32_t R, double alpha_deg, int32_t *nbr, int32_t *deg);

/* Reverse-edge union (Algorithm 2, Algorithm 5): row
 * u = N(u) together with every v that has u in N(v).  nbr [n][R], deg [n]
 * in; off [n+1] and ids out (ids needs capacity >= 2 * sum(deg); entries
 * within a row are in no particular order).  *host_total (host, may be
 * NULL) receives off[n] and makes the call synchronous. */
pg_status pg_reverse_union(pg_ctx *ctx, const int32_t *nbr, const int32_t *deg, int64_t n,
                           int32_t R, int64_t *off, int32_t *ids, int64_t ids_capacity,
                           int64_t *host_total);

/* Entry point: the point nearest the centroid (Section 3.1, search phase),
 * exact argmin by (s, id); the centroid is summed in FP64 per coordinate
 * in blocks of 1024 consecutive points (each in index order, then the block
 * sums in order) and divided by n.  *host_ep (host) receives the id. */
pg_status pg_medoid(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                    int64_t *host_ep);

/* Connectivity step (Algorithm 2, Algorithm 5),
 * in place on nbr/deg: S = nodes reachable from ep; while S != V the
 * smallest unreached id r is linked from p = argmin over x in S with
 * deg(x) < R of (s(x,r), x), and everything reachable from r joins S.
 * *host_added (host, may be NULL) receives the number of edges added.
 * PG_ERR_CAPACITY if no reached node has a free slot.  Synchronous. */
pg_status pg_connect(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                     int32_t *nbr, int32_t *deg, int32_t R, int64_t ep, int64_t *host_added);

/* The connectivity step with edge replacement (a reading for graphs whose
 * reached nodes are all full; the paper only says that extra edges join the
 * components).  As pg_connect while some reached node has a free slot;
 * when none has one for the smallest unreached id r, the reached node p
 * nearest to r by (s, id) that still holds an edge not added by this call
 * gives up the last such edge in its list (its farthest original
 * neighbour) for r, and the reached set is recomputed from ep.  Equal to
 * pg_connect whenever pg_connect succeeds.  *host_added / *host_replaced
 * (host, may be NULL): edges added (replacements included) and
 * replacements.  PG_ERR_CAPACITY when no reached node has a free slot or
 * an original edge. */
pg_status pg_connect_replace(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                             int32_t *nbr, int32_t *deg, int32_t R, int64_t ep,
                             int64_t *host_added, int64_t *host_replaced);

/* k-CNA acquisition by search on the refined graph (the search step of
 * Algorithm 5): for every u, KANNSearch(G, u, L, L, u) of Algorithm 1; row
 * u of cand [n][L] receives the final pool minus u, in (s, id) order, padded
 * with -1.  nbr [n][R] / deg [n] is the graph.  1 <= L <= 256, R <= 64.
 * PG_PREC_BF16_SCREEN gathers byte rows (a u8 copy of D) when the rows are
 * exact bytes (same result as FP32); PG_PREC_FP8_SCREEN is refused. */
pg_status pg_acquire_candidates(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                                pg_metric metric, const int32_t *nbr, const int32_t *deg,
                                int32_t R, int32_t L, pg_precision precision, int32_t *cand);

/* Batched beam search, KANNSearch(G, q, k, L, ep) of Algorithm 1, on one
 * graph: query i starts at starts[i] (device, nq entries).  rows (device,
 * may be NULL) maps a point id to its adjacency row when the graph covers
 * a subset of D (a layer of a hierarchical index); NULL = row id.  Output
 * out_ids / out_dist [nq][k], padded with -1 / +inf.  1 <= k <= L <= 256.
 * precision: PG_PREC_FP32 or PG_PREC_BF16_SCREEN (both FP32 rows here). */
pg_status pg_search_graph(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                          const int32_t *nbr, const int32_t *deg, int32_t R,
                          const int32_t *rows, const float *Q, int64_t nq,
                          const int32_t *starts, int32_t k, int32_t L, pg_precision precision,
                          int32_t *out_ids, float *out_dist);

/* ----------------------------------------------------------------- builds */

/* IterNSG with a fixed number of iterations (Algorithm 6 with the
 * OptKCNA iterations of Algorithm 5; final refinement with the refinement
 * steps of Algorithm 2: pruning, reverse-edge union, connectivity).  With
 * route_layers set, NSWG upper layers (Algorithm 7, i >= 1) are added so
 * that queries enter the graph near their target.  D stays owned by the
 * caller and must outlive the index.  Synchronous. */
pg_status pg_build_rng(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                       const pg_build_params *params, pg_index **out);

/* Quality examination of the k-CNA lists (Section 5.2): for each sampled
 * point u = sample[i] (DEVICE, ns ids in [0, n)), recall[i] (DEVICE,
 * double) = r(u), the share of the first k entries of row u of cand
 * (DEVICE [n][L], -1 padded, the k-CNA lists C(u)) that are among the exact
 * k nearest points of u other than u: an entry counts once when its id is
 * valid, not u and not repeated, and its FP64 distance to u is at most the
 * exact k-th distance (ties count).  *host_mean (host, may be NULL) receives
 * the mean over the sample, the estimator r^(S) / n_s.  1 <= k <= min(L,
 * 255), k < n.  Synchronous.  An id outside [0, n) in sample gives
 * PG_ERR_DEVICE_CHECK. */
pg_status pg_kcna_recall(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                         const int32_t *cand, int32_t L, int32_t k, const int32_t *sample,
                         int64_t ns, double *recall, double *host_mean);

/* Sample size of Theorem 3 (host only): the smallest n_s with
 * n_s >= (8 + 2 eps) l ln(n) / eps^2, so that the sampled mean of r(u) is
 * within eps / 2 of the exact mean with probability >= 1 - n^-l.  -1 for
 * n < 2, eps <= 0 or l <= 0. */
int64_t pg_quality_sample_size(int64_t n, double eps, double l);

/* The sample the builds draw (host only): ns distinct ids of [0, n),
 * ascending, from SplitMix64 outputs of seed XOR (0x51a3c0ffee000000 + c),
 * c = 0, 1, ..., each mapped to the high 64 bits of z * n, repeats
 * skipped.  host_ids [ns].  PG_ERR_INVALID_ARG unless 0 <= ns <= n < 2^31. */
pg_status pg_quality_sample(int64_t n, int64_t ns, uint64_t seed, int32_t *host_ids);

/* Quality examination record of the last build of this index (layer 0):
 * *iters_run (host) = OptKCNA iterations run, *sample_size (host) = n_s
 * (0 when the examination was off), host_estimates [iters_run] (host, may
 * be NULL; at most 16) = the estimate after each iteration. */
pg_status pg_index_quality(const pg_index *index, int32_t *iters_run, int64_t *sample_size,
                           double *host_estimates);

/* pg_build_rng from HOST memory: D_host [n][d] (host, pinned or pageable)
 * is copied to a device buffer that the index owns, the build runs as
 * pg_build_rng, and the base graph (layer 0) is copied back to the host
 * arrays nbr_host [n][R] and deg_host [n].  Synchronous.  out may be NULL
 * (the index is then destroyed before returning); otherwise *out is an
 * index that owns its points. */
pg_status pg_build_rng_host(pg_ctx *ctx, const float *D_host, int64_t n, int32_t d,
                            const pg_build_params *params, int32_t *nbr_host, int32_t *deg_host,
                            pg_index **out);

/* Global NSWG construction, OptHNSW (Algorithm 7): levels drawn up front
 * (l(u) = floor(-ln U / ln M), U from SplitMix64(seed XOR u)); layer i
 * holds D_i = {u : l(u) >= i}; a layer with |D_i| <= its degree bound is
 * complete, any other is an IterNSG build of D_i without the final
 * connectivity step.  Layer 0 bound R, upper layers M.  Synchronous. */
pg_status pg_build_nswg(pg_ctx *ctx, const float *D, int64_t n, int32_t d,
                        const pg_build_params *params, pg_index **out);

#define PG_SEARCH_FLAT 1 /* ignore routing layers: start at the medoid */

/* k-ANN queries on an index: from the top layer down to layer 1,
 * w <- first of KANNSearch(G_i, q, 1, upper_beam, w); then
 * KANNSearch(G_0, q, k, beam, w) (pattern of Algorithm 4, where
 * upper_beam = 1 is the greedy routing of the paper); an index without
 * upper layers (or with PG_SEARCH_FLAT) starts at its medoid.
 * Q [nq][d] device; out [nq][k].  1 <= k <= beam <= 256,
 * 1 <= upper_beam <= 256.  precision: PG_PREC_FP8_SCREEN screens the
 * base-layer search (see pg_precision); PG_PREC_FP32 and
 * PG_PREC_BF16_SCREEN search FP32 rows. */
pg_status pg_search(pg_ctx *ctx, const pg_index *index, const float *Q, int64_t nq, int32_t k,
                    int32_t beam, int32_t upper_beam, int32_t flags, pg_precision precision,
                    int32_t *out_ids, float *out_dist);

/* Same as pg_search with HOST buffers (Q, out_ids, out_dist in host
 * memory, pinned or pageable): copies in, searches, copies out and
 * synchronises. */
pg_status pg_search_host(pg_ctx *ctx, const pg_index *index, const float *Q, int64_t nq,
                         int32_t k, int32_t beam, int32_t upper_beam, int32_t flags,
                         pg_precision precision, int32_t *out_ids, float *out_dist);

void pg_index_destroy(pg_index *index);

/* The layer of each point id 0..n-1 that pg_build_nswg (and insertion)
 * assign, host only (no context, no device): l(u) = floor(-ln U / ln M)
 * with U = ((z >> 11) + 1) 2^-53, z = SplitMix64(seed XOR u) (the
 * exponentially decaying level draw of Algorithm 7).  host_levels [n]. */
pg_status pg_levels(int64_t n, uint64_t seed, int32_t M, int32_t *host_levels);

/* Shape of an index: number of layers, points, entry points (host outs). */
pg_status pg_index_info(const pg_index *index, int32_t *n_layers, int64_t *n, int64_t *ep_top,
                        int64_t *ep_base);

/* Device pointers of layer `layer` (owned by the index): *count nodes,
 * degree bound *R, gid [count] (ascending point ids; NULL for layer 0,
 * which holds every point), nbr [count][R] of point ids, deg [count]. */
pg_status pg_index_layer(const pg_index *index, int32_t layer, int64_t *count, int32_t *R,
                         const int32_t **gid, const int32_t **nbr, const int32_t **deg);

/* Copy layer `layer` of an index into caller DEVICE buffers: gid [count]
 * (may be NULL; for layer 0 it receives 0..n-1), nbr [count][R] and deg
 * [count] (shapes from pg_index_layer).  Synchronous. */
pg_status pg_index_export_layer(pg_ctx *ctx, const pg_index *index, int32_t layer, int32_t *gid,
                                int32_t *nbr, int32_t *deg);

/* ------------------------------------------------------------ insertion */

/* Make `index` growable (serving): the index takes a private DEVICE copy of
 * its points in a buffer of `capacity` rows (the caller's D is no longer
 * read afterwards) and grows every layer to hold the points inserted up to
 * that capacity.  n <= capacity < 2^31.  Synchronous.  Errors:
 * PG_ERR_INVALID_ARG, PG_ERR_CUDA (allocation). */
pg_status pg_index_reserve(pg_ctx *ctx, pg_index *index, int64_t capacity);

/* Batched insertion of m points X (DEVICE, [m][d] row-major, caller-owned;
 * copied into the index) with ids n .. n+m-1: the search and refinement
 * phases of Algorithm 4 for every new point, all against the graph as it
 * was before the batch (one batch = one snapshot).  Each new point u takes
 * the level of the build's SplitMix64 draw (Algorithm 7), capped at
 * the top layer; w = the top entry, w <- best of a pool-`upper_beam`
 * search in each layer above l(u) (1 = the paper's greedy routing); for
 * i = l(u)..0: W_i <- KANNSearch(G_i, u, ef, ef, w), w <- W_i[0],
 * N_i(u) <- Prune(u, W_i, R_i) at the build's final angle (Algorithm 3 with
 * the Section 4.1 rule).  Every old node v that gained in-edges I_i(v)
 * re-prunes N_i(v) | I_i(v) (the reverse-edge step of Algorithm 4); new
 * nodes are appended to the layers in id order.  Needs pg_index_reserve
 * with capacity >= n + m (else PG_ERR_CAPACITY); 1 <= ef, upper_beam <= 256.
 * The batch is built in copies of the layers' graph arrays (those of an
 * earlier version that no search reads any more are reused, else new ones
 * are allocated) and published when it ends, so a search running meanwhile
 * on another context (pg_search, pg_search_host, the serving loop) reads
 * the version it started on.  Insertions into one index must not overlap
 * each other (the serving loop runs them one at a time).  Synchronous. */
pg_status pg_index_insert(pg_ctx *ctx, pg_index *index, const float *X, int64_t m, int32_t ef,
                          int32_t upper_beam);

/* Build parameters and dimension of an index (host outs, each nullable). */
pg_status pg_index_params(const pg_index *index, pg_build_params *params, int32_t *d);

/* ---------------------------------------------------------- index files */

/* Write `index` to the file `path`: its build parameters, entry points,
 * every layer (members, degrees, neighbour lists) and its n points, then a
 * checksum.  The layout, little-endian, version 1:
 *   "PGINDEX\0", u32 version, u32 byte-order mark 0x01020304,
 *   i64 n, i32 d, i32 metric, i64 ep_top, i64 ep_base,
 *   i32 metric, precision, K, L, R, M; f64 alpha_deg, alpha_final_deg;
 *   i32 iters, connect_final, route_layers, 0; u64 seed;
 *   i32 layers, i32 0; per layer i64 count, i32 R, i32 has_gid;
 *   per layer: gid i32[count] (upper layers only), deg i32[count],
 *   nbr i32[count][R] (point ids);
 *   points f32[n][d];
 *   u64 checksum: FNV-1a (offset basis 0xcbf29ce484222325, prime
 *   0x100000001b3) over the preceding bytes read as little-endian 64-bit
 *   words, the last partial word zero-padded.
 * The file is written under a temporary name and renamed when complete,
 * so `path` never holds a partial index.  Synchronous (device -> host
 * copies on the context stream).  Errors: PG_ERR_INVALID_ARG (null
 * argument), PG_ERR_CUDA, PG_ERR_IO (the message names the failing step). */
pg_status pg_index_save(pg_ctx *ctx, const pg_index *index, const char *path);

/* Read an index written by pg_index_save.  The whole file is checked on
 * the host before the index is returned: magic, version, byte order,
 * parameter ranges (those of pg_build_rng), layer 0 holding every point,
 * upper layers holding strictly ascending ids, each a subset of the layer
 * below, degrees within [0, R], every listed neighbour a member of its
 * layer, the entry points (ep_top in the top layer), no trailing bytes and
 * the checksum.  The index owns a private DEVICE copy of its points
 * (pg_index_reserve grows it for insertion).  Synchronous.  Errors:
 * PG_ERR_IO (open / short read), PG_ERR_INVALID_ARG (a failed check; the
 * message says which), PG_ERR_CUDA (allocation or copy); *out is NULL on
 * error. */
pg_status pg_index_load(pg_ctx *ctx, const char *path, pg_index **out);

/* The checks of pg_index_load without a context or a device: n, d and the
 * number of layers of a valid file go to the host outs (each nullable);
 * on error a one-line reason is written to msg (msg_len bytes, nullable). */
pg_status pg_index_file_check(const char *path, int64_t *n, int32_t *d, int32_t *n_layers,
                              char *msg, size_t msg_len);

/* The FP8 rows that PG_PREC_FP8_SCREEN searches use, for n DEVICE rows
 * D [n][d]: scale[i] = max_j |D[i][j]| / 448 in FP32 (1 for a zero row),
 * codes[i][j] = E4M3 (OCP FP8, 1-4-3 bits, bias 7, no infinities) of
 * D[i][j] * (1 / scale[i]) (both steps in FP32) rounded to nearest even
 * and saturated at +-448.  Caller DEVICE buffers codes [n][d], scale [n].
 * Synchronous. */
pg_status pg_encode_fp8(pg_ctx *ctx, const float *D, int64_t n, int32_t d, uint8_t *codes,
                        float *scale);

/* -------------------------------------------------------------- serving */

/* A serving loop over a growable index: a dispatcher thread takes query
 * and insertion requests in submission order and hands query groups to
 * `slots` worker threads, each with its own context on its own CUDA stream,
 * so that groups of different requests run concurrently on the device.
 * Consecutive query requests with equal (k, beam, upper_beam, precision)
 * are merged into one group of at most max_batch queries.  A group is admitted when a
 * worker is free and the device scratch of the groups in flight plus its
 * own (queries, results and search state: rows x (4 d + 8 k + 12) bytes)
 * fits the HBM budget of ctx (0 = no limit); a group larger than the budget
 * fails with PG_ERR_BUDGET.  A query group searches the version of the
 * index pinned when it was dispatched.  An insertion (pg_index_insert on a
 * free worker's context) runs beside the groups in flight: it builds the
 * next version in copies of the graph arrays, publishes it when it ends,
 * and nothing submitted after it is dispatched before then, so a query sees
 * exactly the points inserted before it was submitted.  The arrays of a
 * version are freed once no group pins it.  Tickets complete out of
 * order.  While the server runs, ctx and index belong to it (the caller
 * issues no other call on them until pg_serve_stop).  Host buffers of a
 * request must stay valid until it completes. */
typedef struct pg_server pg_server;

/* Start the dispatcher and the workers on ctx's device (1 <= max_batch <=
 * 65536, 1 <= slots <= 16; the workers' streams and contexts are created
 * here and freed by pg_serve_stop). */
pg_status pg_serve_start(pg_ctx *ctx, pg_index *index, int32_t max_batch, int32_t slots,
                         pg_server **out);

/* Enqueue nq HOST query rows Q [nq][d]; results go to HOST out_ids [nq][k]
 * and out_dist [nq][k] (pg_search semantics).  *ticket identifies it.  A
 * refused submission (bad arguments, stopping: PG_ERR_INVALID_ARG; full:
 * PG_ERR_CAPACITY) returns its status and records no message. */
pg_status pg_serve_submit_query(pg_server *server, const float *Q, int64_t nq, int32_t k,
                                int32_t beam, int32_t upper_beam, int32_t *out_ids,
                                float *out_dist, int64_t *ticket);

/* Enqueue the insertion of m HOST rows X [m][d] (pg_index_insert). */
pg_status pg_serve_submit_insert(pg_server *server, const float *X, int64_t m, int32_t ef,
                                 int32_t upper_beam, int64_t *ticket);

/* Wait up to timeout_s seconds (0: poll) for `ticket`; *done = 1 once it has
 * completed, and the return value is then that request's status.
 * PG_ERR_INVALID_ARG for a ticket that was never issued. */
pg_status pg_serve_wait(pg_server *server, int64_t ticket, double timeout_s, int32_t *done);

/* Seconds from the submission of `ticket` to its completion (host clock),
 * for a completed ticket among the last 65,536 issued; else
 * PG_ERR_INVALID_ARG. */
pg_status pg_serve_latency(pg_server *server, int64_t ticket, double *seconds);

/* Admission control: a submit is refused with PG_ERR_CAPACITY (nothing
 * enqueued, no ticket) while `limit` requests are pending (queued or
 * running); 0 = no limit (the default). */
pg_status pg_serve_set_queue_limit(pg_server *server, int64_t limit);

/* Distance form of the query requests submitted from now on (PG_PREC_FP32,
 * the default, PG_PREC_BF16_SCREEN or PG_PREC_FP8_SCREEN, as pg_search);
 * requests of different forms are not merged. */
pg_status pg_serve_set_precision(pg_server *server, pg_precision precision);

/* Admission budget: bytes of device scratch the groups in flight may hold
 * together (0 = no limit; the default is ctx's HBM budget).  A group larger
 * than the budget fails with PG_ERR_BUDGET when it is dispatched. */
pg_status pg_serve_set_budget(pg_server *server, int64_t bytes);

/* The first `count` (<= 6) of {groups run (query groups and insertions),
 * requests completed, queries, inserted points, most groups in flight at
 * once, dispatches that waited for a worker, for memory or for the groups
 * before an insertion} go to host_stats. */
pg_status pg_serve_stats(pg_server *server, int64_t *host_stats, int32_t count);

/* Finish every queued request, join the threads and free the server. */
pg_status pg_serve_stop(pg_server *server);

/* The scheduler of the serving loop with simulated work, host only (no
 * context, no device): `count` requests submitted at once, request i a
 * query of rows[i] queries with merge key shape[i] (kind[i] = 0) or an
 * insertion of rows[i] points (kind[i] = 1).  Running a group sleeps
 * work_us x (1 + rows / 64) microseconds; its scratch is rows x
 * bytes_per_row against budget_bytes.  Per request (caller arrays of
 * `count`, left untouched for requests refused with PG_ERR_BUDGET):
 * start_seq / end_seq, the positions of the start and the end of its group
 * in one sequence of events shared by all threads; slot_of, the worker
 * that ran it; group_of, its group; version_of (nullable), for a query the
 * version of the index its group pinned when dispatched and for an
 * insertion the version it published (versions count the insertions that
 * have ended, from 0).  host_stats6 as pg_serve_stats (nullable).  Returns
 * once every request has completed. */
pg_status pg_serve_simulate(int32_t slots, int32_t max_batch, int64_t budget_bytes,
                            int32_t count, const int32_t *kind, const int32_t *rows,
                            const int32_t *shape, int32_t work_us, int64_t bytes_per_row,
                            int64_t *start_seq, int64_t *end_seq, int32_t *slot_of,
                            int64_t *group_of, int64_t *version_of, int64_t *host_stats6);

/* ------------------------------------------------------------ self test */

/* Failure path of the bounded device waits, without a fault: one thread
 * waits on an mbarrier that nothing completes, gives up after `seconds`
 * (0 < seconds <= 5), records a timeout in the context's error word and
 * returns; the call then returns PG_ERR_TIMEOUT, like a kernel whose
 * pipeline wait expired, and the context stays usable. */
pg_status pg_selftest_wait_timeout(pg_ctx *ctx, double seconds);

/* Measured FP32 FMA throughput of the context's device (not from the paper:
 * the SIMT roofline of the FP32 form's distance tiles): eight independent
 * fused multiply-add chains per thread, 2048 threads per SM, timed with CUDA
 * events on the context's stream; *host_tflops receives the best of three
 * timed launches (2 flop per FMA).  Synchronous. */
pg_status pg_measure_fp32_peak(pg_ctx *ctx, double *host_tflops);

/* Seconds spent per build phase by the last build on this index:
 * knn, prune, union, connect, acquire, layers (host array of 6). */
pg_status pg_index_phase_seconds(const pg_index *index, double *host_seconds6);

#ifdef __cplusplus
}
#endif
#endif /* PG_H */
