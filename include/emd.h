/*
 * emd.h -- C ABI of the GB300 (sm_103a) library for the linear-complexity EMD lower
 * bounds of Atasu & Mittelholzer, "Low-Complexity Data-Parallel Earth Mover's Distance
 * Approximations" (ICML 2019): LC-RWMD, OMR (Alg. 1), LC-ACT (Alg. 3, Section 5) and
 * ICT (Alg. 2), for query histograms against a device-resident database of sparse
 * histograms, in either direction or the maximum of both, plus top-K neighbours.
 *
 * Problem statement (Section 2.2 and Section 6): one query histogram q is compared with
 * n database histograms over a vocabulary of v coordinates with m-dimensional
 * embeddings; the ground cost is the Euclidean distance between embeddings (Section 6)
 * or, in cost-matrix mode, any nonnegative v x v matrix (Section 4, remark on p-th
 * Wasserstein distances).  Every histogram is L1-normalised (Section 2).
 *
 * Conventions shared by every entry point
 *   - Status codes only; nothing throws across the ABI.  On failure the thread-local
 *     message behind emd_last_error() says why.
 *   - Ownership: the caller owns every buffer it passes.  Host inputs are copied during
 *     the call; nothing keeps a caller pointer after the call returns.  Handles are
 *     released only by the matching *_destroy call.
 *   - Threads: one handle must not be used by two host threads at the same time.
 *   - Index types: vocabulary ids and per-histogram sizes are int32; offsets int64.
 */
#ifndef EMD_GB300_H
#define EMD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EMD_OK = 0,
    EMD_ERR_INVALID_ARG = 1,   /* a size, index, weight or option is out of range */
    EMD_ERR_OUT_OF_MEMORY = 2, /* a device or pinned-host allocation failed */
    EMD_ERR_CUDA = 3,          /* a CUDA call or kernel reported an error */
    EMD_ERR_TIMEOUT = 4,       /* a bounded wait ran out */
    EMD_ERR_BUSY = 5,          /* admission refused: no free slot or workspace */
    EMD_ERR_SHUTDOWN = 6,      /* the server is shutting down */
    EMD_ERR_UNSUPPORTED = 7    /* a valid request this build does not serve */
} emd_status;

/* Which lower bound.  RWMD is ACT with k = 1 (Alg. 3); OMR is Alg. 1 (k ignored);
 * ACT is Alg. 3 with top-k width k, i.e. k-1 capacity-limited transfers and the rest of
 * the mass to the k-th nearest (the evaluation's "ACT-j" is k = j+1); ICT is Alg. 2,
 * equal to ACT with k = the destination's histogram size.  In the forward direction an ICT
 * table row holds only the nearest query bins that the row's largest database weight can
 * reach (Section 5 form of Alg. 2: the transfers stop once the mass is placed), at most
 * max_table_k of them; a query that needs more is recomputed with rows of full width. */
typedef enum { EMD_RWMD = 0, EMD_OMR = 1, EMD_ACT = 2, EMD_ICT = 3 } emd_measure;

/* FWD moves each database histogram's mass into the query (the direction of the
 * linear-complexity Phase 2, Section 5); REV moves the query's mass into each database
 * histogram; MAX is the symmetric bound max(FWD, REV) of Sections 4 and 6. */
typedef enum { EMD_DIR_FWD = 0, EMD_DIR_REV = 1, EMD_DIR_MAX = 2 } emd_direction;

/* Arithmetic of the Phase-1 distance matrix (Section 5).  FP32 is the plain method (FP32
 * FFMA on the CUDA cores).  FP32_TC computes the same FP32-grade distances on the tensor
 * cores: each embedding row is scaled by its absmax and split into two FP16 parts
 * (hi + lo * 2^-11), and the three products hi*hi, hi*lo, lo*hi are accumulated in FP32,
 * which reproduces the dot product to about 2^-22 relative.  BF16 and FP8_E4M3 compute the
 * matrix from one low-precision product on the tensor cores (operands scaled per row by
 * their absmax; E4M3 maps the absmax to 448), FP32 accumulation; the Phase-1 table then
 * takes each row's k + rerank_margin smallest approximate distances and recomputes them
 * exactly in FP32 as sqrt(sum (v - q)^2) before keeping the k smallest.  Forward distances
 * are exact whenever the true k nearest are among those candidates; reverse distances use
 * the approximate matrix except for the re-ranked entries.  These two forms require
 * min(table width + rerank_margin, h_q) <= 32 for forward directions (else UNSUPPORTED).
 * Cost-matrix databases ignore the precision. */
typedef enum {
    EMD_PREC_FP32 = 0,
    EMD_PREC_BF16 = 1,
    EMD_PREC_FP8_E4M3 = 2,
    EMD_PREC_FP32_TC = 3
} emd_precision;

typedef struct emd_db emd_db; /* opaque; owns device memory on one GPU */

typedef struct {
    int32_t device;          /* CUDA device ordinal (default 0) */
    emd_precision precision; /* default EMD_PREC_FP32 */
    int32_t rerank_margin;   /* BF16/FP8 only: extra candidates re-ranked in FP32 (default 8) */
    int32_t max_query_h;     /* largest query histogram accepted; sizes the workspace (default 2048) */
    int32_t max_table_k;     /* largest forward table width: k of ACT, and the entries an ICT row may
                                hold before the query is recomputed at full width (default 64) */
    int32_t max_batch;       /* queries staged per device pass (default 64) */
    int32_t prune_topk;      /* 1 (default): exact pruned max-direction top-K for K <= 16 */
    int32_t lanes;           /* per-query pipelines, each with its own stream and workspace
                                (default 1, 1..16); with batched = 0 a batch's queries are spread
                                over them and joined back into the caller's stream */
    int32_t batched;         /* 1 (default): each step of a batch is one launch over all its
                                queries; 0: one query after another on the lanes.  Results are
                                bit-identical either way */
    int32_t batch_columns;   /* batched form: distance-matrix columns of one batch (sum over its
                                queries of h_q rounded up to 32; default 16384, at least
                                max_query_h).  Device memory: 4 x v_used x batch_columns bytes */
    int32_t graphs;          /* batched form: 1 (default) replays each (measure, k, K, direction)
                                sequence from a captured CUDA graph; 0: launches directly.
                                Profiling (emd_db_set_profiling) launches directly */
    int32_t autotune;        /* batched form: 1 (default) times the free parameters of the batched
                                kernels on a synthetic batch at creation and keeps the fastest
                                (results do not depend on them); 0: fixed defaults */
    int32_t fused_phase1;    /* batched pruned top-K (EMD_DIR_MAX, K <= 16) with RWMD, OMR or ACT
                                (k <= 16), tensor-core precisions.  The fused form keeps each row's
                                k smallest distances (FP32_TC) or k + rerank_margin <= 16 smallest
                                approximate ones (BF16, FP8_E4M3) in the product's epilogue, and
                                computes the reverse direction's distances only on the candidate
                                documents' rows, in the FP32-grade split, so no v_used x h_q
                                matrix is written.  FP32_TC: bit-identical to the full-matrix
                                form.  BF16: each table row is re-ranked exactly and certified
                                (the k + margin-th approximate value minus the operand-rounding
                                bound exceeds the k-th exact value) or recomputed exactly over all
                                bins, so results meet the FP32 tolerance.  FP8_E4M3: the re-ranked
                                candidates as the table (no certificate), exact reverse distances.
                                0: always the full matrix and a separate table pass; 1 (default):
                                the fused form for FP32_TC; 2: also for BF16 and FP8_E4M3 (exact
                                but, on the serving-size database, slower than their full-matrix
                                form: the wide candidate lists and their FP32 re-rank cost about
                                what the cheaper product saves) */
    int32_t fwd_kernel;      /* form of the batched forward sweep (Phase 2+3 over the CSR for a
                                group of eight queries): 0 (default) the autotuner's choice; 1 each
                                table entry loaded when the residual mass needs it; 2 query-major
                                table rows, four entries loaded up front; 3 the first two entries up
                                front, column ids and weights read 32 at a time; 4 as 1 with each
                                lane's next column ids and weights read ahead.  Same results */
    int32_t tc_pair;         /* the fused FP32_TC table (fused_phase1 >= 1) on clusters of two SMs
                                (tcgen05 cta_group::2: 256 vocabulary rows per product, each SM
                                staging half of each query chunk): 0 (default) one SM per tile;
                                1 pairs with 64-column tiles; 2 pairs with 128-column tiles.
                                Same results */
} emd_db_options;

typedef struct {
    int64_t v, v_used, n_docs, nnz; /* vocabulary, used vocabulary (Section 2.2), database size */
    int32_t m;                      /* embedding width (0 in cost-matrix mode) */
    int32_t cost_matrix_mode;       /* 1 when a v x v ground-cost matrix replaced embeddings */
    int64_t device_bytes;           /* device memory held by the handle */
    int32_t autotuned;              /* 1 when the parameters below were timed at creation */
    int32_t tc_group_mult;          /* batched tensor-core Phase 1: query groups per vocabulary tile
                                       (multiple of the load-balance minimum) */
    int32_t tc_stages;              /* its query-chunk stages (0: as many as fit) */
    int32_t rev_warps;              /* pruned reverse pass: warps per candidate document */
    int32_t fwd_kernel;             /* the batched forward sweep's form (1..4, see emd_db_options) */
    int32_t tc_pair;                /* the fused table's SM-pair form in use (0..2, see emd_db_options) */
} emd_db_info;

/* A batch of query histograms in CSR form: query i has bins
 * idx[row_ptr[i] .. row_ptr[i+1]) with weights w[...]. */
typedef struct {
    int64_t n_queries;
    const int64_t* row_ptr; /* [n_queries + 1], row_ptr[0] == 0 */
    const int32_t* idx;     /* vocabulary ids, distinct within a query */
    const float* w;         /* weights, >= 0, summing to 1 per query (|sum - 1| <= 1e-5) */
} emd_queries;

/* Per-phase device time (CUDA events on the launch stream) and launch counts collected
 * while profiling is on.  Phases: 0 query staging, 1 distance matrix (Phase 1), 2 top-k
 * table (Phase 1), 3 forward sparse pass (Phase 2+3), 4 reverse pass + max, 5 top-K
 * selection, 6 other. */
#define EMD_N_PHASES 7
typedef struct {
    double ms[EMD_N_PHASES];
    int64_t launches[EMD_N_PHASES];
    int64_t total_launches; /* every kernel launch since creation, profiling on or off */
    int64_t pruned_queries; /* max-direction top-K queries answered by the pruned path */
    int64_t prune_fallbacks; /* of those, queries recomputed over all documents */
    int64_t graph_launches;  /* batch sequences replayed from captured graphs (their kernels are
                                included in the launch counts) */
    int64_t ict_wide;        /* ICT queries recomputed with tables of full width h because a
                                vocabulary row needed more than max_table_k entries */
    int64_t fused_retries;   /* pruned queries of the fused form whose candidate documents held
                                more distinct rows than its exact distance block; each was run
                                again with the full distance matrix (its answer is unchanged) */
} emd_profile;

/* Fill *opt with the defaults listed above.  Never fails. */
void emd_db_options_default(emd_db_options* opt);

/* Build the device-resident database (Section 5: X in CSR form; V, the embeddings).
 *   emb          host float [v * m] row-major embeddings, or NULL in cost-matrix mode
 *   v, m         vocabulary size (>= 1) and embedding width (1..4096; ignored if emb NULL)
 *   cost_matrix  host float [v * v] row-major nonnegative ground costs with a zero
 *                diagonal, or NULL (then emb is required).  Exactly one of emb and
 *                cost_matrix is non-NULL.
 *   row_ptr      host int64 [n_docs + 1], row_ptr[0] == 0, non-decreasing, nnz < 2^31
 *   col, val     host int32 / float [nnz]: vocabulary ids (0 <= col < v, distinct
 *                within a row) and weights (> 0, each row summing to 1 within 1e-5)
 *   n_docs       >= 1; every row must have at least one bin
 *   opt          options or NULL for the defaults
 *   out          receives the handle
 * The used vocabulary (the union of database coordinates, Section 2.2) is compacted on
 * the device; database columns are renumbered into it.
 * Errors: INVALID_ARG for any violated condition above (nothing is allocated),
 * OUT_OF_MEMORY, CUDA. */
emd_status emd_db_create(const float* emb, int64_t v, int32_t m, const float* cost_matrix,
                         const int64_t* row_ptr, const int32_t* col, const float* val,
                         int64_t n_docs, const emd_db_options* opt, emd_db** out);

/* Release every device and host resource of the handle.  NULL is accepted.  BUSY while a
 * server (below) is attached to the handle. */
emd_status emd_db_destroy(emd_db* db);

/* Sizes and memory of the handle.  INVALID_ARG on NULL arguments. */
emd_status emd_db_info_get(const emd_db* db, emd_db_info* out);

/* Distances from each query to every database histogram (Section 5: the vector t of
 * size n per query; Section 6: the maximum of both directions for EMD_DIR_MAX).
 *   q         host query batch (see emd_queries); every h_q in 1..max_query_h
 *   meas, k   measure and top-k width (k >= 1; ignored by RWMD, OMR, ICT)
 *   dir       direction
 *   out_dist  host float [n_queries * n_docs], row-major by query
 * Synchronous: returns after the results are in out_dist.
 * Errors: INVALID_ARG (bad query: weight < 0, sum off by > 1e-5, id out of range or
 * repeated, h_q out of range, k < 1), UNSUPPORTED (ACT with k > max_table_k; with the
 * approximate precisions, ICT forward with h_q > max_table_k or a re-rank width above 32),
 * CUDA. */
emd_status emd_query_batch(emd_db* db, const emd_queries* q, emd_measure meas, int32_t k,
                           emd_direction dir, float* out_dist);

/* The K nearest database histograms of each query (Section 6, top-l neighbours), in
 * ascending (distance, document id) order.
 * For EMD_DIR_MAX with K <= 16 (and prune_topk set) the reverse direction is evaluated
 * only where it can matter: max(fwd, rev) >= fwd, so the documents are taken in ascending
 * forward order, the reverse pass runs on the 63 best, and the answer is certified when the
 * K-th symmetric value is strictly below the 64th forward value; a query that fails the
 * test is recomputed over all documents.  The result equals the unpruned one.
 *   K         1..min(n_docs, 256)
 *   out_idx   host int64 [n_queries * K]; out_dist host float [n_queries * K]
 * Otherwise as emd_query_batch. */
emd_status emd_topk(emd_db* db, const emd_queries* q, emd_measure meas, int32_t k,
                    emd_direction dir, int32_t K, int64_t* out_idx, float* out_dist);

/* Device-resident variants: the same computations with inputs and outputs already in
 * device memory, stream-ordered on `stream` (a cudaStream_t; NULL is the CUDA default
 * stream, as in the CUDA runtime).  They return once the work is enqueued; the
 * workspace they use belongs to the handle, so two calls on one handle must be ordered
 * (same stream, or synchronised).
 *   q_row_ptr_host  HOST int64 [n_queries + 1] (launch sizes are taken from it)
 *   q_idx_dev, q_w_dev  DEVICE int32 / float [q_row_ptr_host[n_queries]]
 *   out_*_dev       DEVICE outputs with the host variants' layouts
 * Query weights are not validated (the caller guarantees them); ids outside 0..v-1 are
 * caught by a device-side bounds check that skips the access and latches an error read
 * by emd_db_check_device_errors.  The pruned top-K path (see emd_topk) reads one
 * certification flag per batch of max_batch queries, so emd_topk_device synchronises
 * `stream` once per such batch. */
emd_status emd_query_batch_device(emd_db* db, int64_t n_queries, const int64_t* q_row_ptr_host,
                                  const int32_t* q_idx_dev, const float* q_w_dev,
                                  emd_measure meas, int32_t k, emd_direction dir,
                                  float* out_dist_dev, void* stream);
emd_status emd_topk_device(emd_db* db, int64_t n_queries, const int64_t* q_row_ptr_host,
                           const int32_t* q_idx_dev, const float* q_w_dev, emd_measure meas,
                           int32_t k, emd_direction dir, int32_t K, int64_t* out_idx_dev,
                           float* out_dist_dev, void* stream);

/* Top-K selection over distance rows already in device memory, with no allocation.
 * The paper has no counterpart: this is a library service for callers that must not call
 * cudaMalloc -- code inside a host framework whose caching allocator owns all device
 * memory, or a serving loop that cannot absorb cudaMalloc's implicit synchronisation.
 * The selection kernels are the ones emd_topk / emd_topk_device run; their block-partial
 * scratch is a fixed 2 MiB array in the library's device memory (every GPU that loads
 * the library holds it until the process exits).
 *   t_dev        DEVICE float [n_rows * n], row-major distances (>= 0)
 *   n_rows       0..64 (the array holds partials for 64 rows); 0 is a no-op
 *   n            1..2^32-1; K in 1..min(n, 64)
 *   out_idx_dev  DEVICE int64 [n_rows * K]; out_dist_dev DEVICE float [n_rows * K]; each row
 *                in ascending (distance, index) order
 *   stream       cudaStream_t or NULL (the legacy default stream); returns once enqueued
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Calls share
 * the array, so calls whose kernels overlap on the GPU race; order them on one stream.
 * Errors: INVALID_ARG for sizes beyond the limits above or NULL pointers (nothing is
 * launched), CUDA. */
emd_status emd_topk_select_static(const float* t_dev, int64_t n_rows, int64_t n, int32_t K,
                                  int64_t* out_idx_dev, float* out_dist_dev, void* stream);

/* Synchronise the handle's streams and report (then clear) a latched device-side error:
 * EMD_OK, or INVALID_ARG when a kernel met an out-of-range id, or CUDA. */
emd_status emd_db_check_device_errors(emd_db* db);

/* Phase-1 table of one query, for inspection (Section 5: Z, S and W, each v_used x k,
 * rows in used-vocabulary order = ascending vocabulary id).
 *   used_ids  host int32 [v_used] (may be NULL): vocabulary id of each table row
 *   z, w      host float [v_used * k]; s host int32 [v_used * k] (query bin index)
 * Entries l >= h_q hold z = +inf, s = -1, w = 0.  k in 1..max_table_k. */
emd_status emd_phase1_table(emd_db* db, const int32_t* q_idx, const float* q_w, int32_t h_q,
                            int32_t k, int32_t* used_ids, float* z, int32_t* s, float* w);

/* Profiling: when on, every kernel launch is bracketed by CUDA events on its stream and
 * its time is added to its phase.  emd_db_profile_get synchronises and reads the sums;
 * emd_db_profile_reset clears them. */
emd_status emd_db_set_profiling(emd_db* db, int32_t on);
emd_status emd_db_profile_get(emd_db* db, emd_profile* out);
emd_status emd_db_profile_reset(emd_db* db);

/* All-pairs top-K over the database itself, the shape of the paper's evaluation (Section 6:
 * every histogram ranked against all others).  For each database histogram a, the K smallest
 * max(fwd(b -> a), fwd(a -> b)) over b != a, ordered by (distance, id), where fwd(x -> y) is
 * the forward bound (Section 5, Eq. 6-9) with histogram y as the query: the reverse bound of
 * a pair is the forward bound of the transposed pair, so one forward pass per histogram
 * gives both directions.  out_idx / out_dist: n_docs x K host arrays.  Needs 4 n_docs^2
 * bytes of device memory for the forward matrix during the call (OUT_OF_MEMORY otherwise);
 * every histogram must be within max_query_h bins (INVALID_ARG).  K <= 64, K < n_docs. */
emd_status emd_all_pairs_topk(emd_db* db, emd_measure meas, int32_t k, int32_t K, int64_t* out_idx,
                              float* out_dist);

/* The two cheap baselines the paper compares against (Section 6), on the same resident
 * database and query format:
 *   EMD_BOW_COSINE  bag-of-words cosine similarity: the dot product of the two weight
 *                   vectors after L2 normalisation (no embeddings, any database mode);
 *   EMD_WCD         word centroid distance: the Euclidean distance between the two
 *                   weight-averaged embedding vectors (embedding databases only, else
 *                   EMD_ERR_UNSUPPORTED).
 * emd_baseline_batch: out is n_queries x n_docs host floats (cosine similarity, or WCD).
 * emd_baseline_topk: the K nearest documents per query, by 1 - cosine (returned in
 * out_dist, clamped at 0) or by WCD, ties by lower document id; K <= 64.  Queries as for
 * emd_query_batch (1..max_query_h bins, distinct ids in range, weights summing to 1). */
typedef enum { EMD_BOW_COSINE = 0, EMD_WCD = 1 } emd_baseline;
emd_status emd_baseline_batch(emd_db* db, const emd_queries* q, emd_baseline kind, float* out);
emd_status emd_baseline_topk(emd_db* db, const emd_queries* q, emd_baseline kind, int32_t K, int64_t* out_idx,
                             float* out_dist);

/* Database sharding (several processes or devices, each holding a contiguous slice of the
 * documents in its own emd_db): the exact global top-K from the shards' top-K lists.
 * Every document of the global top-K is among its own shard's K_shard >= K best, so the K
 * smallest (distance, global id) pairs of the union are the answer; ties go to the lower
 * global id, as in emd_topk.  shard_idx[s] / shard_dist[s]: n_queries x K_shard host arrays
 * of shard s (local ids; negative ids are skipped); id_offset[s]: the global id of shard s's
 * first document.  out_idx / out_dist: n_queries x K.  Host computation only (no device is
 * needed); INVALID_ARG when a query has fewer than K results. */
emd_status emd_topk_merge(int32_t n_shards, const int64_t* const* shard_idx, const float* const* shard_dist,
                          const int64_t* id_offset, int64_t n_queries, int32_t K_shard, int32_t K,
                          int64_t* out_idx, float* out_dist);

/* ------------------------------------------------------------------ serving
 *
 * A request loop over a resident database.  Single queries are submitted as they arrive; a
 * worker thread forms batches from the head of the queue -- requests with the head's
 * (measure, k, K), in arrival order -- and runs each on one of two executors, each with its
 * own batch workspace and stream, with the batched kernel sequence of emd_topk (direction
 * EMD_DIR_MAX, Section 6).  Requests that arrive while a batch is on the GPU join the next
 * batch as soon as an executor is free (continuous batching).  Every query of a batch is
 * computed exactly as alone, so a result is bit-identical whether it was served alone or in
 * any mix, and equals emd_topk's.
 *
 * Admission: a batch takes requests while its executor's workspace holds them: the sum over
 * the batch of round_up(h_q, 32) distance-matrix columns (4 x v_used bytes each) may not
 * exceed the executor's columns (workspace_bytes / 2, or the database's batch_columns), at
 * most max_batch requests, and at most max_inflight requests on the device in all.  A
 * request that does not fit an empty executor is refused at submit.
 *
 * Threads: submit, poll and stats may be called from any host threads; one worker thread
 * per server issues the GPU work.  Calls on the database handle made while a server is
 * attached are serialised with the worker's launches. */
typedef struct emd_server emd_server;

typedef struct {
    int32_t max_inflight;    /* requests on the device at once, over both executors (default 128) */
    int32_t queue_capacity;  /* submitted but not yet admitted requests; beyond it submit
                                returns BUSY.  Default 4096 */
    int64_t workspace_bytes; /* device memory for the two executors' distance matrices; 0
                                (default): each gets the database's batch_columns.  Must hold at
                                least one request of max_query_h per executor */
    int32_t max_query_h;     /* largest accepted h_q; 0 (default) = the database's */
} emd_server_options;

typedef struct {
    int64_t submitted, completed, rejected_busy, failed, prune_fallbacks;
    int64_t queued, in_flight, max_in_flight;
    int64_t pool_bytes, pool_used_max;  /* executors' distance-matrix bytes; the most one batch used */
    double qps;              /* completed / (last completion - first submit), since reset */
    double latency_p50_us, latency_p99_us, latency_mean_us, latency_max_us; /* submit -> done */
} emd_server_stats;

void emd_server_options_default(emd_server_options* opt);

/* Attach a server to db (the handle must outlive it).  K is limited to 64 per request.  INVALID_ARG on bad options,
 * OUT_OF_MEMORY if the executors' workspaces or pinned staging cannot be allocated, CUDA. */
emd_status emd_server_create(emd_db* db, const emd_server_options* opt, emd_server** out);

/* Queue one query (h_q bins: vocabulary ids idx, weights w summing to 1, host memory, copied
 * during the call) for the symmetric top-K with measure meas and width k.  *ticket
 * identifies the result.  INVALID_ARG for the argument checks of emd_topk or a request
 * larger than an executor's workspace, BUSY when the queue is full, SHUTDOWN after destroy
 * began. */
emd_status emd_server_submit(emd_server* s, const int32_t* idx, const float* w, int32_t h_q,
                             emd_measure meas, int32_t k, int32_t K, uint64_t* ticket);

/* Wait up to timeout_ms (negative: no limit, 0: do not wait) for the result of ticket.
 * Ready: out_idx / out_dist (K entries each, host) are written, the ticket is released and
 * the status is OK (or the request's own failure status).  TIMEOUT if not ready yet (the
 * ticket stays valid); INVALID_ARG for an unknown or already collected ticket. */
emd_status emd_server_poll(emd_server* s, uint64_t ticket, int32_t timeout_ms, int64_t* out_idx,
                           float* out_dist);

/* Counters and latency percentiles since creation or the last reset. */
emd_status emd_server_stats_get(emd_server* s, emd_server_stats* out);
emd_status emd_server_stats_reset(emd_server* s);

/* Stop accepting requests, finish every admitted and queued request, release the server.
 * Results not collected are discarded.  NULL is accepted. */
emd_status emd_server_destroy(emd_server* s);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* emd_last_error(void);

/* Library version string. */
const char* emd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EMD_GB300_H */
