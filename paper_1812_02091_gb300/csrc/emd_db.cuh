// The database handle and the per-query kernel sequence, shared by the query entry points
// (emd_api.cu) and the server (emd_server.cu).  Internal to the library.
#pragma once

#include <cuda_fp16.h>

#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "emd_internal.cuh"

namespace emd {

// Record a formatted failure for emd_last_error() and return st.
emd_status fail(emd_status st, const char* fmt, ...);
emd_status cuda_fail(cudaError_t e, const char* what);

// One concurrent per-query pipeline: its stream and the workspace a query needs from
// Phase 1 to its distances (or its pruned top-K).
struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    float* Q = nullptr;          // qrows_max x ldm
    float* qnorm = nullptr;      // qrows_max
    __half* q_hi = nullptr;      // npad_max x kpad (tensor-core precision)
    __half* q_lo = nullptr;
    float* q_scale = nullptr;    // npad_max
    float* D = nullptr;          // v_used x ldd (ldd <= ldd_max)
    float2* tab = nullptr;       // v_used x max_table_k
    float* t_fwd = nullptr;      // n
    float* t_rev = nullptr;      // n
    int64_t* sel_idx = nullptr;  // kPruneMaxK forward top-K
    float* sel_val = nullptr;
    int64_t* cand_idx = nullptr; // kPruneCap candidates
    float* cand_sym = nullptr;   // 2 x kPruneCap
    int* cand_count = nullptr;
    unsigned long long* scratch = nullptr;  // kTopkScratchRow selection partials
};

}  // namespace emd

#define EMD_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return emd::cuda_fail(e_, what); \
    } while (0)

namespace emd {
// One captured batch sequence (launch_sequence) and the kernel launches it holds.
struct GraphKey {
    int meas, k, K, dir, pruned, slot, qcap;  // qcap: queries the grids cover (power of two)
    int fused;                                // fused pruned path allowed
    bool operator<(const GraphKey& o) const
    {
        if (fused != o.fused) return fused < o.fused;
        if (meas != o.meas) return meas < o.meas;
        if (k != o.k) return k < o.k;
        if (K != o.K) return K < o.K;
        if (dir != o.dir) return dir < o.dir;
        if (pruned != o.pruned) return pruned < o.pruned;
        if (slot != o.slot) return slot < o.slot;
        return qcap < o.qcap;
    }
};
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t launches[EMD_N_PHASES] = {};
    int64_t total = 0;
};
}  // namespace emd

namespace emd {
// Workspace of the batched form: every buffer a batch of up to max_batch queries and
// b_cols distance-matrix columns needs, the descriptor ring and the captured graphs (which
// bake these pointers in).  The database handle owns one for the host-API calls; each
// server executor owns its own.
struct BatchWS {
    static constexpr int kDescRing = 4;
    int max_batch = 0;
    std::vector<int64_t> order;   // host: query of each descriptor position (fill_descriptors)
    int64_t b_cols = 0, b_qrows = 0, b_prows = 0, b_tabcols = 0;
    float* bD = nullptr;          // v_used x b_cols: the batch's distance matrices side by side
    float* bQ = nullptr;          // b_qrows x ldm
    float* bqnorm = nullptr;      // b_qrows
    __half* bq_hi = nullptr;      // b_prows x kpad packed panels
    __half* bq_lo = nullptr;
    float* bq_scale = nullptr;    // b_prows
    float2* btab = nullptr;       // v_used x b_tabcols tables
    float* bt_fwd = nullptr;      // max_batch x n
    float* bt_rev = nullptr;      // max_batch x n
    float* bt_out = nullptr;      // max_batch x n (distances of unpruned top-K batches)
    int64_t* bsel_idx = nullptr;  // max_batch x kPruneMaxK
    float* bsel_val = nullptr;
    int64_t* bcand = nullptr;     // max_batch x kPruneCap
    float* bcand_sym = nullptr;   // max_batch x 2 kPruneCap
    int* bcand_count = nullptr;   // max_batch
    int* cand_ok = nullptr;       // max_batch certification flags
    int* ict_over = nullptr;      // max_batch ICT table overflow flags
    unsigned long long* topk_scratch = nullptr;  // max_batch x kTopkScratchRow
    // fused pruned path (allocated when the database can use it)
    bool fused = false;
    int32_t* bqpos = nullptr;     // max_batch x v_used, -1 between batches
    int32_t* brmap = nullptr;     // max_batch x v_used, -1 between batches
    int32_t* bcrows = nullptr;    // max_batch x kCandRows
    int* bncrows = nullptr;       // max_batch
    __half* bc_hi = nullptr;      // max_batch x kCandRows x kpad
    __half* bc_lo = nullptr;
    float* bc_scale = nullptr;    // max_batch x kCandRows
    float* bc_norm = nullptr;
    float* bDc = nullptr;         // kCandRows x b_cols
    __half* bqs_hi = nullptr;     // split query panels (BF16 / E4M3 databases), b_prows x kpad
    __half* bqs_lo = nullptr;
    float* bqs_scale = nullptr;
    int32_t* bcb = nullptr;       // max_batch x v_used x kCandPerRow candidate bins
    float* bcmax = nullptr;       // max_batch x v_used
    int32_t* brr = nullptr;       // max_batch x v_used uncertified rows
    int* brr_count = nullptr;     // max_batch
    QDesc* qd_dev = nullptr;      // kDescRing x max_batch descriptors
    int* nq_dev = nullptr;        // kDescRing counts
    QDesc* qd_host = nullptr;     // pinned mirror of the ring
    int* nq_host = nullptr;
    cudaEvent_t desc_ev[kDescRing] = {};
    int desc_slot = 0;
    cudaStream_t cap_stream = nullptr;  // graph capture
    std::map<GraphKey, GraphEntry> graphs;
};
}  // namespace emd

struct emd_db {
    int dev = 0;
    cudaStream_t stream = nullptr;  // host-buffer entry points run here
    cudaEvent_t fork = nullptr;
    emd_db_options opt{};
    int64_t v = 0, v_used = 0, n = 0, nnz = 0;
    int m = 0, ldm = 0;
    bool cost_mode = false;

    // resident database
    float* emb = nullptr;        // v x ldm, full vocabulary (queries gather from it)
    float* emb_used = nullptr;   // v_used x ldm, used vocabulary (Section 2.2)
    float* norm_used = nullptr;  // v_used, squared norms
    int32_t* used_ids = nullptr; // v_used, vocabulary id of each used row (ascending)
    float* cost = nullptr;       // v x v ground costs (cost-matrix mode)
    int32_t* row_ptr = nullptr;  // n + 1
    std::vector<int64_t> row_ptr_host;  // the same offsets on the host (all-pairs batching)
    int32_t* col = nullptr;      // nnz, renumbered into the used vocabulary
    float* val = nullptr;        // nnz
    int* err = nullptr;

    // tensor-core operands of the used vocabulary (precisions FP32_TC, BF16, FP8_E4M3)
    bool tc = false;
    int tcfmt = -1;              // TC_SPLIT, TC_BF16, TC_E4M3 (TC_NONE: SIMT FP32)
    bool approx = false;         // BF16 / E4M3: the table re-ranks with exact FP32 distances
    int margin = 8;              // re-rank candidates beyond k
    int kpad = 0;
    int64_t mpad = 0;
    __half* a_hi = nullptr;      // mpad x kpad packed panels (2-byte elements; E4M3 uses half the bytes)
    __half* a_lo = nullptr;      // TC_SPLIT only
    float* a_scale = nullptr;    // mpad
    // FP16-split panels of the used vocabulary for the fused path's exact candidate block: the
    // panels above for FP32_TC, a copy in the split format for BF16 / E4M3 databases
    __half* as_hi = nullptr;
    __half* as_lo = nullptr;
    float* as_scale = nullptr;

    // per-lane workspace
    int ldd_max = 0, qrows_max = 0;
    std::vector<emd::Lane> lanes;
    int32_t* tab_s = nullptr;    // v_used x max_table_k (inspection entry point only)

    // batch workspace (shared by the lanes, one row per query of a batch)
    unsigned long long* topk_scratch = nullptr;  // max_batch x kTopkScratchRow
    int* cand_ok = nullptr;        // max_batch certification flags
    int* ict_over = nullptr;       // max_batch ICT table overflow flags (lanes path)
    float* xmax = nullptr;         // v_used, the largest database weight at each used row
    int32_t* vslot = nullptr;      // v: used-vocabulary row of each id, -1 if unused
    int64_t stage_bins = 0;
    int32_t* stage_idx = nullptr;
    float* stage_w = nullptr;
    float* stage_out = nullptr;      // max_batch x n
    int64_t* stage_oidx = nullptr;   // max_batch x kMaxTopK
    float* stage_odist = nullptr;    // max_batch x kMaxTopK

    int64_t bytes = 0;
    std::vector<void*> allocs;

    // profiling
    bool profiling = false;
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[EMD_N_PHASES] = {};
    int64_t launches[EMD_N_PHASES] = {};
    int64_t total_launches = 0;
    int64_t pruned_queries = 0, prune_fallbacks = 0;

    // batched form (opt.batched): the workspace of the host-API batches
    emd::BatchWS bw;
    int64_t graph_launches = 0;   // batch sequences replayed from graphs (all workspaces)
    int64_t ict_wide = 0;         // ICT queries recomputed with full-width tables
    int64_t fused_retries = 0;    // pruned queries rerun with the full matrix (candidate block overflow)

    // free parameters of the batched kernels (autotune at creation)
    bool autotuned = false;
    int tune_group_mult = 1;   // query groups per vocabulary tile, times the balance minimum
    int tune_stages = 0;       // B stages of the batched tensor-core kernel (0: as many as fit)
    int tune_rev_warps = 4;    // warps per candidate document in the pruned reverse pass
    int tune_fwd = 0;          // form of the grouped forward sweep (kFwd*)
    std::map<emd::GraphKey, emd::GraphEntry> graphs;

    // Section 6 baselines (allocated and prepared at first use)
    float* bow_dense = nullptr;     // ceil(max_batch / 8) x v_used x 8 interleaved query vectors
    float* doc_inv_norm = nullptr;  // n
    float* doc_centroid = nullptr;  // n x ldc (word centroid distance)
    float* q_centroid = nullptr;    // max_batch x ldc
    int64_t* base_rp = nullptr;     // max_batch + 1 query offsets of a batch
    int ldc = 0;
    bool bow_ready = false, wcd_ready = false;

    // Serialises the entry points that launch work or touch the counters above (host
    // threads, and the server's worker thread).
    std::mutex mu;
    std::atomic<int> servers{0};  // attached servers (emd_server_create)
};


namespace emd {

cudaEvent_t take_event(emd_db* db);

// Brackets the kernels of one phase with events (when profiling) and counts launches.
// With several lanes the phases of different queries overlap, so phase sums can exceed
// the wall time of a batch.
struct Phase {
    emd_db* db;
    int ph;
    int nlaunch;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Phase(emd_db* d, int p, int nl, cudaStream_t s) : db(d), ph(p), nlaunch(nl), st(s)
    {
        if (db->profiling) {
            a = take_event(db);
            cudaEventRecord(a, st);
        }
    }
    ~Phase()
    {
        db->launches[ph] += nlaunch;
        db->total_launches += nlaunch;
        if (db->profiling) {
            cudaEvent_t b = take_event(db);
            cudaEventRecord(b, st);
            db->recs.push_back({ph, a, b});
        }
    }
};

// Forward table width of a query with h bins.  ICT (FP32 distances): at most max_table_k
// entries, rows ending where the largest database weight of the row is placed.
int table_width(const emd_db* db, int meas, int k, int h);
// Candidates per row re-ranked by the table kernel of the approximate precisions.
int rerank_width(const emd_db* db, int tk, int h);
emd_status check_query_values(const emd_db* db, const emd_queries* q);
bool prunable(const emd_db* db, int meas, int k, int dir, int K);
int topk_launch_count(int64_t n);

// One query through Phase 1 and the forward and/or reverse pass on lane L's workspace;
// out_t (n floats, device) receives the distances.  ICT: with `over` (device flag) the
// table is at most max_table_k wide and *over = 1 marks a query that needed more; without
// it the table is h wide (temporary device memory when above max_table_k), always exact.
// Caller holds db->mu.
emd_status run_query(emd_db* db, Lane& L, const int32_t* qidx, const float* qw, int h, int meas, int k,
                     int dir, float* out_t, int* over, cudaStream_t st);

// Pruned max-direction top-K of one query (K <= kPruneMaxK); *ok (device) receives the
// certificate, *over the ICT overflow flag.  Caller holds db->mu.
emd_status run_topk_pruned(emd_db* db, Lane& L, const int32_t* qidx, const float* qw, int h, int meas, int k,
                           int K, int* ok, int* over, int64_t* out_idx, float* out_dist, cudaStream_t st);

// Batch workspaces (emd_api.cu).  alloc_batch_ws records its device allocations in
// `allocs` (freed by the owner) and adds their size to *bytes; free_batch_ws releases the
// rest (pinned ring, events, capture stream, graphs).
emd_status alloc_batch_ws(emd_db* db, BatchWS& ws, int max_batch, int64_t cols, std::vector<void*>& allocs,
                          int64_t* bytes);
void free_batch_ws(BatchWS& ws);

// Sub-batch j0..j1-1 of the queries i0.. (host rp, device qidx / qw relative to query i0)
// on ws, in ring slot order: descriptors, then the batched sequence (graph replay when
// enabled) on st.  Outputs: out_t rows (K = 0), else out_idx / out_dist rows, relative to
// i0; certification flags in ws.cand_ok[i - i0] on the pruned path.  Caller holds db->mu.
emd_status run_subbatch(emd_db* db, BatchWS& ws, const int64_t* rp, const int32_t* qidx, const float* qw,
                        int64_t i0, int64_t j0, int64_t j1, int meas, int k, int dir, int K, bool pruned,
                        float* out_t, int64_t* out_idx, float* out_dist, cudaStream_t st, bool allow_fused = true);
// Pruned query i (of the batch starting at i0) whose fused candidate block overflowed: run
// again alone on ws with the full distance matrix; *ok receives its new certification flag.
emd_status retry_materialized(emd_db* db, BatchWS& ws, const int64_t* rp, const int32_t* qidx, const float* qw,
                              int64_t i0, int64_t i, int meas, int k, int K, int64_t* out_idx, float* out_dist,
                              cudaStream_t st, int* ok);
// Whether the batch (rp entries i0..i1) fits one sub-batch of ws.
bool batch_fits(const emd_db* db, const BatchWS& ws, const int64_t* rp, int64_t i0, int64_t i1, int meas, int k,
                int dir);

}  // namespace emd
