// C ABI (include/emd.h): argument checks, the device-resident database, the workspace,
// and the per-query sequence of kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <string>
#include <vector>

#include "emd_db.cuh"

using namespace emd;

namespace {
thread_local std::string g_err;
}  // namespace

namespace emd {

emd_status fail(emd_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

emd_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? EMD_ERR_OUT_OF_MEMORY : EMD_ERR_CUDA,
                "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace emd

namespace emd {
// Record a failure message for emd_last_error() from another translation unit.
emd_status set_error(emd_status st, const char* msg)
{
    g_err = msg;
    return st;
}
void clear_error() { g_err.clear(); }
}  // namespace emd

namespace emd {

template <typename T>
emd_status dalloc(emd_db* db, T** p, int64_t count)
{
    size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EMD_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    db->allocs.push_back(q);
    db->bytes += (int64_t)bytes;
    *p = (T*)q;
    return EMD_OK;
}

void release(emd_db* db)
{
    if (!db) return;
    cudaSetDevice(db->dev);
    cudaDeviceSynchronize();
    for (void* p : db->allocs) cudaFree(p);
    free_batch_ws(db->bw);
    for (auto& r : db->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : db->pool) cudaEventDestroy(e);
    for (auto& L : db->lanes) {
        if (L.done) cudaEventDestroy(L.done);
        if (L.st) cudaStreamDestroy(L.st);
    }
    if (db->fork) cudaEventDestroy(db->fork);
    if (db->stream) cudaStreamDestroy(db->stream);
    delete db;
}

cudaEvent_t take_event(emd_db* db)
{
    if (!db->pool.empty()) {
        cudaEvent_t e = db->pool.back();
        db->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Whether a batch's forward tables are interleaved in groups of kFwdGroup queries (one CSR
// sweep per group): register-width tables, and ICT tables (the loop form) when a group of
// them fits the workspace's table columns.
// The fused FP32_TC table runs on SM pairs when the option asks for it and the panel fits.
bool use_tc_pair(const emd_db* db)
{
    return db->opt.tc_pair > 0 && db->tc && db->tcfmt == TC_SPLIT && !db->cost_mode && db->mpad % 256 == 0 &&
           tc_table_pair_fits(db->kpad);
}

bool grouped_tables(const BatchWS& ws, int meas, int tk_b)
{
    return tk_b > 0 && (tk_b <= 16 || (meas == M_ICT && (int64_t)kFwdGroup * tk_b <= ws.b_tabcols));
}

// Row width of a query's table in the grouped, query-major layout (the forward kernel's
// register width), or 0 for the entry-interleaved layout of wide ICT tables.
int grouped_width(const emd_db* db, int meas, int tk_b)
{
    if (db->tune_fwd != kFwdRowMajor || (meas == M_ICT && tk_b > 16)) return 0;
    return fwd_reg_width(tk_b);
}

int topk_launch_count(int64_t n) { return topk_blocks(n) > 1 ? 2 : 1; }

int table_width(const emd_db* db, int meas, int k, int h)
{
    switch (meas) {
    case M_RWMD: return 1;
    case M_OMR: return std::min(2, h);
    case M_ICT: return db->approx ? h : std::min(h, db->opt.max_table_k);
    default: return std::min(k, h);
    }
}

emd_status check_request(const emd_db* db, int meas, int k, int dir)
{
    if (meas < EMD_RWMD || meas > EMD_ICT) return fail(EMD_ERR_INVALID_ARG, "unknown measure %d", meas);
    if (dir < EMD_DIR_FWD || dir > EMD_DIR_MAX) return fail(EMD_ERR_INVALID_ARG, "unknown direction %d", dir);
    if (meas == EMD_ACT && k < 1) return fail(EMD_ERR_INVALID_ARG, "k must be >= 1 (got %d)", k);
    (void)db;
    return EMD_OK;
}

emd_status check_sizes(const emd_db* db, int64_t nq, const int64_t* rp, int meas, int k, int dir)
{
    if (nq < 0) return fail(EMD_ERR_INVALID_ARG, "n_queries < 0");
    if (nq == 0) return EMD_OK;
    if (!rp) return fail(EMD_ERR_INVALID_ARG, "query row_ptr is NULL");
    if (rp[0] != 0) return fail(EMD_ERR_INVALID_ARG, "query row_ptr[0] != 0");
    for (int64_t i = 0; i < nq; ++i) {
        int64_t h = rp[i + 1] - rp[i];
        if (h < 1 || h > db->opt.max_query_h)
            return fail(EMD_ERR_INVALID_ARG, "query %lld has %lld bins (allowed 1..%d)", (long long)i,
                        (long long)h, db->opt.max_query_h);
        if (dir != EMD_DIR_REV && table_width(db, meas, k, (int)h) > db->opt.max_table_k)
            return fail(EMD_ERR_UNSUPPORTED, "forward table width %d exceeds max_table_k %d",
                        table_width(db, meas, k, (int)h), db->opt.max_table_k);
        if (dir != EMD_DIR_REV && db->approx && rerank_width(db, table_width(db, meas, k, (int)h), (int)h) > kRerankMax)
            return fail(EMD_ERR_UNSUPPORTED, "re-rank width %d exceeds %d (approximate precisions)",
                        rerank_width(db, table_width(db, meas, k, (int)h), (int)h), kRerankMax);
    }
    return EMD_OK;
}

emd_status check_query_values(const emd_db* db, const emd_queries* q)
{
    if (q->n_queries == 0) return EMD_OK;
    if (!q->idx || !q->w) return fail(EMD_ERR_INVALID_ARG, "query idx or w is NULL");
    std::vector<int64_t> stamp((size_t)db->v, -1);
    for (int64_t i = 0; i < q->n_queries; ++i) {
        double s = 0.0;
        for (int64_t e = q->row_ptr[i]; e < q->row_ptr[i + 1]; ++e) {
            int32_t id = q->idx[e];
            float w = q->w[e];
            if (id < 0 || id >= db->v)
                return fail(EMD_ERR_INVALID_ARG, "query %lld: id %d out of range", (long long)i, id);
            if (stamp[id] == i)
                return fail(EMD_ERR_INVALID_ARG, "query %lld: id %d repeated", (long long)i, id);
            stamp[id] = i;
            if (!(w >= 0.f) || !isfinite(w))
                return fail(EMD_ERR_INVALID_ARG, "query %lld: weight %g invalid", (long long)i, (double)w);
            s += w;
        }
        if (fabs(s - 1.0) > 1e-5)
            return fail(EMD_ERR_INVALID_ARG, "query %lld: weights sum to %.9g, not 1", (long long)i, s);
    }
    return EMD_OK;
}

// Phase 1 (distances, or the cost-matrix gather) for one query into the lane's D.
emd_status run_phase1(emd_db* db, Lane& L, const int32_t* qidx, int h, cudaStream_t st)
{
    const int ldd = (int)round_up(h, 32);
    const int qrows = (int)round_up(ldd, kDistBN);
    if (db->cost_mode) {
        Phase p(db, 1, 1, st);
        EMD_CUDA(launch_dist_gather(db->cost, db->v, db->used_ids, db->v_used, qidx, h, L.D, ldd,
                                    db->err, st), "distance gather");
        return EMD_OK;
    }
    {
        Phase p(db, 0, db->tc ? 2 : 1, st);
        EMD_CUDA(launch_gather_rows(db->emb, db->v, db->ldm, db->m, qidx, h, qrows, L.Q, L.qnorm,
                                    db->err, st), "query gather");
        if (db->tc)
            EMD_CUDA(launch_pack(db->tcfmt, L.Q, db->ldm, db->m, h, round_up(h, 128), db->kpad, L.q_hi,
                                 db->tcfmt == TC_SPLIT ? L.q_lo : nullptr, L.q_scale, st), "query pack");
    }
    Phase p(db, 1, db->tc ? 2 : 1, st);
    if (db->tc) {
        EMD_CUDA(launch_tc_dist(db->tcfmt, db->a_hi, db->a_lo, db->mpad, db->a_scale, db->norm_used, db->v_used,
                                L.q_hi, db->tcfmt == TC_SPLIT ? L.q_lo : nullptr, round_up(h, 128), L.q_scale,
                                L.qnorm, h, db->kpad, L.D, ldd, db->err, st),
                 "distance matrix (tensor cores)");
        EMD_CUDA(launch_zero_ident(qidx, h, db->vslot, db->v, L.D, ldd, st), "identical ids");
    } else
        EMD_CUDA(launch_dist_fp32(db->emb_used, db->v_used, db->ldm, db->norm_used, db->used_ids, L.Q, h,
                                  db->ldm, L.qnorm, qidx, db->m, L.D, ldd, st), "distance matrix");
    return EMD_OK;
}

int rerank_width(const emd_db* db, int tk, int h) { return std::min(tk + db->margin, h); }

// The Phase-1 table of width tk from lane L's D (re-ranked for the approximate precisions).
emd_status run_table(emd_db* db, Lane& L, const float* qw, int h, int meas, int tk, float2* tab, int32_t* tab_s,
                     int* over, cudaStream_t st)
{
    const int ldd = (int)round_up(h, 32);
    Phase p(db, 2, 1, st);
    if (meas == M_ICT && !db->approx)
        EMD_CUDA(launch_table_ict(L.D, ldd, db->v_used, h, tk, qw, db->xmax, tab, tab_s, over, !db->cost_mode, st),
                 "ICT table");
    else if (db->approx)
        EMD_CUDA(launch_table_rerank(L.D, ldd, db->v_used, h, tk, rerank_width(db, tk, h), db->emb_used, L.Q,
                                     db->ldm, qw, tab, tab_s, st), "top-k table (re-ranked)");
    else
        EMD_CUDA(launch_table(L.D, ldd, db->v_used, h, tk, qw, tab, tab_s, !db->cost_mode, st), "top-k table");
    return EMD_OK;
}

// One query through Phase 1, the forward and/or reverse pass; out_t (n floats) receives
// the distances.
emd_status run_query(emd_db* db, Lane& L, const int32_t* qidx, const float* qw, int h, int meas, int k,
                     int dir, float* out_t, int* over, cudaStream_t st)
{
    emd_status s0 = run_phase1(db, L, qidx, h, st);
    if (s0 != EMD_OK) return s0;
    const int ldd = (int)round_up(h, 32);
    if (dir != EMD_DIR_REV) {
        const bool wide = meas == M_ICT && !db->approx && !over;  // the whole row if needed
        const int tk = wide ? h : table_width(db, meas, k, h);
        float2* tab = L.tab;
        if (tk > db->opt.max_table_k)
            EMD_CUDA(cudaMallocAsync((void**)&tab, (size_t)db->v_used * tk * sizeof(float2), st), "ICT table memory");
        emd_status s1 = run_table(db, L, qw, h, meas, tk, tab, nullptr, over, st);
        if (s1 == EMD_OK) {
            Phase p(db, 3, 1, st);
            const cudaError_t e = launch_fwd(meas, db->row_ptr, db->col, db->val, db->n, tab, tk, tk,
                                             dir == EMD_DIR_FWD ? out_t : L.t_fwd, st);
            if (e != cudaSuccess) s1 = cuda_fail(e, "forward pass");
        }
        if (tab != L.tab) cudaFreeAsync(tab, st);
        if (s1 != EMD_OK) return s1;
    }
    if (dir != EMD_DIR_FWD) {
        Phase p(db, 4, 1, st);
        EMD_CUDA(launch_rev(meas, k, db->row_ptr, db->col, db->val, db->n, L.D, ldd, h, qw,
                            L.t_fwd, dir == EMD_DIR_REV ? out_t : L.t_rev,
                            dir == EMD_DIR_MAX ? out_t : nullptr, nullptr, !db->cost_mode, st),
                 "reverse pass");
    }
    return EMD_OK;
}

bool prunable(const emd_db* db, int meas, int k, int dir, int K)
{
    return db->opt.prune_topk != 0 && dir == EMD_DIR_MAX && K <= kPruneMaxK &&
           (meas != EMD_ICT || !db->approx) && (meas != EMD_ACT || k <= kMaxRegK);
}

// Pruned symmetric top-K of one query (see emd_topk in include/emd.h): forward pass over
// all documents, forward top-K, candidates within the margin, reverse pass on them, final
// selection with the certification flag in *ok.
emd_status run_topk_pruned(emd_db* db, Lane& L, const int32_t* qidx, const float* qw, int h, int meas, int k,
                           int K, int* ok, int* over, int64_t* out_idx, float* out_dist, cudaStream_t st)
{
    emd_status s = run_phase1(db, L, qidx, h, st);
    if (s != EMD_OK) return s;
    const int ldd = (int)round_up(h, 32);
    const int tk = table_width(db, meas, k, h);
    s = run_table(db, L, qw, h, meas, tk, L.tab, nullptr, over, st);
    if (s != EMD_OK) return s;
    {
        Phase p(db, 3, 1, st);
        EMD_CUDA(launch_fwd(meas, db->row_ptr, db->col, db->val, db->n, L.tab, tk, tk, L.t_fwd, st),
                 "forward pass");
    }
    {
        Phase p(db, 5, topk_launch_count(db->n), st);
        EMD_CUDA(launch_topk(L.t_fwd, db->n, K, L.scratch, L.sel_idx, L.sel_val, st), "forward top-K");
    }
    Phase p(db, 4, 3, st);
    EMD_CUDA(launch_prune(meas, k, db->row_ptr, db->col, db->val, db->n, L.D, ldd, h, qw, L.t_fwd,
                          L.sel_idx, L.sel_val, K, L.cand_idx, L.cand_count, L.cand_sym, out_idx,
                          out_dist, ok, !db->cost_mode, st),
             "pruned reverse pass");
    return EMD_OK;
}

// Top-K of `rows` distance rows (row stride n) in one selection launch.
emd_status select_topk(emd_db* db, const float* t, int64_t rows, int K, int64_t* out_idx,
                       float* out_dist, cudaStream_t st)
{
    Phase p(db, 5, topk_launch_count(db->n), st);
    EMD_CUDA(launch_topk_rows(t, rows, db->n, db->n, K, db->topk_scratch, out_idx, out_dist, st), "top-K");
    return EMD_OK;
}

// Queries i0..i1-1 (at most max_batch) on the lanes, ordered after and joined back into
// `st`.  qidx / qw point at query i0's bins (rp gives every query's offset).  With K > 0
// the top-K goes to out_idx / out_dist (rows relative to i0); otherwise the distances go
// to out_t (rows relative to i0, row stride n).  The pruned path reads its certification
// flags once (synchronising `st`) and recomputes uncertified queries over all documents.
emd_status run_lanes(emd_db* db, const int64_t* rp, const int32_t* qidx, const float* qw, int64_t i0,
                     int64_t i1, int meas, int k, int dir, int K, bool pruned, float* out_t, int64_t* out_idx,
                     float* out_dist, cudaStream_t st);

// The kernels of one sub-batch whose descriptors sit in ring slot `slot`.  Grids are sized
// from bounds (qcap queries, max_query_h bins, the table width of k) and every block checks
// the query count on the device, so the same sequence serves every batch of at most qcap
// queries with these parameters and can be captured into a graph.  hd (host descriptors of
// nb queries) only when Phase 1 must run per query.
emd_status launch_sequence(BatchWS& ws, emd_db* db, int slot, int meas, int k, int K, int dir, bool pruned, const QDesc* hd,
                           int nb, int qcap, cudaStream_t st, bool allow_fused = true)
{
    const int B = qcap;  // grids cover qcap queries (>= the batch's count)
    const QDesc* D_ = ws.qd_dev + (int64_t)slot * ws.max_batch;
    const int* nqd = ws.nq_dev + slot;
    const int64_t n = db->n;
    const int H = db->opt.max_query_h;
    const int tk_b = dir != EMD_DIR_REV ? table_width(db, meas, k, H) : 0;
    const int kc_b = db->approx ? std::min(rerank_width(db, tk_b, H), kRerankMax) : tk_b;
    if (pruned && allow_fused && ws.fused && !hd && meas != M_ICT && tk_b <= 16 &&
        (!db->approx || kc_b <= kCandPerRow)) {
        // fused form: the table from the product's epilogue (approximate formats: candidates
        // re-ranked exactly); the reverse direction's distances on the candidate documents' rows
        // only, exact in the FP16 split
        {
            Phase p(db, 0, db->approx ? 3 : 2, st);
            const int prow = (int)round_up(H, 128);
            EMD_CUDA(launch_gather_rows_b(D_, nqd, B, db->qrows_max, db->emb, db->v, db->ldm, db->m, db->err, st),
                     "query gather");
            EMD_CUDA(launch_pack_b(db->tcfmt, D_, nqd, B, prow, db->ldm, db->m, db->kpad, st), "query pack");
            if (db->approx)
                EMD_CUDA(launch_pack_b(TC_SPLIT, D_, nqd, B, prow, db->ldm, db->m, db->kpad, st, true),
                         "query pack (split)");
        }
        {
            Phase p(db, 1, 2, st);
            EMD_CUDA(launch_qpos_b(D_, nqd, B, db->vslot, db->v, true, st), "identical ids");
            if (use_tc_pair(db))
                EMD_CUDA(launch_tc_table_pair(db->a_hi, db->a_lo, db->mpad, db->a_scale, db->norm_used, db->v_used,
                                              D_, nqd, B, db->kpad, db->m, tk_b, db->tune_group_mult,
                                              db->opt.tc_pair == 1 ? 64 : 128, db->err, st),
                         "Phase-1 table (tensor cores on SM pairs, fused)");
            else
                EMD_CUDA(launch_tc_table_batch(db->tcfmt, db->a_hi, db->a_lo, db->mpad, db->a_scale, db->norm_used,
                                               db->v_used, D_, nqd, B, db->kpad, db->m, db->approx ? kc_b : tk_b,
                                               db->tune_group_mult, db->tune_stages, db->err, st),
                         db->approx ? "Phase-1 candidates (tensor cores, fused)"
                                    : "Phase-1 table (tensor cores, fused)");
        }
        if (db->approx) {
            // BF16: certified rows exact by construction; E4M3's rounding bound is too wide for a
            // certificate, its tables are the re-ranked candidates (R15)
            const bool certify = db->tcfmt == TC_BF16;
            const double u = 1.0 / 256.0;
            const float eps_rel = (float)(2.0 * (2.0 * u + u * u + 4e-5) * (1.0 + 1.0 / 1024.0));
            const float eps_abs = (float)(8.0 / 16777216.0);
            EMD_CUDA(cudaMemsetAsync(ws.brr_count, 0, sizeof(int) * B, st), "re-rank rows");
            Phase p(db, 2, certify ? 2 : 1, st);
            EMD_CUDA(launch_rerank_cand_b(D_, nqd, B, db->v_used, H, db->emb_used, db->ldm, db->norm_used, certify,
                                          eps_rel, eps_abs, st),
                     "top-k table (re-ranked candidates)");
            if (certify)
                EMD_CUDA(launch_rerank_full_b(D_, nqd, B, tk_b, db->emb_used, db->ldm, st), "top-k table (full rows)");
        }
        {
            Phase p(db, 3, 1, st);
            EMD_CUDA(launch_fwd_b(meas, D_, nqd, B, db->row_ptr, db->col, db->val, n, false,
                                  grouped_tables(ws, meas, tk_b), tk_b, st, db->tune_fwd),
                     "forward pass");
        }
        {
            Phase p(db, 5, topk_launch_count(n), st);
            EMD_CUDA(launch_topk_b(D_, nqd, B, n, K, ws.topk_scratch, true, st), "forward top-K");
        }
        EMD_CUDA(cudaMemsetAsync(ws.bcand_count, 0, sizeof(int) * B, st), "candidate counts");
        EMD_CUDA(cudaMemsetAsync(ws.bncrows, 0, sizeof(int) * B, st), "candidate rows");
        {
            Phase p(db, 4, 1, st);
            EMD_CUDA(launch_prune_compact_b(D_, nqd, B, n, K, st), "candidates");
        }
        {
            Phase p(db, 1, 3, st);
            EMD_CUDA(launch_cand_rows_b(D_, nqd, B, db->row_ptr, db->col, false, st), "candidate rows");
            EMD_CUDA(launch_cand_pack_b(D_, nqd, B, db->as_hi, db->as_lo, db->mpad, db->as_scale, db->norm_used,
                                        db->kpad, st),
                     "candidate panels");
            EMD_CUDA(launch_tc_cand_batch(D_, nqd, B, db->kpad, db->tune_stages, db->err, st),
                     "candidate distances (tensor cores)");
        }
        {
            Phase p(db, 4, 2, st);
            EMD_CUDA(launch_prune_mapped_b(meas, k, D_, nqd, B, db->row_ptr, db->col, db->val, K, db->tune_rev_warps,
                                           st),
                     "pruned reverse pass");
        }
        Phase p(db, 6, 2, st);
        EMD_CUDA(launch_cand_rows_b(D_, nqd, B, db->row_ptr, db->col, true, st), "candidate reset");
        EMD_CUDA(launch_qpos_b(D_, nqd, B, db->vslot, db->v, false, st), "identical ids");
        return EMD_OK;
    }
    if (db->cost_mode) {
        Phase p(db, 1, 1, st);
        EMD_CUDA(launch_dist_gather_b(D_, nqd, B, db->cost, db->v, db->used_ids, db->v_used, db->err, st),
                 "distance gather");
    } else {
        {
            Phase p(db, 0, db->tc ? 2 : 1, st);
            EMD_CUDA(launch_gather_rows_b(D_, nqd, B, db->qrows_max, db->emb, db->v, db->ldm, db->m, db->err, st),
                     "query gather");
            if (db->tc)
                EMD_CUDA(launch_pack_b(db->tcfmt, D_, nqd, B, (int)round_up(H, 128), db->ldm, db->m, db->kpad, st),
                         "query pack");
        }
        if (db->tc && !hd) {
            Phase p(db, 1, 2, st);
            EMD_CUDA(launch_tc_dist_batch(db->tcfmt, db->a_hi, db->a_lo, db->mpad, db->a_scale, db->norm_used,
                                          db->v_used, D_, nqd, B, db->kpad, db->m, db->tune_group_mult,
                                          db->tune_stages,
                                          db->err, st),
                     "distance matrices (tensor cores, batched)");
            EMD_CUDA(launch_zero_ident_b(D_, nqd, B, H, db->vslot, db->v, st), "identical ids");
        } else if (db->tc) {
            Phase p(db, 1, nb + 1, st);
            for (int q = 0; q < nb; ++q) {
                const QDesc& d = hd[q];
                EMD_CUDA(launch_tc_dist(db->tcfmt, db->a_hi, db->a_lo, db->mpad, db->a_scale, db->norm_used,
                                        db->v_used, d.q_hi, d.q_lo, d.npad, d.q_scale, d.qnorm, d.h, db->kpad, d.D,
                                        d.ldd, db->err, st),
                         "distance matrix (tensor cores)");
            }
            EMD_CUDA(launch_zero_ident_b(D_, nqd, B, H, db->vslot, db->v, st), "identical ids");
        } else {
            Phase p(db, 1, 1, st);
            EMD_CUDA(launch_dist_fp32_b(D_, nqd, B, db->ldd_max, db->emb_used, db->v_used, db->ldm, db->norm_used,
                                        db->used_ids, db->m, st),
                     "distance matrix");
        }
    }
    if (dir != EMD_DIR_REV) {
        {
            Phase p(db, 2, 1, st);
            if (meas == M_ICT && !db->approx)
                EMD_CUDA(launch_table_ict_b(D_, nqd, B, db->v_used, db->xmax, st), "ICT table");
            else
                EMD_CUDA(launch_table_b(D_, nqd, B, db->v_used, tk_b, db->approx, kc_b, H, db->emb_used, db->ldm, st),
                         "top-k table");
        }
        Phase p(db, 3, 1, st);
        EMD_CUDA(launch_fwd_b(meas, D_, nqd, B, db->row_ptr, db->col, db->val, n, dir == EMD_DIR_FWD,
                              grouped_tables(ws, meas, tk_b), tk_b, st, db->tune_fwd),
                 "forward pass");
    }
    if (pruned) {
        {
            Phase p(db, 5, topk_launch_count(n), st);
            EMD_CUDA(launch_topk_b(D_, nqd, B, n, K, ws.topk_scratch, true, st), "forward top-K");
        }
        EMD_CUDA(cudaMemsetAsync(ws.bcand_count, 0, sizeof(int) * B, st), "candidate counts");
        Phase p(db, 4, 3, st);
        EMD_CUDA(launch_prune_b(meas, k, D_, nqd, B, db->row_ptr, db->col, db->val, n, K, db->tune_rev_warps, st),
                 "pruned reverse pass");
        return EMD_OK;
    }
    if (dir != EMD_DIR_FWD) {
        Phase p(db, 4, 1, st);
        EMD_CUDA(launch_rev_b(meas, k, dir, D_, nqd, B, db->row_ptr, db->col, db->val, n, st), "reverse pass");
    }
    if (K > 0) {
        Phase p(db, 5, topk_launch_count(n), st);
        EMD_CUDA(launch_topk_b(D_, nqd, B, n, K, ws.topk_scratch, false, st), "top-K");
    }
    return EMD_OK;
}

// Captures launch_sequence for these parameters into an executable graph (on the handle's
// capture stream); the launch counts of one replay are kept beside it.
emd_status capture_sequence(BatchWS& ws, emd_db* db, int slot, int meas, int k, int K, int dir, bool pruned, int qcap,
                            GraphEntry* g, bool allow_fused)
{
    int64_t l0[EMD_N_PHASES], t0 = db->total_launches;
    for (int p = 0; p < EMD_N_PHASES; ++p) l0[p] = db->launches[p];
    cudaStream_t cs = ws.cap_stream;
    EMD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "graph capture");
    emd_status s = launch_sequence(ws, db, slot, meas, k, K, dir, pruned, nullptr, 0, qcap, cs, allow_fused);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    for (int p = 0; p < EMD_N_PHASES; ++p) {
        g->launches[p] = db->launches[p] - l0[p];
        db->launches[p] = l0[p];
    }
    g->total = db->total_launches - t0;
    db->total_launches = t0;
    if (s != EMD_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return s != EMD_OK ? s : cuda_fail(e, "graph capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        g->exec = nullptr;
        cudaGetLastError();
        return cuda_fail(ei, "graph instantiate");
    }
    return EMD_OK;
}

emd_status alloc_batch_ws(emd_db* db, BatchWS& ws, int max_batch, int64_t cols, std::vector<void*>& allocs,
                          int64_t* bytes)
{
    auto dal = [&](auto** p, int64_t count) -> emd_status {
        using T = std::remove_reference_t<decltype(**p)>;
        const size_t nb = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(EMD_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s", nb, cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *bytes += (int64_t)nb;
        *p = static_cast<T*>(q);
        return EMD_OK;
    };
#define TRYW(x)                           \
    do {                                  \
        emd_status s_ = (x);              \
        if (s_ != EMD_OK) return s_;      \
    } while (0)
    const int64_t B = max_batch, vu = db->v_used, n = db->n;
    ws.max_batch = max_batch;
    ws.b_cols = std::max<int64_t>(round_up(cols, 32), round_up(db->opt.max_query_h, 32));
    ws.b_qrows = ws.b_cols + 32 * B;
    ws.b_prows = ws.b_cols + 96 * B;
    ws.b_tabcols = std::max<int64_t>(db->opt.max_table_k, 16 * round_up(B, kFwdGroup));  // whole interleaved groups
    TRYW(dal(&ws.bD, vu * ws.b_cols));
    if (!db->cost_mode) {
        TRYW(dal(&ws.bQ, ws.b_qrows * db->ldm));
        TRYW(dal(&ws.bqnorm, ws.b_qrows));
        if (db->tc) {
            TRYW(dal(&ws.bq_hi, ws.b_prows * db->kpad));
            if (db->tcfmt == TC_SPLIT) TRYW(dal(&ws.bq_lo, ws.b_prows * db->kpad));
            TRYW(dal(&ws.bq_scale, ws.b_prows));
        }
    }
    TRYW(dal(&ws.btab, vu * ws.b_tabcols));
    TRYW(dal(&ws.bt_fwd, B * n));
    TRYW(dal(&ws.bt_rev, B * n));
    TRYW(dal(&ws.bt_out, B * n));
    TRYW(dal(&ws.bsel_idx, B * kPruneMaxK));
    TRYW(dal(&ws.bsel_val, B * kPruneMaxK));
    TRYW(dal(&ws.bcand, B * kPruneCap));
    TRYW(dal(&ws.bcand_sym, B * 2 * kPruneCap));
    TRYW(dal(&ws.bcand_count, B));
    TRYW(dal(&ws.cand_ok, B));
    TRYW(dal(&ws.ict_over, B));
    TRYW(dal(&ws.topk_scratch, B * kTopkScratchRow));
    TRYW(dal(&ws.qd_dev, BatchWS::kDescRing * B));
    TRYW(dal(&ws.nq_dev, BatchWS::kDescRing));
    ws.fused = db->tc && !db->cost_mode && db->opt.fused_phase1 >= (db->approx ? 2 : 1) && db->as_hi != nullptr &&
               tc_table_fits(db->tcfmt, db->kpad) && tc_batch_stages(TC_SPLIT, db->kpad / 64) >= 2;
    if (ws.fused) {
        TRYW(dal(&ws.bqpos, B * vu));
        TRYW(dal(&ws.brmap, B * vu));
        TRYW(dal(&ws.bcrows, B * kCandRows));
        TRYW(dal(&ws.bncrows, B));
        TRYW(dal(&ws.bc_hi, B * kCandRows * db->kpad));
        TRYW(dal(&ws.bc_lo, B * kCandRows * db->kpad));
        TRYW(dal(&ws.bc_scale, B * kCandRows));
        TRYW(dal(&ws.bc_norm, B * kCandRows));
        TRYW(dal(&ws.bDc, (int64_t)kCandRows * ws.b_cols));
        if (db->approx) {
            TRYW(dal(&ws.bqs_hi, ws.b_prows * db->kpad));
            TRYW(dal(&ws.bqs_lo, ws.b_prows * db->kpad));
            TRYW(dal(&ws.bqs_scale, ws.b_prows));
            TRYW(dal(&ws.bcb, B * vu * kCandPerRow));
            TRYW(dal(&ws.bcmax, B * vu));
            TRYW(dal(&ws.brr, B * vu));
            TRYW(dal(&ws.brr_count, B));
        }
        // the row maps start (and every batch leaves them) at -1
        EMD_CUDA(cudaMemset(ws.bqpos, 0xff, sizeof(int32_t) * B * vu), "memset");
        EMD_CUDA(cudaMemset(ws.brmap, 0xff, sizeof(int32_t) * B * vu), "memset");
        EMD_CUDA(cudaDeviceSynchronize(), "synchronize");
    }
#undef TRYW
    EMD_CUDA(cudaHostAlloc((void**)&ws.qd_host, sizeof(QDesc) * BatchWS::kDescRing * B, cudaHostAllocDefault),
             "pinned descriptors");
    EMD_CUDA(cudaHostAlloc((void**)&ws.nq_host, sizeof(int) * BatchWS::kDescRing, cudaHostAllocDefault),
             "pinned descriptors");
    for (auto& e : ws.desc_ev) EMD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    EMD_CUDA(cudaStreamCreateWithFlags(&ws.cap_stream, cudaStreamNonBlocking), "stream");
    return EMD_OK;
}

void free_batch_ws(BatchWS& ws)
{
    for (auto& kv : ws.graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ws.graphs.clear();
    if (ws.cap_stream) cudaStreamDestroy(ws.cap_stream);
    for (auto& e : ws.desc_ev)
        if (e) cudaEventDestroy(e);
    if (ws.qd_host) cudaFreeHost(ws.qd_host);
    if (ws.nq_host) cudaFreeHost(ws.nq_host);
    ws = BatchWS();
}

// Fills ring slot `slot` with the descriptors of queries j0..j1-1 of the batch i0.. (the
// batch fits the batch workspace) and uploads them on st.  Outputs as run_batch.
emd_status fill_descriptors(BatchWS& ws, int slot, emd_db* db, const int64_t* rp, const int32_t* qidx, const float* qw, int64_t i0,
                        int64_t j0, int64_t j1, int meas, int k, int dir, int K, bool pruned, float* out_t,
                        int64_t* out_idx, float* out_dist, cudaStream_t st)
{
    const int nb = (int)(j1 - j0);
    const int tk_b = dir != EMD_DIR_REV ? table_width(db, meas, k, db->opt.max_query_h) : 0;
    const bool grouped = grouped_tables(ws, meas, tk_b);
    const int lw_b = grouped_width(db, meas, tk_b);
    QDesc* hd = ws.qd_host + (int64_t)slot * ws.max_batch;
    QDesc* dd = ws.qd_dev + (int64_t)slot * ws.max_batch;
    int* nqd = ws.nq_dev + slot;
    const int64_t n = db->n;
    int max_rows = 0, max_npad = 0, max_ldd = 0, max_tk = 0, max_kc = 0;
    int64_t c_D = 0, c_Q = 0, c_P = 0, c_T = 0;
    // Descriptor position p holds query order[p].  With grouped tables the forward sweep runs
    // a group of kFwdGroup consecutive positions in one warp, whose lanes step through the
    // longest transfer chain of the group (longer for larger h_q, whose capacities are
    // smaller), so the queries are placed by h_q, largest first: groups of alike lengths.
    // Every output is addressed per query (b = i - i0), so results do not depend on the order.
    std::vector<int64_t>& order = ws.order;
    order.resize((size_t)nb);
    for (int p = 0; p < nb; ++p) order[p] = j0 + p;
    if (grouped)
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t x, int64_t y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
    for (int p = 0; p < nb; ++p) {
        const int64_t i = order[p];
        QDesc& d = hd[p];
        memset(&d, 0, sizeof(d));
        const int64_t off = rp[i] - rp[i0];
        const int b = (int)(i - i0);
        d.h = (int)(rp[i + 1] - rp[i]);
        d.ldd = (int)round_up(d.h, 32);
        d.qrows = (int)round_up(d.ldd, kDistBN);
        d.npad = (int)round_up(d.h, 128);
        d.tk = dir != EMD_DIR_REV ? table_width(db, meas, k, d.h) : 0;
        d.kc = db->approx && d.tk > 0 ? rerank_width(db, d.tk, d.h) : d.tk;
        d.qidx = qidx + off;
        d.qw = qw + off;
        if (!db->cost_mode) {
            d.Q = ws.bQ + c_Q * db->ldm;
            d.qnorm = ws.bqnorm + c_Q;
            if (db->tc) {
                d.q_hi = ws.bq_hi + c_P * db->kpad;
                d.q_lo = db->tcfmt == TC_SPLIT ? ws.bq_lo + c_P * db->kpad : nullptr;
                d.q_scale = ws.bq_scale + c_P;
            }
        }
        d.D = ws.bD + c_D * db->v_used;
        if (grouped && lw_b > 0) {
            const int64_t bs = p;  // position in the sub-batch: group bs / kFwdGroup
            d.tab = ws.btab + (bs / kFwdGroup) * (db->v_used * lw_b * kFwdGroup) + (bs % kFwdGroup) * lw_b;
            d.tab_rs = lw_b * kFwdGroup;
            d.tab_es = 1;
        } else if (grouped) {
            const int64_t bs = p;
            d.tab = ws.btab + (bs / kFwdGroup) * (db->v_used * tk_b * kFwdGroup) + bs % kFwdGroup;
            d.tab_rs = tk_b * kFwdGroup;
            d.tab_es = kFwdGroup;
        } else {
            d.tab = ws.btab + c_T * db->v_used;
            d.tab_rs = d.tk;
            d.tab_es = 1;
        }
        d.t_fwd = ws.bt_fwd + (int64_t)b * n;
        d.t_rev = ws.bt_rev + (int64_t)b * n;
        d.t_out = (K > 0 ? ws.bt_out : out_t) + (int64_t)b * n;
        if (pruned) {
            d.sel_idx = ws.bsel_idx + (int64_t)b * K;
            d.sel_val = ws.bsel_val + (int64_t)b * K;
            d.cand = ws.bcand + (int64_t)b * kPruneCap;
            d.cand_sym = ws.bcand_sym + (int64_t)b * 2 * kPruneCap;
            d.cand_count = ws.bcand_count + p;  // position in the sub-batch: zeroed by its sequence
            d.ok = ws.cand_ok + b;
        }
        if (meas == M_ICT) d.over = ws.ict_over + b;
        if (ws.fused) {
            const int64_t bs = p;  // position in the sub-batch
            d.qpos = ws.bqpos + bs * db->v_used;
            d.rmap = ws.brmap + bs * db->v_used;
            d.crows = ws.bcrows + bs * kCandRows;
            d.ncrows = ws.bncrows + bs;  // zeroed by the sub-batch's sequence
            d.c_hi = ws.bc_hi + bs * kCandRows * db->kpad;
            d.c_lo = ws.bc_lo + bs * kCandRows * db->kpad;
            d.c_scale = ws.bc_scale + bs * kCandRows;
            d.c_norm = ws.bc_norm + bs * kCandRows;
            d.Dc = ws.bDc + c_D * kCandRows;
            if (db->approx) {
                d.qs_hi = ws.bqs_hi + c_P * db->kpad;
                d.qs_lo = ws.bqs_lo + c_P * db->kpad;
                d.qs_scale = ws.bqs_scale + c_P;
                d.cbin = ws.bcb + bs * db->v_used * kCandPerRow;
                d.camax = ws.bcmax + bs * db->v_used;
                d.rr = ws.brr + bs * db->v_used;
                d.rr_count = ws.brr_count + bs;
            } else {
                d.qs_hi = d.q_hi;
                d.qs_lo = d.q_lo;
                d.qs_scale = d.q_scale;
            }
        }
        d.sq = db->cost_mode ? 0 : 1;
        if (K > 0) {
            d.out_idx = out_idx + (int64_t)b * K;
            d.out_dist = out_dist + (int64_t)b * K;
        }
        c_D += d.ldd;
        c_Q += d.qrows;
        c_P += d.npad;
        c_T += d.tk;
        max_rows = std::max(max_rows, d.qrows);
        max_npad = std::max(max_npad, d.npad);
        max_ldd = std::max(max_ldd, d.ldd);
        max_tk = std::max(max_tk, d.tk);
        max_kc = std::max(max_kc, d.kc);
    }
    // the caller sizes sub-batches with batch_fits; never let one overrun the workspace
    const int64_t tab_used = grouped ? (int64_t)(nb + kFwdGroup - 1) / kFwdGroup * kFwdGroup * (lw_b ? lw_b : tk_b) : c_T;
    if (nb > ws.max_batch || c_D > ws.b_cols || c_Q > ws.b_qrows || c_P > ws.b_prows || tab_used > ws.b_tabcols)
        return fail(EMD_ERR_INVALID_ARG, "internal: sub-batch of %d queries exceeds the batch workspace", nb);
    ws.nq_host[slot] = nb;
    EMD_CUDA(cudaMemcpyAsync(dd, hd, sizeof(QDesc) * nb, cudaMemcpyHostToDevice, st), "descriptor upload");
    EMD_CUDA(cudaMemcpyAsync(nqd, ws.nq_host + slot, sizeof(int), cudaMemcpyHostToDevice, st), "descriptor upload");
    (void)max_rows; (void)max_npad; (void)max_ldd; (void)max_tk; (void)max_kc;
    return EMD_OK;
}

// Runs the sub-batch whose descriptors fill_descriptors put in `slot` (nb queries).
emd_status run_subbatch_launch(BatchWS& ws, int slot, emd_db* db, int nb, int meas, int k, int dir, int K, bool pruned,
                               cudaStream_t st, bool allow_fused)
{
    const QDesc* hd = ws.qd_host + (int64_t)slot * ws.max_batch;
    int qcap = 1;  // size class of the batch: the next power of two
    while (qcap < nb) qcap *= 2;
    qcap = std::min(qcap, ws.max_batch);
    if (db->tc && tc_batch_stages(db->tcfmt, db->kpad / 64) < 2) {
        // embeddings too wide for the batched panel: Phase 1 per query, the rest batched
        return launch_sequence(ws, db, slot, meas, k, K, dir, pruned, hd, nb, qcap, st);
    }
    if (!db->opt.graphs || db->profiling)
        return launch_sequence(ws, db, slot, meas, k, K, dir, pruned, nullptr, 0, qcap, st, allow_fused);
    const GraphKey key{meas, k, K, dir, pruned ? 1 : 0, slot, qcap, allow_fused ? 1 : 0};
    auto it = ws.graphs.find(key);
    if (it == ws.graphs.end()) {
        GraphEntry g;
        emd_status cs = capture_sequence(ws, db, slot, meas, k, K, dir, pruned, qcap, &g, allow_fused);
        if (cs != EMD_OK) {
            g_err.clear();
            g.exec = nullptr;  // capture refused: this key launches directly from now on
        }
        it = ws.graphs.emplace(key, g).first;
    }
    if (!it->second.exec) return launch_sequence(ws, db, slot, meas, k, K, dir, pruned, nullptr, 0, qcap, st, allow_fused);
    EMD_CUDA(cudaGraphLaunch(it->second.exec, st), "graph launch");
    for (int p = 0; p < EMD_N_PHASES; ++p) db->launches[p] += it->second.launches[p];
    db->total_launches += it->second.total;
    db->graph_launches += 1;
    return EMD_OK;
}

// Ring slots are reused only after the work that reads them (pinned host copy and device
// descriptors) has finished, whatever stream it ran on.
emd_status run_subbatch(emd_db* db, BatchWS& ws, const int64_t* rp, const int32_t* qidx, const float* qw, int64_t i0,
                        int64_t j0, int64_t j1, int meas, int k, int dir, int K, bool pruned, float* out_t,
                        int64_t* out_idx, float* out_dist, cudaStream_t st, bool allow_fused)
{
    const int slot = ws.desc_slot;
    ws.desc_slot = (slot + 1) % BatchWS::kDescRing;
    EMD_CUDA(cudaEventSynchronize(ws.desc_ev[slot]), "descriptor ring");
    if (meas == M_ICT)
        EMD_CUDA(cudaMemsetAsync(ws.ict_over + (j0 - i0), 0, (j1 - j0) * sizeof(int), st), "flag reset");
    emd_status s = fill_descriptors(ws, slot, db, rp, qidx, qw, i0, j0, j1, meas, k, dir, K, pruned, out_t, out_idx,
                                    out_dist, st);
    if (s == EMD_OK) s = run_subbatch_launch(ws, slot, db, (int)(j1 - j0), meas, k, dir, K, pruned, st, allow_fused);
    EMD_CUDA(cudaEventRecord(ws.desc_ev[slot], st), "descriptor ring");
    return s;
}

emd_status retry_materialized(emd_db* db, BatchWS& ws, const int64_t* rp, const int32_t* qidx, const float* qw,
                              int64_t i0, int64_t i, int meas, int k, int K, int64_t* out_idx, float* out_dist,
                              cudaStream_t st, int* ok)
{
    const int64_t off = rp[i] - rp[i0];
    // a sub-batch of its own: query i with offsets relative to itself, outputs at row i - i0
    const int64_t rp1[2] = {0, rp[i + 1] - rp[i]};
    emd_status s = run_subbatch(db, ws, rp1, qidx + off, qw + off, 0, 0, 1, meas, k, EMD_DIR_MAX, K, true, nullptr,
                                out_idx + (i - i0) * K, out_dist + (i - i0) * K, st, false);
    if (s != EMD_OK) return s;
    EMD_CUDA(cudaMemcpyAsync(ok, ws.cand_ok, sizeof(int), cudaMemcpyDeviceToHost, st), "flag read");
    EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
    return EMD_OK;
}

bool batch_fits(const emd_db* db, const BatchWS& ws, const int64_t* rp, int64_t i0, int64_t i1, int meas, int k,
                int dir)
{
    int64_t cD = 0, cQ = 0, cP = 0, cT = 0;
    if (i1 - i0 > ws.max_batch) return false;
    const int tk_b = dir != EMD_DIR_REV ? table_width(db, meas, k, db->opt.max_query_h) : 0;
    const bool grouped = grouped_tables(ws, meas, tk_b);
    for (int64_t i = i0; i < i1; ++i) {
        const int h = (int)(rp[i + 1] - rp[i]);
        const int64_t ldd = round_up(h, 32);
        cD += ldd;
        cQ += round_up(ldd, kDistBN);
        cP += round_up(h, 128);
        cT += dir != EMD_DIR_REV ? table_width(db, meas, k, h) : 0;
    }
    if (grouped) {  // whole groups of kFwdGroup tables
        const int lw = grouped_width(db, meas, tk_b);
        cT = (i1 - i0 + kFwdGroup - 1) / kFwdGroup * kFwdGroup * (lw ? lw : tk_b);
    }
    return cD <= ws.b_cols && cQ <= ws.b_qrows && cP <= ws.b_prows && cT <= ws.b_tabcols;
}

emd_status run_batch(emd_db* db, const int64_t* rp, const int32_t* qidx, const float* qw, int64_t i0,
                     int64_t i1, int meas, int k, int dir, int K, float* out_t, int64_t* out_idx,
                     float* out_dist, cudaStream_t st)
{
    const bool pruned = K > 0 && prunable(db, meas, k, dir, K);
    const bool ict = meas == M_ICT && dir != EMD_DIR_REV && !db->approx;
    if (db->opt.batched) {
        // split into sub-batches that fit the batch workspace
        BatchWS& ws = db->bw;
        int64_t j0 = i0;
        while (j0 < i1) {
            int64_t j1 = j0 + 1;
            while (j1 < i1 && batch_fits(db, ws, rp, j0, j1 + 1, meas, k, dir)) ++j1;
            emd_status s = run_subbatch(db, ws, rp, qidx, qw, i0, j0, j1, meas, k, dir, K, pruned, out_t, out_idx,
                                        out_dist, st);
            if (s != EMD_OK) return s;
            j0 = j1;
        }
    } else {
        if (ict) EMD_CUDA(cudaMemsetAsync(db->ict_over, 0, (i1 - i0) * sizeof(int), st), "flag reset");
        emd_status s = run_lanes(db, rp, qidx, qw, i0, i1, meas, k, dir, K, pruned, out_t, out_idx, out_dist, st);
        if (s != EMD_OK) return s;
        if (K > 0 && !pruned) {
            s = select_topk(db, db->stage_out, i1 - i0, K, out_idx, out_dist, st);
            if (s != EMD_OK) return s;
        }
    }
    if (!pruned && !ict) return EMD_OK;
    // uncertified pruned queries and ICT queries whose table overflowed: recomputed alone
    // over all documents (ICT with tables of full width)
    std::vector<int> ok((size_t)(i1 - i0), 1), over((size_t)(i1 - i0), 0);
    if (pruned)
        EMD_CUDA(cudaMemcpyAsync(ok.data(), db->opt.batched ? db->bw.cand_ok : db->cand_ok, (i1 - i0) * sizeof(int),
                                 cudaMemcpyDeviceToHost, st),
                 "flag read");
    if (ict)
        EMD_CUDA(cudaMemcpyAsync(over.data(), db->opt.batched ? db->bw.ict_over : db->ict_over,
                                 (i1 - i0) * sizeof(int), cudaMemcpyDeviceToHost, st),
                 "flag read");
    EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
    if (pruned) db->pruned_queries += i1 - i0;
    for (int64_t i = i0; i < i1; ++i) {
        if (db->opt.batched && pruned && ok[i - i0] == 2) {  // the fused candidate block overflowed
            ++db->fused_retries;
            emd_status s = retry_materialized(db, db->bw, rp, qidx, qw, i0, i, meas, k, K, out_idx, out_dist, st,
                                              &ok[i - i0]);
            if (s != EMD_OK) return s;
        }
        if (ok[i - i0] == 1 && !over[i - i0]) continue;
        if (over[i - i0]) ++db->ict_wide; else ++db->prune_fallbacks;
        const int64_t off = rp[i] - rp[i0];
        const int h = (int)(rp[i + 1] - rp[i]);
        float* dst = K > 0 ? db->stage_out : out_t + (i - i0) * db->n;
        emd_status s = run_query(db, db->lanes[0], qidx + off, qw + off, h, meas, k, dir, dst, nullptr, st);
        if (s != EMD_OK) return s;
        if (K > 0) s = select_topk(db, db->stage_out, 1, K, out_idx + (i - i0) * K, out_dist + (i - i0) * K, st);
        if (s != EMD_OK) return s;
    }
    return EMD_OK;
}

// Queries i0..i1-1 one after another on the lanes (opt.batched = 0).
emd_status run_lanes(emd_db* db, const int64_t* rp, const int32_t* qidx, const float* qw, int64_t i0,
                     int64_t i1, int meas, int k, int dir, int K, bool pruned, float* out_t, int64_t* out_idx,
                     float* out_dist, cudaStream_t st)
{
    const int nl = (int)std::min<int64_t>((int64_t)db->lanes.size(), i1 - i0);
    EMD_CUDA(cudaEventRecord(db->fork, st), "fork");
    for (int l = 0; l < nl; ++l) EMD_CUDA(cudaStreamWaitEvent(db->lanes[l].st, db->fork, 0), "fork");
    for (int64_t i = i0; i < i1; ++i) {
        Lane& L = db->lanes[(i - i0) % nl];
        const int64_t off = rp[i] - rp[i0];
        const int h = (int)(rp[i + 1] - rp[i]);
        emd_status s;
        if (pruned)
            s = run_topk_pruned(db, L, qidx + off, qw + off, h, meas, k, K, db->cand_ok + (i - i0), db->ict_over + (i - i0),
                                out_idx + (i - i0) * K, out_dist + (i - i0) * K, L.st);
        else
            s = run_query(db, L, qidx + off, qw + off, h, meas, k, dir,
                          (K > 0 ? db->stage_out : out_t) + (i - i0) * db->n, db->ict_over + (i - i0), L.st);
        if (s != EMD_OK) return s;
    }
    for (int l = 0; l < nl; ++l) {
        EMD_CUDA(cudaEventRecord(db->lanes[l].done, db->lanes[l].st), "join");
        EMD_CUDA(cudaStreamWaitEvent(st, db->lanes[l].done, 0), "join");
    }
    return EMD_OK;
}

emd_status read_device_errors(emd_db* db)
{
    int h_err = 0;
    EMD_CUDA(cudaMemcpyAsync(&h_err, db->err, sizeof(int), cudaMemcpyDeviceToHost, db->stream), "error read");
    EMD_CUDA(cudaStreamSynchronize(db->stream), "synchronize");
    if (h_err) {
        int zero = 0;
        cudaMemcpy(db->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (h_err & ERR_TIMEOUT)
            return fail(EMD_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its time limit");
        if (h_err & ERR_PAIR_TMEM)
            return fail(EMD_ERR_CUDA, "the SM-pair Phase-1 kernel found different TMEM addresses in a pair");
        return fail(EMD_ERR_INVALID_ARG, "a kernel met a vocabulary id outside 0..%lld", (long long)db->v - 1);
    }
    return EMD_OK;
}

// Folds the finished profiling event pairs into the per-phase sums.
emd_status collect_profile(emd_db* db)
{
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    for (auto& r : db->recs) {
        EMD_CUDA(cudaEventSynchronize(r.b), "event synchronize");
        float ms = 0.f;
        EMD_CUDA(cudaEventElapsedTime(&ms, r.a, r.b), "event time");
        db->ms[r.phase] += ms;
        db->pool.push_back(r.a);
        db->pool.push_back(r.b);
    }
    db->recs.clear();
    return EMD_OK;
}

// Host-buffer driver shared by emd_query_batch and emd_topk.
emd_status host_batches(emd_db* db, const emd_queries* q, int meas, int k, int dir, int K,
                        float* out_dist_all, int64_t* out_idx, float* out_dist)
{
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    cudaStream_t st = db->stream;
    int64_t i0 = 0;
    while (i0 < q->n_queries) {
        int64_t i1 = i0;
        while (i1 < q->n_queries && i1 - i0 < db->opt.max_batch &&
               q->row_ptr[i1 + 1] - q->row_ptr[i0] <= db->stage_bins)
            ++i1;
        const int64_t base = q->row_ptr[i0];
        const int64_t bins = q->row_ptr[i1] - base;
        EMD_CUDA(cudaMemcpyAsync(db->stage_idx, q->idx + base, bins * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st), "query copy");
        EMD_CUDA(cudaMemcpyAsync(db->stage_w, q->w + base, bins * sizeof(float),
                                 cudaMemcpyHostToDevice, st), "query copy");
        emd_status s = run_batch(db, q->row_ptr, db->stage_idx, db->stage_w, i0, i1, meas, k, dir, K,
                                 db->stage_out, db->stage_oidx, db->stage_odist, st);
        if (s != EMD_OK) return s;
        if (K > 0) {
            EMD_CUDA(cudaMemcpyAsync(out_idx + i0 * K, db->stage_oidx, (i1 - i0) * K * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st), "result copy");
            EMD_CUDA(cudaMemcpyAsync(out_dist + i0 * K, db->stage_odist, (i1 - i0) * K * sizeof(float),
                                     cudaMemcpyDeviceToHost, st), "result copy");
        } else {
            EMD_CUDA(cudaMemcpyAsync(out_dist_all + i0 * db->n, db->stage_out,
                                     (i1 - i0) * db->n * sizeof(float), cudaMemcpyDeviceToHost, st),
                     "result copy");
        }
        EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
        i0 = i1;
    }
    return read_device_errors(db);
}

// Picks the batched kernels' free parameters (query groups per vocabulary tile and B
// stages of the tensor-core Phase 1, warps per candidate in the pruned reverse pass) by
// timing them on a synthetic batch of max_batch queries of up to 128 consecutive used
// vocabulary rows, uniform weights.  Every choice gives bit-identical results; only the time differs.
emd_status autotune(emd_db* db, const std::vector<int32_t>& used_host)
{
    const int h = (int)std::min<int64_t>(std::min<int64_t>(128, db->opt.max_query_h), db->v_used);
    const int k = std::min(4, db->opt.max_table_k);
    const int K = (int)std::min<int64_t>(16, db->n);
    // as many queries as one sub-batch of the workspace holds, at most max_batch
    std::vector<int64_t> rp((size_t)db->opt.max_batch + 1);
    for (size_t i = 0; i < rp.size(); ++i) rp[i] = (int64_t)i * h;
    int nb = 1;
    while (nb < db->opt.max_batch && batch_fits(db, db->bw, rp.data(), 0, nb + 1, EMD_ACT, k, EMD_DIR_MAX)) ++nb;
    std::vector<int32_t> idx((size_t)nb * h);
    std::vector<float> w((size_t)nb * h, 1.0f / (float)h);
    for (int i = 0; i < nb; ++i) {
        const int64_t start = (int64_t)i * (db->v_used / nb);
        for (int j = 0; j < h; ++j) idx[(size_t)i * h + j] = used_host[(size_t)((start + j) % db->v_used)];
    }
    cudaStream_t st = db->stream;
    BatchWS& ws = db->bw;
    EMD_CUDA(cudaMemcpyAsync(db->stage_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, st), "tune copy");
    EMD_CUDA(cudaMemcpyAsync(db->stage_w, w.data(), w.size() * 4, cudaMemcpyHostToDevice, st), "tune copy");
    const bool pruned = prunable(db, EMD_ACT, k, EMD_DIR_MAX, K);
    emd_status s = fill_descriptors(ws, 0, db, rp.data(), db->stage_idx, db->stage_w, 0, 0, nb, EMD_ACT, k, EMD_DIR_MAX, K,
                                    pruned, nullptr, db->stage_oidx, db->stage_odist, st);
    if (s != EMD_OK) return s;
    const bool per_query_tc = db->tc && tc_batch_stages(db->tcfmt, db->kpad / 64) < 2;
    s = launch_sequence(ws, db, 0, EMD_ACT, k, K, EMD_DIR_MAX, pruned, per_query_tc ? ws.qd_host : nullptr, nb,
                        ws.max_batch, st);
    if (s != EMD_OK) return s;
    EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
    cudaEvent_t a = nullptr, b = nullptr;
    EMD_CUDA(cudaEventCreate(&a), "event");
    EMD_CUDA(cudaEventCreate(&b), "event");
    auto timed = [&](auto&& launch) -> float {
        float best = 1e30f;
        for (int r = 0; r < 8; ++r) {
            cudaEventRecord(a, st);
            launch();
            cudaEventRecord(b, st);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (r > 0) best = std::min(best, ms);
        }
        return best;
    };
    const QDesc* D_ = ws.qd_dev;
    const int* nqd = ws.nq_dev;
    if (db->tc && tc_batch_stages(db->tcfmt, db->kpad / 64) >= 2) {
        // a candidate replaces the current choice only when at least 5% faster (timing noise
        // on short launches would otherwise pick at random)
        const int fit = tc_batch_stages(db->tcfmt, db->kpad / 64);
        float best = 1e30f;
        std::vector<int> stage_set;
        for (int sg : {fit, (fit + 2) / 2, 2})
            if (sg >= 2 && sg <= fit && std::find(stage_set.begin(), stage_set.end(), sg) == stage_set.end())
                stage_set.push_back(sg);
        for (int gm : {1, 2, 4})
            for (int sg : stage_set) {
                const float ms = timed([&] {
                    launch_tc_dist_batch(db->tcfmt, db->a_hi, db->a_lo, db->mpad, db->a_scale, db->norm_used,
                                         db->v_used, D_, nqd, db->opt.max_batch, db->kpad, db->m, gm, sg, db->err,
                                         st);
                });
                if (ms < 0.95f * best) {
                    best = ms;
                    db->tune_group_mult = gm;
                    db->tune_stages = sg;
                }
            }
    }
    if (pruned) {
        // Warps per candidate document: 4 unless 8 is clearly faster.  Two warps are not tried:
        // on the synthetic batch (consecutive frequent ids) they could time well while on the
        // serving database's own queries they took 1.7x as long (2.9 against 1.7 ms per batch).
        float best = 1e30f;
        for (int wp : {4, 8}) {  // the default first
            const float ms = timed([&] {
                cudaMemsetAsync(ws.bcand_count, 0, sizeof(int) * db->opt.max_batch, st);
                launch_prune_b(EMD_ACT, k, D_, nqd, db->opt.max_batch, db->row_ptr, db->col, db->val, db->n, K, wp,
                               st);
            });
            if (ms < 0.90f * best) {
                best = ms;
                db->tune_rev_warps = wp;
            }
        }
    }
    if (db->opt.fwd_kernel == 0) {
        // the grouped forward sweep: each variant with its own table layout (descriptors and
        // tables rebuilt), timed on the same batch
        float best = 1e30f;
        int choice = kFwdChain;
        for (int v : {kFwdChain, kFwdPrefetch, kFwdCoalesced, kFwdRowMajor}) {
            db->tune_fwd = v;
            s = fill_descriptors(ws, 0, db, rp.data(), db->stage_idx, db->stage_w, 0, 0, nb, EMD_ACT, k, EMD_DIR_MAX,
                                 K, pruned, nullptr, db->stage_oidx, db->stage_odist, st);
            if (s == EMD_OK)
                s = launch_sequence(ws, db, 0, EMD_ACT, k, K, EMD_DIR_MAX, pruned, per_query_tc ? ws.qd_host : nullptr,
                                    nb, ws.max_batch, st);
            if (s != EMD_OK) return s;
            const int tk = table_width(db, EMD_ACT, k, db->opt.max_query_h);
            const float ms = timed([&] {
                launch_fwd_b(EMD_ACT, D_, nqd, db->opt.max_batch, db->row_ptr, db->col, db->val, db->n, false,
                             grouped_tables(ws, EMD_ACT, tk), tk, st, v);
            });
            if (ms < 0.95f * best) {
                best = ms;
                choice = v;
            }
        }
        db->tune_fwd = choice;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
    EMD_CUDA(cudaGetLastError(), "autotune");
    db->autotuned = true;
    for (int p = 0; p < EMD_N_PHASES; ++p) db->launches[p] = 0;
    db->total_launches = 0;
    return EMD_OK;
}

}  // namespace emd

extern "C" {

void emd_db_options_default(emd_db_options* opt)
{
    if (!opt) return;
    opt->device = 0;
    opt->precision = EMD_PREC_FP32;
    opt->rerank_margin = 8;
    opt->max_query_h = 2048;
    opt->max_table_k = 64;
    opt->max_batch = 64;
    opt->prune_topk = 1;
    opt->lanes = 1;
    opt->batched = 1;
    opt->batch_columns = 16384;
    opt->graphs = 1;
    opt->autotune = 1;
    opt->fused_phase1 = 1;
    opt->fwd_kernel = 0;
    opt->tc_pair = 0;
}

emd_status emd_db_create(const float* emb, int64_t v, int32_t m, const float* cost_matrix,
                         const int64_t* row_ptr, const int32_t* col, const float* val,
                         int64_t n_docs, const emd_db_options* opt_in, emd_db** out)
{
    g_err.clear();
    if (!out) return fail(EMD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    emd_db_options opt;
    emd_db_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if ((emb == nullptr) == (cost_matrix == nullptr))
        return fail(EMD_ERR_INVALID_ARG, "exactly one of emb and cost_matrix must be given");
    if (v < 1 || v >= (1ll << 31)) return fail(EMD_ERR_INVALID_ARG, "v out of range");
    if (emb && (m < 1 || m > 4096)) return fail(EMD_ERR_INVALID_ARG, "m out of range (1..4096)");
    if (n_docs < 1) return fail(EMD_ERR_INVALID_ARG, "n_docs must be >= 1");
    if (!row_ptr || !col || !val) return fail(EMD_ERR_INVALID_ARG, "CSR arrays must be non-NULL");
    if (opt.precision < EMD_PREC_FP32 || opt.precision > EMD_PREC_FP32_TC)
        return fail(EMD_ERR_INVALID_ARG, "unknown precision %d", (int)opt.precision);
    if (opt.rerank_margin < 0 || opt.rerank_margin > kRerankMax)
        return fail(EMD_ERR_INVALID_ARG, "rerank_margin must be 0..%d", kRerankMax);
    if (opt.max_query_h < 1 || opt.max_query_h > (1 << 16) || opt.max_table_k < 1 ||
        opt.max_table_k > (1 << 16) || opt.max_batch < 1 || opt.max_batch > 4096 || opt.lanes < 1 ||
        opt.lanes > 16 || opt.batch_columns < 1)
        return fail(EMD_ERR_INVALID_ARG, "option out of range");
    if (opt.fused_phase1 < 0 || opt.fused_phase1 > 2) return fail(EMD_ERR_INVALID_ARG, "fused_phase1 must be 0..2");
    if (opt.fwd_kernel < 0 || opt.fwd_kernel > kFwdVariants)
        return fail(EMD_ERR_INVALID_ARG, "fwd_kernel must be 0..%d", kFwdVariants);
    if (opt.tc_pair < 0 || opt.tc_pair > 2) return fail(EMD_ERR_INVALID_ARG, "tc_pair must be 0..2");
    if ((opt.precision == EMD_PREC_BF16 || opt.precision == EMD_PREC_FP8_E4M3) && opt.max_query_h > 6400)
        return fail(EMD_ERR_INVALID_ARG, "max_query_h above 6400 with an approximate precision (the re-rank "
                                         "stages 32 bytes per query bin in shared memory)");
    if (row_ptr[0] != 0) return fail(EMD_ERR_INVALID_ARG, "row_ptr[0] != 0");
    const int64_t nnz = row_ptr[n_docs];
    if (nnz >= (1ll << 31)) return fail(EMD_ERR_UNSUPPORTED, "nnz must be < 2^31");
    std::vector<int64_t> stamp((size_t)v, -1);
    std::vector<char> used((size_t)v, 0);
    for (int64_t d = 0; d < n_docs; ++d) {
        if (row_ptr[d + 1] <= row_ptr[d])
            return fail(EMD_ERR_INVALID_ARG, "document %lld is empty or row_ptr decreases", (long long)d);
        double s = 0.0;
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
            int32_t c = col[e];
            if (c < 0 || c >= v) return fail(EMD_ERR_INVALID_ARG, "document %lld: id %d out of range", (long long)d, c);
            if (stamp[c] == d) return fail(EMD_ERR_INVALID_ARG, "document %lld: id %d repeated", (long long)d, c);
            stamp[c] = d;
            if (!(val[e] > 0.f) || !isfinite(val[e]))
                return fail(EMD_ERR_INVALID_ARG, "document %lld: weight %g invalid", (long long)d, (double)val[e]);
            s += val[e];
            used[c] = 1;
        }
        if (fabs(s - 1.0) > 1e-5)
            return fail(EMD_ERR_INVALID_ARG, "document %lld: weights sum to %.9g, not 1", (long long)d, s);
    }
    if (cost_matrix) {
        for (int64_t a = 0; a < v; ++a)
            for (int64_t b = 0; b < v; ++b) {
                float c = cost_matrix[a * v + b];
                if (!(c >= 0.f) || !isfinite(c) || (a == b && c != 0.f))
                    return fail(EMD_ERR_INVALID_ARG, "cost matrix entry (%lld,%lld) invalid", (long long)a, (long long)b);
            }
    }

    // used vocabulary (Section 2.2) and renumbered columns
    std::vector<int32_t> slot((size_t)v, -1), used_ids;
    for (int64_t u = 0; u < v; ++u)
        if (used[u]) { slot[u] = (int32_t)used_ids.size(); used_ids.push_back((int32_t)u); }
    std::vector<int32_t> col_used((size_t)nnz), rp32((size_t)n_docs + 1);
    for (int64_t e = 0; e < nnz; ++e) col_used[e] = slot[col[e]];
    for (int64_t d = 0; d <= n_docs; ++d) rp32[d] = (int32_t)row_ptr[d];

    emd_db* db = new emd_db();
    db->row_ptr_host.assign(row_ptr, row_ptr + n_docs + 1);
    db->opt = opt;
    db->dev = opt.device;
    db->tune_fwd = opt.fwd_kernel > 0 ? opt.fwd_kernel - 1 : kFwdChain;
    db->margin = opt.rerank_margin;
    db->v = v;
    db->v_used = (int64_t)used_ids.size();
    db->n = n_docs;
    db->nnz = nnz;
    db->cost_mode = cost_matrix != nullptr;
    db->m = db->cost_mode ? 0 : m;
    db->ldm = db->cost_mode ? 0 : (int)round_up(m, 4);

    emd_status s = EMD_OK;
#define TRY(x)                          \
    do {                                \
        s = (x);                        \
        if (s != EMD_OK) { release(db); return s; } \
    } while (0)
#define TRYC(x, what)                                        \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) { release(db); return cuda_fail(e_, what); } \
    } while (0)

    TRYC(cudaSetDevice(db->dev), "cudaSetDevice");
    TRYC(cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking), "stream");
    TRYC(cudaEventCreateWithFlags(&db->fork, cudaEventDisableTiming), "event");
    db->lanes.resize((size_t)opt.lanes);
    for (auto& L : db->lanes) {
        TRYC(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking), "stream");
        TRYC(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming), "event");
    }
    cudaStream_t st = db->stream;

    const int64_t vu = db->v_used;
    TRY(dalloc(db, &db->used_ids, vu));
    TRY(dalloc(db, &db->row_ptr, n_docs + 1));
    TRY(dalloc(db, &db->col, nnz));
    TRY(dalloc(db, &db->val, nnz));
    TRY(dalloc(db, &db->err, 1));
    TRYC(cudaMemsetAsync(db->err, 0, sizeof(int), st), "memset");
    TRYC(cudaMemcpyAsync(db->used_ids, used_ids.data(), vu * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
    TRY(dalloc(db, &db->vslot, v));
    TRYC(launch_vslot(db->used_ids, vu, v, db->vslot, st), "vocabulary slots");
    db->total_launches += 1;
    db->launches[6] += 1;
    TRYC(cudaMemcpyAsync(db->row_ptr, rp32.data(), (n_docs + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
    TRYC(cudaMemcpyAsync(db->col, col_used.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
    TRYC(cudaMemcpyAsync(db->val, val, nnz * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    {
        // the largest weight any document puts on each used row: how far an ICT table row
        // must reach (Algorithm 2 moves at most that much mass out of a bin of the row)
        std::vector<float> xmax((size_t)vu, 0.f);
        for (int64_t e = 0; e < nnz; ++e) xmax[col_used[e]] = std::max(xmax[col_used[e]], val[e]);
        TRY(dalloc(db, &db->xmax, vu));
        TRYC(cudaMemcpy(db->xmax, xmax.data(), vu * sizeof(float), cudaMemcpyHostToDevice), "copy");
    }

    if (db->cost_mode) {
        TRY(dalloc(db, &db->cost, v * v));
        TRYC(cudaMemcpyAsync(db->cost, cost_matrix, v * v * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    } else {
        const int ldm = db->ldm;
        TRY(dalloc(db, &db->emb, v * ldm));
        TRY(dalloc(db, &db->emb_used, vu * ldm));
        TRY(dalloc(db, &db->norm_used, vu));
        TRYC(cudaMemcpy2DAsync(db->emb, ldm * sizeof(float), emb, m * sizeof(float), m * sizeof(float), v,
                               cudaMemcpyHostToDevice, st), "copy");
        if (ldm > m)
            TRYC(cudaMemset2DAsync(db->emb + m, ldm * sizeof(float), 0, (ldm - m) * sizeof(float), v, st), "memset");
        TRYC(launch_gather_rows(db->emb, v, ldm, ldm, db->used_ids, vu, vu, db->emb_used, db->norm_used,
                                db->err, st), "embedding gather");
        db->total_launches += 1;
        db->launches[6] += 1;
        db->qrows_max = (int)round_up(round_up(opt.max_query_h, 32), kDistBN);
        if (opt.precision != EMD_PREC_FP32) {
            db->tc = true;
            db->tcfmt = opt.precision == EMD_PREC_FP32_TC ? TC_SPLIT
                        : opt.precision == EMD_PREC_BF16  ? TC_BF16
                                                          : TC_E4M3;
            db->approx = db->tcfmt != TC_SPLIT;
            db->kpad = (int)round_up(m, 64);
            db->mpad = round_up(vu, 256);  // whole row tiles of 128, and of 256 for the SM-pair form
            TRY(dalloc(db, &db->a_hi, db->mpad * db->kpad));
            if (db->tcfmt == TC_SPLIT) TRY(dalloc(db, &db->a_lo, db->mpad * db->kpad));
            TRY(dalloc(db, &db->a_scale, db->mpad));
            TRYC(launch_pack(db->tcfmt, db->emb_used, ldm, m, vu, db->mpad, db->kpad, db->a_hi, db->a_lo,
                             db->a_scale, st),
                 "embedding pack");
            db->total_launches += 1;
            db->launches[6] += 1;
            if (db->approx && opt.batched && opt.fused_phase1 >= 2) {
                TRY(dalloc(db, &db->as_hi, db->mpad * db->kpad));
                TRY(dalloc(db, &db->as_lo, db->mpad * db->kpad));
                TRY(dalloc(db, &db->as_scale, db->mpad));
                TRYC(launch_pack(TC_SPLIT, db->emb_used, ldm, m, vu, db->mpad, db->kpad, db->as_hi, db->as_lo,
                                 db->as_scale, st),
                     "embedding pack (split)");
                db->total_launches += 1;
                db->launches[6] += 1;
            } else if (!db->approx) {
                db->as_hi = db->a_hi;
                db->as_lo = db->a_lo;
                db->as_scale = db->a_scale;
            }
        }
    }

    db->ldd_max = (int)round_up(opt.max_query_h, 32);
    const int64_t npad = round_up(opt.max_query_h, 128);
    for (auto& L : db->lanes) {
        if (!db->cost_mode) {
            TRY(dalloc(db, &L.Q, (int64_t)db->qrows_max * db->ldm));
            TRY(dalloc(db, &L.qnorm, db->qrows_max));
            if (db->tc) {
                TRY(dalloc(db, &L.q_hi, npad * db->kpad));
                if (db->tcfmt == TC_SPLIT) TRY(dalloc(db, &L.q_lo, npad * db->kpad));
                TRY(dalloc(db, &L.q_scale, npad));
            }
        }
        TRY(dalloc(db, &L.D, vu * db->ldd_max));
        TRY(dalloc(db, &L.tab, vu * opt.max_table_k));
        TRY(dalloc(db, &L.t_fwd, n_docs));
        TRY(dalloc(db, &L.t_rev, n_docs));
        TRY(dalloc(db, &L.sel_idx, kPruneMaxK));
        TRY(dalloc(db, &L.sel_val, kPruneMaxK));
        TRY(dalloc(db, &L.cand_idx, kPruneCap));
        TRY(dalloc(db, &L.cand_sym, 2 * kPruneCap));
        TRY(dalloc(db, &L.cand_count, 1));
        TRY(dalloc(db, &L.scratch, kTopkScratchRow));
    }
    TRY(dalloc(db, &db->tab_s, vu * opt.max_table_k));
    TRY(dalloc(db, &db->topk_scratch, (int64_t)opt.max_batch * kTopkScratchRow));
    TRY(dalloc(db, &db->cand_ok, opt.max_batch));
    TRY(dalloc(db, &db->ict_over, opt.max_batch));
    if (opt.batched) TRY(alloc_batch_ws(db, db->bw, opt.max_batch, opt.batch_columns, db->allocs, &db->bytes));
    db->stage_bins = (int64_t)opt.max_batch * opt.max_query_h;
    TRY(dalloc(db, &db->stage_idx, db->stage_bins));
    TRY(dalloc(db, &db->stage_w, db->stage_bins));
    TRY(dalloc(db, &db->stage_out, (int64_t)opt.max_batch * n_docs));
    TRY(dalloc(db, &db->stage_oidx, (int64_t)opt.max_batch * kMaxTopK));
    TRY(dalloc(db, &db->stage_odist, (int64_t)opt.max_batch * kMaxTopK));
    TRYC(cudaStreamSynchronize(st), "synchronize");
    if (opt.batched && opt.autotune) TRY(autotune(db, used_ids));
#undef TRY
#undef TRYC
    *out = db;
    return EMD_OK;
}

emd_status emd_db_destroy(emd_db* db)
{
    g_err.clear();
    if (db && db->servers.load() > 0) return fail(EMD_ERR_BUSY, "a server is attached to the database");
    release(db);
    return EMD_OK;
}

emd_status emd_db_info_get(const emd_db* db, emd_db_info* out)
{
    if (!db || !out) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    out->v = db->v;
    out->v_used = db->v_used;
    out->n_docs = db->n;
    out->nnz = db->nnz;
    out->m = db->m;
    out->cost_matrix_mode = db->cost_mode ? 1 : 0;
    out->device_bytes = db->bytes;
    out->autotuned = db->autotuned ? 1 : 0;
    out->tc_group_mult = db->tune_group_mult;
    out->tc_stages = db->tune_stages;
    out->rev_warps = db->tune_rev_warps;
    out->fwd_kernel = db->tune_fwd + 1;
    out->tc_pair = use_tc_pair(db) ? db->opt.tc_pair : 0;
    return EMD_OK;
}

emd_status emd_query_batch(emd_db* db, const emd_queries* q, emd_measure meas, int32_t k,
                           emd_direction dir, float* out_dist)
{
    g_err.clear();
    if (!db || !q) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(db->mu);
    emd_status s = check_request(db, meas, k, dir);
    if (s != EMD_OK) return s;
    if ((s = check_sizes(db, q->n_queries, q->row_ptr, meas, k, dir)) != EMD_OK) return s;
    if ((s = check_query_values(db, q)) != EMD_OK) return s;
    if (q->n_queries == 0) return EMD_OK;
    if (!out_dist) return fail(EMD_ERR_INVALID_ARG, "out_dist is NULL");
    return host_batches(db, q, meas, k, dir, 0, out_dist, nullptr, nullptr);
}

emd_status emd_topk(emd_db* db, const emd_queries* q, emd_measure meas, int32_t k,
                    emd_direction dir, int32_t K, int64_t* out_idx, float* out_dist)
{
    g_err.clear();
    if (!db || !q) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(db->mu);
    emd_status s = check_request(db, meas, k, dir);
    if (s != EMD_OK) return s;
    if (K < 1 || K > kMaxTopK || K > db->n)
        return fail(EMD_ERR_INVALID_ARG, "K must be in 1..min(n_docs, %d)", kMaxTopK);
    if ((s = check_sizes(db, q->n_queries, q->row_ptr, meas, k, dir)) != EMD_OK) return s;
    if ((s = check_query_values(db, q)) != EMD_OK) return s;
    if (q->n_queries == 0) return EMD_OK;
    if (!out_idx || !out_dist) return fail(EMD_ERR_INVALID_ARG, "output is NULL");
    return host_batches(db, q, meas, k, dir, K, nullptr, out_idx, out_dist);
}

emd_status emd_query_batch_device(emd_db* db, int64_t n_queries, const int64_t* q_row_ptr_host,
                                  const int32_t* q_idx_dev, const float* q_w_dev,
                                  emd_measure meas, int32_t k, emd_direction dir,
                                  float* out_dist_dev, void* stream)
{
    g_err.clear();
    if (!db) return fail(EMD_ERR_INVALID_ARG, "NULL handle");
    emd_status s = check_request(db, meas, k, dir);
    std::lock_guard<std::mutex> lock(db->mu);
    if (s != EMD_OK) return s;
    if ((s = check_sizes(db, n_queries, q_row_ptr_host, meas, k, dir)) != EMD_OK) return s;
    if (n_queries == 0) return EMD_OK;
    if (!q_idx_dev || !q_w_dev || !out_dist_dev) return fail(EMD_ERR_INVALID_ARG, "NULL device pointer");
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);  // NULL: the default stream
    for (int64_t i0 = 0; i0 < n_queries; i0 += db->opt.max_batch) {
        const int64_t i1 = std::min<int64_t>(n_queries, i0 + db->opt.max_batch);
        s = run_batch(db, q_row_ptr_host, q_idx_dev + q_row_ptr_host[i0], q_w_dev + q_row_ptr_host[i0], i0, i1,
                      meas, k, dir, 0, out_dist_dev + i0 * db->n, nullptr, nullptr, st);
        if (s != EMD_OK) return s;
    }
    return EMD_OK;
}

emd_status emd_topk_device(emd_db* db, int64_t n_queries, const int64_t* q_row_ptr_host,
                           const int32_t* q_idx_dev, const float* q_w_dev, emd_measure meas,
                           int32_t k, emd_direction dir, int32_t K, int64_t* out_idx_dev,
                           float* out_dist_dev, void* stream)
{
    g_err.clear();
    if (!db) return fail(EMD_ERR_INVALID_ARG, "NULL handle");
    emd_status s = check_request(db, meas, k, dir);
    std::lock_guard<std::mutex> lock(db->mu);
    if (s != EMD_OK) return s;
    if (K < 1 || K > kMaxTopK || K > db->n)
        return fail(EMD_ERR_INVALID_ARG, "K must be in 1..min(n_docs, %d)", kMaxTopK);
    if ((s = check_sizes(db, n_queries, q_row_ptr_host, meas, k, dir)) != EMD_OK) return s;
    if (n_queries == 0) return EMD_OK;
    if (!q_idx_dev || !q_w_dev || !out_idx_dev || !out_dist_dev)
        return fail(EMD_ERR_INVALID_ARG, "NULL device pointer");
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);  // NULL: the default stream
    for (int64_t i0 = 0; i0 < n_queries; i0 += db->opt.max_batch) {
        const int64_t i1 = std::min<int64_t>(n_queries, i0 + db->opt.max_batch);
        s = run_batch(db, q_row_ptr_host, q_idx_dev + q_row_ptr_host[i0], q_w_dev + q_row_ptr_host[i0], i0, i1,
                      meas, k, dir, K, nullptr, out_idx_dev + i0 * K, out_dist_dev + i0 * K, st);
        if (s != EMD_OK) return s;
    }
    return EMD_OK;
}

emd_status emd_all_pairs_topk(emd_db* db, emd_measure meas, int32_t k, int32_t K, int64_t* out_idx, float* out_dist)
{
    g_err.clear();
    if (!db || !out_idx || !out_dist) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(db->mu);
    emd_status s = check_request(db, meas, k, EMD_DIR_FWD);
    if (s != EMD_OK) return s;
    const int64_t n = db->n;
    if (K < 1 || K > kMaxTopK || K >= n) return fail(EMD_ERR_INVALID_ARG, "K must be in 1..min(n_docs - 1, %d)", kMaxTopK);
    const int64_t* rp = db->row_ptr_host.data();
    if ((s = check_sizes(db, n, rp, meas, k, EMD_DIR_FWD)) != EMD_OK) return s;
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    cudaStream_t st = db->stream;
    float* F = nullptr;
    int32_t* qidx = nullptr;
    cudaError_t e = cudaMalloc(&F, (size_t)n * (size_t)n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&qidx, (size_t)std::max<int64_t>(db->nnz, 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (F) cudaFree(F);
        return fail(EMD_ERR_OUT_OF_MEMORY, "all-pairs: the %lld x %lld forward matrix does not fit", (long long)n,
                    (long long)n);
    }
    struct Free {
        float* f;
        int32_t* q;
        ~Free()
        {
            cudaFree(f);
            cudaFree(q);
        }
    } guard{F, qidx};
    {
        Phase p(db, 6, 1, st);
        EMD_CUDA(launch_map_ids(db->col, db->nnz, db->used_ids, qidx, st), "query bins");
    }
    // every database histogram as a query: forward values F[a][b] = fwd(b -> a)
    for (int64_t i0 = 0; i0 < n; i0 += db->opt.max_batch) {
        const int64_t i1 = std::min<int64_t>(n, i0 + db->opt.max_batch);
        s = run_batch(db, rp, qidx + rp[i0], db->val + rp[i0], i0, i1, meas, k, EMD_DIR_FWD, 0, F + i0 * n, nullptr,
                      nullptr, st);
        if (s != EMD_OK) return s;
    }
    {
        Phase p(db, 6, 1, st);
        EMD_CUDA(launch_sym_max(F, n, st), "symmetric maximum");
    }
    for (int64_t i0 = 0; i0 < n; i0 += db->opt.max_batch) {
        const int64_t rows = std::min<int64_t>(db->opt.max_batch, n - i0);
        {
            Phase p(db, 5, topk_launch_count(n), st);
            EMD_CUDA(launch_topk_rows(F + i0 * n, rows, n, n, K, db->topk_scratch, db->stage_oidx, db->stage_odist, st),
                     "top-K");
        }
        EMD_CUDA(cudaMemcpyAsync(out_idx + i0 * K, db->stage_oidx, rows * K * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 st),
                 "result copy");
        EMD_CUDA(cudaMemcpyAsync(out_dist + i0 * K, db->stage_odist, rows * K * sizeof(float), cudaMemcpyDeviceToHost,
                                 st),
                 "result copy");
        EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
    }
    return read_device_errors(db);
}

emd_status emd_db_check_device_errors(emd_db* db)
{
    g_err.clear();
    if (!db) return fail(EMD_ERR_INVALID_ARG, "NULL handle");
    std::lock_guard<std::mutex> lock(db->mu);
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    EMD_CUDA(cudaDeviceSynchronize(), "synchronize");
    return read_device_errors(db);
}

emd_status emd_phase1_table(emd_db* db, const int32_t* q_idx, const float* q_w, int32_t h_q,
                            int32_t k, int32_t* used_ids, float* z, int32_t* s_out, float* w)
{
    g_err.clear();
    if (!db || !q_idx || !q_w || !z || !s_out || !w) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    if (h_q < 1 || h_q > db->opt.max_query_h) return fail(EMD_ERR_INVALID_ARG, "h_q out of range");
    if (k < 1 || k > db->opt.max_table_k) return fail(EMD_ERR_INVALID_ARG, "k out of range");
    std::lock_guard<std::mutex> lock(db->mu);
    int64_t rp[2] = {0, h_q};
    emd_queries q{1, rp, q_idx, q_w};
    emd_status s = check_query_values(db, &q);
    if (s != EMD_OK) return s;
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    cudaStream_t st = db->stream;
    Lane& L = db->lanes[0];
    EMD_CUDA(cudaMemcpyAsync(db->stage_idx, q_idx, h_q * sizeof(int32_t), cudaMemcpyHostToDevice, st), "copy");
    EMD_CUDA(cudaMemcpyAsync(db->stage_w, q_w, h_q * sizeof(float), cudaMemcpyHostToDevice, st), "copy");
    const int ldd = (int)round_up(h_q, 32);
    s = run_phase1(db, L, db->stage_idx, h_q, st);
    if (s != EMD_OK) return s;
    if (db->approx && rerank_width(db, k, h_q) > kRerankMax)
        return fail(EMD_ERR_UNSUPPORTED, "re-rank width %d exceeds %d", rerank_width(db, k, h_q), kRerankMax);
    s = run_table(db, L, db->stage_w, h_q, M_ACT, k, L.tab, db->tab_s, nullptr, st);
    if (s != EMD_OK) return s;
    const int64_t cnt = db->v_used * k;
    std::vector<float2> tz((size_t)cnt);
    EMD_CUDA(cudaMemcpyAsync(tz.data(), L.tab, cnt * sizeof(float2), cudaMemcpyDeviceToHost, st), "copy");
    EMD_CUDA(cudaMemcpyAsync(s_out, db->tab_s, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy");
    if (used_ids)
        EMD_CUDA(cudaMemcpyAsync(used_ids, db->used_ids, db->v_used * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy");
    EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
    for (int64_t i = 0; i < cnt; ++i) { z[i] = tz[i].x; w[i] = tz[i].y; }
    return read_device_errors(db);
}

emd_status emd_db_set_profiling(emd_db* db, int32_t on)
{
    if (!db) return fail(EMD_ERR_INVALID_ARG, "NULL handle");
    std::lock_guard<std::mutex> lock(db->mu);
    db->profiling = on != 0;
    return EMD_OK;
}

emd_status emd_db_profile_get(emd_db* db, emd_profile* out)
{
    if (!db || !out) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(db->mu);
    emd_status s = collect_profile(db);
    if (s != EMD_OK) return s;
    for (int p = 0; p < EMD_N_PHASES; ++p) { out->ms[p] = db->ms[p]; out->launches[p] = db->launches[p]; }
    out->total_launches = db->total_launches;
    out->pruned_queries = db->pruned_queries;
    out->prune_fallbacks = db->prune_fallbacks;
    out->graph_launches = db->graph_launches;
    out->ict_wide = db->ict_wide;
    out->fused_retries = db->fused_retries;
    return EMD_OK;
}

emd_status emd_db_profile_reset(emd_db* db)
{
    if (!db) return fail(EMD_ERR_INVALID_ARG, "NULL handle");
    std::lock_guard<std::mutex> lock(db->mu);
    emd_status s = collect_profile(db);
    if (s != EMD_OK) return s;
    for (int p = 0; p < EMD_N_PHASES; ++p) { db->ms[p] = 0.0; db->launches[p] = 0; }
    db->pruned_queries = db->prune_fallbacks = db->graph_launches = db->ict_wide = db->fused_retries = 0;
    return EMD_OK;
}

const char* emd_last_error(void) { return g_err.c_str(); }

const char* emd_version(void) { return "emd-lc-gb300 0.1 (sm_103a)"; }

}  // extern "C"
