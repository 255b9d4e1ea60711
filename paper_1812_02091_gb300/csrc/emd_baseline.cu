// Entry points of the Section 6 baselines (bag-of-words cosine similarity, word centroid
// distance) on the resident database; see include/emd.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "emd.h"
#include "emd_db.cuh"

using namespace emd;

namespace emd {
cudaError_t launch_bow_prep(const int64_t* rp, int nq, const int32_t* idx, const float* w, const int32_t* vslot,
                            float* dense, int64_t v_used, bool clear, cudaStream_t st);
cudaError_t launch_bow_sweep(const int32_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                             const float* inv_norm, const float* dense, int64_t v_used, int nq, float* out,
                             int64_t ldo, bool as_dist, cudaStream_t st);
cudaError_t launch_doc_inv_norm(const int32_t* row_ptr, const float* val, int64_t n, float* inv_norm,
                                cudaStream_t st);
cudaError_t launch_doc_centroids(const int32_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                                 const float* E, int lde, int m, float* C, int ldc, cudaStream_t st);
cudaError_t launch_query_centroids(const int64_t* rp, int nq, const int32_t* idx, const float* w, const float* E,
                                   int lde, int m, float* C, int ldc, cudaStream_t st);
cudaError_t launch_wcd(const float* Cd, int64_t n, const float* Cq, int nq, int ldc, float* out, int64_t ldo,
                       cudaStream_t st);
}  // namespace emd

namespace {

template <typename T>
emd_status balloc(emd_db* db, T** p, int64_t count)
{
    const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EMD_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    db->allocs.push_back(q);
    db->bytes += (int64_t)bytes;
    *p = (T*)q;
    return EMD_OK;
}

#define BTRY(x)                               \
    do {                                      \
        const emd_status s_ = (x);            \
        if (s_ != EMD_OK) return s_;          \
    } while (0)

// Device state of one baseline, made on its first use (caller holds db->mu).
emd_status prepare(emd_db* db, int kind)
{
    cudaStream_t st = db->stream;
    if (!db->base_rp) BTRY(balloc(db, &db->base_rp, (int64_t)db->opt.max_batch + 1));
    if (kind == EMD_BOW_COSINE && !db->bow_ready) {
        const int64_t groups = (db->opt.max_batch + kFwdGroup - 1) / kFwdGroup;
        BTRY(balloc(db, &db->bow_dense, groups * db->v_used * kFwdGroup));
        BTRY(balloc(db, &db->doc_inv_norm, db->n));
        EMD_CUDA(cudaMemsetAsync(db->bow_dense, 0, (size_t)groups * db->v_used * kFwdGroup * sizeof(float), st),
                 "memset");
        EMD_CUDA(launch_doc_inv_norm(db->row_ptr, db->val, db->n, db->doc_inv_norm, st), "document norms");
        db->total_launches += 1;
        db->launches[6] += 1;
        db->bow_ready = true;
    }
    if (kind == EMD_WCD && !db->wcd_ready) {
        db->ldc = (int)((db->m + 31) / 32 * 32);
        BTRY(balloc(db, &db->doc_centroid, db->n * db->ldc));
        BTRY(balloc(db, &db->q_centroid, (int64_t)db->opt.max_batch * db->ldc));
        EMD_CUDA(launch_doc_centroids(db->row_ptr, db->col, db->val, db->n, db->emb_used, db->ldm, db->m,
                                      db->doc_centroid, db->ldc, st),
                 "document centroids");
        db->total_launches += 1;
        db->launches[6] += 1;
        db->wcd_ready = true;
    }
    return EMD_OK;
}

// Queries i0..i1-1, bins already in stage_idx / stage_w, offsets in base_rp: values (or,
// with as_dist, distances for the top-K) into stage_out rows.
emd_status run_baseline(emd_db* db, int kind, int nb, bool as_dist, cudaStream_t st)
{
    if (kind == EMD_BOW_COSINE) {
        {
            Phase p(db, 0, 1, st);
            EMD_CUDA(launch_bow_prep(db->base_rp, nb, db->stage_idx, db->stage_w, db->vslot, db->bow_dense,
                                     db->v_used, false, st),
                     "query vectors");
        }
        {
            Phase p(db, 3, 1, st);
            EMD_CUDA(launch_bow_sweep(db->row_ptr, db->col, db->val, db->n, db->doc_inv_norm, db->bow_dense,
                                      db->v_used, nb, db->stage_out, db->n, as_dist, st),
                     "cosine sweep");
        }
        Phase p(db, 6, 1, st);
        EMD_CUDA(launch_bow_prep(db->base_rp, nb, db->stage_idx, db->stage_w, db->vslot, db->bow_dense, db->v_used,
                                 true, st),
                 "query vectors");
        return EMD_OK;
    }
    {
        Phase p(db, 0, 1, st);
        EMD_CUDA(launch_query_centroids(db->base_rp, nb, db->stage_idx, db->stage_w, db->emb, db->ldm, db->m,
                                        db->q_centroid, db->ldc, st),
                 "query centroids");
    }
    Phase p(db, 1, 1, st);
    EMD_CUDA(launch_wcd(db->doc_centroid, db->n, db->q_centroid, nb, db->ldc, db->stage_out, db->n, st),
             "centroid distances");
    return EMD_OK;
}

emd_status baseline_entry(emd_db* db, const emd_queries* q, int kind, int K, float* out_all, int64_t* out_idx,
                          float* out_dist)
{
    clear_error();
    if (!db || !q) return fail(EMD_ERR_INVALID_ARG, "NULL argument");
    if (kind != EMD_BOW_COSINE && kind != EMD_WCD) return fail(EMD_ERR_INVALID_ARG, "unknown baseline %d", kind);
    std::lock_guard<std::mutex> lock(db->mu);
    if (kind == EMD_WCD && db->cost_mode)
        return fail(EMD_ERR_UNSUPPORTED, "the word centroid distance needs embeddings (cost-matrix database)");
    if (K > 0 && (K > kMaxTopK || K > db->n))
        return fail(EMD_ERR_INVALID_ARG, "K must be in 1..min(n_docs, %d)", kMaxTopK);
    if (q->n_queries < 0) return fail(EMD_ERR_INVALID_ARG, "n_queries < 0");
    if (q->n_queries == 0) return EMD_OK;
    if (!q->row_ptr || q->row_ptr[0] != 0) return fail(EMD_ERR_INVALID_ARG, "query row_ptr invalid");
    for (int64_t i = 0; i < q->n_queries; ++i) {
        const int64_t h = q->row_ptr[i + 1] - q->row_ptr[i];
        if (h < 1 || h > db->opt.max_query_h)
            return fail(EMD_ERR_INVALID_ARG, "query %lld has %lld bins (allowed 1..%d)", (long long)i, (long long)h,
                        db->opt.max_query_h);
    }
    emd_status s = check_query_values(db, q);
    if (s != EMD_OK) return s;
    if (K > 0 ? (!out_idx || !out_dist) : !out_all) return fail(EMD_ERR_INVALID_ARG, "output is NULL");
    EMD_CUDA(cudaSetDevice(db->dev), "cudaSetDevice");
    BTRY(prepare(db, kind));
    cudaStream_t st = db->stream;
    std::vector<int64_t> rp((size_t)db->opt.max_batch + 1);
    int64_t i0 = 0;
    while (i0 < q->n_queries) {
        int64_t i1 = i0;
        while (i1 < q->n_queries && i1 - i0 < db->opt.max_batch && q->row_ptr[i1 + 1] - q->row_ptr[i0] <= db->stage_bins)
            ++i1;
        const int nb = (int)(i1 - i0);
        const int64_t base = q->row_ptr[i0];
        for (int i = 0; i <= nb; ++i) rp[i] = q->row_ptr[i0 + i] - base;
        EMD_CUDA(cudaMemcpyAsync(db->base_rp, rp.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st),
                 "query copy");
        EMD_CUDA(cudaMemcpyAsync(db->stage_idx, q->idx + base, rp[nb] * sizeof(int32_t), cudaMemcpyHostToDevice, st),
                 "query copy");
        EMD_CUDA(cudaMemcpyAsync(db->stage_w, q->w + base, rp[nb] * sizeof(float), cudaMemcpyHostToDevice, st),
                 "query copy");
        BTRY(run_baseline(db, kind, nb, K > 0, st));
        if (K > 0) {
            {
                Phase p(db, 5, topk_launch_count(db->n), st);
                EMD_CUDA(launch_topk_rows(db->stage_out, nb, db->n, db->n, K, db->topk_scratch, db->stage_oidx,
                                          db->stage_odist, st),
                         "top-K");
            }
            EMD_CUDA(cudaMemcpyAsync(out_idx + i0 * K, db->stage_oidx, (size_t)nb * K * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st),
                     "result copy");
            EMD_CUDA(cudaMemcpyAsync(out_dist + i0 * K, db->stage_odist, (size_t)nb * K * sizeof(float),
                                     cudaMemcpyDeviceToHost, st),
                     "result copy");
        } else {
            EMD_CUDA(cudaMemcpyAsync(out_all + i0 * db->n, db->stage_out, (size_t)nb * db->n * sizeof(float),
                                     cudaMemcpyDeviceToHost, st),
                     "result copy");
        }
        EMD_CUDA(cudaStreamSynchronize(st), "synchronize");
        i0 = i1;
    }
    return EMD_OK;
}

}  // namespace

emd_status emd_baseline_batch(emd_db* db, const emd_queries* q, emd_baseline kind, float* out)
{
    return baseline_entry(db, q, (int)kind, 0, out, nullptr, nullptr);
}

emd_status emd_baseline_topk(emd_db* db, const emd_queries* q, emd_baseline kind, int32_t K, int64_t* out_idx,
                             float* out_dist)
{
    if (K < 1) return fail(EMD_ERR_INVALID_ARG, "K must be >= 1");
    return baseline_entry(db, q, (int)kind, K, nullptr, out_idx, out_dist);
}
