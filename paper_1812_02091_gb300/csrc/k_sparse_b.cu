// Sparse passes over the database for a batch of queries (one launch over all its queries,
// descriptors in QDesc): the reverse direction, the pruned symmetric top-K with its
// candidate rows, and the top-K selection.
#include "k_sparse_dev.cuh"

namespace emd {

cudaError_t launch_rev_b(int meas, int k, int dir, const QDesc* qd, const int* nq, int max_q,
                         const int32_t* row_ptr, const int32_t* col, const float* val, int64_t n, cudaStream_t st)
{
    if (max_q <= 0 || n <= 0) return cudaSuccess;
    if (dir != EMD_DIR_REV && dir != EMD_DIR_MAX) return cudaErrorInvalidValue;
    switch (meas) {
    case M_RWMD: return rev_meas_b<M_RWMD>(k, dir, qd, nq, max_q, row_ptr, col, val, n, st);
    case M_OMR: return rev_meas_b<M_OMR>(k, dir, qd, nq, max_q, row_ptr, col, val, n, st);
    case M_ICT: return rev_meas_b<M_ICT>(k, dir, qd, nq, max_q, row_ptr, col, val, n, st);
    default: return rev_meas_b<M_ACT>(k, dir, qd, nq, max_q, row_ptr, col, val, n, st);
    }
}


cudaError_t launch_prune_compact_b(const QDesc* qd, const int* nq, int max_q, int64_t n, int K, cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 4);
    k_prune_compact_b<<<dim3((unsigned)blocks, (unsigned)max_q), 256, 0, st>>>(qd, nq, n, K);
    return cudaGetLastError();
}

cudaError_t launch_cand_rows_b(const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr, const int32_t* col,
                               bool reset, cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    const dim3 g(kPruneCap, (unsigned)max_q);
    if (reset)
        k_cand_reset_b<<<g, 128, 0, st>>>(qd, nq, row_ptr, col);
    else
        k_cand_rows_b<<<g, 128, 0, st>>>(qd, nq, row_ptr, col);
    return cudaGetLastError();
}


cudaError_t launch_topk_b(const QDesc* qd, const int* nq, int max_q, int64_t n, int K,
                          unsigned long long* scratch, bool fwd_rows, cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    if (K <= 16) return topk_kt_b<16>(qd, nq, max_q, n, K, scratch, fwd_rows, st);
    if (K <= 32) return topk_kt_b<32>(qd, nq, max_q, n, K, scratch, fwd_rows, st);
    return topk_kt_b<64>(qd, nq, max_q, n, K, scratch, fwd_rows, st);
}

}  // namespace emd
