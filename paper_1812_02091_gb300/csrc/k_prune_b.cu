// Sparse passes over the database for a batch of queries: the pruned symmetric top-K's reverse pass over
// the full distance matrix, in a translation unit of its own (its template instances
// are many; the build compiles the units in parallel).
#include "k_sparse_dev.cuh"

namespace emd {

cudaError_t launch_prune_b(int meas, int k, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                           const int32_t* col, const float* val, int64_t n, int K, int rev_warps, cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 4);
    k_prune_compact_b<<<dim3((unsigned)blocks, (unsigned)max_q), 256, 0, st>>>(qd, nq, n, K);
    cudaError_t e;
    switch (meas) {
    case M_RWMD: e = rev_meas_blk_b<M_RWMD>(k, rev_warps, qd, nq, max_q, row_ptr, col, val, st); break;
    case M_OMR: e = rev_meas_blk_b<M_OMR>(k, rev_warps, qd, nq, max_q, row_ptr, col, val, st); break;
    case M_ICT:
        k_rev_generic_cand_b<M_ICT><<<dim3(kPruneCap, (unsigned)max_q), kRevW * 32, 0, st>>>(qd, nq, row_ptr, col,
                                                                                            val, k);
        e = cudaGetLastError();
        break;
    default: e = rev_meas_blk_b<M_ACT>(k, rev_warps, qd, nq, max_q, row_ptr, col, val, st); break;
    }
    if (e != cudaSuccess) return e;
    k_prune_select_b<<<(unsigned)max_q, kPruneCap, 0, st>>>(qd, nq, K, false);
    return cudaGetLastError();
}

}  // namespace emd
