// Sparse passes over the database for a batch of queries: the pruned symmetric top-K's reverse pass over
// the candidate rows' exact block, in a translation unit of its own (its template instances
// are many; the build compiles the units in parallel).
#include "k_sparse_dev.cuh"

namespace emd {

cudaError_t launch_prune_mapped_b(int meas, int k, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                                  const int32_t* col, const float* val, int K, int rev_warps, cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    cudaError_t e;
    switch (meas) {
    case M_RWMD: e = rev_meas_blk_b<M_RWMD, true>(k, rev_warps, qd, nq, max_q, row_ptr, col, val, st); break;
    case M_OMR: e = rev_meas_blk_b<M_OMR, true>(k, rev_warps, qd, nq, max_q, row_ptr, col, val, st); break;
    case M_ACT: e = rev_meas_blk_b<M_ACT, true>(k, rev_warps, qd, nq, max_q, row_ptr, col, val, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    k_prune_select_b<<<(unsigned)max_q, kPruneCap, 0, st>>>(qd, nq, K, true);
    return cudaGetLastError();
}

}  // namespace emd
