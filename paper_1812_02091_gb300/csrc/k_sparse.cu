// Sparse passes over the database (Section 5; Section 6, the reverse direction and the
// symmetric maximum) and the top-K neighbour selection: the per-query launchers, the
// all-pairs helpers and the allocation-free top-K entry point.
#include "k_sparse_dev.cuh"

namespace emd {

cudaError_t launch_rev(int meas, int k, const int32_t* row_ptr, const int32_t* col,
                       const float* val, int64_t n, const float* D, int ldd, int h,
                       const float* q_w, const float* t_fwd, float* t_rev, float* t_max,
                       const int64_t* doc_ids, bool sq, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    switch (meas) {
    case M_RWMD: return rev_meas<M_RWMD>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, doc_ids, nullptr, sq, st);
    case M_OMR: return rev_meas<M_OMR>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, doc_ids, nullptr, sq, st);
    case M_ICT: return rev_meas<M_ICT>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, doc_ids, nullptr, sq, st);
    default: return rev_meas<M_ACT>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, doc_ids, nullptr, sq, st);
    }
}

cudaError_t launch_prune(int meas, int k, const int32_t* row_ptr, const int32_t* col, const float* val,
                         int64_t n, const float* D, int ldd, int h, const float* q_w, const float* t_fwd,
                         const int64_t* sel_idx, const float* sel_val, int K, int64_t* cand, int* count,
                         float* sym, int64_t* out_idx, float* out_dist, int* ok, bool sq, cudaStream_t st)
{
    (void)sel_idx;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 4);
    k_prune_compact<<<blocks, 256, 0, st>>>(t_fwd, n, sel_val, K, kPruneCap, cand, count);
    // reverse pass on the candidate slots (t_rev into sym + kPruneCap, max into sym)
    switch (meas) {
    case M_RWMD: e = rev_meas_blk<M_RWMD>(k, row_ptr, col, val, kPruneCap, D, ldd, h, q_w, t_fwd, sym + kPruneCap, sym, cand, count, sq, st); break;
    case M_OMR: e = rev_meas_blk<M_OMR>(k, row_ptr, col, val, kPruneCap, D, ldd, h, q_w, t_fwd, sym + kPruneCap, sym, cand, count, sq, st); break;
    case M_ICT:
        k_rev_generic_blk<M_ICT><<<kPruneCap, kRevW * 32, 0, st>>>(row_ptr, col, val, D, ldd, h, q_w, k, t_fwd,
                                                                  sym + kPruneCap, sym, cand, count, sq);
        e = cudaGetLastError();
        break;
    default: e = rev_meas_blk<M_ACT>(k, row_ptr, col, val, kPruneCap, D, ldd, h, q_w, t_fwd, sym + kPruneCap, sym, cand, count, sq, st); break;
    }
    if (e != cudaSuccess) return e;
    k_prune_select<<<1, kPruneCap, 0, st>>>(cand, sym, count, kPruneCap, sel_val, K, out_idx, out_dist, ok);
    return cudaGetLastError();
}

}  // namespace emd


namespace {

__global__ void k_map_ids(const int32_t* __restrict__ col, int64_t nnz, const int32_t* __restrict__ used_ids,
                          int32_t* __restrict__ out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = used_ids[col[e]];
}

// One 32 x 32 tile pair (I, J), I <= J, per block: both tiles through shared memory, the
// element-wise max written to both (the symmetric bound of Section 6 from the forward values
// of a pair and of its transpose); the diagonal becomes +inf (no self-match).
__global__ void k_sym_max(float* __restrict__ F, int64_t n)
{
    const int64_t I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    __shared__ float a[32][33], b[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = I * 32 + r, j = J * 32 + tx;
        a[r][tx] = (i < n && j < n) ? F[i * n + j] : 0.f;
        const int64_t i2 = J * 32 + r, j2 = I * 32 + tx;
        b[r][tx] = (i2 < n && j2 < n) ? F[i2 * n + j2] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = I * 32 + r, j = J * 32 + tx;
        if (i < n && j < n) F[i * n + j] = (i == j) ? INFINITY : fmaxf(a[r][tx], b[tx][r]);
        const int64_t i2 = J * 32 + r, j2 = I * 32 + tx;
        if (I != J && i2 < n && j2 < n) F[i2 * n + j2] = fmaxf(b[r][tx], a[tx][r]);
    }
}

}  // namespace

namespace emd {

cudaError_t launch_map_ids(const int32_t* col, int64_t nnz, const int32_t* used_ids, int32_t* out, cudaStream_t st)
{
    if (nnz <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    k_map_ids<<<(unsigned)blocks, 256, 0, st>>>(col, nnz, used_ids, out);
    return cudaGetLastError();
}

cudaError_t launch_sym_max(float* F, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nt = (n + 31) / 32;
    if (nt > 65535) return cudaErrorInvalidValue;
    k_sym_max<<<dim3((unsigned)nt, (unsigned)nt), dim3(32, 8), 0, st>>>(F, n);
    return cudaGetLastError();
}

cudaError_t launch_topk_rows(const float* t, int64_t rows, int64_t n, int64_t ldt, int K,
                             unsigned long long* scratch, int64_t* out_idx, float* out_dist,
                             cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    if (K <= 16) return topk_kt<16>(t, rows, n, ldt, K, scratch, out_idx, out_dist, st);
    if (K <= 32) return topk_kt<32>(t, rows, n, ldt, K, scratch, out_idx, out_dist, st);
    return topk_kt<64>(t, rows, n, ldt, K, scratch, out_idx, out_dist, st);
}

cudaError_t launch_topk(const float* t, int64_t n, int K, unsigned long long* scratch,
                        int64_t* out_idx, float* out_dist, cudaStream_t st)
{
    return launch_topk_rows(t, 1, n, n, K, scratch, out_idx, out_dist, st);
}

}  // namespace emd

// ------------------------------------------------------------------ top-K without allocation
//
// emd_topk_select_static: the top-K selection kernels above, with their block-partial
// scratch in a fixed device array instead of memory the caller or the library
// allocates.  It is meant for callers that may not call cudaMalloc: code that runs
// inside a host framework whose own caching allocator owns all device memory (a raw
// cudaMalloc would bypass its accounting), or a latency-bound serving loop where the
// implicit device synchronisation of cudaMalloc/cudaFree would stall work in flight.
//
// The array lives for the life of the process on every device that loads the library.
// Every call shares it and it keeps the last call's contents; nothing in it needs to
// start at zero (each block writes its partial list before the merge reads it).  Calls
// whose kernels overlap on the GPU (different streams, no ordering between them) race
// on the array.

#include <mutex>

namespace {

constexpr int kStaticMaxRows = 64;  // rows (queries) per call
constexpr size_t kStaticScratchKeys = (size_t)kStaticMaxRows * emd::kTopkScratchRow;

static __device__ __align__(256) unsigned long long g_topk_static_scratch[kStaticScratchKeys];

std::mutex g_static_mu;
constexpr int kStaticMaxDevices = 64;
unsigned long long* g_static_ptr[kStaticMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
cudaError_t static_scratch(unsigned long long** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_topk_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" emd_status emd_topk_select_static(const float* t_dev, int64_t n_rows, int64_t n,
                                             int32_t K, int64_t* out_idx_dev, float* out_dist_dev,
                                             void* stream)
{
    emd::clear_error();
    if (n_rows < 0 || n_rows > kStaticMaxRows)
        return emd::set_error(EMD_ERR_INVALID_ARG,
                              "emd_topk_select_static: n_rows must be 0..64 (the static scratch holds 64 rows)");
    if (n < 1 || n > 0xffffffffll)
        return emd::set_error(EMD_ERR_INVALID_ARG, "emd_topk_select_static: n must be 1..2^32-1");
    if (K < 1 || K > emd::kMaxTopK || K > n)
        return emd::set_error(EMD_ERR_INVALID_ARG, "emd_topk_select_static: K must be 1..min(n, 64)");
    if (n_rows == 0) return EMD_OK;
    if (!t_dev || !out_idx_dev || !out_dist_dev)
        return emd::set_error(EMD_ERR_INVALID_ARG, "emd_topk_select_static: NULL device pointer");
    unsigned long long* scratch = nullptr;
    cudaError_t e = static_scratch(&scratch);
    if (e != cudaSuccess)
        return emd::set_error(EMD_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = emd::launch_topk_rows(t_dev, n_rows, n, n, K, scratch, out_idx_dev, out_dist_dev, st);
    if (e != cudaSuccess) return emd::set_error(EMD_ERR_CUDA, cudaGetErrorString(e));
    return EMD_OK;
}
