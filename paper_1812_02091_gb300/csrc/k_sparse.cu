// Sparse passes over the database (Section 4, Phase 2 and 3; Section 5, the reverse
// direction and the symmetric maximum) and the top-K neighbour selection.
#include <math.h>

#include <algorithm>

#include "emd_internal.cuh"

namespace emd {
namespace {

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ------------------------------------------------------------------ forward pass
//
// Phase 2 (Eq. 6-8) and Phase 3 (Eq. 9) evaluated per nonzero: a database weight x at
// vocabulary row u is moved into the query along row u's table, k-1 capacity-limited
// transfers then the rest at the k-th distance.  The per-nonzero costs are summed per
// document (t_fwd).  One warp per document, lanes over its nonzeros (coalesced col/val
// loads), table rows gathered from L2, warp-shuffle sum.

template <int MEAS>
__device__ __forceinline__ float fwd_cost(float x, const float2* __restrict__ T, int keff)
{
    if (MEAS == M_RWMD) return x * T[0].x;
    if (MEAS == M_OMR) {
        const float2 t0 = T[0];
        if (t0.x == 0.f && keff >= 2) {
            const float r = x - fminf(x, t0.y);  // free transfer to the overlapping bin
            return r != 0.f ? r * T[1].x : 0.f;
        }
        return x * t0.x;
    }
    float r = x, c = 0.f;
    for (int l = 0; l < keff - 1; ++l) {
        const float2 t = T[l];
        const float tau = fminf(r, t.y);
        c = fmaf(tau, t.x, c);
        r -= tau;
        if (r == 0.f) return c;
    }
    return fmaf(r, T[keff - 1].x, c);
}

template <int MEAS>
__global__ void k_fwd(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                      const float* __restrict__ val, int64_t n, const float2* __restrict__ tab,
                      int k, int keff, float* __restrict__ t_fwd)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float acc = 0.f;
        for (int32_t e = a + lane; e < b; e += 32) {
            const int32_t u = col[e];
            acc += fwd_cost<MEAS>(val[e], tab + (int64_t)u * k, keff);
        }
        acc = warp_sum(acc);
        if (lane == 0) t_fwd[d] = acc;
    }
}

// ------------------------------------------------------------------ reverse pass
//
// The query's bins are the sources (mass q_j), the document's bins the destinations
// (capacities x_u), the cost block D[supp(d), j] is gathered from the Phase-1 matrix.
// One warp per document; lane j' of chunk c handles query bin j = 32c + j' and keeps a
// register top-KT of (distance, capacity) over the document's bins, visited in CSR
// order (strict '<' keeps the earlier bin first on equal distance).  Reads of
// D[u, 32c .. 32c+31] are one 128-byte line per bin.

template <int MEAS>
__device__ __forceinline__ float rev_cost_sorted(float qj, const float* z, const float* cap,
                                                 int keff)
{
    if (MEAS == M_RWMD) return qj * z[0];
    if (MEAS == M_OMR) {
        if (z[0] == 0.f && keff >= 2) {
            const float r = qj - fminf(qj, cap[0]);
            return r != 0.f ? r * z[1] : 0.f;
        }
        return qj * z[0];
    }
    float r = qj, c = 0.f;
    for (int l = 0; l < keff - 1; ++l) {
        const float tau = fminf(r, cap[l]);
        c = fmaf(tau, z[l], c);
        r -= tau;
        if (r == 0.f) return c;
    }
    return fmaf(r, z[keff - 1], c);
}

template <int MEAS, int KT>
__global__ void k_rev(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                      const float* __restrict__ val, int64_t n, const float* __restrict__ D,
                      int ldd, int h, const float* __restrict__ q_w, int k,
                      const float* __restrict__ t_fwd, float* __restrict__ t_rev,
                      float* __restrict__ t_max)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        const int hd = b - a;
        const int keff = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? min(2, hd) : min(k, hd));
        float total = 0.f;
        for (int jc = 0; jc < h; jc += 32) {
            const int j = jc + lane;
            float z[KT], cap[KT];
#pragma unroll
            for (int l = 0; l < KT; ++l) { z[l] = INFINITY; cap[l] = 0.f; }
            for (int32_t eb = a; eb < b; eb += 32) {
                const int32_t e = eb + lane;
                const int32_t u = e < b ? col[e] : 0;
                const float x = e < b ? val[e] : 0.f;
                const int cnt = min(32, b - eb);
                for (int i = 0; i < cnt; ++i) {
                    const int32_t ui = __shfl_sync(0xffffffffu, u, i);
                    const float xi = __shfl_sync(0xffffffffu, x, i);
                    const float dd = D[(int64_t)ui * ldd + j];  // j < ldd: padding holds +inf
                    if (dd < z[KT - 1]) {
                        z[KT - 1] = dd;
                        cap[KT - 1] = xi;
#pragma unroll
                        for (int l = KT - 1; l > 0; --l) {
                            if (z[l] < z[l - 1]) {
                                float tz = z[l]; z[l] = z[l - 1]; z[l - 1] = tz;
                                float tc = cap[l]; cap[l] = cap[l - 1]; cap[l - 1] = tc;
                            }
                        }
                    }
                }
            }
            if (j < h) total += rev_cost_sorted<MEAS>(q_w[j], z, cap, keff);
        }
        total = warp_sum(total);
        if (lane == 0) {
            t_rev[d] = total;
            if (t_max) t_max[d] = fmaxf(t_fwd[d], total);
        }
    }
}

// k above the register width (ICT, large k): per lane, successive minima over the
// document's bins, each strictly after the previous in (distance, bin position) order,
// until the source mass is placed.  O(steps * h_d) per query bin.
template <int MEAS>
__global__ void k_rev_generic(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const float* __restrict__ val, int64_t n, const float* __restrict__ D,
                              int ldd, int h, const float* __restrict__ q_w, int k,
                              const float* __restrict__ t_fwd, float* __restrict__ t_rev,
                              float* __restrict__ t_max)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        const int hd = b - a;
        const int keff = MEAS == M_ICT ? hd : min(k, hd);
        float total = 0.f;
        for (int j = lane; j < h; j += 32) {
            float r = q_w[j], c = 0.f;
            float pz = -INFINITY;
            int pe = -1;
            for (int l = 0; l < keff; ++l) {
                float bz = INFINITY, bx = 0.f;
                int be = INT32_MAX;
                for (int32_t e = a; e < b; ++e) {
                    const float dd = D[(int64_t)col[e] * ldd + j];
                    const int pos = e - a;
                    const bool after = dd > pz || (dd == pz && pos > pe);
                    if (after && (dd < bz || (dd == bz && pos < be))) { bz = dd; be = pos; bx = val[e]; }
                }
                if (l < keff - 1) {
                    const float tau = fminf(r, bx);
                    c = fmaf(tau, bz, c);
                    r -= tau;
                    if (r == 0.f) break;
                } else {
                    c = fmaf(r, bz, c);
                }
                pz = bz;
                pe = be;
            }
            total += c;
        }
        total = warp_sum(total);
        if (lane == 0) {
            t_rev[d] = total;
            if (t_max) t_max[d] = fmaxf(t_fwd[d], total);
        }
    }
}

// ------------------------------------------------------------------ top-K selection
//
// Keys are (float bits of the distance << 32) | document id: distances are >= 0, so the
// unsigned order of the keys is the (distance, id) order and every key is unique.
// Each thread keeps a sorted register list of its KT smallest keys; the block merges the
// lists pairwise in shared memory (log2(threads) levels).  With several blocks per query
// the block results go to scratch and one more block merges them.

template <int KT>
__device__ __forceinline__ void list_insert(unsigned long long (&L)[KT], unsigned long long key)
{
    if (key < L[KT - 1]) {
        L[KT - 1] = key;
#pragma unroll
        for (int l = KT - 1; l > 0; --l) {
            if (L[l] < L[l - 1]) { unsigned long long t = L[l]; L[l] = L[l - 1]; L[l - 1] = t; }
        }
    }
}

template <int KT>
__device__ void block_merge_and_emit(unsigned long long (&L)[KT], int K, unsigned long long* out_keys,
                                     int64_t* out_idx, float* out_dist)
{
    extern __shared__ unsigned long long sm[];  // [blockDim.x][KT]
    const int tid = threadIdx.x;
#pragma unroll
    for (int l = 0; l < KT; ++l) sm[tid * KT + l] = L[l];
    __syncthreads();
    for (int active = blockDim.x; active > 1; active >>= 1) {
        const int half = active >> 1;
        if (tid < half) {
            const unsigned long long* A = sm + tid * KT;
            const unsigned long long* B = sm + (tid + half) * KT;
            unsigned long long M[KT];
            int ia = 0, ib = 0;
#pragma unroll
            for (int l = 0; l < KT; ++l) {
                const unsigned long long x = A[ia], y = B[ib];
                if (x <= y) { M[l] = x; ++ia; } else { M[l] = y; ++ib; }
            }
#pragma unroll
            for (int l = 0; l < KT; ++l) sm[tid * KT + l] = M[l];
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int l = 0; l < K; ++l) {
            const unsigned long long key = sm[l];
            if (out_keys) out_keys[l] = key;
            if (out_idx) {
                out_idx[l] = (key == ~0ull) ? -1 : (int64_t)(key & 0xffffffffull);
                out_dist[l] = (key == ~0ull) ? INFINITY : __uint_as_float((unsigned)(key >> 32));
            }
        }
    }
}

template <int KT>
__global__ void __launch_bounds__(kTopkThreads)
k_topk_values(const float* __restrict__ t, int64_t n, int K, int64_t per_block,
              unsigned long long* __restrict__ scratch, int64_t* __restrict__ out_idx,
              float* __restrict__ out_dist)
{
    unsigned long long L[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) L[l] = ~0ull;
    const int64_t lo = (int64_t)blockIdx.x * per_block;
    const int64_t hi = min(n, lo + per_block);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(t[i]) << 32) | (unsigned long long)(uint32_t)i;
        list_insert<KT>(L, key);
    }
    if (gridDim.x == 1)
        block_merge_and_emit<KT>(L, K, nullptr, out_idx, out_dist);
    else
        block_merge_and_emit<KT>(L, KT, scratch + (int64_t)blockIdx.x * KT, nullptr, nullptr);
}

template <int KT>
__global__ void __launch_bounds__(kTopkThreads)
k_topk_keys(const unsigned long long* __restrict__ keys, int64_t count, int K,
            int64_t* __restrict__ out_idx, float* __restrict__ out_dist)
{
    unsigned long long L[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) L[l] = ~0ull;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) list_insert<KT>(L, keys[i]);
    block_merge_and_emit<KT>(L, K, nullptr, out_idx, out_dist);
}

template <int KT>
cudaError_t topk_kt(const float* t, int64_t n, int K, unsigned long long* scratch,
                    int64_t* out_idx, float* out_dist, cudaStream_t st)
{
    const size_t smem = (size_t)kTopkThreads * KT * sizeof(unsigned long long);
    int blocks = (int)std::min<int64_t>(kTopkMaxBlocks, std::max<int64_t>(1, n / 8192));
    const int64_t per_block = (n + blocks - 1) / blocks;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_topk_values<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_topk_keys<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_topk_values<KT><<<blocks, kTopkThreads, smem, st>>>(t, n, K, per_block, scratch, out_idx, out_dist);
    if (blocks > 1)
        k_topk_keys<KT><<<1, kTopkThreads, smem, st>>>(scratch, (int64_t)blocks * KT, K, out_idx, out_dist);
    return cudaGetLastError();
}

template <int MEAS>
cudaError_t rev_meas(int k, const int32_t* row_ptr, const int32_t* col, const float* val,
                     int64_t n, const float* D, int ldd, int h, const float* q_w,
                     const float* t_fwd, float* t_rev, float* t_max, cudaStream_t st)
{
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks));
    const int kt = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? 2 : (MEAS == M_ICT ? 1 << 30 : k));
    if (kt <= 1) k_rev<MEAS, 1><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max);
    else if (kt <= 2) k_rev<MEAS, 2><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max);
    else if (kt <= 4) k_rev<MEAS, 4><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max);
    else if (kt <= 8) k_rev<MEAS, 8><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max);
    else if (kt <= 16) k_rev<MEAS, 16><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max);
    else k_rev_generic<MEAS><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fwd(int meas, const int32_t* row_ptr, const int32_t* col, const float* val,
                       int64_t n, const float2* tab, int k, int keff, float* t_fwd,
                       cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks));
    switch (meas) {
    case M_RWMD: k_fwd<M_RWMD><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, tab, k, keff, t_fwd); break;
    case M_OMR: k_fwd<M_OMR><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, tab, k, keff, t_fwd); break;
    default: k_fwd<M_ACT><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, tab, k, keff, t_fwd); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_rev(int meas, int k, const int32_t* row_ptr, const int32_t* col,
                       const float* val, int64_t n, const float* D, int ldd, int h,
                       const float* q_w, const float* t_fwd, float* t_rev, float* t_max,
                       cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    switch (meas) {
    case M_RWMD: return rev_meas<M_RWMD>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, st);
    case M_OMR: return rev_meas<M_OMR>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, st);
    case M_ICT: return rev_meas<M_ICT>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, st);
    default: return rev_meas<M_ACT>(k, row_ptr, col, val, n, D, ldd, h, q_w, t_fwd, t_rev, t_max, st);
    }
}

cudaError_t launch_topk(const float* t, int64_t n, int K, unsigned long long* scratch,
                        int64_t* out_idx, float* out_dist, cudaStream_t st)
{
    if (K <= 16) return topk_kt<16>(t, n, K, scratch, out_idx, out_dist, st);
    if (K <= 32) return topk_kt<32>(t, n, K, scratch, out_idx, out_dist, st);
    return topk_kt<64>(t, n, K, scratch, out_idx, out_dist, st);
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
constexpr size_t kStaticScratchKeys = (size_t)kStaticMaxRows * emd::kTopkMaxBlocks * emd::kMaxTopK;

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
    for (int64_t r = 0; r < n_rows; ++r) {
        e = emd::launch_topk(t_dev + r * n, n, K, scratch + r * (int64_t)emd::kTopkMaxBlocks * emd::kMaxTopK,
                             out_idx_dev + r * K, out_dist_dev + r * K, st);
        if (e != cudaSuccess) return emd::set_error(EMD_ERR_CUDA, cudaGetErrorString(e));
    }
    return EMD_OK;
}
