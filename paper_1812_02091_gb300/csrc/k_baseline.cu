// The two cheap baselines of Section 6, on the database resident for the EMD bounds:
//
//  * bag-of-words cosine similarity: the dot product of the query's and each document's
//    weights after L2 normalisation (no embeddings).  The query side is scattered into a
//    dense vector over the used vocabulary, eight queries interleaved (entry u of query g
//    at dense[u * 8 + g]); one CSR sweep serves the eight: a warp takes a document, lane =
//    8 x phase + query, as in the grouped forward pass, so the gather of one nonzero for
//    the eight queries is one 32-byte sector.
//  * word centroid distance: the Euclidean distance between the weight-averaged embedding
//    vectors.  Centroids are formed with compensated products and sums (Ogita, Rump and
//    Oishi, "Accurate sum and dot product", 2005) and rounded to FP32 once; distances take
//    the differences directly (no norm expansion, so nothing cancels).

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "emd_internal.cuh"

namespace emd {
namespace {

// Error-free transformations (Knuth's TwoSum; TwoProduct through one FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}

// s + c accumulates sum(x_i * y_i) with the error terms carried in c.
__device__ __forceinline__ void dot2_step(float x, float y, float& s, float& c)
{
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    c += te + pe;
}

// One block per query: the query's squared norm (block reduction), then its weights
// divided by the norm scattered into its group's dense vector (ids outside the used
// vocabulary have no document to meet and are skipped).  clear: write zeros instead, so the
// dense vectors are all-zero between batches without a full memset.
__global__ void k_bow_prep(const int64_t* __restrict__ rp, int nq, const int32_t* __restrict__ idx,
                           const float* __restrict__ w, const int32_t* __restrict__ vslot, float* __restrict__ dense,
                           int64_t v_used, bool clear)
{
    const int q = blockIdx.x;
    if (q >= nq) return;
    const int64_t a = rp[q], b = rp[q + 1];
    float* dq = dense + (int64_t)(q / kFwdGroup) * v_used * kFwdGroup + (q % kFwdGroup);
    if (clear) {
        for (int64_t j = a + threadIdx.x; j < b; j += blockDim.x) {
            const int32_t s = vslot[idx[j]];
            if (s >= 0) dq[(int64_t)s * kFwdGroup] = 0.f;
        }
        return;
    }
    __shared__ float part[32];
    float acc = 0.f;
    for (int64_t j = a + threadIdx.x; j < b; j += blockDim.x) acc = fmaf(w[j], w[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[0] = t;
    }
    __syncthreads();
    const float nrm = sqrtf(part[0]);
    for (int64_t j = a + threadIdx.x; j < b; j += blockDim.x) {
        const int32_t s = vslot[idx[j]];
        if (s >= 0) dq[(int64_t)s * kFwdGroup] = nrm > 0.f ? w[j] / nrm : 0.f;
    }
}

// One warp per document and group of eight queries (blockIdx.y): lane = 8 x phase + query;
// phase p sums the nonzeros a + p, a + p + 4, ..., then (p0 + p1) + (p2 + p3).
__global__ void k_bow_sweep(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const float* __restrict__ val, int64_t n, const float* __restrict__ inv_norm,
                            const float* __restrict__ dense, int64_t v_used, int nq, float* __restrict__ out,
                            int64_t ldo, bool as_dist)
{
    const int lane = threadIdx.x & 31, g = lane & 7, ph = lane >> 3;
    const int q = blockIdx.y * kFwdGroup + g;
    const float* dg = dense + (int64_t)blockIdx.y * v_used * kFwdGroup + g;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float acc = 0.f;
        int32_t e = a + ph;
        for (; e + 12 < b; e += 16) {  // four independent gathers in flight, summed in order
            const int32_t c0 = col[e], c1 = col[e + 4], c2 = col[e + 8], c3 = col[e + 12];
            const float v0 = val[e], v1 = val[e + 4], v2 = val[e + 8], v3 = val[e + 12];
            const float x0 = dg[(int64_t)c0 * kFwdGroup], x1 = dg[(int64_t)c1 * kFwdGroup];
            const float x2 = dg[(int64_t)c2 * kFwdGroup], x3 = dg[(int64_t)c3 * kFwdGroup];
            acc = fmaf(v0, x0, acc);
            acc = fmaf(v1, x1, acc);
            acc = fmaf(v2, x2, acc);
            acc = fmaf(v3, x3, acc);
        }
        for (; e < b; e += 4) acc = fmaf(val[e], dg[(int64_t)col[e] * kFwdGroup], acc);
        const float o8 = __shfl_xor_sync(0xffffffffu, acc, 8);
        const float s01 = (ph & 1) ? o8 + acc : acc + o8;  // (p0 + p1) on phases 0/1, (p2 + p3) on 2/3
        const float o16 = __shfl_xor_sync(0xffffffffu, s01, 16);
        const float tot = (ph & 2) ? o16 + s01 : s01 + o16;
        if (ph == 0 && q < nq) {
            const float c = tot * inv_norm[d];
            out[(int64_t)q * ldo + d] = as_dist ? fmaxf(1.f - c, 0.f) : c;
        }
    }
}

// Inverse L2 norms of the documents' weights (0 for an empty document): one warp each.
__global__ void k_doc_inv_norm(const int32_t* __restrict__ row_ptr, const float* __restrict__ val, int64_t n,
                               float* __restrict__ inv_norm)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        float acc = 0.f;
        for (int32_t e = row_ptr[d] + lane; e < row_ptr[d + 1]; e += 32) acc = fmaf(val[e], val[e], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) inv_norm[d] = acc > 0.f ? 1.f / sqrtf(acc) : 0.f;
    }
}

__global__ void k_vslot(const int32_t* __restrict__ used_ids, int64_t v_used, int32_t* __restrict__ vslot)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < v_used; u += (int64_t)gridDim.x * blockDim.x)
        vslot[used_ids[u]] = (int32_t)u;
}

// Centroid of each document: sum_e val[e] * E[col[e]] / sum_e val[e], one warp per document,
// lanes over the dimensions, compensated accumulation; zero padding up to ldc.
__global__ void k_doc_centroids(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ val, int64_t n, const float* __restrict__ E, int lde, int m,
                                float* __restrict__ C, int ldc)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float ws = 0.f, wc = 0.f;
        for (int32_t e = a; e < b; ++e) {
            float t, te;
            two_sum(ws, val[e], t, te);
            ws = t;
            wc += te;
        }
        const float wsum = ws + wc;
        for (int i0 = 0; i0 < ldc; i0 += 32) {
            const int i = i0 + lane;
            float s = 0.f, c = 0.f;
            if (i < m)
                for (int32_t e = a; e < b; ++e) dot2_step(val[e], E[(int64_t)col[e] * lde + i], s, c);
            C[d * ldc + i] = (i < m && wsum > 0.f) ? (s + c) / wsum : 0.f;
        }
    }
}

// Centroid of each query of a batch (rp relative offsets into idx / w).  Block (query,
// 32-dimension chunk), 8 warps: warp w accumulates bins w, w + 8, ... (compensated, lane =
// dimension), then warp 0 adds the eight partial (sum, error) pairs in warp order.
__global__ void __launch_bounds__(256) k_query_centroids(const int64_t* __restrict__ rp, int nq,
                                                         const int32_t* __restrict__ idx, const float* __restrict__ w,
                                                         const float* __restrict__ E, int lde, int m,
                                                         float* __restrict__ C, int ldc)
{
    const int q = blockIdx.x;
    if (q >= nq) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int i = blockIdx.y * 32 + lane;
    const int64_t a = rp[q], b = rp[q + 1];
    __shared__ float ps[8][32], pc[8][32], ws_[8], wc_[8];
    float s = 0.f, c = 0.f, sw = 0.f, cw = 0.f;
    for (int64_t j = a + wp; j < b; j += 8) {
        const float wj = w[j];
        float t, te;
        two_sum(sw, wj, t, te);
        sw = t;
        cw += te;
        if (i < m) dot2_step(wj, E[(int64_t)idx[j] * lde + i], s, c);
    }
    ps[wp][lane] = s;
    pc[wp][lane] = c;
    if (lane == 0) { ws_[wp] = sw; wc_[wp] = cw; }
    __syncthreads();
    if (wp == 0) {
        float S = 0.f, Cc = 0.f, SW = 0.f, CW = 0.f;
        for (int v = 0; v < 8; ++v) {
            float t, te;
            two_sum(S, ps[v][lane], t, te);
            S = t;
            Cc += te + pc[v][lane];
            two_sum(SW, ws_[v], t, te);
            SW = t;
            CW += te + wc_[v];
        }
        const float wsum = SW + CW;
        if (i < ldc) C[(int64_t)q * ldc + i] = (i < m && wsum > 0.f) ? (S + Cc) / wsum : 0.f;
    }
}

// out[q * ldo + d] = sqrt(sum_i (Cd[d, i] - Cq[q, i])^2).  Block: 64 documents x 64
// queries, 256 threads of 4 documents (4tx..4tx+3) x 4 queries (4ty..4ty+3) read from shared
// memory as float4; dimension tiles of 16 loaded as float4 along the dimensions (rows padded
// to 68 floats: 2-way bank conflicts at most on the transposing stores).
constexpr int kWcdT = 64, kWcdK = 16, kWcdLd = kWcdT + 4;

__global__ void __launch_bounds__(256) k_wcd(const float* __restrict__ Cd, int64_t n, const float* __restrict__ Cq,
                                             int nq, int ldc, float* __restrict__ out, int64_t ldo)
{
    __shared__ __align__(16) float sd[kWcdK][kWcdLd];
    __shared__ __align__(16) float sq[kWcdK][kWcdLd];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int lr = tid >> 2, lk = 4 * (tid & 3);  // loader: row lr, dimensions lk..lk+3
    const int64_t d0 = (int64_t)blockIdx.x * kWcdT;
    const int q0 = blockIdx.y * kWcdT;
    const int64_t dl = d0 + lr;
    const int ql = q0 + lr;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < ldc; k0 += kWcdK) {
        const float4 va = dl < n ? *reinterpret_cast<const float4*>(Cd + dl * ldc + k0 + lk) : make_float4(0, 0, 0, 0);
        const float4 vb = ql < nq ? *reinterpret_cast<const float4*>(Cq + (int64_t)ql * ldc + k0 + lk)
                                  : make_float4(0, 0, 0, 0);
        sd[lk][lr] = va.x; sd[lk + 1][lr] = va.y; sd[lk + 2][lr] = va.z; sd[lk + 3][lr] = va.w;
        sq[lk][lr] = vb.x; sq[lk + 1][lr] = vb.y; sq[lk + 2][lr] = vb.z; sq[lk + 3][lr] = vb.w;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kWcdK; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(&sd[kk][4 * tx]);
            const float4 b4 = *reinterpret_cast<const float4*>(&sq[kk][4 * ty]);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w};
            const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float diff = a[r] - b[c];
                    acc[r][c] = fmaf(diff, diff, acc[r][c]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t d = d0 + 4 * tx + r;
            const int q = q0 + 4 * ty + c;
            if (d < n && q < nq) out[(int64_t)q * ldo + d] = sqrtf(acc[r][c]);
        }
}

}  // namespace

cudaError_t launch_bow_prep(const int64_t* rp, int nq, const int32_t* idx, const float* w, const int32_t* vslot,
                            float* dense, int64_t v_used, bool clear, cudaStream_t st)
{
    if (nq <= 0) return cudaSuccess;
    k_bow_prep<<<nq, 256, 0, st>>>(rp, nq, idx, w, vslot, dense, v_used, clear);
    return cudaGetLastError();
}

cudaError_t launch_bow_sweep(const int32_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                             const float* inv_norm, const float* dense, int64_t v_used, int nq, float* out,
                             int64_t ldo, bool as_dist, cudaStream_t st)
{
    if (nq <= 0 || n <= 0) return cudaSuccess;
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    const dim3 grid((unsigned)blocks, (unsigned)((nq + kFwdGroup - 1) / kFwdGroup));
    k_bow_sweep<<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, inv_norm, dense, v_used, nq, out, ldo, as_dist);
    return cudaGetLastError();
}

cudaError_t launch_doc_inv_norm(const int32_t* row_ptr, const float* val, int64_t n, float* inv_norm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    k_doc_inv_norm<<<(unsigned)blocks, warps * 32, 0, st>>>(row_ptr, val, n, inv_norm);
    return cudaGetLastError();
}

cudaError_t launch_vslot(const int32_t* used_ids, int64_t v_used, int64_t v, int32_t* vslot, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(vslot, 0xff, (size_t)v * sizeof(int32_t), st);  // -1
    if (e != cudaSuccess || v_used <= 0) return e;
    const int64_t blocks = std::min<int64_t>((v_used + 255) / 256, 152 * 8);
    k_vslot<<<(unsigned)blocks, 256, 0, st>>>(used_ids, v_used, vslot);
    return cudaGetLastError();
}

cudaError_t launch_doc_centroids(const int32_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                                 const float* E, int lde, int m, float* C, int ldc, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (ldc % 32 != 0 || ldc < m) return cudaErrorInvalidValue;
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    k_doc_centroids<<<(unsigned)blocks, warps * 32, 0, st>>>(row_ptr, col, val, n, E, lde, m, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_query_centroids(const int64_t* rp, int nq, const int32_t* idx, const float* w, const float* E,
                                   int lde, int m, float* C, int ldc, cudaStream_t st)
{
    if (nq <= 0) return cudaSuccess;
    if (ldc % 32 != 0 || ldc < m) return cudaErrorInvalidValue;
    k_query_centroids<<<dim3((unsigned)nq, (unsigned)(ldc / 32)), 256, 0, st>>>(rp, nq, idx, w, E, lde, m, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_wcd(const float* Cd, int64_t n, const float* Cq, int nq, int ldc, float* out, int64_t ldo,
                       cudaStream_t st)
{
    if (n <= 0 || nq <= 0) return cudaSuccess;
    if (ldc % kWcdK != 0) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((n + kWcdT - 1) / kWcdT), (unsigned)((nq + kWcdT - 1) / kWcdT));
    k_wcd<<<grid, 256, 0, st>>>(Cd, n, Cq, nq, ldc, out, ldo);
    return cudaGetLastError();
}

}  // namespace emd
