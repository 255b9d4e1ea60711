// Phase 1 of LC-ACT (Section 5): the distance matrix D between the used vocabulary and
// the query's coordinates, and the per-row top-k table (Z, S, W).
//
// This file holds the plain FP32 path: a register-tiled SIMT distance kernel (FP32 FFMA,
// norm expansion ||a||^2 + ||b||^2 - 2<a,b>), the cost-matrix gather of the image
// workloads, and the per-row top-k selection shared by every precision.
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

// ------------------------------------------------------------------ row gather + norms

__device__ __forceinline__ void gather_rows_body(const float* __restrict__ src, int64_t v, int ld, int m,
                              const int32_t* __restrict__ ids, int64_t nrows, int64_t nrows_pad,
                              float* __restrict__ dst, float* __restrict__ norm2, int* err)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= nrows_pad) return;
    float* out = dst + r * ld;
    int64_t id = -1;
    if (r < nrows) {
        id = ids[r];
        if (id < 0 || id >= v) {
            if (lane == 0) atomicOr(err, ERR_BAD_INDEX);
            id = -1;
        }
    }
    float s = 0.f;
    for (int c = lane; c < ld; c += 32) {
        float x = (id >= 0 && c < m) ? src[id * ld + c] : 0.f;
        out[c] = x;
        s = fmaf(x, x, s);
    }
    s = warp_sum(s);
    if (lane == 0) norm2[r] = s;
}

__global__ void k_gather_rows(const float* __restrict__ src, int64_t v, int ld, int m,
                              const int32_t* __restrict__ ids, int64_t nrows, int64_t nrows_pad,
                              float* __restrict__ dst, float* __restrict__ norm2, int* err)
{
    gather_rows_body(src, v, ld, m, ids, nrows, nrows_pad, dst, norm2, err);
}

// ------------------------------------------------------------------ FP32 distance tile
//
// Block tile 128 (vocabulary rows) x 64 (query columns), K step 16, 128 threads, each
// thread an 8 x 8 register tile (rows tr*4+{0..3} and 64+tr*4+{0..3}, columns tc*4+{0..3}
// and 32+tc*4+{0..3}).  Both operands are staged k-major in shared memory (double
// buffered, one barrier per K step) so that the inner loop is 4 LDS.128 + 64 FFMA.
// Operand rows are zero-padded to a multiple of 4 floats, so the K tail reads zeros.

__device__ __forceinline__ void dist_fp32_body(const float* __restrict__ A, int64_t M, int lda, const float* __restrict__ anorm,
            const int32_t* __restrict__ a_ids, const float* __restrict__ B, int N, int ldb,
            const float* __restrict__ bnorm, const int32_t* __restrict__ b_ids, int K,
            float* __restrict__ D, int ldd)
{
    constexpr int BM = kDistBM, BN = kDistBN, BK = kDistBK;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int tr = tid >> 3, tc = tid & 7;

    // loader mapping: A row tid (16 floats); B row tid>>1, half (tid&1)
    const int64_t arow = m0 + tid;
    const bool a_ok = arow < M;
    const float* Ap = A + (a_ok ? arow : 0) * lda;
    const int brow = n0 + (tid >> 1);
    const int bk = (tid & 1) * 8;
    const float* Bp = B + (int64_t)brow * ldb;

    float4 ra[4], rb[2];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk = k0 + q * 4;
            ra[q] = (a_ok && kk < lda) ? *reinterpret_cast<const float4*>(Ap + kk)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int kk = k0 + bk + q * 4;
            rb[q] = (kk < ldb) ? *reinterpret_cast<const float4*>(Bp + kk)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            As[buf][q * 4 + 0][tid] = ra[q].x;
            As[buf][q * 4 + 1][tid] = ra[q].y;
            As[buf][q * 4 + 2][tid] = ra[q].z;
            As[buf][q * 4 + 3][tid] = ra[q].w;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            Bs[buf][bk + q * 4 + 0][tid >> 1] = rb[q].x;
            Bs[buf][bk + q * 4 + 1][tid >> 1] = rb[q].y;
            Bs[buf][bk + q * 4 + 2][tid >> 1] = rb[q].z;
            Bs[buf][bk + q * 4 + 3][tid >> 1] = rb[q].w;
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int Kpad = (int)round_up(K, BK);
    load(0);
    store(0);
    __syncthreads();
    for (int k0 = 0; k0 < Kpad; k0 += BK) {
        const int buf = (k0 / BK) & 1;
        const bool more = k0 + BK < Kpad;
        if (more) load(k0 + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][tr * 4]);
            float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + tr * 4]);
            float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tc * 4]);
            float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][32 + tc * 4]);
            float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
    }

    // epilogue: the squared distance |a|^2 + |b|^2 - 2<a,b> (unclamped); identical ids give exactly 0
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = m0 + (i < 4 ? tr * 4 + i : 64 + tr * 4 + (i - 4));
        if (row >= M) continue;
        const float an = anorm[row];
        const int32_t aid = a_ids[row];
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
            const int col0 = n0 + jh * 32 + tc * 4;
            if (col0 >= ldd) continue;
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = col0 + e;
                float d = INFINITY;
                if (col < N) {
                    const float d2 = fmaf(-2.f, acc[i][jh * 4 + e], an + bnorm[col]);
                    d = (aid == b_ids[col]) ? 0.f : d2;
                }
                o[e] = d;
            }
            *reinterpret_cast<float4*>(D + row * ldd + col0) = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

__global__ void __launch_bounds__(128) k_dist_fp32(const float* __restrict__ A, int64_t M, int lda, const float* __restrict__ anorm,
            const int32_t* __restrict__ a_ids, const float* __restrict__ B, int N, int ldb,
            const float* __restrict__ bnorm, const int32_t* __restrict__ b_ids, int K,
            float* __restrict__ D, int ldd)
{
    dist_fp32_body(A, M, lda, anorm, a_ids, B, N, ldb, bnorm, b_ids, K, D, ldd);
}

// ------------------------------------------------------------------ cost-matrix gather

__device__ __forceinline__ void dist_gather_body(const float* __restrict__ cost, int64_t v,
                              const int32_t* __restrict__ a_ids, int64_t M,
                              const int32_t* __restrict__ b_ids, int N, float* __restrict__ D,
                              int ldd, int* err)
{
    const int64_t u = blockIdx.x;
    if (u >= M) return;
    const int64_t a = a_ids[u];
    for (int j = threadIdx.x; j < ldd; j += blockDim.x) {
        float d = INFINITY;
        if (j < N) {
            const int64_t b = b_ids[j];
            if (b < 0 || b >= v || a < 0 || a >= v) {
                atomicOr(err, ERR_BAD_INDEX);
                d = 0.f;
            } else {
                d = cost[a * v + b];
            }
        }
        D[u * ldd + j] = d;
    }
}

__global__ void k_dist_gather(const float* __restrict__ cost, int64_t v,
                              const int32_t* __restrict__ a_ids, int64_t M,
                              const int32_t* __restrict__ b_ids, int N, float* __restrict__ D,
                              int ldd, int* err)
{
    dist_gather_body(cost, v, a_ids, M, b_ids, N, D, ldd, err);
}

// ------------------------------------------------------------------ top-k table
//
// One thread per vocabulary row: the row of D is read with 16-byte loads in column order
// and kept in a branch-free sorted register list of the KT smallest (d, j); strict '<'
// keeps the earlier column first on equal d, the order the definition uses.

template <int KCT>
__device__ __forceinline__ void insert_dj_tie(float (&z)[KCT], int (&s)[KCT], float d, int j)
{
    bool p[KCT];
#pragma unroll
    for (int l = 0; l < KCT; ++l) p[l] = d < z[l] || (d == z[l] && j < s[l]);
#pragma unroll
    for (int l = KCT - 1; l > 0; --l) {
        z[l] = p[l - 1] ? z[l - 1] : (p[l] ? d : z[l]);
        s[l] = p[l - 1] ? s[l - 1] : (p[l] ? j : s[l]);
    }
    z[0] = p[0] ? d : z[0];
    s[0] = p[0] ? j : s[0];
}

template <int KT>
__device__ __forceinline__ void insert_dj(float (&z)[KT], int (&s)[KT], float d, int j)
{
    bool p[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) p[l] = d < z[l];
#pragma unroll
    for (int l = KT - 1; l > 0; --l) {
        z[l] = p[l - 1] ? z[l - 1] : (p[l] ? d : z[l]);
        s[l] = p[l - 1] ? s[l - 1] : (p[l] ? j : s[l]);
    }
    z[0] = p[0] ? d : z[0];
    s[0] = p[0] ? j : s[0];
}

template <int KT>
__device__ __forceinline__ void table_body(const float* __restrict__ D, int ldd, int64_t M, int h, int k, const float* __restrict__ q_w,
        float2* __restrict__ tab, int32_t* __restrict__ tab_s, int rs, int es, bool sq)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= M) return;
    const float* Dr = D + row * ldd;
    // two independent lists (columns 8i..8i+3 and 8i+4..8i+7, ldd % 32 == 0 so both loads
    // stay in the row) for instruction-level parallelism, merged by (value, column)
    float z[KT], zb[KT];
    int s[KT], sb[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) { z[l] = zb[l] = INFINITY; s[l] = sb[l] = INT32_MAX; }
    for (int j = 0; j < h; j += 8) {
        const float4 v = *reinterpret_cast<const float4*>(Dr + j);
        const float4 w = *reinterpret_cast<const float4*>(Dr + j + 4);
        insert_dj<KT>(z, s, v.x, j);
        if (j + 4 < h) insert_dj<KT>(zb, sb, w.x, j + 4);
        if (j + 1 < h) insert_dj<KT>(z, s, v.y, j + 1);
        if (j + 5 < h) insert_dj<KT>(zb, sb, w.y, j + 5);
        if (j + 2 < h) insert_dj<KT>(z, s, v.z, j + 2);
        if (j + 6 < h) insert_dj<KT>(zb, sb, w.z, j + 6);
        if (j + 3 < h) insert_dj<KT>(z, s, v.w, j + 3);
        if (j + 7 < h) insert_dj<KT>(zb, sb, w.w, j + 7);
    }
#pragma unroll
    for (int l = 0; l < KT; ++l)
        if (sb[l] != INT32_MAX) insert_dj_tie<KT>(z, s, zb[l], sb[l]);
#pragma unroll
    for (int l = 0; l < KT; ++l) {
        if (l < k) {
            const bool valid = s[l] != INT32_MAX;
            tab[row * rs + l * es] = make_float2(valid ? d_value(z[l], sq) : INFINITY, valid ? q_w[s[l]] : 0.f);
            if (tab_s) tab_s[row * k + l] = valid ? s[l] : -1;
        }
    }
}

template <int KT>
__global__ void __launch_bounds__(128) k_table(const float* __restrict__ D, int ldd, int64_t M, int h, int k, const float* __restrict__ q_w,
        float2* __restrict__ tab, int32_t* __restrict__ tab_s, bool sq)
{
    table_body<KT>(D, ldd, M, h, k, q_w, tab, tab_s, k, 1, sq);
}

// k larger than the register lists: successive minima, each strictly after the previous
// in (d, j) order.  O(k * h / 32) per lane; used for ICT on small queries.
__device__ __forceinline__ void table_generic_body(const float* __restrict__ D, int ldd, int64_t M, int h, int k,
                                const float* __restrict__ q_w, float2* __restrict__ tab,
                                int32_t* __restrict__ tab_s, int rs, int es, bool sq)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    const float* Dr = D + row * ldd;
    float pz = -INFINITY;
    int ps = -1;
    for (int l = 0; l < k; ++l) {
        float bz = INFINITY;
        int bs = INT32_MAX;
        for (int j = lane; j < h; j += 32) {
            float d = Dr[j];
            bool after = d > pz || (d == pz && j > ps);
            if (after && (d < bz || (d == bz && j < bs))) { bz = d; bs = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float oz = __shfl_xor_sync(0xffffffffu, bz, o);
            int os = __shfl_xor_sync(0xffffffffu, bs, o);
            if (oz < bz || (oz == bz && os < bs)) { bz = oz; bs = os; }
        }
        if (lane == 0) {
            const bool valid = bs != INT32_MAX;
            tab[row * rs + l * es] = make_float2(valid ? d_value(bz, sq) : INFINITY, valid ? q_w[bs] : 0.f);
            if (tab_s) tab_s[row * k + l] = valid ? bs : -1;
        }
        pz = bz;
        ps = bs;
    }
}

// One warp per vocabulary row.  Each step finds the next smallest (distance, column) after
// the previous one (lane-strided scan, shuffle reduction), writes it and moves
// min(residual, weight) of xmax[row] -- the steps of the forward cost, so for every database
// weight x <= xmax[row] the forward walk along this row ends (residual 0) within the
// entries written (fl(r - min(r, w)) is non-decreasing in r).
__device__ __forceinline__ void table_ict_body(const float* __restrict__ D, int ldd, int64_t M, int h, int W,
                                               const float* __restrict__ q_w, const float* __restrict__ xmax,
                                               float2* __restrict__ tab, int32_t* __restrict__ tab_s, int rs,
                                               int es, int* __restrict__ over, bool sq)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    if (tab[row * rs].y >= 0.f) return;  // finished by the register pass (ict_fast_body)
    const float* Dr = D + row * ldd;
    const int lim = min(W, h);
    float r = xmax[row];
    float pz = -INFINITY;
    int ps = -1, l = 0;
    do {
        float bz = INFINITY;
        int bs = INT32_MAX;
        for (int j = lane; j < h; j += 32) {
            const float d = Dr[j];
            const bool after = d > pz || (d == pz && j > ps);
            if (after && (d < bz || (d == bz && j < bs))) { bz = d; bs = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oz = __shfl_xor_sync(0xffffffffu, bz, o);
            const int os = __shfl_xor_sync(0xffffffffu, bs, o);
            if (oz < bz || (oz == bz && os < bs)) { bz = oz; bs = os; }
        }
        const bool valid = bs != INT32_MAX;  // always while l < h, unless D holds NaN
        const float w = valid ? q_w[bs] : 0.f;
        if (lane == 0) {
            tab[row * rs + (int64_t)l * es] = make_float2(valid ? d_value(bz, sq) : INFINITY, w);
            if (tab_s) tab_s[row * W + l] = valid ? bs : -1;
        }
        if (!valid) break;
        r -= fminf(r, w);
        pz = bz;
        ps = bs;
        ++l;
    } while (r != 0.f && l < lim);
    if (r != 0.f && lim < h && lane == 0 && over) *over = 1;
}

// Register pass of the ICT table, one thread per row: the row's kIctFast smallest (d, j) in
// ascending order (strict '<' over ascending j), then the same residual steps as
// table_ict_body.  A row whose residual reaches 0 within them -- or that has no more
// entries to take -- is written here in full; any other row gets entry 0 = (NaN, -1), and
// table_ict_body, which skips rows with a nonnegative entry-0 weight, computes it.  Both
// write identical entries for a row.
constexpr int kIctFast = 8;

__device__ __forceinline__ void ict_fast_body(const float* __restrict__ D, int ldd, int64_t M, int h, int W,
                                              const float* __restrict__ q_w, const float* __restrict__ xmax,
                                              float2* __restrict__ tab, int32_t* __restrict__ tab_s, int rs, int es,
                                              int* __restrict__ over, bool sq)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= M) return;
    const float* Dr = D + row * ldd;
    // two independent lists (columns 8i..8i+3 and 8i+4..8i+7; ldd % 32 == 0 keeps both loads
    // in the row), merged by (value, column)
    float z[kIctFast], zb[kIctFast];
    int s[kIctFast], sb[kIctFast];
#pragma unroll
    for (int l = 0; l < kIctFast; ++l) { z[l] = zb[l] = INFINITY; s[l] = sb[l] = INT32_MAX; }
    for (int j = 0; j < h; j += 8) {
        const float4 v = *reinterpret_cast<const float4*>(Dr + j);
        const float4 w = *reinterpret_cast<const float4*>(Dr + j + 4);
        insert_dj<kIctFast>(z, s, v.x, j);
        if (j + 4 < h) insert_dj<kIctFast>(zb, sb, w.x, j + 4);
        if (j + 1 < h) insert_dj<kIctFast>(z, s, v.y, j + 1);
        if (j + 5 < h) insert_dj<kIctFast>(zb, sb, w.y, j + 5);
        if (j + 2 < h) insert_dj<kIctFast>(z, s, v.z, j + 2);
        if (j + 6 < h) insert_dj<kIctFast>(zb, sb, w.z, j + 6);
        if (j + 3 < h) insert_dj<kIctFast>(z, s, v.w, j + 3);
        if (j + 7 < h) insert_dj<kIctFast>(zb, sb, w.w, j + 7);
    }
#pragma unroll
    for (int l = 0; l < kIctFast; ++l)
        if (sb[l] != INT32_MAX) insert_dj_tie<kIctFast>(z, s, zb[l], sb[l]);
    const int lim = min(W, h), lf = min(lim, kIctFast);
    float r = xmax[row];
    int L = 0;
    bool go = true;  // the first entry is always taken; then while mass remains
#pragma unroll
    for (int l = 0; l < kIctFast; ++l) {
        if (l < lf && go) {
            const bool valid = s[l] != INT32_MAX;  // false only where D held NaN
            L = l + 1;
            if (valid) {
                r -= fminf(r, q_w[s[l]]);
                go = r != 0.f;
            } else {
                go = false;
            }
        }
    }
    if (r != 0.f && lf < lim) {  // needs more than kIctFast entries: the warp pass
        tab[row * rs] = make_float2(__int_as_float(0x7fc00000), -1.f);
        return;
    }
    if (r != 0.f && lim < h && over) *over = 1;  // more than W entries needed
#pragma unroll
    for (int l = 0; l < kIctFast; ++l) {
        if (l < L) {
            const bool valid = s[l] != INT32_MAX;
            tab[row * rs + (int64_t)l * es] = make_float2(valid ? d_value(z[l], sq) : INFINITY, valid ? q_w[s[l]] : 0.f);
            if (tab_s) tab_s[row * W + l] = valid ? s[l] : -1;
        }
    }
}

__global__ void __launch_bounds__(128) k_table_ict_fast(const float* __restrict__ D, int ldd, int64_t M, int h, int W,
                                 const float* __restrict__ q_w, const float* __restrict__ xmax,
                                 float2* __restrict__ tab, int32_t* __restrict__ tab_s, int* __restrict__ over, bool sq)
{
    ict_fast_body(D, ldd, M, h, W, q_w, xmax, tab, tab_s, W, 1, over, sq);
}

__global__ void k_table_ict(const float* __restrict__ D, int ldd, int64_t M, int h, int W,
                            const float* __restrict__ q_w, const float* __restrict__ xmax, float2* __restrict__ tab,
                            int32_t* __restrict__ tab_s, int* __restrict__ over, bool sq)
{
    table_ict_body(D, ldd, M, h, W, q_w, xmax, tab, tab_s, W, 1, over, sq);
}

__global__ void k_table_generic(const float* __restrict__ D, int ldd, int64_t M, int h, int k,
                                const float* __restrict__ q_w, float2* __restrict__ tab,
                                int32_t* __restrict__ tab_s, bool sq)
{
    table_generic_body(D, ldd, M, h, k, q_w, tab, tab_s, k, 1, sq);
}

// Re-rank form of the table, for approximate distance matrices (BF16 / E4M3 Phase 1).
// Per vocabulary row u: the kc smallest approximate D[u, .] (squared distances; ties: lower
// j) are the candidates; their squared distances are recomputed exactly in FP32 as
// sum_i (V_u,i - Q_j,i)^2 -- differences, not the norm expansion -- and written back into D;
// the k smallest exact values (ties: lower j) form the table, with z = their square roots.  Selection runs one thread per
// row, the recomputation one warp per row (lanes over float4 slices of the embedding;
// rows are zero beyond m, so the padded width adds nothing).

// Block: kRrRows rows, one thread each.  Selection as in table_body (each thread scans its
// own row, four entries per load).  Exact sums: over the embedding in chunks of kRrDims (4)
// dimensions, the chunk of every query row staged in shared memory once per block, each
// thread holding its own row's chunk in registers and adding the squared differences to
// each of its kc candidates (sequential over the dimensions).  Then the k smallest exact
// sums (ties: lower j) are selected and the exact squared distances written back into D.
// Dynamic shared memory: rerank_smem_bytes(h).
constexpr int kRrRows = 256, kRrDims = 4;

__host__ __device__ constexpr size_t rerank_smem_bytes(int h) { return (size_t)h * kRrDims * 4; }

template <int KCT>
__device__ __forceinline__ void table_rerank_body(float* __restrict__ D, int ldd, int64_t M, int h, int k, int kc, const float* __restrict__ V,
               const float* __restrict__ Q, int ldv, const float* __restrict__ q_w, float2* __restrict__ tab,
               int32_t* __restrict__ tab_s, int64_t tile, int rs, int es)
{
    extern __shared__ float4 qs4[];  // [h]: Q[j][d0 .. d0 + 4)
    const int tid = threadIdx.x;
    const int64_t row = tile * kRrRows + tid;
    const bool rok = row < M;
    int s[KCT];
    {
        float z[KCT];
#pragma unroll
        for (int l = 0; l < KCT; ++l) { z[l] = INFINITY; s[l] = INT32_MAX; }
        if (rok) {
            const float* Dr = D + row * ldd;
            for (int j = 0; j < h; j += 4) {
                const float4 v = *reinterpret_cast<const float4*>(Dr + j);
                insert_dj<KCT>(z, s, v.x, j);
                if (j + 1 < h) insert_dj<KCT>(z, s, v.y, j + 1);
                if (j + 2 < h) insert_dj<KCT>(z, s, v.z, j + 2);
                if (j + 3 < h) insert_dj<KCT>(z, s, v.w, j + 3);
            }
        }
    }
    float acc[KCT];
#pragma unroll
    for (int l = 0; l < KCT; ++l) acc[l] = 0.f;
    for (int d0 = 0; d0 < ldv; d0 += kRrDims) {  // ldv % 4 == 0
        __syncthreads();  // the previous chunk's readers are done
        for (int j = tid; j < h; j += blockDim.x)
            qs4[j] = *reinterpret_cast<const float4*>(Q + (int64_t)j * ldv + d0);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rok) v = *reinterpret_cast<const float4*>(V + row * ldv + d0);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < KCT; ++c) {
            if (c < kc && s[c] != INT32_MAX) {
                const float4 a = qs4[s[c]];
                float t = v.x - a.x;
                acc[c] = fmaf(t, t, acc[c]);
                t = v.y - a.y;
                acc[c] = fmaf(t, t, acc[c]);
                t = v.z - a.z;
                acc[c] = fmaf(t, t, acc[c]);
                t = v.w - a.w;
                acc[c] = fmaf(t, t, acc[c]);
            }
        }
    }
    if (!rok) return;
    float z[KCT];
    int s2[KCT];
#pragma unroll
    for (int l = 0; l < KCT; ++l) { z[l] = INFINITY; s2[l] = INT32_MAX; }
#pragma unroll
    for (int c = 0; c < KCT; ++c) {
        if (c < kc && s[c] != INT32_MAX) {
            D[row * ldd + s[c]] = acc[c];
            insert_dj_tie<KCT>(z, s2, acc[c], s[c]);
        }
    }
#pragma unroll
    for (int l = 0; l < KCT; ++l) {
        if (l < k) {
            const bool valid = s2[l] != INT32_MAX;
            tab[row * rs + l * es] = make_float2(valid ? sq_to_dist(z[l]) : INFINITY, valid ? q_w[s2[l]] : 0.f);
            if (tab_s) tab_s[row * k + l] = valid ? s2[l] : -1;
        }
    }
}

template <int KCT>
__global__ void __launch_bounds__(kRrRows) k_table_rerank(float* __restrict__ D, int ldd, int64_t M, int h, int k, int kc, const float* __restrict__ V,
               const float* __restrict__ Q, int ldv, const float* __restrict__ q_w, float2* __restrict__ tab,
               int32_t* __restrict__ tab_s)
{
    table_rerank_body<KCT>(D, ldd, M, h, k, kc, V, Q, ldv, q_w, tab, tab_s, blockIdx.x, k, 1);
}

// ------------------------------------------------------------------ batched forms

__global__ void k_gather_rows_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const float* __restrict__ src,
                                int64_t v, int ld, int m, int* err)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    gather_rows_body(src, v, ld, m, d.qidx, d.h, d.qrows, d.Q, d.qnorm, err);
}

__global__ void __launch_bounds__(128)
k_dist_fp32_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const float* __restrict__ A, int64_t M,
              int lda, const float* __restrict__ anorm, const int32_t* __restrict__ a_ids, int K)
{
    if ((int)blockIdx.z >= *nq) return;
    const QDesc& d = qd[blockIdx.z];
    if ((int)blockIdx.y * kDistBN >= d.ldd) return;
    dist_fp32_body(A, M, lda, anorm, a_ids, d.Q, d.h, lda, d.qnorm, d.qidx, K, d.D, d.ldd);
}

__global__ void k_dist_gather_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const float* __restrict__ cost,
                                int64_t v, const int32_t* __restrict__ a_ids, int64_t M, int* err)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    dist_gather_body(cost, v, a_ids, M, d.qidx, d.h, d.D, d.ldd, err);
}

template <int KT>
__global__ void __launch_bounds__(128)
k_table_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t M)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    table_body<KT>(d.D, d.ldd, M, d.h, d.tk, d.qw, d.tab, nullptr, d.tab_rs, d.tab_es, d.sq != 0);
}

// D[vslot[q_idx[j]], j] = 0 for the query bins whose id is a used vocabulary row (ids
// outside 0..v-1 are skipped; the query gather latches them as errors).
__device__ __forceinline__ void zero_ident_body(const int32_t* __restrict__ q_idx, int h,
                                                const int32_t* __restrict__ vslot, int64_t v, float* __restrict__ D,
                                                int ldd)
{
    for (int j = threadIdx.x; j < h; j += blockDim.x) {
        const int32_t id = q_idx[j];
        const int32_t s = (id >= 0 && id < v) ? vslot[id] : -1;
        if (s >= 0) D[(int64_t)s * ldd + j] = 0.f;
    }
}

__global__ void k_zero_ident(const int32_t* __restrict__ q_idx, int h, const int32_t* __restrict__ vslot, int64_t v,
                             float* __restrict__ D, int ldd)
{
    zero_ident_body(q_idx, h, vslot, v, D, ldd);
}

__global__ void k_zero_ident_b(const QDesc* __restrict__ qd, const int* __restrict__ nq,
                               const int32_t* __restrict__ vslot, int64_t v)
{
    if ((int)blockIdx.x >= *nq) return;
    const QDesc& d = qd[blockIdx.x];
    zero_ident_body(d.qidx, d.h, vslot, v, d.D, d.ldd);
}

// The fused path's map from used row to query bin: qpos[vslot[q_idx[j]]] = j (set) or -1
// (clear, restoring the state every batch starts from).
__global__ void k_qpos_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ vslot,
                         int64_t v, bool set)
{
    if ((int)blockIdx.x >= *nq) return;
    const QDesc& d = qd[blockIdx.x];
    for (int j = threadIdx.x; j < d.h; j += blockDim.x) {
        const int32_t id = d.qidx[j];
        const int32_t s = (id >= 0 && id < v) ? vslot[id] : -1;
        if (s >= 0) d.qpos[s] = set ? j : -1;
    }
}

__global__ void __launch_bounds__(128) k_table_ict_fast_b(const QDesc* __restrict__ qd, const int* __restrict__ nq,
                                                          int64_t M, const float* __restrict__ xmax)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    ict_fast_body(d.D, d.ldd, M, d.h, d.tk, d.qw, xmax, d.tab, nullptr, d.tab_rs, d.tab_es, d.over, d.sq != 0);
}

__global__ void k_table_ict_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t M,
                              const float* __restrict__ xmax)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    table_ict_body(d.D, d.ldd, M, d.h, d.tk, d.qw, xmax, d.tab, nullptr, d.tab_rs, d.tab_es, d.over, d.sq != 0);
}

__global__ void k_table_generic_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t M)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    table_generic_body(d.D, d.ldd, M, d.h, d.tk, d.qw, d.tab, nullptr, d.tab_rs, d.tab_es, d.sq != 0);
}

// Queries vary fastest (blockIdx.x) so that the blocks of one vocabulary tile for all
// queries of the batch run together and its FP32 rows are read from HBM once.
template <int KCT>
__global__ void __launch_bounds__(kRrRows)
k_table_rerank_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t M, const float* __restrict__ V,
                 int ldv)
{
    if ((int)blockIdx.x >= *nq) return;
    const QDesc& d = qd[blockIdx.x];
    table_rerank_body<KCT>(d.D, d.ldd, M, d.h, d.tk, d.kc, V, d.Q, ldv, d.qw, d.tab, nullptr, blockIdx.y, d.tab_rs,
                           d.tab_es);
}

// Fused approximate forms: the re-rank from the candidate bins the product's epilogue kept
// (qd[q].cbin, kc per row) instead of a scan of the distance matrix; exact sums as in
// table_rerank_body (same dimension order, so the same values), k smallest by (value, bin).
// Certificate (BF16): every bin outside the candidates has an approximate squared distance of
// at least camax (the kc-th smallest), hence an exact one of at least camax - eps; when that
// exceeds the k-th exact value (with its own FP32 rounding allowed for) the row is exact.
// Uncertified rows are listed for k_rerank_full_b.  Block: kRrRows rows of one query.
template <int KCT>
__global__ void __launch_bounds__(kRrRows)
k_rerank_cand_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t M, const float* __restrict__ V,
                int ldv, const float* __restrict__ vnorm, bool certify, float eps_rel, float eps_abs)
{
    if ((int)blockIdx.x >= *nq) return;
    const QDesc& d = qd[blockIdx.x];
    extern __shared__ float4 qs4[];  // [h]: Q[j][d0 .. d0 + 4)
    __shared__ float wmax[kRrRows / 32];
    const int tid = threadIdx.x;
    const int64_t row = (int64_t)blockIdx.y * kRrRows + tid;
    const bool rok = row < M;
    const int h = d.h, k = d.tk, kc = d.kc;
    float qmax = 0.f;  // largest squared norm of the query's bins
    if (certify) {
        float qm = 0.f;
        for (int j = tid; j < h; j += blockDim.x) qm = fmaxf(qm, d.qnorm[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qm = fmaxf(qm, __shfl_xor_sync(0xffffffffu, qm, o));
        if ((tid & 31) == 0) wmax[tid >> 5] = qm;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kRrRows / 32; ++w) qmax = fmaxf(qmax, wmax[w]);
    }
    int s[KCT];
#pragma unroll
    for (int c = 0; c < KCT; ++c) s[c] = (rok && c < kc) ? d.cbin[row * kCandPerRow + c] : INT32_MAX;
    float acc[KCT];
#pragma unroll
    for (int c = 0; c < KCT; ++c) acc[c] = 0.f;
    for (int d0 = 0; d0 < ldv; d0 += kRrDims) {
        __syncthreads();
        for (int j = tid; j < h; j += blockDim.x) qs4[j] = *reinterpret_cast<const float4*>(d.Q + (int64_t)j * ldv + d0);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rok) v = *reinterpret_cast<const float4*>(V + row * ldv + d0);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < KCT; ++c) {
            if (s[c] != INT32_MAX) {
                const float4 a = qs4[s[c]];
                float t = v.x - a.x;
                acc[c] = fmaf(t, t, acc[c]);
                t = v.y - a.y;
                acc[c] = fmaf(t, t, acc[c]);
                t = v.z - a.z;
                acc[c] = fmaf(t, t, acc[c]);
                t = v.w - a.w;
                acc[c] = fmaf(t, t, acc[c]);
            }
        }
    }
    if (!rok) return;
    float z[KCT];
    int s2[KCT];
#pragma unroll
    for (int l = 0; l < KCT; ++l) { z[l] = INFINITY; s2[l] = INT32_MAX; }
#pragma unroll
    for (int c = 0; c < KCT; ++c)
        if (s[c] != INT32_MAX) insert_dj_tie<KCT>(z, s2, acc[c], s[c]);
    float ek = INFINITY;
#pragma unroll
    for (int l = 0; l < KCT; ++l) {
        if (l < k) {
            const bool valid = s2[l] != INT32_MAX;
            d.tab[row * d.tab_rs + l * d.tab_es] = make_float2(valid ? sq_to_dist(z[l]) : INFINITY, valid ? d.qw[s2[l]] : 0.f);
        }
        if (l == k - 1) ek = z[l];
    }
    if (certify) {
        const float nv = vnorm[row];
        const float eps = eps_rel * sqrtf(nv * qmax) + eps_abs * (nv + qmax);
        if (!(d.camax[row] - eps > ek * (1.0f + 4e-5f))) {
            const int idx = atomicAdd(d.rr_count, 1);
            d.rr[idx] = (int32_t)row;
        }
    }
}

// Exact table rows over all bins for the rows the certificate left out: a warp per row,
// each lane the exact squared distances (sums as above) of bins lane, lane + 32, ... kept as
// its KT smallest (bins ascending per lane, so ties keep the lower bin), then k successive
// minima across the warp by (value, bin).
template <int KT>
__global__ void __launch_bounds__(256)
k_rerank_full_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const float* __restrict__ V, int ldv)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    const int cnt = *d.rr_count;
    const int lane = threadIdx.x & 31;
    const int nw = (int)(gridDim.x * (blockDim.x >> 5));
    for (int t = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); t < cnt; t += nw) {
        const int64_t row = d.rr[t];
        const float* vr = V + row * ldv;
        float z[KT];
        int s[KT];
#pragma unroll
        for (int l = 0; l < KT; ++l) { z[l] = INFINITY; s[l] = INT32_MAX; }
        for (int j = lane; j < d.h; j += 32) {
            const float* qr = d.Q + (int64_t)j * ldv;
            float acc = 0.f;
            for (int d0 = 0; d0 < ldv; d0 += 4) {
                const float4 v = *reinterpret_cast<const float4*>(vr + d0);
                const float4 a = *reinterpret_cast<const float4*>(qr + d0);
                float e = v.x - a.x;
                acc = fmaf(e, e, acc);
                e = v.y - a.y;
                acc = fmaf(e, e, acc);
                e = v.z - a.z;
                acc = fmaf(e, e, acc);
                e = v.w - a.w;
                acc = fmaf(e, e, acc);
            }
            if (acc < z[KT - 1]) insert_dj<KT>(z, s, acc, j);
        }
        for (int l = 0; l < d.tk; ++l) {
            float bz = z[0];
            int bs = s[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oz = __shfl_xor_sync(0xffffffffu, bz, o);
                const int os = __shfl_xor_sync(0xffffffffu, bs, o);
                if (oz < bz || (oz == bz && os < bs)) { bz = oz; bs = os; }
            }
            if (lane == 0) {
                const bool valid = bs != INT32_MAX;
                d.tab[row * d.tab_rs + l * d.tab_es] = make_float2(valid ? sq_to_dist(bz) : INFINITY, valid ? d.qw[bs] : 0.f);
            }
            if (s[0] == bs && bs != INT32_MAX) {  // the owner pops its head
#pragma unroll
                for (int q = 0; q < KT - 1; ++q) { z[q] = z[q + 1]; s[q] = s[q + 1]; }
                z[KT - 1] = INFINITY;
                s[KT - 1] = INT32_MAX;
            }
        }
    }
}

// Opt-in dynamic shared memory of the re-rank kernels (above 48 KB for long queries).
cudaError_t rerank_smem_attr(size_t smem)
{
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int b = (int)std::max<size_t>(smem, 1);
    cudaError_t e = cudaFuncSetAttribute(k_table_rerank<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank_b<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank_b<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank_b<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_table_rerank_b<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rerank_cand_b<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

}  // namespace

cudaError_t launch_gather_rows(const float* src, int64_t v, int ld, int m, const int32_t* ids,
                               int64_t nrows, int64_t nrows_pad, float* dst, float* norm2,
                               int* err, cudaStream_t st)
{
    if (nrows_pad <= 0) return cudaSuccess;
    const int warps = 8;
    dim3 grid((unsigned)((nrows_pad + warps - 1) / warps));
    k_gather_rows<<<grid, warps * 32, 0, st>>>(src, v, ld, m, ids, nrows, nrows_pad, dst, norm2, err);
    return cudaGetLastError();
}

cudaError_t launch_dist_fp32(const float* A, int64_t M, int lda, const float* anorm,
                             const int32_t* a_ids, const float* B, int N, int ldb,
                             const float* bnorm, const int32_t* b_ids, int K, float* D,
                             int ldd, cudaStream_t st)
{
    if (M <= 0 || ldd <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + kDistBM - 1) / kDistBM), (unsigned)((ldd + kDistBN - 1) / kDistBN));
    k_dist_fp32<<<grid, 128, 0, st>>>(A, M, lda, anorm, a_ids, B, N, ldb, bnorm, b_ids, K, D, ldd);
    return cudaGetLastError();
}

cudaError_t launch_dist_gather(const float* cost, int64_t v, const int32_t* a_ids, int64_t M,
                               const int32_t* b_ids, int N, float* D, int ldd, int* err,
                               cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    k_dist_gather<<<(unsigned)M, 128, 0, st>>>(cost, v, a_ids, M, b_ids, N, D, ldd, err);
    return cudaGetLastError();
}

cudaError_t launch_table(const float* D, int ldd, int64_t M, int h, int k, const float* q_w,
                         float2* tab, int32_t* tab_s, bool sq, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    const dim3 tgrid((unsigned)((M + 127) / 128));
    if (k <= 1) k_table<1><<<tgrid, 128, 0, st>>>(D, ldd, M, h, k, q_w, tab, tab_s, sq);
    else if (k <= 2) k_table<2><<<tgrid, 128, 0, st>>>(D, ldd, M, h, k, q_w, tab, tab_s, sq);
    else if (k <= 4) k_table<4><<<tgrid, 128, 0, st>>>(D, ldd, M, h, k, q_w, tab, tab_s, sq);
    else if (k <= 8) k_table<8><<<tgrid, 128, 0, st>>>(D, ldd, M, h, k, q_w, tab, tab_s, sq);
    else if (k <= 16) k_table<16><<<tgrid, 128, 0, st>>>(D, ldd, M, h, k, q_w, tab, tab_s, sq);
    else {
        const int warps = 8;
        dim3 grid((unsigned)((M + warps - 1) / warps));
        k_table_generic<<<grid, warps * 32, 0, st>>>(D, ldd, M, h, k, q_w, tab, tab_s, sq);
    }
    return cudaGetLastError();
}

cudaError_t launch_zero_ident(const int32_t* q_idx, int h, const int32_t* vslot, int64_t v, float* D, int ldd,
                              cudaStream_t st)
{
    if (h <= 0) return cudaSuccess;
    k_zero_ident<<<1, 256, 0, st>>>(q_idx, h, vslot, v, D, ldd);
    return cudaGetLastError();
}

cudaError_t launch_table_ict(const float* D, int ldd, int64_t M, int h, int W, const float* q_w,
                             const float* xmax, float2* tab, int32_t* tab_s, int* over, bool sq, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    if (W < 1 || h < 1) return cudaErrorInvalidValue;
    const int warps = 8;
    k_table_ict_fast<<<(unsigned)((M + 127) / 128), 128, 0, st>>>(D, ldd, M, h, W, q_w, xmax, tab, tab_s, over, sq);
    k_table_ict<<<(unsigned)((M + warps - 1) / warps), warps * 32, 0, st>>>(D, ldd, M, h, W, q_w, xmax, tab, tab_s,
                                                                           over, sq);
    return cudaGetLastError();
}

}  // namespace emd

namespace emd {

cudaError_t launch_table_rerank(float* D, int ldd, int64_t M, int h, int k, int kc, const float* V,
                                const float* Q, int ldv, const float* q_w, float2* tab, int32_t* tab_s,
                                cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    if (k < 1 || kc < k || kc > h || kc > kRerankMax || ldv % 4 != 0) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((M + kRrRows - 1) / kRrRows);
    const size_t smem = rerank_smem_bytes(h);
    cudaError_t e = rerank_smem_attr(smem);
    if (e != cudaSuccess) return e;
    if (kc <= 8) k_table_rerank<8><<<grid, kRrRows, smem, st>>>(D, ldd, M, h, k, kc, V, Q, ldv, q_w, tab, tab_s);
    else if (kc <= 12) k_table_rerank<12><<<grid, kRrRows, smem, st>>>(D, ldd, M, h, k, kc, V, Q, ldv, q_w, tab, tab_s);
    else if (kc <= 16) k_table_rerank<16><<<grid, kRrRows, smem, st>>>(D, ldd, M, h, k, kc, V, Q, ldv, q_w, tab, tab_s);
    else k_table_rerank<32><<<grid, kRrRows, smem, st>>>(D, ldd, M, h, k, kc, V, Q, ldv, q_w, tab, tab_s);
    return cudaGetLastError();
}

}  // namespace emd

namespace emd {

cudaError_t launch_gather_rows_b(const QDesc* qd, const int* nq, int max_q, int max_rows, const float* src,
                                 int64_t v, int ld, int m, int* err, cudaStream_t st)
{
    if (max_q <= 0 || max_rows <= 0) return cudaSuccess;
    const int warps = 8;
    k_gather_rows_b<<<dim3((unsigned)((max_rows + warps - 1) / warps), (unsigned)max_q), warps * 32, 0, st>>>(
        qd, nq, src, v, ld, m, err);
    return cudaGetLastError();
}

cudaError_t launch_dist_fp32_b(const QDesc* qd, const int* nq, int max_q, int max_ldd, const float* A, int64_t M,
                               int lda, const float* anorm, const int32_t* a_ids, int K, cudaStream_t st)
{
    if (max_q <= 0 || M <= 0 || max_ldd <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + kDistBM - 1) / kDistBM), (unsigned)((max_ldd + kDistBN - 1) / kDistBN), (unsigned)max_q);
    k_dist_fp32_b<<<grid, 128, 0, st>>>(qd, nq, A, M, lda, anorm, a_ids, K);
    return cudaGetLastError();
}

cudaError_t launch_dist_gather_b(const QDesc* qd, const int* nq, int max_q, const float* cost, int64_t v,
                                 const int32_t* a_ids, int64_t M, int* err, cudaStream_t st)
{
    if (max_q <= 0 || M <= 0) return cudaSuccess;
    k_dist_gather_b<<<dim3((unsigned)M, (unsigned)max_q), 128, 0, st>>>(qd, nq, cost, v, a_ids, M, err);
    return cudaGetLastError();
}

cudaError_t launch_zero_ident_b(const QDesc* qd, const int* nq, int max_q, int max_h, const int32_t* vslot, int64_t v,
                                cudaStream_t st)
{
    if (max_q <= 0 || max_h <= 0) return cudaSuccess;
    k_zero_ident_b<<<(unsigned)max_q, 256, 0, st>>>(qd, nq, vslot, v);
    return cudaGetLastError();
}

cudaError_t launch_qpos_b(const QDesc* qd, const int* nq, int max_q, const int32_t* vslot, int64_t v, bool set,
                          cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    k_qpos_b<<<(unsigned)max_q, 256, 0, st>>>(qd, nq, vslot, v, set);
    return cudaGetLastError();
}

cudaError_t launch_table_ict_b(const QDesc* qd, const int* nq, int max_q, int64_t M, const float* xmax,
                               cudaStream_t st)
{
    if (max_q <= 0 || M <= 0) return cudaSuccess;
    const int warps = 8;
    k_table_ict_fast_b<<<dim3((unsigned)((M + 127) / 128), (unsigned)max_q), 128, 0, st>>>(qd, nq, M, xmax);
    k_table_ict_b<<<dim3((unsigned)((M + warps - 1) / warps), (unsigned)max_q), warps * 32, 0, st>>>(qd, nq, M, xmax);
    return cudaGetLastError();
}

cudaError_t launch_table_b(const QDesc* qd, const int* nq, int max_q, int64_t M, int max_tk, bool rerank,
                           int max_kc, int max_h, const float* V, int ldv, cudaStream_t st)
{
    if (max_q <= 0 || M <= 0) return cudaSuccess;
    const dim3 g((unsigned)((M + 127) / 128), (unsigned)max_q);
    if (rerank) {
        const int64_t tiles = (M + kRrRows - 1) / kRrRows;
        if (max_kc > kRerankMax || tiles > 65535 || ldv % 4 != 0) return cudaErrorInvalidValue;
        const dim3 gq((unsigned)max_q, (unsigned)tiles);
        const size_t smem = rerank_smem_bytes(max_h);
        cudaError_t e = rerank_smem_attr(smem);
        if (e != cudaSuccess) return e;
        if (max_kc <= 8) k_table_rerank_b<8><<<gq, kRrRows, smem, st>>>(qd, nq, M, V, ldv);
        else if (max_kc <= 12) k_table_rerank_b<12><<<gq, kRrRows, smem, st>>>(qd, nq, M, V, ldv);
        else if (max_kc <= 16) k_table_rerank_b<16><<<gq, kRrRows, smem, st>>>(qd, nq, M, V, ldv);
        else k_table_rerank_b<32><<<gq, kRrRows, smem, st>>>(qd, nq, M, V, ldv);
    } else if (max_tk <= 1) k_table_b<1><<<g, 128, 0, st>>>(qd, nq, M);
    else if (max_tk <= 2) k_table_b<2><<<g, 128, 0, st>>>(qd, nq, M);
    else if (max_tk <= 4) k_table_b<4><<<g, 128, 0, st>>>(qd, nq, M);
    else if (max_tk <= 8) k_table_b<8><<<g, 128, 0, st>>>(qd, nq, M);
    else if (max_tk <= 16) k_table_b<16><<<g, 128, 0, st>>>(qd, nq, M);
    else {
        const int warps = 8;
        k_table_generic_b<<<dim3((unsigned)((M + warps - 1) / warps), (unsigned)max_q), warps * 32, 0, st>>>(qd, nq, M);
    }
    return cudaGetLastError();
}

}  // namespace emd

namespace emd {

cudaError_t launch_rerank_cand_b(const QDesc* qd, const int* nq, int max_q, int64_t M, int max_h, const float* V,
                                 int ldv, const float* vnorm, bool certify, float eps_rel, float eps_abs,
                                 cudaStream_t st)
{
    if (max_q <= 0 || M <= 0) return cudaSuccess;
    const int64_t tiles = (M + kRrRows - 1) / kRrRows;
    if (tiles > 65535 || ldv % 4 != 0) return cudaErrorInvalidValue;
    const size_t smem = rerank_smem_bytes(max_h);
    cudaError_t e = rerank_smem_attr(smem);
    if (e != cudaSuccess) return e;
    k_rerank_cand_b<16><<<dim3((unsigned)max_q, (unsigned)tiles), kRrRows, smem, st>>>(qd, nq, M, V, ldv, vnorm,
                                                                                       certify, eps_rel, eps_abs);
    return cudaGetLastError();
}

cudaError_t launch_rerank_full_b(const QDesc* qd, const int* nq, int max_q, int max_tk, const float* V, int ldv,
                                 cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    if (max_tk > 16 || ldv % 4 != 0) return cudaErrorInvalidValue;
    const dim3 g(64, (unsigned)max_q);
    if (max_tk <= 4)
        k_rerank_full_b<4><<<g, 256, 0, st>>>(qd, nq, V, ldv);
    else if (max_tk <= 8)
        k_rerank_full_b<8><<<g, 256, 0, st>>>(qd, nq, V, ldv);
    else
        k_rerank_full_b<16><<<g, 256, 0, st>>>(qd, nq, V, ldv);
    return cudaGetLastError();
}

}  // namespace emd
