// The forward direction's sparse pass over the database (Section 5, Phase 2 and 3): per
// nonzero, a database weight moved along its vocabulary row's table; the per-query form and
// the grouped forms of the batched path (one CSR sweep per group of eight queries).
#include <math.h>

#include <algorithm>

#include "emd_internal.cuh"

namespace emd {
namespace {

// ------------------------------------------------------------------ forward pass
//
// Phase 2 (Eq. 6-8) and Phase 3 (Eq. 9) evaluated per nonzero: a database weight x at
// vocabulary row u is moved into the query along row u's table, k-1 capacity-limited
// transfers then the rest at the k-th distance.  The per-nonzero costs are summed per
// document (t_fwd).  One warp per document, lanes over its nonzeros (coalesced col/val
// loads), table rows gathered from L2, warp-shuffle sum.

// Cost of one nonzero along its table row T (entries es apart).  Products and sums that the
// compiler could otherwise contract into an FMA in one kernel and not in another are written
// with __fmul_rn / __fadd_rn, so every kernel that shares these bodies rounds alike.
template <int MEAS>
__device__ __forceinline__ float fwd_cost_s(float x, const float2* __restrict__ T, int es, int keff)
{
    if (MEAS == M_RWMD) return __fmul_rn(x, T[0].x);
    if (MEAS == M_OMR) {
        const float2 t0 = T[0];
        if (t0.x == 0.f && keff >= 2) {
            const float r = x - fminf(x, t0.y);  // free transfer to the overlapping bin
            return r != 0.f ? __fmul_rn(r, T[es].x) : 0.f;
        }
        return __fmul_rn(x, t0.x);
    }
    float r = x, c = 0.f;
    for (int l = 0; l < keff - 1; ++l) {
        const float2 t = T[l * es];
        const float tau = fminf(r, t.y);
        c = fmaf(tau, t.x, c);
        r -= tau;
        if (r == 0.f) return c;
    }
    return fmaf(r, T[(keff - 1) * es].x, c);
}

template <int MEAS>
__device__ __forceinline__ float fwd_cost(float x, const float2* __restrict__ T, int keff)
{
    return fwd_cost_s<MEAS>(x, T, 1, keff);
}

// fwd_cost_s for keff <= KT without branches: the loop over the row is unrolled to KT and
// each step is predicated on (l < keff - 1 and residual > 0), so lanes whose residual ran
// out earlier neither diverge nor load.  Same operations in the same order: bit-identical.
// KT = 0: rows wider than 16, the loop form.
template <int MEAS, int KT>
__device__ __forceinline__ float fwd_cost_p(float x, const float2* __restrict__ T, int es, int keff)
{
    if (KT == 0 || MEAS != M_ACT) return fwd_cost_s<MEAS>(x, T, es, keff);
    float r = x, c = 0.f;
#pragma unroll
    for (int l = 0; l < (KT > 1 ? KT - 1 : 0); ++l) {
        if (l < keff - 1 && r != 0.f) {
            const float2 t = T[l * es];
            const float tau = fminf(r, t.y);
            c = fmaf(tau, t.x, c);
            r -= tau;
        }
    }
    return r != 0.f ? fmaf(r, T[(keff - 1) * es].x, c) : c;
}

// Summation order of a document's forward value, shared by every form of the pass: the
// nonzeros are split into four phases (position e - a mod 4), each summed in CSR order,
// then (p0 + p1) + (p2 + p3).  The per-query form gives each warp eight documents (lane =
// 8 x phase + document slot); the grouped form gives each warp one document for eight
// queries (lane = 8 x phase + query), so both compute every value identically.
template <int MEAS, int KT>
__device__ __forceinline__ void fwd_body(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                      const float* __restrict__ val, int64_t n, const float2* __restrict__ tab,
                      int k, int keff, float* __restrict__ t_fwd)
{
    const int lane = threadIdx.x & 31, slot = lane & 7, ph = lane >> 3;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 8; base < n;
         base += warps * 8) {
        const int64_t d = base + slot;
        const bool valid = d < n;
        const int32_t a = valid ? row_ptr[d] : 0, b = valid ? row_ptr[d + 1] : 0;
        float acc = 0.f;
        int32_t e = a + ph;
        for (; e + 12 < b; e += 16) {  // four nonzeros' costs in flight, added in order
            const int32_t u0 = col[e], u1 = col[e + 4], u2 = col[e + 8], u3 = col[e + 12];
            const float c0 = fwd_cost_p<MEAS, KT>(val[e], tab + (int64_t)u0 * k, 1, keff);
            const float c1 = fwd_cost_p<MEAS, KT>(val[e + 4], tab + (int64_t)u1 * k, 1, keff);
            const float c2 = fwd_cost_p<MEAS, KT>(val[e + 8], tab + (int64_t)u2 * k, 1, keff);
            const float c3 = fwd_cost_p<MEAS, KT>(val[e + 12], tab + (int64_t)u3 * k, 1, keff);
            acc = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(acc, c0), c1), c2), c3);
        }
        for (; e < b; e += 4)
            acc = __fadd_rn(acc, fwd_cost_p<MEAS, KT>(val[e], tab + (int64_t)col[e] * k, 1, keff));
        acc += __shfl_xor_sync(0xffffffffu, acc, 8);
        acc += __shfl_xor_sync(0xffffffffu, acc, 16);
        if (ph == 0 && valid) t_fwd[d] = acc;
    }
}

template <int MEAS, int KT>
__global__ void k_fwd(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                      const float* __restrict__ val, int64_t n, const float2* __restrict__ tab,
                      int k, int keff, float* __restrict__ t_fwd)
{
    fwd_body<MEAS, KT>(row_ptr, col, val, n, tab, k, keff, t_fwd);
}

// ------------------------------------------------------------------ batched forms

template <int MEAS, int KT>
__global__ void k_fwd_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
                        const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n, bool to_out)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    fwd_body<MEAS, KT>(row_ptr, col, val, n, d.tab, d.tk, d.tk, to_out ? d.t_out : d.t_fwd);
}

// One sweep of the CSR for a group of kFwdGroup (8) consecutive queries of the batch: a warp
// takes a document, lane = 8 x phase + query.  The 8 lanes of a nonzero read the same col /
// val and adjacent table entries (the group's tables are interleaved by entry), so a gather
// instruction touches 4 table rows instead of 32; the CSR is read once per group.  Values
// are bit-identical to the per-query form (same phases, same order).  The sweep is bound by
// the latency of its dependent gathers, not by bandwidth: 32 registers give 8 blocks (all 64
// warps) per SM, and two nonzeros per lane per step fit in them (four spill or cost occupancy;
// measured on 1e6 documents, 64 mixed-size queries: 19.6 ms at 6 blocks and four nonzeros,
// 16.9 ms at 8 blocks and two).
template <int MEAS, int KT>
__global__ void __launch_bounds__(256, 8)
k_fwd_g(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
        const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n, bool to_out)
{
    const int q0 = blockIdx.y * kFwdGroup;
    const int nqv = *nq;
    if (q0 >= nqv) return;
    const int lane = threadIdx.x & 31, g = lane & 7, ph = lane >> 3;
    const bool act = q0 + g < nqv;
    const QDesc& dq = qd[act ? q0 + g : q0];
    const float2* tq = dq.tab;
    const int kq = dq.tk;
    float* oq = to_out ? dq.t_out : dq.t_fwd;
    const int rs = dq.tab_rs, es = dq.tab_es;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float acc = 0.f;
        int32_t e = a + ph;
        for (; e + 4 < b; e += 8) {  // two nonzeros' costs in flight, added in order
            const int32_t u0 = col[e], u1 = col[e + 4];
            const float x0 = val[e], x1 = val[e + 4];
            if (act) {
                const float c0 = fwd_cost_p<MEAS, KT>(x0, tq + (int64_t)u0 * rs, es, kq);
                const float c1 = fwd_cost_p<MEAS, KT>(x1, tq + (int64_t)u1 * rs, es, kq);
                acc = __fadd_rn(__fadd_rn(acc, c0), c1);
            }
        }
        if (e < b) {
            const int32_t u = col[e];
            const float x = val[e];
            if (act) acc = __fadd_rn(acc, fwd_cost_p<MEAS, KT>(x, tq + (int64_t)u * rs, es, kq));
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 8);
        acc += __shfl_xor_sync(0xffffffffu, acc, 16);
        if (ph == 0 && act) oq[d] = acc;
    }
}

// Cost of one nonzero from the first KR entries of its table row already in registers
// (entries KR.. are loaded here, only while mass remains; entry l at T[l * es]).  The same
// operations in the same order as fwd_cost_p, so the values are bit-identical.
template <int MEAS, int KT, int KR>
__device__ __forceinline__ float fwd_cost_reg(float x, const float2 (&E)[KR], const float2* __restrict__ T, int es,
                                              int keff)
{
    if (MEAS == M_RWMD) return __fmul_rn(x, E[0].x);
    if (MEAS == M_OMR) {
        if (E[0].x == 0.f && keff >= 2) {
            const float r = x - fminf(x, E[0].y);
            return r != 0.f ? __fmul_rn(r, (KR > 1 ? E[KR > 1 ? 1 : 0] : T[es]).x) : 0.f;
        }
        return __fmul_rn(x, E[0].x);
    }
    float r = x, c = 0.f;
#pragma unroll
    for (int l = 0; l < (KT > 1 ? KT - 1 : 0); ++l) {
        if (l < keff - 1 && r != 0.f) {
            const float2 t = l < KR ? E[l < KR ? l : 0] : T[l * es];
            const float tau = fminf(r, t.y);
            c = fmaf(tau, t.x, c);
            r -= tau;
        }
    }
    if (r == 0.f) return c;
    const int lk = keff - 1;
    float zl;
    if (lk < KR) {
        zl = E[0].x;
#pragma unroll
        for (int l = 1; l < KR; ++l) zl = lk == l ? E[l].x : zl;
    } else {
        zl = T[lk * es].x;
    }
    return fmaf(r, zl, c);
}

// Forward pass of a group of kFwdGroup queries in one sweep of the CSR, tables of width
// <= KT (1, 2, 4, 8, 16) stored query-major within a row: query g's entries of row u at
// tab + u * tab_rs + l (tab_rs = 8 KT, the query's own offset g KT is in its descriptor), so
// a lane reads its first min(KT, 4) entries with independent vector loads before any
// arithmetic -- no chain of dependent loads per nonzero.  A warp takes a document; the
// column ids and weights of 32 consecutive nonzeros are read with one coalesced load per
// lane and handed to the lanes that use them by shuffles (lane = 8 x phase + query, phase
// = nonzero position mod 4).  Each phase sums its nonzeros in CSR order, then (p0 + p1) +
// (p2 + p3): the order of every other form of the pass, so values are bit-identical.
template <int MEAS, int KT>
__global__ void __launch_bounds__(256, 3)
k_fwd_gv(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
         const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n, bool to_out)
{
    constexpr int KR = KT < 4 ? KT : 4;
    const int q0 = blockIdx.y * kFwdGroup;
    const int nqv = *nq;
    if (q0 >= nqv) return;
    const int lane = threadIdx.x & 31, g = lane & 7, ph = lane >> 3;
    const bool act = q0 + g < nqv;
    const QDesc& dq = qd[act ? q0 + g : q0];
    const float2* tq = dq.tab;
    const int kq = dq.tk;
    float* oq = to_out ? dq.t_out : dq.t_fwd;
    const int rs = dq.tab_rs;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float acc = 0.f;
        for (int32_t eb = a; eb < b; eb += 32) {
            const bool lin = eb + lane < b;
            const int32_t cu = lin ? col[eb + lane] : 0;
            const float cx = lin ? val[eb + lane] : 0.f;
#pragma unroll
            for (int r = 0; r < 8; r += 4) {  // four nonzeros per lane in flight
                float2 E[4][KR];
                float xs[4];
                int32_t us[4];
                bool ok[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int src = 4 * (r + i) + ph;
                    us[i] = __shfl_sync(0xffffffffu, cu, src);
                    xs[i] = __shfl_sync(0xffffffffu, cx, src);
                    ok[i] = act && eb + src < b;
                    const float2* T = tq + (int64_t)us[i] * rs;
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    if constexpr (KR == 4) {
                        const float4 v0 = ok[i] ? *reinterpret_cast<const float4*>(T) : z4;
                        const float4 v1 = ok[i] ? *reinterpret_cast<const float4*>(T + 2) : z4;
                        E[i][0] = make_float2(v0.x, v0.y);
                        E[i][1] = make_float2(v0.z, v0.w);
                        E[i][2] = make_float2(v1.x, v1.y);
                        E[i][3] = make_float2(v1.z, v1.w);
                    } else if constexpr (KR == 2) {
                        const float4 v0 = ok[i] ? *reinterpret_cast<const float4*>(T) : z4;
                        E[i][0] = make_float2(v0.x, v0.y);
                        E[i][1] = make_float2(v0.z, v0.w);
                    } else {
                        E[i][0] = ok[i] ? T[0] : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (ok[i]) acc = __fadd_rn(acc, fwd_cost_reg<MEAS, KT, KR>(xs[i], E[i], tq + (int64_t)us[i] * rs, 1, kq));
            }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 8);
        acc += __shfl_xor_sync(0xffffffffu, acc, 16);
        if (ph == 0 && act) oq[d] = acc;
    }
}

// The entry-chain sweep of k_fwd_g with the CSR read one group ahead: each lane (four
// nonzeros of its phase per step) loads the column ids and weights of its next four
// nonzeros before it evaluates the current ones, so the DRAM latency of the stream overlaps
// the table gathers.  Same steps and summation order as k_fwd_g: bit-identical.
template <int MEAS, int KT>
__global__ void k_fwd_gp(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n, bool to_out)
{
    const int q0 = blockIdx.y * kFwdGroup;
    const int nqv = *nq;
    if (q0 >= nqv) return;
    const int lane = threadIdx.x & 31, g = lane & 7, ph = lane >> 3;
    const bool act = q0 + g < nqv;
    const QDesc& dq = qd[act ? q0 + g : q0];
    const float2* tq = dq.tab;
    const int kq = dq.tk;
    float* oq = to_out ? dq.t_out : dq.t_fwd;
    const int rs = dq.tab_rs, es = dq.tab_es;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float acc = 0.f;
        int32_t e = a + ph;
        int32_t pu[4];
        float px[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool v = e + 4 * i < b;
            pu[i] = v ? col[e + 4 * i] : 0;
            px[i] = v ? val[e + 4 * i] : 0.f;
        }
        while (e < b) {
            int32_t u[4];
            float x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                u[i] = pu[i];
                x[i] = px[i];
            }
            const int32_t en = e + 16;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool v = en + 4 * i < b;
                pu[i] = v ? col[en + 4 * i] : 0;
                px[i] = v ? val[en + 4 * i] : 0.f;
            }
            if (act) {
                float c[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    c[i] = e + 4 * i < b ? fwd_cost_p<MEAS, KT>(x[i], tq + (int64_t)u[i] * rs, es, kq) : 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (e + 4 * i < b) acc = __fadd_rn(acc, c[i]);
            }
            e = en;
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 8);
        acc += __shfl_xor_sync(0xffffffffu, acc, 16);
        if (ph == 0 && act) oq[d] = acc;
    }
}

// Forward pass of a group of kFwdGroup queries, entry-interleaved tables (row u, entry l,
// query g at tab[u * tab_rs + l * kFwdGroup], so the group's entry l of a row is 64
// contiguous bytes): the column ids and weights of 32 nonzeros are read with one coalesced
// load and handed out by shuffles as in k_fwd_gv; the first two entries of each row are
// loaded before any arithmetic, later ones only while mass remains.  Fewer registers than
// k_fwd_gv (more resident warps), fewer bytes per nonzero.  Same values as every other form.
template <int MEAS, int KT>
__global__ void __launch_bounds__(256, 4)
k_fwd_gc(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
         const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n, bool to_out)
{
    constexpr int KR = KT < 2 ? KT : 2;
    const int q0 = blockIdx.y * kFwdGroup;
    const int nqv = *nq;
    if (q0 >= nqv) return;
    const int lane = threadIdx.x & 31, g = lane & 7, ph = lane >> 3;
    const bool act = q0 + g < nqv;
    const QDesc& dq = qd[act ? q0 + g : q0];
    const float2* tq = dq.tab;
    const int kq = dq.tk;
    float* oq = to_out ? dq.t_out : dq.t_fwd;
    const int rs = dq.tab_rs, es = dq.tab_es;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int32_t a = row_ptr[d], b = row_ptr[d + 1];
        float acc = 0.f;
        for (int32_t eb = a; eb < b; eb += 32) {
            const bool lin = eb + lane < b;
            const int32_t cu = lin ? col[eb + lane] : 0;
            const float cx = lin ? val[eb + lane] : 0.f;
#pragma unroll
            for (int r = 0; r < 8; r += 4) {  // four nonzeros per lane in flight
                float2 E[4][KR];
                float xs[4];
                int32_t us[4];
                bool ok[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int src = 4 * (r + i) + ph;
                    us[i] = __shfl_sync(0xffffffffu, cu, src);
                    xs[i] = __shfl_sync(0xffffffffu, cx, src);
                    ok[i] = act && eb + src < b;
                    const float2* T = tq + (int64_t)us[i] * rs;
#pragma unroll
                    for (int l = 0; l < KR; ++l) E[i][l] = ok[i] ? T[l * es] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (ok[i]) acc = __fadd_rn(acc, fwd_cost_reg<MEAS, KT, KR>(xs[i], E[i], tq + (int64_t)us[i] * rs, es, kq));
            }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 8);
        acc += __shfl_xor_sync(0xffffffffu, acc, 16);
        if (ph == 0 && act) oq[d] = acc;
    }
}

}  // namespace

// Register width of the forward cost for table width kw (0: the loop form).
static int fwd_kt(int kw) { return fwd_reg_width(kw); }

#define EMD_FWD_KT_SWITCH(KTV, LAUNCH)             \
    switch (KTV) {                                 \
    case 1: LAUNCH(1); break;                      \
    case 2: LAUNCH(2); break;                      \
    case 4: LAUNCH(4); break;                      \
    case 8: LAUNCH(8); break;                      \
    case 16: LAUNCH(16); break;                    \
    default: LAUNCH(0); break;                     \
    }

cudaError_t launch_fwd(int meas, const int32_t* row_ptr, const int32_t* col, const float* val,
                       int64_t n, const float2* tab, int k, int keff, float* t_fwd,
                       cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int warps = 8;  // eight documents per warp
    const int64_t blocks = std::min<int64_t>((n + 8 * warps - 1) / (8 * warps), 152 * 64);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks));
    switch (meas) {
    case M_RWMD: k_fwd<M_RWMD, 0><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, tab, k, keff, t_fwd); break;
    case M_OMR: k_fwd<M_OMR, 0><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, tab, k, keff, t_fwd); break;
    default: {
#define EMD_L(KT) k_fwd<M_ACT, KT><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, tab, k, keff, t_fwd)
        EMD_FWD_KT_SWITCH(fwd_kt(keff), EMD_L)
#undef EMD_L
        break;
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_fwd_b(int meas, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                         const int32_t* col, const float* val, int64_t n, bool to_out, bool grouped, int max_tk,
                         cudaStream_t st, int variant)
{
    const int kt = fwd_kt(max_tk);
    if (max_q <= 0 || n <= 0) return cudaSuccess;
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    if (grouped) {  // one document per warp, eight queries
        dim3 gg((unsigned)std::max<int64_t>(1, blocks), (unsigned)((max_q + kFwdGroup - 1) / kFwdGroup));
        const int m = meas == M_ICT ? M_ACT : meas;  // ICT tables: the ACT steps over the written entries
        const int kw = meas == M_RWMD ? 1 : meas == M_OMR ? 2 : (meas == M_ICT && kt == 0 ? 0 : kt);
        if (variant == kFwdPrefetch) {  // the entry chain with the CSR read one group ahead
            switch (m) {
            case M_RWMD: k_fwd_gp<M_RWMD, 0><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out); break;
            case M_OMR: k_fwd_gp<M_OMR, 0><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out); break;
            default: {
#define EMD_L(KT) k_fwd_gp<M_ACT, KT><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out)
                EMD_FWD_KT_SWITCH(kw, EMD_L)
#undef EMD_L
                break;
            }
            }
            return cudaGetLastError();
        }
        if (kw == 0 || variant == kFwdChain) {  // entry-interleaved rows, loads while mass remains
            switch (m) {
            case M_RWMD: k_fwd_g<M_RWMD, 0><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out); break;
            case M_OMR: k_fwd_g<M_OMR, 0><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out); break;
            default: {
#define EMD_L(KT) k_fwd_g<M_ACT, KT><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out)
                EMD_FWD_KT_SWITCH(kw, EMD_L)
#undef EMD_L
                break;
            }
            }
            return cudaGetLastError();
        }
#define EMD_GV(M, KT)                                                                                       \
    do {                                                                                                    \
        if (variant == kFwdRowMajor)                                                                        \
            k_fwd_gv<M, KT><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out);               \
        else                                                                                                \
            k_fwd_gc<M, KT><<<gg, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out);               \
    } while (0)
        switch (m) {
        case M_RWMD: EMD_GV(M_RWMD, 1); break;
        case M_OMR: EMD_GV(M_OMR, 2); break;
        default:
            switch (kw) {
            case 1: EMD_GV(M_ACT, 1); break;
            case 2: EMD_GV(M_ACT, 2); break;
            case 4: EMD_GV(M_ACT, 4); break;
            case 8: EMD_GV(M_ACT, 8); break;
            default: EMD_GV(M_ACT, 16); break;
            }
        }
#undef EMD_GV
        return cudaGetLastError();
    }
    const int64_t qblocks = std::min<int64_t>((n + 8 * warps - 1) / (8 * warps), 152 * 64);  // eight documents per warp
    dim3 grid((unsigned)std::max<int64_t>(1, qblocks), (unsigned)max_q);
    switch (meas) {
    case M_RWMD: k_fwd_b<M_RWMD, 0><<<grid, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out); break;
    case M_OMR: k_fwd_b<M_OMR, 0><<<grid, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out); break;
    default: {
#define EMD_L(KT) k_fwd_b<M_ACT, KT><<<grid, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, to_out)
        EMD_FWD_KT_SWITCH(kt, EMD_L)
#undef EMD_L
        break;
    }
    }
    return cudaGetLastError();
}

}  // namespace emd
