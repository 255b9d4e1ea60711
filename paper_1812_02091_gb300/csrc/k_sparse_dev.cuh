// Device code of the sparse passes over the database (Section 5, the reverse direction of
// Section 6 and the symmetric maximum) and of the top-K selection, shared by the per-query
// launchers (k_sparse.cu) and the batched ones (k_sparse_b.cu); every kernel here is a
// template or small, and each translation unit instantiates what its launchers use.
#pragma once
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

// ------------------------------------------------------------------ reverse pass
//
// The query's bins are the sources (mass q_j), the document's bins the destinations
// (capacities x_u), the cost block D[supp(d), j] is gathered from the Phase-1 matrix.
// One warp per document.  Lane l of a pass handles the NJ consecutive query bins
// j = jbase + NJ*l .. +NJ-1 and keeps, for each, a register list of the KT smallest
// (distance, capacity) over the document's bins, visited in CSR order.  A D row segment
// for one document bin is one NJ-float vector load per lane (a warp reads 128*NJ
// contiguous bytes); four bins' loads are issued before their insertions.  Insertion is
// branch-free: with 32*NJ lists per warp some list almost always changes, so a branch
// would diverge on nearly every bin.  Strict '<' keeps the earlier bin first on equal
// distance.

// Cost of moving source mass qj along a sorted destination list (Alg. 3 / Alg. 1).  The loop
// runs over the compile-time width with predicates so that the lists stay in registers;
// transfers after the residual reaches zero add exactly zero.
// sq: the lists hold squared distances (ordered the same way); they are converted here,
// KT square roots per query bin instead of one per gathered entry.
template <int MEAS, int KT>
__device__ __forceinline__ float rev_cost_sorted(float qj, const float (&zs)[KT], const float (&cap)[KT],
                                                 int keff, bool sq)
{
    float z[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) z[l] = d_value(zs[l], sq);
    if (MEAS == M_RWMD) return __fmul_rn(qj, z[0]);
    if (MEAS == M_OMR) {
        if (KT >= 2 && z[0] == 0.f && keff >= 2) {
            const float r = qj - fminf(qj, cap[0]);
            return r != 0.f ? __fmul_rn(r, z[KT >= 2 ? 1 : 0]) : 0.f;
        }
        return __fmul_rn(qj, z[0]);
    }
    // z is ascending, so z[keff-1] is the largest of the first keff entries (distances >= 0)
    float r = qj, c = 0.f, zlast = 0.f;
#pragma unroll
    for (int l = 0; l < KT; ++l) {
        const bool capped = l < keff - 1;
        const float tau = fminf(r, cap[l]);
        c = capped ? fmaf(tau, z[l], c) : c;
        r = capped ? r - tau : r;
        zlast = fmaxf(zlast, l < keff ? z[l] : 0.f);
    }
    return r != 0.f ? fmaf(r, zlast, c) : c;
}

// Insert (d, x) into the ascending list z (payload c), keeping the KT smallest.
template <int KT>
__device__ __forceinline__ void insert_sorted(float (&z)[KT], float (&c)[KT], float d, float x)
{
    bool p[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) p[l] = d < z[l];
#pragma unroll
    for (int l = KT - 1; l > 0; --l) {
        z[l] = p[l - 1] ? z[l - 1] : (p[l] ? d : z[l]);
        c[l] = p[l - 1] ? c[l - 1] : (p[l] ? x : c[l]);
    }
    z[0] = p[0] ? d : z[0];
    c[0] = p[0] ? x : c[0];
}

__device__ __forceinline__ void load_vec(const float* p, bool ok, float (&o)[1])
{
    o[0] = ok ? *p : INFINITY;
}
__device__ __forceinline__ void load_vec(const float* p, bool ok, float (&o)[2])
{
    const float2 v = ok ? *reinterpret_cast<const float2*>(p) : make_float2(INFINITY, INFINITY);
    o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void load_vec(const float* p, bool ok, float (&o)[4])
{
    const float4 v = ok ? *reinterpret_cast<const float4*>(p) : make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

template <int MEAS, int KT, int NJ>
__device__ __forceinline__ void rev_body(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
      const float* __restrict__ val, int64_t n, const float* __restrict__ D, int ldd, int h,
      const float* __restrict__ q_w, int k, const float* __restrict__ t_fwd,
      float* __restrict__ t_rev, float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
      const int* __restrict__ n_dev, bool sq)
{
    constexpr int U = 4;  // bins whose loads are in flight together
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    if (n_dev) n = min(n, (int64_t)*n_dev);  // slots filled on the device (candidate lists)
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int64_t dd = doc_ids ? doc_ids[d] : d;  // document of this output slot
        const int32_t a = row_ptr[dd], b = row_ptr[dd + 1];
        const int hd = b - a;
        const int keff = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? min(2, hd) : min(k, hd));
        float total = 0.f;
        for (int jbase = 0; jbase < h; jbase += 32 * NJ) {
            const int j0 = jbase + lane * NJ;
            const bool jin = j0 < ldd;  // ldd % 32 == 0 and NJ | 32: the whole vector is in the row
            float z[NJ][KT], cap[NJ][KT];
#pragma unroll
            for (int t = 0; t < NJ; ++t)
#pragma unroll
                for (int l = 0; l < KT; ++l) { z[t][l] = INFINITY; cap[t][l] = 0.f; }
            for (int32_t eb = a; eb < b; eb += 32) {
                const int32_t e = eb + lane;
                const int32_t u = e < b ? col[e] : 0;
                const float x = e < b ? val[e] : 0.f;
                const int cnt = min(32, b - eb);
                int i = 0;
                for (; i + U <= cnt; i += U) {
                    float dv[U][NJ], xv[U];
#pragma unroll
                    for (int s = 0; s < U; ++s) {
                        const int32_t ui = __shfl_sync(0xffffffffu, u, i + s);
                        xv[s] = __shfl_sync(0xffffffffu, x, i + s);
                        load_vec(D + (int64_t)ui * ldd + j0, jin, dv[s]);
                    }
#pragma unroll
                    for (int s = 0; s < U; ++s)
#pragma unroll
                        for (int t = 0; t < NJ; ++t) insert_sorted<KT>(z[t], cap[t], dv[s][t], xv[s]);
                }
                for (; i < cnt; ++i) {
                    const int32_t ui = __shfl_sync(0xffffffffu, u, i);
                    const float xi = __shfl_sync(0xffffffffu, x, i);
                    float dv[NJ];
                    load_vec(D + (int64_t)ui * ldd + j0, jin, dv);
#pragma unroll
                    for (int t = 0; t < NJ; ++t) insert_sorted<KT>(z[t], cap[t], dv[t], xi);
                }
            }
#pragma unroll
            for (int t = 0; t < NJ; ++t)
                if (j0 + t < h) total = __fadd_rn(total, rev_cost_sorted<MEAS, KT>(q_w[j0 + t], z[t], cap[t], keff, sq));
        }
        total = warp_sum(total);
        if (lane == 0) {
            t_rev[d] = total;
            if (t_max) t_max[d] = fmaxf(t_fwd[dd], total);
        }
    }
}

template <int MEAS, int KT, int NJ>
__global__ void __launch_bounds__(256, 2) k_rev(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
      const float* __restrict__ val, int64_t n, const float* __restrict__ D, int ldd, int h,
      const float* __restrict__ q_w, int k, const float* __restrict__ t_fwd,
      float* __restrict__ t_rev, float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
      const int* __restrict__ n_dev, bool sq)
{
    rev_body<MEAS, KT, NJ>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq);
}

// Candidate-list form: a block of W warps per candidate slot.  Warp w scans the w-th
// contiguous chunk of the document's bins; warp 0 then inserts the other chunks' lists in
// chunk order.  Strict '<' keeps an earlier chunk's entry ahead of an equal distance from a
// later one, so the merged list (and the cost, summed in the same lane order) is
// bit-identical to the one-warp kernel above.  W times the warps on a few hundred
// documents, whose single-warp scans are latency-bound.
template <int MEAS, int KT, int NJ, int W>
__device__ __forceinline__ void rev_blk_body(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
          const float* __restrict__ val, const float* __restrict__ D, int ldd, int h,
          const float* __restrict__ q_w, int k, const float* __restrict__ t_fwd,
          float* __restrict__ t_rev, float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
          const int* __restrict__ n_dev, bool sq, const int32_t* __restrict__ rmap = nullptr)
{
    constexpr int U = 4;
    __shared__ float sz[W - 1][32 * NJ][KT];
    __shared__ float sc[W - 1][32 * NJ][KT];
    const int slot = blockIdx.x;
    if (slot >= min(*n_dev, (int)gridDim.x)) return;  // uniform over the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t dd = doc_ids[slot];
    const int32_t a = row_ptr[dd], b = row_ptr[dd + 1];
    const int hd = b - a;
    const int keff = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? min(2, hd) : min(k, hd));
    const int chunk = (hd + W - 1) / W;
    const int32_t ca = a + min(hd, warp * chunk), cb = a + min(hd, (warp + 1) * chunk);
    float total = 0.f;
    for (int jbase = 0; jbase < h; jbase += 32 * NJ) {
        const int j0 = jbase + lane * NJ;
        const bool jin = j0 < ldd;
        float z[NJ][KT], cap[NJ][KT];
#pragma unroll
        for (int t = 0; t < NJ; ++t)
#pragma unroll
            for (int l = 0; l < KT; ++l) { z[t][l] = INFINITY; cap[t][l] = 0.f; }
        for (int32_t eb = ca; eb < cb; eb += 32) {
            const int32_t e = eb + lane;
            const int32_t u = e < cb ? col[e] : 0;
            const float x = e < cb ? val[e] : 0.f;
            const int cnt = min(32, cb - eb);
            int i = 0;
            for (; i + U <= cnt; i += U) {
                float dv[U][NJ], xv[U];
#pragma unroll
                for (int s = 0; s < U; ++s) {
                    const int32_t ui = __shfl_sync(0xffffffffu, u, i + s);
                    xv[s] = __shfl_sync(0xffffffffu, x, i + s);
                    load_vec(D + (rmap ? (int64_t)rmap[ui] : (int64_t)ui) * ldd + j0, jin, dv[s]);
                }
#pragma unroll
                for (int s = 0; s < U; ++s)
#pragma unroll
                    for (int t = 0; t < NJ; ++t) insert_sorted<KT>(z[t], cap[t], dv[s][t], xv[s]);
            }
            for (; i < cnt; ++i) {
                const int32_t ui = __shfl_sync(0xffffffffu, u, i);
                const float xi = __shfl_sync(0xffffffffu, x, i);
                float dv[NJ];
                load_vec(D + (rmap ? (int64_t)rmap[ui] : (int64_t)ui) * ldd + j0, jin, dv);
#pragma unroll
                for (int t = 0; t < NJ; ++t) insert_sorted<KT>(z[t], cap[t], dv[t], xi);
            }
        }
        if (warp > 0) {
#pragma unroll
            for (int t = 0; t < NJ; ++t)
#pragma unroll
                for (int l = 0; l < KT; ++l) {
                    sz[warp - 1][lane * NJ + t][l] = z[t][l];
                    sc[warp - 1][lane * NJ + t][l] = cap[t][l];
                }
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int w = 0; w < W - 1; ++w)
#pragma unroll
                for (int t = 0; t < NJ; ++t)
#pragma unroll
                    for (int l = 0; l < KT; ++l)
                        insert_sorted<KT>(z[t], cap[t], sz[w][lane * NJ + t][l], sc[w][lane * NJ + t][l]);
#pragma unroll
            for (int t = 0; t < NJ; ++t)
                if (j0 + t < h) total = __fadd_rn(total, rev_cost_sorted<MEAS, KT>(q_w[j0 + t], z[t], cap[t], keff, sq));
        }
        __syncthreads();
    }
    if (warp == 0) {
        total = warp_sum(total);
        if (lane == 0) {
            t_rev[slot] = total;
            if (t_max) t_max[slot] = fmaxf(t_fwd[dd], total);
        }
    }
}

// 24 resident warps per SM whatever W, as the batched form (80 registers, no spills).
template <int MEAS, int KT, int NJ, int W>
__global__ void __launch_bounds__(W * 32, (W >= 8 ? 3 : (W >= 4 ? 6 : 12)))
k_rev_blk(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
          const float* __restrict__ val, const float* __restrict__ D, int ldd, int h,
          const float* __restrict__ q_w, int k, const float* __restrict__ t_fwd,
          float* __restrict__ t_rev, float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
          const int* __restrict__ n_dev, bool sq)
{
    rev_blk_body<MEAS, KT, NJ, W>(row_ptr, col, val, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq);
}

// k above the register width (ICT, large k): per lane, successive minima over the
// document's bins, each strictly after the previous in (distance, bin position) order,
// until the source mass is placed.  O(steps * h_d) per query bin.  The query bins are
// taken in tiles of 32 (lane = bin within the tile); a lane's costs are summed per tile
// residue t mod kRevW, and the kRevW partial sums are then added in order -- the same
// arithmetic whether one warp walks all tiles (rev_generic_body) or kRevW warps split them
// (rev_generic_blk_body, for candidate lists).
constexpr int kRevW = 8;

template <int MEAS>
__device__ __forceinline__ float rev_generic_bin(const int32_t* __restrict__ col, const float* __restrict__ val,
                                                 int32_t a, int32_t b, int keff, const float* __restrict__ D, int ldd,
                                                 int j, float qj, bool sq)
{
    float r = qj, c = 0.f;
    float pz = -INFINITY;
    int pe = -1;
    for (int l = 0; l < keff; ++l) {
        float bz = INFINITY, bx = 0.f;
        int be = INT32_MAX;
        for (int32_t e = a; e < b; ++e) {
            const float dv = D[(int64_t)col[e] * ldd + j];
            const int pos = e - a;
            const bool after = dv > pz || (dv == pz && pos > pe);
            if (after && (dv < bz || (dv == bz && pos < be))) { bz = dv; be = pos; bx = val[e]; }
        }
        const float zd = d_value(bz, sq);
        if (l < keff - 1) {
            const float tau = fminf(r, bx);
            c = fmaf(tau, zd, c);
            r -= tau;
            if (r == 0.f) break;
        } else {
            c = fmaf(r, zd, c);
        }
        pz = bz;
        pe = be;
    }
    return c;
}

template <int MEAS>
__device__ __forceinline__ void rev_generic_body(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const float* __restrict__ val, int64_t n, const float* __restrict__ D,
                              int ldd, int h, const float* __restrict__ q_w, int k,
                              const float* __restrict__ t_fwd, float* __restrict__ t_rev,
                              float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
                              const int* __restrict__ n_dev, bool sq)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    if (n_dev) n = min(n, (int64_t)*n_dev);
    for (int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n; d += warps) {
        const int64_t dd = doc_ids ? doc_ids[d] : d;
        const int32_t a = row_ptr[dd], b = row_ptr[dd + 1];
        const int hd = b - a;
        const int keff = MEAS == M_ICT ? hd : min(k, hd);
        float part[kRevW];
#pragma unroll
        for (int w = 0; w < kRevW; ++w) part[w] = 0.f;
        for (int t0 = 0; t0 * 32 < h; t0 += kRevW) {
#pragma unroll
            for (int w = 0; w < kRevW; ++w) {
                const int j = (t0 + w) * 32 + lane;
                if (j < h) part[w] = __fadd_rn(part[w], rev_generic_bin<MEAS>(col, val, a, b, keff, D, ldd, j, q_w[j], sq));
            }
        }
        float total = part[0];
#pragma unroll
        for (int w = 1; w < kRevW; ++w) total = __fadd_rn(total, part[w]);
        total = warp_sum(total);
        if (lane == 0) {
            t_rev[d] = total;
            if (t_max) t_max[d] = fmaxf(t_fwd[dd], total);
        }
    }
}

// Candidate-list form: a block of kRevW warps per slot, warp w taking the query-bin tiles
// t = w, w + kRevW, ...; warp 0 adds the partial sums in warp order.  Same values as
// rev_generic_body.
template <int MEAS>
__device__ __forceinline__ void rev_generic_blk_body(const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col, const float* __restrict__ val,
                                                     const float* __restrict__ D, int ldd, int h,
                                                     const float* __restrict__ q_w, int k,
                                                     const float* __restrict__ t_fwd, float* __restrict__ t_rev,
                                                     float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
                                                     const int* __restrict__ n_dev, bool sq)
{
    __shared__ float sp[kRevW][32];
    const int slot = blockIdx.x;
    if (slot >= min(*n_dev, (int)gridDim.x)) return;  // uniform over the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t dd = doc_ids[slot];
    const int32_t a = row_ptr[dd], b = row_ptr[dd + 1];
    const int hd = b - a;
    const int keff = MEAS == M_ICT ? hd : min(k, hd);
    float part = 0.f;
    for (int t = warp; t * 32 < h; t += kRevW) {
        const int j = t * 32 + lane;
        if (j < h) part = __fadd_rn(part, rev_generic_bin<MEAS>(col, val, a, b, keff, D, ldd, j, q_w[j], sq));
    }
    sp[warp][lane] = part;
    __syncthreads();
    if (warp == 0) {
        float total = sp[0][lane];
#pragma unroll
        for (int w = 1; w < kRevW; ++w) total = __fadd_rn(total, sp[w][lane]);
        total = warp_sum(total);
        if (lane == 0) {
            t_rev[slot] = total;
            if (t_max) t_max[slot] = fmaxf(t_fwd[dd], total);
        }
    }
}

template <int MEAS>
__global__ void __launch_bounds__(kRevW * 32) k_rev_generic_blk(const int32_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col, const float* __restrict__ val,
                                  const float* __restrict__ D, int ldd, int h, const float* __restrict__ q_w, int k,
                                  const float* __restrict__ t_fwd, float* __restrict__ t_rev,
                                  float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
                                  const int* __restrict__ n_dev, bool sq)
{
    rev_generic_blk_body<MEAS>(row_ptr, col, val, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq);
}

template <int MEAS>
__global__ void k_rev_generic(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const float* __restrict__ val, int64_t n, const float* __restrict__ D,
                              int ldd, int h, const float* __restrict__ q_w, int k,
                              const float* __restrict__ t_fwd, float* __restrict__ t_rev,
                              float* __restrict__ t_max, const int64_t* __restrict__ doc_ids,
                              const int* __restrict__ n_dev, bool sq)
{
    rev_generic_body<MEAS>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq);
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
__device__ __forceinline__ void topk_values_body(const float* __restrict__ t, int64_t n, int K, int64_t per_block,
                                                 unsigned long long* __restrict__ scratch_row,
                                                 int64_t* __restrict__ out_idx, float* __restrict__ out_dist)
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
        block_merge_and_emit<KT>(L, KT, scratch_row + (int64_t)blockIdx.x * KT, nullptr, nullptr);
}

template <int KT>
__device__ __forceinline__ void topk_keys_body(const unsigned long long* __restrict__ keys, int64_t count, int K,
                                               int64_t* __restrict__ out_idx, float* __restrict__ out_dist)
{
    unsigned long long L[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) L[l] = ~0ull;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) list_insert<KT>(L, keys[i]);
    block_merge_and_emit<KT>(L, K, nullptr, out_idx, out_dist);
}

template <int KT>
__global__ void __launch_bounds__(kTopkThreads)
k_topk_values(const float* __restrict__ t, int64_t n, int64_t ldt, int K, int64_t per_block,
              unsigned long long* __restrict__ scratch, int64_t* __restrict__ out_idx,
              float* __restrict__ out_dist)
{
    const int64_t row = blockIdx.y;
    topk_values_body<KT>(t + row * ldt, n, K, per_block, scratch + row * kTopkScratchRow, out_idx + row * K,
                         out_dist + row * K);
}

template <int KT>
__global__ void __launch_bounds__(kTopkThreads)
k_topk_keys(const unsigned long long* __restrict__ keys, int64_t count, int K,
            int64_t* __restrict__ out_idx, float* __restrict__ out_dist)
{
    const int64_t row = blockIdx.x;
    topk_keys_body<KT>(keys + row * kTopkScratchRow, count, K, out_idx + row * K, out_dist + row * K);
}

// Batched forms: row q of the batch reads qd[q].t_fwd and writes sel_idx / sel_val (the
// forward top-K of the pruned path, fwd_rows) or reads t_out and writes out_idx / out_dist.
template <int KT>
__global__ void __launch_bounds__(kTopkThreads)
k_topk_values_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t n, int K, int64_t per_block,
                unsigned long long* __restrict__ scratch, bool fwd_rows)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    topk_values_body<KT>(fwd_rows ? d.t_fwd : d.t_out, n, K, per_block,
                         scratch + (int64_t)blockIdx.y * kTopkScratchRow, fwd_rows ? d.sel_idx : d.out_idx,
                         fwd_rows ? d.sel_val : d.out_dist);
}

template <int KT>
__global__ void __launch_bounds__(kTopkThreads)
k_topk_keys_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t count, int K,
              const unsigned long long* __restrict__ scratch, bool fwd_rows)
{
    if ((int)blockIdx.x >= *nq) return;
    const QDesc& d = qd[blockIdx.x];
    topk_keys_body<KT>(scratch + (int64_t)blockIdx.x * kTopkScratchRow, count, K, fwd_rows ? d.sel_idx : d.out_idx,
                       fwd_rows ? d.sel_val : d.out_dist);
}

template <int KT>
cudaError_t topk_kt_b(const QDesc* qd, const int* nq, int max_q, int64_t n, int K, unsigned long long* scratch,
                      bool fwd_rows, cudaStream_t st)
{
    const size_t smem = (size_t)kTopkThreads * KT * sizeof(unsigned long long);
    const int blocks = topk_blocks(n);
    const int64_t per_block = (n + blocks - 1) / blocks;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_topk_values_b<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_topk_keys_b<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_topk_values_b<KT><<<dim3(blocks, (unsigned)max_q), kTopkThreads, smem, st>>>(qd, nq, n, K, per_block, scratch,
                                                                                    fwd_rows);
    if (blocks > 1)
        k_topk_keys_b<KT><<<(unsigned)max_q, kTopkThreads, smem, st>>>(qd, nq, (int64_t)blocks * KT, K, scratch,
                                                                        fwd_rows);
    return cudaGetLastError();
}

template <int KT>
cudaError_t topk_kt(const float* t, int64_t rows, int64_t n, int64_t ldt, int K,
                    unsigned long long* scratch, int64_t* out_idx, float* out_dist, cudaStream_t st)
{
    const size_t smem = (size_t)kTopkThreads * KT * sizeof(unsigned long long);
    const int blocks = topk_blocks(n);
    const int64_t per_block = (n + blocks - 1) / blocks;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_topk_values<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_topk_keys<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_topk_values<KT><<<dim3(blocks, (unsigned)rows), kTopkThreads, smem, st>>>(t, n, ldt, K, per_block, scratch,
                                                                                 out_idx, out_dist);
    if (blocks > 1)
        k_topk_keys<KT><<<(unsigned)rows, kTopkThreads, smem, st>>>(scratch, (int64_t)blocks * KT, K, out_idx,
                                                                     out_dist);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pruned symmetric top-K
//
// max(fwd, rev) >= fwd.  With theta = fwd_K * (1 + 2^-7) (fwd_K the K-th smallest forward
// value), the candidates are the documents with fwd <= theta; every other document has
// sym >= fwd > theta.  Once the K-th smallest symmetric value among the candidates is
// <= theta, no other document can enter the top-K, not even by the id tie-break.

__device__ __forceinline__ float prune_theta(float fwd_k) { return fwd_k * (1.0f + 0.0078125f); }

__device__ __forceinline__ void prune_compact_body(const float* __restrict__ t_fwd, int64_t n, const float* __restrict__ sel_val,
                                int K, int cap, int64_t* __restrict__ cand, int* __restrict__ count)
{
    const float theta = prune_theta(sel_val[K - 1]);
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x) {
        if (t_fwd[d] <= theta) {
            const int pos = atomicAdd(count, 1);
            if (pos < cap) cand[pos] = d;
        }
    }
}

__global__ void k_prune_compact(const float* __restrict__ t_fwd, int64_t n, const float* __restrict__ sel_val,
                                int K, int cap, int64_t* __restrict__ cand, int* __restrict__ count)
{
    prune_compact_body(t_fwd, n, sel_val, K, cap, cand, count);
}

// Final selection over the candidates: thread i ranks candidate i in (sym, id) order
// against the other filled slots (one 64-bit key compare each: distances are >= 0, so the
// key order is the (distance, id) order); ranks < K are written; ok = no overflow and
// K-th <= theta.
__device__ __forceinline__ void prune_select_body(const int64_t* __restrict__ cand, const float* __restrict__ sym,
                               const int* __restrict__ count, int cap, const float* __restrict__ sel_val,
                               int K, int64_t* __restrict__ out_idx, float* __restrict__ out_dist,
                               int* __restrict__ ok, bool complete = true)
{
    __shared__ unsigned long long key[kPruneCap];
    __shared__ float kth;
    const int c = min(*count, cap);
    const int i = threadIdx.x;
    const unsigned long long me =
        i < c ? ((unsigned long long)__float_as_uint(sym[i]) << 32) | (unsigned long long)(uint32_t)cand[i] : ~0ull;
    key[i] = me;
    if (i == 0) kth = INFINITY;
    __syncthreads();
    int r = 0;
    for (int j = 0; j < c; ++j) r += key[j] < me ? 1 : 0;
    if (i < c && r < K) {
        out_idx[r] = (int64_t)(me & 0xffffffffull);
        out_dist[r] = __uint_as_float((unsigned)(me >> 32));
    }
    if (i < c && r == K - 1) kth = __uint_as_float((unsigned)(me >> 32));
    __syncthreads();
    // 1: certified; 0: not certified (recompute over all documents); 2: the candidate
    // block of the fused path overflowed (retry with the full distance matrix)
    if (i == 0) *ok = !complete ? 2 : (*count <= cap && c >= K && kth <= prune_theta(sel_val[K - 1])) ? 1 : 0;
}

__global__ void k_prune_select(const int64_t* __restrict__ cand, const float* __restrict__ sym,
                               const int* __restrict__ count, int cap, const float* __restrict__ sel_val,
                               int K, int64_t* __restrict__ out_idx, float* __restrict__ out_dist,
                               int* __restrict__ ok)
{
    prune_select_body(cand, sym, count, cap, sel_val, K, out_idx, out_dist, ok);
}

template <int MEAS>
cudaError_t rev_meas_blk(int k, const int32_t* row_ptr, const int32_t* col, const float* val, int slots,
                         const float* D, int ldd, int h, const float* q_w, const float* t_fwd,
                         float* t_rev, float* t_max, const int64_t* doc_ids, const int* n_dev, bool sq,
                         cudaStream_t st)
{
    constexpr int W = 4;
    const int kt = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? 2 : k);
    const bool wide = h > 32;
#define EMD_REVB(KT, NJ) k_rev_blk<MEAS, KT, NJ, W><<<slots, W * 32, 0, st>>>(row_ptr, col, val, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq)
    if (kt <= 1) { if (wide) EMD_REVB(1, 4); else EMD_REVB(1, 1); }
    else if (kt <= 2) { if (wide) EMD_REVB(2, 4); else EMD_REVB(2, 1); }
    else if (kt <= 4) { if (wide) EMD_REVB(4, 4); else EMD_REVB(4, 1); }
    else if (kt <= 8) { if (wide) EMD_REVB(8, 2); else EMD_REVB(8, 1); }
    else EMD_REVB(16, 1);
#undef EMD_REVB
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched forms

// NJ follows the per-query launcher: NJW bins per lane when h > 32, else one.
template <int MEAS, int KT, int NJW>
__global__ void __launch_bounds__(256, 2)
k_rev_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
        const int32_t* __restrict__ col, const float* __restrict__ val, int64_t n, int k, int dir)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    float* t_rev = dir == EMD_DIR_REV ? d.t_out : d.t_rev;
    float* t_max = dir == EMD_DIR_MAX ? d.t_out : nullptr;
    if (d.h > 32)
        rev_body<MEAS, KT, NJW>(row_ptr, col, val, n, d.D, d.ldd, d.h, d.qw, k, d.t_fwd, t_rev, t_max, nullptr,
                                nullptr, d.sq != 0);
    else
        rev_body<MEAS, KT, 1>(row_ptr, col, val, n, d.D, d.ldd, d.h, d.qw, k, d.t_fwd, t_rev, t_max, nullptr,
                              nullptr, d.sq != 0);
}

template <int MEAS>
__global__ void k_rev_generic_b(const QDesc* __restrict__ qd, const int* __restrict__ nq,
                                const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ val, int64_t n, int k, int dir)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    float* t_rev = dir == EMD_DIR_REV ? d.t_out : d.t_rev;
    float* t_max = dir == EMD_DIR_MAX ? d.t_out : nullptr;
    rev_generic_body<MEAS>(row_ptr, col, val, n, d.D, d.ldd, d.h, d.qw, k, d.t_fwd, t_rev, t_max, nullptr, nullptr,
                           d.sq != 0);
}

__global__ void k_prune_compact_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int64_t n, int K)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    prune_compact_body(d.t_fwd, n, d.sel_val, K, kPruneCap, d.cand, d.cand_count);
}

// MAPPED: the distances come from the query's candidate-row block (fused path): used row u
// is row rmap[u] of Dc.  A query whose candidate documents hold more than kCandRows distinct
// rows has no complete block; it is skipped here and reported uncertified by the selection.
// 24 resident warps per SM whatever W (80 registers, no spills; the unbounded form took 106-112
// and left 16): the gathers of the distance block are latency-bound.
template <int MEAS, int KT, int NJW, int W, bool MAPPED>
__global__ void __launch_bounds__(W * 32, (W >= 8 ? 3 : (W >= 4 ? 6 : 12)))
k_rev_blk_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
            const int32_t* __restrict__ col, const float* __restrict__ val, int k)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    if (MAPPED && *d.ncrows > kCandRows) return;
    const float* D = MAPPED ? d.Dc : d.D;
    const int32_t* rmap = MAPPED ? d.rmap : nullptr;
    if (d.h > 32)
        rev_blk_body<MEAS, KT, NJW, W>(row_ptr, col, val, D, d.ldd, d.h, d.qw, k, d.t_fwd, d.cand_sym + kPruneCap,
                                       d.cand_sym, d.cand, d.cand_count, d.sq != 0, rmap);
    else
        rev_blk_body<MEAS, KT, 1, W>(row_ptr, col, val, D, d.ldd, d.h, d.qw, k, d.t_fwd, d.cand_sym + kPruneCap,
                                     d.cand_sym, d.cand, d.cand_count, d.sq != 0, rmap);
}

// Reverse values of the candidate documents, rows of any width (ICT): a block of kRevW
// warps each.
template <int MEAS>
__global__ void __launch_bounds__(kRevW * 32)
k_rev_generic_cand_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const int32_t* __restrict__ row_ptr,
                     const int32_t* __restrict__ col, const float* __restrict__ val, int k)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    rev_generic_blk_body<MEAS>(row_ptr, col, val, d.D, d.ldd, d.h, d.qw, k, d.t_fwd, d.cand_sym + kPruneCap,
                               d.cand_sym, d.cand, d.cand_count, d.sq != 0);
}

__global__ void k_prune_select_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int K, bool mapped)
{
    if ((int)blockIdx.x >= *nq) return;
    const QDesc& d = qd[blockIdx.x];
    prune_select_body(d.cand, d.cand_sym, d.cand_count, kPruneCap, d.sel_val, K, d.out_idx, d.out_dist, d.ok,
                      !mapped || *d.ncrows <= kCandRows);
}

template <int MEAS>
cudaError_t rev_meas_b(int k, int dir, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                       const int32_t* col, const float* val, int64_t n, cudaStream_t st)
{
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks), (unsigned)max_q);
    const int kt = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? 2 : (MEAS == M_ICT ? 1 << 30 : k));
#define EMD_REVQ(KT, NJ) k_rev_b<MEAS, KT, NJ><<<grid, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, k, dir)
    if (kt <= 1) EMD_REVQ(1, 4);
    else if (kt <= 2) EMD_REVQ(2, 4);
    else if (kt <= 4) EMD_REVQ(4, 4);
    else if (kt <= 8) EMD_REVQ(8, 2);
    else if (kt <= 16) EMD_REVQ(16, 1);
    else k_rev_generic_b<MEAS><<<grid, warps * 32, 0, st>>>(qd, nq, row_ptr, col, val, n, k, dir);
#undef EMD_REVQ
    return cudaGetLastError();
}

template <int MEAS, int W, bool MAPPED>
cudaError_t rev_meas_blk_bw(int k, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                            const int32_t* col, const float* val, cudaStream_t st)
{
    const int kt = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? 2 : k);
    const dim3 grid(kPruneCap, (unsigned)max_q);
#define EMD_REVBQ(KT, NJ) k_rev_blk_b<MEAS, KT, NJ, W, MAPPED><<<grid, W * 32, 0, st>>>(qd, nq, row_ptr, col, val, k)
    if (kt <= 1) EMD_REVBQ(1, 4);
    else if (kt <= 2) EMD_REVBQ(2, 4);
    else if (kt <= 4) EMD_REVBQ(4, 4);
    else if (kt <= 8) EMD_REVBQ(8, 2);
    else EMD_REVBQ(16, 1);
#undef EMD_REVBQ
    return cudaGetLastError();
}

// Warps per candidate document: 2, 4 or 8 (the merge in chunk order makes the result
// independent of the choice).
template <int MEAS, bool MAPPED = false>
cudaError_t rev_meas_blk_b(int k, int warps, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                           const int32_t* col, const float* val, cudaStream_t st)
{
    if (warps <= 2) return rev_meas_blk_bw<MEAS, 2, MAPPED>(k, qd, nq, max_q, row_ptr, col, val, st);
    if (warps <= 4) return rev_meas_blk_bw<MEAS, 4, MAPPED>(k, qd, nq, max_q, row_ptr, col, val, st);
    return rev_meas_blk_bw<MEAS, 8, MAPPED>(k, qd, nq, max_q, row_ptr, col, val, st);
}

// Candidate rows of the fused pruned path: every used row of every candidate document of
// query q gets a row of q's candidate block (first come, first served: the block's row
// order does not matter, each entry is computed independently).  A block per candidate
// document.
__global__ void k_cand_rows_b(const QDesc* __restrict__ qd, const int* __restrict__ nq,
                              const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    if ((int)blockIdx.x >= min(*d.cand_count, kPruneCap)) return;
    const int64_t doc = d.cand[blockIdx.x];
    for (int32_t e = row_ptr[doc] + (int32_t)threadIdx.x; e < row_ptr[doc + 1]; e += blockDim.x) {
        const int32_t u = col[e];
        if (atomicCAS(&d.rmap[u], -1, -2) == -1) {
            const int idx = atomicAdd(d.ncrows, 1);
            if (idx < kCandRows) d.crows[idx] = u;
            atomicExch(&d.rmap[u], idx);
        }
    }
}

// Returns the row map of the candidate documents' rows to -1 (the state every batch
// starts from).
__global__ void k_cand_reset_b(const QDesc* __restrict__ qd, const int* __restrict__ nq,
                               const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    if ((int)blockIdx.x >= min(*d.cand_count, kPruneCap)) return;
    const int64_t doc = d.cand[blockIdx.x];
    for (int32_t e = row_ptr[doc] + (int32_t)threadIdx.x; e < row_ptr[doc + 1]; e += blockDim.x) d.rmap[col[e]] = -1;
}

template <int MEAS>
cudaError_t rev_meas(int k, const int32_t* row_ptr, const int32_t* col, const float* val,
                     int64_t n, const float* D, int ldd, int h, const float* q_w,
                     const float* t_fwd, float* t_rev, float* t_max, const int64_t* doc_ids,
                     const int* n_dev, bool sq, cudaStream_t st)
{
    const int warps = 8;
    const int64_t blocks = std::min<int64_t>((n + warps - 1) / warps, 152 * 64);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks));
    const int kt = MEAS == M_RWMD ? 1 : (MEAS == M_OMR ? 2 : (MEAS == M_ICT ? 1 << 30 : k));
    const bool wide = h > 32;  // several 32-bin chunks: vector loads of consecutive bins
#define EMD_REV(KT, NJ) k_rev<MEAS, KT, NJ><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq)
    if (kt <= 1) { if (wide) EMD_REV(1, 4); else EMD_REV(1, 1); }
    else if (kt <= 2) { if (wide) EMD_REV(2, 4); else EMD_REV(2, 1); }
    else if (kt <= 4) { if (wide) EMD_REV(4, 4); else EMD_REV(4, 1); }
    else if (kt <= 8) { if (wide) EMD_REV(8, 2); else EMD_REV(8, 1); }
    else if (kt <= 16) EMD_REV(16, 1);
    else k_rev_generic<MEAS><<<grid, warps * 32, 0, st>>>(row_ptr, col, val, n, D, ldd, h, q_w, k, t_fwd, t_rev, t_max, doc_ids, n_dev, sq);
#undef EMD_REV
    return cudaGetLastError();
}

}  // namespace
}  // namespace emd
