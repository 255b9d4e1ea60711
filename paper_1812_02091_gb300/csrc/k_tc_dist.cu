// Phase 1 of LC-ACT (Section 5) on the 5th-generation tensor cores of sm_103a: the
// distance matrix D = dist(V, Q) from the product V Q^T (Section 5: "a matrix-matrix
// multiplication between V and the transpose of Q") with FP32 accumulators in TMEM.
//
// Operands carry a per-row absmax scale s (x = s * stored value).  Three operand formats:
//  * TC_SPLIT: FP16 hi + lo * 2^-11 (hi = fp16(x/s), lo = fp16((x/s - hi) * 2^11)); three
//    products hi*hi (accumulator 0) and hi*lo + lo*hi (accumulator 1) reconstruct the dot
//    product to about 2^-22 relative: FP32-grade distances on the tensor pipe (kind::f16).
//  * TC_BF16: bf16(x/s), one product (kind::f16 with BF16 inputs).
//  * TC_E4M3: e4m3(448 x / amax), s = amax / 448, one product (kind::f8f6f4).
// The BF16 and E4M3 distances are approximate; the top-k table kernel re-ranks each row's
// candidates with exact FP32 sums of squared differences.
//
// Data movement: both operands are pre-packed in global memory in the canonical K-major,
// no-swizzle UMMA layout -- core matrices of 8 rows x 16 bytes (128 contiguous bytes);
// inside a 64-element K chunk the core matrices of a row group are adjacent (leading byte
// offset 128 B) and row groups follow each other 8 x (bytes of a 64-element row segment)
// apart (stride byte offset: 1 KB for 2-byte types, 512 B for E4M3).  A tile's K chunk is
// therefore one contiguous block and moves with one 1-D bulk copy (cp.async.bulk, the TMA
// engine) completing on an mbarrier.
//
// Roles (320 threads, one persistent CTA per SM): warp 0 lane 0 issues the copies into a
// ring of stages; warp 1 allocates TMEM and its lane 0 issues tcgen05.mma (M = 128 rows of
// V, N <= 128 query columns, K = 16 (32 for E4M3) per instruction) and tcgen05.commit;
// warps 2..9 read
// their TMEM lane quarter with tcgen05.ld and write the squared distance |v|^2 + |q|^2 -
// 2 v.q (the readers of D take the square root of the entries they use; the exact zeros
// of identical vocabulary ids are written after the kernel).  Every wait is bounded in time; a timeout
// latches ERR_TIMEOUT, raises a block-wide abort flag and the block tears down.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <algorithm>

#include "emd_internal.cuh"

namespace emd {
namespace {

constexpr int TC_BM = 128;          // rows per tile = TMEM lanes
constexpr int TC_BN = 128;          // largest column tile
constexpr int TC_THREADS = 320;  // warp 0 copies, warp 1 MMA, warps 2..9 epilogue
constexpr uint64_t TC_TIMEOUT_NS = 2000000000ull;
constexpr int TCB_EPI_WARPS = 16;                  // batched form: epilogue warps
constexpr int TCB_THREADS = 64 + 32 * TCB_EPI_WARPS;  // + copy warp + MMA warp

// Per-format constants: bytes of a 64-element row segment, operand parts, MMAs per
// 64-element chunk (each advances 2 core matrices = 256 B along K).
template <int FMT> struct TcFmt;
template <> struct TcFmt<TC_SPLIT> { static constexpr uint32_t EB = 128, parts = 2, mmas = 4, atype = 0; };
template <> struct TcFmt<TC_BF16> { static constexpr uint32_t EB = 128, parts = 1, mmas = 4, atype = 1; };
template <> struct TcFmt<TC_E4M3> { static constexpr uint32_t EB = 64, parts = 1, mmas = 2, atype = 0; };

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false once the deadline has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline)
{
    while (!mbar_try_wait(bar, parity))
        if (global_ns() > deadline) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: canonical K-major layout without swizzle, leading
// byte offset 128 (next core matrix along K), stride byte offset `sbo` (next 8-row group),
// descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// D[tmem] (+)= A[smem] * B[smem]^T with FP32 accumulation: kind::f16 (FP16 or BF16 inputs,
// both the same type) or kind::f8f6f4 (E4M3 inputs).
template <int FMT>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    if (FMT == TC_E4M3)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrive on the mbarrier once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive TMEM columns of this thread's lane (32x32b shape, 32 repetitions).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// 16 consecutive TMEM columns of this thread's lane (32x32b shape, 16 repetitions).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane from registers (32x32b shape).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent form: each CTA (one per SM) walks tiles t = blockIdx.x, += gridDim.x in
// column-tile-major order (t -> column tile t / m_tiles, row tile t % m_tiles), so a CTA's
// consecutive tiles nearly always share their query columns.  The query panel (all K
// chunks of the tile's columns, hi and lo) is loaded once into shared memory and reloaded
// only when the column tile changes; the vocabulary panels stream through a ring of
// `stages` stages.  Every SM reading the same small query panel for every tile would
// otherwise concentrate the L2 traffic on a few slices.  The accumulators alternate
// between two TMEM buffers, so the MMA warp fills one while the eight epilogue warps drain
// the other (two warps per TMEM lane quarter, each taking half of the columns).
template <int FMT>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_dist(const uint8_t* __restrict__ A_hi, const uint8_t* __restrict__ A_lo, int64_t Mpad,
          const float* __restrict__ a_scale, const float* __restrict__ a_norm,
          int64_t M, const uint8_t* __restrict__ B_hi, const uint8_t* __restrict__ B_lo, int64_t Npad,
          const float* __restrict__ b_scale, const float* __restrict__ b_norm,
          int N, int KC, int stages, float* __restrict__ D, int ldd, int* __restrict__ err)
{
    constexpr bool SPLIT = FMT == TC_SPLIT;
    constexpr uint32_t EB = TcFmt<FMT>::EB;
    constexpr int kParts = (int)TcFmt<FMT>::parts;
    constexpr uint32_t kABytes = TC_BM * EB;                       // one 64-element K chunk of 128 rows
    constexpr uint32_t kBBytes = TC_BN * EB;
    constexpr uint32_t kSbo = 8 * EB;
    constexpr uint32_t kStage = kParts * kABytes;                  // vocabulary chunk: hi (and lo)
    constexpr uint32_t kBChunk = kParts * kBBytes;                 // query chunk: hi (and lo)
    constexpr uint32_t kAcc = SPLIT ? 256 : 128;  // TMEM columns per accumulator buffer (acc0 | acc1)
    constexpr uint32_t kCols = 2 * kAcc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* bpanel = smem + (size_t)stages * kStage;              // KC query chunks
    uint64_t* full = reinterpret_cast<uint64_t*>(bpanel + (size_t)KC * kBChunk);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;   // [2] accumulator ready (MMA commit)
    uint64_t* tempty = tfull + 2;       // [2] accumulator drained (8 epilogue warps)
    uint64_t* bfull = tempty + 2;       // query panel loaded
    uint64_t* bfree = bfull + 1;        // MMAs reading the query panel done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bfree + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tiles = (int)(Mpad / TC_BM);
    const int n_tiles = (N + TC_BN - 1) / TC_BN;
    const int total = m_tiles * n_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(bfull, 1);
        mbar_init(bfree, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
    };

    if (warp == 0 && lane == 0) {
        // producer: the query panel when the column tile changes, vocabulary chunks always
        int64_t g = 0;
        int cur_n = -1, reloads = 0;
        for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
            const int64_t m0 = (int64_t)(t % m_tiles) * TC_BM;
            const int nt = t / m_tiles;
            if (nt != cur_n) {
                if (reloads > 0 && !mbar_wait(bfree, (uint32_t)(reloads - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    break;
                }
                const int n0 = nt * TC_BN;
                const int Nt = min(TC_BN, (int)round_up(N - n0, 16));
                const uint32_t b_bytes = (uint32_t)Nt * EB;
                mbar_expect_tx(bfull, (uint32_t)(kParts * KC) * b_bytes);
                for (int c = 0; c < KC; ++c) {
                    uint8_t* bst = bpanel + (size_t)c * kBChunk;
                    bulk_g2s(bst, B_hi + ((int64_t)c * Npad + n0) * EB, b_bytes, bfull);
                    if (SPLIT) bulk_g2s(bst + kBBytes, B_lo + ((int64_t)c * Npad + n0) * EB, b_bytes, bfull);
                }
                cur_n = nt;
                ++reloads;
            }
            for (int c = 0; c < KC; ++c, ++g) {
                const int s = (int)(g % stages);
                if (g >= stages && !mbar_wait(&empty[s], (uint32_t)((g / stages) - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    break;
                }
                uint8_t* st = smem + (size_t)s * kStage;
                mbar_expect_tx(&full[s], kStage);
                bulk_g2s(st, A_hi + ((int64_t)c * Mpad + m0) * EB, kABytes, &full[s]);
                if (SPLIT) bulk_g2s(st + kABytes, A_lo + ((int64_t)c * Mpad + m0) * EB, kABytes, &full[s]);
            }
        }
        // no copy may still be landing in shared memory when the block leaves
        const uint64_t tail = global_ns() + TC_TIMEOUT_NS;
        for (int64_t c = g > stages ? g - stages : 0; c < g; ++c)
            if (!mbar_wait(&full[c % stages], (uint32_t)(c / stages) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
        if (reloads > 0 && !mbar_wait(bfull, (uint32_t)(reloads - 1) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: D format F32 (bit 4), A/B format at bits 7 and 10 (F16 or E4M3 = 0,
        // BF16 = 1), K-major A and B, N >> 3 at bit 17, M >> 4 at bit 24
        int64_t g = 0;
        int it = 0, cur_n = -1, reloads = 0;
        for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++it) {
            const int nt = t / m_tiles;
            const int n0 = nt * TC_BN;
            const int Nt = min(TC_BN, (int)round_up(N - n0, 16));
            const uint32_t idesc = (1u << 4) | (TcFmt<FMT>::atype << 7) | (TcFmt<FMT>::atype << 10) |
                                   ((uint32_t)(Nt >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
            if (nt != cur_n) {
                if (reloads > 0) mma_commit(bfree);  // the old panel is released once its MMAs finish
                if (!mbar_wait(bfull, (uint32_t)reloads & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    break;
                }
                cur_n = nt;
                ++reloads;
            }
            const int buf = it & 1;
            if (it >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((it >> 1) - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            tc_fence_after();
            const uint32_t acc0 = tmem + (uint32_t)buf * kAcc;
            bool ok = true;
            for (int c = 0; c < KC; ++c, ++g) {
                const int s = (int)(g % stages);
                if (!mbar_wait(&full[s], (uint32_t)(g / stages) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + (size_t)s * kStage);
                const uint32_t sa_lo = sa + kABytes;
                const uint32_t sb = smem_u32(bpanel + (size_t)c * kBChunk);
                const uint32_t sb_lo = sb + kBBytes;
                // descriptors of the chunk's first K step; a step of 16 elements (256 B) adds 16 to the
                // address field (addresses stay below 2^18, so no carry leaves the 14-bit field)
                const uint64_t dA0 = smem_desc(sa, kSbo), dB0 = smem_desc(sb, kSbo);
                const uint64_t dAl0 = smem_desc(sa_lo, kSbo), dBl0 = smem_desc(sb_lo, kSbo);
#pragma unroll
                for (int ks = 0; ks < (int)TcFmt<FMT>::mmas; ++ks) {  // each MMA: 2 core matrices = 256 B of K
                    const uint32_t ko = (uint32_t)ks * 256u;
                    const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                    const uint64_t kd = (uint64_t)(ko >> 4);
                    const uint64_t da = dA0 + kd, db = dB0 + kd;
                    mma_issue<FMT>(acc0, da, db, idesc, acc);
                    if (SPLIT) {
                        mma_issue<FMT>(acc0 + 128, da, dBl0 + kd, idesc, acc);
                        mma_issue<FMT>(acc0 + 128, dAl0 + kd, db, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&tfull[buf]);
            if (!ok) break;
        }
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 = tile rows, columns of its half
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        int it = 0;
        for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++it) {
            const int64_t m0 = (int64_t)(t % m_tiles) * TC_BM;
            const int n0 = (t / m_tiles) * TC_BN;
            const int Nt = min(TC_BN, (int)round_up(N - n0, 16));
            const int buf = it & 1;
            if (!mbar_wait(&tfull[buf], (uint32_t)(it >> 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            tc_fence_after();
            const int64_t u = m0 + row;
            const bool row_ok = u < M;
            const float su = row_ok ? a_scale[u] : 0.f;
            const float nu = row_ok ? a_norm[u] : 0.f;
            const uint32_t tbase = tmem + (uint32_t)buf * kAcc + ((uint32_t)(q * 32) << 16);
            for (int cc = half * 64; cc < half * 64 + 64 && cc < Nt; cc += 32) {
                uint32_t r0[32], r1[32];
                tmem_ld32(tbase + (uint32_t)cc, r0);
                if (SPLIT) tmem_ld32(tbase + 128u + (uint32_t)cc, r1);
                tmem_wait_ld();
                // lane l fetches the constants of column n0 + cc + l once (coalesced); inside
                // the element loop they are broadcast by shuffles
                const int lcol = n0 + cc + lane;
                const bool lok = lcol < N;
                const float cb_l = lok ? -2.f * b_scale[lcol] : 0.f;
                const float nb_l = lok ? b_norm[lcol] : 0.f;
                // every lane runs the loop (full-warp shuffles); rows past M only skip the stores
                float* out = D + (row_ok ? u : 0) * ldd + n0 + cc;
#pragma unroll
                for (int e4 = 0; e4 < 8; ++e4) {
                    float o[4];
#pragma unroll
                    for (int tt = 0; tt < 4; ++tt) {
                        const int e = e4 * 4 + tt;
                        const float cb = __shfl_sync(0xffffffffu, cb_l, e);
                        const float nb = __shfl_sync(0xffffffffu, nb_l, e);
                        float dot = __uint_as_float(r0[e]);
                        if (SPLIT) dot = fmaf(__uint_as_float(r1[e]), 1.0f / 2048.0f, dot);
                        o[tt] = fmaf(cb * su, dot, nu + nb);  // squared distance, unclamped
                    }
                    if (row_ok && n0 + cc + e4 * 4 < ldd)
                        *reinterpret_cast<float4*>(out + e4 * 4) = make_float4(o[0], o[1], o[2], o[3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// Batched form: every query of a batch against the same vocabulary.  Work item = (row tile
// r, query group g): the CTA loads all K chunks of the vocabulary tile once into shared
// memory (the "A panel", resident for the whole item) and streams the column tiles of the
// group's queries (each query's tiles n0 = 0, 128, ... < h) through a ring of B-chunk
// stages.  The vocabulary is thus read from HBM once per batch (once per group) instead of
// once per query.  MMA order, accumulators and epilogue are those of k_tc_dist, so each
// D[u, j] is bit-identical to the per-query kernel's.  Barriers: afull (A panel landed),
// afree (the item's MMAs are done with it), full/empty per B stage, tfull/tempty per TMEM
// accumulator buffer; every wait is bounded as in k_tc_dist.
template <int FMT>
__global__ void __launch_bounds__(TCB_THREADS, 1)
k_tc_dist_batch(const uint8_t* __restrict__ A_hi, const uint8_t* __restrict__ A_lo, int64_t Mpad,
                const float* __restrict__ a_scale, const float* __restrict__ a_norm,
                int64_t M, const QDesc* __restrict__ qd,
                const int* __restrict__ nq_dev, int groups, int KC, int stages, int klast, int* __restrict__ err)
{
    constexpr bool SPLIT = FMT == TC_SPLIT;
    constexpr uint32_t EB = TcFmt<FMT>::EB;
    constexpr int kParts = (int)TcFmt<FMT>::parts;
    constexpr uint32_t kABytes = TC_BM * EB;
    constexpr uint32_t kBBytes = TC_BN * EB;
    constexpr uint32_t kSbo = 8 * EB;
    constexpr uint32_t kAChunk = kParts * kABytes;
    constexpr uint32_t kBStage = kParts * kBBytes;
    constexpr uint32_t kAcc = SPLIT ? 256 : 128;
    constexpr uint32_t kCols = 2 * kAcc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* apanel = smem;                                   // KC A chunks (hi | lo)
    uint8_t* bring = apanel + (size_t)KC * kAChunk;           // stages B chunks (hi | lo)
    uint64_t* full = reinterpret_cast<uint64_t*>(bring + (size_t)stages * kBStage);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* afull = tempty + 2;
    uint64_t* afree = afull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(afree + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = *nq_dev;
    const int m_tiles = (int)(Mpad / TC_BM);
    const int total = m_tiles * groups;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], TCB_EPI_WARPS);
        }
        mbar_init(afull, 1);
        mbar_init(afree, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
    };
    auto qrange = [&](int g, int& qa, int& qb) {
        qa = (int)((int64_t)g * nq / groups);
        qb = (int)((int64_t)(g + 1) * nq / groups);
    };

    if (warp == 0 && lane == 0) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int items = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x, ++items) {
            const int64_t m0 = (int64_t)(w % m_tiles) * TC_BM;
            if (items > 0 && !mbar_wait(afree, (uint32_t)(items - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            mbar_expect_tx(afull, (uint32_t)KC * kAChunk);
            for (int c = 0; c < KC; ++c) {
                uint8_t* ast = apanel + (size_t)c * kAChunk;
                bulk_g2s(ast, A_hi + ((int64_t)c * Mpad + m0) * EB, kABytes, afull);
                if (SPLIT) bulk_g2s(ast + kABytes, A_lo + ((int64_t)c * Mpad + m0) * EB, kABytes, afull);
            }
            int qa, qb;
            qrange(w / m_tiles, qa, qb);
            for (int q = qa; q < qb && ok; ++q) {
                const QDesc& d = qd[q];
                const uint8_t* bh = static_cast<const uint8_t*>(d.q_hi);
                const uint8_t* bl = static_cast<const uint8_t*>(d.q_lo);
                for (int n0 = 0; n0 < d.h && ok; n0 += TC_BN) {
                    const int Nt = min(TC_BN, (int)round_up(d.h - n0, 16));
                    const uint32_t b_bytes = (uint32_t)Nt * EB;
                    for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                        const int s = rs;
                        if (gb >= stages &&
                            !mbar_wait(&empty[s], rp ^ 1u, global_ns() + TC_TIMEOUT_NS)) {
                            fail();
                            ok = false;
                            break;
                        }
                        uint8_t* bst = bring + (size_t)s * kBStage;
                        mbar_expect_tx(&full[s], (uint32_t)kParts * b_bytes);
                        bulk_g2s(bst, bh + ((int64_t)c * d.npad + n0) * EB, b_bytes, &full[s]);
                        if (SPLIT) bulk_g2s(bst + kBBytes, bl + ((int64_t)c * d.npad + n0) * EB, b_bytes, &full[s]);
                    }
                }
            }
        }
        // no copy may still be landing in shared memory when the block leaves
        const uint64_t tail = global_ns() + TC_TIMEOUT_NS;
        for (int64_t c = gb > stages ? gb - stages : 0; c < gb; ++c)
            if (!mbar_wait(&full[c % stages], (uint32_t)(c / stages) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
        if (items > 0 && !mbar_wait(afull, (uint32_t)(items - 1) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int it = 0, items = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x, ++items) {
            if (!mbar_wait(afull, (uint32_t)items & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            int qa, qb;
            qrange(w / m_tiles, qa, qb);
            for (int q = qa; q < qb && ok; ++q) {
                const int h = qd[q].h;
                for (int n0 = 0; n0 < h && ok; n0 += TC_BN, ++it) {
                    const int Nt = min(TC_BN, (int)round_up(h - n0, 16));
                    const uint32_t idesc = (1u << 4) | (TcFmt<FMT>::atype << 7) | (TcFmt<FMT>::atype << 10) |
                                           ((uint32_t)(Nt >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
                    const int buf = it & 1;
                    if (it >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((it >> 1) - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t acc0 = tmem + (uint32_t)buf * kAcc;
                    for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                        const int s = rs;
                        if (!mbar_wait(&full[s], rp, global_ns() + TC_TIMEOUT_NS)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(apanel + (size_t)c * kAChunk);
                        const uint32_t sa_lo = sa + kABytes;
                        const uint32_t sb = smem_u32(bring + (size_t)s * kBStage);
                        const uint32_t sb_lo = sb + kBBytes;
                        // descriptors of the chunk's first K step; a step of 16 elements (256 B) adds 16 to the
                        // address field (addresses stay below 2^18, so no carry leaves the 14-bit field)
                        const uint64_t dA0 = smem_desc(sa, kSbo), dB0 = smem_desc(sb, kSbo);
                        const uint64_t dAl0 = smem_desc(sa_lo, kSbo), dBl0 = smem_desc(sb_lo, kSbo);
#pragma unroll
                        for (int ks = 0; ks < (int)TcFmt<FMT>::mmas; ++ks) {
                            if (c == KC - 1 && ks >= klast) break;  // the last chunk's zero K steps
                            const uint32_t ko = (uint32_t)ks * 256u;
                            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                            const uint64_t kd = (uint64_t)(ko >> 4);
                            const uint64_t da = dA0 + kd, db = dB0 + kd;
                            mma_issue<FMT>(acc0, da, db, idesc, acc);
                            if (SPLIT) {
                                mma_issue<FMT>(acc0 + 128, da, dBl0 + kd, idesc, acc);
                                mma_issue<FMT>(acc0 + 128, dAl0 + kd, db, idesc, 1u);
                            }
                        }
                        mma_commit(&empty[s]);
                    }
                    mma_commit(&tfull[buf]);
                }
            }
            mma_commit(afree);  // the A panel is free once this item's MMAs complete
        }
    } else if (warp >= 2) {
        // epilogue: 16 warps, four per TMEM lane quarter (warp w reads lanes 32*(w%4) ..
        // +31 = tile rows), each draining 32 of the tile's columns
        const int qw4 = warp & 3;
        const int cc = ((warp - 2) >> 2) * 32;
        const int row = qw4 * 32 + lane;
        int it = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
            const int64_t m0 = (int64_t)(w % m_tiles) * TC_BM;
            const int64_t u = m0 + row;
            const bool row_ok = u < M;
            const float su = row_ok ? a_scale[u] : 0.f;
            const float nu = row_ok ? a_norm[u] : 0.f;
            int qa, qb;
            qrange(w / m_tiles, qa, qb);
            for (int q = qa; q < qb && ok; ++q) {
                const QDesc& d = qd[q];
                const int N = d.h, ldd = d.ldd;
                const float* qsc = d.q_scale;
                const float* qnm = d.qnorm;
                float* Dq = d.D;
                for (int n0 = 0; n0 < N; n0 += TC_BN, ++it) {
                    const int Nt = min(TC_BN, (int)round_up(N - n0, 16));
                    const int buf = it & 1;
                    // this warp's column constants, fetched before the wait (coalesced)
                    const int lcol = n0 + cc + lane;
                    const bool lok = lcol < N;
                    const float cb_l = lok ? -2.f * qsc[lcol] : 0.f;
                    const float nb_l = lok ? qnm[lcol] : 0.f;
                    if (!mbar_wait(&tfull[buf], (uint32_t)(it >> 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (cc < Nt) {
                        const uint32_t tbase = tmem + (uint32_t)buf * kAcc + ((uint32_t)(qw4 * 32) << 16);
                        const float su2 = su;
                        float* out = Dq + (row_ok ? u : 0) * ldd + n0 + cc;
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {  // two halves of 16 columns
                        uint32_t r0[16], r1[16];
                        tmem_ld16(tbase + (uint32_t)(cc + 16 * hh), r0);
                        if (SPLIT) tmem_ld16(tbase + 128u + (uint32_t)(cc + 16 * hh), r1);
                        tmem_wait_ld();
#pragma unroll
                        for (int e4 = 4 * hh; e4 < 4 * hh + 4; ++e4) {
                            float o[4];
#pragma unroll
                            for (int tt = 0; tt < 4; ++tt) {
                                const int e = e4 * 4 + tt;
                                const int er = e - 16 * hh;
                                const float cb = __shfl_sync(0xffffffffu, cb_l, e);
                                const float nb = __shfl_sync(0xffffffffu, nb_l, e);
                                float dot = __uint_as_float(r0[er]);
                                if (SPLIT) dot = fmaf(__uint_as_float(r1[er]), 1.0f / 2048.0f, dot);
                                o[tt] = fmaf(cb * su2, dot, nu + nb);  // squared distance, unclamped
                            }
                            if (row_ok && n0 + cc + e4 * 4 < ldd)
                                *reinterpret_cast<float4*>(out + e4 * 4) = make_float4(o[0], o[1], o[2], o[3]);
                        }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[buf]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// ------------------------------------------------------------------ fused Phase-1 table
//
// Phase 1 with the per-row top-k folded into the product's epilogue (Section 5, Fig. 6:
// V Q^T, then per row the k smallest with their query bins): the squared distances of a
// vocabulary row to a query's bins never leave the registers of the thread that owns the
// row, which keeps the KT smallest (value, bin) pairs and writes only the table (z =
// square root, w = the bin's weight).
//
// Work item = (vocabulary row tile, query group) as in k_tc_dist_batch, same operand
// panels, copies, MMA order and epilogue arithmetic, so every squared distance is
// bit-identical to the batched matrix kernel's (and the exact zero of an identical
// vocabulary id is applied to the same entry).  The item's column tiles run in two
// streams: each query belongs to one stream, a stream takes the group's next query when
// its current one is done, and tiles are issued alternately from the two streams.  Stream
// s has TMEM accumulator buffer s and epilogue warpgroup s (warps 2+4s .. 5+4s, one per
// TMEM lane quarter), so all tiles of a query reach the same 128 threads and a row's list
// lives in one thread for the whole query: no merge across threads.  A thread sees its
// row's columns in increasing bin order and inserts only strictly smaller values, so ties
// keep the lower bin -- the order the table kernel applies to the matrix.
constexpr int TCT_THREADS = 64 + 32 * 16;  // copy warp, MMA warp, two epilogue warpgroups per stream

// The interleaved two-stream tile order of one work item (every role walks it alike).
// Scalar fields (no arrays indexed at run time, which would live in local memory).
struct TileSeq {
    int qb, nextq, cq0, cq1, c0, c1, turn, bn;
    __device__ __forceinline__ void init(int qa, int qb_, int bn_ = TC_BN)
    {
        bn = bn_;
        qb = qb_;
        nextq = qa;
        cq0 = cq1 = -1;
        c0 = c1 = 0;
        turn = 0;
    }
    // Next tile (query q, first column n0, stream s); false when the item is done.
    __device__ __forceinline__ bool next(const QDesc* __restrict__ qd, int& q, int& n0, int& s)
    {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int st = turn ^ t;
            int cq = st ? cq1 : cq0, c = st ? c1 : c0;
            if (cq < 0 && nextq < qb) {
                cq = nextq++;
                c = 0;
            }
            if (cq >= 0) {
                q = cq;
                n0 = c;
                s = st;
                c += bn;
                if (c >= qd[cq].h) cq = -1;
                if (st) { cq1 = cq; c1 = c; } else { cq0 = cq; c0 = c; }
                turn = st ^ 1;
                return true;
            }
            if (st) { cq1 = cq; c1 = c; } else { cq0 = cq; c0 = c; }
        }
        return false;
    }
};

// Sorted insertion of (d, j) into the KT smallest; strict '<' keeps the earlier bin first.
template <int KT>
__device__ __forceinline__ void tc_insert(float (&z)[KT], int (&s)[KT], float d, int j)
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

// Insertion by (value, bin): merging two lists whose bins interleave keeps the k smallest
// pairs of their union, the set a scan of all columns in bin order keeps.
template <int KT>
__device__ __forceinline__ void tc_insert_key(float (&z)[KT], int (&s)[KT], float d, int j)
{
    bool p[KT];
#pragma unroll
    for (int l = 0; l < KT; ++l) p[l] = d < z[l] || (d == z[l] && j < s[l]);
#pragma unroll
    for (int l = KT - 1; l > 0; --l) {
        z[l] = p[l - 1] ? z[l - 1] : (p[l] ? d : z[l]);
        s[l] = p[l - 1] ? s[l - 1] : (p[l] ? j : s[l]);
    }
    z[0] = p[0] ? d : z[0];
    s[0] = p[0] ? j : s[0];
}

// CAND (approximate formats): instead of the table, each row's kc = qd[q].kc smallest
// approximate values are kept and written as candidate bins (cbin, kCandPerRow per row)
// with the kc-th approximate value (camax; +inf when every bin is a candidate), for the
// exact re-rank and its certificate.
template <int FMT, int KT, bool CAND>
__global__ void __launch_bounds__(TCT_THREADS, 1)
k_tc_table_batch(const uint8_t* __restrict__ A_hi, const uint8_t* __restrict__ A_lo, int64_t Mpad,
                 const float* __restrict__ a_scale, const float* __restrict__ a_norm, int64_t M,
                 const QDesc* __restrict__ qd, const int* __restrict__ nq_dev, int groups, int KC, int stages,
                 int klast, int* __restrict__ err)
{
    constexpr bool SPLIT = FMT == TC_SPLIT;
    constexpr uint32_t EB = TcFmt<FMT>::EB;
    constexpr int kParts = (int)TcFmt<FMT>::parts;
    constexpr uint32_t kABytes = TC_BM * EB;
    constexpr uint32_t kBBytes = TC_BN * EB;
    constexpr uint32_t kSbo = 8 * EB;
    constexpr uint32_t kAChunk = kParts * kABytes;
    constexpr uint32_t kBStage = kParts * kBBytes;
    constexpr uint32_t kAcc = SPLIT ? 256 : 128;
    constexpr uint32_t kCols = 2 * kAcc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* apanel = smem;
    uint8_t* bring = apanel + (size_t)KC * kAChunk;
    uint64_t* full = reinterpret_cast<uint64_t*>(bring + (size_t)stages * kBStage);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;   // [2] stream s's accumulator ready
    uint64_t* tempty = tfull + 2;       // [2] stream s's accumulator drained (4 warps)
    uint64_t* afull = tempty + 2;
    uint64_t* afree = afull + 1;
    uint64_t* xbar = afree + 1;         // [2][4] per stream and lane quarter: the upper half's list is in TMEM
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xbar + 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = *nq_dev;
    const int m_tiles = (int)(Mpad / TC_BM);
    const int total = m_tiles * groups;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(afull, 1);
        mbar_init(afree, 1);
        for (int x = 0; x < 8; ++x) mbar_init(&xbar[x], 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
    };
    auto qrange = [&](int g, int& qa, int& qb) {
        qa = (int)((int64_t)g * nq / groups);
        qb = (int)((int64_t)(g + 1) * nq / groups);
    };

    if (warp == 0 && lane == 0) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int items = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x, ++items) {
            const int64_t m0 = (int64_t)(w % m_tiles) * TC_BM;
            if (items > 0 && !mbar_wait(afree, (uint32_t)(items - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            mbar_expect_tx(afull, (uint32_t)KC * kAChunk);
            for (int c = 0; c < KC; ++c) {
                uint8_t* ast = apanel + (size_t)c * kAChunk;
                bulk_g2s(ast, A_hi + ((int64_t)c * Mpad + m0) * EB, kABytes, afull);
                if (SPLIT) bulk_g2s(ast + kABytes, A_lo + ((int64_t)c * Mpad + m0) * EB, kABytes, afull);
            }
            int qa, qb, q, n0, s;
            qrange(w / m_tiles, qa, qb);
            TileSeq ts;
            ts.init(qa, qb);
            while (ok && ts.next(qd, q, n0, s)) {
                const QDesc& d = qd[q];
                const int Nt = min(TC_BN, (int)round_up(d.h - n0, 16));
                const uint32_t b_bytes = (uint32_t)Nt * EB;
                const uint8_t* bh = static_cast<const uint8_t*>(d.q_hi);
                const uint8_t* bl = static_cast<const uint8_t*>(d.q_lo);
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int st = rs;
                    if (gb >= stages &&
                        !mbar_wait(&empty[st], rp ^ 1u, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* bst = bring + (size_t)st * kBStage;
                    mbar_expect_tx(&full[st], (uint32_t)kParts * b_bytes);
                    bulk_g2s(bst, bh + ((int64_t)c * d.npad + n0) * EB, b_bytes, &full[st]);
                    if (SPLIT) bulk_g2s(bst + kBBytes, bl + ((int64_t)c * d.npad + n0) * EB, b_bytes, &full[st]);
                }
            }
        }
        const uint64_t tail = global_ns() + TC_TIMEOUT_NS;
        for (int64_t c = gb > stages ? gb - stages : 0; c < gb; ++c)
            if (!mbar_wait(&full[c % stages], (uint32_t)(c / stages) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
        if (items > 0 && !mbar_wait(afull, (uint32_t)(items - 1) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int cnt0 = 0, cnt1 = 0, items = 0;  // tiles issued per stream
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x, ++items) {
            if (!mbar_wait(afull, (uint32_t)items & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            int qa, qb, q, n0, s;
            qrange(w / m_tiles, qa, qb);
            TileSeq ts;
            ts.init(qa, qb);
            while (ok && ts.next(qd, q, n0, s)) {
                const int Nt = min(TC_BN, (int)round_up(qd[q].h - n0, 16));
                const uint32_t idesc = (1u << 4) | (TcFmt<FMT>::atype << 7) | (TcFmt<FMT>::atype << 10) |
                                       ((uint32_t)(Nt >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
                const int cs = s ? cnt1 : cnt0;
                if (cs >= 1 && !mbar_wait(&tempty[s], (uint32_t)(cs - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc0 = tmem + (uint32_t)s * kAcc;
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int st = rs;
                    if (!mbar_wait(&full[st], rp, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(apanel + (size_t)c * kAChunk);
                    const uint32_t sa_lo = sa + kABytes;
                    const uint32_t sb = smem_u32(bring + (size_t)st * kBStage);
                    const uint32_t sb_lo = sb + kBBytes;
                    // descriptors of the chunk's first K step; a step of 16 elements (256 B) adds 16 to the
                    // address field (addresses stay below 2^18, so no carry leaves the 14-bit field)
                    const uint64_t dA0 = smem_desc(sa, kSbo), dB0 = smem_desc(sb, kSbo);
                    const uint64_t dAl0 = smem_desc(sa_lo, kSbo), dBl0 = smem_desc(sb_lo, kSbo);
#pragma unroll
                    for (int ks = 0; ks < (int)TcFmt<FMT>::mmas; ++ks) {
                        if (c == KC - 1 && ks >= klast) break;  // the last chunk's zero K steps
                        const uint32_t ko = (uint32_t)ks * 256u;
                        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                        const uint64_t kd = (uint64_t)(ko >> 4);
                        const uint64_t da = dA0 + kd, db = dB0 + kd;
                        mma_issue<FMT>(acc0, da, db, idesc, acc);
                        if (SPLIT) {
                            mma_issue<FMT>(acc0 + 128, da, dBl0 + kd, idesc, acc);
                            mma_issue<FMT>(acc0 + 128, dAl0 + kd, db, idesc, 1u);
                        }
                    }
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&tfull[s]);
                if (s) ++cnt1; else ++cnt0;
            }
            mma_commit(afree);
        }
    } else if (warp >= 2) {
        // epilogue: stream sme = warps 2 + 8 sme .. 9 + 8 sme; warp w reads TMEM lane quarter
        // w % 4; the lower four take columns 0..63 of each tile, the upper four 64..127
        const int ew = warp - 2;
        const int qw4 = warp & 3;
        const int sme = ew >> 3;
        const int half = (ew >> 2) & 1;
        const int cb0 = half * (TC_BN / 2);
        const int row = qw4 * 32 + lane;
        uint64_t* xb = &xbar[sme * 4 + qw4];
        int cnt = 0, nx = 0;
        bool ok = true;
        float z[KT];
        int sj[KT];
        int jstar = -1;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
            const int64_t m0 = (int64_t)(w % m_tiles) * TC_BM;
            const int64_t u = m0 + row;
            const bool row_ok = u < M;
            const float su = row_ok ? a_scale[u] : 0.f;
            const float nu = row_ok ? a_norm[u] : 0.f;
            int qa, qb, q, n0, s;
            qrange(w / m_tiles, qa, qb);
            TileSeq ts;
            ts.init(qa, qb);
            while (ok && ts.next(qd, q, n0, s)) {
                if (s != sme) continue;
                const QDesc& d = qd[q];
                const int N = d.h;
                const int Nt = min(TC_BN, (int)round_up(N - n0, 16));
                if (n0 == 0) {
#pragma unroll
                    for (int l = 0; l < KT; ++l) {
                        z[l] = INFINITY;
                        sj[l] = INT32_MAX;
                    }
                    // the query bin of this row's own vocabulary id, if any: its squared distance is 0
                    jstar = row_ok ? d.qpos[u] : -1;
                }
                // lane l holds the constants of columns n0 + cb0 + 32 c + l, broadcast by shuffles
                float cbl[2], nbl[2];
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2) {
                    const int col = n0 + cb0 + 32 * c2 + lane;
                    const bool cok = col < N;
                    cbl[c2] = cok ? -2.f * d.q_scale[col] : 0.f;
                    nbl[c2] = cok ? d.qnorm[col] : 0.f;
                }
                if (!mbar_wait(&tfull[sme], (uint32_t)cnt & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem + (uint32_t)sme * kAcc + ((uint32_t)(qw4 * 32) << 16);
#pragma unroll
                for (int cc = 0; cc < TC_BN / 2; cc += 16) {
                    if (cb0 + cc < Nt) {
                        uint32_t r0[16], r1[16];
                        tmem_ld16(tbase + (uint32_t)(cb0 + cc), r0);
                        if (SPLIT) tmem_ld16(tbase + 128u + (uint32_t)(cb0 + cc), r1);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int jc = cc + e;
                            const float cb = __shfl_sync(0xffffffffu, cbl[jc >> 5], jc & 31);
                            const float nb = __shfl_sync(0xffffffffu, nbl[jc >> 5], jc & 31);
                            float dot = __uint_as_float(r0[e]);
                            if (SPLIT) dot = fmaf(__uint_as_float(r1[e]), 1.0f / 2048.0f, dot);
                            const int j = n0 + cb0 + jc;
                            float d2 = fmaf(cb * su, dot, nu + nb);  // as k_tc_dist_batch writes it
                            d2 = j == jstar ? 0.f : d2;
                            if (j < N && d2 < z[KT - 1]) tc_insert<KT>(z, sj, d2, j);
                        }
                    }
                }
                const bool last = n0 + TC_BN >= N;
                if (last && N > TC_BN / 2) {
                    // the query's last tile: the upper half hands its list to the lower half
                    // through its own (already drained) TMEM columns cb0 .. cb0 + 31
                    if (half == 1) {
                        uint32_t x[32];
#pragma unroll
                        for (int l = 0; l < 16; ++l) {
                            x[l] = __float_as_uint(l < KT ? z[l < KT ? l : 0] : INFINITY);
                            x[16 + l] = (uint32_t)(l < KT ? sj[l < KT ? l : 0] : INT32_MAX);
                        }
                        tmem_st32(tbase + (uint32_t)cb0, x);
                        tmem_wait_st();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(xb);
                    } else {
                        if (!mbar_wait(xb, (uint32_t)nx & 1u, global_ns() + TC_TIMEOUT_NS)) {
                            fail();
                            ok = false;
                        } else {
                            tc_fence_after();
                            uint32_t x[32];
                            tmem_ld32(tbase + (uint32_t)(TC_BN / 2), x);
                            tmem_wait_ld();
#pragma unroll
                            for (int l = 0; l < KT; ++l)
                                tc_insert_key<KT>(z, sj, __uint_as_float(x[l]), (int)x[16 + l]);
                        }
                    }
                    ++nx;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[sme]);
                ++cnt;
                if (!ok) break;
                if (last && half == 0 && row_ok) {  // write the query's table row
                    if (CAND) {
                        const int kc = d.kc;
#pragma unroll
                        for (int l = 0; l < KT; ++l)
                            if (l < kc) d.cbin[u * kCandPerRow + l] = sj[l];
                        float zc = z[0];
#pragma unroll
                        for (int l = 1; l < KT; ++l) zc = l == kc - 1 ? z[l] : zc;
                        d.camax[u] = kc < N ? zc : INFINITY;
                    } else {
#pragma unroll
                        for (int l = 0; l < KT; ++l) {
                            if (l < d.tk) {
                                const bool valid = sj[l] != INT32_MAX;
                                d.tab[u * d.tab_rs + (int64_t)l * d.tab_es] =
                                    make_float2(valid ? sq_to_dist(z[l]) : INFINITY, valid ? d.qw[sj[l]] : 0.f);
                            }
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// ------------------------------------------------------------------ fused table on SM pairs
//
// The fused Phase-1 table of k_tc_table_batch on a cluster of two CTAs (two SMs) issuing
// tcgen05.mma.cta_group::2: M = 256 vocabulary rows per product, each CTA holding its own 128
// rows in shared memory and its own TMEM accumulators, and half of each query chunk's columns
// -- the pair's tensor cores read the other half from the peer CTA's shared memory.  Each SM
// therefore stages half the query bytes per product of the single-CTA form, and twice as
// many chunk stages fit beside the resident vocabulary panel; that ring, not the tensor pipe,
// bounds the single-CTA form.  Per CTA the arithmetic of a row is unchanged (same operands,
// K order, accumulator split and epilogue), so the tables are bit-identical to it.
//
// Roles in both CTAs: warp 0 lane 0 copies this CTA's vocabulary rows and its half of each
// chunk; warp 1 allocates TMEM for the pair; warps 2..9 drain this CTA's accumulators (two
// tile streams as in k_tc_table_batch).  In the leader (rank 0) warp 1 lane 0 issues the
// pair's MMAs and commits to both CTAs' barriers; in the peer it forwards the completion of
// its own copies to the leader (an arrive on the leader's barrier after its local wait).  The
// peer's epilogue warps release an accumulator with arrives on the leader's barrier.  Every
// wait is bounded; both CTAs meet at a cluster barrier before TMEM is released and before
// either exits, so no remote arrive targets a finished CTA.
constexpr int TCP_THREADS = 64 + 32 * 8;

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared::cluster address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// A wait on a barrier that the peer CTA arrives on (acquire at cluster scope).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, uint64_t deadline)
{
    while (!mbar_try_wait_cluster(bar, parity))
        if (global_ns() > deadline) return false;
    return true;
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_issue_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                               uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the barrier at this offset in both CTAs once the pair's MMAs so far are done.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// BN: the pair's largest column tile (64 or 128); each CTA stages BN / 2 columns of a chunk.
template <int KT, int BN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TCP_THREADS, 1)
k_tc_table_pair(const uint8_t* __restrict__ A_hi, const uint8_t* __restrict__ A_lo, int64_t Mpad,
                const float* __restrict__ a_scale, const float* __restrict__ a_norm, int64_t M,
                const QDesc* __restrict__ qd, const int* __restrict__ nq_dev, int groups, int KC, int stages,
                int klast, int* __restrict__ err)
{
    constexpr uint32_t EB = 128;  // FP16 split: bytes of a 64-element row segment
    constexpr uint32_t kABytes = TC_BM * EB;
    constexpr uint32_t kBBytes = (BN / 2) * EB;
    constexpr uint32_t kSbo = 8 * EB;
    constexpr uint32_t kAChunk = 2 * kABytes;
    constexpr uint32_t kBStage = 2 * kBBytes;
    constexpr uint32_t kAcc = 2 * BN;  // per stream: hi.hi, then the cross terms
    constexpr uint32_t kCols = 2 * kAcc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* apanel = smem;
    uint8_t* bring = apanel + (size_t)KC * kAChunk;
    uint64_t* full = reinterpret_cast<uint64_t*>(bring + (size_t)stages * kBStage);  // own copies landed
    uint64_t* pfull = full + stages;    // leader: the peer's copies of the stage landed
    uint64_t* empty = pfull + stages;   // the pair's MMAs on the stage done (both CTAs)
    uint64_t* tfull = empty + stages;   // [2] stream s's accumulators ready (both CTAs)
    uint64_t* tempty = tfull + 2;       // [2] leader: stream s drained by 8 warps of the pair
    uint64_t* afull = tempty + 2;       // own vocabulary rows landed
    uint64_t* pafull = afull + 1;       // leader: the peer's rows landed
    uint64_t* afree = pafull + 1;       // the pair's MMAs on the item done (both CTAs)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(afree + 1);
    uint32_t* peer_tmem = tmem_slot + 1;  // leader: the peer's TMEM address
    volatile int* abort_flag = reinterpret_cast<volatile int*>(peer_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int nq = *nq_dev;
    const int pairs = (int)(Mpad / (2 * TC_BM));
    const int total = pairs * groups;
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&pfull[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(afull, 1);
        mbar_init(pafull, 1);
        mbar_init(afree, 1);
        *peer_tmem = 0xFFFFFFFFu;
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, kCols);
    tc_fence_before();
    cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated in both
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the pair must hold its accumulators at the same TMEM address: each CTA hands its own to
    // the other, and both skip every role (issuing nothing) when they differ
    if (threadIdx.x == 0) {
        const uint32_t dst = peer_addr(peer_tmem, rank ^ 1u);
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(dst), "r"(tmem) : "memory");
    }
    cluster_sync_all();
    const bool pair_ok = *peer_tmem == tmem;
    if (!pair_ok && threadIdx.x == 0 && rank == 0) atomicOr(err, ERR_PAIR_TMEM);

    auto fail = [&]() {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
    };
    auto qrange = [&](int g, int& qa, int& qb) {
        qa = (int)((int64_t)g * nq / groups);
        qb = (int)((int64_t)(g + 1) * nq / groups);
    };
    if (warp == 0 && lane == 0 && pair_ok) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int items = 0;
        bool ok = true;
        for (int w = cid; w < total && ok && !*abort_flag; w += ncl, ++items) {
            const int64_t m0 = (int64_t)(w % pairs) * (2 * TC_BM) + (int64_t)rank * TC_BM;
            if (items > 0 && !mbar_wait_cluster(afree, (uint32_t)(items - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            mbar_expect_tx(afull, (uint32_t)KC * kAChunk);
            for (int c = 0; c < KC; ++c) {
                uint8_t* ast = apanel + (size_t)c * kAChunk;
                bulk_g2s(ast, A_hi + ((int64_t)c * Mpad + m0) * EB, kABytes, afull);
                bulk_g2s(ast + kABytes, A_lo + ((int64_t)c * Mpad + m0) * EB, kABytes, afull);
            }
            int qa, qb, q, n0, s;
            qrange(w / pairs, qa, qb);
            TileSeq ts;
            ts.init(qa, qb, BN);
            while (ok && ts.next(qd, q, n0, s)) {
                const QDesc& d = qd[q];
                const int Nt = min(BN, (int)round_up(d.h - n0, 16));
                const int nh = Nt >> 1;  // this CTA's columns: n0 + rank * nh ..
                const uint32_t b_bytes = (uint32_t)nh * EB;
                const int64_t c0 = n0 + (int64_t)rank * nh;
                const uint8_t* bh = static_cast<const uint8_t*>(d.q_hi);
                const uint8_t* bl = static_cast<const uint8_t*>(d.q_lo);
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int st = rs;
                    if (gb >= stages && !mbar_wait_cluster(&empty[st], rp ^ 1u,
                                                           global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* bst = bring + (size_t)st * kBStage;
                    mbar_expect_tx(&full[st], 2u * b_bytes);
                    bulk_g2s(bst, bh + ((int64_t)c * d.npad + c0) * EB, b_bytes, &full[st]);
                    bulk_g2s(bst + kBBytes, bl + ((int64_t)c * d.npad + c0) * EB, b_bytes, &full[st]);
                }
            }
        }
        const uint64_t tail = global_ns() + TC_TIMEOUT_NS;
        for (int64_t c = gb > stages ? gb - stages : 0; c < gb; ++c)
            if (!mbar_wait(&full[c % stages], (uint32_t)(c / stages) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
        if (items > 0 && !mbar_wait(afull, (uint32_t)(items - 1) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
    } else if (warp == 1 && lane == 0 && rank == 1 && pair_ok) {
        // peer: forward the completion of its own copies to the leader, in the copy order
        const uint32_t r_pfull = peer_addr(pfull, 0), r_pafull = peer_addr(pafull, 0);
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int items = 0;
        bool ok = true;
        for (int w = cid; w < total && ok && !*abort_flag; w += ncl, ++items) {
            if (!mbar_wait(afull, (uint32_t)items & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            mbar_arrive_cluster(r_pafull);
            int qa, qb, q, n0, s;
            qrange(w / pairs, qa, qb);
            TileSeq ts;
            ts.init(qa, qb, BN);
            while (ok && ts.next(qd, q, n0, s)) {
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int st = rs;
                    if (!mbar_wait(&full[st], rp, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(r_pfull + (uint32_t)st * 8u);
                }
            }
        }
    } else if (warp == 1 && lane == 0 && rank == 0 && pair_ok) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int cnt0 = 0, cnt1 = 0, items = 0;  // tiles issued per stream
        bool ok = true;
        for (int w = cid; w < total && ok && !*abort_flag; w += ncl, ++items) {
            if (!mbar_wait(afull, (uint32_t)items & 1u, global_ns() + TC_TIMEOUT_NS) ||
                !mbar_wait_cluster(pafull, (uint32_t)items & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            int qa, qb, q, n0, s;
            qrange(w / pairs, qa, qb);
            TileSeq ts;
            ts.init(qa, qb, BN);
            while (ok && ts.next(qd, q, n0, s)) {
                const int Nt = min(BN, (int)round_up(qd[q].h - n0, 16));
                const uint32_t idesc = (1u << 4) | ((uint32_t)(Nt >> 3) << 17) | ((uint32_t)((2 * TC_BM) >> 4) << 24);
                const int cs = s ? cnt1 : cnt0;
                if (cs >= 1 &&
                    !mbar_wait_cluster(&tempty[s], (uint32_t)(cs - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc0 = tmem + (uint32_t)s * kAcc;
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int st = rs;
                    if (!mbar_wait(&full[st], rp, global_ns() + TC_TIMEOUT_NS) ||
                        !mbar_wait_cluster(&pfull[st], rp, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(apanel + (size_t)c * kAChunk);
                    const uint32_t sa_lo = sa + kABytes;
                    const uint32_t sb = smem_u32(bring + (size_t)st * kBStage);
                    const uint32_t sb_lo = sb + kBBytes;
                    // descriptors of the chunk's first K step; a step of 16 elements (256 B) adds 16 to the
                    // address field (addresses stay below 2^18, so no carry leaves the 14-bit field)
                    const uint64_t dA0 = smem_desc(sa, kSbo), dB0 = smem_desc(sb, kSbo);
                    const uint64_t dAl0 = smem_desc(sa_lo, kSbo), dBl0 = smem_desc(sb_lo, kSbo);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        if (c == KC - 1 && ks >= klast) break;  // the last chunk's zero K steps
                        const uint32_t ko = (uint32_t)ks * 256u;
                        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                        const uint64_t kd = (uint64_t)(ko >> 4);
                        const uint64_t da = dA0 + kd, db = dB0 + kd;
                        mma_issue_pair(acc0, da, db, idesc, acc);
                        mma_issue_pair(acc0 + BN, da, dBl0 + kd, idesc, acc);
                        mma_issue_pair(acc0 + BN, dAl0 + kd, db, idesc, 1u);
                    }
                    mma_commit_pair(&empty[st]);
                }
                if (!ok) break;
                mma_commit_pair(&tfull[s]);
                if (s) ++cnt1; else ++cnt0;
            }
            mma_commit_pair(afree);
        }
    } else if (warp >= 2 && pair_ok) {
        // epilogue: warpgroup sme = stream sme; warp w reads TMEM lane quarter w % 4
        const int qw4 = warp & 3;
        const int sme = (warp - 2) >> 2;
        const int row = qw4 * 32 + lane;
        const uint32_t r_tempty = rank == 0 ? smem_u32(&tempty[sme]) : peer_addr(&tempty[sme], 0);
        int cnt = 0;
        bool ok = true;
        float z[KT];
        int sj[KT];
        int jstar = -1;
        for (int w = cid; w < total && ok && !*abort_flag; w += ncl) {
            const int64_t m0 = (int64_t)(w % pairs) * (2 * TC_BM) + (int64_t)rank * TC_BM;
            const int64_t u = m0 + row;
            const bool row_ok = u < M;
            const float su = row_ok ? a_scale[u] : 0.f;
            const float nu = row_ok ? a_norm[u] : 0.f;
            int qa, qb, q, n0, s;
            qrange(w / pairs, qa, qb);
            TileSeq ts;
            ts.init(qa, qb, BN);
            while (ok && ts.next(qd, q, n0, s)) {
                if (s != sme) continue;
                const QDesc& d = qd[q];
                const int N = d.h;
                const int Nt = min(BN, (int)round_up(N - n0, 16));
                if (n0 == 0) {
#pragma unroll
                    for (int l = 0; l < KT; ++l) {
                        z[l] = INFINITY;
                        sj[l] = INT32_MAX;
                    }
                    // the query bin of this row's own vocabulary id, if any: its squared distance is 0
                    jstar = row_ok ? d.qpos[u] : -1;
                }
                // lane l holds the constants of columns n0 + 32 c + l, broadcast by shuffles
                float cbl[BN / 32], nbl[BN / 32];
#pragma unroll
                for (int c4 = 0; c4 < BN / 32; ++c4) {
                    const int col = n0 + 32 * c4 + lane;
                    const bool cok = col < N;
                    cbl[c4] = cok ? -2.f * d.q_scale[col] : 0.f;
                    nbl[c4] = cok ? d.qnorm[col] : 0.f;
                }
                if (!mbar_wait_cluster(&tfull[sme], (uint32_t)cnt & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem + (uint32_t)sme * kAcc + ((uint32_t)(qw4 * 32) << 16);
#pragma unroll
                for (int cc = 0; cc < BN; cc += 16) {
                    if (cc < Nt) {
                        uint32_t r0[16], r1[16];
                        tmem_ld16(tbase + (uint32_t)cc, r0);
                        tmem_ld16(tbase + (uint32_t)BN + (uint32_t)cc, r1);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int jc = cc + e;
                            const float cb = __shfl_sync(0xffffffffu, cbl[jc >> 5], jc & 31);
                            const float nb = __shfl_sync(0xffffffffu, nbl[jc >> 5], jc & 31);
                            float dot = __uint_as_float(r0[e]);
                            dot = fmaf(__uint_as_float(r1[e]), 1.0f / 2048.0f, dot);
                            const int j = n0 + jc;
                            float d2 = fmaf(cb * su, dot, nu + nb);  // as k_tc_dist_batch writes it
                            d2 = j == jstar ? 0.f : d2;
                            if (j < N && d2 < z[KT - 1]) tc_insert<KT>(z, sj, d2, j);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(r_tempty);
                ++cnt;
                if (n0 + BN >= N && row_ok) {  // the query's last tile: write its table row
#pragma unroll
                    for (int l = 0; l < KT; ++l) {
                        if (l < d.tk) {
                            const bool valid = sj[l] != INT32_MAX;
                            d.tab[u * d.tab_rs + (int64_t)l * d.tab_es] =
                                make_float2(valid ? sq_to_dist(z[l]) : INFINITY, valid ? d.qw[sj[l]] : 0.f);
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // no remote arrive may reach a CTA that has left
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, kCols);
    }
}

// ------------------------------------------------------------------ candidate-row block
//
// The reverse direction of the fused pruned path needs D only on the used rows of the
// candidate documents.  Their packed panel rows are gathered (k_cand_pack_b) and this
// kernel computes their squared distances to the query's bins with the same operands, MMA
// order and epilogue as k_tc_dist_batch, so each entry equals the full matrix's entry.
// Work item = (query q, 128-row tile r of q's candidate rows); items past a query's row
// count are skipped by every role alike.
template <int FMT>
__global__ void __launch_bounds__(TCB_THREADS, 1)
k_tc_cand_batch(const QDesc* __restrict__ qd, const int* __restrict__ nq_dev, int max_q, int KC, int stages,
                int* __restrict__ err)
{
    constexpr bool SPLIT = FMT == TC_SPLIT;
    constexpr uint32_t EB = TcFmt<FMT>::EB;
    constexpr int kParts = (int)TcFmt<FMT>::parts;
    constexpr uint32_t kABytes = TC_BM * EB;
    constexpr uint32_t kBBytes = TC_BN * EB;
    constexpr uint32_t kSbo = 8 * EB;
    constexpr uint32_t kAChunk = kParts * kABytes;
    constexpr uint32_t kBStage = kParts * kBBytes;
    constexpr uint32_t kAcc = SPLIT ? 256 : 128;
    constexpr uint32_t kCols = 2 * kAcc;
    constexpr int kRT = kCandRows / TC_BM;  // row tiles per query
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* apanel = smem;
    uint8_t* bring = apanel + (size_t)KC * kAChunk;
    uint64_t* full = reinterpret_cast<uint64_t*>(bring + (size_t)stages * kBStage);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* afull = tempty + 2;
    uint64_t* afree = afull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(afree + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = *nq_dev;
    const int total = max_q * kRT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], TCB_EPI_WARPS);
        }
        mbar_init(afull, 1);
        mbar_init(afree, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
    };
    // rows of item w (0 when the item is past its query's candidate rows)
    auto item_rows = [&](int w) -> int {
        const int q = w / kRT, r = w % kRT;
        if (q >= nq) return 0;
        const int nr = min(*qd[q].ncrows, kCandRows);
        return max(0, min(TC_BM, nr - r * TC_BM));
    };

    if (warp == 0 && lane == 0) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int items = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
            if (item_rows(w) == 0) continue;
            const QDesc& d = qd[w / kRT];
            const int64_t m0 = (int64_t)(w % kRT) * TC_BM;
            if (items > 0 && !mbar_wait(afree, (uint32_t)(items - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            const uint8_t* ah = static_cast<const uint8_t*>(d.c_hi);
            const uint8_t* al = static_cast<const uint8_t*>(d.c_lo);
            mbar_expect_tx(afull, (uint32_t)KC * kAChunk);
            for (int c = 0; c < KC; ++c) {
                uint8_t* ast = apanel + (size_t)c * kAChunk;
                bulk_g2s(ast, ah + ((int64_t)c * kCandRows + m0) * EB, kABytes, afull);
                if (SPLIT) bulk_g2s(ast + kABytes, al + ((int64_t)c * kCandRows + m0) * EB, kABytes, afull);
            }
            ++items;
            const uint8_t* bh = static_cast<const uint8_t*>(d.qs_hi);
            const uint8_t* bl = static_cast<const uint8_t*>(d.qs_lo);
            for (int n0 = 0; n0 < d.h && ok; n0 += TC_BN) {
                const int Nt = min(TC_BN, (int)round_up(d.h - n0, 16));
                const uint32_t b_bytes = (uint32_t)Nt * EB;
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int s = rs;
                    if (gb >= stages &&
                        !mbar_wait(&empty[s], rp ^ 1u, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* bst = bring + (size_t)s * kBStage;
                    mbar_expect_tx(&full[s], (uint32_t)kParts * b_bytes);
                    bulk_g2s(bst, bh + ((int64_t)c * d.npad + n0) * EB, b_bytes, &full[s]);
                    if (SPLIT) bulk_g2s(bst + kBBytes, bl + ((int64_t)c * d.npad + n0) * EB, b_bytes, &full[s]);
                }
            }
        }
        const uint64_t tail = global_ns() + TC_TIMEOUT_NS;
        for (int64_t c = gb > stages ? gb - stages : 0; c < gb; ++c)
            if (!mbar_wait(&full[c % stages], (uint32_t)(c / stages) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
        if (items > 0 && !mbar_wait(afull, (uint32_t)(items - 1) & 1u, tail)) atomicOr(err, ERR_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        int64_t gb = 0;
        int rs = 0;          // ring stage gb % stages
        uint32_t rp = 0;     // its round's parity (gb / stages) & 1
        int it = 0, items = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
            if (item_rows(w) == 0) continue;
            const int h = qd[w / kRT].h;
            if (!mbar_wait(afull, (uint32_t)items & 1u, global_ns() + TC_TIMEOUT_NS)) {
                fail();
                break;
            }
            ++items;
            for (int n0 = 0; n0 < h && ok; n0 += TC_BN, ++it) {
                const int Nt = min(TC_BN, (int)round_up(h - n0, 16));
                const uint32_t idesc = (1u << 4) | (TcFmt<FMT>::atype << 7) | (TcFmt<FMT>::atype << 10) |
                                       ((uint32_t)(Nt >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
                const int buf = it & 1;
                if (it >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((it >> 1) - 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc0 = tmem + (uint32_t)buf * kAcc;
                for (int c = 0; c < KC; ++c, ++gb, rs = rs + 1 == stages ? (rp ^= 1u, 0) : rs + 1) {
                    const int s = rs;
                    if (!mbar_wait(&full[s], rp, global_ns() + TC_TIMEOUT_NS)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(apanel + (size_t)c * kAChunk);
                    const uint32_t sa_lo = sa + kABytes;
                    const uint32_t sb = smem_u32(bring + (size_t)s * kBStage);
                    const uint32_t sb_lo = sb + kBBytes;
                    // descriptors of the chunk's first K step; a step of 16 elements (256 B) adds 16 to the
                    // address field (addresses stay below 2^18, so no carry leaves the 14-bit field)
                    const uint64_t dA0 = smem_desc(sa, kSbo), dB0 = smem_desc(sb, kSbo);
                    const uint64_t dAl0 = smem_desc(sa_lo, kSbo), dBl0 = smem_desc(sb_lo, kSbo);
#pragma unroll
                    for (int ks = 0; ks < (int)TcFmt<FMT>::mmas; ++ks) {
                        const uint32_t ko = (uint32_t)ks * 256u;
                        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                        const uint64_t kd = (uint64_t)(ko >> 4);
                        const uint64_t da = dA0 + kd, db = dB0 + kd;
                        mma_issue<FMT>(acc0, da, db, idesc, acc);
                        if (SPLIT) {
                            mma_issue<FMT>(acc0 + 128, da, dBl0 + kd, idesc, acc);
                            mma_issue<FMT>(acc0 + 128, dAl0 + kd, db, idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[buf]);
            }
            mma_commit(afree);
        }
    } else if (warp >= 2) {
        const int qw4 = warp & 3;
        const int cc = ((warp - 2) >> 2) * 32;
        const int row = qw4 * 32 + lane;
        int it = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
            const int nr = item_rows(w);
            if (nr == 0) continue;
            const QDesc& d = qd[w / kRT];
            const int64_t u = (int64_t)(w % kRT) * TC_BM + row;  // candidate row
            const bool row_ok = row < nr;
            const float su = row_ok ? d.c_scale[u] : 0.f;
            const float nu = row_ok ? d.c_norm[u] : 0.f;
            const int jstar = row_ok ? d.qpos[d.crows[u]] : -1;
            const int N = d.h, ldd = d.ldd;
            for (int n0 = 0; n0 < N; n0 += TC_BN, ++it) {
                const int Nt = min(TC_BN, (int)round_up(N - n0, 16));
                const int buf = it & 1;
                const int lcol = n0 + cc + lane;
                const bool lok = lcol < N;
                const float cb_l = lok ? -2.f * d.qs_scale[lcol] : 0.f;
                const float nb_l = lok ? d.qnorm[lcol] : 0.f;
                if (!mbar_wait(&tfull[buf], (uint32_t)(it >> 1) & 1u, global_ns() + TC_TIMEOUT_NS)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (cc < Nt) {
                    const uint32_t tbase = tmem + (uint32_t)buf * kAcc + ((uint32_t)(qw4 * 32) << 16);
                    float* out = d.Dc + (row_ok ? u : 0) * ldd + n0 + cc;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        uint32_t r0[16], r1[16];
                        tmem_ld16(tbase + (uint32_t)(cc + 16 * hh), r0);
                        if (SPLIT) tmem_ld16(tbase + 128u + (uint32_t)(cc + 16 * hh), r1);
                        tmem_wait_ld();
#pragma unroll
                        for (int e4 = 4 * hh; e4 < 4 * hh + 4; ++e4) {
                            float o[4];
#pragma unroll
                            for (int tt = 0; tt < 4; ++tt) {
                                const int e = e4 * 4 + tt;
                                const int er = e - 16 * hh;
                                const float cb = __shfl_sync(0xffffffffu, cb_l, e);
                                const float nb = __shfl_sync(0xffffffffu, nb_l, e);
                                float dot = __uint_as_float(r0[er]);
                                if (SPLIT) dot = fmaf(__uint_as_float(r1[er]), 1.0f / 2048.0f, dot);
                                o[tt] = fmaf(cb * su, dot, nu + nb);
                                o[tt] = n0 + cc + e == jstar ? 0.f : o[tt];
                            }
                            if (row_ok && n0 + cc + e4 * 4 < ldd)
                                *reinterpret_cast<float4*>(out + e4 * 4) = make_float4(o[0], o[1], o[2], o[3]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// Gathers the packed FP16-split panel rows (hi and lo), scales and squared norms of each
// query's candidate rows (qd[q].crows) from the vocabulary panels: one warp per row, 16-byte
// pieces (a row's 8 consecutive K elements of one core matrix).
__global__ void k_cand_pack_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, const uint8_t* __restrict__ a_hi,
                              const uint8_t* __restrict__ a_lo, int64_t Mpad, const float* __restrict__ a_scale,
                              const float* __restrict__ a_norm, int KC)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    const int nr = min(*d.ncrows, kCandRows);
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    uint8_t* ch = static_cast<uint8_t*>(d.c_hi);
    uint8_t* cl = static_cast<uint8_t*>(d.c_lo);
    for (int i = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); i < nr; i += warps) {
        const int64_t u = d.crows[i];
        for (int p = lane; p < KC * 8; p += 32) {  // piece p: chunk p / 8, core matrix p % 8
            const int64_t c = p >> 3, kk = p & 7;
            const int64_t src = 2 * (c * Mpad * 64 + (u >> 3) * 512 + kk * 64 + (u & 7) * 8);
            const int64_t dst = 2 * (c * (int64_t)kCandRows * 64 + (int64_t)(i >> 3) * 512 + kk * 64 + (i & 7) * 8);
            *reinterpret_cast<uint4*>(ch + dst) = *reinterpret_cast<const uint4*>(a_hi + src);
            *reinterpret_cast<uint4*>(cl + dst) = *reinterpret_cast<const uint4*>(a_lo + src);
        }
        if (lane == 0) {
            d.c_scale[i] = a_scale[u];
            d.c_norm[i] = a_norm[u];
        }
    }
}

// Pack rows of an FP32 matrix (ld floats per row, first m used) into the canonical layout
// above.  For 2-byte formats element (r, k) of a matrix with Rpad rows lives at byte
// 2 * ((k/64)*Rpad*64 + (r/8)*512 + ((k%64)/8)*64 + (r%8)*8 + k%8); for E4M3 at byte
// (k/64)*Rpad*64 + (r/8)*512 + ((k%64)/16)*128 + (r%8)*16 + k%16.  One warp per row; rows
// R..Rpad-1 and columns m..Kpad-1 are zero.  scale[r]: the factor that turns stored
// values back into x (amax for FP16/BF16, amax / 448 for E4M3; 0 for a zero row).
template <int FMT>
__device__ __forceinline__ void pack_body(const float* __restrict__ src, int ld, int m, int64_t R, int64_t Rpad, int Kpad,
                       uint8_t* __restrict__ hi, uint8_t* __restrict__ lo, float* __restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= Rpad) return;
    const bool live = r < R;
    float amax = 0.f;
    if (live)
        for (int k = lane; k < m; k += 32) amax = fmaxf(amax, fabsf(src[r * ld + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    constexpr float kTop = FMT == TC_E4M3 ? 448.0f : 1.0f;  // largest stored magnitude
    const float inv = amax > 0.f ? kTop / amax : 0.f;
    for (int k = lane; k < Kpad; k += 32) {
        const float y = (live && k < m) ? src[r * ld + k] * inv : 0.f;
        const int64_t chunk = (int64_t)(k >> 6) * Rpad * 64;
        if (FMT == TC_E4M3) {
            const int64_t off = chunk + (r >> 3) * 512 + ((k & 63) >> 4) * 128 + (r & 7) * 16 + (k & 15);
            hi[off] = (uint8_t)__nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
        } else {
            const int64_t off = chunk + (r >> 3) * 512 + ((k & 63) >> 3) * 64 + (r & 7) * 8 + (k & 7);
            if (FMT == TC_BF16) {
                reinterpret_cast<__nv_bfloat16*>(hi)[off] = __float2bfloat16_rn(y);
            } else {
                const __half h = __float2half_rn(y);
                reinterpret_cast<__half*>(hi)[off] = h;
                if (lo) reinterpret_cast<__half*>(lo)[off] = __float2half_rn((y - __half2float(h)) * 2048.0f);
            }
        }
    }
    if (lane == 0) scale[r] = amax / kTop;
}

template <int FMT>
__global__ void k_pack(const float* __restrict__ src, int ld, int m, int64_t R, int64_t Rpad, int Kpad,
                       uint8_t* __restrict__ hi, uint8_t* __restrict__ lo, float* __restrict__ scale)
{
    pack_body<FMT>(src, ld, m, R, Rpad, Kpad, hi, lo, scale);
}

// to_split: into the query's FP16-split panels of the candidate block (qs_*).
template <int FMT>
__global__ void k_pack_b(const QDesc* __restrict__ qd, const int* __restrict__ nq, int ld, int m, int Kpad,
                         bool to_split)
{
    if ((int)blockIdx.y >= *nq) return;
    const QDesc& d = qd[blockIdx.y];
    if (to_split)
        pack_body<FMT>(d.Q, ld, m, d.h, d.npad, Kpad, static_cast<uint8_t*>(d.qs_hi), static_cast<uint8_t*>(d.qs_lo),
                       d.qs_scale);
    else
        pack_body<FMT>(d.Q, ld, m, d.h, d.npad, Kpad, static_cast<uint8_t*>(d.q_hi), static_cast<uint8_t*>(d.q_lo),
                       d.q_scale);
}

}  // namespace

size_t tc_dist_smem_bytes(int fmt, int stages, int KC)
{
    const size_t eb = fmt == TC_E4M3 ? 64 : 128;
    const size_t parts = fmt == TC_SPLIT ? 2 : 1;
    return 1024 + (size_t)stages * parts * TC_BM * eb + (size_t)KC * parts * TC_BN * eb +
           (2 * (size_t)stages + 6) * 8 + 16;
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    }
    return n;
}

// Vocabulary stages (2..8) that fit beside the resident query panel (0 when the panel
// alone does not leave room for two stages).
int tc_dist_stages(int fmt, int KC)
{
    const size_t budget = 227 * 1024;
    int s = 8;
    while (s >= 2 && tc_dist_smem_bytes(fmt, s, KC) > budget) --s;
    return s >= 2 ? s : 0;
}

cudaError_t launch_pack_b(int fmt, const QDesc* qd, const int* nq, int max_q, int max_rows, int ld, int m,
                          int Kpad, cudaStream_t st, bool to_split)
{
    if (max_q <= 0 || max_rows <= 0) return cudaSuccess;
    const int warps = 8;
    const dim3 g((unsigned)((max_rows + warps - 1) / warps), (unsigned)max_q);
    switch (fmt) {
    case TC_SPLIT: k_pack_b<TC_SPLIT><<<g, warps * 32, 0, st>>>(qd, nq, ld, m, Kpad, to_split); break;
    case TC_BF16: k_pack_b<TC_BF16><<<g, warps * 32, 0, st>>>(qd, nq, ld, m, Kpad, false); break;
    case TC_E4M3: k_pack_b<TC_E4M3><<<g, warps * 32, 0, st>>>(qd, nq, ld, m, Kpad, false); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(int fmt, const float* src, int ld, int m, int64_t R, int64_t Rpad, int Kpad, void* hi,
                        void* lo, float* scale, cudaStream_t st)
{
    if (Rpad <= 0) return cudaSuccess;
    const int warps = 8;
    const unsigned blocks = (unsigned)((Rpad + warps - 1) / warps);
    uint8_t* h = static_cast<uint8_t*>(hi);
    uint8_t* l = static_cast<uint8_t*>(lo);
    switch (fmt) {
    case TC_SPLIT: k_pack<TC_SPLIT><<<blocks, warps * 32, 0, st>>>(src, ld, m, R, Rpad, Kpad, h, l, scale); break;
    case TC_BF16: k_pack<TC_BF16><<<blocks, warps * 32, 0, st>>>(src, ld, m, R, Rpad, Kpad, h, nullptr, scale); break;
    case TC_E4M3: k_pack<TC_E4M3><<<blocks, warps * 32, 0, st>>>(src, ld, m, R, Rpad, Kpad, h, nullptr, scale); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int FMT>
static cudaError_t tc_launch(dim3 grid, size_t smem, cudaStream_t st, const void* A_hi, const void* A_lo,
                             int64_t Mpad, const float* a_scale, const float* a_norm, int64_t M,
                             const void* B_hi, const void* B_lo, int64_t Npad, const float* b_scale,
                             const float* b_norm, int N, int KC, int stages, float* D, int ldd,
                             int* err)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_dist<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_dist<FMT><<<grid, TC_THREADS, smem, st>>>(
        static_cast<const uint8_t*>(A_hi), static_cast<const uint8_t*>(A_lo), Mpad, a_scale, a_norm, M,
        static_cast<const uint8_t*>(B_hi), static_cast<const uint8_t*>(B_lo), Npad, b_scale, b_norm, N, KC,
        stages, D, ldd, err);
    return cudaGetLastError();
}

// MMAs of the last 64-element K chunk that touch data (m elements of K, the rest zero
// padding): zero steps add exact zeros, so leaving them out changes no value.
static int last_chunk_steps(int fmt, int m, int KC)
{
    const int step = fmt == TC_E4M3 ? 32 : 16, mmas = 64 / step;
    if (m <= 0) return mmas;
    return std::max(1, std::min(mmas, (m - 64 * (KC - 1) + step - 1) / step));
}

size_t tc_batch_smem_bytes(int fmt, int stages, int KC)
{
    const size_t eb = fmt == TC_E4M3 ? 64 : 128;
    const size_t parts = fmt == TC_SPLIT ? 2 : 1;
    return 1024 + (size_t)KC * parts * TC_BM * eb + (size_t)stages * parts * TC_BN * eb + (2 * (size_t)stages + 6) * 8 + 16;
}

// B stages (2..8) beside the resident vocabulary panel; 0 when the panel leaves no room.
int tc_batch_stages(int fmt, int KC)
{
    const size_t budget = 227 * 1024;
    int s = 8;
    while (s >= 2 && tc_batch_smem_bytes(fmt, s, KC) > budget) --s;
    return s >= 2 ? s : 0;
}

// The fused table kernel: the matrix kernel's layout plus eight list-exchange barriers.
static size_t tct_smem_bytes(int fmt, int stages, int KC) { return tc_batch_smem_bytes(fmt, stages, KC) + 8 * 8; }

static int tct_stages(int fmt, int KC)
{
    const size_t budget = 227 * 1024;
    int s = 8;
    while (s >= 2 && tct_smem_bytes(fmt, s, KC) > budget) --s;
    return s >= 2 ? s : 0;
}

template <int FMT>
static cudaError_t tc_batch_launch(dim3 grid, size_t smem, cudaStream_t st, const void* A_hi, const void* A_lo,
                                   int64_t Mpad, const float* a_scale, const float* a_norm,
                                   int64_t M, const QDesc* qd, const int* nq, int groups, int KC, int stages, int klast,
                                   int* err)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_dist_batch<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_dist_batch<FMT><<<grid, TCB_THREADS, smem, st>>>(static_cast<const uint8_t*>(A_hi),
                                                         static_cast<const uint8_t*>(A_lo), Mpad, a_scale, a_norm,
                                                         M, qd, nq, groups, KC, stages, klast, err);
    return cudaGetLastError();
}

cudaError_t launch_tc_dist_batch(int fmt, const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                                 const float* a_norm, int64_t M, const QDesc* qd, const int* nq,
                                 int max_q, int Kpad, int m, int group_mult, int stages_req, int* err, cudaStream_t st)
{
    if (M <= 0 || max_q <= 0) return cudaSuccess;
    const int KC = Kpad / 64;
    const int klast = last_chunk_steps(fmt, m, KC);
    const int fit = tc_batch_stages(fmt, KC);
    if (fit < 2) return cudaErrorInvalidValue;
    const int stages = stages_req >= 2 ? std::min(stages_req, fit) : fit;
    const size_t smem = tc_batch_smem_bytes(fmt, stages, KC);
    const int m_tiles = (int)(Mpad / TC_BM);
    const int sms = sm_count();
    const int groups =
        std::max(1, std::min(max_q, std::max(1, group_mult) * ((2 * sms + m_tiles - 1) / m_tiles)));
    dim3 grid((unsigned)std::min<int64_t>((int64_t)m_tiles * groups, sms));
    switch (fmt) {
    case TC_SPLIT:
        return tc_batch_launch<TC_SPLIT>(grid, smem, st, A_hi, A_lo, Mpad, a_scale, a_norm, M, qd, nq, groups,
                                         KC, stages, klast, err);
    case TC_BF16:
        return tc_batch_launch<TC_BF16>(grid, smem, st, A_hi, nullptr, Mpad, a_scale, a_norm, M, qd, nq,
                                        groups, KC, stages, klast, err);
    case TC_E4M3:
        return tc_batch_launch<TC_E4M3>(grid, smem, st, A_hi, nullptr, Mpad, a_scale, a_norm, M, qd, nq,
                                        groups, KC, stages, klast, err);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tc_dist(int fmt, const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                           const float* a_norm, int64_t M, const void* B_hi, const void* B_lo,
                           int64_t Npad, const float* b_scale, const float* b_norm, int N,
                           int Kpad, float* D, int ldd, int* err, cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int KC = Kpad / 64;
    const int stages = tc_dist_stages(fmt, KC);
    if (stages < 2) return cudaErrorInvalidValue;  // embeddings wider than the resident panel allows
    const size_t smem = tc_dist_smem_bytes(fmt, stages, KC);
    const int64_t tiles = (Mpad / TC_BM) * ((N + TC_BN - 1) / TC_BN);
    dim3 grid((unsigned)std::min<int64_t>(tiles, sm_count()));
    switch (fmt) {
    case TC_SPLIT:
        return tc_launch<TC_SPLIT>(grid, smem, st, A_hi, A_lo, Mpad, a_scale, a_norm, M, B_hi, B_lo, Npad,
                                   b_scale, b_norm, N, KC, stages, D, ldd, err);
    case TC_BF16:
        return tc_launch<TC_BF16>(grid, smem, st, A_hi, nullptr, Mpad, a_scale, a_norm, M, B_hi, nullptr,
                                  Npad, b_scale, b_norm, N, KC, stages, D, ldd, err);
    case TC_E4M3:
        return tc_launch<TC_E4M3>(grid, smem, st, A_hi, nullptr, Mpad, a_scale, a_norm, M, B_hi, nullptr,
                                  Npad, b_scale, b_norm, N, KC, stages, D, ldd, err);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace emd

namespace emd {

template <int FMT, int KT, bool CAND>
static cudaError_t tc_table_launch(dim3 grid, size_t smem, cudaStream_t st, const void* A_hi, const void* A_lo,
                                   int64_t Mpad, const float* a_scale, const float* a_norm, int64_t M, const QDesc* qd,
                                   const int* nq, int groups, int KC, int stages, int klast, int* err)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_table_batch<FMT, KT, CAND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_table_batch<FMT, KT, CAND><<<grid, TCT_THREADS, smem, st>>>(static_cast<const uint8_t*>(A_hi),
                                                                     static_cast<const uint8_t*>(A_lo), Mpad, a_scale,
                                                                     a_norm, M, qd, nq, groups, KC, stages, klast, err);
    return cudaGetLastError();
}

cudaError_t launch_tc_table_batch(int fmt, const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                                  const float* a_norm, int64_t M, const QDesc* qd, const int* nq, int max_q, int Kpad,
                                  int m, int max_tk, int group_mult, int stages_req, int* err, cudaStream_t st)
{
    if (M <= 0 || max_q <= 0) return cudaSuccess;
    if (max_tk < 1 || max_tk > 16) return cudaErrorInvalidValue;
    const int KC = Kpad / 64;
    const int klast = last_chunk_steps(fmt, m, KC);
    const int fit = tct_stages(fmt, KC);
    if (fit < 2) return cudaErrorInvalidValue;
    const int stages = stages_req >= 2 ? std::min(stages_req, fit) : fit;
    const size_t smem = tct_smem_bytes(fmt, stages, KC);
    const int m_tiles = (int)(Mpad / TC_BM);
    const int sms = sm_count();
    const int groups = std::max(1, std::min(max_q, std::max(1, group_mult) * ((2 * sms + m_tiles - 1) / m_tiles)));
    const dim3 grid((unsigned)std::min<int64_t>((int64_t)m_tiles * groups, sms));
    // approximate formats keep max_tk = the candidate count in candidate mode (at most 16)
    if (fmt == TC_BF16)
        return tc_table_launch<TC_BF16, 16, true>(grid, smem, st, A_hi, nullptr, Mpad, a_scale, a_norm, M, qd, nq,
                                                  groups, KC, stages, klast, err);
    if (fmt == TC_E4M3)
        return tc_table_launch<TC_E4M3, 16, true>(grid, smem, st, A_hi, nullptr, Mpad, a_scale, a_norm, M, qd, nq,
                                                  groups, KC, stages, klast, err);
    if (fmt != TC_SPLIT) return cudaErrorInvalidValue;
#define EMD_TT(KT) \
    return tc_table_launch<TC_SPLIT, KT, false>(grid, smem, st, A_hi, A_lo, Mpad, a_scale, a_norm, M, qd, nq, groups, KC, \
                                                stages, klast, err)
    if (max_tk <= 1) EMD_TT(1);
    if (max_tk <= 2) EMD_TT(2);
    if (max_tk <= 4) EMD_TT(4);
    if (max_tk <= 8) EMD_TT(8);
    EMD_TT(16);
#undef EMD_TT
}

static size_t tcp_smem_bytes(int bn, int stages, int KC)
{
    return 1024 + (size_t)KC * 2 * TC_BM * 128 + (size_t)stages * 2 * (bn / 2) * 128 + (3 * (size_t)stages + 7) * 8 +
           16;
}

static int tcp_stages(int bn, int KC)
{
    const size_t budget = 227 * 1024;
    int s = 8;
    while (s >= 2 && tcp_smem_bytes(bn, s, KC) > budget) --s;
    return s >= 2 ? s : 0;
}

bool tc_table_fits(int fmt, int Kpad) { return tct_stages(fmt, Kpad / 64) >= 2; }

bool tc_table_pair_fits(int Kpad) { return tcp_stages(128, Kpad / 64) >= 2 && tcp_stages(64, Kpad / 64) >= 2; }

template <int KT, int BN>
static cudaError_t tc_pair_launch(dim3 grid, size_t smem, cudaStream_t st, const void* A_hi, const void* A_lo,
                                  int64_t Mpad, const float* a_scale, const float* a_norm, int64_t M, const QDesc* qd,
                                  const int* nq, int groups, int KC, int stages, int klast, int* err)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_table_pair<KT, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_table_pair<KT, BN><<<grid, TCP_THREADS, smem, st>>>(static_cast<const uint8_t*>(A_hi),
                                                             static_cast<const uint8_t*>(A_lo), Mpad, a_scale, a_norm,
                                                             M, qd, nq, groups, KC, stages, klast, err);
    return cudaGetLastError();
}

cudaError_t launch_tc_table_pair(const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                                 const float* a_norm, int64_t M, const QDesc* qd, const int* nq, int max_q, int Kpad,
                                 int m, int max_tk, int group_mult, int bn, int* err, cudaStream_t st)
{
    if (M <= 0 || max_q <= 0) return cudaSuccess;
    if (max_tk < 1 || max_tk > 16 || (bn != 64 && bn != 128) || Mpad % (2 * TC_BM) != 0)
        return cudaErrorInvalidValue;
    const int KC = Kpad / 64;
    const int klast = last_chunk_steps(TC_SPLIT, m, KC);
    const int stages = tcp_stages(bn, KC);
    if (stages < 2) return cudaErrorInvalidValue;
    const size_t smem = tcp_smem_bytes(bn, stages, KC);
    const int pairs = (int)(Mpad / (2 * TC_BM));
    const int clusters_max = std::max(1, sm_count() / 2);
    const int groups =
        std::max(1, std::min(max_q, std::max(1, group_mult) * ((2 * clusters_max + pairs - 1) / pairs)));
    const dim3 grid((unsigned)(2 * std::min<int64_t>((int64_t)pairs * groups, clusters_max)));
#define EMD_TP(KT)                                                                                                    \
    return bn == 64 ? tc_pair_launch<KT, 64>(grid, smem, st, A_hi, A_lo, Mpad, a_scale, a_norm, M, qd, nq, groups, KC, \
                                             stages, klast, err)                                                              \
                    : tc_pair_launch<KT, 128>(grid, smem, st, A_hi, A_lo, Mpad, a_scale, a_norm, M, qd, nq, groups,    \
                                              KC, stages, klast, err)
    if (max_tk <= 1) EMD_TP(1);
    if (max_tk <= 2) EMD_TP(2);
    if (max_tk <= 4) EMD_TP(4);
    if (max_tk <= 8) EMD_TP(8);
    EMD_TP(16);
#undef EMD_TP
}

cudaError_t launch_cand_pack_b(const QDesc* qd, const int* nq, int max_q, const void* a_hi, const void* a_lo,
                               int64_t Mpad, const float* a_scale, const float* a_norm, int Kpad, cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    const dim3 g(256, (unsigned)max_q);
    k_cand_pack_b<<<g, 256, 0, st>>>(qd, nq, static_cast<const uint8_t*>(a_hi), static_cast<const uint8_t*>(a_lo), Mpad,
                                     a_scale, a_norm, Kpad / 64);
    return cudaGetLastError();
}

cudaError_t launch_tc_cand_batch(const QDesc* qd, const int* nq, int max_q, int Kpad, int stages_req, int* err,
                                 cudaStream_t st)
{
    if (max_q <= 0) return cudaSuccess;
    const int KC = Kpad / 64;
    const int fit = tc_batch_stages(TC_SPLIT, KC);
    if (fit < 2) return cudaErrorInvalidValue;
    const int stages = stages_req >= 2 ? std::min(stages_req, fit) : fit;
    const size_t smem = tc_batch_smem_bytes(TC_SPLIT, stages, KC);
    cudaError_t e = cudaFuncSetAttribute(k_tc_cand_batch<TC_SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)std::min<int64_t>((int64_t)max_q * (kCandRows / TC_BM), sm_count()));
    k_tc_cand_batch<TC_SPLIT><<<grid, TCB_THREADS, smem, st>>>(qd, nq, max_q, KC, stages, err);
    return cudaGetLastError();
}

}  // namespace emd
