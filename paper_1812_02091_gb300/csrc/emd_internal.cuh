// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/emd.h is).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/emd.h"

namespace emd {

constexpr int kWarp = 32;

// Measures as kernel template arguments (same numbering as emd_measure).
enum : int { M_RWMD = 0, M_OMR = 1, M_ACT = 2, M_ICT = 3 };

// Phase-1 matrices D of embedding databases hold squared distances |v_u - q_j|^2 (the
// distance kernels leave the square root to the readers, which take it only for the
// entries they use: the k table entries of a row, the distances a reverse pass gathers);
// cost-matrix databases hold the costs themselves.  sq tells a reader which.
__device__ __forceinline__ float sq_to_dist(float x) { return __fsqrt_rn(fmaxf(x, 0.f)); }
__device__ __forceinline__ float d_value(float x, bool sq) { return sq ? sq_to_dist(x) : x; }

// Device error latch bits (written by kernels, read by emd_db_check_device_errors).
enum : int { ERR_BAD_INDEX = 1, ERR_TIMEOUT = 2, ERR_PAIR_TMEM = 4 };

// Distance-matrix tiling of the FP32 SIMT kernel.
constexpr int kDistBM = 128;
constexpr int kDistBN = 64;
constexpr int kDistBK = 16;

// Row strides: embeddings are padded to a multiple of 4 floats (16-byte rows); the
// distance matrix D to a multiple of 32 columns (one warp-wide chunk); staged query
// coordinates to a multiple of the distance tile width.
__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Largest top-K of the neighbour selection and largest register top-k width.
constexpr int kMaxTopK = 64;
constexpr int kMaxRegK = 16;
constexpr int kTopkThreads = 128;
constexpr int kTopkMaxBlocks = 64;
constexpr int64_t kTopkScratchRow = (int64_t)kTopkMaxBlocks * kMaxTopK;  // keys per selection row

// Blocks per row of the top-K selection (one block per 2048 values, at most 64).
__host__ __device__ inline int topk_blocks(int64_t n)
{
    int64_t b = n / 2048;
    return (int)(b < 1 ? 1 : (b > kTopkMaxBlocks ? kTopkMaxBlocks : b));
}

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns cudaGetLastError().

// Gather rows of `src` (ld floats per row) into `dst` (ld floats per row) and write
// their squared L2 norms; ids outside [0, v) latch ERR_BAD_INDEX and produce zero rows.
// Rows nrows..nrows_pad-1 of dst are zero-filled with zero norm.
cudaError_t launch_gather_rows(const float* src, int64_t v, int ld, int m, const int32_t* ids,
                               int64_t nrows, int64_t nrows_pad, float* dst, float* norm2,
                               int* err, cudaStream_t st);

// D[u, j] = squared Euclidean distance between A row u and B row j by the norm expansion
// (unclamped), exactly 0 when a_ids[u] == b_ids[j]; +inf for j in [N, ldd).
cudaError_t launch_dist_fp32(const float* A, int64_t M, int lda, const float* anorm,
                             const int32_t* a_ids, const float* B, int N, int ldb,
                             const float* bnorm, const int32_t* b_ids, int K, float* D,
                             int ldd, cudaStream_t st);

// Cost-matrix mode: D[u, j] = cost[a_ids[u] * v + b_ids[j]]; +inf for j in [N, ldd).
cudaError_t launch_dist_gather(const float* cost, int64_t v, const int32_t* a_ids, int64_t M,
                               const int32_t* b_ids, int N, float* D, int ldd, int* err,
                               cudaStream_t st);

// Phase-1 table (Section 5): per row u the k smallest D[u, 0..h) (ties by column),
// written as tab[u * k + l] = (z, w = q_w[s]) and optionally tab_s[u * k + l] = s; z is the
// distance (the square root of the entry when sq).
cudaError_t launch_table(const float* D, int ldd, int64_t M, int h, int k, const float* q_w,
                         float2* tab, int32_t* tab_s, bool sq, cudaStream_t st);

// vslot[id] = the used-vocabulary row of each vocabulary id (v entries), -1 for unused ids.
cudaError_t launch_vslot(const int32_t* used_ids, int64_t v_used, int64_t v, int32_t* vslot, cudaStream_t st);

// Exact zeros of identical ids in squared-distance matrices: D[s(j), j] = 0 for every query
// bin j whose vocabulary id has used row s(j) = vslot[q_idx[j]] >= 0.
cudaError_t launch_zero_ident(const int32_t* q_idx, int h, const int32_t* vslot, int64_t v, float* D, int ldd,
                              cudaStream_t st);

// ICT table (Section 4.2, Algorithm 2, in the linear form of Section 5): per row u the
// smallest D[u, 0..h) in ascending (distance, column) order, only as many as the largest
// database weight at u, xmax[u], needs before its residual reaches 0 (capacity-limited
// transfers in FP32, the same steps as the forward pass), at most W entries.  Entries past
// that point are not written: no database weight at u reaches them.  A row that would need
// more than W < h entries sets *over = 1 (the query's values are then incomplete).
cudaError_t launch_table_ict(const float* D, int ldd, int64_t M, int h, int W, const float* q_w,
                             const float* xmax, float2* tab, int32_t* tab_s, int* over, bool sq, cudaStream_t st);

// Forward direction (Phase 2 and 3, Eq. 6-9): t_fwd[d] for every document.
cudaError_t launch_fwd(int meas, const int32_t* row_ptr, const int32_t* col, const float* val,
                       int64_t n, const float2* tab, int k, int keff, float* t_fwd,
                       cudaStream_t st);

// Reverse direction: the query's mass moved into each document, cost block gathered
// from D; t_rev[d], and t_max[d] = max(t_fwd[d], t_rev[d]) when t_max != nullptr.  With
// doc_ids, output slot i holds document doc_ids[i] (n slots) and t_fwd is indexed by
// document.
cudaError_t launch_rev(int meas, int k, const int32_t* row_ptr, const int32_t* col,
                       const float* val, int64_t n, const float* D, int ldd, int h,
                       const float* q_w, const float* t_fwd, float* t_rev, float* t_max,
                       const int64_t* doc_ids, bool sq, cudaStream_t st);

// Exact pruned symmetric top-K (K <= kPruneMaxK).  sel_val holds the K smallest forward
// values (ascending); the candidates are the documents with fwd <= fwd_K (1 + 2^-7), at
// most kPruneCap of them, and the reverse pass runs only there.  Writes the K smallest
// (max(fwd, rev), id) among the candidates and ok = 1 when the K-th is <= that threshold
// (then no other document can enter) and the candidates did not overflow.  cand holds
// kPruneCap ids, sym 2 * kPruneCap values, count one int (all workspace).
constexpr int kPruneMaxK = 16;
constexpr int kPruneCap = 256;
cudaError_t launch_prune(int meas, int k, const int32_t* row_ptr, const int32_t* col, const float* val,
                         int64_t n, const float* D, int ldd, int h, const float* q_w, const float* t_fwd,
                         const int64_t* sel_idx, const float* sel_val, int K, int64_t* cand, int* count,
                         float* sym, int64_t* out_idx, float* out_dist, int* ok, bool sq, cudaStream_t st);

// Top-K smallest of t[0..n) by (value, index), into out_idx / out_dist (K <= kMaxTopK).
// scratch must hold kTopkScratchRow uint64 keys.
cudaError_t launch_topk(const float* t, int64_t n, int K, unsigned long long* scratch,
                        int64_t* out_idx, float* out_dist, cudaStream_t st);

// The same for `rows` rows of t (row stride ldt) in one launch; outputs are rows x K and
// scratch holds rows * kTopkScratchRow keys.
cudaError_t launch_topk_rows(const float* t, int64_t rows, int64_t n, int64_t ldt, int K,
                             unsigned long long* scratch, int64_t* out_idx, float* out_dist,
                             cudaStream_t st);

// Tensor-core operand formats (k_tc_dist.cu).
constexpr int TC_NONE = -1;
constexpr int TC_SPLIT = 0;  // FP16 hi + lo * 2^-11, three products: FP32-grade
constexpr int TC_BF16 = 1;   // BF16, one product: approximate
constexpr int TC_E4M3 = 2;   // FP8 E4M3, one product: approximate

// Tensor-core distance matrix.  Operands are panels in the canonical K-major core-matrix
// layout (see launch_pack) with Mpad / Npad rows (multiples of 128) and Kpad = m rounded
// up to 64; A_lo / B_lo only for TC_SPLIT.  D[u, j] = the squared distance by the norm
// expansion (unclamped); the zeros of identical ids are left to launch_zero_ident.
cudaError_t launch_tc_dist(int fmt, const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                           const float* a_norm, int64_t M, const void* B_hi, const void* B_lo,
                           int64_t Npad, const float* b_scale, const float* b_norm, int N,
                           int Kpad, float* D, int ldd, int* err, cudaStream_t st);

// Pack R rows of an FP32 matrix (ld floats per row, m used) into format `fmt` panels of
// Rpad rows and Kpad columns with per-row scales (x = scale * stored); lo (TC_SPLIT only,
// may be null) receives the scaled remainder (x/s - hi) * 2^11.  Panel bytes: Rpad * Kpad
// * (2 for FP16/BF16, 1 for E4M3) per part.
cudaError_t launch_pack(int fmt, const float* src, int ld, int m, int64_t R, int64_t Rpad, int Kpad, void* hi,
                        void* lo, float* scale, cudaStream_t st);

// Table from an approximate D: per row the kc smallest approximate values are re-ranked
// with exact FP32 distances sqrt(sum (V_u - Q_j)^2) (V: M rows, Q: h rows, both ldv floats
// per row, zero beyond m), which are also written back into D; then the k smallest exact
// values form the table (as launch_table).  k <= kc <= min(h, kRerankMax).
constexpr int kRerankMax = 32;
cudaError_t launch_table_rerank(float* D, int ldd, int64_t M, int h, int k, int kc, const float* V,
                                const float* Q, int ldv, const float* q_w, float2* tab, int32_t* tab_s,
                                cudaStream_t st);

// ------------------------------------------------------------------ batched forms
//
// A batch of queries runs each step as one launch: query q of the batch is blockIdx.y
// (blockIdx.z for the SIMT distance tile), its pointers and sizes are qd[q] (device
// memory), and blocks of queries q >= *nq exit at once.  Every batched kernel calls the
// same device body as its per-query form with the same template widths, so a query's
// results are bit-identical either way.
struct QDesc {
    const int32_t* qidx;    // h bins: vocabulary ids and weights
    const float* qw;
    float* Q;               // qrows x ldm gathered rows (zero beyond h and m)
    float* qnorm;           // qrows squared norms
    void* q_hi;             // npad x Kpad packed panel(s) (tensor-core precisions)
    void* q_lo;
    float* q_scale;
    float* D;               // v_used x ldd distance matrix
    float2* tab;            // v_used x tk table
    float* t_fwd;           // n forward values
    float* t_rev;           // n reverse values
    float* t_out;           // n requested distances (FWD, REV or MAX)
    int64_t* sel_idx;       // kPruneMaxK forward top-K (pruned top-K)
    float* sel_val;
    int64_t* cand;          // kPruneCap candidate documents
    float* cand_sym;        // 2 * kPruneCap: max values, then reverse values
    int* cand_count;
    int* ok;                // certification flag
    int* over;              // ICT: set to 1 when a table row needed more than tk entries
    int sq;                 // D holds squared distances (embedding databases)
    int64_t* out_idx;       // K top-K result
    float* out_dist;
    int h, ldd, qrows, npad, tk, kc;
    int tab_rs, tab_es;     // table layout: entry l of row u at tab[u * tab_rs + l * tab_es]
    // fused form of the pruned path (Phase-1 table in the product's epilogue, no full matrix)
    int32_t* qpos;          // v_used: the query bin whose vocabulary id is used row u, else -1
    int32_t* rmap;          // v_used: row of used row u in the candidate block, else -1
    int32_t* crows;         // kCandRows used rows of the candidate documents
    int* ncrows;            // their count (may exceed kCandRows: the query is then recomputed)
    void* c_hi;             // kCandRows x Kpad packed FP16-split panels of those rows
    void* c_lo;
    float* c_scale;         // kCandRows scales and squared norms
    float* c_norm;
    float* Dc;              // kCandRows x ldd squared distances of those rows to the query's bins
    // FP16-split query panels for the candidate block (the query panels above when the
    // database's format is the split; separate ones for BF16 / E4M3 databases)
    void* qs_hi;
    void* qs_lo;
    float* qs_scale;
    // fused approximate formats: per used row the kc candidate bins of the product's epilogue
    // (kCandPerRow apart) and the kc-th approximate squared distance; rows the re-rank cannot
    // certify (rr, count rr_count) are recomputed exactly over all bins
    int32_t* cbin;
    float* camax;
    int32_t* rr;
    int* rr_count;
};

// Candidate bins kept per vocabulary row by the fused approximate forms (k + margin <= 16).
constexpr int kCandPerRow = 16;

// Largest number of distinct used rows among the candidate documents of one query in the
// fused pruned path (their distance block is computed exactly; beyond it the query is
// recomputed over all documents with the full distance matrix).
constexpr int kCandRows = 32768;

// Queries whose forward pass shares one sweep of the CSR (batched form).  Tables of width
// <= 16 are stored query-major within a row -- row u, query g, entry l at
// base[(u * kFwdGroup + g) * W + l] with W the register width of the table (1, 2, 4, 8 or
// 16) -- so that a lane reads its query's first entries with vector loads; ICT tables of
// other widths are interleaved by entry, base[(u * width + l) * kFwdGroup + g].
constexpr int kFwdGroup = 8;
__host__ __device__ inline int fwd_reg_width(int kw)
{
    return kw <= 1 ? 1 : kw <= 2 ? 2 : kw <= 4 ? 4 : kw <= 8 ? 8 : kw <= 16 ? 16 : 0;
}

cudaError_t launch_gather_rows_b(const QDesc* qd, const int* nq, int max_q, int max_rows, const float* src,
                                 int64_t v, int ld, int m, int* err, cudaStream_t st);
cudaError_t launch_pack_b(int fmt, const QDesc* qd, const int* nq, int max_q, int max_rows, int ld, int m,
                          int Kpad, cudaStream_t st, bool to_split = false);
cudaError_t launch_dist_fp32_b(const QDesc* qd, const int* nq, int max_q, int max_ldd, const float* A, int64_t M,
                               int lda, const float* anorm, const int32_t* a_ids, int K, cudaStream_t st);
cudaError_t launch_dist_gather_b(const QDesc* qd, const int* nq, int max_q, const float* cost, int64_t v,
                                 const int32_t* a_ids, int64_t M, int* err, cudaStream_t st);
// Tensor-core distance matrices of every query of a batch (qd[q].q_hi / q_lo / q_scale /
// qnorm / qidx / h / npad -> qd[q].D, ldd); the vocabulary panel stays resident while the
// batch's column tiles stream past it.  max_q: queries the grid is sized for (the actual
// count is *nq).  cudaErrorInvalidValue when the panel does not fit in shared memory
// (tc_batch_stages == 0): use launch_tc_dist per query instead.
int tc_batch_stages(int fmt, int KC);
// group_mult scales the number of query groups per row tile (load balance against
// vocabulary re-reads); stages caps the B ring (0: as many as fit).  Same results for any
// choice.
cudaError_t launch_tc_dist_batch(int fmt, const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                                 const float* a_norm, int64_t M, const QDesc* qd, const int* nq,
                                 int max_q, int Kpad, int m, int group_mult, int stages, int* err, cudaStream_t st);
// max_tk: the largest table width of the batch; rerank: the approximate precisions' form
// (V: the used vocabulary rows, ldv floats each).
// Exact zeros of identical ids (launch_zero_ident) for every query of a batch.
cudaError_t launch_zero_ident_b(const QDesc* qd, const int* nq, int max_q, int max_h, const int32_t* vslot, int64_t v,
                                cudaStream_t st);

// ---- fused pruned path (tensor-core precision FP32_TC; RWMD, OMR, ACT with tables of width
// <= 16): the Phase-1 table from the product's epilogue, the reverse direction from an exact
// block over the candidate documents' rows only.  No v_used x h_q matrix is written.
// qd[q].qpos for every query of a batch: set (qpos[vslot[q_idx[j]]] = j) or cleared (-1).
cudaError_t launch_qpos_b(const QDesc* qd, const int* nq, int max_q, const int32_t* vslot, int64_t v, bool set,
                          cudaStream_t st);
// The table of every query (qd[q].tab, width qd[q].tk <= max_tk <= 16); format TC_SPLIT.
// The fused table on clusters of two SMs (tcgen05 cta_group::2, M = 256 per product): FP16
// split only; Mpad a multiple of 256; bn = 64 or 128 (the pair's largest column tile).
bool tc_table_pair_fits(int Kpad);
// The one-SM fused table kernel fits beside this panel width (format fmt).
bool tc_table_fits(int fmt, int Kpad);
cudaError_t launch_tc_table_pair(const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                                 const float* a_norm, int64_t M, const QDesc* qd, const int* nq, int max_q, int Kpad,
                                 int m, int max_tk, int group_mult, int bn, int* err, cudaStream_t st);
cudaError_t launch_tc_table_batch(int fmt, const void* A_hi, const void* A_lo, int64_t Mpad, const float* a_scale,
                                  const float* a_norm, int64_t M, const QDesc* qd, const int* nq, int max_q, int Kpad,
                                  int m, int max_tk, int group_mult, int stages, int* err, cudaStream_t st);
// Candidate compaction of the pruned path alone (counts must be zeroed).
cudaError_t launch_prune_compact_b(const QDesc* qd, const int* nq, int max_q, int64_t n, int K, cudaStream_t st);
// The distinct used rows of the candidate documents (qd[q].crows, ncrows zeroed, rmap), or
// with reset the row map returned to -1.
cudaError_t launch_cand_rows_b(const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr, const int32_t* col,
                               bool reset, cudaStream_t st);
// Their FP16-split panel rows, scales and norms gathered from the vocabulary panels.
cudaError_t launch_cand_pack_b(const QDesc* qd, const int* nq, int max_q, const void* a_hi, const void* a_lo,
                               int64_t Mpad, const float* a_scale, const float* a_norm, int Kpad, cudaStream_t st);
// Their squared distances to the query's bins (qd[q].Dc, ldd columns), exact zeros of
// identical ids from qd[q].qpos.
cudaError_t launch_tc_cand_batch(const QDesc* qd, const int* nq, int max_q, int Kpad, int stages, int* err,
                                 cudaStream_t st);
// Fused approximate forms: the table from each row's candidate bins (qd[q].cbin), exact
// squared distances sum (V_u - Q_j)^2 in FP32; with certify (BF16), a row is certified when
// its kc-th approximate value minus the rounding bound eps_rel |v_u| max|q| + eps_abs (|v_u|^2
// + max|q|^2) exceeds the k-th exact value: then no bin outside the candidates can be among
// the k nearest.  Other rows go to qd[q].rr (rr_count zeroed) for launch_rerank_full_b.
cudaError_t launch_rerank_cand_b(const QDesc* qd, const int* nq, int max_q, int64_t M, int max_h, const float* V,
                                 int ldv, const float* vnorm, bool certify, float eps_rel, float eps_abs,
                                 cudaStream_t st);
// The table rows listed in qd[q].rr recomputed exactly over all bins (same sums as above).
cudaError_t launch_rerank_full_b(const QDesc* qd, const int* nq, int max_q, int max_tk, const float* V, int ldv,
                                 cudaStream_t st);
// Reverse pass on the candidates through the row map, then the final selection (queries
// whose block overflowed are reported uncertified).
cudaError_t launch_prune_mapped_b(int meas, int k, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                                  const int32_t* col, const float* val, int K, int rev_warps, cudaStream_t st);
cudaError_t launch_table_b(const QDesc* qd, const int* nq, int max_q, int64_t M, int max_tk, bool rerank,
                           int max_kc, int max_h, const float* V, int ldv, cudaStream_t st);
// The ICT table of every query of a batch (width qd[q].tk, overflow flag qd[q].over).
cudaError_t launch_table_ict_b(const QDesc* qd, const int* nq, int max_q, int64_t M, const float* xmax,
                               cudaStream_t st);
// Forward values into t_out (to_out) or t_fwd.  grouped: the tables are interleaved in
// groups of kFwdGroup queries and each group shares one sweep of the CSR.  variant: the form
// of the grouped sweep (same values for each; the grouped table layout follows it, see
// fwd_layout_rowmajor):
//   kFwdChain     entry-interleaved rows, each entry loaded once the residual needs it
//   kFwdRowMajor  query-major rows, the first four entries loaded up front (vector loads)
//   kFwdCoalesced entry-interleaved rows, the first two entries up front, coalesced CSR reads
//   kFwdPrefetch  the entry chain with each lane's next four column ids and weights read ahead
enum : int { kFwdChain = 0, kFwdRowMajor = 1, kFwdCoalesced = 2, kFwdPrefetch = 3, kFwdVariants = 4 };
cudaError_t launch_fwd_b(int meas, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                         const int32_t* col, const float* val, int64_t n, bool to_out, bool grouped, int max_tk,
                         cudaStream_t st, int variant);
// Reverse pass over all documents; dir FWD is not accepted, REV writes t_out, MAX writes
// t_rev and max(t_fwd, t_rev) into t_out.
cudaError_t launch_rev_b(int meas, int k, int dir, const QDesc* qd, const int* nq, int max_q,
                         const int32_t* row_ptr, const int32_t* col, const float* val, int64_t n, cudaStream_t st);
// Top-K of each query of a batch: from t_fwd into sel_idx / sel_val (fwd_rows: the
// forward top-K of the pruned path) or from t_out into out_idx / out_dist.  scratch holds
// max_q * kTopkScratchRow keys.
cudaError_t launch_topk_b(const QDesc* qd, const int* nq, int max_q, int64_t n, int K,
                          unsigned long long* scratch, bool fwd_rows, cudaStream_t st);
// Pruned top-K after the forward top-K (sel_idx / sel_val): candidate compaction (counts
// must be zeroed), reverse pass on the candidates, final selection and certificate.
// rev_warps: warps per candidate document in the reverse pass (2, 4 or 8; same results).
cudaError_t launch_prune_b(int meas, int k, const QDesc* qd, const int* nq, int max_q, const int32_t* row_ptr,
                           const int32_t* col, const float* val, int64_t n, int K, int rev_warps, cudaStream_t st);

// All-pairs form (Section 6's evaluation over the database itself).  Vocabulary ids of
// the database's nonzeros (used_ids[col[e]]), the query bins of the database histograms.
cudaError_t launch_map_ids(const int32_t* col, int64_t nnz, const int32_t* used_ids, int32_t* out, cudaStream_t st);
// F (n x n, row stride n): F[a][b] <- max(F[a][b], F[b][a]) for all a, b and F[a][a] <- +inf.
cudaError_t launch_sym_max(float* F, int64_t n, cudaStream_t st);

// Failure message for emd_last_error() (defined beside the C ABI).
emd_status set_error(emd_status st, const char* msg);
void clear_error();

}  // namespace emd
