/*
 * Input generation helper for emd_synth (synthetic histograms only; nothing of the EMD
 * relaxations).  For each row: map uniform draws to Zipf-distributed vocabulary ids by
 * inverse CDF, keep the first `len` distinct ids in draw order, and write them sorted.
 * It is the per-row loop of emd_synth._zipf_sets_chunk written in C for speed; the two
 * produce identical rows from identical draws.
 */
#include <stdint.h>
#include <stdlib.h>

static int cmp_i32(const void* a, const void* b)
{
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Number of cdf entries <= u (numpy searchsorted, side="right"). */
static int64_t upper_bound(const double* cdf, int64_t V, double u)
{
    int64_t lo = 0, hi = V;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] <= u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * cdf[V]      ascending cumulative probabilities (last entry 1)
 * u           uniform draws of all rows back to back; row r owns draws[r] of them
 * lens[r]     distinct ids wanted for row r
 * stamp[V]    scratch, every entry < tag0 on entry (row r marks ids with tag0 + r)
 * out         row r's ids go to out[out_off[r] .. out_off[r] + lens[r]) in ascending order
 * ok[r]       1 when the draws held lens[r] distinct ids, else 0 (row left unwritten)
 * buf         scratch of at least max(lens) entries
 */
void zipf_first_distinct(const double* cdf, int64_t V, const double* u, const int64_t* draws, const int64_t* lens,
                         int64_t nrows, int64_t* stamp, int64_t tag0, int32_t* out, const int64_t* out_off,
                         uint8_t* ok, int32_t* buf)
{
    int64_t pos = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t tag = tag0 + r, L = lens[r];
        int64_t cnt = 0;
        for (int64_t t = 0; t < draws[r] && cnt < L; ++t) {
            int64_t id = upper_bound(cdf, V, u[pos + t]);
            if (id > V - 1) id = V - 1;
            if (stamp[id] != tag) {
                stamp[id] = tag;
                buf[cnt++] = (int32_t)id;
            }
        }
        pos += draws[r];
        if (cnt == L) {
            qsort(buf, (size_t)L, sizeof(int32_t), cmp_i32);
            for (int64_t j = 0; j < L; ++j) out[out_off[r] + j] = buf[j];
            ok[r] = 1;
        } else {
            ok[r] = 0;
        }
    }
}
