/*
 * FP64 CPU oracle for the EMD relaxations of Atasu & Mittelholzer, "Low-Complexity
 * Data-Parallel Earth Mover's Distance Approximations" (ICML 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls this
 * file: it exists so that tests, the smoke check and the benchmark's CPU baseline can
 * compare the CUDA path against a plain, slow, obviously correct implementation.  It
 * shares no code, header or constant with the CUDA library.
 *
 * Every quantity is FP64.  Inputs that come from the synthetic data are FP32 and are
 * promoted without renormalisation.  Readings taken where the paper is silent or
 * garbled (each marked "reading" below):
 *   R1 (Alg. 3)  the cost update inside the loop uses C[i, s[l]] (the printed C[i, j]
 *                leaves j undefined; Alg. 2 uses C[i, s[l]]).
 *   R2 (Alg. 1/3) when fewer than k destinations exist, k_eff = min(k, h_dest); OMR
 *                with one destination moves nothing further after the free transfer.
 *   R3 (Alg. 2)  the while-loop stops after the last destination, which absorbs what
 *                is left (ICT == ACT with k = h_dest; guards FP round-off in sum q).
 *   R4 (Alg. 1-3) argsort / argmin_k order ties by destination position.
 *   R5 (Eq. 6)   the minimum is element-wise: Y[d,u] = min(X[d,u], w_u^(l)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_RWMD 0
#define ORACLE_OMR 1
#define ORACLE_ACT 2
#define ORACLE_ICT 3

/* ------------------------------------------------------------------ ground cost */

/* Section 6: the transportation cost between two coordinates is the Euclidean (L2)
 * distance of their embedding vectors. */
static double euclid(const float* a, const float* b, int32_t m)
{
    double s = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        double d = (double)a[i] - (double)b[i];
        s += d * d;
    }
    return sqrt(s);
}

static double ground_cost(const float* emb, int32_t m, const float* cost, int64_t v,
                          int32_t a, int32_t b)
{
    if (cost) return (double)cost[(int64_t)a * v + b];
    return euclid(emb + (int64_t)a * m, emb + (int64_t)b * m, m);
}

/* Section 2: the h_p x h_q cost matrix between the bins of two histograms. */
void oracle_cost_block(const float* emb, int32_t m, const float* cost, int64_t v,
                       const int32_t* ia, int32_t ha, const int32_t* ib, int32_t hb,
                       double* C)
{
    for (int32_t i = 0; i < ha; ++i)
        for (int32_t j = 0; j < hb; ++j)
            C[(int64_t)i * hb + j] = ground_cost(emb, m, cost, v, ia[i], ib[j]);
}

/* ------------------------------------------------------------------ row sort */

typedef struct { double c; int32_t pos; } keyed;

static int keyed_cmp(const void* x, const void* y)
{
    const keyed* a = (const keyed*)x;
    const keyed* b = (const keyed*)y;
    if (a->c < b->c) return -1;
    if (a->c > b->c) return 1;
    return (a->pos > b->pos) - (a->pos < b->pos); /* R4 */
}

/* s = argsort(row) with ties ordered by position (R4). */
static void argsort_row(const double* row, int32_t h, int32_t* s, keyed* buf)
{
    for (int32_t j = 0; j < h; ++j) { buf[j].c = row[j]; buf[j].pos = j; }
    qsort(buf, (size_t)h, sizeof(keyed), keyed_cmp);
    for (int32_t j = 0; j < h; ++j) s[j] = buf[j].pos;
}

/* ------------------------------------------------------------------ pairwise measures */

/* Section 2.1 (RWMD, one direction): drop the in-flow constraints (Eq. 3); every bin of
 * p then moves all its mass to its nearest bin of q: sum_i p_i * min_j C[i,j]. */
double oracle_rwmd(const double* p, int32_t hp, const double* q, int32_t hq, const double* C)
{
    (void)q;
    double t = 0.0;
    for (int32_t i = 0; i < hp; ++i) {
        double mn = INFINITY;
        for (int32_t j = 0; j < hq; ++j) mn = fmin(mn, C[(int64_t)i * hq + j]);
        t += p[i] * mn;
    }
    return t;
}

/* Algorithm 1 (OMR). */
double oracle_omr(const double* p, int32_t hp, const double* q, int32_t hq, const double* C)
{
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)hq);
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)hq);
    double t = 0.0;
    for (int32_t i = 0; i < hp; ++i) {
        const double* Ci = C + (int64_t)i * hq;
        argsort_row(Ci, hq, s, buf); /* top-2 = first two of the sorted order */
        double pi = p[i];
        if (Ci[s[0]] == 0.0) {
            double r = fmin(pi, q[s[0]]); /* free transfer to the overlapping bin */
            pi = pi - r;
            if (hq > 1) t = t + pi * Ci[s[1]]; /* R2: nothing is left to move when hq == 1 */
        } else {
            t = t + pi * Ci[s[0]];
        }
    }
    free(buf);
    free(s);
    return t;
}

/* Algorithm 2 (ICT). */
double oracle_ict(const double* p, int32_t hp, const double* q, int32_t hq, const double* C)
{
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)hq);
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)hq);
    double t = 0.0;
    for (int32_t i = 0; i < hp; ++i) {
        const double* Ci = C + (int64_t)i * hq;
        argsort_row(Ci, hq, s, buf);
        double pi = p[i];
        int32_t l = 0;
        while (pi > 0.0 && l < hq) {
            double r = (l == hq - 1) ? pi : fmin(pi, q[s[l]]); /* R3 */
            pi = pi - r;
            t = t + r * Ci[s[l]];
            l = l + 1;
        }
    }
    free(buf);
    free(s);
    return t;
}

/* Algorithm 3 (ACT): k-1 capacity-limited transfers to the nearest bins, then the rest
 * of the mass to the k-th nearest. */
double oracle_act(const double* p, int32_t hp, const double* q, int32_t hq, const double* C,
                  int32_t k)
{
    int32_t keff = k < hq ? k : hq; /* R2 */
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)hq);
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)hq);
    double t = 0.0;
    for (int32_t i = 0; i < hp; ++i) {
        const double* Ci = C + (int64_t)i * hq;
        argsort_row(Ci, hq, s, buf); /* top-k = first k of the sorted order */
        double pi = p[i];
        int32_t l = 0;
        while (l < keff - 1) {
            double r = fmin(pi, q[s[l]]);
            pi = pi - r;
            t = t + r * Ci[s[l]]; /* R1 */
            l = l + 1;
        }
        if (pi != 0.0) t = t + pi * Ci[s[keff - 1]];
    }
    free(buf);
    free(s);
    return t;
}

double oracle_measure(int32_t measure, const double* p, int32_t hp, const double* q,
                      int32_t hq, const double* C, int32_t k)
{
    switch (measure) {
    case ORACLE_RWMD: return oracle_act(p, hp, q, hq, C, 1);
    case ORACLE_OMR: return oracle_omr(p, hp, q, hq, C);
    case ORACLE_ACT: return oracle_act(p, hp, q, hq, C, k);
    case ORACLE_ICT: return oracle_ict(p, hp, q, hq, C);
    default: return NAN;
    }
}

/* ------------------------------------------------------------------ exact EMD */

/* Eq. 1-3: EMD(p, q) = min sum F C subject to the out-flow and in-flow constraints,
 * solved as a min-cost flow on the bipartite graph by successive shortest augmenting
 * paths (Bellman-Ford on the residual network).  For tiny histograms only. */
double oracle_emd(const double* p, int32_t hp, const double* q, int32_t hq, const double* C)
{
    const double EPS = 1e-15;
    const int32_t N = hp + hq;
    double* F = (double*)calloc((size_t)hp * hq, sizeof(double));
    double* sup = (double*)malloc(sizeof(double) * (size_t)hp);
    double* dem = (double*)malloc(sizeof(double) * (size_t)hq);
    double* dist = (double*)malloc(sizeof(double) * (size_t)N);
    int32_t* pred = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    memcpy(sup, p, sizeof(double) * (size_t)hp);
    memcpy(dem, q, sizeof(double) * (size_t)hq);

    for (int64_t iter = 0; iter < 4 * (int64_t)N * N + 16; ++iter) {
        for (int32_t i = 0; i < hp; ++i) { dist[i] = sup[i] > EPS ? 0.0 : INFINITY; pred[i] = -1; }
        for (int32_t j = 0; j < hq; ++j) { dist[hp + j] = INFINITY; pred[hp + j] = -1; }
        for (int32_t round = 0; round < N; ++round) {
            int changed = 0;
            for (int32_t i = 0; i < hp; ++i) {
                if (dist[i] == INFINITY) continue;
                for (int32_t j = 0; j < hq; ++j) { /* forward arc i -> j, unbounded */
                    double nd = dist[i] + C[(int64_t)i * hq + j];
                    if (nd < dist[hp + j] - 1e-14) { dist[hp + j] = nd; pred[hp + j] = i; changed = 1; }
                }
            }
            for (int32_t j = 0; j < hq; ++j) {
                if (dist[hp + j] == INFINITY) continue;
                for (int32_t i = 0; i < hp; ++i) { /* backward arc j -> i while F[i,j] > 0 */
                    if (F[(int64_t)i * hq + j] <= EPS) continue;
                    double nd = dist[hp + j] - C[(int64_t)i * hq + j];
                    if (nd < dist[i] - 1e-14) { dist[i] = nd; pred[i] = hp + j; changed = 1; }
                }
            }
            if (!changed) break;
        }
        int32_t best = -1;
        for (int32_t j = 0; j < hq; ++j)
            if (dem[j] > EPS && dist[hp + j] < INFINITY && (best < 0 || dist[hp + j] < dist[hp + best]))
                best = j;
        if (best < 0) break;
        /* bottleneck along the path back to a root source */
        double b = dem[best];
        int32_t node = hp + best;
        while (1) {
            int32_t i = pred[node];            /* node is a sink; arrived by i -> node */
            if (pred[i] < 0) { b = fmin(b, sup[i]); break; }
            int32_t jj = pred[i] - hp;         /* arrived at i by the backward arc jj -> i */
            b = fmin(b, F[(int64_t)i * hq + jj]);
            node = hp + jj;
        }
        node = hp + best;
        while (1) {
            int32_t i = pred[node];
            int32_t j = node - hp;
            F[(int64_t)i * hq + j] += b;
            if (pred[i] < 0) { sup[i] -= b; break; }
            int32_t jj = pred[i] - hp;
            F[(int64_t)i * hq + jj] -= b;
            node = hp + jj;
        }
        dem[best] -= b;
    }
    double t = 0.0;
    for (int64_t e = 0; e < (int64_t)hp * hq; ++e) t += F[e] * C[e];
    free(pred); free(dist); free(dem); free(sup); free(F);
    return t;
}

/* ------------------------------------------------------------------ per-pair, whole database */

/* The plain definition for one query against every database histogram: for document d
 * build C[supp(d), supp(q)] afresh and run the pairwise algorithm.
 *   fwd(d) = measure(p = doc d, q = query, C)          (doc mass moved into the query)
 *   rev(d) = measure(p = query, q = doc d, C^T)        (query mass moved into the doc)
 * Either output may be NULL. */
int32_t oracle_pair_db(const float* emb, int32_t m, const float* cost, int64_t v,
                       const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                       const int32_t* q_idx, const float* q_w, int32_t hq,
                       int32_t measure, int32_t k, double* t_fwd, double* t_rev)
{
    double* qw = (double*)malloc(sizeof(double) * (size_t)hq);
    for (int32_t j = 0; j < hq; ++j) qw[j] = (double)q_w[j];
    for (int64_t d = 0; d < n; ++d) {
        int64_t a = row_ptr[d], b = row_ptr[d + 1];
        int32_t hd = (int32_t)(b - a);
        double* pw = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1));
        double* C = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1) * hq);
        double* CT = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1) * hq);
        for (int32_t i = 0; i < hd; ++i) pw[i] = (double)val[a + i];
        oracle_cost_block(emb, m, cost, v, col + a, hd, q_idx, hq, C);
        for (int32_t i = 0; i < hd; ++i)
            for (int32_t j = 0; j < hq; ++j) CT[(int64_t)j * hd + i] = C[(int64_t)i * hq + j];
        if (t_fwd) t_fwd[d] = oracle_measure(measure, pw, hd, qw, hq, C, k);
        if (t_rev) t_rev[d] = oracle_measure(measure, qw, hq, pw, hd, CT, k);
        free(CT); free(C); free(pw);
    }
    free(qw);
    return 0;
}

/* ------------------------------------------------------------------ LC-ACT (Section 5) */

/* Linear-complexity form for one query against the database.
 *
 * Phase 1: D[u, j] = ground cost between vocabulary coordinate u and query bin j, for
 *   every u in the used vocabulary (the union of database coordinates, Section 2.2);
 *   per row the top-k smallest give Z (distances), S (query bins) and W = q_S.
 * Phase 2 (Eq. 6-8): for l = 1..k-1, Y^(l) = min(X^(l-1), w^(l)) element-wise,
 *   X^(l) = X^(l-1) - Y^(l), t^(l) = t^(l-1) + Y^(l) z^(l).
 * Phase 3 (Eq. 9): t^(k) = t^(k-1) + X^(k-1) z^(k).
 * Measures: RWMD is k = 1; ICT is k = h_q; OMR runs the Phase-2 step l = 1 only on rows
 *   whose nearest distance is exactly zero (Alg. 1), i.e. k_u = 2 there and 1 elsewhere.
 *
 * The reverse direction has no vocabulary-level reuse: for document d it is the
 * pairwise algorithm with the query as source, the document as destination, and the
 * cost block gathered from D (rows supp(d), all query bins).
 *
 * Any of t_fwd / t_rev may be NULL.  Returns 0, or -1 on allocation failure. */
int32_t oracle_lc_query(const float* emb, int32_t m, const float* cost, int64_t v,
                        const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                        const int32_t* q_idx, const float* q_w, int32_t hq,
                        int32_t measure, int32_t k, double* t_fwd, double* t_rev)
{
    int64_t nnz = row_ptr[n];
    int32_t kk = measure == ORACLE_RWMD ? 1 : measure == ORACLE_OMR ? 2
               : measure == ORACLE_ICT ? hq : (k < hq ? k : hq);
    if (kk > hq) kk = hq;

    /* used vocabulary: the union of the database coordinates */
    int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)v);
    if (!slot) return -1;
    for (int64_t u = 0; u < v; ++u) slot[u] = -1;
    int64_t vu = 0;
    for (int64_t e = 0; e < nnz; ++e)
        if (slot[col[e]] < 0) slot[col[e]] = vu++;
    int32_t* used = (int32_t*)malloc(sizeof(int32_t) * (size_t)(vu > 0 ? vu : 1));
    for (int64_t u = 0; u < v; ++u) if (slot[u] >= 0) used[slot[u]] = (int32_t)u;

    /* Phase 1: D (vu x hq), then Z, W per row (top-kk) */
    double* D = (double*)malloc(sizeof(double) * (size_t)(vu > 0 ? vu : 1) * hq);
    double* Z = (double*)malloc(sizeof(double) * (size_t)(vu > 0 ? vu : 1) * kk);
    double* W = (double*)malloc(sizeof(double) * (size_t)(vu > 0 ? vu : 1) * kk);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)hq);
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)hq);
    if (!used || !D || !Z || !W || !s || !buf) {
        free(buf); free(s); free(W); free(Z); free(D); free(used); free(slot);
        return -1;
    }
    for (int64_t u = 0; u < vu; ++u) {
        double* Du = D + u * hq;
        for (int32_t j = 0; j < hq; ++j) Du[j] = ground_cost(emb, m, cost, v, used[u], q_idx[j]);
        argsort_row(Du, hq, s, buf);
        for (int32_t l = 0; l < kk; ++l) {
            Z[u * kk + l] = Du[s[l]];
            W[u * kk + l] = (double)q_w[s[l]];
        }
    }

    if (t_fwd) {
        /* per-row number of transfer columns: k_u */
        int32_t* ku = (int32_t*)malloc(sizeof(int32_t) * (size_t)(vu > 0 ? vu : 1));
        double* X = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
        for (int64_t u = 0; u < vu; ++u)
            ku[u] = measure == ORACLE_OMR ? ((Z[u * kk] == 0.0 && hq > 1) ? 2 : 1) : kk;
        for (int64_t e = 0; e < nnz; ++e) X[e] = (double)val[e]; /* X^(0) = X */
        for (int64_t d = 0; d < n; ++d) t_fwd[d] = 0.0;          /* t^(0) = 0 */
        /* Phase 2 */
        for (int32_t l = 0; l < kk - 1; ++l) {
            for (int64_t d = 0; d < n; ++d) {
                for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
                    int64_t u = slot[col[e]];
                    if (l >= ku[u] - 1) continue;
                    double y = fmin(X[e], W[u * kk + l]);  /* Eq. 6 (R5) */
                    X[e] = X[e] - y;                         /* Eq. 7 */
                    t_fwd[d] = t_fwd[d] + y * Z[u * kk + l]; /* Eq. 8 */
                }
            }
        }
        /* Phase 3 (Eq. 9) */
        for (int64_t d = 0; d < n; ++d)
            for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
                int64_t u = slot[col[e]];
                t_fwd[d] = t_fwd[d] + X[e] * Z[u * kk + (ku[u] - 1)];
            }
        free(X);
        free(ku);
    }

    if (t_rev) {
        double* qw = (double*)malloc(sizeof(double) * (size_t)hq);
        for (int32_t j = 0; j < hq; ++j) qw[j] = (double)q_w[j];
        for (int64_t d = 0; d < n; ++d) {
            int64_t a = row_ptr[d];
            int32_t hd = (int32_t)(row_ptr[d + 1] - a);
            double* pw = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1));
            double* CT = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1) * hq);
            for (int32_t i = 0; i < hd; ++i) {
                pw[i] = (double)val[a + i];
                const double* Du = D + slot[col[a + i]] * hq;
                for (int32_t j = 0; j < hq; ++j) CT[(int64_t)j * hd + i] = Du[j];
            }
            t_rev[d] = oracle_measure(measure, qw, hq, pw, hd, CT, k);
            free(CT);
            free(pw);
        }
        free(qw);
    }

    free(buf); free(s); free(W); free(Z); free(D); free(used); free(slot);
    return 0;
}

/* Phase 2 (Eq. 6-8) and Phase 3 (Eq. 9) alone, from Phase-1 tables computed elsewhere
 * (oracle_phase1 on the rows of the used vocabulary): the same steps, in the same order,
 * as the forward part of oracle_lc_query.  Table row r belongs to vocabulary id used[r];
 * row_of_id[c] = r for every column id c of the database (v entries).  Z and W are
 * (number of rows) x kk.  Returns 0, or -1 on allocation failure. */
int32_t oracle_lc_phase23(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                          const int64_t* row_of_id, const double* Z, const double* W, int32_t kk,
                          int32_t measure, int32_t hq, double* t_fwd)
{
    int64_t nnz = row_ptr[n];
    double* X = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!X) return -1;
    for (int64_t e = 0; e < nnz; ++e) X[e] = (double)val[e]; /* X^(0) = X */
    for (int64_t d = 0; d < n; ++d) t_fwd[d] = 0.0;          /* t^(0) = 0 */
    /* Phase 2 */
    for (int32_t l = 0; l < kk - 1; ++l) {
        for (int64_t d = 0; d < n; ++d) {
            for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
                int64_t u = row_of_id[col[e]];
                int32_t ku = measure == ORACLE_OMR ? ((Z[u * kk] == 0.0 && hq > 1) ? 2 : 1) : kk;
                if (l >= ku - 1) continue;
                double y = fmin(X[e], W[u * kk + l]);  /* Eq. 6 (R5) */
                X[e] = X[e] - y;                         /* Eq. 7 */
                t_fwd[d] = t_fwd[d] + y * Z[u * kk + l]; /* Eq. 8 */
            }
        }
    }
    /* Phase 3 (Eq. 9) */
    for (int64_t d = 0; d < n; ++d)
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
            int64_t u = row_of_id[col[e]];
            int32_t ku = measure == ORACLE_OMR ? ((Z[u * kk] == 0.0 && hq > 1) ? 2 : 1) : kk;
            t_fwd[d] = t_fwd[d] + X[e] * Z[u * kk + (ku - 1)];
        }
    free(X);
    return 0;
}

/* The reverse direction of oracle_lc_query alone, from a Phase-1 distance block computed
 * elsewhere: D is (number of rows) x hq, row r for vocabulary id used[r], row_of_id[c] = r
 * for every column id c of the database.  For each document the same steps as in
 * oracle_lc_query: the pairwise algorithm with the query as source and the document as
 * destination, cost block gathered from D.  Returns 0, or -1 on allocation failure. */
int32_t oracle_lc_rev(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                      const int64_t* row_of_id, const double* D, const float* q_w, int32_t hq,
                      int32_t measure, int32_t k, double* t_rev)
{
    double* qw = (double*)malloc(sizeof(double) * (size_t)hq);
    if (!qw) return -1;
    for (int32_t j = 0; j < hq; ++j) qw[j] = (double)q_w[j];
    for (int64_t d = 0; d < n; ++d) {
        int64_t a = row_ptr[d];
        int32_t hd = (int32_t)(row_ptr[d + 1] - a);
        double* pw = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1));
        double* CT = (double*)malloc(sizeof(double) * (size_t)(hd > 0 ? hd : 1) * hq);
        if (!pw || !CT) { free(CT); free(pw); free(qw); return -1; }
        for (int32_t i = 0; i < hd; ++i) {
            pw[i] = (double)val[a + i];
            const double* Du = D + row_of_id[col[a + i]] * hq;
            for (int32_t j = 0; j < hq; ++j) CT[(int64_t)j * hd + i] = Du[j];
        }
        t_rev[d] = oracle_measure(measure, qw, hq, pw, hd, CT, k);
        free(CT);
        free(pw);
    }
    free(qw);
    return 0;
}

/* Phase 1 alone (for inspecting the Z / S / W tables of Section 5): rows are the given
 * vocabulary ids; outputs are rows x kk, row-major. */
void oracle_phase1(const float* emb, int32_t m, const float* cost, int64_t v,
                   const int32_t* rows, int64_t nrows, const int32_t* q_idx, const float* q_w,
                   int32_t hq, int32_t kk, double* Z, int32_t* S, double* W)
{
    double* Du = (double*)malloc(sizeof(double) * (size_t)hq);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)hq);
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)hq);
    for (int64_t r = 0; r < nrows; ++r) {
        for (int32_t j = 0; j < hq; ++j) Du[j] = ground_cost(emb, m, cost, v, rows[r], q_idx[j]);
        argsort_row(Du, hq, s, buf);
        for (int32_t l = 0; l < kk; ++l) {
            Z[r * kk + l] = l < hq ? Du[s[l]] : INFINITY;
            S[r * kk + l] = l < hq ? s[l] : -1;
            W[r * kk + l] = l < hq ? (double)q_w[s[l]] : 0.0;
        }
    }
    free(buf); free(s); free(Du);
}

/* ------------------------------------------------------------------ Section 6 baselines */

/* Bag-of-words cosine similarity of the query with every database histogram (Section 6:
 * the dot product of the two weight vectors after L2 normalisation; it ignores the
 * embeddings).  Coordinates held by one side only contribute nothing.  A histogram with
 * zero norm has similarity 0.  Returns 0, or -1 on allocation failure. */
int32_t oracle_bow_db(int64_t v, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                      const int32_t* q_idx, const float* q_w, int32_t hq, double* out)
{
    double* dense = (double*)calloc((size_t)(v > 0 ? v : 1), sizeof(double));
    if (!dense) return -1;
    double qn = 0.0;
    for (int32_t j = 0; j < hq; ++j) {
        dense[q_idx[j]] = (double)q_w[j];
        qn += (double)q_w[j] * (double)q_w[j];
    }
    qn = sqrt(qn);
    for (int64_t d = 0; d < n; ++d) {
        double dot = 0.0, dn = 0.0;
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
            dot += (double)val[e] * dense[col[e]];
            dn += (double)val[e] * (double)val[e];
        }
        dn = sqrt(dn);
        out[d] = (qn > 0.0 && dn > 0.0) ? dot / (qn * dn) : 0.0;
    }
    free(dense);
    return 0;
}

/* Word centroid distance (Section 6, after Kusner et al.): the Euclidean distance between
 * the weighted averages sum_i p_i E_i / sum_i p_i of the two histograms' embedding vectors.
 * Returns 0, or -1 on allocation failure. */
int32_t oracle_wcd_db(const float* emb, int32_t m, const int64_t* row_ptr, const int32_t* col, const float* val,
                      int64_t n, const int32_t* q_idx, const float* q_w, int32_t hq, double* out)
{
    double* cq = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double* cd = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    if (!cq || !cd) { free(cq); free(cd); return -1; }
    double sq = 0.0;
    for (int32_t j = 0; j < hq; ++j) {
        sq += (double)q_w[j];
        for (int32_t i = 0; i < m; ++i) cq[i] += (double)q_w[j] * (double)emb[(int64_t)q_idx[j] * m + i];
    }
    for (int32_t i = 0; i < m; ++i) cq[i] /= sq;
    for (int64_t d = 0; d < n; ++d) {
        double sd = 0.0;
        for (int32_t i = 0; i < m; ++i) cd[i] = 0.0;
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
            sd += (double)val[e];
            for (int32_t i = 0; i < m; ++i) cd[i] += (double)val[e] * (double)emb[(int64_t)col[e] * m + i];
        }
        double s = 0.0;
        for (int32_t i = 0; i < m; ++i) {
            const double diff = cd[i] / sd - cq[i];
            s += diff * diff;
        }
        out[d] = sqrt(s);
    }
    free(cq);
    free(cd);
    return 0;
}
