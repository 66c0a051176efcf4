/*
 * erq_oracle.c -- plain FP64 CPU oracle for extended RaBitQ search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA path; the two meet only in the
 * seeded inputs of synthetic/.
 *
 * Every function restates one step of the paper (arXiv 2409.09913) in the
 * most direct form: FP64 arithmetic, sequential loops, library sort.  Inputs
 * stored as FP32 are read as exact values.  Compile with -ffp-contract=off so
 * that no multiply-add is fused.
 *
 * Readings of the paper that this file fixes (each is repeated beside the code
 * it governs):
 *  R1  centroid c = mean of the rows assigned to the cluster (Section 5.1,
 *      "center every cluster ... with its local centroid"), summed in FP64 in
 *      ascending row order and rounded once to FP32.
 *  R2  the residual o_r - c is rounded once to FP32, and the rotated residual
 *      o' = P^{-1}(o_r - c) = P^T(o_r - c) (Section 3.3 workflow) is
 *      accumulated in FP64 in ascending input index and rounded once to FP32.
 *      Algorithm 1 is scale invariant, so it runs on this unnormalised o'.
 *  R3  Algorithm 1 state: |y_i| = m_i + 1/2, m_i in {0..2^(B-1)-1}; the
 *      initial state (t -> 0+) is evaluated before any event, so that B = 1
 *      returns the RaBitQ sign code (Section 3.1, B = 1 remark).
 *  R4  critical values: coordinate i moves from m to m+1 at t = (m+1)/|o'_i|
 *      (the half-integer-grid form of "(x+0.5)/o'[i]", Section 3.1); events
 *      are ordered by the exact rational value, ties by ascending i.
 *  R5  <y_cur, o'> is updated in FP64 in event order; ||y_cur||^2 is exact;
 *      v = ip / sqrt(n2) with correctly rounded sqrt and division; the
 *      maximum is strict (first state reaching it wins); the returned code is
 *      the recorded state, not a re-rounding of t_max * o'.
 *  R6  sign convention sgn(0) = + (Appendix B, proof of Lemma B.3).
 *  R7  the stored norm ||o_r - c|| is read as ||o'|| (equal in exact
 *      arithmetic because P is orthogonal), and the second stored float is
 *      1/(||ybar|| <o, obar>) (Section 5.1 metrics paragraph, with ||ybar||
 *      in place of the printed ||y_u||, as Eq. 3.3 requires).
 *  R8  o_r = c (zero residual): code of all +1/2 entries, both factors 0, so
 *      the estimate is ||q_r - c||^2.
 *  R9  inner-product metric (Section 7 points to RaBitQ for it): split
 *      <o_r, q_r> = <c, q_r> + ||o_r - c|| <o, q_r> with o the unit residual,
 *      and estimate <o, q^> for the unit query q^ = q_r/||q_r|| (no centroid
 *      subtracted) by the same unbiased estimator <obar, q^>/<obar, o> as the
 *      distance (Section 3.3); so est = <c, q_r> + ||o_r - c|| ||q_r|| *
 *      <obar, q^>/<obar, o>.  Probing takes the nprobe largest <q_r, c_j>,
 *      the re-rank the exact <o_r, q_r>; results are ordered by decreasing
 *      inner product, ties by lower id (internally: ascending -<.,.>).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* R1: local centroids.                                                     */
/* ------------------------------------------------------------------------ */
void orc_centroids(const float* X, int64_t n, int d, const int32_t* assign, int nlist, float* C)
{
    double* acc = (double*)calloc((size_t)nlist * d, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)nlist, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int32_t j = assign[i];
        double* a = acc + (size_t)j * d;
        const float* x = X + (size_t)i * d;
        for (int k = 0; k < d; ++k) a[k] += (double)x[k];
        cnt[j] += 1;
    }
    for (int j = 0; j < nlist; ++j)
        for (int k = 0; k < d; ++k)
            C[(size_t)j * d + k] = cnt[j] ? (float)(acc[(size_t)j * d + k] / (double)cnt[j]) : 0.0f;
    free(acc);
    free(cnt);
}

/* ------------------------------------------------------------------------ */
/* R2: rotation.  out[i][j] = fl32( sum_k r_k * P[k][j] ), r_k = fl32(x_k -   */
/* c_k) (or x_k when C is NULL), i.e. the row form of P^T r.                  */
/* ------------------------------------------------------------------------ */
void orc_rotate(const float* X, const float* C, const int32_t* assign, int64_t n, int d,
                const float* P, float* out)
{
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * d);
        float* r = (float*)malloc(sizeof(float) * d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const float* x = X + (size_t)i * d;
            if (C) {
                const float* c = C + (size_t)(assign ? assign[i] : 0) * d;
                for (int k = 0; k < d; ++k) r[k] = (float)((double)x[k] - (double)c[k]);
            } else {
                for (int k = 0; k < d; ++k) r[k] = x[k];
            }
            for (int j = 0; j < d; ++j) acc[j] = 0.0;
            for (int k = 0; k < d; ++k) {
                const double rk = (double)r[k];
                const float* p = P + (size_t)k * d;
                for (int j = 0; j < d; ++j) acc[j] += rk * (double)p[j];
            }
            for (int j = 0; j < d; ++j) out[(size_t)i * d + j] = (float)acc[j];
        }
        free(acc);
        free(r);
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Quantize), Section 3.1, with the min-heap of critical values */
/* described in the complexity paragraph.                                     */
/* ------------------------------------------------------------------------ */
typedef struct { int i; int m; } orc_event; /* coordinate i goes from m to m+1 */

/* R4: t_x < t_y  <=>  (m_x+1)/a_x < (m_y+1)/a_y  <=>  (m_x+1)*a_y < (m_y+1)*a_x.
 * a_* are FP32 magnitudes and m+1 <= 2^9, so both products are exact in FP64. */
static int ev_before(const double* a, orc_event x, orc_event y)
{
    const double lhs = (double)(x.m + 1) * a[y.i];
    const double rhs = (double)(y.m + 1) * a[x.i];
    if (lhs != rhs) return lhs < rhs;
    return x.i < y.i;
}

static void heap_push(orc_event* h, int* n, orc_event e, const double* a)
{
    int k = (*n)++;
    h[k] = e;
    while (k > 0) {
        int p = (k - 1) / 2;
        if (!ev_before(a, h[k], h[p])) break;
        orc_event t = h[k]; h[k] = h[p]; h[p] = t;
        k = p;
    }
}

static orc_event heap_pop(orc_event* h, int* n, const double* a)
{
    orc_event top = h[0];
    h[0] = h[--(*n)];
    int k = 0;
    for (;;) {
        int l = 2 * k + 1, r = l + 1, s = k;
        if (l < *n && ev_before(a, h[l], h[s])) s = l;
        if (r < *n && ev_before(a, h[r], h[s])) s = r;
        if (s == k) break;
        orc_event t = h[k]; h[k] = h[s]; h[s] = t;
        k = s;
    }
    return top;
}

/* Quantize one rotated residual rp[0..d-1] with B bits per coordinate.
 * Writes the unsigned code ybar_u (16 bits per coordinate, B <= 9) and
 * stats[0..4] = { <ybar,|o'|> (ip at the optimum), ||ybar||^2, v_max,
 * ||o'||^2, number of events }. */
void orc_quantize(const float* rp, int d, int B, uint16_t* code, double* stats)
{
    const int M = (1 << (B - 1)) - 1;           /* events per coordinate */
    const int half = 1 << (B - 1);
    double* a = (double*)malloc(sizeof(double) * d);
    int* m = (int*)malloc(sizeof(int) * d);
    orc_event* heap = (orc_event*)malloc(sizeof(orc_event) * (d > 0 ? d : 1));
    double s = 0.0, nr2 = 0.0;
    for (int i = 0; i < d; ++i) {
        a[i] = fabs((double)rp[i]);
        s += a[i];
        nr2 += (double)rp[i] * (double)rp[i];
    }
    /* R3: initial state y_cur = (1/2,...,1/2) in the orthant of o'. */
    double ip = 0.5 * s;
    double n2 = 0.25 * (double)d;
    double vmax = ip / sqrt(n2);
    double ip_best = ip, n2_best = n2;
    long long kbest = 0, k = 0;
    int hn = 0;
    if (M > 0)
        for (int i = 0; i < d; ++i)
            if (a[i] > 0.0) heap_push(heap, &hn, (orc_event){i, 0}, a);
    while (hn > 0) {
        orc_event e = heap_pop(heap, &hn, a);
        ++k;
        ip += a[e.i];                            /* R5: O(1) update */
        n2 += 2.0 * (double)(e.m + 1);           /* (m+3/2)^2 - (m+1/2)^2 */
        double v = ip / sqrt(n2);
        if (v > vmax) { vmax = v; kbest = k; ip_best = ip; n2_best = n2; }
        if (e.m + 1 < M) heap_push(heap, &hn, (orc_event){e.i, e.m + 1}, a);
    }
    /* R5: replay the first kbest events to recover the recorded state. */
    for (int i = 0; i < d; ++i) m[i] = 0;
    hn = 0;
    if (M > 0 && kbest > 0)
        for (int i = 0; i < d; ++i)
            if (a[i] > 0.0) heap_push(heap, &hn, (orc_event){i, 0}, a);
    for (long long j = 0; j < kbest; ++j) {
        orc_event e = heap_pop(heap, &hn, a);
        m[e.i] = e.m + 1;
        if (e.m + 1 < M) heap_push(heap, &hn, (orc_event){e.i, e.m + 1}, a);
    }
    /* ybar_u = ybar + (2^B-1)/2: +(m+1/2) -> half+m, -(m+1/2) -> half-1-m (R6). */
    for (int i = 0; i < d; ++i)
        code[i] = (uint16_t)(rp[i] >= 0.0f ? half + m[i] : half - 1 - m[i]);
    stats[0] = ip_best;
    stats[1] = n2_best;
    stats[2] = vmax;
    stats[3] = nr2;
    stats[4] = (double)k;
    free(a);
    free(m);
    free(heap);
}

void orc_quantize_batch(const float* Rp, int64_t n, int d, int B, uint16_t* codes, double* stats)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        orc_quantize(Rp + (size_t)i * d, d, B, codes + (size_t)i * d, stats + (size_t)i * 5);
}

/* ------------------------------------------------------------------------ */
/* Eq. (eq:dis to ip) + Eq. 3.3: estimated squared distance.                */
/* ------------------------------------------------------------------------ */
/* Per-vector stored quantities (R7): nr = ||o_r - c||, inv = 1/(||ybar|| <o,obar>). */
static void vec_factors(const double* st, double* nr, double* inv)
{
    const double nr2 = st[3];
    if (nr2 > 0.0) {
        *nr = sqrt(nr2);
        const double ybar_norm = sqrt(st[1]);
        const double o_obar = st[2] / *nr;      /* <o, obar> = v_max / ||o'|| */
        *inv = 1.0 / (ybar_norm * o_obar);
    } else {                                     /* R8 */
        *nr = 0.0;
        *inv = 0.0;
    }
}

/* Query-side quantities for one (query, centroid) pair: the normalised,
 * rotated query q' = P^{-1} (q_r - c)/||q_r - c|| (Section 3.3 workflow),
 * sum_i q'[i], and ||q_r - c||. */
static void query_side(const double* q, const float* c, const float* P, int d,
                       double* qn, double* qp, double* sum_qp, double* qc_norm)
{
    double n2 = 0.0;
    for (int k = 0; k < d; ++k) { qn[k] = q[k] - (double)c[k]; n2 += qn[k] * qn[k]; }
    *qc_norm = sqrt(n2);
    if (n2 > 0.0)
        for (int k = 0; k < d; ++k) qn[k] /= *qc_norm;
    for (int j = 0; j < d; ++j) qp[j] = 0.0;
    for (int k = 0; k < d; ++k) {
        const float* p = P + (size_t)k * d;
        for (int j = 0; j < d; ++j) qp[j] += qn[k] * (double)p[j];
    }
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += qp[j];
    *sum_qp = s;
}

static double estimate_one(const uint16_t* code, const double* st, int d, int B,
                           const double* qp, double sum_qp, double qc_norm)
{
    double nr, inv;
    vec_factors(st, &nr, &inv);
    double ipu = 0.0;                            /* <ybar_u, q'> */
    for (int j = 0; j < d; ++j) ipu += (double)code[j] * qp[j];
    const double obar_q = ipu - 0.5 * (double)((1 << B) - 1) * sum_qp;  /* ||ybar|| <obar, q> */
    /* <o,q> estimate = <obar,q>/<obar,o> = (||ybar||<obar,q>) * inv */
    const double ip_est = obar_q * inv;
    return nr * nr + qc_norm * qc_norm - 2.0 * nr * qc_norm * ip_est;
}

/* R9: estimated inner product <o_r, q_r>.  qp = P^{-1} q^ with q^ = q_r/||q_r||
 * (query_ip_side), sum_qp = sum_i qp[i], q_norm = ||q_r||, c_q = <c, q_r>. */
static double estimate_ip_one(const uint16_t* code, const double* st, int d, int B,
                              const double* qp, double sum_qp, double q_norm, double c_q)
{
    double nr, inv;
    vec_factors(st, &nr, &inv);
    double ipu = 0.0;                            /* <ybar_u, q'> */
    for (int j = 0; j < d; ++j) ipu += (double)code[j] * qp[j];
    const double obar_q = ipu - 0.5 * (double)((1 << B) - 1) * sum_qp;  /* ||ybar|| <obar, q^> */
    return c_q + nr * q_norm * (obar_q * inv);
}

/* Query-side quantities of the inner-product metric for one centroid:
 * q' = P^{-1} q_r/||q_r||, its coordinate sum, ||q_r|| and <c, q_r>. */
static void query_ip_side(const double* q, const float* c, const float* P, int d,
                          double* qn, double* qp, double* sum_qp, double* q_norm, double* c_q)
{
    double n2 = 0.0, cq = 0.0;
    for (int k = 0; k < d; ++k) { qn[k] = q[k]; n2 += q[k] * q[k]; cq += (double)c[k] * q[k]; }
    *q_norm = sqrt(n2);
    *c_q = cq;
    if (n2 > 0.0)
        for (int k = 0; k < d; ++k) qn[k] /= *q_norm;
    for (int j = 0; j < d; ++j) qp[j] = 0.0;
    for (int k = 0; k < d; ++k) {
        const float* p = P + (size_t)k * d;
        for (int j = 0; j < d; ++j) qp[j] += qn[k] * (double)p[j];
    }
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += qp[j];
    *sum_qp = s;
}

/* Index arrays (cluster-major): list_off[nlist+1] row offsets, list_ids[n]
 * original row id of each stored row, codes[n][d], stats[n][5] from
 * orc_quantize, X[n][d] raw rows in ORIGINAL order (for exact distances). */
typedef struct {
    int d, B, nlist;
    const float* P;
    const float* C;
    const int64_t* list_off;
    const int64_t* list_ids;
    const uint16_t* codes;
    const double* stats;
    const float* X;
} orc_index;

typedef struct { double key; int64_t id; } orc_pair;

static int pair_cmp(const void* x, const void* y)
{
    const orc_pair* a = (const orc_pair*)x;
    const orc_pair* b = (const orc_pair*)y;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

static double exact_dist(const float* x, const double* q, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) { double t = (double)x[k] - q[k]; s += t * t; }
    return s;
}

static double exact_ip(const float* x, const double* q, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += (double)x[k] * q[k];
    return s;
}

/* IVF probe (Section 4.1): the nprobe centroids nearest to q (metric 0) or
 * with the largest <q, c> (metric 1, R9), ties by id. */
static void probe_one(const orc_index* ix, const double* q, int nprobe, int metric, int32_t* out)
{
    orc_pair* cd = (orc_pair*)malloc(sizeof(orc_pair) * ix->nlist);
    for (int j = 0; j < ix->nlist; ++j) {
        const float* c = ix->C + (size_t)j * ix->d;
        cd[j].key = metric ? -exact_ip(c, q, ix->d) : exact_dist(c, q, ix->d);
        cd[j].id = j;
    }
    qsort(cd, ix->nlist, sizeof(orc_pair), pair_cmp);
    for (int p = 0; p < nprobe; ++p) out[p] = (int32_t)cd[p].id;
    free(cd);
}

/* One query of the search path: probe -> estimate every candidate -> top-k'
 * by estimate -> exact re-rank of those k' -> top-k.  With kprime <= 0 the
 * estimated top-k is returned (the paper's no-re-rank setting, Section 4.1).
 * probe may be given (nprobe entries) or computed when probe_in is NULL.
 * metric 0: squared distances, ascending; metric 1: inner products (R9),
 * descending -- sorted as ascending -<.,.> and reported with their sign. */
static void search_one(const orc_index* ix, const double* q, int nprobe, const int32_t* probe_in,
                       int kprime, int k, int metric, int64_t* ids, double* dists,
                       int64_t* cand_ids, double* cand_est, int32_t* probe_out)
{
    const int d = ix->d;
    const double sgn = metric ? -1.0 : 1.0;
    int32_t* probe = (int32_t*)malloc(sizeof(int32_t) * (nprobe > 0 ? nprobe : 1));
    if (probe_in) memcpy(probe, probe_in, sizeof(int32_t) * nprobe);
    else probe_one(ix, q, nprobe, metric, probe);
    if (probe_out) memcpy(probe_out, probe, sizeof(int32_t) * nprobe);
    int64_t ncand = 0;
    for (int p = 0; p < nprobe; ++p) ncand += ix->list_off[probe[p] + 1] - ix->list_off[probe[p]];
    orc_pair* cand = (orc_pair*)malloc(sizeof(orc_pair) * (ncand > 0 ? ncand : 1));
    double* qn = (double*)malloc(sizeof(double) * d);
    double* qp = (double*)malloc(sizeof(double) * d);
    int64_t w = 0;
    for (int p = 0; p < nprobe; ++p) {
        const int c = probe[p];
        double sum_qp, qc_norm, q_norm, c_q;
        if (metric)
            query_ip_side(q, ix->C + (size_t)c * d, ix->P, d, qn, qp, &sum_qp, &q_norm, &c_q);
        else
            query_side(q, ix->C + (size_t)c * d, ix->P, d, qn, qp, &sum_qp, &qc_norm);
        for (int64_t r = ix->list_off[c]; r < ix->list_off[c + 1]; ++r) {
            const uint16_t* code = ix->codes + (size_t)r * d;
            const double* st = ix->stats + (size_t)r * 5;
            cand[w].key = metric ? -estimate_ip_one(code, st, d, ix->B, qp, sum_qp, q_norm, c_q)
                                 : estimate_one(code, st, d, ix->B, qp, sum_qp, qc_norm);
            cand[w].id = ix->list_ids[r];
            ++w;
        }
    }
    qsort(cand, (size_t)ncand, sizeof(orc_pair), pair_cmp);
    const int kp = kprime > 0 ? kprime : k;
    const int64_t nk = ncand < kp ? ncand : kp;
    for (int j = 0; j < kp; ++j) {
        if (cand_ids) cand_ids[j] = j < nk ? cand[j].id : -1;
        if (cand_est) cand_est[j] = j < nk ? sgn * cand[j].key : sgn * INFINITY;
    }
    if (kprime > 0) {
        for (int64_t j = 0; j < nk; ++j) {
            const float* x = ix->X + (size_t)cand[j].id * d;
            cand[j].key = metric ? -exact_ip(x, q, d) : exact_dist(x, q, d);
        }
        qsort(cand, (size_t)nk, sizeof(orc_pair), pair_cmp);
    }
    for (int j = 0; j < k; ++j) {
        ids[j] = j < nk ? cand[j].id : -1;
        dists[j] = j < nk ? sgn * cand[j].key : sgn * INFINITY;
    }
    free(probe); free(cand); free(qn); free(qp);
}

void orc_search(int d, int B, int nlist, const float* P, const float* C, const int64_t* list_off,
                const int64_t* list_ids, const uint16_t* codes, const double* stats, const float* X,
                const double* Q, int64_t nq, const int32_t* nprobe, const int32_t* probe_in, int max_probe,
                int kprime, int k, int metric, int64_t* ids, double* dists, int64_t* cand_ids, double* cand_est,
                int32_t* probe_out)
{
    orc_index ix = {d, B, nlist, P, C, list_off, list_ids, codes, stats, X};
    const int kp = kprime > 0 ? kprime : k;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nq; ++i)
        search_one(&ix, Q + (size_t)i * d, nprobe[i], probe_in ? probe_in + (size_t)i * max_probe : NULL,
                   kprime, k, metric, ids + (size_t)i * k, dists + (size_t)i * k,
                   cand_ids ? cand_ids + (size_t)i * kp : NULL, cand_est ? cand_est + (size_t)i * kp : NULL,
                   probe_out ? probe_out + (size_t)i * max_probe : NULL);
}

/* Centroid distances ||q - c_j||^2 for every query and centroid (FP64). */
void orc_centroid_dists(const float* C, int nlist, int d, const double* Q, int64_t nq, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nq; ++i)
        for (int j = 0; j < nlist; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) { double t = Q[(size_t)i * d + k] - (double)C[(size_t)j * d + k]; s += t * t; }
            out[(size_t)i * nlist + j] = s;
        }
}

/* Estimated distance (metric 0) or inner product (metric 1, R9) for explicit
 * (query, stored row) pairs; rows index the cluster-major arrays and cl gives
 * the cluster of each row. */
void orc_estimate_rows(int d, int B, const float* P, const float* C, const uint16_t* codes, const double* stats,
                       const double* Q, int64_t nq, int nc, const int64_t* rows, const int32_t* cl, int metric,
                       double* out)
{
#pragma omp parallel
    {
        double* qn = (double*)malloc(sizeof(double) * d);
        double* qp = (double*)malloc(sizeof(double) * d);
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nq; ++i)
            for (int j = 0; j < nc; ++j) {
                const int64_t r = rows[(size_t)i * nc + j];
                if (r < 0) { out[(size_t)i * nc + j] = NAN; continue; }
                double sum_qp, qc_norm, q_norm, c_q;
                if (metric) {
                    query_ip_side(Q + (size_t)i * d, C + (size_t)cl[r] * d, P, d, qn, qp, &sum_qp, &q_norm, &c_q);
                    out[(size_t)i * nc + j] = estimate_ip_one(codes + (size_t)r * d, stats + (size_t)r * 5, d, B,
                                                              qp, sum_qp, q_norm, c_q);
                } else {
                    query_side(Q + (size_t)i * d, C + (size_t)cl[r] * d, P, d, qn, qp, &sum_qp, &qc_norm);
                    out[(size_t)i * nc + j] = estimate_one(codes + (size_t)r * d, stats + (size_t)r * 5, d, B,
                                                           qp, sum_qp, qc_norm);
                }
            }
        free(qn);
        free(qp);
    }
}

/* Gradient of the estimated scores w.r.t. the raw query, codes and ids fixed.
 * From Eq. (eq:dis to ip) and Eq. 3.3 with unnormalised q~ = P^T(q_r - c):
 *   est = ||o'||^2 + ||q_r - c||^2 + f * <ybar, P^T (q_r - c)>,
 *   f   = -2 ||o_r - c|| * inv,  ybar = ybar_u - (2^B-1)/2,
 * so d est / d q_r = 2 (q_r - c) + f * P ybar.  grad_q = sum_j g_j d est_j/d q_r. */
void orc_backward(int d, int B, const float* P, const float* C, const uint16_t* codes, const double* stats,
                  const double* Q, int64_t nq, int nc, const int64_t* rows, const int32_t* cl,
                  const double* g, int metric, double* grad)
{
#pragma omp parallel
    {
        double* v = (double*)malloc(sizeof(double) * d);
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nq; ++i) {
            double* gq = grad + (size_t)i * d;
            for (int k = 0; k < d; ++k) gq[k] = 0.0;
            for (int j = 0; j < nc; ++j) {
                const int64_t r = rows[(size_t)i * nc + j];
                if (r < 0) continue;
                const double gj = g[(size_t)i * nc + j];
                double nr, inv;
                vec_factors(stats + (size_t)r * 5, &nr, &inv);
                const double f = -2.0 * nr * inv;
                const float* c = C + (size_t)cl[r] * d;
                const uint16_t* code = codes + (size_t)r * d;
                for (int k = 0; k < d; ++k) v[k] = (double)code[k] - 0.5 * (double)((1 << B) - 1);
                for (int k = 0; k < d; ++k) {
                    double pv = 0.0;                /* (P ybar)[k] */
                    const float* p = P + (size_t)k * d;
                    for (int m = 0; m < d; ++m) pv += (double)p[m] * v[m];
                    /* R9: est = <c, q_r> + ||o_r - c|| inv <ybar, P^T q_r>, so
                     * d est / d q_r = c - (f / 2) P ybar */
                    gq[k] += metric ? gj * ((double)c[k] - 0.5 * f * pv)
                                    : gj * (2.0 * (Q[(size_t)i * d + k] - (double)c[k]) + f * pv);
                }
            }
        }
        free(v);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
