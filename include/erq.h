/*
 * erq.h -- C ABI of the GB300 extended-RaBitQ search library (liberq.so).
 *
 * Extended RaBitQ (Gao et al., arXiv 2409.09913) quantizes each data vector
 * o_r, after local centring o_r - c and a random orthogonal rotation
 * o' = P^{-1}(o_r - c), to a B-bit-per-coordinate code ybar_u (Section 3.1,
 * Algorithm 1) and estimates squared distances to a query q_r from the code,
 * two per-vector floats and the rotated query (Eq. 3.3 with
 * Eq. (eq:dis to ip)), or inner products with the same estimator (the
 * adaptation Section 7 defers to RaBitQ; see erq_search).  Combined with an
 * IVF index (Section 4.1) this gives approximate nearest-neighbour or
 * maximum-inner-product search; the library adds exact re-ranking of the
 * estimated top-k' and the gradient of the estimated scores with respect to
 * the query.
 *
 * Conventions for every entry point:
 *  - Array arguments are caller-owned CUDA device pointers unless the name
 *    ends in _host.  The library never frees caller memory.
 *  - Matrices are row-major and contiguous: X[N][D], P[D][D], Q[nq][D].
 *  - D must be a multiple of 64 (the paper pads to a multiple of 64,
 *    Section 5.1) and at most 4096; B is 1..9; N < 2^31.
 *  - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  Host-side validation errors return before any work is
 *    queued.  Device-side errors (a wait that ran out, a bound that failed) are
 *    recorded in a status word held by the index and returned by the next call
 *    on that index or by erq_index_status().
 *  - Every function returns an erq_status; on failure erq_last_error() gives a
 *    thread-local message.
 *  - A single erq_index may be used by one host thread at a time (it owns one
 *    search workspace).
 */
#ifndef ERQ_H
#define ERQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ERQ_OK = 0,
    ERQ_EINVAL = 1,          /* bad argument (shape, range, null pointer)      */
    ERQ_ENOMEM = 2,          /* device or host allocation failed               */
    ERQ_ECUDA = 3,           /* a CUDA runtime call or kernel launch failed    */
    ERQ_ETIMEOUT = 4,        /* a bounded device-side wait ran out             */
    ERQ_EUNSUPPORTED = 5,    /* valid request the library or GPU cannot serve  */
    ERQ_EIO = 6              /* file error in save/load                        */
} erq_status;

/* Arithmetic of the code-by-query contraction in erq_search. */
typedef enum {
    ERQ_PREC_FP32 = 0,       /* CUDA-core FP32 FFMA scan (reference GPU path)           */
    ERQ_PREC_FP16 = 1,       /* tcgen05 kind::f16: codes exact, rotated query in FP16,
                                FP32 accumulation in tensor memory                       */
    ERQ_PREC_FP8 = 2,        /* tcgen05 kind::f8f6f4: query rounded to e4m3 after a
                                per-query power-of-two scale, centred codes exact in
                                e4m3 (B <= 4 directly; B = 5..8 as 16 hc + lc, two
                                e4m3 parts of magnitude <= 15 each, Section 3.3;
                                B = 9 -> ERQ_EUNSUPPORTED), FP32 accumulation in
                                tensor memory                                            */
    ERQ_PREC_INT8 = 3        /* int8 tensor MMA: unavailable on sm_103a (ptxas rejects
                                tcgen05 kind::i8) -> ERQ_EUNSUPPORTED                    */
} erq_precision;

typedef struct erq_index erq_index;   /* opaque; owns all of its device memory */

/* Index construction parameters (Section 3.3 workflow, Section 4.1 IVF). */
typedef struct {
    int32_t B;                /* bits per coordinate, 1..9                               */
    int32_t nlist;            /* IVF clusters; 1 = no IVF (one cluster, c = mean of X)   */
    const float* P;           /* device [D][D] orthogonal matrix (the method's random
                                 draw, Section 3.1 Eq. equ:rotation); required            */
    const int32_t* assign;    /* device [N] cluster of each row, or NULL: the library runs
                                 k-means (Lloyd) on the GPU to make one                   */
    int32_t kmeans_iters;     /* Lloyd iterations when assign == NULL (default 10)        */
    int32_t kmeans_sample;    /* rows sampled for k-means training, 0 = all              */
    uint64_t seed;            /* k-means initialisation seed                             */
    int32_t keep_raw;         /* keep the FP32 rows in the index (exact re-rank needs it)*/
    int32_t normalize;        /* 1: scale every row to unit length first (FP64 norm, one
                                 rounding), so that ERQ_METRIC_COS searches are the
                                 inner product of unit vectors; kept raw rows are the
                                 scaled ones                                              */
    const float* centroids;   /* optional device [nlist][D] centroids to use instead of the
                                 means of the rows (requires assign; lists may then be
                                 empty): an index over one shard of a larger index's lists
                                 keeps the larger index's centroids, codes and probe      */
} erq_build_params;

/* Search parameters. */
typedef struct {
    int32_t k;                /* neighbours returned per query (>= 1)                    */
    int32_t rerank_k;         /* k' >= k candidates (by estimate) re-ranked with exact
                                 distances; 0 = return the estimated top-k (no re-rank)  */
    int32_t nprobe;           /* clusters probed per query (1..nlist) when
                                 nprobe_per_query is NULL                                */
    int32_t precision;        /* erq_precision                                           */
    const int32_t* nprobe_per_query; /* optional device [nq], each 1..nlist               */
    const int32_t* probe;     /* optional device [nq][probe_stride] explicit probe lists
                                 (distinct cluster ids; replaces the centroid search)    */
    int32_t probe_stride;     /* row stride of `probe` (>= max nprobe)                   */
    int32_t flags;            /* ERQ_SEARCH_TIMING: record per-phase CUDA events         */
    int64_t* cand_ids;        /* optional device out [nq][kc], kc = max(k, rerank_k):
                                 ids of the estimated top-kc, ascending by estimate      */
    float* cand_est;          /* optional device out [nq][kc]: their estimates            */
    int32_t metric;           /* erq_metric (0 = ERQ_METRIC_L2)                          */
} erq_search_params;

/* erq_search_params.metric */
typedef enum {
    ERQ_METRIC_L2 = 0,        /* squared Euclidean distance, smallest first               */
    ERQ_METRIC_IP = 1,        /* inner product, largest first (see erq_search)            */
    ERQ_METRIC_COS = 2        /* cosine similarity, largest first: the inner product of
                                 unit vectors.  Needs an index built with normalize = 1;
                                 the query is scaled to unit length, then searched as
                                 ERQ_METRIC_IP; dists / cand_est hold cosines.  Search
                                 only (erq_search, erq_search_host)                       */
} erq_metric;

/* erq_search_params.flags */
#define ERQ_SEARCH_TIMING 1      /* record per-phase CUDA events (erq_search_timing)        */
#define ERQ_SEARCH_SIMT_GEMM 2   /* run the query rotation and centroid distances on the
                                    CUDA-core SGEMM instead of the tensor-core FP32 GEMM    */
#define ERQ_SEARCH_ASYNC 4       /* no host synchronisation inside the call: work buffers are
                                    sized from host-side upper bounds, so the call can be
                                    recorded into a CUDA graph once a first call with the
                                    same (nq, nprobe, k') has sized them; device-side errors
                                    surface at the next synchronous call or erq_index_status.
                                    Ignored with explicit probe lists, which are sized from a
                                    read-back (their distinctness is not checked)          */

/* Read-only description of an index. */
typedef struct {
    int64_t N;
    int32_t D, B, nlist, keep_raw;
    int64_t max_list;         /* rows in the largest cluster                             */
    int64_t device_bytes;     /* device memory held by the index                         */
} erq_index_info;

/* Fields copied out by erq_index_export (cluster-major order unless noted). */
typedef enum {
    ERQ_FIELD_CENTROIDS = 0,      /* float  [nlist][D]  c_j (means of their rows)          */
    ERQ_FIELD_ROT_CENTROIDS = 1,  /* float  [nlist][D]  c'_j = P^T c_j (FP64 accumulated)  */
    ERQ_FIELD_LIST_OFFSETS = 2,   /* int64  [nlist+1]   first stored row of each cluster   */
    ERQ_FIELD_LIST_IDS = 3,       /* int64  [N]         original row id of each stored row */
    ERQ_FIELD_CODES = 4,          /* [N][D] ybar_u: uint8 (B <= 8) or little-endian uint16 (B = 9) */
    ERQ_FIELD_F_ADD = 5,          /* float  [N]         ||o'||^2                           */
    ERQ_FIELD_F_RES = 6,          /* float  [N]         -2 ||o'||^2 / <ybar, |o'|>          */
    ERQ_FIELD_P = 7,              /* float  [D][D]                                         */
    ERQ_FIELD_RAW = 8,            /* float  [N][D] original order (keep_raw only)          */
    ERQ_FIELD_PACKED_CODES = 9    /* uint8  [Np*D*B/8] the tensor-core scan's packed copy:  */
                                  /* each cluster padded to a multiple of 32 rows (Np rows  */
                                  /* in all; padding rows hold code 0), stored as 64-bit    */
                                  /* words [tile of 32 rows][block of 64 coordinates][B][32]*/
                                  /* (little-endian).  In block k, for codes u[0..63] of a  */
                                  /* row, the two 32-bit halves h = 0..7 of words 0-3 hold  */
                                  /* (B >= 4) byte L = u[8h+L] & 15 | (u[8h+4+L] & 15) << 4, */
                                  /* and word b (b >= 4, or every b < B when B < 4) is bit  */
                                  /* plane b: bit 8L + (m & 7) of half m >> 3 is bit b of   */
                                  /* u[4m + L].  B bits per coordinate exactly.             */
} erq_field;

const char* erq_version(void);
/* Message of the last failed call on this host thread ("" if none). */
const char* erq_last_error(void);

/* Build an IVF + extended-RaBitQ index from X (device [N][D]) -- Section 3.3
 * workflow and Section 4.1:
 *   c_j  = mean of the rows of cluster j (FP64 sum in ascending row id, rounded
 *          once to FP32; Section 5.1 local centring),
 *   o'   = fl32(P^T fl32(o_r - c)) accumulated in FP64 in ascending index,
 *   code = Algorithm 1 on o' (FP64 comparisons; bit-identical to a sequential
 *          FP64 implementation),
 *   plus the per-vector factors (Section 5.1 metrics paragraph).
 * X and P are read during the call only.  *out receives a new index owned by the
 * caller (free with erq_free_index).  The call synchronises `stream` before it
 * returns.  Errors: EINVAL (shape/B/nlist/assign range), ENOMEM, ECUDA. */
erq_status erq_build_index(const float* X, int64_t N, int32_t D, const erq_build_params* params,
                           void* stream, erq_index** out);

void erq_free_index(erq_index* index);
erq_status erq_index_info_get(const erq_index* index, erq_index_info* info);
/* Synchronise `stream` and return (then clear) the device status word. */
erq_status erq_index_status(erq_index* index, void* stream);

/* out[n][D] = X[n][D] * P, i.e. each row becomes P^T x = P^{-1} x (Section 2.2,
 * Eq. sec 2 qprime; Section 3.3 workflow).  accurate != 0: FP64 accumulation in
 * ascending index, one rounding to FP32 (index time); accurate == 0: FP32
 * accumulation (query time).  Errors: EINVAL, ECUDA. */
erq_status erq_rotate(const float* X, int64_t n, int32_t D, const float* P, float* out, int32_t accurate,
                      void* stream);

/* Algorithm 1 (Section 3.1) on each row of Rrot (device [n][D], rotated
 * residuals o', any scale).  Writes codes[n][D] (ybar_u: one byte per
 * coordinate for B <= 8, a little-endian 16-bit word per coordinate for
 * B = 9 and 10, i.e. 2 n D bytes), f_add[n] = fl32(||o'||^2), f_res[n] = fl32(-2 ||o'||^2 / ip*) with
 * ip* = <ybar, |o'|> at the optimum (0 for o' = 0), and optionally stats[n][2] =
 * (ip*, ||ybar||^2) in FP64.  Critical values are visited in ascending exact
 * rational order, ties by coordinate; <y_cur,o'> accumulates in FP64 in that
 * order; the first state of maximal <y/||y||, o'> wins.  B = 10 (the widest
 * code of Table 4) is accepted here, for the encoder alone; an index stores
 * at most B = 9 bits per coordinate (erq_build_index).
 * Errors: EINVAL (B outside 1..10, D), EUNSUPPORTED (a row whose non-zero
 * magnitudes span more than 2^118), ECUDA. */
erq_status erq_encode(const float* Rrot, int64_t n, int32_t D, int32_t B, uint8_t* codes, float* f_add,
                      float* f_res, double* stats, void* stream);

/* Batched IVF search (Section 4.1) for Q (device [nq][D]):
 *   q' = P^T q_r (once per query), probe the nprobe nearest centroids (ties by
 *   lower id), estimate every candidate of the probed clusters with Eq. 3.3 +
 *   Eq. (eq:dis to ip), keep the k' = max(k, rerank_k) smallest estimates (ties by
 *   lower id), and -- when rerank_k > 0 -- re-rank them by exact squared distance.
 * ids[nq][k] (int64, -1 where fewer than k candidates exist) and dists[nq][k]
 * (FP32: exact squared distances after re-rank, estimates otherwise).
 * metric = ERQ_METRIC_IP (the inner-product adaptation Section 7 refers to
 * RaBitQ for): probe the nprobe centroids with the largest <q_r, c> (ties by
 * lower id); estimate <o_r, q_r> = <c, q_r> + ||o_r - c|| <o, q_r> with the
 * same unbiased estimator of <o, q_r> and the same codes and factors, i.e.
 * <c, q_r> - (f_res / 2) <ybar, q'>; keep the k' largest estimates (ties by
 * lower id) and re-rank them by the exact inner product.  ids are then in
 * decreasing order of inner product and dists (and cand_est) hold the inner
 * products themselves (-INFINITY where fewer than k exist).
 * Errors: EINVAL (k, nprobe, probe ids, rerank without raw rows), EUNSUPPORTED
 * (precision), ENOMEM (workspace), ECUDA, ETIMEOUT (device status). */
erq_status erq_search(erq_index* index, const float* Q, int64_t nq, const erq_search_params* params,
                      int64_t* ids, float* dists, void* stream);

/* Two-stage (MSB-first) search of Section 4.2, for few queries per probed
 * cluster, on CUDA cores in FP32 (params->precision is ignored; metric l2).
 * The probe is erq_search's.  Stage 1 reads only the most significant bit
 * plane of every probed row -- the 1-bit RaBitQ code of its residual -- and
 * forms Lemma 2.1's estimate est1 and error bound eps0 * err1 * ||q_r - c||
 * (err1 = 2 ||o'|| sqrt(1 - a^2) / (a sqrt(D - 1)), a = sum|o'_i| / (sqrt(D) ||o'||)).
 * Per query, tau = the k'-th smallest est1 + bound over its probed rows (+inf
 * with fewer rows); rows with est1 - bound > tau are dropped.  Stage 2 reads
 * the other B - 1 bits of the survivors and completes their estimate by
 * Eq. 4.2; the k' = max(k, rerank_k) smallest (estimate, id) survivors are
 * re-ranked as in erq_search (cand_ids / cand_est as there).  eps0 = INFINITY
 * keeps every row (erq_search's result up to FP32 rounding); eps0 = 0 keeps
 * the k' smallest est1.
 * stats: optional HOST int64_t[2] out = {probed rows, survivors} summed over
 * the queries (reading them synchronises the stream).  The first call on an
 * index computes the stage-1 factors (16 bytes per row, kept) from the raw
 * rows.  The call synchronises the stream (the row count sizes its buffers).
 * Errors: EINVAL (as erq_search; eps0 < 0 or NaN; no raw rows),
 * EUNSUPPORTED (metric ip; B = 4, whose top bit sits inside the packed nibble
 * words), ENOMEM, ECUDA. */
erq_status erq_search_two_stage(erq_index* index, const float* Q, int64_t nq, const erq_search_params* params,
                                float eps0, int64_t* ids, float* dists, int64_t* stats, void* stream);

/* The same search from HOST buffers: Q_host[nq][D] is copied to the device,
 * searched, and ids_host/dists_host are copied back before the call returns.
 * Pinned (page-locked) host memory gives asynchronous copies. */
erq_status erq_search_host(erq_index* index, const float* Q_host, int64_t nq, const erq_search_params* params,
                           int64_t* ids_host, float* dists_host, void* stream);

/* Estimated squared distance (Eq. 3.3 + Eq. eq:dis to ip, FP32 path) of query i
 * to each original id in ids[i][0..nc-1]; ids < 0 give NaN.  Q device [nq][D],
 * ids device [nq][nc], est device [nq][nc].  Errors: EINVAL, ECUDA. */
erq_status erq_estimate(erq_index* index, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                        float* est, void* stream);

/* Gradient of sum_j grad_scores[i][j] * est(q_i, ids[i][j]) with respect to the
 * raw query q_i, codes and ids fixed.  From Eq. (eq:dis to ip) and Eq. 3.3:
 *   d est / d q_r = 2 (q_r - c) + f_res * P ybar,  ybar = ybar_u - (2^B-1)/2,
 * evaluated as grad_Q = 2 (G q_r - sum_j g_j c_j) + (sum_j g_j f_res,j ybar_j) P^T
 * (a gather over the codes, then one GEMM with P).  grad_Q device [nq][D] is
 * overwritten.  ids < 0 contribute nothing.  Errors: EINVAL, ENOMEM, ECUDA. */
erq_status erq_search_backward(erq_index* index, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                               const float* grad_scores, float* grad_Q, void* stream);

/* erq_estimate and erq_search_backward for a given erq_metric.  With
 * ERQ_METRIC_IP, est is the estimated inner product
 *   <c, q_r> - (f_res / 2) <ybar, P^T q_r>   (see erq_search)
 * and its gradient is d est / d q_r = c - (f_res / 2) P ybar, evaluated as
 * grad_Q = sum_j g_j c_j - (sum_j g_j (f_res,j / 2) ybar_j) P^T.  ERQ_METRIC_L2
 * is exactly erq_estimate / erq_search_backward.  Errors: as those, and EINVAL
 * for an unknown metric. */
erq_status erq_estimate_metric(erq_index* index, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                               int32_t metric, float* est, void* stream);
erq_status erq_search_backward_metric(erq_index* index, const float* Q, int64_t nq, int32_t nc,
                                      const int64_t* ids, const float* grad_scores, int32_t metric,
                                      float* grad_Q, void* stream);

/* Copy one field of the index to host memory (dst_host must hold dst_bytes).
 * Errors: EINVAL (field, size), ECUDA. */
erq_status erq_index_export(const erq_index* index, int32_t field, void* dst_host, int64_t dst_bytes);

/* Versioned flat file holding every field; load rebuilds the device index. */
erq_status erq_index_save(const erq_index* index, const char* path);
erq_status erq_index_load(const char* path, void* stream, erq_index** out);

/* Diagnostics.
 * erq_search_timing: device time in milliseconds of the phases of the last
 * erq_search on this index that ran with ERQ_SEARCH_TIMING, measured with CUDA
 * events on the search stream: ms[0] query rotation, ms[1] centroid probe,
 * ms[2] planning (probe inversion, pair scalars, one host read-back),
 * ms[3] code scan (estimator + per-item top-k'), ms[4] merge, ms[5] re-rank.
 * Synchronises those events.  n must be >= 6.  Errors: EINVAL (no timed search).
 * erq_kernel_launches: number of kernels this library has launched in the
 * process so far (all entry points, all threads).
 * erq_search_stats: work of the last erq_search on this index: out[0] estimated
 * (query, candidate) pairs, out[1] rows of the distinct probed clusters (codes
 * that had to be read at least once), out[2] work items, out[3] per-(query,
 * item) candidate lists, and for the tensor-core scan out[4] 128-row blocks
 * streamed through the tensor cores and out[5] the sum over those blocks of the
 * item's query count padded to the MMA width (0 for the FP32 path).  Fills
 * min(n, 6) entries; n must be >= 4.  Synchronises the device. */
erq_status erq_search_timing(const erq_index* index, float* ms, int32_t n);
/* erq_search_timing_total: per-phase device milliseconds summed over the timed
 * searches since the previous call (at most the last 512 of them; *count says
 * how many were summed), same phase order as erq_search_timing.  Synchronises
 * on those searches' events.  Errors: EINVAL for null arguments or n < 6. */
erq_status erq_search_timing_total(erq_index* index, float* ms, int32_t n, int64_t* count);
uint64_t erq_kernel_launches(void);
erq_status erq_search_stats(const erq_index* index, int64_t* out, int32_t n);

/* Work-item shape of the code scan (no counterpart in the paper; a tuning
 * interface of this implementation).  A work item is (cluster, up to
 * queries_per_item of the queries that probe it, up to rows_per_item of its
 * rows); on the tensor-core path queries_per_item is the MMA's N extent.
 * erq_autotune: times erq_search over the caller's query batch and params for
 * every supported shape (queries_per_item 32, 64 or 128 for k' <= 32, 32 for larger k',
 * rows_per_item in {2048, 4096, 8192}), reps searches each after one warm-up,
 * and keeps the fastest for later searches on this index whose nq * nprobe is
 * within 4x of the tuned one (one entry for k' <= 32, one for larger k');
 * best_out (optional, host [2]) receives it.  Synchronises the stream.  Errors
 * as erq_search; EUNSUPPORTED for the FP32 path.
 * erq_set_scan_config: force the shape (0 = automatic) for later searches;
 * EINVAL for values other than 0/32/64/128 and 0 or multiples of 256.
 * erq_scan_config: out[0..1] = the shape used by the last search. */
erq_status erq_autotune(erq_index* index, const float* Q, int64_t nq, const erq_search_params* params, int32_t reps,
                        void* stream, int32_t* best_out);
erq_status erq_set_scan_config(erq_index* index, int32_t queries_per_item, int32_t rows_per_item);
erq_status erq_scan_config(const erq_index* index, int32_t* out, int32_t n);

/* Merge of caller-given candidate lists (no counterpart in the paper; the
 * exchange step of a search whose IVF lists are split over several indices,
 * one per GPU, see Section 4.1 for the single-index search it reproduces).
 * For query i, the k smallest (values[i][j], cand_ids[i][j]) pairs over
 * j < m, ascending by value and then by id (ERQ_METRIC_IP: the k largest
 * values, descending, ties by lower id); ids < 0 are empty.  ids_out[nq][k]
 * gets -1 and vals_out[nq][k] +inf (-inf for ERQ_METRIC_IP) past the
 * available pairs.  All arrays are device memory; the call allocates and
 * frees its workspace in stream order.  Errors: EINVAL (m outside [1, 8192],
 * k outside [1, 1024], null pointer, metric), ECUDA. */
erq_status erq_merge_topk(const int64_t* cand_ids, const float* values, int64_t nq, int32_t m, int32_t k,
                          int32_t metric, int64_t* ids_out, float* vals_out, void* stream);

/* Exact re-rank of caller-given ids (the re-rank step of erq_search, which the
 * paper's search leaves to the caller, Section 4.1): for query i, the exact
 * squared distance (ERQ_METRIC_IP: inner product) to every id in
 * ids[i][0..nc-1] that the index holds (0 <= id < N; other ids are skipped),
 * the k best by (distance, id) ascending (ERQ_METRIC_IP: largest inner
 * product first, ties by lower id) into ids_out[nq][k] / dists_out[nq][k],
 * with -1 / +inf (-inf) past the available ones.  Needs keep_raw.  Q device
 * [nq][D].  Errors: EINVAL (k, nc outside 1 <= k <= nc <= 1024, no raw rows,
 * metric), ECUDA. */
erq_status erq_rerank_ids(erq_index* index, const float* Q, int64_t nq, int32_t nc, const int64_t* ids, int32_t k,
                          int32_t metric, int64_t* ids_out, float* dists_out, void* stream);

/* Limit of every bounded device-side wait of the tensor-core scan on this
 * index, in nanoseconds (0 = the default, 2 s); no counterpart in the paper.
 * A wait that runs out makes the scan stop, drain its copies, free its tensor
 * memory and report ERQ_ETIMEOUT through the index's status word; the index
 * stays usable.  stall_stage >= 0 is a test of that path: in later scans the
 * first MMA issuer of every CTA, at its stage number stall_stage, waits on a
 * barrier that nothing arrives on, so the wait runs out after the limit;
 * -1 turns it off.  Errors: EINVAL (null index, stall_stage < -1). */
erq_status erq_set_wait_limit(erq_index* index, uint64_t ns, int64_t stall_stage);

/* Allocation-free variant of erq_search_backward (no counterpart in the paper;
 * an interface for callers that cannot allocate device memory while they run,
 * e.g. a host that owns all device memory through its own pool).  Same arguments, result and errors as erq_search_backward.  Its
 * intermediates (2 * nq * D floats and nq ints) live in one static device array
 * of ERQ_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * keeps until the process exits; requests with 8*nq*D + 4*nq + 512 bytes above
 * that size are rejected with ERQ_EINVAL (at D = 1024: nq <= 2046).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and keeps it for the life of the process; the kept address is no longer
 * valid once the device's
 * primary context is destroyed (cudaDeviceReset), after which this entry point
 * must not be called again in that process.  All calls share the array and the previous call's
 * contents are never read, but calls that can overlap on the GPU (different
 * streams or threads) race on it and must be serialised by the caller.  No
 * memory is allocated or freed by this call. */
#define ERQ_NOALLOC_SCRATCH_BYTES (16u << 20)
erq_status erq_search_backward_noalloc(erq_index* index, const float* Q, int64_t nq, int32_t nc,
                                       const int64_t* ids, const float* grad_scores, float* grad_Q, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ERQ_H */
