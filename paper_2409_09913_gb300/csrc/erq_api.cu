// C ABI of liberq.so: argument validation, index lifecycle, and the order of
// kernel launches for build / encode / search / estimate / backward.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "erq_kernels.cuh"
#include "erq_search.cuh"

namespace erq {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_err = msg; }
erq_status fail(erq_status st, const std::string& msg) {
    g_err = msg;
    return st;
}
erq_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ERQ_ENOMEM : ERQ_ECUDA;
}

// k-means helpers (k_linalg.cu)
cudaError_t launch_row_argmin(const float* V, int64_t rows, int ncols, int32_t* out, cudaStream_t s);
cudaError_t launch_gather_rows(const float* X, const int64_t* idx, int64_t n, int D, float* out, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s);
cudaError_t launch_strided_ids(int64_t* out, int64_t n, int64_t N, uint64_t seed, cudaStream_t s);
// k_scan_tc.cu
erq_status scan_tc(const ScanLaunch& L, int precision, cudaStream_t s);
bool tc_available(int precision, int D, int kp);
cudaError_t launch_to_half(const float* x, __half* y, int64_t n, cudaStream_t s);

namespace {

template <typename T>
erq_status dalloc(T** p, size_t count, int64_t* tally = nullptr) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if (tally) *tally += (int64_t)(count * sizeof(T));
    return ERQ_OK;
}

void free_index_arrays(erq_index* ix) {
    void* ptrs[] = {ix->PT,    ix->eP,    ix->ePT,     ix->eC,   ix->corder,
                    ix->P,     ix->C,     ix->Cp,      ix->cnorm2, ix->list_off, ix->list_ids,
                    ix->row_of, ix->cl_of_row, ix->codes, ix->f_add, ix->f_res,  ix->g_const,
                    ix->X,     ix->status, ix->ws,      ix->ws_b,   ix->io,    ix->rowmeta, ix->poff, ix->codes_p,
                    ix->dstats, ix->PT_hi, ix->C_hi, ix->dctr, ix->rowmeta1, ix->ws_ts};   // PT_lo / C_lo live inside those blocks
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (ix->pinned) cudaFreeHost(ix->pinned);
    if (ix->ev_ring) {
        for (int i = 0; i < erq_index::kTimingRing * 7; ++i)
            if (ix->ev_ring[i]) cudaEventDestroy(ix->ev_ring[i]);
        delete[] ix->ev_ring;
    }
    delete ix->host_list_off;
}

// Bump allocator over a device workspace.
struct Carver {
    char* base;
    size_t off = 0, cap;
    Carver(void* b, size_t c) : base((char*)b), cap(c) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) / 256 * 256;
        T* p = (T*)(base ? base + off : nullptr);
        off += std::max<size_t>(count, 1) * sizeof(T);
        return p;
    }
};

erq_status ensure_ws(void** ws, size_t* have, size_t need) {
    if (*have >= need) return ERQ_OK;
    if (*ws) cudaFree(*ws);
    *ws = nullptr;
    *have = 0;
    const size_t bytes = need + need / 8 + (1 << 20);
    cudaError_t e = cudaMalloc(ws, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "workspace cudaMalloc");
    *have = bytes;
    return ERQ_OK;
}

erq_status check_status(erq_index* ix, cudaStream_t s) {
    uint32_t st = 0;
    ERQ_CHECK_CUDA(cudaMemcpyAsync(&st, ix->status, 4, cudaMemcpyDeviceToHost, s));
    ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
    if (st) {
        ERQ_CHECK_CUDA(cudaMemsetAsync(ix->status, 0, 4, s));
        ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
        if (st & kStatusTimeout) return fail(ERQ_ETIMEOUT, "a device-side wait ran out of iterations");
        if (st & kStatusRange)
            return fail(ERQ_EUNSUPPORTED, "a rotated residual has a non-zero coordinate below 2^-118 of its largest");
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "a device-side bound check failed (cluster id, probe id, nprobe or row id out of range; "
                 "checked-build sites 0x%06x)", st >> 8);
        return fail(ERQ_EINVAL, msg);
    }
    return ERQ_OK;
}

bool valid_d(int32_t D) { return D >= 64 && D <= 4096 && D % 64 == 0; }

// P^T and the row exponents used by the tensor-core GEMM (from P and C).
erq_status derive_gemm_arrays(erq_index* ix, cudaStream_t s) {
    const int D = ix->D;
    if (!ix->PT && cudaMalloc(&ix->PT, sizeof(float) * D * D) != cudaSuccess) return fail(ERQ_ENOMEM, "cudaMalloc P^T");
    if (!ix->eP && cudaMalloc(&ix->eP, sizeof(int32_t) * D) != cudaSuccess) return fail(ERQ_ENOMEM, "cudaMalloc");
    if (!ix->ePT && cudaMalloc(&ix->ePT, sizeof(int32_t) * D) != cudaSuccess) return fail(ERQ_ENOMEM, "cudaMalloc");
    if (!ix->eC && cudaMalloc(&ix->eC, sizeof(int32_t) * ix->nlist) != cudaSuccess) return fail(ERQ_ENOMEM, "cudaMalloc");
    ix->device_bytes += (int64_t)D * D * 4 + 8 * D + 4 * ix->nlist;
    cudaError_t e;
    if ((e = launch_transpose(ix->P, D, D, ix->PT, s)) != cudaSuccess) return cuda_fail(e, "transpose P");
    if ((e = launch_row_exp(ix->P, D, D, ix->eP, s)) != cudaSuccess) return cuda_fail(e, "row exp");
    if ((e = launch_row_exp(ix->PT, D, D, ix->ePT, s)) != cudaSuccess) return cuda_fail(e, "row exp");
    if ((e = launch_row_exp(ix->C, ix->nlist, D, ix->eC, s)) != cudaSuccess) return cuda_fail(e, "row exp");
    // FP16 hi / lo splits of P^T and the centroids for the query-time GEMMs
    {
        const size_t pd = (size_t)D * D, cd = (size_t)ix->nlist * D;
        if (!ix->PT_hi && cudaMalloc(&ix->PT_hi, 2 * pd * sizeof(__half)) != cudaSuccess)
            return fail(ERQ_ENOMEM, "cudaMalloc P^T split");
        if (!ix->C_hi && cudaMalloc(&ix->C_hi, 2 * cd * sizeof(__half)) != cudaSuccess)
            return fail(ERQ_ENOMEM, "cudaMalloc centroid split");
        ix->PT_lo = ix->PT_hi + pd;
        ix->C_lo = ix->C_hi + cd;
        ix->device_bytes += (int64_t)(4 * (pd + cd));
        if ((e = launch_split_hilo(ix->PT, ix->ePT, D, D, ix->PT_hi, ix->PT_lo, s)) != cudaSuccess)
            return cuda_fail(e, "split P^T");
        if ((e = launch_split_hilo(ix->C, ix->eC, ix->nlist, D, ix->C_hi, ix->C_lo, s)) != cudaSuccess)
            return cuda_fail(e, "split centroids");
    }
    // tiled, padded copy of the codes and per-row factors for the tensor-core scan
    {
        const std::vector<int64_t>& lo = *ix->host_list_off;
        std::vector<int64_t> po(ix->nlist + 1, 0);
        for (int c = 0; c < ix->nlist; ++c) po[c + 1] = po[c] + (lo[c + 1] - lo[c] + 31) / 32 * 32;
        ix->Np = po[ix->nlist];
        if (!ix->poff && cudaMalloc(&ix->poff, sizeof(int64_t) * (ix->nlist + 1)) != cudaSuccess)
            return fail(ERQ_ENOMEM, "cudaMalloc padded offsets");
        ERQ_CHECK_CUDA(cudaMemcpyAsync(ix->poff, po.data(), sizeof(int64_t) * (ix->nlist + 1), cudaMemcpyHostToDevice, s));
        const size_t np = (size_t)std::max<int64_t>(ix->Np, 32);
        const size_t np32 = (np + 31) / 32 * 32;
        const size_t pbytes = np32 * (size_t)D * ix->B / 8;      // B bits per coordinate
        if (!ix->codes_p && cudaMalloc(&ix->codes_p, pbytes) != cudaSuccess)
            return fail(ERQ_ENOMEM, "cudaMalloc packed codes");
        if (!ix->rowmeta && cudaMalloc(&ix->rowmeta, sizeof(float4) * np) != cudaSuccess)
            return fail(ERQ_ENOMEM, "cudaMalloc row factors");
        ix->device_bytes += (int64_t)(pbytes + 16 * np + 8 * (ix->nlist + 1));
        if ((e = launch_scan_layout(ix->codes, ix->g_const, ix->f_res, ix->list_ids, ix->list_off, ix->poff, ix->nlist,
                                    ix->Np, D, ix->B, ix->codes_p, ix->rowmeta, s)) != cudaSuccess)
            return cuda_fail(e, "scan layout");
        ERQ_CHECK_CUDA(cudaStreamSynchronize(s));   // po (host) goes out of scope
    }
    // clusters by decreasing size: work items of the largest clusters are scheduled first
    std::vector<int32_t> order(ix->nlist);
    for (int j = 0; j < ix->nlist; ++j) order[j] = j;
    const std::vector<int64_t>& off = *ix->host_list_off;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return off[x + 1] - off[x] > off[y + 1] - off[y]; });
    if (!ix->corder && cudaMalloc(&ix->corder, sizeof(int32_t) * ix->nlist) != cudaSuccess)
        return fail(ERQ_ENOMEM, "cudaMalloc");
    ERQ_CHECK_CUDA(cudaMemcpyAsync(ix->corder, order.data(), sizeof(int32_t) * ix->nlist, cudaMemcpyHostToDevice, s));
    ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
    return ERQ_OK;
}

}  // namespace
}  // namespace erq

using namespace erq;

extern "C" const char* erq_version(void) { return "erq 0.1 (sm_103a)"; }
extern "C" const char* erq_last_error(void) { return g_err.c_str(); }

extern "C" void erq_free_index(erq_index* index) {
    if (!index) return;
    free_index_arrays(index);
    delete index;
}

extern "C" erq_status erq_index_info_get(const erq_index* ix, erq_index_info* info) {
    if (!ix || !info) return fail(ERQ_EINVAL, "null argument");
    info->N = ix->N;
    info->D = ix->D;
    info->B = ix->B;
    info->nlist = ix->nlist;
    info->keep_raw = ix->keep_raw;
    info->max_list = ix->max_list;
    info->device_bytes = ix->device_bytes;
    return ERQ_OK;
}

extern "C" erq_status erq_index_status(erq_index* ix, void* stream) {
    if (!ix) return fail(ERQ_EINVAL, "null index");
    return check_status(ix, (cudaStream_t)stream);
}

extern "C" erq_status erq_rotate(const float* X, int64_t n, int32_t D, const float* P, float* out, int32_t accurate,
                      void* stream) {
    if (n < 0 || !valid_d(D)) return fail(ERQ_EINVAL, "erq_rotate: D must be a multiple of 64 in [64, 4096], n >= 0");
    if (n == 0) return ERQ_OK;
    if (!X || !P || !out) return fail(ERQ_EINVAL, "erq_rotate: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = accurate ? launch_rotate_fp64(X, nullptr, nullptr, nullptr, P, out, n, D, s)
                             : launch_sgemm(false, X, P, out, n, D, D, 1.f, nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "erq_rotate launch");
    return ERQ_OK;
}

extern "C" erq_status erq_encode(const float* Rrot, int64_t n, int32_t D, int32_t B, uint8_t* codes, float* f_add, float* f_res,
                      double* stats, void* stream) {
    if (n < 0 || !valid_d(D)) return fail(ERQ_EINVAL, "erq_encode: D must be a multiple of 64 in [64, 4096], n >= 0");
    if (B < 1 || B > 10) return fail(ERQ_EINVAL, "erq_encode: B must be in [1, 10]");
    if (n == 0) return ERQ_OK;
    if (!Rrot || !codes || !f_add || !f_res) return fail(ERQ_EINVAL, "erq_encode: null pointer");
    uint32_t* status = nullptr;
    ERQ_CHECK_CUDA(cudaMalloc(&status, 4));
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(status, 0, 4, s);
    cudaError_t e = launch_encode(Rrot, n, D, B, codes, f_add, f_res, stats, status, s);
    if (e != cudaSuccess) {
        cudaFree(status);
        return cuda_fail(e, "erq_encode launch");
    }
    uint32_t st = 0;
    cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(e, "erq_encode");
    if (st & kStatusRange)
        return fail(ERQ_EUNSUPPORTED, "erq_encode: a row has a non-zero coordinate below 2^-118 of its largest");
    if (st) return fail(ERQ_EINVAL, "erq_encode: window bound violated (non-finite input?)");
    return ERQ_OK;
}

// ---------------------------------------------------------------------------
// Build
// ---------------------------------------------------------------------------
static erq_status build_kmeans(const float* X, int64_t N, int D, int nlist, const erq_build_params* p, int32_t* assign,
                               erq_index* ix, cudaStream_t s) {
    const int iters = p->kmeans_iters > 0 ? p->kmeans_iters : 10;
    int64_t S = p->kmeans_sample > 0 ? std::min<int64_t>(p->kmeans_sample, N) : N;
    if (S < nlist) S = std::min<int64_t>(N, nlist);
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)(512ll << 20) / (4ll * nlist)));
    // workspace: sample rows, their norms, ids, assignment, distance chunk, grouping
    size_t need = 0;
    {
        Carver cv(nullptr, 0);
        cv.take<float>((size_t)S * D);
        cv.take<float>(S);
        cv.take<int64_t>(S);
        cv.take<int32_t>(S);
        cv.take<float>((size_t)chunk * nlist);
        cv.take<int64_t>(nlist + 1);
        cv.take<int64_t>(S);
        cv.take<char>(group_scratch_bytes(S, nlist));
        cv.take<float>(N);
        need = cv.off;
    }
    ERQ_TRY(ensure_ws(&ix->ws, &ix->ws_bytes, need));
    Carver cv(ix->ws, ix->ws_bytes);
    float* Xs = cv.take<float>((size_t)S * D);
    float* xn = cv.take<float>(S);
    int64_t* sid = cv.take<int64_t>(S);
    int32_t* sa = cv.take<int32_t>(S);
    float* dist = cv.take<float>((size_t)chunk * nlist);
    int64_t* soff = cv.take<int64_t>(nlist + 1);
    int64_t* sids = cv.take<int64_t>(S);
    const size_t gbytes = group_scratch_bytes(S, nlist);
    void* gscr = cv.take<char>(gbytes);
    float* xall = cv.take<float>(N);
    cudaError_t e;
    if ((e = launch_strided_ids(sid, S, N, p->seed, s)) != cudaSuccess) return cuda_fail(e, "kmeans ids");
    if ((e = launch_gather_rows(X, sid, S, D, Xs, s)) != cudaSuccess) return cuda_fail(e, "kmeans gather");
    if ((e = launch_row_sqnorm(Xs, S, D, xn, s)) != cudaSuccess) return cuda_fail(e, "kmeans norms");
    // initial centroids: nlist evenly spaced sample rows
    std::vector<int64_t> init(nlist);
    for (int j = 0; j < nlist; ++j) init[j] = (int64_t)((double)j * (double)S / nlist);
    int64_t* init_d = sids;  // temporarily
    ERQ_CHECK_CUDA(cudaMemcpyAsync(init_d, init.data(), sizeof(int64_t) * nlist, cudaMemcpyHostToDevice, s));
    if ((e = launch_gather_rows(Xs, init_d, nlist, D, ix->C, s)) != cudaSuccess) return cuda_fail(e, "kmeans init");
    ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int it = 0; it < iters; ++it) {
        if ((e = launch_row_sqnorm(ix->C, nlist, D, ix->cnorm2, s)) != cudaSuccess) return cuda_fail(e, "kmeans cn");
        for (int64_t r0 = 0; r0 < S; r0 += chunk) {
            const int64_t m = std::min(chunk, S - r0);
            if ((e = launch_sqdist(Xs + r0 * D, xn + r0, ix->C, ix->cnorm2, dist, m, nlist, D, s)) != cudaSuccess)
                return cuda_fail(e, "kmeans dist");
            if ((e = launch_row_argmin(dist, m, nlist, sa + r0, s)) != cudaSuccess) return cuda_fail(e, "kmeans argmin");
        }
        if ((e = launch_group(sa, S, nlist, soff, sids, nullptr, nullptr, gscr, gbytes, ix->status, s)) != cudaSuccess)
            return cuda_fail(e, "kmeans group");
        if ((e = launch_centroids(Xs, soff, sids, nlist, D, ix->C, 1, s)) != cudaSuccess)
            return cuda_fail(e, "kmeans centroids");
    }
    // final assignment of every row
    if ((e = launch_row_sqnorm(ix->C, nlist, D, ix->cnorm2, s)) != cudaSuccess) return cuda_fail(e, "kmeans cn");
    if ((e = launch_row_sqnorm(X, N, D, xall, s)) != cudaSuccess) return cuda_fail(e, "kmeans xn");
    for (int64_t r0 = 0; r0 < N; r0 += chunk) {
        const int64_t m = std::min(chunk, N - r0);
        if ((e = launch_sqdist(X + r0 * D, xall + r0, ix->C, ix->cnorm2, dist, m, nlist, D, s)) != cudaSuccess)
            return cuda_fail(e, "kmeans dist");
        if ((e = launch_row_argmin(dist, m, nlist, assign + r0, s)) != cudaSuccess) return cuda_fail(e, "kmeans argmin");
    }
    ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
    return ERQ_OK;
}

extern "C" erq_status erq_build_index(const float* X, int64_t N, int32_t D, const erq_build_params* p, void* stream,
                                      erq_index** out) {
    if (!out) return fail(ERQ_EINVAL, "erq_build_index: out is null");
    *out = nullptr;
    if (!p || !X || !p->P) return fail(ERQ_EINVAL, "erq_build_index: X, params and params->P are required");
    if (N < 1 || N >= (1ll << 31)) return fail(ERQ_EINVAL, "erq_build_index: N must be in [1, 2^31)");
    if (!valid_d(D)) return fail(ERQ_EINVAL, "erq_build_index: D must be a multiple of 64 in [64, 4096]");
    if (p->B < 1 || p->B > 9) return fail(ERQ_EINVAL, "erq_build_index: B must be in [1, 9]");
    if (p->centroids && (!p->assign || p->nlist < 2))
        return fail(ERQ_EINVAL, "erq_build_index: explicit centroids need an explicit assignment and nlist >= 2");
    if (p->nlist < 1 || p->nlist > 65536 || (p->nlist > N && !p->centroids))
        return fail(ERQ_EINVAL, "erq_build_index: nlist must be in [1, min(N, 65536)]");
    cudaStream_t s = (cudaStream_t)stream;
    erq_index* ix = new erq_index();
    ix->N = N;
    ix->D = D;
    ix->B = p->B;
    ix->nlist = p->nlist;
    ix->keep_raw = p->keep_raw ? 1 : 0;
    ix->normalized = p->normalize ? 1 : 0;
    ix->host_list_off = new std::vector<int64_t>();
    float* Xn = nullptr;                 // rows scaled to unit length (normalize = 1)
    auto bail = [&](erq_status st) {
        cudaStreamSynchronize(s);
        if (Xn && Xn != ix->X) cudaFree(Xn);
        erq_free_index(ix);
        return st;
    };
    const int nlist = p->nlist;
    erq_status st;
#define ALLOC(ptr, cnt)                                         \
    if ((st = dalloc(&ix->ptr, (cnt), &ix->device_bytes)) != ERQ_OK) return bail(st);
    ALLOC(P, (size_t)D * D);
    ALLOC(C, (size_t)nlist * D);
    ALLOC(Cp, (size_t)nlist * D);
    ALLOC(cnorm2, nlist);
    ALLOC(list_off, nlist + 1);
    ALLOC(list_ids, N);
    ALLOC(row_of, N);
    ALLOC(cl_of_row, N);
    ALLOC(codes, (size_t)N * D * code_bytes(p->B));
    ALLOC(f_add, N);
    ALLOC(f_res, N);
    ALLOC(g_const, N);
    ALLOC(status, 1);
    if (ix->keep_raw) ALLOC(X, (size_t)N * D);
#undef ALLOC
    cudaError_t e;
    if ((e = cudaMemsetAsync(ix->status, 0, 4, s)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
    if (ix->normalized) {                // every later step sees the unit rows
        if (ix->keep_raw) {
            Xn = ix->X;
        } else if (cudaMalloc(&Xn, sizeof(float) * (size_t)N * D) != cudaSuccess) {
            Xn = nullptr;
            return bail(fail(ERQ_ENOMEM, "erq_build_index: unit-row copy"));
        }
        if ((e = launch_normalize_rows(X, N, D, Xn, s)) != cudaSuccess) return bail(cuda_fail(e, "normalize rows"));
        X = Xn;
    }
    if ((e = cudaMemcpyAsync(ix->P, p->P, sizeof(float) * D * D, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return bail(cuda_fail(e, "copy P"));
    if (ix->keep_raw && X != ix->X &&
        (e = cudaMemcpyAsync(ix->X, X, sizeof(float) * (size_t)N * D, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return bail(cuda_fail(e, "copy X"));
    // --- assignment
    int32_t* assign = nullptr;
    if ((st = dalloc(&assign, N)) != ERQ_OK) return bail(st);
    auto bail2 = [&](erq_status st2) {
        cudaStreamSynchronize(s);
        cudaFree(assign);
        return bail(st2);
    };
    if (nlist == 1) {
        if ((e = launch_fill_i32(assign, N, 0, s)) != cudaSuccess) return bail2(cuda_fail(e, "fill"));
    } else if (p->assign) {
        if ((e = cudaMemcpyAsync(assign, p->assign, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return bail2(cuda_fail(e, "copy assign"));
    } else {
        if ((st = build_kmeans(X, N, D, nlist, p, assign, ix, s)) != ERQ_OK) return bail2(st);
    }
    // --- group rows by cluster, centroids, rotated centroids
    {
        const size_t gbytes = group_scratch_bytes(N, nlist);
        if ((st = ensure_ws(&ix->ws, &ix->ws_bytes, gbytes)) != ERQ_OK) return bail2(st);
        if ((e = launch_group(assign, N, nlist, ix->list_off, ix->list_ids, ix->row_of, ix->cl_of_row, ix->ws,
                              ix->ws_bytes, ix->status, s)) != cudaSuccess)
            return bail2(cuda_fail(e, "group"));
        if ((st = check_status(ix, s)) != ERQ_OK)
            return bail2(fail(ERQ_EINVAL, "erq_build_index: assign holds a cluster id outside [0, nlist)"));
    }
    if (p->centroids) {
        if ((e = cudaMemcpyAsync(ix->C, p->centroids, sizeof(float) * (size_t)nlist * D, cudaMemcpyDeviceToDevice,
                                 s)) != cudaSuccess)
            return bail2(cuda_fail(e, "copy centroids"));
    } else if ((e = launch_centroids(X, ix->list_off, ix->list_ids, nlist, D, ix->C, 0, s)) != cudaSuccess) {
        return bail2(cuda_fail(e, "centroids"));
    }
    if ((e = launch_rotate_fp64(ix->C, nullptr, nullptr, nullptr, ix->P, ix->Cp, nlist, D, s)) != cudaSuccess)
        return bail2(cuda_fail(e, "rotate centroids"));
    if ((e = launch_row_sqnorm(ix->C, nlist, D, ix->cnorm2, s)) != cudaSuccess) return bail2(cuda_fail(e, "cnorm"));
    // --- rotate residuals and encode, in chunks of rows
    {
        const int64_t chunk = std::min<int64_t>(N, std::max<int64_t>(4096, (int64_t)(1ll << 30) / (4ll * D)));
        if ((st = ensure_ws(&ix->ws, &ix->ws_bytes, (size_t)chunk * D * 4)) != ERQ_OK) return bail2(st);
        float* R = (float*)ix->ws;
        for (int64_t r0 = 0; r0 < N; r0 += chunk) {
            const int64_t m = std::min(chunk, N - r0);
            if ((e = launch_rotate_fp64(X, ix->list_ids + r0, ix->C, ix->cl_of_row + r0, ix->P, R, m, D, s)) !=
                cudaSuccess)
                return bail2(cuda_fail(e, "rotate residuals"));
            if ((e = launch_encode(R, m, D, ix->B, ix->codes + r0 * D * code_bytes(ix->B), ix->f_add + r0, ix->f_res + r0, nullptr,
                                   ix->status, s)) != cudaSuccess)
                return bail2(cuda_fail(e, "encode"));
        }
    }
    if ((e = launch_gconst(ix->codes, ix->f_add, ix->f_res, ix->Cp, ix->cl_of_row, N, D, ix->B, ix->g_const, s)) !=
        cudaSuccess)
        return bail2(cuda_fail(e, "gconst"));
    ix->host_list_off->resize(nlist + 1);
    if ((e = cudaMemcpyAsync(ix->host_list_off->data(), ix->list_off, sizeof(int64_t) * (nlist + 1),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return bail2(cuda_fail(e, "list_off"));
    if ((st = check_status(ix, s)) != ERQ_OK) return bail2(st);
    if ((st = derive_gemm_arrays(ix, s)) != ERQ_OK) return bail2(st);
    cudaFree(assign);
    if (Xn && Xn != ix->X) cudaFree(Xn);   // (derive_gemm_arrays synchronised the stream)
    int64_t mx = 0;
    for (int j = 0; j < nlist; ++j) mx = std::max(mx, (*ix->host_list_off)[j + 1] - (*ix->host_list_off)[j]);
    ix->max_list = mx;
    *out = ix;
    return ERQ_OK;
}

// ---------------------------------------------------------------------------
// Search
// ---------------------------------------------------------------------------
// Work-item shape of the scan: queries per item (the tensor-core MMA's N
// extent) and rows per item.  Heuristic for k' <= 32: 128 queries per item when
// a probed cluster has more than 96 probing queries on average, else 64; for
// larger k' 32; 4,096 rows; the autotuned or forced shape wins.
static void choose_scan_shape(const erq_index* ix, int prec, int kp, int64_t nq, int maxp, int* qn, int* rr) {
    if (prec == ERQ_PREC_FP32) {
        *qn = 64;
        *rr = ix->force_rr > 0 ? ix->force_rr : 4096;
        return;
    }
    const int cls = kp <= 32 ? 0 : 1;
    const int64_t work = nq * (int64_t)maxp;
    int q = cls == 0 ? ((double)work / ix->nlist > 96.0 ? 128 : 64) : 32, r = 4096;
    const erq_index::ScanTune& t = ix->tune[cls];
    if (t.valid && work <= 4 * t.work && 4 * work >= t.work) {
        q = t.qn;
        r = t.rr;
    }
    if (ix->force_qn > 0 && scan_tc_shape_ok(ix->force_qn, kp)) q = ix->force_qn;
    if (ix->force_rr > 0) r = ix->force_rr;
    *qn = q;
    *rr = r;
}

// Stage 1, pruning, stage 2 and the selection of the two-stage search
// (k_two_stage.cu), after the probe, then the exact re-rank.
static erq_status two_stage_tail(erq_index* ix, const float* Q, int64_t nq, const erq_search_params* p, int64_t* ids,
                                 float* dists, cudaStream_t s, float eps0, int64_t* stats_out, const int32_t* probe_c,
                                 const float* dqc, const float* Qrot, int maxp, int kp, int k, bool do_rerank,
                                 uint64_t* cand, const DevChecks& ck) {
    const int D = ix->D;
    cudaError_t e;
    // slots for every probed row: bounded on the host (nq x the rows of the maxp
    // largest lists) so that nothing is read back, unless the probe lists are
    // explicit (their distinctness is not checked) or the bound would take more
    // than 2 GB of scratch, when the exact count is read back instead
    int64_t rows = 0;
    {
        const std::vector<int64_t>& off = *ix->host_list_off;
        std::vector<int64_t> sz((size_t)ix->nlist);
        for (int c = 0; c < ix->nlist; ++c) sz[c] = off[c + 1] - off[c];
        const int top = std::min(maxp, ix->nlist);
        std::partial_sort(sz.begin(), sz.begin() + top, sz.end(), std::greater<int64_t>());
        int64_t per_q = 0;
        for (int i = 0; i < top; ++i) per_q += sz[i];
        rows = nq * per_q;
    }
    const bool exact = p->probe != nullptr || rows * 20 > (1ll << 31);
    // one index-owned scratch block (kept between calls):
    //   rbase [nq][maxp] i32 | qrows [nq] i64 | qoffr [nq+1] i64 | ub, lb, s1 [rows] f32 |
    //   skey [rows] u64 | T [nq][4D] f32 | tau [nq] f32 | scnt [nq] i32
    // (every part starts on a 256-byte boundary: the tables are read as float4)
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t off_qrows = up(4 * (size_t)nq * maxp), off_qoffr = up(off_qrows + 8 * (size_t)nq);
    const size_t off_rows = up(off_qoffr + 8 * (size_t)(nq + 1));
    ERQ_TRY(ensure_ws(&ix->ws_ts, &ix->ws_ts_bytes, off_rows));
    int32_t* rbase = (int32_t*)ix->ws_ts;
    int64_t* qrows = (int64_t*)((char*)ix->ws_ts + off_qrows);
    int64_t* qoffr = (int64_t*)((char*)ix->ws_ts + off_qoffr);
    if ((e = launch_two_stage_rows(probe_c, nq, maxp, ix->list_off, rbase, qrows, s)) != cudaSuccess ||
        (e = launch_excl_scan_i64(qrows, qoffr, nq, s)) != cudaSuccess)
        return cuda_fail(e, "two-stage: row offsets");
    if (exact) {
        if ((e = cudaMemcpyAsync(&rows, qoffr + nq, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "two-stage: row count");
    }
    const size_t r = (size_t)std::max<int64_t>(rows, 1);
    const size_t off_skey = up(off_rows + 12 * r), off_T = up(off_skey + 8 * r);
    const size_t off_tau = up(off_T + (size_t)nq * 16 * D), off_cnt = up(off_tau + 4 * (size_t)nq);
    const size_t need = off_cnt + 4 * (size_t)nq;
    if (ix->ws_ts_bytes < need) {        // growing replaces the block: keep the offsets computed so far
        ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
        std::vector<char> head(off_rows);
        ERQ_CHECK_CUDA(cudaMemcpy(head.data(), ix->ws_ts, off_rows, cudaMemcpyDeviceToHost));
        ERQ_TRY(ensure_ws(&ix->ws_ts, &ix->ws_ts_bytes, need));
        ERQ_CHECK_CUDA(cudaMemcpy(ix->ws_ts, head.data(), off_rows, cudaMemcpyHostToDevice));
        rbase = (int32_t*)ix->ws_ts;
        qoffr = (int64_t*)((char*)ix->ws_ts + off_qoffr);
    }
    char* b = (char*)ix->ws_ts;          // the offsets are from the block's start
    TwoStageLaunch L;
    L.probe_c = probe_c; L.dqc = dqc; L.list_off = ix->list_off; L.poff = ix->poff; L.codes_p = ix->codes_p;
    L.rowmeta = ix->rowmeta; L.meta1 = ix->rowmeta1; L.Qrot = Qrot; L.T = (float*)(b + off_T);
    L.rbase = rbase; L.qoffr = qoffr;
    L.ub = (float*)(b + off_rows); L.lb = L.ub + r; L.s1 = L.ub + 2 * r;   // 4-byte elements
    L.skey = (uint64_t*)(b + off_skey); L.scratch = (uint32_t*)(b + off_skey);
    L.tau = (float*)(b + off_tau); L.scnt = (int32_t*)(b + off_cnt); L.cand = cand;
    L.nq = nq; L.maxp = maxp; L.D = D; L.B = ix->B; L.kp = kp; L.eps0 = eps0;
    if ((e = launch_two_stage(L, s)) != cudaSuccess) return cuda_fail(e, "two-stage");
    if ((e = launch_rerank(cand, nq, kp, ix->X, Q, D, k, do_rerank ? 1 : 0, 0, ids, dists, p->cand_ids, p->cand_est,
                           ck, s)) != cudaSuccess)
        return cuda_fail(e, "two-stage: rerank");
    if (stats_out) {
        std::vector<int32_t> cnt((size_t)nq);
        int64_t total = 0;
        if ((e = cudaMemcpyAsync(cnt.data(), L.scnt, sizeof(int32_t) * (size_t)nq, cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(&total, qoffr + nq, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "two-stage: survivors");
        int64_t sv = 0;
        for (int32_t v : cnt) sv += v;
        stats_out[0] = total;
        stats_out[1] = sv;
    }
    return ERQ_OK;
}

// Two-stage search request (erq_search_two_stage): Lemma 2.1's eps0 and an
// optional host output {probed rows, survivors} summed over the queries.
struct TwoStageReq {
    float eps0;
    int64_t* stats;
};

// Stage-1 factors of every stored row (rowmeta1), from the rotated residuals
// of the raw rows (the same FP64 rotation as the build).
static erq_status ensure_stage1(erq_index* ix, cudaStream_t s) {
    if (ix->rowmeta1) return ERQ_OK;
    const int D = ix->D;
    const size_t np = (size_t)std::max<int64_t>(ix->Np, 32);
    if (cudaMalloc(&ix->rowmeta1, sizeof(float4) * np) != cudaSuccess) {
        ix->rowmeta1 = nullptr;
        return fail(ERQ_ENOMEM, "cudaMalloc two-stage factors");
    }
    ix->device_bytes += (int64_t)(16 * np);
    ERQ_CHECK_CUDA(cudaMemsetAsync(ix->rowmeta1, 0, sizeof(float4) * np, s));
    const int64_t N = ix->N;
    const int64_t chunk = std::min<int64_t>(N, std::max<int64_t>(4096, (int64_t)(1ll << 30) / (4ll * D)));
    ERQ_TRY(ensure_ws(&ix->ws, &ix->ws_bytes, (size_t)std::max<int64_t>(chunk, 1) * D * 4));
    float* R = (float*)ix->ws;
    cudaError_t e;
    for (int64_t r0 = 0; r0 < N; r0 += chunk) {
        const int64_t m = std::min(chunk, N - r0);
        if ((e = launch_rotate_fp64(ix->X, ix->list_ids + r0, ix->C, ix->cl_of_row + r0, ix->P, R, m, D, s)) !=
            cudaSuccess)
            return cuda_fail(e, "two-stage factors: rotate residuals");
        if ((e = launch_stage1_factors(R, r0, m, D, ix->B, ix->codes, ix->f_add, ix->Cp, ix->cl_of_row, ix->list_off,
                                       ix->poff, ix->rowmeta1, s)) != cudaSuccess)
            return cuda_fail(e, "two-stage factors");
    }
    ERQ_CHECK_CUDA(cudaStreamSynchronize(s));   // the workspace is carved by the search next
    return ERQ_OK;
}

static erq_status search_impl(erq_index* ix, const float* Q, int64_t nq, const erq_search_params* p, int64_t* ids,
                              float* dists, cudaStream_t s, const TwoStageReq* ts = nullptr) {
    const int D = ix->D, nlist = ix->nlist;
    const int k = p->k;
    const int kp = std::max(p->k, p->rerank_k);
    const bool do_rerank = p->rerank_k > 0;
    int maxp = p->probe ? p->nprobe : (nlist == 1 ? 1 : p->nprobe);
    const bool explicit_probe = p->probe != nullptr;
    const int prec = p->precision;
    const int ip = p->metric == ERQ_METRIC_IP ? 1 : 0;   // rank by -<o_r, q_r> (probe: -<q_r, c_j>)
    // e4m3 query rows: padded to whole 128-byte stages (B <= 4), or every
    // 64-coordinate block twice for the split form of wider codes
    const int split8 = ix->B > 4;
    const int64_t Dq = split8 ? 2 * (int64_t)D : (D + 127) / 128 * 128;
    // ---- phase A workspace (sizes known on the host)
    // queries per work item of the scan kernels
    int QT = 64, RR = 4096;
    choose_scan_shape(ix, prec, kp, nq, maxp, &QT, &RR);
    ix->last_qn = QT;
    ix->last_rr = RR;
    Carver plan(nullptr, 0);
    auto layout = [&](Carver& cv, bool carve, void** slots) {
        int i = 0;
        auto T = [&](auto* dummy, size_t n) {
            using TT = std::remove_pointer_t<decltype(dummy)>;
            void* ptr = cv.take<TT>(n);
            if (carve) slots[i] = ptr;
            ++i;
        };
        T((float*)nullptr, (size_t)nq * D);                              // 0 Qrot
        T((float*)nullptr, nq);                                          // 1 qn
        T((float*)nullptr, (!explicit_probe && nlist > 1) ? (size_t)nq * nlist : 1);  // 2 sqd
        T((int32_t*)nullptr, (size_t)nq * maxp);                         // 3 probe (computed)
        T((int32_t*)nullptr, nq);                                        // 4 npr
        T((float*)nullptr, (size_t)nq * maxp);                           // 5 dqc
        T((int32_t*)nullptr, (size_t)nq * maxp);                         // 6 probe_c
        T((int32_t*)nullptr, (size_t)nq * maxp);                         // 7 slot_nr
        T((int32_t*)nullptr, (size_t)nq * maxp);                         // 8 slot_off
        T((int64_t*)nullptr, nq);                                        // 9 qtot
        T((int64_t*)nullptr, nq + 1);                                    // 10 qbase
        T((int32_t*)nullptr, 2 * (size_t)nlist);                         // 11 cnt_c (per phase cluster)
        T((int32_t*)nullptr, 2 * (size_t)nlist);                         // 12 pos_c
        T((int64_t*)nullptr, 2 * (size_t)nlist);                         // 13 cnt64
        T((int64_t*)nullptr, 2 * (size_t)nlist);                         // 14 items_c
        T((int64_t*)nullptr, 2 * (size_t)nlist + 1);                     // 15 qoff
        T((int64_t*)nullptr, 2 * (size_t)nlist + 1);                     // 16 item_off
        T((int64_t*)nullptr, (size_t)nq * maxp);                         // 17 qlist
        T((uint64_t*)nullptr, (size_t)nq * kp);                          // 18 cand
        T((uint64_t*)nullptr, 1);                                        // 19 (unused)
        T((__half*)nullptr, prec == ERQ_PREC_FP16 ? (size_t)nq * D : 1); // 20 Qh
        T((int32_t*)nullptr, nq);                                        // 21 eQ
        T((uint64_t*)nullptr, prec == ERQ_PREC_FP32 ? 1 : nq);           // 22 query-wide thresholds
        T((__half*)nullptr, (size_t)nq * D);                              // 23 Q hi
        T((__half*)nullptr, (size_t)nq * D);                              // 24 Q lo
        T((float*)nullptr, (!explicit_probe && nlist > 1) ? (size_t)nq * ((nlist + 31) / 32) : 1);  // 25 group minima
        T((unsigned char*)nullptr, prec == ERQ_PREC_FP8 ? (size_t)nq * Dq : 1);   // 26 e4m3 queries
        T((float*)nullptr, prec == ERQ_PREC_FP8 ? (size_t)nq : 1);                // 27 their scales
        T((int32_t*)nullptr, nlist);                                     // 28 touch_c
    };
    void* sl[29];
    layout(plan, false, sl);
    ERQ_TRY(ensure_ws(&ix->ws, &ix->ws_bytes, plan.off));
    Carver cv(ix->ws, ix->ws_bytes);
    layout(cv, true, sl);
    float* Qrot = (float*)sl[0];
    float* qn = (float*)sl[1];
    float* sqd = (float*)sl[2];
    int32_t* probe = (int32_t*)sl[3];
    int32_t* npr = (int32_t*)sl[4];
    float* dqc = (float*)sl[5];
    PlanArgs pa;
    pa.probe_c = (int32_t*)sl[6];
    pa.slot_nr = (int32_t*)sl[7];
    pa.slot_off = (int32_t*)sl[8];
    pa.qtot = (int64_t*)sl[9];
    pa.qbase = (int64_t*)sl[10];
    pa.cnt_c = (int32_t*)sl[11];
    pa.pos_c = (int32_t*)sl[12];
    pa.cnt64 = (int64_t*)sl[13];
    pa.items_c = (int64_t*)sl[14];
    pa.qoff = (int64_t*)sl[15];
    pa.item_off = (int64_t*)sl[16];
    pa.qlist = (int64_t*)sl[17];
    pa.touch_c = (int32_t*)sl[28];
    uint64_t* cand = (uint64_t*)sl[18];
    if (!ix->dstats && cudaMalloc(&ix->dstats, 4 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(ERQ_ENOMEM, "cudaMalloc search counters");
    if (!ix->dctr && cudaMalloc(&ix->dctr, 256) != cudaSuccess) return fail(ERQ_ENOMEM, "cudaMalloc scan counter");
    pa.stats = ix->dstats;
    cudaError_t e;
    const bool timed = (p->flags & ERQ_SEARCH_TIMING) != 0;
    ix->timed = 0;
    if (timed && !ix->ev_ring) ix->ev_ring = new cudaEvent_t[erq_index::kTimingRing * 7]();
    cudaEvent_t* ev = timed ? ix->ev_ring + (ix->timing_seq % erq_index::kTimingRing) * 7 : nullptr;
    if (timed)
        for (int i = 0; i < 7; ++i)
            if (!ev[i]) ERQ_CHECK_CUDA(cudaEventCreate(&ev[i]));
    auto mark = [&](int i) -> erq_status {
        if (timed) ERQ_CHECK_CUDA(cudaEventRecord(ev[i], s));
        return ERQ_OK;
    };
    ERQ_TRY(mark(0));
    // ---- q' = P^T q_r
    const bool simt = (p->flags & ERQ_SEARCH_SIMT_GEMM) != 0;
    int32_t* eQ = (int32_t*)sl[21];
    const bool need_qn = !explicit_probe && nlist > 1 && !ip;   // ||q_r||^2 for the distance probe
    bool qn_done = false, qh_done = false;
    if (simt) {
        if ((e = launch_sgemm(false, Q, ix->P, Qrot, nq, D, D, 1.f, nullptr, s)) != cudaSuccess)
            return cuda_fail(e, "query rotation");
    } else {
        // row exponents, ||q_r||^2 and the hi/lo split in one pass; the rotation
        // GEMM also writes the FP16 copy of q' that the tensor-core scan reads
        if ((e = launch_query_prep(Q, nq, D, eQ, need_qn ? qn : nullptr, (__half*)sl[23], (__half*)sl[24], s)) !=
            cudaSuccess)
            return cuda_fail(e, "query split");
        qn_done = need_qn;
        __half* qh = prec == ERQ_PREC_FP16 ? (__half*)sl[20] : nullptr;
        if ((e = launch_gemm_tma((__half*)sl[23], (__half*)sl[24], eQ, nq, ix->PT_hi, ix->PT_lo, ix->ePT, D, D, Qrot,
                                 D, 0, nullptr, nullptr, nullptr, ix->status, s, qh)) != cudaSuccess)
            return cuda_fail(e, "query rotation");
        qh_done = qh != nullptr;
    }
    if (prec == ERQ_PREC_FP8 &&
        (e = launch_quant_e4m3(Qrot, nq, D, (int)Dq, split8, (unsigned char*)sl[26], (float*)sl[27], s)) != cudaSuccess)
        return cuda_fail(e, "query e4m3");
    if (prec == ERQ_PREC_FP16 && !qh_done &&
        (e = launch_to_half(Qrot, (__half*)sl[20], (int64_t)nq * D, s)) != cudaSuccess)
        return cuda_fail(e, "query half");
    ERQ_TRY(mark(1));
    // ---- probe
    const int32_t* probe_use = probe;
    int64_t probe_stride = maxp;
    if (explicit_probe) {
        probe_use = p->probe;
        probe_stride = p->probe_stride;
    } else if (nlist == 1) {
        if ((e = launch_fill_i32(probe, nq, 0, s)) != cudaSuccess) return cuda_fail(e, "probe fill");
    } else {
        if (need_qn && !qn_done && (e = launch_row_sqnorm(Q, nq, D, qn, s)) != cudaSuccess)
            return cuda_fail(e, "query norms");
        if (simt)
            e = ip ? launch_sgemm(true, Q, ix->C, sqd, nq, nlist, D, -1.f, nullptr, s)
                   : launch_sqdist(Q, qn, ix->C, ix->cnorm2, sqd, nq, nlist, D, s);
        else
            e = launch_gemm_tma((__half*)sl[23], (__half*)sl[24], eQ, nq, ix->C_hi, ix->C_lo, ix->eC, nlist, D, sqd,
                                nlist, ip ? 2 : 1, ip ? nullptr : qn, ip ? nullptr : ix->cnorm2,
                                maxp <= 32 ? (float*)sl[25] : nullptr, ix->status, s);
        if (e != cudaSuccess) return cuda_fail(e, "centroid distances");
        e = (!simt && maxp <= 32) ? launch_row_topk_groups(sqd, (float*)sl[25], nq, nlist, nlist, maxp, probe, maxp, s)
                                  : launch_row_topk_fast(sqd, nq, nlist, nlist, maxp, probe, nullptr, maxp, s);
        if (e != cudaSuccess) return cuda_fail(e, "probe select");
    }
    ERQ_TRY(mark(2));
    // ---- plan
    pa.probe = probe_use;
    pa.probe_stride = probe_stride;
    pa.npr_in = p->nprobe_per_query;
    pa.npr_uniform = maxp;
    pa.nq = nq;
    pa.maxp = maxp;
    pa.nlist = nlist;
    pa.QT = QT;
    pa.RR = RR;
    pa.list_off = ix->list_off;
    pa.corder = ix->corder;
    pa.npr = npr;
    pa.status = ix->status;
    // ||q_r - c||^2 (or -<q_r, c>) of the probed pairs: the probe's own values
    // when it computed them (the FP32 expansion ||q_r||^2 + ||c||^2 - 2<q_r, c>
    // with an FP32-accurate product), else computed directly below
    const bool dqc_from_probe = !explicit_probe && nlist > 1;
    pa.sqd = dqc_from_probe ? sqd : nullptr;
    pa.dqc = dqc;
    DevChecks ck;
    ck.status = ix->status;
    ck.qlist = nq * (int64_t)maxp;
    ck.rows = ix->N;
    ck.nlist = nlist;
    ck.items = 0;                 // set once phase B is sized; the plan kernels below use qlist only
    ck.lists = 0;
    pa.ck = ck;
    if ((e = launch_plan(pa, s)) != cudaSuccess) return cuda_fail(e, "plan");
    // dqc needs the validated probe ids
    if (!dqc_from_probe && (e = launch_dqc(Q, ix->C, pa.probe_c, npr, nq, maxp, D, ip, dqc, s)) != cudaSuccess)
        return cuda_fail(e, "dqc");
    if (ts) return two_stage_tail(ix, Q, nq, p, ids, dists, s, ts->eps0, ts->stats, pa.probe_c, dqc, Qrot, maxp, kp,
                                  k, do_rerank, cand, ck);
    int64_t Ltot = 0, nitems = 0;
    // host-side bounds assume distinct probed lists per query, which the
    // centroid search guarantees; explicit probe lists are sized exactly
    const bool async = (p->flags & ERQ_SEARCH_ASYNC) != 0 && !explicit_probe;
    if (async) {
        // upper bounds from the cluster sizes (no read-back):
        //   items <= maxR * ceil(nq * maxp / QT) + sum_c nr_c,  lists <= nq * (sum of the maxp largest nr_c)
        const std::vector<int64_t>& off = *ix->host_list_off;
        std::vector<int64_t> nr(nlist);
        int64_t maxR = 0, sumR = 0;
        for (int c = 0; c < nlist; ++c) {
            nr[c] = (off[c + 1] - off[c] + RR - 1) / RR;
            maxR = std::max(maxR, nr[c]);
            sumR += nr[c];
        }
        std::partial_sort(nr.begin(), nr.begin() + std::min(maxp, nlist), nr.end(), std::greater<int64_t>());
        int64_t topR = 0;
        for (int i = 0; i < std::min(maxp, nlist); ++i) topR += nr[i];
        nitems = maxR * ceil_div(nq * (int64_t)maxp, QT) + 2 * sumR;   // two phases per cluster
        Ltot = nq * topR;
    } else {
        int64_t tot[2] = {0, 0};
        ERQ_CHECK_CUDA(cudaMemcpyAsync(&tot[0], pa.qbase + nq, 8, cudaMemcpyDeviceToHost, s));
        ERQ_CHECK_CUDA(cudaMemcpyAsync(&tot[1], pa.item_off + 2 * nlist, 8, cudaMemcpyDeviceToHost, s));
        ERQ_TRY(check_status(ix, s));
        Ltot = tot[0];
        nitems = tot[1];
        ix->last_stats[2] = nitems;
        ix->last_stats[3] = Ltot;
    }
    // ---- phase B workspace
    Carver pb(nullptr, 0);
    pb.take<int4>(nitems);
    const int lstride = scan_list_stride(prec, kp, QT);
    pb.take<uint64_t>((size_t)Ltot * lstride);
    pb.take<int32_t>(Ltot);
    pb.take<int64_t>(1);
    const bool tcp = prec != ERQ_PREC_FP32;
    pb.take<int4>(tcp ? nitems : 0);
    pb.take<int4>(tcp ? nitems * QT : 0);
    if (async && ix->ws_b_bytes < pb.off)
        ERQ_CHECK_CUDA(cudaStreamSynchronize(s));   // growing the buffer frees the old one
    ERQ_TRY(ensure_ws(&ix->ws_b, &ix->ws_b_bytes, pb.off));
    Carver cb(ix->ws_b, ix->ws_b_bytes);
    int4* items = cb.take<int4>(nitems);
    uint64_t* inter = cb.take<uint64_t>((size_t)Ltot * lstride);
    int32_t* inter_cnt = cb.take<int32_t>(Ltot);
    int64_t* n_items_d = cb.take<int64_t>(1);
    int4* itemd = cb.take<int4>(tcp ? nitems : 0);
    int4* itemq = cb.take<int4>(tcp ? nitems * QT : 0);
    ERQ_CHECK_CUDA(cudaMemcpyAsync(n_items_d, pa.item_off + 2 * nlist, 8, cudaMemcpyDeviceToDevice, s));
    ck.items = nitems;
    ck.lists = Ltot;
    pa.ck = ck;
    if (Ltot > 0) ERQ_CHECK_CUDA(cudaMemsetAsync(inter_cnt, 0, sizeof(int32_t) * Ltot, s));

    if ((e = launch_plan_items(pa, items, s)) != cudaSuccess) return cuda_fail(e, "plan items");
    if (tcp && (e = launch_item_tables(items, n_items_d, nitems, ix->list_off, ix->poff, pa.qoff, pa.qlist, dqc,
                                       pa.qbase, pa.slot_off, maxp, RR, QT, nlist, itemd, itemq, pa.stats, ck, s)) !=
                   cudaSuccess)
        return cuda_fail(e, "item tables");
    ERQ_TRY(mark(3));
    // ---- scan
    ScanLaunch L;
    L.Qrot = Qrot; L.Qh = sl[20]; L.Q8 = sl[26]; L.qscale = (const float*)sl[27]; L.Dq = Dq; L.status = ix->status; L.N = ix->N; L.codes = ix->codes; L.g_const = ix->g_const; L.f_res = ix->f_res; L.list_off = ix->list_off;
    L.list_ids = ix->list_ids; L.qlist = pa.qlist; L.qoff = pa.qoff; L.items = items; L.n_items = n_items_d;
    L.dqc = dqc; L.slot_off = pa.slot_off; L.qbase = pa.qbase; L.inter = inter; L.inter_cnt = inter_cnt;
    L.maxp = maxp; L.D = D; L.B = ix->B; L.kp = kp; L.RR = RR; L.qn = QT; L.nlist = nlist;
    L.itemd = itemd; L.itemq = itemq; L.rowmeta = ix->rowmeta; L.codes_p = ix->codes_p; L.Np = ix->Np;
    L.tq = (unsigned long long*)sl[22];
    L.ip = ip;
    L.ck = ck;
    L.nq = nq;
    L.work_ctr = ix->dctr;
    L.wait_ns = ix->wait_ns;
    L.stall_stage = ix->stall_stage;
    if (tcp) ERQ_CHECK_CUDA(cudaMemsetAsync(L.tq, 0xff, sizeof(uint64_t) * nq, s));
    ERQ_CHECK_CUDA(cudaMemsetAsync(ix->dctr, 0, sizeof(unsigned int), s));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    L.grid = (int)std::min<int64_t>(nitems, (int64_t)sms * (prec == ERQ_PREC_FP32 ? scan_fp32_blocks_per_sm(kp, ix->B) : 1));
    if (prec == ERQ_PREC_FP32) {
        if ((e = launch_scan_fp32(L, s)) != cudaSuccess) return cuda_fail(e, "scan fp32");
    } else {
        ERQ_TRY(scan_tc(L, prec, s));
    }
    ERQ_TRY(mark(4));
    // ---- merge, re-rank
    if ((e = launch_merge(inter, inter_cnt, pa.qbase, nq, kp, lstride, cand, ck, s)) != cudaSuccess)
        return cuda_fail(e, "merge");
    ERQ_TRY(mark(5));
    if ((e = launch_rerank(cand, nq, kp, ix->X, Q, D, k, do_rerank ? 1 : 0, ip, ids, dists, p->cand_ids, p->cand_est,
                           ck, s)) != cudaSuccess)
        return cuda_fail(e, "rerank");
    ERQ_TRY(mark(6));
    if (timed) {
        ix->timed = 1;
        ++ix->timing_seq;
    }
    return ERQ_OK;
}

static erq_status validate_search(const erq_index* ix, const float* Q, int64_t nq, const erq_search_params* p,
                                  const void* ids, const void* dists, bool two_stage = false) {
    if (!ix || !p) return fail(ERQ_EINVAL, "erq_search: null index or params");
    if (nq < 0) return fail(ERQ_EINVAL, "erq_search: nq < 0");
    if (nq > 0 && (!Q || !ids || !dists)) return fail(ERQ_EINVAL, "erq_search: null Q/ids/dists");
    if (p->k < 1) return fail(ERQ_EINVAL, "erq_search: k must be >= 1");
    if (p->rerank_k != 0 && p->rerank_k < p->k) return fail(ERQ_EINVAL, "erq_search: rerank_k must be 0 or >= k");
    const int kp = std::max(p->k, p->rerank_k);
    if (kp > 1024) return fail(ERQ_EUNSUPPORTED, "erq_search: max(k, rerank_k) > 1024");
    if (p->rerank_k > 0 && !ix->keep_raw) return fail(ERQ_EINVAL, "erq_search: re-ranking needs keep_raw");
    if (p->probe) {
        if (p->nprobe < 1 || p->probe_stride < p->nprobe)
            return fail(ERQ_EINVAL, "erq_search: explicit probe needs nprobe >= 1 and probe_stride >= nprobe");
        if (p->nprobe > ix->nlist) return fail(ERQ_EINVAL, "erq_search: nprobe > nlist");
    } else if (ix->nlist > 1 && (p->nprobe < 1 || p->nprobe > ix->nlist)) {
        return fail(ERQ_EINVAL, "erq_search: nprobe must be in [1, nlist]");
    }
    if (two_stage) {
        if (p->metric != ERQ_METRIC_L2) return fail(ERQ_EUNSUPPORTED, "erq_search_two_stage: metric l2 only");
        if (ix->B == 4)
            return fail(ERQ_EUNSUPPORTED, "erq_search_two_stage: B = 4 keeps its top bit inside the nibble words "
                                          "of the packed layout (no separate plane to read first)");
        if (!ix->keep_raw) return fail(ERQ_EINVAL, "erq_search_two_stage: needs keep_raw (stage-1 factors)");
        return ERQ_OK;
    }
    if (p->precision == ERQ_PREC_INT8)
        return fail(ERQ_EUNSUPPORTED, "erq_search: int8 tensor MMA (tcgen05 kind::i8) is not available on sm_103a");
    if (p->precision < 0 || p->precision > ERQ_PREC_INT8) return fail(ERQ_EINVAL, "erq_search: unknown precision");
    if (p->precision == ERQ_PREC_FP8 && ix->B > 8)
        return fail(ERQ_EUNSUPPORTED, "erq_search: fp8 holds the split code parts (16 hc + lc) only for B <= 8");
    if (p->precision != ERQ_PREC_FP32 && !tc_available(p->precision, ix->D, kp))
        return fail(ERQ_EUNSUPPORTED, "erq_search: tensor-core path unavailable for this D / k'");
    if (scan_fp32_smem(kp) > 220 * 1024 && p->precision == ERQ_PREC_FP32)
        return fail(ERQ_EUNSUPPORTED, "erq_search: k' too large for the FP32 scan");
    if (p->metric != ERQ_METRIC_L2 && p->metric != ERQ_METRIC_IP && p->metric != ERQ_METRIC_COS)
        return fail(ERQ_EINVAL, "erq_search: unknown metric");
    if (p->metric == ERQ_METRIC_COS && !ix->normalized)
        return fail(ERQ_EINVAL, "erq_search: the cosine metric needs an index built with normalize = 1");
    return ERQ_OK;
}

extern "C" erq_status erq_search(erq_index* ix, const float* Q, int64_t nq, const erq_search_params* p, int64_t* ids,
                                 float* dists, void* stream) {
    ERQ_TRY(validate_search(ix, Q, nq, p, ids, dists));
    if (nq == 0) return ERQ_OK;
    if (p->metric != ERQ_METRIC_COS) return search_impl(ix, Q, nq, p, ids, dists, (cudaStream_t)stream);
    // cosine: the inner-product search of the unit query over the unit rows
    cudaStream_t s = (cudaStream_t)stream;
    float* Qn = nullptr;
    ERQ_CHECK_CUDA(cudaMallocAsync((void**)&Qn, sizeof(float) * (size_t)nq * ix->D, s));
    erq_search_params q = *p;
    q.metric = ERQ_METRIC_IP;
    cudaError_t e = launch_normalize_rows(Q, nq, ix->D, Qn, s);
    const erq_status st = e == cudaSuccess ? search_impl(ix, Qn, nq, &q, ids, dists, s) : cuda_fail(e, "normalize query");
    const cudaError_t ef = cudaFreeAsync(Qn, s);
    if (st != ERQ_OK) return st;
    if (ef != cudaSuccess) return cuda_fail(ef, "erq_search: cudaFreeAsync");
    return ERQ_OK;
}

extern "C" erq_status erq_search_two_stage(erq_index* ix, const float* Q, int64_t nq, const erq_search_params* p,
                                           float eps0, int64_t* ids, float* dists, int64_t* stats, void* stream) {
    ERQ_TRY(validate_search(ix, Q, nq, p, ids, dists, true));
    if (!(eps0 >= 0.f)) return fail(ERQ_EINVAL, "erq_search_two_stage: eps0 must be >= 0");
    if (stats) stats[0] = stats[1] = 0;
    if (nq == 0) return ERQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ERQ_TRY(ensure_stage1(ix, s));
    erq_search_params q = *p;
    q.precision = ERQ_PREC_FP32;          // the probe's FP32 path; no tensor-core query copies
    q.flags &= ~(ERQ_SEARCH_ASYNC | ERQ_SEARCH_TIMING);
    TwoStageReq ts{eps0, stats};
    return search_impl(ix, Q, nq, &q, ids, dists, s, &ts);
}

extern "C" erq_status erq_search_host(erq_index* ix, const float* Q_host, int64_t nq, const erq_search_params* p,
                                      int64_t* ids_host, float* dists_host, void* stream) {
    ERQ_TRY(validate_search(ix, Q_host, nq, p, ids_host, dists_host));
    if (nq == 0) return ERQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t qb = (size_t)nq * ix->D * 4, ib = (size_t)nq * p->k * 8, db = (size_t)nq * p->k * 4;
    ERQ_TRY(ensure_ws(&ix->io, &ix->io_bytes, qb + ib + db + 1024));
    char* base = (char*)ix->io;
    float* Qd = (float*)base;
    int64_t* idd = (int64_t*)(base + (qb + 255) / 256 * 256);
    float* dd = (float*)((char*)idd + (ib + 255) / 256 * 256);
    ERQ_CHECK_CUDA(cudaMemcpyAsync(Qd, Q_host, qb, cudaMemcpyHostToDevice, s));
    erq_search_params q = *p;
    if (p->metric == ERQ_METRIC_COS) {   // the unit query, in place in the staging buffer
        q.metric = ERQ_METRIC_IP;
        cudaError_t e = launch_normalize_rows(Qd, nq, ix->D, Qd, s);
        if (e != cudaSuccess) return cuda_fail(e, "normalize query");
    }
    ERQ_TRY(search_impl(ix, Qd, nq, &q, idd, dd, s));
    ERQ_CHECK_CUDA(cudaMemcpyAsync(ids_host, idd, ib, cudaMemcpyDeviceToHost, s));
    ERQ_CHECK_CUDA(cudaMemcpyAsync(dists_host, dd, db, cudaMemcpyDeviceToHost, s));
    ERQ_CHECK_CUDA(cudaStreamSynchronize(s));
    return ERQ_OK;
}

extern "C" erq_status erq_estimate_metric(erq_index* ix, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                                          int32_t metric, float* est, void* stream) {
    if (!ix || nq < 0 || nc < 0) return fail(ERQ_EINVAL, "erq_estimate: bad arguments");
    if (metric != ERQ_METRIC_L2 && metric != ERQ_METRIC_IP) return fail(ERQ_EINVAL, "erq_estimate: unknown metric");
    if (nq == 0 || nc == 0) return ERQ_OK;
    if (!Q || !ids || !est) return fail(ERQ_EINVAL, "erq_estimate: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    ERQ_TRY(ensure_ws(&ix->ws, &ix->ws_bytes, (size_t)nq * ix->D * 4));
    float* Qrot = (float*)ix->ws;
    cudaError_t e;
    if ((e = launch_sgemm(false, Q, ix->P, Qrot, nq, ix->D, ix->D, 1.f, nullptr, s)) != cudaSuccess)
        return cuda_fail(e, "estimate rotation");
    if ((e = launch_estimate(Q, Qrot, ids, nq, nc, ix, metric == ERQ_METRIC_IP ? 1 : 0, est, s)) != cudaSuccess)
        return cuda_fail(e, "estimate");
    return ERQ_OK;
}

extern "C" erq_status erq_estimate(erq_index* ix, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                                   float* est, void* stream) {
    return erq_estimate_metric(ix, Q, nq, nc, ids, ERQ_METRIC_L2, est, stream);
}

extern "C" erq_status erq_search_backward_metric(erq_index* ix, const float* Q, int64_t nq, int32_t nc,
                                                 const int64_t* ids, const float* grad_scores, int32_t metric,
                                                 float* grad_Q, void* stream) {
    if (!ix || nq < 0 || nc < 0) return fail(ERQ_EINVAL, "erq_search_backward: bad arguments");
    if (metric != ERQ_METRIC_L2 && metric != ERQ_METRIC_IP)
        return fail(ERQ_EINVAL, "erq_search_backward: unknown metric");
    if (nq == 0) return ERQ_OK;
    if (!Q || !grad_Q || (nc > 0 && (!ids || !grad_scores))) return fail(ERQ_EINVAL, "erq_search_backward: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t mat = (size_t)nq * ix->D;
    ERQ_TRY(ensure_ws(&ix->ws, &ix->ws_bytes, 2 * mat * 4 + (size_t)nq * 4 + 1024));
    float* V = (float*)ix->ws;
    float* Wv = V + (mat + 63) / 64 * 64;
    int32_t* eV = (int32_t*)(Wv + (mat + 63) / 64 * 64);
    cudaError_t e;
    if ((e = launch_backward_gather(Q, ids, grad_scores, nq, nc, ix, metric == ERQ_METRIC_IP ? 1 : 0, V, Wv, s)) !=
        cudaSuccess)
        return cuda_fail(e, "backward gather");
    // grad_Q = V P^T + Wv  (B = P read as [n][k])
    if ((e = launch_row_exp(V, nq, ix->D, eV, s)) != cudaSuccess) return cuda_fail(e, "backward exponents");
    if ((e = launch_gemm_tc(V, eV, nq, ix->P, ix->eP, ix->D, ix->D, grad_Q, ix->D, 0, Wv, nullptr, nullptr, ix->status,
                            s)) != cudaSuccess)
        return cuda_fail(e, "backward gemm");
    return ERQ_OK;
}

extern "C" erq_status erq_search_backward(erq_index* ix, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                                          const float* grad_scores, float* grad_Q, void* stream) {
    return erq_search_backward_metric(ix, Q, nq, nc, ids, grad_scores, ERQ_METRIC_L2, grad_Q, stream);
}

// ---------------------------------------------------------------------------
// Export / save / load
// ---------------------------------------------------------------------------
struct FieldDesc {
    const void* ptr;
    size_t bytes;
};

static FieldDesc field_of(const erq_index* ix, int f) {
    const size_t N = ix->N, D = ix->D, nl = ix->nlist;
    switch (f) {
        case ERQ_FIELD_CENTROIDS: return {ix->C, nl * D * 4};
        case ERQ_FIELD_ROT_CENTROIDS: return {ix->Cp, nl * D * 4};
        case ERQ_FIELD_LIST_OFFSETS: return {ix->list_off, (nl + 1) * 8};
        case ERQ_FIELD_LIST_IDS: return {ix->list_ids, N * 8};
        case ERQ_FIELD_CODES: return {ix->codes, N * D * code_bytes(ix->B)};
        case ERQ_FIELD_F_ADD: return {ix->f_add, N * 4};
        case ERQ_FIELD_F_RES: return {ix->f_res, N * 4};
        case ERQ_FIELD_P: return {ix->P, D * D * 4};
        case ERQ_FIELD_RAW: return {ix->keep_raw ? ix->X : nullptr, ix->keep_raw ? N * D * 4 : 0};
        case ERQ_FIELD_PACKED_CODES: return {ix->codes_p, ix->codes_p ? ix->Np * D * ix->B / 8 : 0};
        default: return {nullptr, 0};
    }
}

extern "C" erq_status erq_index_export(const erq_index* ix, int32_t field, void* dst_host, int64_t dst_bytes) {
    if (!ix || !dst_host) return fail(ERQ_EINVAL, "erq_index_export: null argument");
    const FieldDesc fd = field_of(ix, field);
    if (!fd.ptr) return fail(ERQ_EINVAL, "erq_index_export: unknown or absent field");
    if ((size_t)dst_bytes < fd.bytes) return fail(ERQ_EINVAL, "erq_index_export: destination too small");
    ERQ_CHECK_CUDA(cudaMemcpy(dst_host, fd.ptr, fd.bytes, cudaMemcpyDeviceToHost));
    return ERQ_OK;
}

static const char kMagic[8] = {'E', 'R', 'Q', 'I', 'D', 'X', '0', '2'};

extern "C" erq_status erq_index_save(const erq_index* ix, const char* path) {
    if (!ix || !path) return fail(ERQ_EINVAL, "erq_index_save: null argument");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(ERQ_EIO, std::string("erq_index_save: cannot open ") + path);
    int64_t hdr[7] = {ix->N, ix->D, ix->B, ix->nlist, ix->keep_raw, ix->max_list, ix->normalized};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, 8, 7, f) == 7;
    const void* arrays[] = {ix->P, ix->C, ix->Cp, ix->cnorm2, ix->list_off, ix->list_ids, ix->row_of,
                            ix->cl_of_row, ix->codes, ix->f_add, ix->f_res, ix->g_const, ix->X};
    const size_t N = ix->N, D = ix->D, nl = ix->nlist;
    const size_t sizes[] = {D * D * 4, nl * D * 4, nl * D * 4, nl * 4, (nl + 1) * 8, N * 8, N * 8,
                            N * 4, N * D * code_bytes(ix->B), N * 4, N * 4, N * 4, ix->keep_raw ? N * D * 4 : 0};
    std::vector<char> host;
    for (int i = 0; i < 13 && ok; ++i) {
        if (!sizes[i]) continue;
        host.resize(sizes[i]);
        if (cudaMemcpy(host.data(), arrays[i], sizes[i], cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(f);
            return fail(ERQ_ECUDA, "erq_index_save: device copy failed");
        }
        ok = fwrite(host.data(), 1, sizes[i], f) == sizes[i];
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? ERQ_OK : fail(ERQ_EIO, "erq_index_save: write failed");
}

extern "C" erq_status erq_index_load(const char* path, void* stream, erq_index** out) {
    if (!path || !out) return fail(ERQ_EINVAL, "erq_index_load: null argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(ERQ_EIO, std::string("erq_index_load: cannot open ") + path);
    char magic[8];
    int64_t hdr[7];
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kMagic, 8) != 0 || fread(hdr, 8, 7, f) != 7) {
        fclose(f);
        return fail(ERQ_EIO, "erq_index_load: not an index file (bad magic or header)");
    }
    erq_index* ix = new erq_index();
    ix->N = hdr[0];
    ix->D = (int32_t)hdr[1];
    ix->B = (int32_t)hdr[2];
    ix->nlist = (int32_t)hdr[3];
    ix->keep_raw = (int32_t)hdr[4];
    ix->max_list = hdr[5];
    ix->normalized = (int32_t)hdr[6];
    ix->host_list_off = new std::vector<int64_t>(ix->nlist + 1);
    if (ix->N < 1 || !valid_d(ix->D) || ix->B < 1 || ix->B > 9 || ix->nlist < 1) {
        fclose(f);
        erq_free_index(ix);
        return fail(ERQ_EIO, "erq_index_load: corrupt header");
    }
    const size_t N = ix->N, D = ix->D, nl = ix->nlist;
    erq_status st = ERQ_OK;
    void** dst[] = {(void**)&ix->P, (void**)&ix->C, (void**)&ix->Cp, (void**)&ix->cnorm2, (void**)&ix->list_off,
                    (void**)&ix->list_ids, (void**)&ix->row_of, (void**)&ix->cl_of_row, (void**)&ix->codes,
                    (void**)&ix->f_add, (void**)&ix->f_res, (void**)&ix->g_const, (void**)&ix->X};
    const size_t sizes[] = {D * D * 4, nl * D * 4, nl * D * 4, nl * 4, (nl + 1) * 8, N * 8, N * 8,
                            N * 4, N * D * code_bytes(ix->B), N * 4, N * 4, N * 4, ix->keep_raw ? N * D * 4 : 0};
    std::vector<char> host;
    for (int i = 0; i < 13 && st == ERQ_OK; ++i) {
        if (!sizes[i]) continue;
        if (cudaMalloc(dst[i], sizes[i]) != cudaSuccess) {
            st = fail(ERQ_ENOMEM, "erq_index_load: cudaMalloc");
            break;
        }
        ix->device_bytes += sizes[i];
        host.resize(sizes[i]);
        if (fread(host.data(), 1, sizes[i], f) != sizes[i]) {
            st = fail(ERQ_EIO, "erq_index_load: truncated file");
            break;
        }
        if (cudaMemcpy(*dst[i], host.data(), sizes[i], cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(ERQ_ECUDA, "erq_index_load: upload");
        if (i == 4) memcpy(ix->host_list_off->data(), host.data(), sizes[i]);
    }
    fclose(f);
    if (st == ERQ_OK && cudaMalloc(&ix->status, 4) != cudaSuccess) st = fail(ERQ_ENOMEM, "erq_index_load: status");
    if (st == ERQ_OK && cudaMemset(ix->status, 0, 4) != cudaSuccess) st = fail(ERQ_ECUDA, "erq_index_load: status");
    if (st == ERQ_OK) st = derive_gemm_arrays(ix, (cudaStream_t)stream);
    if (st == ERQ_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        st = fail(ERQ_ECUDA, "erq_index_load: derive");
    if (st != ERQ_OK) {
        erq_free_index(ix);
        return st;
    }
    *out = ix;
    return ERQ_OK;
}


extern "C" erq_status erq_search_timing(const erq_index* ix, float* ms, int32_t n) {
    if (!ix || !ms || n < 6) return fail(ERQ_EINVAL, "erq_search_timing: bad arguments");
    if (!ix->timed) return fail(ERQ_EINVAL, "erq_search_timing: no search ran with ERQ_SEARCH_TIMING");
    const cudaEvent_t* ev = ix->ev_ring + ((ix->timing_seq - 1) % erq_index::kTimingRing) * 7;
    ERQ_CHECK_CUDA(cudaEventSynchronize(ev[6]));
    for (int i = 0; i < 6; ++i) ERQ_CHECK_CUDA(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
    return ERQ_OK;
}

extern "C" erq_status erq_search_timing_total(erq_index* ix, float* ms, int32_t n, int64_t* count) {
    if (!ix || !ms || n < 6 || !count) return fail(ERQ_EINVAL, "erq_search_timing_total: bad arguments");
    for (int i = 0; i < 6; ++i) ms[i] = 0.f;
    const int64_t first = std::max(ix->timing_base, ix->timing_seq - erq_index::kTimingRing);
    for (int64_t t = first; t < ix->timing_seq; ++t) {
        const cudaEvent_t* ev = ix->ev_ring + (t % erq_index::kTimingRing) * 7;
        ERQ_CHECK_CUDA(cudaEventSynchronize(ev[6]));
        for (int i = 0; i < 6; ++i) {
            float x = 0.f;
            ERQ_CHECK_CUDA(cudaEventElapsedTime(&x, ev[i], ev[i + 1]));
            ms[i] += x;
        }
    }
    *count = ix->timing_seq - first;
    ix->timing_base = ix->timing_seq;
    return ERQ_OK;
}

extern "C" erq_status erq_set_scan_config(erq_index* ix, int32_t queries_per_item, int32_t rows_per_item) {
    if (!ix) return fail(ERQ_EINVAL, "erq_set_scan_config: null index");
    if (queries_per_item != 0 && queries_per_item != 32 && queries_per_item != 64 && queries_per_item != 128)
        return fail(ERQ_EINVAL, "erq_set_scan_config: queries_per_item must be 0, 32, 64 or 128");
    if (rows_per_item != 0 && (rows_per_item < 256 || rows_per_item % 256 != 0 || rows_per_item > (1 << 20)))
        return fail(ERQ_EINVAL, "erq_set_scan_config: rows_per_item must be 0 or a multiple of 256 in [256, 2^20]");
    ix->force_qn = queries_per_item;
    ix->force_rr = rows_per_item;
    return ERQ_OK;
}

extern "C" erq_status erq_scan_config(const erq_index* ix, int32_t* out, int32_t n) {
    if (!ix || !out || n < 2) return fail(ERQ_EINVAL, "erq_scan_config: bad arguments");
    out[0] = ix->last_qn;
    out[1] = ix->last_rr;
    return ERQ_OK;
}

extern "C" erq_status erq_autotune(erq_index* ix, const float* Q, int64_t nq, const erq_search_params* p,
                                   int32_t reps, void* stream, int32_t* best_out) {
    ERQ_TRY(validate_search(ix, Q, nq, p, p ? (const void*)p : nullptr, p ? (const void*)p : nullptr));
    if (nq == 0 || reps < 1) return fail(ERQ_EINVAL, "erq_autotune: nq and reps must be positive");
    if (p->precision == ERQ_PREC_FP32) return fail(ERQ_EUNSUPPORTED, "erq_autotune: tunes the tensor-core scan");
    cudaStream_t s = (cudaStream_t)stream;
    const int kp = std::max(p->k, p->rerank_k);
    const int cls = kp <= 32 ? 0 : 1;
    const int maxp = p->probe ? p->nprobe : (ix->nlist == 1 ? 1 : p->nprobe);
    const int qns[3] = {32, 64, 128};
    const int rrs[3] = {2048, 4096, 8192};
    int64_t* ids = nullptr;
    float* dists = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    erq_status st = ERQ_OK;
    if (cudaMalloc(&ids, sizeof(int64_t) * nq * p->k) != cudaSuccess ||
        cudaMalloc(&dists, sizeof(float) * nq * p->k) != cudaSuccess)
        st = fail(ERQ_ENOMEM, "erq_autotune: cudaMalloc");
    if (st == ERQ_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(ERQ_ECUDA, "erq_autotune: cudaEventCreate");
    const int keep_qn = ix->force_qn, keep_rr = ix->force_rr;
    float best = -1.f;
    int bq = 0, br = 0;
    erq_search_params pp = *p;
    pp.flags &= ~ERQ_SEARCH_TIMING;
    pp.cand_ids = nullptr;
    pp.cand_est = nullptr;
    for (int qi = 0; qi < 3 && st == ERQ_OK; ++qi) {
        if (!scan_tc_shape_ok(qns[qi], kp)) continue;
        for (int ri = 0; ri < 3 && st == ERQ_OK; ++ri) {
            ix->force_qn = qns[qi];
            ix->force_rr = rrs[ri];
            if ((st = search_impl(ix, Q, nq, &pp, ids, dists, s)) != ERQ_OK) break;   // warm-up, sizes buffers
            if (cudaEventRecord(e0, s) != cudaSuccess) { st = fail(ERQ_ECUDA, "erq_autotune: event"); break; }
            for (int r = 0; r < reps && st == ERQ_OK; ++r) st = search_impl(ix, Q, nq, &pp, ids, dists, s);
            if (st != ERQ_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = fail(ERQ_ECUDA, "erq_autotune: timing");
                break;
            }
            if (best < 0.f || ms < best) {
                best = ms;
                bq = qns[qi];
                br = rrs[ri];
            }
        }
    }
    ix->force_qn = keep_qn;
    ix->force_rr = keep_rr;
    if (st == ERQ_OK) st = check_status(ix, s);
    if (st == ERQ_OK && best >= 0.f) {
        ix->tune[cls].valid = 1;
        ix->tune[cls].work = nq * (int64_t)maxp;
        ix->tune[cls].qn = bq;
        ix->tune[cls].rr = br;
        if (best_out) {
            best_out[0] = bq;
            best_out[1] = br;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ids) cudaFree(ids);
    if (dists) cudaFree(dists);
    return st;
}

extern "C" uint64_t erq_kernel_launches(void) { return g_launches.load(); }

extern "C" erq_status erq_search_stats(const erq_index* ix, int64_t* out, int32_t n) {
    if (!ix || !out || n < 4) return fail(ERQ_EINVAL, "erq_search_stats: bad arguments");
    unsigned long long d[4] = {0, 0, 0, 0};
    if (ix->dstats) {
        ERQ_CHECK_CUDA(cudaDeviceSynchronize());
        ERQ_CHECK_CUDA(cudaMemcpy(d, ix->dstats, sizeof(d), cudaMemcpyDeviceToHost));
    }
    const int64_t v[6] = {(int64_t)d[0], (int64_t)d[1], ix->last_stats[2], ix->last_stats[3], (int64_t)d[2],
                          (int64_t)d[3]};
    for (int i = 0; i < n && i < 6; ++i) out[i] = v[i];
    return ERQ_OK;
}

// ---------------------------------------------------------------------------
// Merging and re-ranking of caller-given candidate lists (cluster-sharded
// search: each shard's top-k' are merged into the single index's top-k', whose
// exact distances each shard then computes for the rows it holds).
// ---------------------------------------------------------------------------
extern "C" erq_status erq_merge_topk(const int64_t* cand_ids, const float* values, int64_t nq, int32_t m, int32_t k,
                                     int32_t metric, int64_t* ids_out, float* vals_out, void* stream) {
    if (nq < 0 || m < 1 || m > 8192 || k < 1 || k > 1024)
        return fail(ERQ_EINVAL, "erq_merge_topk: need nq >= 0, 1 <= m <= 8192, 1 <= k <= 1024");
    if (metric != ERQ_METRIC_L2 && metric != ERQ_METRIC_IP) return fail(ERQ_EINVAL, "erq_merge_topk: unknown metric");
    if (nq == 0) return ERQ_OK;
    if (!cand_ids || !values || !ids_out || !vals_out) return fail(ERQ_EINVAL, "erq_merge_topk: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int neg = metric == ERQ_METRIC_IP ? 1 : 0;
    Carver plan(nullptr, 0);
    plan.take<uint64_t>((size_t)nq * m);
    plan.take<int32_t>(nq);
    plan.take<int64_t>(nq + 1);
    plan.take<uint64_t>((size_t)nq * k);
    void* ws = nullptr;
    ERQ_CHECK_CUDA(cudaMallocAsync(&ws, plan.off, s));
    Carver cv(ws, plan.off);
    uint64_t* keys = cv.take<uint64_t>((size_t)nq * m);
    int32_t* counts = cv.take<int32_t>(nq);
    int64_t* off = cv.take<int64_t>(nq + 1);
    uint64_t* cand = cv.take<uint64_t>((size_t)nq * k);
    DevChecks ck;
    ck.lists = nq;
    cudaError_t e = launch_make_keys(cand_ids, values, nq * (int64_t)m, 0, neg, keys, s);
    if (e == cudaSuccess) e = launch_one_list_per_query(nq, m, counts, off, s);
    if (e == cudaSuccess) e = launch_merge(keys, counts, off, nq, k, m, cand, ck, s);
    if (e == cudaSuccess) e = launch_keys_to_pairs(cand, nq * (int64_t)k, neg, ids_out, vals_out, s);
    const cudaError_t ef = cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return cuda_fail(e, "erq_merge_topk");
    if (ef != cudaSuccess) return cuda_fail(ef, "erq_merge_topk: cudaFreeAsync");
    return ERQ_OK;
}

extern "C" erq_status erq_rerank_ids(erq_index* ix, const float* Q, int64_t nq, int32_t nc, const int64_t* ids,
                                     int32_t k, int32_t metric, int64_t* ids_out, float* dists_out, void* stream) {
    if (!ix || nq < 0 || nc < 1 || nc > 1024 || k < 1 || k > nc)
        return fail(ERQ_EINVAL, "erq_rerank_ids: need an index, 1 <= k <= nc <= 1024");
    if (metric != ERQ_METRIC_L2 && metric != ERQ_METRIC_IP) return fail(ERQ_EINVAL, "erq_rerank_ids: unknown metric");
    if (!ix->keep_raw) return fail(ERQ_EINVAL, "erq_rerank_ids: the index keeps no raw rows (keep_raw = 0)");
    if (nq == 0) return ERQ_OK;
    if (!Q || !ids || !ids_out || !dists_out) return fail(ERQ_EINVAL, "erq_rerank_ids: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* keys = nullptr;
    ERQ_CHECK_CUDA(cudaMallocAsync((void**)&keys, sizeof(uint64_t) * (size_t)nq * nc, s));
    DevChecks ck;
    ck.status = ix->status;
    ck.rows = ix->N;
    cudaError_t e = launch_make_keys(ids, nullptr, nq * (int64_t)nc, ix->N, 0, keys, s);
    if (e == cudaSuccess)
        e = launch_rerank(keys, nq, nc, ix->X, Q, ix->D, k, 1, metric == ERQ_METRIC_IP ? 1 : 0, ids_out, dists_out,
                          nullptr, nullptr, ck, s);
    const cudaError_t ef = cudaFreeAsync(keys, s);
    if (e != cudaSuccess) return cuda_fail(e, "erq_rerank_ids");
    if (ef != cudaSuccess) return cuda_fail(ef, "erq_rerank_ids: cudaFreeAsync");
    return ERQ_OK;
}

extern "C" erq_status erq_set_wait_limit(erq_index* ix, uint64_t ns, int64_t stall_stage) {
    if (!ix) return fail(ERQ_EINVAL, "erq_set_wait_limit: null index");
    if (stall_stage < -1) return fail(ERQ_EINVAL, "erq_set_wait_limit: stall_stage must be >= -1");
    ix->wait_ns = ns;
    ix->stall_stage = stall_stage;
    return ERQ_OK;
}
