// Dense linear algebra and grouping kernels of the index build and the query
// prologue:
//   * rotation o' = P^T (o_r - c) with FP64 accumulation (index time) -- the
//     Section 3.3 workflow step "apply P^{-1} to the data vectors";
//   * FP32 SGEMM (query rotation q' = P^T q_r, centroid distances for the IVF
//     probe of Section 4.1, the P-multiply of the backward pass);
//   * cluster means (Section 5.1 local centring) and a stable counting sort
//     that groups rows by cluster (IVF lists, Section 4.1);
//   * per-row selection of the p smallest entries (probe lists, k-means).
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "warp_sort.cuh"

namespace erq {

// ---------------------------------------------------------------------------
// Rotation with FP64 accumulation.
//   out[r][j] = fl32( sum_{k=0..D-1, ascending} (double)res_k * (double)P[k][j] )
//   res_k     = fl32(X[src][k] - C[cl][k])  (or X[src][k] when C == nullptr)
// Products of two FP32 values are exact in FP64, so fma(res, p, acc) equals the
// sequential "acc += res * p" of a plain FP64 loop: the result is bit-identical
// to any implementation that sums in ascending k.
// Tile 64 rows x 64 columns, 256 threads, 4x4 outputs per thread, BK = 16.
// ---------------------------------------------------------------------------
constexpr int R64_BM = 64, R64_BN = 64, R64_BK = 16;

__global__ void __launch_bounds__(256) rotate_fp64_kernel(const float* __restrict__ X,
                                                          const int64_t* __restrict__ gather,
                                                          const float* __restrict__ C,
                                                          const int32_t* __restrict__ cl,
                                                          const float* __restrict__ P, float* __restrict__ out,
                                                          int64_t n, int D) {
    __shared__ float As[R64_BK][R64_BM + 4];
    __shared__ float Bs[R64_BK][R64_BN + 4];
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.y * R64_BM;
    const int col0 = blockIdx.x * R64_BN;
    const int tr = tid / 16, tc = tid % 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    // loader mapping: A tile 64 rows x 16 k = 1024 floats, 4 per thread
    const int a_row = tid / 4, a_k = (tid % 4) * 4;
    const int64_t grow = row0 + a_row;
    const float* xrow = nullptr;
    const float* crow = nullptr;
    if (grow < n) {
        const int64_t src = gather ? gather[grow] : grow;
        xrow = X + src * (int64_t)D;
        if (C) crow = C + (int64_t)(cl ? cl[grow] : 0) * D;
    }
    // B tile 16 k x 64 cols = 1024 floats, 4 per thread
    const int b_k = tid / 16, b_c = (tid % 16) * 4;

    for (int k0 = 0; k0 < D; k0 += R64_BK) {
        float4 av = make_float4(0.f, 0.f, 0.f, 0.f);
        if (xrow) {
            av = *reinterpret_cast<const float4*>(xrow + k0 + a_k);
            if (crow) {
                const float4 cv = *reinterpret_cast<const float4*>(crow + k0 + a_k);
                av.x = __fsub_rn(av.x, cv.x);
                av.y = __fsub_rn(av.y, cv.y);
                av.z = __fsub_rn(av.z, cv.z);
                av.w = __fsub_rn(av.w, cv.w);
            }
        }
        As[a_k + 0][a_row] = av.x;
        As[a_k + 1][a_row] = av.y;
        As[a_k + 2][a_row] = av.z;
        As[a_k + 3][a_row] = av.w;
        const float4 bv = *reinterpret_cast<const float4*>(P + (int64_t)(k0 + b_k) * D + col0 + b_c);
        *reinterpret_cast<float4*>(&Bs[b_k][b_c]) = bv;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < R64_BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = (double)As[kk][tr * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = (double)Bs[kk][tc * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = row0 + tr * 4 + i;
        if (r >= n) continue;
        float4 o;
        o.x = __double2float_rn(acc[i][0]);
        o.y = __double2float_rn(acc[i][1]);
        o.z = __double2float_rn(acc[i][2]);
        o.w = __double2float_rn(acc[i][3]);
        *reinterpret_cast<float4*>(out + r * D + col0 + tc * 4) = o;
    }
}

cudaError_t launch_rotate_fp64(const float* X, const int64_t* gather, const float* C, const int32_t* cl,
                               const float* P, float* out, int64_t n, int D, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t slab = 65535ll * R64_BM;
    for (int64_t r0 = 0; r0 < n; r0 += slab) {
        const int64_t m = n - r0 < slab ? n - r0 : slab;
        dim3 grid(D / R64_BN, (unsigned)ceil_div(m, R64_BM));
        // rows are addressed through `gather` when given, else directly
        count_launch();
        rotate_fp64_kernel<<<grid, 256, 0, s>>>(gather ? X : X + r0 * D, gather ? gather + r0 : nullptr, C,
                                                cl ? cl + r0 : nullptr, P, out + r0 * D, m, D);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 SGEMM  C[M][N] = A[M][K] * op(B), op(B) = B[K][N] (NN) or B[N][K]^T (NT).
// 128x128 tile, BK = 8, 256 threads, 8x8 outputs per thread (split 4+4 in both
// dimensions), register prefetch of the next tile.  K % 8 == 0; for NN N % 4 == 0.
// Epilogues:
//   EPI_PLAIN : C = alpha * acc + (addend ? addend[m][n] : 0)
//   EPI_DIST  : C = rown[m] + coln[n] - 2 * acc      (squared L2 distances)
// ---------------------------------------------------------------------------
enum { EPI_PLAIN = 0, EPI_DIST = 1 };

template <bool NT, int EPI>
__global__ void __launch_bounds__(256) sgemm_kernel(const float* __restrict__ A, const float* __restrict__ Bm,
                                                    float* __restrict__ Cm, int64_t M, int N, int K, float alpha,
                                                    const float* __restrict__ addend,
                                                    const float* __restrict__ rown,
                                                    const float* __restrict__ coln, int64_t ldc) {
    __shared__ __align__(16) float As[2][8][128];
    __shared__ __align__(16) float Bs[2][8][128];
    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.y * 128;
    const int n0 = blockIdx.x * 128;
    // A loader: row tid/2, k offset (tid%2)*4
    const int la_r = tid >> 1, la_k = (tid & 1) * 4;
    const bool a_ok = (m0 + la_r) < M;
    const float* a_ptr = A + (a_ok ? (m0 + la_r) : 0) * (int64_t)K + la_k;
    // B loader
    int lb_k, lb_n;
    bool b_ok;
    const float* b_ptr;
    if (NT) {
        lb_n = tid >> 1;
        lb_k = (tid & 1) * 4;
        b_ok = (n0 + lb_n) < N;
        b_ptr = Bm + (int64_t)(b_ok ? (n0 + lb_n) : 0) * K + lb_k;
    } else {
        lb_k = tid >> 5;
        lb_n = (tid & 31) * 4;
        b_ok = (n0 + lb_n) < N;
        b_ptr = Bm + (int64_t)lb_k * N + (b_ok ? n0 + lb_n : 0);
    }
    float4 ra, rb;
    auto load_regs = [&](int k0) {
        ra = a_ok ? *reinterpret_cast<const float4*>(a_ptr + k0) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (NT)
            rb = b_ok ? *reinterpret_cast<const float4*>(b_ptr + k0) : make_float4(0.f, 0.f, 0.f, 0.f);
        else
            rb = b_ok ? *reinterpret_cast<const float4*>(b_ptr + (int64_t)k0 * N) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto store_smem = [&](int buf) {
        As[buf][la_k + 0][la_r] = ra.x;
        As[buf][la_k + 1][la_r] = ra.y;
        As[buf][la_k + 2][la_r] = ra.z;
        As[buf][la_k + 3][la_r] = ra.w;
        if (NT) {
            Bs[buf][lb_k + 0][lb_n] = rb.x;
            Bs[buf][lb_k + 1][lb_n] = rb.y;
            Bs[buf][lb_k + 2][lb_n] = rb.z;
            Bs[buf][lb_k + 3][lb_n] = rb.w;
        } else {
            *reinterpret_cast<float4*>(&Bs[buf][lb_k][lb_n]) = rb;
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int ty = tid / 16, tx = tid % 16;
    load_regs(0);
    store_smem(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += 8) {
        const bool more = (k0 + 8) < K;
        if (more) load_regs(k0 + 8);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            float a[8], b[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store_smem(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int nn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (nn >= N) continue;
            float v;
            if (EPI == EPI_DIST) {
                v = rown[m] + coln[nn] - 2.f * acc[i][j];
            } else {
                v = alpha * acc[i][j];
                if (addend) v += addend[m * ldc + nn];
            }
            Cm[m * ldc + nn] = v;
        }
    }
}

constexpr int64_t kMaxSlabRows = 65535ll * 128;  // gridDim.y limit x tile rows

cudaError_t launch_sgemm(bool nt, const float* A, const float* B, float* C, int64_t M, int N, int K, float alpha,
                         const float* addend, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    for (int64_t m0 = 0; m0 < M; m0 += kMaxSlabRows) {
        const int64_t m = M - m0 < kMaxSlabRows ? M - m0 : kMaxSlabRows;
        dim3 grid((unsigned)ceil_div(N, 128), (unsigned)ceil_div(m, 128));
        const float* add = addend ? addend + m0 * N : nullptr;
        count_launch();
        if (nt)
            sgemm_kernel<true, EPI_PLAIN><<<grid, 256, 0, s>>>(A + m0 * K, B, C + m0 * N, m, N, K, alpha, add, nullptr,
                                                               nullptr, N);
        else
            sgemm_kernel<false, EPI_PLAIN><<<grid, 256, 0, s>>>(A + m0 * K, B, C + m0 * N, m, N, K, alpha, add,
                                                                nullptr, nullptr, N);
    }
    return cudaGetLastError();
}

cudaError_t launch_sqdist(const float* Q, const float* qn, const float* C, const float* cn, float* out, int64_t nq,
                          int nc, int D, cudaStream_t s) {
    if (nq <= 0 || nc <= 0) return cudaSuccess;
    for (int64_t m0 = 0; m0 < nq; m0 += kMaxSlabRows) {
        const int64_t m = nq - m0 < kMaxSlabRows ? nq - m0 : kMaxSlabRows;
        dim3 grid((unsigned)ceil_div(nc, 128), (unsigned)ceil_div(m, 128));
        count_launch();
        sgemm_kernel<true, EPI_DIST><<<grid, 256, 0, s>>>(Q + m0 * D, C, out + m0 * nc, m, nc, D, 1.f, nullptr,
                                                          qn + m0, cn, nc);
    }
    return cudaGetLastError();
}

// Squared norms of rows (FP32, one warp per row).
__global__ void row_sqnorm_kernel(const float* __restrict__ X, int64_t n, int D, float* __restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const float* x = X + w * D;
    float s = 0.f;
    for (int k = lane * 4; k < D; k += 128) {
        const float4 v = *reinterpret_cast<const float4*>(x + k);
        s = fmaf(v.x, v.x, s);
        s = fmaf(v.y, v.y, s);
        s = fmaf(v.z, v.z, s);
        s = fmaf(v.w, v.w, s);
    }
    s = warp_sum(s);
    if (lane == 0) out[w] = s;
}

// Rows scaled to unit length (cosine similarity as the inner product of unit
// vectors): y = fl32(x / sqrt(sum x^2)) with the sum in FP64, one warp per
// row; a zero row stays zero.  X and Y may be the same array (each thread
// rewrites only the elements it read).
__global__ void normalize_rows_kernel(const float* X, int64_t n, int D, float* Y) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float* x = X + r * D;
    double s = 0.0;
    for (int k = lane; k < D; k += 32) s += (double)x[k] * (double)x[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double nrm = sqrt(s);
    float* y = Y + r * D;
    for (int k = lane; k < D; k += 32) y[k] = nrm > 0.0 ? (float)((double)x[k] / nrm) : 0.f;
}

cudaError_t launch_normalize_rows(const float* X, int64_t n, int D, float* Y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    normalize_rows_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(X, n, D, Y);
    return cudaGetLastError();
}

cudaError_t launch_row_sqnorm(const float* X, int64_t n, int D, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    row_sqnorm_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(X, n, D, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cluster means (reading of Section 5.1 "local centroid"): one thread per
// (cluster, coordinate), FP64 sum over the cluster's rows in stored order
// (ascending original id), one division and one rounding to FP32.  Empty
// clusters keep `keep_empty ? old value : 0`.
// ---------------------------------------------------------------------------
__global__ void centroid_kernel(const float* __restrict__ X, const int64_t* __restrict__ list_off,
                                const int64_t* __restrict__ list_ids, int nlist, int D, float* __restrict__ C,
                                int keep_empty) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nlist * D) return;
    const int j = (int)(t / D), k = (int)(t % D);
    const int64_t b = list_off[j], e = list_off[j + 1];
    if (b == e) {
        if (!keep_empty) C[t] = 0.f;
        return;
    }
    double acc = 0.0;
    int64_t r = b;
    // four independent loads in flight; the additions stay in ascending order
    for (; r + 4 <= e; r += 4) {
        const float x0 = X[list_ids[r] * D + k];
        const float x1 = X[list_ids[r + 1] * D + k];
        const float x2 = X[list_ids[r + 2] * D + k];
        const float x3 = X[list_ids[r + 3] * D + k];
        acc = __dadd_rn(acc, (double)x0);
        acc = __dadd_rn(acc, (double)x1);
        acc = __dadd_rn(acc, (double)x2);
        acc = __dadd_rn(acc, (double)x3);
    }
    for (; r < e; ++r) acc = __dadd_rn(acc, (double)X[list_ids[r] * D + k]);
    C[t] = __double2float_rn(__ddiv_rn(acc, (double)(e - b)));
}

cudaError_t launch_centroids(const float* X, const int64_t* list_off, const int64_t* list_ids, int nlist, int D,
                             float* C, int keep_empty, cudaStream_t s) {
    const int64_t tot = (int64_t)nlist * D;
    count_launch();
    centroid_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(X, list_off, list_ids, nlist, D, C, keep_empty);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable counting sort of rows by cluster id.
//   pass 1: counts[b][c] = rows of chunk b in cluster c       (one warp per chunk)
//   pass 2: base[b][c] = list_off[c] + sum_{b'<b} counts[b'][c] (one thread per c)
//   pass 3: each chunk walks its rows in order; rank among equal clusters inside
//           a 32-row step comes from __match_any_sync, so rows land in ascending
//           id order within their cluster.
// ---------------------------------------------------------------------------
__global__ void group_count_kernel(const int32_t* __restrict__ assign, int64_t n, int64_t chunk, int nlist,
                                   int32_t* __restrict__ counts, uint32_t* __restrict__ status) {
    const int b = blockIdx.x;
    const int lane = threadIdx.x;
    const int64_t r0 = (int64_t)b * chunk, r1 = min(n, r0 + chunk);
    int32_t* cnt = counts + (int64_t)b * nlist;
    for (int64_t r = r0 + lane; r < r1; r += 32) {
        const int c = assign[r];
        if (c < 0 || c >= nlist) {
            atomicOr(status, kStatusBounds);
            continue;
        }
        atomicAdd(&cnt[c], 1);
    }
}

__global__ void group_scan_kernel(const int32_t* __restrict__ counts, int nb, int nlist,
                                  int64_t* __restrict__ total, int64_t* __restrict__ base) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nlist) return;
    int64_t s = 0;
    for (int b = 0; b < nb; ++b) {
        base[(int64_t)b * nlist + c] = s;
        s += counts[(int64_t)b * nlist + c];
    }
    total[c] = s;
}

// exclusive scan of nlist totals into list_off (single block, sequential per thread chunk)
__global__ void offsets_scan_kernel(const int64_t* __restrict__ total, int nlist, int64_t* __restrict__ off) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int per = (nlist + 1023) / 1024;
    const int c0 = t * per, c1 = min(nlist, c0 + per);
    int64_t s = 0;
    for (int c = c0; c < c1; ++c) s += total[c];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        off[nlist] = run;
    }
    __syncthreads();
    s = part[t];
    for (int c = c0; c < c1; ++c) {
        off[c] = s;
        s += total[c];
    }
}

__global__ void group_scatter_kernel(const int32_t* __restrict__ assign, int64_t n, int64_t chunk, int nlist,
                                     const int64_t* __restrict__ list_off, int64_t* __restrict__ base,
                                     int64_t* __restrict__ list_ids, int64_t* __restrict__ row_of,
                                     int32_t* __restrict__ cl_of_row) {
    const int b = blockIdx.x;
    const int lane = threadIdx.x;
    const int64_t r0 = (int64_t)b * chunk, r1 = min(n, r0 + chunk);
    int64_t* bs = base + (int64_t)b * nlist;
    for (int64_t s = r0; s < r1; s += 32) {
        const int64_t r = s + lane;
        const bool ok = r < r1;
        int c = ok ? assign[r] : -1;
        if (c < 0 || c >= nlist) c = -1;
        const unsigned active = __ballot_sync(0xffffffffu, ok && c >= 0);
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const unsigned grp = peers & active;
        if (ok && c >= 0) {
            const int leader = __ffs(grp) - 1;
            const int rank = __popc(grp & ((1u << lane) - 1u));
            int64_t old = 0;
            if (lane == leader) {
                old = bs[c];
                bs[c] = old + __popc(grp);
            }
            old = __shfl_sync(grp, old, leader);
            const int64_t pos = list_off[c] + old + rank;
            list_ids[pos] = r;
            if (row_of) row_of[r] = pos;
            if (cl_of_row) cl_of_row[pos] = c;
        }
        __syncwarp();
    }
}

cudaError_t launch_group(const int32_t* assign, int64_t n, int nlist, int64_t* list_off, int64_t* list_ids,
                         int64_t* row_of, int32_t* cl_of_row, void* scratch, size_t scratch_bytes,
                         uint32_t* status, cudaStream_t s) {
    int64_t chunk = 2048;
    // layout: counts (nb*nlist int32, 256-aligned) | base (nb*nlist int64) | total (nlist int64)
    while (ceil_div(n, chunk) * (int64_t)nlist * 12 + (int64_t)nlist * 8 + 512 > (int64_t)scratch_bytes) chunk *= 2;
    const int nb = (int)ceil_div(n, chunk);
    int32_t* counts = (int32_t*)scratch;
    int64_t* base = (int64_t*)((char*)scratch + ((size_t)nb * nlist * 4 + 255) / 256 * 256);
    int64_t* total = base + (int64_t)nb * nlist;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nb * nlist * 4, s);
    if (e != cudaSuccess) return e;
    count_launch();
    group_count_kernel<<<nb, 32, 0, s>>>(assign, n, chunk, nlist, counts, status);
    count_launch();
    group_scan_kernel<<<(unsigned)ceil_div(nlist, 256), 256, 0, s>>>(counts, nb, nlist, total, base);
    count_launch();
    offsets_scan_kernel<<<1, 1024, 0, s>>>(total, nlist, list_off);
    count_launch();
    group_scatter_kernel<<<nb, 32, 0, s>>>(assign, n, chunk, nlist, list_off, base, list_ids, row_of, cl_of_row);
    return cudaGetLastError();
}

size_t group_scratch_bytes(int64_t n, int nlist) {
    const int64_t nb = ceil_div(n, 2048);
    const size_t want = (size_t)nb * nlist * 12 + (size_t)nlist * 8 + 512;
    const size_t floor_bytes = (size_t)nlist * 8 * 3 + 4096;  // room for one chunk row
    const size_t cap = ((size_t)1 << 30) > floor_bytes ? ((size_t)1 << 30) : floor_bytes;
    return want < cap ? want : cap;
}

// ---------------------------------------------------------------------------
// Per-row selection of the p smallest values (ties by lower column) of a
// [rows][ncols] FP32 matrix.  One block per row; the row is processed in
// chunks of CH columns: the chunk's keys plus the running best p are sorted
// with a block-wide bitonic network in shared memory and the first p kept.
// out_idx[row][0..p-1] ascending; out_val optional.
// ---------------------------------------------------------------------------
__device__ void block_bitonic_sort_u64(uint64_t* a, int n) {
    // n is a power of two, blockDim.x threads cooperate
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const uint64_t x = a[lo], y = a[hi];
                if ((x > y) == up) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(512) row_topk_kernel(const float* __restrict__ V, int64_t rows, int ncols,
                                                       int64_t ld, int p, int sortn, int32_t* __restrict__ out_idx,
                                                       float* __restrict__ out_val, int64_t ld_out) {
    extern __shared__ uint64_t sk[];
    const int64_t row = blockIdx.x;
    const float* v = V + row * ld;
    const int chunk = sortn - p;  // new entries per round
    for (int i = threadIdx.x; i < p; i += blockDim.x) sk[i] = kEmptyKey;
    __syncthreads();
    for (int c0 = 0; c0 < ncols; c0 += chunk) {
        for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
            const int c = c0 + i;
            sk[p + i] = c < ncols ? make_key(v[c], (uint32_t)c) : kEmptyKey;
        }
        __syncthreads();
        block_bitonic_sort_u64(sk, sortn);
    }
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        const uint64_t k = sk[i];
        out_idx[row * ld_out + i] = k == kEmptyKey ? -1 : (int32_t)key_id(k);
        if (out_val) out_val[row * ld_out + i] = k == kEmptyKey ? INFINITY : key_value(k);
    }
}

cudaError_t launch_row_topk(const float* V, int64_t rows, int ncols, int64_t ld, int p, int32_t* out_idx,
                            float* out_val, int64_t ld_out, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    int sortn = 1024;
    while (sortn < 2 * p) sortn <<= 1;
    while (sortn < ncols + p && sortn < 8192) sortn <<= 1;
    cudaError_t e = cudaFuncSetAttribute(row_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sortn * 8);
    if (e != cudaSuccess) return e;
    count_launch();
    row_topk_kernel<<<(unsigned)rows, 512, sortn * 8, s>>>(V, rows, ncols, ld, p, sortn, out_idx, out_val, ld_out);
    return cudaGetLastError();
}

}  // namespace erq

namespace erq {

// Column of the smallest value in each row (ties -> lower column); one warp per row.
__global__ void row_argmin_kernel(const float* __restrict__ V, int64_t rows, int ncols, int32_t* __restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows) return;
    const float* v = V + w * ncols;
    uint64_t best = kEmptyKey;
    for (int c = lane; c < ncols; c += 32) {
        const uint64_t k = make_key(v[c], (uint32_t)c);
        best = k < best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t t = __shfl_xor_sync(0xffffffffu, best, o);
        best = t < best ? t : best;
    }
    if (lane == 0) out[w] = (int32_t)key_id(best);
}

cudaError_t launch_row_argmin(const float* V, int64_t rows, int ncols, int32_t* out, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    count_launch();
    row_argmin_kernel<<<(unsigned)ceil_div(rows * 32, 256), 256, 0, s>>>(V, rows, ncols, out);
    return cudaGetLastError();
}

__global__ void gather_rows_kernel(const float* __restrict__ X, const int64_t* __restrict__ idx, int64_t n, int D,
                                   float* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t vecs = (int64_t)n * (D / 4);
    if (t >= vecs) return;
    const int64_t r = t / (D / 4), c = t % (D / 4);
    reinterpret_cast<float4*>(out)[r * (D / 4) + c] = reinterpret_cast<const float4*>(X)[idx[r] * (D / 4) + c];
}

cudaError_t launch_gather_rows(const float* X, const int64_t* idx, int64_t n, int D, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    gather_rows_kernel<<<(unsigned)ceil_div(n * (D / 4), 256), 256, 0, s>>>(X, idx, n, D, out);
    return cudaGetLastError();
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, int32_t v) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = v;
}

cudaError_t launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    fill_i32_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

// k-means training sample: n evenly spaced row ids with a seed-dependent offset.
__global__ void strided_ids_kernel(int64_t* out, int64_t n, int64_t N, uint64_t seed) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double step = (double)N / (double)n;
    const int64_t off = (int64_t)(seed % (uint64_t)(step > 1.0 ? (int64_t)step : 1));
    int64_t r = (int64_t)((double)t * step) + off;
    out[t] = r < N ? r : N - 1;
}

cudaError_t launch_strided_ids(int64_t* out, int64_t n, int64_t N, uint64_t seed, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    strided_ids_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(out, n, N, seed);
    return cudaGetLastError();
}

}  // namespace erq

namespace erq {

// ---------------------------------------------------------------------------
// Per-row selection by radix select (probe lists): the p smallest (value,
// column) pairs of each row, ascending, ties by lower column.  One block of 256
// threads per row; the row's order-preserving keys stay in shared memory
// (ncols <= 16384).  Three histogram passes over 11 + 11 + 10 key bits find the
// p-th smallest key T; the entries below T and the lowest-column entries equal
// to T are gathered and sorted with a small bitonic network.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;

__global__ void __launch_bounds__(RS_THREADS) row_topk_radix_kernel(const float* __restrict__ V, int ncols,
                                                                    int64_t ld, int p, int sortn,
                                                                    int32_t* __restrict__ out_idx,
                                                                    float* __restrict__ out_val, int64_t ld_out) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    // [ncols] keys | [2048] histogram | [sortn] selected (the u64 array must be
    // 8-byte aligned for any ncols, so the key region is padded to 16 bytes)
    const size_t keys_bytes = ((size_t)ncols * 4 + 15) / 16 * 16;
    uint32_t* keys = reinterpret_cast<uint32_t*>(rs_smem);
    int* hist = reinterpret_cast<int*>(rs_smem + keys_bytes);
    uint64_t* sel = reinterpret_cast<uint64_t*>(rs_smem + keys_bytes + 2048 * 4);
    __shared__ int s_bin, s_below, s_nsel;
    const int64_t row = blockIdx.x;
    const float* v = V + row * ld;
    for (int i = threadIdx.x; i < ncols; i += RS_THREADS) keys[i] = float_to_ordered(v[i]);
    uint32_t prefix = 0, pmask = 0;
    int need = p;                       // rank (1-based) of the wanted key among the candidates
    const int shifts[3] = {21, 10, 0};
    const int widths[3] = {11, 11, 10};
    for (int pass = 0; pass < 3; ++pass) {
        const int nb = 1 << widths[pass];
        for (int i = threadIdx.x; i < nb; i += RS_THREADS) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < ncols; i += RS_THREADS) {
            const uint32_t k = keys[i];
            if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shifts[pass]) & (nb - 1)], 1);
        }
        __syncthreads();
        if (threadIdx.x < 32) {           // first bin whose running count reaches `need`
            const int per = nb / 32, lane = threadIdx.x;
            int mine = 0;
            for (int b = lane * per; b < (lane + 1) * per; ++b) mine += hist[b];
            int incl = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int excl = incl - mine;
            const unsigned hit = __ballot_sync(0xffffffffu, incl >= need && excl < need);
            if (lane == __ffs(hit) - 1) {
                int run = excl, b = lane * per;
                for (; b < (lane + 1) * per - 1; ++b) {
                    if (run + hist[b] >= need) break;
                    run += hist[b];
                }
                s_bin = b;
                s_below = run;
            }
        }
        __syncthreads();
        need -= s_below;
        prefix |= (uint32_t)s_bin << shifts[pass];
        pmask |= (uint32_t)(nb - 1) << shifts[pass];
        __syncthreads();
    }
    // T = prefix: `need` entries equal to T are wanted, all smaller ones are in
    const uint32_t T = prefix;
    if (threadIdx.x == 0) s_nsel = 0;
    for (int i = threadIdx.x; i < sortn; i += RS_THREADS) sel[i] = kEmptyKey;
    __syncthreads();
    for (int i = threadIdx.x; i < ncols; i += RS_THREADS) {
        const uint32_t k = keys[i];
        if (k < T) sel[atomicAdd(&s_nsel, 1)] = ((uint64_t)k << 32) | (uint32_t)i;
    }
    __syncthreads();
    // entries equal to T: the `need` lowest columns, found by scanning in column order
    if (threadIdx.x < 32) {
        const int base = s_nsel;
        int taken = 0;
        for (int c0 = 0; c0 < ncols && taken < need; c0 += 32) {
            const int i = c0 + threadIdx.x;
            const bool eq = i < ncols && keys[i] == T;
            const unsigned m = __ballot_sync(0xffffffffu, eq);
            const int rank = __popc(m & ((1u << threadIdx.x) - 1u));
            if (eq && taken + rank < need) sel[base + taken + rank] = ((uint64_t)T << 32) | (uint32_t)i;
            taken += __popc(m);
        }
    }
    __syncthreads();
    // sort the p selected keys
    for (int size = 2; size <= sortn; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < sortn / 2; i += RS_THREADS) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t x = sel[lo], y = sel[hi];
                if ((x > y) == up) { sel[lo] = y; sel[hi] = x; }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < p; i += RS_THREADS) {
        const uint64_t k = sel[i];
        out_idx[row * ld_out + i] = k == kEmptyKey ? -1 : (int32_t)(k & 0xffffffffu);
        if (out_val) out_val[row * ld_out + i] = k == kEmptyKey ? INFINITY : ordered_to_float((uint32_t)(k >> 32));
    }
}

// Smallest p <= 32 entries of each row (keys (value, column), so ties take the
// lower column), one warp per row.  A first pass takes the p-th smallest of the
// 32 lanes' minima over their columns: at least p entries lie at or below it,
// so it is a valid admission bound, and a tight one.  The second pass keeps the
// current p best in a sorted 32-entry list across the lanes; a 32-column chunk
// with an entry below the bound and the list's p-th key is sorted and merged in.
__global__ void __launch_bounds__(256) row_topk_warp_kernel(const float* __restrict__ V, int64_t rows, int ncols,
                                                            int64_t ld, int p, int32_t* __restrict__ out_idx,
                                                            float* __restrict__ out_val, int64_t ld_out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float* v = V + row * ld;
    constexpr int PF = 8;                        // chunks loaded ahead
    uint32_t lmin = 0xffffffffu;                 // this lane's smallest ordered value
    for (int c0 = 0; c0 < ncols; c0 += 32 * PF) {
        uint32_t o[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int c = c0 + 32 * u + lane;
            o[u] = c < ncols ? float_to_ordered(v[c]) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < PF; ++u) lmin = o[u] < lmin ? o[u] : lmin;
    }
    // p-th smallest lane minimum (lanes that saw no column contribute the maximum)
    const uint32_t bound = (uint32_t)(ws_shfl(ws_sort32(((uint64_t)lmin << 32) | (uint32_t)lane, lane), p - 1) >> 32);
    uint64_t list = kEmptyKey, th = kEmptyKey;
    for (int c0 = 0; c0 < ncols; c0 += 32 * PF) {
        uint32_t o[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int c = c0 + 32 * u + lane;
            o[u] = c < ncols ? float_to_ordered(v[c]) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int c = c0 + 32 * u + lane;
            const uint64_t key = ((uint64_t)o[u] << 32) | (uint32_t)c;
            const bool pass = c < ncols && o[u] <= bound && key < th;
            if (!__any_sync(0xffffffffu, pass)) continue;
            list = ws_merge32(list, ws_sort32(pass ? key : kEmptyKey, lane), lane);
            th = ws_shfl(list, p - 1);
        }
    }
    if (lane < p) {
        out_idx[row * ld_out + lane] = list == kEmptyKey ? -1 : (int32_t)(list & 0xffffffffu);
        if (out_val) out_val[row * ld_out + lane] = list == kEmptyKey ? INFINITY : ordered_to_float((uint32_t)(list >> 32));
    }
}

// Smallest p <= 32 entries of each row (keys (value, column), ties to the lower
// column) given the minimum of every 32-column group, one warp per row: the
// p-th smallest group minimum bounds the p-th smallest entry (p groups hold an
// entry at or below it), so only groups whose minimum is at or below it can
// hold an answer; those are read and merged into a sorted 32-entry warp list.
__global__ void __launch_bounds__(256) row_topk_groups_kernel(const float* __restrict__ V,
                                                              const float* __restrict__ gmin, int64_t rows, int ncols,
                                                              int64_t ld, int p, int32_t* __restrict__ out_idx,
                                                              int64_t ld_out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int ng = (ncols + 31) / 32;
    const float* gm = gmin + row * ng;
    // bound: p-th smallest group minimum (groups visited 32 at a time)
    uint64_t best = kEmptyKey;
    for (int g0 = 0; g0 < ng; g0 += 32) {
        const int gi = g0 + lane;
        const uint64_t key = gi < ng ? ((uint64_t)float_to_ordered(gm[gi]) << 32) | (uint32_t)gi : kEmptyKey;
        best = ws_merge32(best, ws_sort32(key, lane), lane);
    }
    const uint32_t bound = (uint32_t)(ws_shfl(best, p - 1) >> 32);
    const float* v = V + row * ld;
    uint64_t list = kEmptyKey, th = kEmptyKey;
    for (int g0 = 0; g0 < ng; g0 += 32) {
        const int gi = g0 + lane;
        uint32_t cand = __ballot_sync(0xffffffffu, gi < ng && float_to_ordered(gm[gi]) <= bound);
        while (cand) {                                   // candidate groups, up to 4 loaded together
            int gsel[4];
            uint32_t o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                gsel[u] = cand ? g0 + __ffs(cand) - 1 : -1;
                if (cand) cand &= cand - 1;
                const int c = gsel[u] * 32 + lane;
                o[u] = (gsel[u] >= 0 && c < ncols) ? float_to_ordered(v[c]) : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (gsel[u] < 0) break;                      // warp-uniform
                const int c = gsel[u] * 32 + lane;
                const uint64_t key = ((uint64_t)o[u] << 32) | (uint32_t)c;
                const bool pass = c < ncols && o[u] <= bound && key < th;
                ws_insert_each(list, th, key, pass, p, lane);
            }
        }
    }
    if (lane < p) out_idx[row * ld_out + lane] = list == kEmptyKey ? -1 : (int32_t)(list & 0xffffffffu);
}

cudaError_t launch_row_topk_groups(const float* V, const float* gmin, int64_t rows, int ncols, int64_t ld, int p,
                                   int32_t* out_idx, int64_t ld_out, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    count_launch();
    row_topk_groups_kernel<<<(unsigned)ceil_div(rows * 32, 256), 256, 0, s>>>(V, gmin, rows, ncols, ld, p, out_idx,
                                                                            ld_out);
    return cudaGetLastError();
}

cudaError_t launch_row_topk_fast(const float* V, int64_t rows, int ncols, int64_t ld, int p, int32_t* out_idx,
                                 float* out_val, int64_t ld_out, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    if (p <= 32) {
        count_launch();
        row_topk_warp_kernel<<<(unsigned)ceil_div(rows * 32, 256), 256, 0, s>>>(V, rows, ncols, ld, p, out_idx, out_val,
                                                                               ld_out);
        return cudaGetLastError();
    }
    if (ncols > 16384 || p > 2048) return launch_row_topk(V, rows, ncols, ld, p, out_idx, out_val, ld_out, s);
    int sortn = 32;
    while (sortn < p) sortn <<= 1;
    const size_t smem = ((size_t)ncols * 4 + 15) / 16 * 16 + 2048 * 4 + (size_t)sortn * 8;
    cudaError_t e = cudaFuncSetAttribute(row_topk_radix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    row_topk_radix_kernel<<<(unsigned)rows, RS_THREADS, smem, s>>>(V, ncols, ld, p, sortn, out_idx, out_val, ld_out);
    return cudaGetLastError();
}

}  // namespace erq

namespace erq {

// out[c][r] = X[r][c] (32x32 tiles through shared memory).
__global__ void transpose_kernel(const float* __restrict__ X, int rows, int cols, float* __restrict__ out) {
    __shared__ float t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = X[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(int64_t)c * rows + r] = t[threadIdx.x][i];
    }
}

cudaError_t launch_transpose(const float* X, int rows, int cols, float* out, cudaStream_t s) {
    count_launch();
    transpose_kernel<<<dim3((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32)), dim3(32, 8), 0, s>>>(X, rows,
                                                                                                         cols, out);
    return cudaGetLastError();
}

}  // namespace erq
