// Two-stage (MSB-first) search of Section 4.2, for the regime of few queries
// per probed cluster, on CUDA cores in FP32.
//
// Stage 1 reads only the most significant bit plane of every probed row (one
// 8-byte word per row and 64 coordinates of the packed layout, i.e. 1/B of
// the code bytes).  Those bits are the 1-bit RaBitQ code of the row's
// residual, so with x0 = 2 msb - 1 the 1-bit estimate is
//     est1 = ||q_r - c||^2 + g1 + (f1 / 2) <x0, P^T q_r>
// (the same constant-folding as the B-bit estimate: g1 = ||o'||^2 -
// f1 <msb - 1/2, P^T c>, f1 = -4 ||o'||^2 / sum_i |o'_i|), and Lemma 2.1
// bounds its error by eps0 * err1 * ||q_r - c|| with
//     err1 = 2 ||o'|| sqrt(1 - a^2) / (a sqrt(D - 1)),  a = sum_i |o'_i| / (sqrt(D) ||o'||).
// <x0, P^T q_r> is read from per-query tables of the 16 signed sums of every
// group of four coordinates that share a nibble of the plane word (the
// table-lookup form of the paper's FastScan, with FP32 entries).
//
// Pruning rule: tau_q = the k'-th smallest upper bound est1 + bound over the
// query's probed rows (+inf with fewer rows); rows with est1 - bound > tau_q
// are dropped.  When every bound holds, each row of the true top-k' has
// est1 - bound <= d <= tau_q and survives.
//
// Stage 2 reads the remaining B - 1 bit words of the survivors only and
// completes <2 ybar_u - (2^B - 1), P^T q_r> by Eq. 4.2:
//     2^(B-1) <x0, P^T q_r> + <2 ylast - (2^(B-1) - 1), P^T q_r>,
// reusing stage 1's product; the survivors' top-k' (estimate, id) keys go to
// the exact re-rank.
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "erq_search.cuh"

namespace erq {

namespace {

constexpr int TS_THREADS = 128;

// One warp per stored row w of rows [r0, r0 + m): R holds their rotated
// residuals o' (FP32, [m][D]).  Writes {g1, f1 / 2, err1, 0} at the row's
// padded position.
__global__ void stage1_factors_kernel(const float* __restrict__ R, int64_t r0, int64_t m, int D, int B,
                                      const uint8_t* __restrict__ codes, const float* __restrict__ f_add,
                                      const float* __restrict__ Cp, const int32_t* __restrict__ cl_of_row,
                                      const int64_t* __restrict__ list_off, const int64_t* __restrict__ poff,
                                      float4* __restrict__ meta1) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= m) return;
    const int64_t w = r0 + i;
    const int c = cl_of_row[w];
    const float* o = R + i * D;
    const float* cp = Cp + (int64_t)c * D;
    double sabs = 0.0, yc = 0.0;
    for (int k = lane; k < D; k += 32) {
        sabs += fabs((double)o[k]);
        yc += ((double)(load_code(codes, B, w * D + k) >> (B - 1)) - 0.5) * (double)cp[k];
    }
    for (int s = 16; s > 0; s >>= 1) {
        sabs += __shfl_xor_sync(0xffffffffu, sabs, s);
        yc += __shfl_xor_sync(0xffffffffu, yc, s);
    }
    if (lane != 0) return;
    const double nr2 = (double)f_add[w];
    float4 v = make_float4((float)nr2, 0.f, 0.f, 0.f);
    if (nr2 > 0.0 && sabs > 0.0) {
        const double f1 = -4.0 * nr2 / sabs;
        const double a = sabs / (sqrt((double)D) * sqrt(nr2));
        const double err = 2.0 * sqrt(nr2) * sqrt(fmax(1.0 - a * a, 0.0)) / (a * sqrt((double)(D - 1)));
        v = make_float4((float)(nr2 - f1 * yc), (float)(0.5 * f1), (float)err, 0.f);
    }
    meta1[poff[c] + (w - list_off[c])] = v;
}

// T[q][g][v], g = 16 kb + n the nibble n of K block kb's plane word, v its
// value: sum over its four bits t of (+-1) * P^T q_r at the bit's coordinate.
// Bit 32h + 8L + j of a plane word is coordinate 32h + 4j + L of the block
// (the packed layout), so nibble n holds coordinates
// 32 (n >> 3) + 16 (n & 1) + ((n >> 1) & 3) + 4t.
__global__ void msb_table_kernel(const float* __restrict__ Qrot, int64_t nq, int D, float* __restrict__ T) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_q = (int64_t)(D / 4) * 16;
    if (t >= nq * per_q) return;
    const int64_t q = t / per_q;
    const int g = (int)((t % per_q) >> 4), v = (int)(t & 15);
    const int kb = g >> 4, n = g & 15;
    const int base = 64 * kb + 32 * (n >> 3) + 16 * (n & 1) + ((n >> 1) & 3);
    const float* x = Qrot + q * D;
    float s = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) s += ((v >> b) & 1) ? x[base + 4 * b] : -x[base + 4 * b];
    T[t] = s;
}

// Warp per query: rbase[q][slot] = rows of the query's earlier valid probes,
// qrows[q] = rows of all of them.
__global__ void ts_rows_kernel(const int32_t* __restrict__ probe_c, int64_t nq, int maxp,
                               const int64_t* __restrict__ list_off, int32_t* __restrict__ rbase,
                               int64_t* __restrict__ qrows) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    int64_t carry = 0;
    for (int s0 = 0; s0 < maxp; s0 += 32) {
        const int s = s0 + lane;
        const int c = s < maxp ? probe_c[q * maxp + s] : -1;
        int64_t sz = c >= 0 ? list_off[c + 1] - list_off[c] : 0;
        int64_t inc = sz;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (s < maxp) rbase[q * maxp + s] = (int32_t)(carry + inc - sz);
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) qrows[q] = carry;
}

struct TsArgs {
    const int32_t* probe_c;     // [nq][maxp] validated probes (-1: none)
    const float* dqc;           // [nq][maxp] ||q_r - c||^2
    const int64_t* list_off;
    const int64_t* poff;
    const uint64_t* codes_p;    // packed codes (layout at unpack_codes in the tensor-core scan)
    const float4* rowmeta;      // [Np] {g, f_res / 2, id, 0}
    const float4* meta1;        // [Np] {g1, f1 / 2, err1, 0}
    const float* T;             // [nq][D/4][16] plane-word nibble tables
    const float* Qrot;          // [nq][D] P^T q_r
    const int32_t* rbase;       // [nq][maxp]
    const int64_t* qoffr;       // [nq + 1] first row slot of each query
    float* ub;                  // per (query, probed row): est1 + bound
    float* lb;                  //                          est1 - bound
    float* s1;                  //                          <x0, P^T q_r>
    const float* tau;           // [nq]
    int32_t* scnt;              // [nq] survivors
    uint64_t* skey;             // per (query, probed row) slot: survivors' keys
    int64_t nq;
    int maxp, D, B;
    float eps0;
};

// Block per (query, probe slot); thread per row of the probed cluster.
__global__ void __launch_bounds__(TS_THREADS) ts_stage1_kernel(TsArgs a) {
    extern __shared__ __align__(16) float tab[];          // [D/4][16]
    const int64_t q = blockIdx.x / a.maxp;
    const int slot = (int)(blockIdx.x % a.maxp);
    const int c = a.probe_c[q * a.maxp + slot];
    if (c < 0) return;
    const int D = a.D, B = a.B, nkb = D / 64;
    const float4* src = reinterpret_cast<const float4*>(a.T + q * (int64_t)D * 4);
    for (int i = threadIdx.x; i < D; i += TS_THREADS) reinterpret_cast<float4*>(tab)[i] = src[i];
    __syncthreads();
    const int64_t size = a.list_off[c + 1] - a.list_off[c], pc = a.poff[c];
    const float dq = a.dqc[q * a.maxp + slot];
    const float bq = a.eps0 * sqrtf(fmaxf(dq, 0.f));
    const int64_t o0 = a.qoffr[q] + a.rbase[q * a.maxp + slot];
    for (int64_t j = threadIdx.x; j < size; j += TS_THREADS) {
        const int64_t p = pc + j;
        const uint64_t* w = a.codes_p + ((p >> 5) * nkb * B + (B - 1)) * 32 + (p & 31);
        float s = 0.f;
        for (int kb = 0; kb < nkb; ++kb) {
            const uint64_t W = __ldg(w + (int64_t)kb * B * 32);
            const float* t = tab + kb * 256;
#pragma unroll
            for (int n = 0; n < 16; ++n) s += t[16 * n + (int)((W >> (4 * n)) & 15u)];
        }
        const float4 m = a.meta1[p];
        const float est1 = dq + m.x + m.y * s, bd = bq * m.z;
        a.ub[o0 + j] = est1 + bd;
        a.lb[o0 + j] = est1 - bd;
        a.s1[o0 + j] = s;
    }
}

// k-th smallest (1-based, k <= n) of n unsigned keys, by one block: a radix
// select over 8-bit digits from the most significant; every thread returns it.
template <typename K>
__device__ K block_select_kth(const K* keys, int64_t n, int64_t k, unsigned* hist, K* s_pre, int64_t* s_k) {
    K prefix = 0, mask = 0;
    for (int shift = 8 * (int)sizeof(K) - 8; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const K v = keys[i];
            if ((v & mask) == prefix) atomicAdd(&hist[(int)((v >> shift) & 255)], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t cum = 0;
            int d = 0;
            for (; d < 255; ++d) {
                if (cum + hist[d] >= k) break;
                cum += hist[d];
            }
            *s_pre = prefix | ((K)d << shift);
            *s_k = k - cum;
        }
        __syncthreads();
        prefix = *s_pre;
        k = *s_k;
        mask |= (K)255 << shift;
        __syncthreads();
    }
    return prefix;
}

// Block per query: tau = k'-th smallest upper bound (+inf with fewer rows).
__global__ void ts_tau_kernel(const float* __restrict__ ub, const int64_t* __restrict__ qoffr, int64_t nq, int kp,
                              float* __restrict__ tau, uint32_t* __restrict__ scratch) {
    __shared__ unsigned hist[256];
    __shared__ uint32_t s_pre;
    __shared__ int64_t s_k;
    const int64_t q = blockIdx.x;
    const int64_t b = qoffr[q], n = qoffr[q + 1] - b;
    if (n < kp) {
        if (threadIdx.x == 0) tau[q] = INFINITY;
        return;
    }
    uint32_t* keys = scratch + b;                           // ordered images of the upper bounds
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) keys[i] = float_to_ordered(ub[b + i]);
    __syncthreads();
    const uint32_t kth = block_select_kth<uint32_t>(keys, n, kp, hist, &s_pre, &s_k);
    if (threadIdx.x == 0) tau[q] = ordered_to_float(kth);
}

// <2 ylast - (2^(B-1) - 1), x> over one 64-coordinate block: `w` points at word
// 0 of the row (word j at w + 32 j), x at the block's 64 query coordinates.
// Coordinates 4m + L: bits 0-3 from the nibble words (B >= 5), bit b >= 4 of
// plane b; for B <= 3 every bit from its plane.
template <int B>
__device__ __forceinline__ float last_bits_dot(const uint64_t* w, const float* x) {
    constexpr float off = (float)((1 << (B - 1)) - 1);
    uint2 W[B > 1 ? B - 1 : 1];
#pragma unroll
    for (int j = 0; j < B - 1; ++j) W[j] = *reinterpret_cast<const uint2*>(w + 32 * j);
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
#pragma unroll
        for (int L = 0; L < 4; ++L) {
            uint32_t u = 0;
            if constexpr (B >= 5) {
                const int h = m >> 1;
                const uint32_t N = (h & 1) ? W[h >> 1].y : W[h >> 1].x;
                u = (N >> (8 * L + ((m & 1) ? 4 : 0))) & 15u;
#pragma unroll
                for (int b = 4; b < B - 1; ++b) {
                    const uint32_t P = m < 8 ? W[b].x : W[b].y;
                    u |= ((P >> (8 * L + (m & 7))) & 1u) << b;
                }
            } else {
#pragma unroll
                for (int b = 0; b < B - 1; ++b) {
                    const uint32_t P = m < 8 ? W[b].x : W[b].y;
                    u |= ((P >> (8 * L + (m & 7))) & 1u) << b;
                }
            }
            acc = fmaf(2.f * (float)u - off, x[4 * m + L], acc);
        }
    }
    return acc;
}

template <int B>
__device__ float last_bits_row(const uint64_t* w0, int nkb, const float* x) {
    float s = 0.f;
    for (int kb = 0; kb < nkb; ++kb) s += last_bits_dot<B>(w0 + (int64_t)kb * B * 32, x + 64 * kb);
    return s;
}

__device__ float last_bits_row_b(int B, const uint64_t* w0, int nkb, const float* x) {
    switch (B) {
        case 1: return 0.f;
        case 2: return last_bits_row<2>(w0, nkb, x);
        case 3: return last_bits_row<3>(w0, nkb, x);
        case 5: return last_bits_row<5>(w0, nkb, x);
        case 6: return last_bits_row<6>(w0, nkb, x);
        case 7: return last_bits_row<7>(w0, nkb, x);
        case 8: return last_bits_row<8>(w0, nkb, x);
        default: return last_bits_row<9>(w0, nkb, x);
    }
}

// Block per (query, probe slot): the survivors' full estimates (Eq. 4.2) and keys.
__global__ void __launch_bounds__(TS_THREADS) ts_stage2_kernel(TsArgs a) {
    extern __shared__ __align__(16) float xq[];            // [D] P^T q_r
    const int64_t q = blockIdx.x / a.maxp;
    const int slot = (int)(blockIdx.x % a.maxp);
    const int c = a.probe_c[q * a.maxp + slot];
    if (c < 0) return;
    const int D = a.D, B = a.B, nkb = D / 64;
    for (int i = threadIdx.x; i < D; i += TS_THREADS) xq[i] = a.Qrot[q * D + i];
    __syncthreads();
    const int64_t size = a.list_off[c + 1] - a.list_off[c], pc = a.poff[c];
    const float dq = a.dqc[q * a.maxp + slot], tq = a.tau[q];
    const int64_t o0 = a.qoffr[q] + a.rbase[q * a.maxp + slot];
    const float hi = (float)(1 << (B - 1));
    for (int64_t j = threadIdx.x; j < size; j += TS_THREADS) {
        if (a.lb[o0 + j] > tq) continue;
        const int64_t p = pc + j;
        const uint64_t* w0 = a.codes_p + ((p >> 5) * nkb * B) * 32 + (p & 31);
        const float s = fmaf(hi, a.s1[o0 + j], last_bits_row_b(B, w0, nkb, xq));
        const float4 m = a.rowmeta[p];
        const float est = dq + fmaf(m.y, s, m.x);
        const int pos = atomicAdd(a.scnt + q, 1);
        a.skey[a.qoffr[q] + pos] = make_key(est, __float_as_uint(m.z));
    }
}

// Block per query: its k' smallest survivor keys, ascending, padded with
// empty keys.
__global__ void ts_select_kernel(const uint64_t* __restrict__ skey, const int64_t* __restrict__ qoffr,
                                 const int32_t* __restrict__ scnt, int64_t nq, int kp, uint64_t* __restrict__ cand) {
    __shared__ unsigned hist[256];
    __shared__ uint64_t s_pre;
    __shared__ int64_t s_k;
    __shared__ int s_cnt;
    __shared__ uint64_t buf[1024];
    const int64_t q = blockIdx.x;
    const uint64_t* keys = skey + qoffr[q];
    const int64_t m = scnt[q];
    uint64_t kth = kEmptyKey;
    if (m > kp) kth = block_select_kth<uint64_t>(keys, m, kp, hist, &s_pre, &s_k);
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        const uint64_t v = keys[i];
        if (v <= kth) {
            const int pos = atomicAdd(&s_cnt, 1);
            if (pos < kp) buf[pos] = v;
        }
    }
    __syncthreads();
    const int cnt = min(s_cnt, kp);
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        if (i >= cnt) buf[i] = kEmptyKey;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)            // bitonic sort, ascending
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t x = buf[i], y = buf[j];
                    if ((x > y) == up) {
                        buf[i] = y;
                        buf[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < kp; i += blockDim.x) cand[q * kp + i] = i < cnt ? buf[i] : kEmptyKey;
}

}  // namespace

cudaError_t launch_stage1_factors(const float* R, int64_t r0, int64_t m, int D, int B, const uint8_t* codes,
                                  const float* f_add, const float* Cp, const int32_t* cl_of_row,
                                  const int64_t* list_off, const int64_t* poff, float4* meta1, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    count_launch();
    stage1_factors_kernel<<<(unsigned)ceil_div(m * 32, 256), 256, 0, s>>>(R, r0, m, D, B, codes, f_add, Cp, cl_of_row,
                                                                         list_off, poff, meta1);
    return cudaGetLastError();
}

cudaError_t launch_two_stage_rows(const int32_t* probe_c, int64_t nq, int maxp, const int64_t* list_off,
                                  int32_t* rbase, int64_t* qrows, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    count_launch();
    ts_rows_kernel<<<(unsigned)ceil_div(nq * 32, 256), 256, 0, s>>>(probe_c, nq, maxp, list_off, rbase, qrows);
    return cudaGetLastError();
}

cudaError_t launch_two_stage(const TwoStageLaunch& L, cudaStream_t s) {
    if (L.nq <= 0) return cudaSuccess;
    if (L.D % 64 != 0 || L.B < 1 || L.B > 9 || L.B == 4 || L.kp < 1 || L.kp > 1024) return cudaErrorInvalidValue;
    // the tables are read as float4, the keys as u64
    if (((uintptr_t)L.T & 15) != 0 || ((uintptr_t)L.skey & 7) != 0 || ((uintptr_t)L.meta1 & 15) != 0)
        return cudaErrorInvalidValue;
    TsArgs a;
    a.probe_c = L.probe_c; a.dqc = L.dqc; a.list_off = L.list_off; a.poff = L.poff; a.codes_p = L.codes_p;
    a.rowmeta = L.rowmeta; a.meta1 = L.meta1; a.T = L.T; a.Qrot = L.Qrot; a.rbase = L.rbase; a.qoffr = L.qoffr;
    a.ub = L.ub; a.lb = L.lb; a.s1 = L.s1; a.tau = L.tau; a.scnt = L.scnt; a.skey = L.skey;
    a.nq = L.nq; a.maxp = L.maxp; a.D = L.D; a.B = L.B; a.eps0 = L.eps0;
    const int64_t blocks = L.nq * L.maxp;
    const size_t tab_bytes = (size_t)L.D * 16;
    cudaError_t e = cudaFuncSetAttribute(ts_stage1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_bytes);
    if (e != cudaSuccess) return e;
    count_launch();
    msb_table_kernel<<<(unsigned)ceil_div(L.nq * (L.D / 4) * 16, 256), 256, 0, s>>>(L.Qrot, L.nq, L.D, L.T);
    count_launch();
    ts_stage1_kernel<<<(unsigned)blocks, TS_THREADS, tab_bytes, s>>>(a);
    count_launch();
    ts_tau_kernel<<<(unsigned)L.nq, 256, 0, s>>>(L.ub, L.qoffr, L.nq, L.kp, L.tau, L.scratch);
    if ((e = cudaMemsetAsync(L.scnt, 0, sizeof(int32_t) * L.nq, s)) != cudaSuccess) return e;
    count_launch();
    ts_stage2_kernel<<<(unsigned)blocks, TS_THREADS, (size_t)L.D * 4, s>>>(a);
    count_launch();
    ts_select_kernel<<<(unsigned)L.nq, 256, 0, s>>>(L.skey, L.qoffr, L.scnt, L.nq, L.kp, L.cand);
    return cudaGetLastError();
}

}  // namespace erq
