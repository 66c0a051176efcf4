// FP32-accurate dense GEMM on the tcgen05 tensor cores:
//   C[M][N] = A[M][K] * B[N][K]^T   (both operands K-major FP32 in memory)
// used for the query rotation q' = P^T q_r (B = P^T), the IVF centroid
// distances ||q - c||^2 = ||q||^2 + ||c||^2 - 2 <q, c> (B = centroids) and the
// P-multiply of the backward pass (B = P).
//
// Each FP32 operand row is first scaled by a power of two 2^-e (exact) so that
// its largest magnitude lies in [2^13, 2^14), then every element x is split into
// two FP16 numbers hi = RN16(x), lo = RN16(x - hi) (x - hi is exact in FP32).
// The product is accumulated in FP32 tensor memory as
//   hi_a*hi_b + hi_a*lo_b + lo_a*hi_b
// (each FP16 x FP16 product is exact in FP32); the dropped lo_a*lo_b term and
// the rounding of lo are below 2^-21 relative, the same order as FP32 SGEMM
// accumulation error.  The epilogue multiplies back by 2^(e_a + e_b).
//
// Tile 128 x 128, K block 64 (one 128-byte swizzle row of FP16), 3 pipeline
// stages of four 16 KB FP16 tiles (A_hi, A_lo, B_hi, B_lo), two TMEM
// accumulators (256 columns), persistent CTAs over output tiles.  Warp roles
// as in the code scan: 4 epilogue warps (TMEM lane = output row), 4 producer
// warps (load, scale, split, swizzle), 1 MMA warp.  All waits are bounded.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "tc_common.cuh"

namespace erq {

namespace gemm {
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3, THREADS = 288;
constexpr int TILE = 128 * BK * 2;                    // one FP16 tile: 16 KB
constexpr int STAGE = 4 * TILE;                        // A_hi, A_lo, B_hi, B_lo
constexpr int OFF_BARS = STAGES * STAGE;
constexpr int NBARS = 2 * STAGES + 4 + 1;
constexpr int OFF_TMEM = OFF_BARS + NBARS * 8;
constexpr int OFF_ABORT = OFF_TMEM + 4;
constexpr int SMEM = OFF_ABORT + 4 + 1024;

enum { EPI_PLAIN = 0, EPI_DIST = 1 };

struct Args {
    const float* A;
    const float* B;
    const int32_t* eA;       // [M] row exponents of A
    const int32_t* eB;       // [N] row exponents of B
    float* C;
    int64_t ldc;
    int64_t M;
    int N, K, epi;
    const float* addend;     // EPI_PLAIN: optional [M][ldc]
    const float* rown;       // EPI_DIST: [M]
    const float* coln;       // EPI_DIST: [N]
    uint32_t* status;
};

// x * 2^-e split into (hi, lo) FP16 halves of 8 consecutive elements.
__device__ __forceinline__ void split8(float4 a, float4 b, float s, uint4& hi, uint4& lo) {
    const float v[8] = {a.x * s, a.y * s, a.z * s, a.w * s, b.x * s, b.y * s, b.z * s, b.w * s};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half h0 = __float2half_rn(v[2 * i]), h1 = __float2half_rn(v[2 * i + 1]);
        const __half l0 = __float2half_rn(v[2 * i] - __half2float(h0));
        const __half l1 = __float2half_rn(v[2 * i + 1] - __half2float(h1));
        const __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
        h[i] = *reinterpret_cast<const uint32_t*>(&hh);
        l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
}  // namespace gemm

using namespace tc;

__global__ void __launch_bounds__(gemm::THREADS, 1) gemm_tc_kernel(gemm::Args a) {
    using namespace gemm;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BARS);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_TMEM);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]);
    const uint32_t tfull0 = smem_u32(&bars[2 * STAGES]), tempty0 = smem_u32(&bars[2 * STAGES + 2]);
    const uint32_t done_bar = smem_u32(&bars[2 * STAGES + 4]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = a.K / BK;
    const int64_t ntm = (a.M + BM - 1) / BM;
    const int ntn = (a.N + BN - 1) / BN;
    const int64_t ntiles = ntm * ntn;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 128);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 128);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= 4 && warp < 8) {
        // ---------------------------------------------------------------- producers
        const int pt = tid - 128;
        const int ch = pt & 7;                                  // 8-element chunk of the K block
        uint32_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int64_t m0 = (tile / ntn) * BM;
            const int n0 = (int)(tile % ntn) * BN;
            // rows pt/8 + 16 i of A and of B
            float sa[8], sb[8];
            const float* pa[8];
            const float* pb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = (pt >> 3) + 16 * i;
                const int64_t m = m0 + r;
                const int n = n0 + r;
                pa[i] = m < a.M ? a.A + m * a.K + ch * 8 : nullptr;
                pb[i] = n < a.N ? a.B + (int64_t)n * a.K + ch * 8 : nullptr;
                sa[i] = m < a.M ? __int_as_float((127 - a.eA[m]) << 23) : 0.f;   // 2^-e
                sb[i] = n < a.N ? __int_as_float((127 - a.eB[n]) << 23) : 0.f;
            }
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % STAGES;
                if (!mbar_wait(empty0 + 8 * s, ((it / STAGES) & 1) ^ 1, abort_flag)) { ok = false; break; }
                unsigned char* st = sm + s * STAGE;
                const int k0 = kb * BK;
                // A then B: 16 loads in flight per operand, then split and store
#pragma unroll
                for (int op = 0; op < 2; ++op) {
                    const float* const* src = op == 0 ? pa : pb;
                    const float* scl = op == 0 ? sa : sb;
                    float4 v[8][2];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (src[i]) {
                            v[i][0] = *reinterpret_cast<const float4*>(src[i] + k0);
                            v[i][1] = *reinterpret_cast<const float4*>(src[i] + k0 + 4);
                        } else {
                            v[i][0] = v[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int r = (pt >> 3) + 16 * i;
                        const int off = r * 128 + ((ch ^ (r & 7)) << 4);
                        uint4 hi, lo;
                        split8(v[i][0], v[i][1], scl[i], hi, lo);
                        *reinterpret_cast<uint4*>(st + (2 * op) * TILE + off) = hi;
                        *reinterpret_cast<uint4*>(st + (2 * op + 1) * TILE + off) = lo;
                    }
                }
                fence_proxy_async();
                mbar_arrive(full0 + 8 * s);
            }
        }
    } else if (warp == 8) {
        // ---------------------------------------------------------------- MMA issuer
        uint32_t it = 0, acc = 0;
        bool ok = true;
        const uint32_t idesc = idesc_f16(BM, BN);
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++acc) {
            const int buf = acc & 1;
            if (!mbar_wait_warp(tempty0 + 8 * buf, ((acc >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t dt = tmem + buf * BN;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % STAGES;
                if (!mbar_wait_warp(full0 + 8 * s, (it / STAGES) & 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t st = smem_u32(sm + s * STAGE);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        const uint64_t ahi = sdesc(st + 0 * TILE + k * 32), alo = sdesc(st + 1 * TILE + k * 32);
                        const uint64_t bhi = sdesc(st + 2 * TILE + k * 32), blo = sdesc(st + 3 * TILE + k * 32);
                        mma_f16(dt, ahi, bhi, idesc, (kb | k) != 0);
                        mma_f16(dt, ahi, blo, idesc, 1);
                        mma_f16(dt, alo, bhi, idesc, 1);
                    }
                    mma_commit(empty0 + 8 * s);
                    if (kb == nkb - 1) mma_commit(tfull0 + 8 * buf);
                }
                __syncwarp();
            }
        }
        if (lane == 0) mma_commit(done_bar);
        __syncwarp();
        mbar_wait_warp(done_bar, 0, abort_flag);
    } else {
        // ---------------------------------------------------------------- epilogue
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        uint32_t acc = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++acc) {
            const int64_t m0 = (tile / ntn) * BM;
            const int n0 = (int)(tile % ntn) * BN;
            const int buf = acc & 1;
            if (!mbar_wait_warp(tfull0 + 8 * buf, (acc >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            const int64_t m = m0 + tid;
            const bool mok = m < a.M;
            const int ea = mok ? a.eA[m] : 0;
            const float rn = (mok && a.epi == EPI_DIST) ? a.rown[m] : 0.f;
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                uint32_t r[32];
                ERQ_TMEM_LD32(tmem + lane_base + buf * BN + cc, r);
                const int nl = n0 + cc + lane;                 // column this lane loads factors for
                int eb = 0;
                float cn = 0.f;
                if (nl < a.N) {
                    eb = a.eB[nl];
                    if (a.epi == EPI_DIST) cn = a.coln[nl];
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float out[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int ebj = __shfl_sync(0xffffffffu, eb, j);
                    const float cnj = __shfl_sync(0xffffffffu, cn, j);
                    const float v = ldexpf(__uint_as_float(r[j]), ea + ebj);
                    out[j] = a.epi == EPI_DIST ? rn + cnj - 2.f * v : v;
                }
                if (mok) {
                    const int nb = n0 + cc;
                    float* crow = a.C + m * a.ldc + nb;
                    const float* arow = (a.epi == EPI_PLAIN && a.addend) ? a.addend + m * a.ldc + nb : nullptr;
                    if (nb + 32 <= a.N && (a.ldc % 4) == 0) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 o = make_float4(out[j], out[j + 1], out[j + 2], out[j + 3]);
                            if (arow) {
                                const float4 ad = *reinterpret_cast<const float4*>(arow + j);
                                o.x += ad.x; o.y += ad.y; o.z += ad.z; o.w += ad.w;
                            }
                            *reinterpret_cast<float4*>(crow + j) = o;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (nb + j < a.N) crow[j] = out[j] + (arow ? arow[j] : 0.f);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty0 + 8 * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(a.status, kStatusTimeout);
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
    }
}

// Row exponents e with max|x| * 2^-e in [2^13, 2^14) (0 for all-zero rows).
__global__ void row_exp_kernel(const float* __restrict__ X, int64_t n, int K, int32_t* __restrict__ e) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const float* x = X + w * K;
    float m = 0.f;
    for (int k = lane * 4; k < K; k += 128) {
        const float4 v = *reinterpret_cast<const float4*>(x + k);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    m = warp_max(m);
    if (lane == 0) {
        int ex = 0;
        if (m > 0.f) {
            frexpf(m, &ex);            // m in [2^(ex-1), 2^ex)
            ex = ex - 14;              // m * 2^-ex in [2^13, 2^14)
            ex = ex < -100 ? -100 : (ex > 100 ? 100 : ex);
        }
        e[w] = ex;
    }
}

cudaError_t launch_row_exp(const float* X, int64_t n, int K, int32_t* e, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    row_exp_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(X, n, K, e);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const float* A, const int32_t* eA, int64_t M, const float* B, const int32_t* eB, int N,
                           int K, float* C, int64_t ldc, int epi, const float* addend, const float* rown,
                           const float* coln, uint32_t* status, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    gemm::Args a;
    a.A = A; a.B = B; a.eA = eA; a.eB = eB; a.C = C; a.ldc = ldc; a.M = M; a.N = N; a.K = K; a.epi = epi;
    a.addend = addend; a.rown = rown; a.coln = coln; a.status = status;
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = ceil_div(M, gemm::BM) * ceil_div(N, gemm::BN);
    const int grid = (int)(tiles < sms ? tiles : sms);
    count_launch();
    gemm_tc_kernel<<<grid, gemm::THREADS, gemm::SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace erq
