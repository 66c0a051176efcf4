// FP32-accurate dense GEMM on the tcgen05 tensor cores with TMA-fed operands:
//   C[M][N] = A[M][K] * B[N][K]^T
// for the query rotation q' = P^T q_r (B = P^T) and the IVF centroid distances
// ||q - c||^2 = ||q||^2 + ||c||^2 - 2 <q, c> (B = centroids).
//
// The operands arrive pre-split: every FP32 row x is scaled by an exact power
// of two 2^-e (largest magnitude in [2^13, 2^14)) and written as two FP16 rows
// hi = RN16(x), lo = RN16(x - hi) (split_hilo_kernel; the centroids and P^T are
// split once per index, the queries once per search).  The product is
// accumulated in FP32 tensor memory as hi_a*hi_b + hi_a*lo_b + lo_a*hi_b; each
// FP16 x FP16 product is exact in FP32, and the dropped lo_a*lo_b term and the
// rounding of lo are below 2^-21 relative, the order of FP32 SGEMM error.  The
// epilogue multiplies back by 2^(e_a + e_b).
//
// The epilogue writes C, the distances, or -C (inner-product probe); for the
// last two it can also write the minimum of every 32-column group of a row
// (used by the probe selection).
// Tile 128 x 256, K block 64 (one 128-byte swizzle row of FP16); a stage is
// four TMA tiles (A_hi, A_lo 16 KB each; B_hi, B_lo 32 KB each), two stages;
// two TMEM accumulators of 256 columns, persistent CTAs over output tiles.
// Warp roles: 4 epilogue warps (TMEM lane = output row), 1 TMA warp, 1 MMA
// warp.  Every wait is bounded (status word on expiry).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "tc_common.cuh"

namespace erq {

namespace gemm2 {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 2, THREADS = 192;
constexpr int TILE_A = BM * BK * 2;                   // 16 KB
constexpr int TILE_B = BN * BK * 2;                   // 32 KB
constexpr int STAGE = 2 * TILE_A + 2 * TILE_B;        // A_hi, A_lo, B_hi, B_lo
constexpr int OFF_BARS = STAGES * STAGE;
constexpr int NBARS = 2 * STAGES + 4 + 1;
constexpr int OFF_CF = (OFF_BARS + NBARS * 8 + 15) / 16 * 16;   // 4 epilogue warps x 32 column factors (float2)
constexpr int OFF_EB = OFF_CF + 4 * 32 * 8;                      // 4 epilogue warps x 32 column exponents
constexpr int OFF_TMEM = OFF_EB + 4 * 32 * 4;
constexpr int OFF_ABORT = OFF_TMEM + 4;
constexpr int SMEM = OFF_ABORT + 4 + 1024;
static_assert(SMEM <= 227 * 1024, "gemm shared memory");

enum { EPI_PLAIN = 0, EPI_DIST = 1, EPI_NEGIP = 2 };   // C, ||a||^2 + ||b||^2 - 2C, -C

struct Args {
    const int32_t* eA;       // [M] row exponents of A
    const int32_t* eB;       // [N] row exponents of B
    float* C;
    int64_t ldc;
    int64_t M;
    int N, K, epi;
    const float* rown;       // EPI_DIST: [M]
    const float* coln;       // EPI_DIST: [N]
    float* gmin;             // EPI_DIST, optional: [M][ceil(N / 32)] minimum of each 32-column group
    __half* Ch;              // optional: an FP16 copy of the output (round to nearest), same layout
    uint32_t* status;
};
}  // namespace gemm2

using namespace tc;

__global__ void __launch_bounds__(gemm2::THREADS, 1)
    gemm_tma_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, gemm2::Args a) {
    using namespace gemm2;
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
            mbar_init(full0 + 8 * s, 1);
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
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        // ---------------------------------------------------------------- TMA
        uint32_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int m0 = (int)((tile / ntn) * BM);
            const int n0 = (int)(tile % ntn) * BN;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % STAGES;
                if (!mbar_wait_warp(empty0 + 8 * s, ((it / STAGES) & 1) ^ 1, abort_flag)) { ok = false; break; }
                if (lane == 0) {
                    const uint32_t st = smem_u32(sm + s * STAGE), bar = full0 + 8 * s;
                    mbar_arrive_expect_tx(bar, STAGE);
                    tma_load_2d(st, &mAh, kb * BK, m0, bar);
                    tma_load_2d(st + TILE_A, &mAl, kb * BK, m0, bar);
                    tma_load_2d(st + 2 * TILE_A, &mBh, kb * BK, n0, bar);
                    tma_load_2d(st + 2 * TILE_A + TILE_B, &mBl, kb * BK, n0, bar);
                }
                __syncwarp();
            }
        }
        // drain: the copies issued to the last stages land before the CTA exits
        for (uint32_t k = 0; k < STAGES && k < it; ++k) {
            const uint32_t gg = it - 1 - k;
            mbar_wait_drain(full0 + 8 * (gg % STAGES), (gg / STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == 5) {
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
                        const uint64_t ahi = sdesc(st + k * 32), alo = sdesc(st + TILE_A + k * 32);
                        const uint64_t bhi = sdesc(st + 2 * TILE_A + k * 32);
                        const uint64_t blo = sdesc(st + 2 * TILE_A + TILE_B + k * 32);
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
        mbar_wait_drain(done_bar, 0);
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float2* cf = reinterpret_cast<float2*>(sm + OFF_CF) + warp * 32;   // this warp's column factors
        int* ebs = reinterpret_cast<int*>(sm + OFF_EB) + warp * 32;
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
                if (n0 + cc >= a.N) break;                     // warp-uniform
                uint32_t r[32];
                ERQ_TMEM_LD32(tmem + lane_base + buf * BN + cc, r);
                const int nl = n0 + cc + lane;                 // column this lane loads factors for
                int eb = 0;
                float cn = 0.f;
                if (nl < a.N) {
                    eb = a.eB[nl];
                    if (a.epi == EPI_DIST) cn = a.coln[nl];
                }
                // v * 2^ea * 2^eb in two exact power-of-two multiplications, which
                // equals ldexpf(v, ea + eb) when 2^ea and 2^eb are normal numbers and
                // v * 2^ea stays normal: v is 0 or at least 2^-48 (a sum of FP16
                // products) and below 2^40, so ea in [-78, 87] suffices; other rows
                // and chunks take ldexpf
                int ebmin = nl < a.N ? eb : 0, ebmax = nl < a.N ? eb : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ebmin = min(ebmin, __shfl_xor_sync(0xffffffffu, ebmin, o));
                    ebmax = max(ebmax, __shfl_xor_sync(0xffffffffu, ebmax, o));
                }
                const bool fast = ebmin >= -126 && ebmax <= 127 && ea >= -78 && ea <= 87;
                __syncwarp();                                  // the previous chunk's factors are consumed
                cf[lane] = make_float2(ebmin >= -126 && ebmax <= 127 ? __int_as_float((eb + 127) << 23) : 0.f, cn);
                ebs[lane] = eb;
                __syncwarp();
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float out[32];
                if (fast) {
                    const float sa = __int_as_float((ea + 127) << 23);
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const float4 f = *reinterpret_cast<const float4*>(cf + j);   // same address in every lane
                        const float v0 = (__uint_as_float(r[j]) * sa) * f.x;
                        const float v1 = (__uint_as_float(r[j + 1]) * sa) * f.z;
                        out[j] = a.epi == EPI_DIST ? rn + f.y - 2.f * v0 : (a.epi == EPI_NEGIP ? -v0 : v0);
                        out[j + 1] = a.epi == EPI_DIST ? rn + f.w - 2.f * v1 : (a.epi == EPI_NEGIP ? -v1 : v1);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float v = ldexpf(__uint_as_float(r[j]), ea + ebs[j]);
                        out[j] = a.epi == EPI_DIST ? rn + cf[j].y - 2.f * v : (a.epi == EPI_NEGIP ? -v : v);
                    }
                }
                if (mok && a.gmin) {                           // group minimum over the valid columns
                    float g = INFINITY;
#pragma unroll
                    for (int j = 0; j < 32; ++j) g = (n0 + cc + j < a.N) ? fminf(g, out[j]) : g;
                    a.gmin[m * ((a.N + 31) / 32) + (n0 + cc) / 32] = g;
                }
                if (mok) {
                    const int nb = n0 + cc;
                    float* crow = a.C + m * a.ldc + nb;
                    if (nb + 32 <= a.N && (a.ldc % 4) == 0) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4*>(crow + j) = make_float4(out[j], out[j + 1], out[j + 2], out[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (nb + j < a.N) crow[j] = out[j];
                    }
                    if (a.Ch) {                                // FP16 copy (16-byte stores when aligned)
                        __half* hrow = a.Ch + m * a.ldc + nb;
                        if (nb + 32 <= a.N && (a.ldc % 8) == 0) {
#pragma unroll
                            for (int j = 0; j < 32; j += 8) {
                                const __half2 h0 = __floats2half2_rn(out[j], out[j + 1]);
                                const __half2 h1 = __floats2half2_rn(out[j + 2], out[j + 3]);
                                const __half2 h2 = __floats2half2_rn(out[j + 4], out[j + 5]);
                                const __half2 h3 = __floats2half2_rn(out[j + 6], out[j + 7]);
                                *reinterpret_cast<uint4*>(hrow + j) = make_uint4(
                                    *reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1),
                                    *reinterpret_cast<const uint32_t*>(&h2), *reinterpret_cast<const uint32_t*>(&h3));
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (nb + j < a.N) hrow[j] = __float2half_rn(out[j]);
                        }
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
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// x * 2^-e -> (hi, lo) FP16 pairs, 8 elements per thread.
__global__ void split_hilo_kernel(const float* __restrict__ X, const int32_t* __restrict__ e, int64_t M, int K,
                                  __half* __restrict__ hi, __half* __restrict__ lo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int per = K / 8;
    if (t >= M * per) return;
    const int64_t m = t / per;
    const float s = __int_as_float((127 - e[m]) << 23);        // 2^-e, |e| <= 100
    const float4 a = reinterpret_cast<const float4*>(X)[2 * t];
    const float4 b = reinterpret_cast<const float4*>(X)[2 * t + 1];
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
    reinterpret_cast<uint4*>(hi)[t] = make_uint4(h[0], h[1], h[2], h[3]);
    reinterpret_cast<uint4*>(lo)[t] = make_uint4(l[0], l[1], l[2], l[3]);
}

// Per-search query preparation in one pass per row (one warp per row): the
// row exponent of row_exp_kernel, optionally the squared norm in the order of
// row_sqnorm_kernel, and the hi/lo split of split_hilo_kernel -- the same
// operations, so the same bits, with the row read twice (the second time from
// cache) instead of three times by three launches.
__global__ void query_prep_kernel(const float* __restrict__ X, int64_t M, int K, int32_t* __restrict__ e,
                                  float* __restrict__ sqn, __half* __restrict__ hi, __half* __restrict__ lo) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= M) return;
    const float* x = X + w * K;
    float mx = 0.f, ss = 0.f;
    for (int k = lane * 4; k < K; k += 128) {
        const float4 v = *reinterpret_cast<const float4*>(x + k);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        ss = fmaf(v.x, v.x, ss);
        ss = fmaf(v.y, v.y, ss);
        ss = fmaf(v.z, v.z, ss);
        ss = fmaf(v.w, v.w, ss);
    }
    mx = warp_max(mx);
    ss = warp_sum(ss);
    int ex = 0;
    if (mx > 0.f) {
        frexpf(mx, &ex);               // mx in [2^(ex-1), 2^ex)
        ex = ex - 14;                  // mx * 2^-ex in [2^13, 2^14)
        ex = ex < -100 ? -100 : (ex > 100 ? 100 : ex);
    }
    if (lane == 0) {
        e[w] = ex;
        if (sqn) sqn[w] = ss;
    }
    const float s = __int_as_float((127 - ex) << 23);          // 2^-e
    const int per = K / 8;
    for (int c = lane; c < per; c += 32) {
        const float4 a = reinterpret_cast<const float4*>(x)[2 * c];
        const float4 b = reinterpret_cast<const float4*>(x)[2 * c + 1];
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
        reinterpret_cast<uint4*>(hi)[w * per + c] = make_uint4(h[0], h[1], h[2], h[3]);
        reinterpret_cast<uint4*>(lo)[w * per + c] = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

cudaError_t launch_query_prep(const float* X, int64_t M, int K, int32_t* e, float* sqn, __half* hi, __half* lo,
                              cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (K % 8 != 0) return cudaErrorInvalidValue;
    count_launch();
    query_prep_kernel<<<(unsigned)ceil_div(M * 32, 256), 256, 0, s>>>(X, M, K, e, sqn, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_split_hilo(const float* X, const int32_t* e, int64_t M, int K, __half* hi, __half* lo,
                              cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    const int64_t n = M * (K / 8);
    count_launch();
    split_hilo_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(X, e, M, K, hi, lo);
    return cudaGetLastError();
}

static bool make_half_map(CUtensorMap* map, const __half* base, int64_t rows, int K, int box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)gemm2::BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_gemm_tma(const __half* Ahi, const __half* Alo, const int32_t* eA, int64_t M, const __half* Bhi,
                            const __half* Blo, const int32_t* eB, int N, int K, float* C, int64_t ldc, int epi,
                            const float* rown, const float* coln, float* gmin, uint32_t* status, cudaStream_t s,
                            __half* Ch) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K % gemm2::BK != 0 || M > 0x7fffffff) return cudaErrorInvalidValue;
    CUtensorMap mAh, mAl, mBh, mBl;
    if (!make_half_map(&mAh, Ahi, M, K, gemm2::BM) || !make_half_map(&mAl, Alo, M, K, gemm2::BM) ||
        !make_half_map(&mBh, Bhi, N, K, gemm2::BN) || !make_half_map(&mBl, Blo, N, K, gemm2::BN))
        return cudaErrorInvalidValue;
    gemm2::Args a;
    a.eA = eA; a.eB = eB; a.C = C; a.ldc = ldc; a.M = M; a.N = N; a.K = K; a.epi = epi;
    a.rown = rown; a.coln = coln; a.gmin = gmin; a.Ch = Ch; a.status = status;
    cudaError_t e = cudaFuncSetAttribute(gemm_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm2::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = ceil_div(M, gemm2::BM) * ceil_div(N, gemm2::BN);
    const int grid = (int)(tiles < sms ? tiles : sms);
    count_launch();
    gemm_tma_kernel<<<grid, gemm2::THREADS, gemm2::SMEM, s>>>(mAh, mAl, mBh, mBl, a);
    return cudaGetLastError();
}

}  // namespace erq
