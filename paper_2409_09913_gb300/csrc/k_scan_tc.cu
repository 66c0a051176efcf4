// Tensor-core code scan (tcgen05, sm_103a): the contraction of Eq. 3.3,
// <2 ybar, q'> for every (query, candidate) pair of a work item, on the
// 5th-generation tensor cores with FP32 accumulation in tensor memory.
//
// Operands of one MMA (kind::f16, M = 128, N = 128, K = 16):
//   A = 128 queries of the item (rotated queries q' in FP16), K-major;
//   B = 128 stored rows of the cluster, codes expanded to 2*ybar_u - (2^B-1),
//       which are odd integers in [-255, 255] and therefore exact in FP16.
// The product is exact up to the FP16 rounding of q' (relative 2^-11 per
// element); accumulation is FP32.  The estimate is then
//   est = ||q_r - c||^2 + g + (f_res / 2) * acc,
// with ||q_r - c||^2 from FP32 and g, f_res the stored per-row factors.
//
// Warp roles (288 threads, one CTA per SM, persistent over work items):
//   warps 0-3  epilogue: tcgen05.ld of 32 accumulator columns per step, an
//              in-register warp transpose so that each query's estimates lie
//              across the warp, warp-wide admission filtering against a per-query
//              threshold and per-query candidate lists in shared memory, compacted
//              by a warp bitonic sort (k' <= 32);
//   warps 4-7  producers: gather FP16 query rows and expand u8 codes into the
//              128B-swizzled K-major layout of a pipeline stage;
//   warp 8     MMA issuer (one elected thread) and TMEM owner.
// Pipeline: 3 stages of (A 16 KB, B 16 KB, raw codes 8 KB) per 64-wide K block; two TMEM
// accumulators of 128 columns so the epilogue of one 128-row block overlaps
// the MMAs of the next.  Every mbarrier wait is bounded: on expiry the kernel
// records ERQ_ETIMEOUT in the status word, stops issuing work, waits (bounded)
// for its MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "erq_search.cuh"
#include "tc_common.cuh"

namespace erq {

namespace tc {

constexpr int QT = 128;          // queries per item (MMA M)
constexpr int NB = 128;          // rows per MMA block (MMA N)
constexpr int KB = 64;           // FP16 elements per K block (one 128-byte swizzle row)
constexpr int STAGES = 3;
constexpr int LOOK = STAGES - 1; // producer lookahead (stages in flight ahead of conversion)
constexpr int KCAP = 32;         // max k' of the tensor-core path
constexpr int KC = 64;           // per-query candidate list capacity (list stride of the output)
constexpr int THREADS = 288;
constexpr int STAGE_A = QT * KB * 2;   // 16 KB
constexpr int STAGE_B = NB * KB * 2;   // 16 KB
constexpr int STAGE_RAW = NB * KB;     // 8 KB of u8 codes (TMA staging)

struct Smem {
    // offsets in bytes from a 1024-aligned base
    static constexpr int a = 0;
    static constexpr int b = a + STAGES * STAGE_A;
    static constexpr int raw = b + STAGES * STAGE_B;               // TMA staging of raw codes
    static constexpr int lists = raw + STAGES * STAGE_RAW;         // [QT][KC] u64 candidate keys
    static constexpr int cnt = lists + QT * KC * 8;                 // [QT] int   list fill
    static constexpr int tau = cnt + QT * 4;                        // [QT] u64   admission threshold
    static constexpr int dqc = tau + QT * 8;                        // [QT] float ||q_r - c||^2
    static constexpr int lidx = dqc + QT * 4;                       // [QT] int64 output list index
    static constexpr int bars = lidx + QT * 8;                      // mbarriers (8 B each)
    static constexpr int nbars = 3 * STAGES + 4 + 1;
    static constexpr int tmem_slot = bars + nbars * 8;
    static constexpr int abort_flag = tmem_slot + 4;
    static constexpr int total = abort_flag + 4 + 1024;             // + alignment slack
};

// 16 u8 codes -> 16 FP16 values 2u - off, exact: 1024 + u is exact in FP16
// (byte u as mantissa of 0x6400), fma(1024 + u, 2, -2048) = 2u is exact, and
// 2u - off is an odd integer of magnitude <= 255 (exact).  off = 2^B - 1 is
// applied separately because -(2048 + off) itself is not representable.
__device__ __forceinline__ void expand16(uint4 u, __half2 two, __half2 m2048, __half2 off2, uint4& lo, uint4& hi) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
    uint32_t o[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t p0 = __byte_perm(w[i], 0x6464u, 0x4140u);   // {b0, 0x64, b1, 0x64}
        const uint32_t p1 = __byte_perm(w[i], 0x6464u, 0x4342u);   // {b2, 0x64, b3, 0x64}
        __half2 h0 = *reinterpret_cast<const __half2*>(&p0);
        __half2 h1 = *reinterpret_cast<const __half2*>(&p1);
        h0 = __hsub2(__hfma2(h0, two, m2048), off2);
        h1 = __hsub2(__hfma2(h1, two, m2048), off2);
        o[2 * i] = *reinterpret_cast<uint32_t*>(&h0);
        o[2 * i + 1] = *reinterpret_cast<uint32_t*>(&h1);
    }
    lo = make_uint4(o[0], o[1], o[2], o[3]);
    hi = make_uint4(o[4], o[5], o[6], o[7]);
}

struct Args {
    const __half* Qh;             // [nq][D] FP16 rotated queries
    const uint8_t* codes;         // [N][D]
    const float* g_const;
    const float* f_res;
    const int64_t* list_off;
    const int64_t* list_ids;
    const int64_t* qlist;
    const int64_t* qoff;
    const int4* items;
    const int64_t* n_items;
    const float* dqc;
    const int32_t* slot_off;
    const int64_t* qbase;
    uint64_t* inter;
    int32_t* inter_cnt;
    uint32_t* status;
    int64_t N;
    int maxp, D, B, kp, RR;
};

}  // namespace tc

using namespace tc;

// 32x32 transpose of a warp's registers (5 butterfly stages, static indices):
// on entry lane t holds row t in v[0..31]; on exit lane l holds column l, i.e.
// v[i] = (old row i)[l].
__device__ __forceinline__ void warp_transpose32(uint32_t (&v)[32], int lane) {
#pragma unroll
    for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool upper = (lane & sft) != 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (i & sft) continue;
            const uint32_t send = upper ? v[i] : v[i ^ sft];
            const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, sft);
            if (upper) v[i] = recv;
            else v[i ^ sft] = recv;
        }
    }
}

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t x, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_u64(uint64_t x, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)x, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(x >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

// Ascending warp bitonic sort of 64 keys held as element e = i*32 + lane in v[i].
__device__ __forceinline__ void warp_sort64(uint64_t (&v)[2], int lane) {
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int e = i * 32 + lane;
                const bool asc = (e & size) == 0 || size == 64;
                if (d == 32) {                     // partner in the other register of this lane
                    if (i == 0) {
                        const uint64_t a = v[0], b = v[1];
                        const bool a_lo = asc;     // e < e ^ 32 here
                        v[0] = (a < b) == a_lo ? a : b;
                        v[1] = (a < b) == a_lo ? b : a;
                    }
                } else {
                    const uint64_t p = shfl_xor_u64(v[i], d);
                    const bool lower = (e & d) == 0;
                    const bool keep_min = lower == asc;
                    v[i] = keep_min ? (p < v[i] ? p : v[i]) : (p > v[i] ? p : v[i]);
                }
            }
        }
    }
}

// Keep the kp smallest keys of one query's list (cnt <= KC entries) in its
// first kp slots, sorted; returns the new admission threshold (the kp-th key).
__device__ __noinline__ uint64_t compact_list(uint64_t* list, int cnt, int kp, int lane) {
    uint64_t v[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int e = i * 32 + lane;
        v[i] = e < cnt ? list[e] : kEmptyKey;
    }
    warp_sort64(v, lane);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int e = i * 32 + lane;
        if (e < kp) list[e] = v[i];
    }
    const int t = kp - 1;
    const uint64_t th = shfl_u64(t >= 32 ? v[1] : v[0], t & 31);
    __syncwarp();
    return th;
}

__global__ void __launch_bounds__(THREADS, 1) scan_tc_kernel(const __grid_constant__ CUtensorMap codes_map, tc::Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Smem::bars);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Smem::tmem_slot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + Smem::abort_flag);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]);
    const uint32_t tfull0 = smem_u32(&bars[2 * STAGES]), tempty0 = smem_u32(&bars[2 * STAGES + 2]);
    const uint32_t done_bar = smem_u32(&bars[2 * STAGES + 4]);
    const uint32_t tma0 = smem_u32(&bars[2 * STAGES + 5]);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = a.D, nkb = D / KB;
    const int64_t nitems = *a.n_items;

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
        for (int s = 0; s < STAGES; ++s) mbar_init(tma0 + 8 * s, 1);
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
        // ------------------------------------------------------------ producers
        // Step t of an item = (128-row block, 64-wide K block).  issue(t): wait
        // until the stage is free, then one thread starts a TMA load of the raw u8
        // codes (128 rows x 64 bytes) into the stage's staging buffer and every
        // thread cp.asyncs its 8 16-byte chunks of FP16 query rows straight into the
        // swizzled A tile (zeros for absent queries).  convert(t), LOOK steps later:
        // wait for the thread's own cp.asyncs and the TMA, expand the codes into the
        // swizzled FP16 B tile, fence the async proxy, and arrive on full[stage].
        const int pt = tid - 128;
        const __half2 two = __floats2half2_rn(2.f, 2.f);
        const __half2 m2048 = __floats2half2_rn(-2048.f, -2048.f);
        const float offv = (float)((1 << a.B) - 1);
        const __half2 off2 = __floats2half2_rn(offv, offv);
        const int achunk = pt & 7, bgrp = pt & 3;
        uint32_t it = 0;                               // global stage counter at the item start
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int4 w = a.items[item];
            const int c = w.x;
            const int64_t qb = a.qoff[c] + (int64_t)w.y * QT;
            const int nqi = (int)imin64(QT, a.qoff[c + 1] - qb);
            const int64_t rb0 = a.list_off[c] + (int64_t)w.z * a.RR;
            const int64_t rb1 = imin64(a.list_off[c + 1], rb0 + a.RR);
            const int nblk = (int)((rb1 - rb0 + NB - 1) / NB);
            const int nsteps = nblk * nkb;
            // query i of the item sits in A row (slot) (i % 4) * 32 + i / 4, so that
            // the active queries spread over all four epilogue warps
            const __half* qsrc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = (pt >> 3) + 16 * i;
                const int qi = (r & 31) * 4 + (r >> 5);
                qsrc[i] = qi < nqi ? a.Qh + (a.qlist[qb + qi] / a.maxp) * D + achunk * 8 : nullptr;
            }
            auto issue = [&](int t) -> bool {
                const uint32_t g = it + t;
                const int s = g % STAGES;
                if (!mbar_wait(empty0 + 8 * s, ((g / STAGES) & 1) ^ 1, abort_flag)) return false;
                const int k0 = (t % nkb) * KB;
                const int64_t r0 = rb0 + (int64_t)(t / nkb) * NB;
                if (pt == 0) {
                    mbar_arrive_expect_tx(tma0 + 8 * s, STAGE_RAW);
                    tma_load_2d(smem_u32(sm + Smem::raw + s * STAGE_RAW), &codes_map, k0, (int)r0, tma0 + 8 * s);
                }
                const uint32_t sa = smem_u32(sm + Smem::a + s * STAGE_A);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = (pt >> 3) + 16 * i;
                    const uint32_t dst = sa + r * 128 + ((achunk ^ (r & 7)) << 4);
                    cp_async16(dst, qsrc[i] ? (const void*)(qsrc[i] + k0) : (const void*)a.Qh, qsrc[i] ? 16u : 0u);
                }
                cp_async_commit();
                return true;
            };
            auto convert = [&](int t, int pending) -> bool {
                const uint32_t g = it + t;
                const int s = g % STAGES;
                // own cp.asyncs of step t done: at most `pending` newer groups may remain
                if (pending >= 3) cp_async_wait<3>();
                else if (pending == 2) cp_async_wait<2>();
                else if (pending == 1) cp_async_wait<1>();
                else cp_async_wait<0>();
                if (!mbar_wait(tma0 + 8 * s, (g / STAGES) & 1, abort_flag)) return false;
                const int nr = (int)imin64(NB, rb1 - (rb0 + (int64_t)(t / nkb) * NB));
                const unsigned char* raw = sm + Smem::raw + s * STAGE_RAW;
                unsigned char* sb = sm + Smem::b + s * STAGE_B;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = (pt >> 2) + 32 * i;
                    uint4 lo, hi;
                    if (r < nr) {
                        const uint4 u = *reinterpret_cast<const uint4*>(raw + r * KB + bgrp * 16);
                        expand16(u, two, m2048, off2, lo, hi);
                    } else {
                        lo = hi = make_uint4(0u, 0u, 0u, 0u);
                    }
                    *reinterpret_cast<uint4*>(sb + r * 128 + (((2 * bgrp) ^ (r & 7)) << 4)) = lo;
                    *reinterpret_cast<uint4*>(sb + r * 128 + (((2 * bgrp + 1) ^ (r & 7)) << 4)) = hi;
                }
                fence_proxy_async();
                mbar_arrive(full0 + 8 * s);
                return true;
            };
            const int pre = nsteps < LOOK ? nsteps : LOOK;
            for (int t = 0; t < pre && ok; ++t) ok = issue(t);
            for (int t = 0; t < nsteps && ok; ++t) {
                if (t + LOOK < nsteps) ok = issue(t + LOOK);
                if (!ok) break;
                const int issued = (t + LOOK < nsteps) ? t + LOOK + 1 : nsteps;
                ok = convert(t, issued - t - 1);
            }
            it += nsteps;
        }
        cp_async_wait<0>();
    } else if (warp == 8) {
        // ------------------------------------------------------------ MMA issuer
        uint32_t it = 0, acc = 0;
        bool ok = true;
        const uint32_t idesc = idesc_f16(QT, NB);
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int4 w = a.items[item];
            const int c = w.x;
            const int64_t rb0 = a.list_off[c] + (int64_t)w.z * a.RR;
            const int64_t rb1 = imin64(a.list_off[c + 1], rb0 + a.RR);
            for (int64_t r0 = rb0; r0 < rb1 && ok; r0 += NB, ++acc) {
                const int buf = acc & 1;
                if (!mbar_wait_warp(tempty0 + 8 * buf, ((acc >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tmem + buf * NB;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait_warp(full0 + 8 * s, (it / STAGES) & 1, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    if (lane == 0) {
                        const uint32_t sa = smem_u32(sm + Smem::a + s * STAGE_A);
                        const uint32_t sb = smem_u32(sm + Smem::b + s * STAGE_B);
#pragma unroll
                        for (int k = 0; k < KB / 16; ++k)
                            mma_f16(dt, sdesc(sa + k * 32), sdesc(sb + k * 32), idesc, (kb | k) != 0);
                        mma_commit(empty0 + 8 * s);            // stage free when these MMAs finish
                        if (kb == nkb - 1) mma_commit(tfull0 + 8 * buf);
                    }
                    __syncwarp();
                }
            }
        }
        // all issued MMAs complete before TMEM is released
        if (lane == 0) mma_commit(done_bar);
        __syncwarp();
        mbar_wait_warp(done_bar, 0, abort_flag);
    } else {
        // ------------------------------------------------------------ epilogue
        // Warp w owns TMEM lanes (query slots) 32w..32w+31.  Per 32-column chunk
        // the accumulator rows are transposed in registers, so lane l holds column
        // l of all 32 slots: the estimates of one query then sit across the warp,
        // are filtered against that query's admission threshold with one ballot,
        // and the survivors are appended to its list; a list that fills is
        // compacted by a warp bitonic sort to its kp smallest keys, which also
        // tightens the threshold.  Each list is a superset of the item's top-kp.
        uint64_t* lists = reinterpret_cast<uint64_t*>(sm + Smem::lists);
        int* s_cnt = reinterpret_cast<int*>(sm + Smem::cnt);
        uint64_t* s_tau = reinterpret_cast<uint64_t*>(sm + Smem::tau);
        float* s_dqc = reinterpret_cast<float*>(sm + Smem::dqc);
        int64_t* s_lidx = reinterpret_cast<int64_t*>(sm + Smem::lidx);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const uint32_t below = (1u << lane) - 1u;
        const int kp = a.kp;
        uint32_t acc = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int4 w = a.items[item];
            const int c = w.x;
            const int64_t qb = a.qoff[c] + (int64_t)w.y * QT;
            const int nqi = (int)imin64(QT, a.qoff[c + 1] - qb);
            const int64_t rb0 = a.list_off[c] + (int64_t)w.z * a.RR;
            const int64_t rb1 = imin64(a.list_off[c + 1], rb0 + a.RR);
            {   // slot setup: slot = warp*32 + lane holds query lane*4 + warp
                const int slot = warp * 32 + lane, qi = lane * 4 + warp;
                s_cnt[slot] = 0;
                s_tau[slot] = kEmptyKey;
                if (qi < nqi) {
                    const int64_t e = a.qlist[qb + qi];
                    s_dqc[slot] = a.dqc[e];
                    s_lidx[slot] = a.qbase[e / a.maxp] + a.slot_off[e] + w.z;
                }
            }
            __syncwarp();
            const int nact = nqi > warp ? (nqi - warp + 3) / 4 : 0;   // active slots of this warp
            for (int64_t r0 = rb0; r0 < rb1; r0 += NB, ++acc) {
                const int nr = (int)imin64(NB, rb1 - r0);
                const int buf = acc & 1;
                if (!mbar_wait_warp(tfull0 + 8 * buf, (acc >> 1) & 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
#pragma unroll 1
                for (int cc = 0; cc < NB; cc += 32) {
                    uint32_t v[32];
                    ERQ_TMEM_LD32(tmem + lane_base + buf * NB + cc, v);
                    const int col = cc + lane;
                    const bool valid = col < nr;
                    float mg = 0.f, mf = 0.f;
                    uint32_t mid = 0;
                    if (valid) {
                        mg = a.g_const[r0 + col];
                        mf = 0.5f * a.f_res[r0 + col];
                        mid = (uint32_t)a.list_ids[r0 + col];
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (nact == 0 || cc >= nr) continue;
                    warp_transpose32(v, lane);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i >= nact) break;                       // warp-uniform
                        const int slot = warp * 32 + i;
                        const float est = s_dqc[slot] + mg + mf * __uint_as_float(v[i]);
                        const uint64_t key = make_key(est, mid);
                        const bool pass = valid && key < s_tau[slot];
                        const uint32_t m = __ballot_sync(0xffffffffu, pass);
                        if (m == 0u) continue;
                        int cnt = s_cnt[slot];
                        if (pass) lists[slot * KC + cnt + __popc(m & below)] = key;
                        cnt += __popc(m);
                        __syncwarp();
                        if (cnt > KC - 32) {
                            const uint64_t th = compact_list(lists + slot * KC, cnt, kp, lane);
                            cnt = kp;
                            if (lane == 0) s_tau[slot] = th;
                        }
                        if (lane == 0) s_cnt[slot] = cnt;
                        __syncwarp();
                    }
                }
                tc_fence_before();
                mbar_arrive(tempty0 + 8 * buf);
            }
            if (ok) {
                for (int i = 0; i < nact; ++i) {                     // write this warp's lists
                    const int slot = warp * 32 + i;
                    const int cnt = s_cnt[slot];
                    const int64_t L = s_lidx[slot];
                    uint64_t* dst = a.inter + L * KC;
                    for (int e = lane; e < cnt; e += 32) dst[e] = lists[slot * KC + e];
                    if (lane == 0) a.inter_cnt[L] = cnt;
                }
            }
            __syncwarp();
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

bool tc_available(int precision, int D, int kp) {
    return precision == ERQ_PREC_FP16 && D % KB == 0 && kp <= KCAP;
}

// Capacity (stride) of the per-(query, item) candidate lists written by the scan.
int scan_list_stride(int precision, int kp) { return precision == ERQ_PREC_FP32 ? kp : KC; }

cudaError_t launch_to_half(const float* x, __half* y, int64_t n, cudaStream_t s);

static bool make_codes_map(CUtensorMap* map, const uint8_t* codes, int64_t N, int D) {
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
    const cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)D};          // bytes between rows
    const cuuint32_t box[2] = {(cuuint32_t)KB, (cuuint32_t)NB};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)codes, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

erq_status scan_tc(const ScanLaunch& L, int precision, cudaStream_t s) {
    if (!tc_available(precision, L.D, L.kp))
        return fail(ERQ_EUNSUPPORTED, "tensor-core scan: needs precision fp16 and k' <= 32");
    if (!L.Qh) return fail(ERQ_EINVAL, "tensor-core scan: FP16 queries missing");
    tc::Args a;
    a.Qh = (const __half*)L.Qh; a.codes = L.codes; a.g_const = L.g_const; a.f_res = L.f_res; a.list_off = L.list_off;
    a.list_ids = L.list_ids; a.qlist = L.qlist; a.qoff = L.qoff; a.items = L.items; a.n_items = L.n_items;
    a.dqc = L.dqc; a.slot_off = L.slot_off; a.qbase = L.qbase; a.inter = L.inter; a.inter_cnt = L.inter_cnt;
    a.status = L.status; a.N = L.N; a.maxp = L.maxp; a.D = L.D; a.B = L.B; a.kp = L.kp; a.RR = L.RR;
    const int smem = Smem::total;
    cudaError_t e = cudaFuncSetAttribute(scan_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "scan_tc smem attribute");
    if (L.grid <= 0) return ERQ_OK;
    CUtensorMap map;
    if (((uintptr_t)L.codes & 15) != 0 || (L.D % 16) != 0 || !make_codes_map(&map, L.codes, L.N, L.D))
        return fail(ERQ_ECUDA, "tensor-core scan: cuTensorMapEncodeTiled failed for the code array");
    count_launch();
    scan_tc_kernel<<<L.grid, THREADS, smem, s>>>(map, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scan_tc launch");
    return ERQ_OK;
}

// FP32 -> FP16 (round to nearest) of the rotated queries.
__global__ void to_half_kernel(const float* __restrict__ x, __half* __restrict__ y, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t * 4 >= n) return;
    const float4 v = reinterpret_cast<const float4*>(x)[t];
    __half2* o = reinterpret_cast<__half2*>(y) + 2 * t;
    o[0] = __floats2half2_rn(v.x, v.y);
    o[1] = __floats2half2_rn(v.z, v.w);
}

cudaError_t launch_to_half(const float* x, __half* y, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    to_half_kernel<<<(unsigned)ceil_div(n / 4, 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

}  // namespace erq
