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
//   warps 0-3  epilogue: TMEM lane = query; tcgen05.ld of the accumulator row,
//              estimator, and a per-query max-heap of the k' best (estimate, id)
//              keys in shared memory (k' <= 64);
//   warps 4-7  producers: gather FP16 query rows and expand u8 codes into the
//              128B-swizzled K-major layout of a pipeline stage;
//   warp 8     MMA issuer (one elected thread) and TMEM owner.
// Pipeline: 4 stages of (A 16 KB, B 16 KB) per 64-wide K block; two TMEM
// accumulators of 128 columns so the epilogue of one 128-row block overlaps
// the MMAs of the next.  Every mbarrier wait is bounded: on expiry the kernel
// records ERQ_ETIMEOUT in the status word, stops issuing work, waits (bounded)
// for its MMAs, frees TMEM and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "erq_search.cuh"

namespace erq {

namespace tc {

constexpr int QT = 128;          // queries per item (MMA M)
constexpr int NB = 128;          // rows per MMA block (MMA N)
constexpr int KB = 64;           // FP16 elements per K block (one 128-byte swizzle row)
constexpr int STAGES = 4;
constexpr int KCAP = 64;         // max k' of the in-shared-memory heaps
constexpr int THREADS = 288;
constexpr int STAGE_A = QT * KB * 2;   // 16 KB
constexpr int STAGE_B = NB * KB * 2;   // 16 KB
constexpr uint64_t kWaitNs = 2000000000ull;   // a bounded wait gives up after 2 s

struct Smem {
    // offsets in bytes from a 1024-aligned base
    static constexpr int a = 0;
    static constexpr int b = a + STAGES * STAGE_A;
    static constexpr int heap = b + STAGES * STAGE_B;              // [KCAP][QT] u64
    static constexpr int bars = heap + KCAP * QT * 8;               // mbarriers (8 B each)
    static constexpr int nbars = 2 * STAGES + 4 + 1;
    static constexpr int tmem_slot = bars + nbars * 8;
    static constexpr int abort_flag = tmem_slot + 4;
    static constexpr int total = abort_flag + 4 + 1024;             // + alignment slack
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait; returns false (and raises the abort flag) when 2 s pass or
// another role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (now_ns() - t0 > kWaitNs) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3fff);        // start address
    d |= (uint64_t)1 << 16;                        // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;              // SBO
    d |= (uint64_t)1 << 46;                        // version
    d |= (uint64_t)2 << 61;                        // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

#define ERQ_TMEM_LD32(taddr, r)                                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"  \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                         \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),          \
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),      \
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),   \
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),   \
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                           \
                 : "r"(taddr))

// 16 u8 codes -> 16 FP16 values 2u - off, exact (1024 + u is exact in FP16).
__device__ __forceinline__ void expand16(uint4 u, __half2 m2, __half2 off2, uint4& lo, uint4& hi) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
    uint32_t o[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t p0 = __byte_perm(w[i], 0x6464u, 0x4140u);   // {b0, 0x64, b1, 0x64}
        const uint32_t p1 = __byte_perm(w[i], 0x6464u, 0x4342u);   // {b2, 0x64, b3, 0x64}
        __half2 h0 = *reinterpret_cast<const __half2*>(&p0);
        __half2 h1 = *reinterpret_cast<const __half2*>(&p1);
        h0 = __hfma2(h0, m2, off2);
        h1 = __hfma2(h1, m2, off2);
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

__global__ void __launch_bounds__(THREADS, 1) scan_tc_kernel(tc::Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* heap = reinterpret_cast<uint64_t*>(sm + Smem::heap);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Smem::bars);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Smem::tmem_slot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + Smem::abort_flag);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]);
    const uint32_t tfull0 = smem_u32(&bars[2 * STAGES]), tempty0 = smem_u32(&bars[2 * STAGES + 2]);
    const uint32_t done_bar = smem_u32(&bars[2 * STAGES + 4]);

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
        const int pt = tid - 128;                      // 0..127
        const __half2 m2 = __floats2half2_rn(2.f, 2.f);
        const float offv = -(2048.f + (float)((1 << a.B) - 1));
        const __half2 off2 = __floats2half2_rn(offv, offv);
        uint32_t it = 0;                               // global stage iteration counter
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int4 w = a.items[item];
            const int c = w.x;
            const int64_t qb = a.qoff[c] + (int64_t)w.y * QT;
            const int nqi = (int)imin64(QT, a.qoff[c + 1] - qb);
            const int64_t rb0 = a.list_off[c] + (int64_t)w.z * a.RR;
            const int64_t rb1 = imin64(a.list_off[c + 1], rb0 + a.RR);
            // the 8 A rows this thread copies: rows pt/8 + 16*i, chunk pt%8
            const int achunk = pt & 7;
            int64_t qrow[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = (pt >> 3) + 16 * i;
                qrow[i] = r < nqi ? a.qlist[qb + r] / a.maxp : -1;
            }
            for (int64_t r0 = rb0; r0 < rb1 && ok; r0 += NB) {
                const int nr = (int)imin64(NB, rb1 - r0);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(empty0 + 8 * s, ((it / STAGES) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    unsigned char* sa = sm + Smem::a + s * STAGE_A;
                    unsigned char* sb = sm + Smem::b + s * STAGE_B;
                    const int k0 = kb * KB;
                    // A: 128 rows x 8 chunks of 16 B
                    uint4 av[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        av[i] = qrow[i] >= 0
                                    ? *reinterpret_cast<const uint4*>(a.Qh + qrow[i] * D + k0 + achunk * 8)
                                    : make_uint4(0u, 0u, 0u, 0u);
                    // B: 128 rows x 4 groups of 16 codes; this thread: rows pt/4 + 32*i, group pt%4
                    const int bgrp = pt & 3;
                    uint4 bv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = (pt >> 2) + 32 * i;
                        bv[i] = r < nr ? *reinterpret_cast<const uint4*>(a.codes + (r0 + r) * D + k0 + bgrp * 16)
                                       : make_uint4(0u, 0u, 0u, 0u);
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int r = (pt >> 3) + 16 * i;
                        *reinterpret_cast<uint4*>(sa + r * 128 + ((achunk ^ (r & 7)) << 4)) = av[i];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = (pt >> 2) + 32 * i;
                        uint4 lo, hi;
                        if (r < nr) {
                            expand16(bv[i], m2, off2, lo, hi);
                        } else {
                            lo = hi = make_uint4(0u, 0u, 0u, 0u);
                        }
                        *reinterpret_cast<uint4*>(sb + r * 128 + (((2 * bgrp) ^ (r & 7)) << 4)) = lo;
                        *reinterpret_cast<uint4*>(sb + r * 128 + (((2 * bgrp + 1) ^ (r & 7)) << 4)) = hi;
                    }
                    fence_proxy_async();
                    mbar_arrive(full0 + 8 * s);
                }
            }
        }
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
                if (!mbar_wait(tempty0 + 8 * buf, ((acc >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tmem + buf * NB;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(full0 + 8 * s, (it / STAGES) & 1, abort_flag)) { ok = false; break; }
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
        mbar_wait(done_bar, 0, abort_flag);
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = tid;                             // TMEM lane = query slot
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        uint32_t acc = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int4 w = a.items[item];
            const int c = w.x;
            const int64_t qb = a.qoff[c] + (int64_t)w.y * QT;
            const int nqi = (int)imin64(QT, a.qoff[c + 1] - qb);
            const int64_t rb0 = a.list_off[c] + (int64_t)w.z * a.RR;
            const int64_t rb1 = imin64(a.list_off[c + 1], rb0 + a.RR);
            const bool active = q < nqi;
            float dqc = 0.f;
            int64_t list = 0;
            if (active) {
                const int64_t e = a.qlist[qb + q];
                const int64_t qq = e / a.maxp;
                dqc = a.dqc[e];
                list = a.qbase[qq] + a.slot_off[e] + w.z;
            }
            int hs = 0;
            uint64_t root = kEmptyKey;                  // heap maximum once full
            const int kp = a.kp;
            for (int64_t r0 = rb0; r0 < rb1; r0 += NB, ++acc) {
                const int nr = (int)imin64(NB, rb1 - r0);
                const int buf = acc & 1;
                if (!mbar_wait(tfull0 + 8 * buf, (acc >> 1) & 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
#pragma unroll 1
                for (int cc = 0; cc < NB; cc += 32) {
                    uint32_t r[32];
                    ERQ_TMEM_LD32(tmem + lane_base + buf * NB + cc, r);
                    // row factors of columns cc..cc+31: one coalesced load, then shuffles
                    const int mc = cc + lane;
                    float mg = 0.f, mf = 0.f;
                    uint32_t mid = 0;
                    if (mc < nr) {
                        mg = a.g_const[r0 + mc];
                        mf = 0.5f * a.f_res[r0 + mc];
                        mid = (uint32_t)a.list_ids[r0 + mc];
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const int ncol = nr - cc < 32 ? nr - cc : 32;
#pragma unroll 4
                    for (int j = 0; j < 32; ++j) {
                        const float gj = __shfl_sync(0xffffffffu, mg, j);
                        const float fj = __shfl_sync(0xffffffffu, mf, j);
                        const uint32_t idj = __shfl_sync(0xffffffffu, mid, j);
                        if (!active || j >= ncol) continue;
                        const float est = dqc + gj + fj * __uint_as_float(r[j]);
                        const uint64_t key = make_key(est, idj);
                        if (hs < kp) {
                            int h = hs++;
                            while (h > 0) {
                                const int p = (h - 1) >> 1;
                                const uint64_t pk = heap[p * QT + q];
                                if (pk >= key) break;
                                heap[h * QT + q] = pk;
                                h = p;
                            }
                            heap[h * QT + q] = key;
                            if (hs == kp) root = heap[q];
                        } else if (key < root) {
                            int h = 0;
                            for (;;) {
                                const int l = 2 * h + 1;
                                if (l >= kp) break;
                                int m = l;
                                uint64_t mk = heap[l * QT + q];
                                if (l + 1 < kp) {
                                    const uint64_t rk = heap[(l + 1) * QT + q];
                                    if (rk > mk) { m = l + 1; mk = rk; }
                                }
                                if (mk <= key) break;
                                heap[h * QT + q] = mk;
                                h = m;
                            }
                            heap[h * QT + q] = key;
                            root = heap[q];
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(tempty0 + 8 * buf);
            }
            if (active && ok) {
                uint64_t* dst = a.inter + list * kp;
                for (int j = 0; j < hs; ++j) dst[j] = heap[j * QT + q];
                a.inter_cnt[list] = hs;
            }
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

cudaError_t launch_to_half(const float* x, __half* y, int64_t n, cudaStream_t s);

erq_status scan_tc(const ScanLaunch& L, int precision, cudaStream_t s) {
    if (!tc_available(precision, L.D, L.kp))
        return fail(ERQ_EUNSUPPORTED, "tensor-core scan: needs precision fp16 and k' <= 64");
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
    count_launch();
    scan_tc_kernel<<<L.grid, THREADS, smem, s>>>(a);
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
