// Encoder: Algorithm 1 (Quantize) of Section 3.1, one warp per vector.
//
// The algorithm walks the rescaling factor t upward through the critical
// values at which the rounding of t*o' changes, keeps <y_cur, o'> and
// ||y_cur||^2 up to date in O(1) per step and records the state of largest
// cosine <y_cur/||y_cur||, o'>.  With |y_i| = m_i + 1/2 the critical values of
// coordinate i are t = (m+1)/|o'_i|, m = 0 .. 2^(B-1)-2.
//
// GPU formulation (bit-identical to a sequential FP64 walk with a min-heap):
//  * The critical values are processed in windows.  A window is the set of
//    remaining events whose FP32 key RN((m+1)/|o'_i|) is <= a threshold T; RN is
//    monotone, so windows never reorder events of different windows.  T is
//    searched so that a window holds at most W >= D events (a coordinate's
//    events all have distinct keys, so one key value never has more than D).
//  * Inside a window the events are sorted by (key, i) with a warp bitonic
//    network; every run of equal FP32 keys is then re-sorted (one lane per run)
//    by the exact rational comparison (m+1)*|o'_j| vs (m'+1)*|o'_i| (exact FP64
//    products).  Ties of the exact value go to the lower coordinate.
//  * <y_cur, o'> is the FP64 sum of the |o'_i| in that order.  Every |o'_i| is
//    an integer multiple of u = 2^ue (ue one below the lowest mantissa bit of
//    the smallest non-zero |o'_i|), and so is every FP64 partial sum.  When the
//    running sum and all of a window's addends are multiples of 2^g and the
//    window's final sum has at most 53 + g significant bits (in units of u),
//    no addition of the window rounds: its partial sums are the exact int64
//    prefix sums, formed in parallel (chunk sums, warp scan, chunk walk).
//    Windows that fail the test (a few per vector at large B, from very small
//    |o'_i|) and rows whose sums could leave int64 are walked serially in FP64
//    by one lane, rounding at every step.  ||y_cur||^2 is an exact integer
//    multiple of 1/4.
//  * All lanes bound each state's cosine in FP32 and only states within 1e-5
//    of the window's best are re-evaluated with correctly rounded FP64 sqrt and
//    division; the first state of strictly largest cosine wins.
//  * The recorded event (i*, m*) defines the final state: m_i = number of
//    events of coordinate i that precede or equal (i*, m*) in the exact order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"

namespace erq {

namespace {

// event word: the FP32 key in the high half, then the coordinate i (22 bits)
// and the level m (10 bits: m <= 2^(B-1) - 2 = 510 at B = 10)
constexpr int EV_MBITS = 10;
constexpr uint64_t EV_MMASK = (1u << EV_MBITS) - 1, EV_IMASK = (1u << (32 - EV_MBITS)) - 1;
__device__ __forceinline__ int ev_i(uint64_t x) { return (int)((x >> EV_MBITS) & EV_IMASK); }
__device__ __forceinline__ int ev_m(uint64_t x) { return (int)(x & EV_MMASK); }

// CntT: the per-coordinate event counter, one byte up to B = 9 (at most 255
// events), two bytes at B = 10 (511); the narrow form leaves room for more
// warps per block in shared memory.
template <typename CntT>
struct EncSmem {
    float* a;         // [D] |o'_i|
    CntT* cnt;        // [D] events of coordinate i already consumed
    uint64_t* keys;   // [W] (key32 << 32) | (i << EV_MBITS) | m
};

// Exponent of the lowest mantissa bit of a positive FP32 value.
__device__ __forceinline__ int lsb_exp(float a) {
    const uint32_t e = (__float_as_uint(a) >> 23) & 0xffu;
    return e == 0 ? -149 : (int)e - 150;
}
// A positive FP32 value as an integer multiple of 2^ue (ue <= lsb_exp(a), and
// the result below 2^62 by the caller's range check).
__device__ __forceinline__ int64_t units_of(float a, int ue) {
    const uint32_t b = __float_as_uint(a);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint64_t mant = e == 0 ? (b & 0x7fffffu) : ((b & 0x7fffffu) | 0x800000u);
    return (int64_t)(mant << (lsb_exp(a) - ue));
}
__device__ __forceinline__ int64_t warp_excl_scan_i64(int64_t v, int64_t& total) {
    const int lane = threadIdx.x & 31;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// k-th event (0-based) of coordinate i has key RN((k+1) * sc / a), sc = 2^e a
// power of two chosen per row so that every key is a finite normal number
// (the product (k+1)*sc is exact, the division correctly rounded, so keys
// are a monotone function of the exact critical value t = (k+1)/a).
__device__ __forceinline__ float ev_key(int k, float a, float sc) { return __fdiv_rn((float)(k + 1) * sc, a); }

// Number of events of a coordinate with key <= T (a > 0), in [0, M].
__device__ __forceinline__ int events_upto(float T, float a, float sc, float inv_sc, int M) {
    if (!(a > 0.f)) return 0;
    if (T == INFINITY) return M;
    float est = floorf(__fmul_rn(T, a * inv_sc));
    int j = est < 0.f ? 0 : (est > (float)M ? M : (int)est);
    while (j < M && ev_key(j, a, sc) <= T) ++j;
    while (j > 0 && ev_key(j - 1, a, sc) > T) --j;
    return j;
}

// Exact order of events: true if (ia, ma) precedes (ib, mb).
__device__ __forceinline__ bool ev_before(const float* a, int ia, int ma, int ib, int mb) {
    const double lhs = (double)(ma + 1) * (double)a[ib];
    const double rhs = (double)(mb + 1) * (double)a[ia];
    if (lhs != rhs) return lhs < rhs;
    return ia < ib;
}

template <typename CntT>
__device__ int window_count(const EncSmem<CntT>& sm, int D, int M, float T, float sc, float inv_sc) {
    const int lane = threadIdx.x & 31;
    int c = 0;
    for (int i = lane; i < D; i += 32) c += events_upto(T, sm.a[i], sc, inv_sc, M) - (int)sm.cnt[i];
    return warp_sum_int(c);
}

}  // namespace

template <typename CntT>
__global__ void __launch_bounds__(256) encode_kernel(const float* __restrict__ Rrot, int64_t n, int D, int B, int W,
                                                     uint8_t* __restrict__ codes, float* __restrict__ f_add,
                                                     float* __restrict__ f_res, double* __restrict__ stats,
                                                     uint32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const size_t per_warp = (size_t)W * 8 + (size_t)D * (4 + sizeof(CntT)) + 64;
    unsigned char* base = smem_raw + (size_t)warp * ((per_warp + 15) / 16 * 16);
    EncSmem<CntT> sm;
    sm.keys = reinterpret_cast<uint64_t*>(base);
    sm.a = reinterpret_cast<float*>(base + (size_t)W * 8);
    sm.cnt = reinterpret_cast<CntT*>(base + (size_t)W * 8 + (size_t)D * 4);

    const int M = (1 << (B - 1)) - 1;
    const int half = 1 << (B - 1);
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp;
    const int64_t stride_w = (int64_t)gridDim.x * nwarps;

    for (int64_t v = gw; v < n; v += stride_w) {
        const float* r = Rrot + v * D;
        int nz = 0;
        float amax = 0.f;
        for (int i = lane; i < D; i += 32) {
            const float x = r[i];
            sm.a[i] = fabsf(x);
            sm.cnt[i] = 0;
            nz += (x != 0.f);
            amax = fmaxf(amax, fabsf(x));
        }
        nz = warp_sum_int(nz);
        amax = warp_max(amax);
        int e2 = 0;
        frexpf(amax, &e2);                       // amax in [2^(e2-1), 2^e2)
        const float sc = ldexpf(1.f, e2 - 1), inv_sc = ldexpf(1.f, 1 - e2);  // both finite for any FP32 amax
        // keys stay finite when every non-zero magnitude is >= 2^-118 * amax
        // (k + 1 <= 2^9 and sc <= amax bound every key by 2^127)
        bool small = false;
        for (int i = lane; i < D; i += 32) small |= (sm.a[i] > 0.f && sm.a[i] < ldexpf(amax, -118));
        if (__any_sync(0xffffffffu, small)) {
            if (lane == 0) atomicOr(status, kStatusRange);
            continue;
        }
        __syncwarp();
        // sum |o'_i| and ||o'||^2 in ascending i (serial FP64 chains on lanes 0, 1)
        double s = 0.0;
        if (lane == 0) {
            for (int i = 0; i < D; ++i) s = __dadd_rn(s, (double)sm.a[i]);
        } else if (lane == 1) {
            for (int i = 0; i < D; ++i) {
                const double x = (double)r[i];
                s = __fma_rn(x, x, s);
            }
        }
        const double sum_a = __shfl_sync(0xffffffffu, s, 0);
        const double nr2 = __shfl_sync(0xffffffffu, s, 1);

        // initial state: all |y_i| = 1/2
        double ip_run = __dmul_rn(0.5, sum_a);    // exact scaling
        uint32_t n2q_run = D;                      // 4 ||y||^2 <= D (2^B - 1)^2 < 2^32 (B <= 10, D <= 4096)
        // integer units of the running sum: u = 2^ue divides every |o'_i| / 2
        int le = 1 << 30;
        for (int i = lane; i < D; i += 32)
            if (sm.a[i] > 0.f) le = min(le, lsb_exp(sm.a[i]));
        le = __reduce_min_sync(0xffffffffu, le);
        const int ue = le - 1;
        // every partial sum stays below (M + 1) * sum |o'_i|; int64 holds it with margin
        const bool in_range = nz > 0 && ldexp((double)(M + 1) * sum_a, -ue) < 0x1p61;
        int64_t S_int = in_range ? __double2ll_rn(ldexp(ip_run, -ue)) : 0;
        double vmax = __ddiv_rn(ip_run, __dsqrt_rn(0.25 * (double)D));
        double ip_best = ip_run;
        uint32_t n2q_best = D;
        int best_i = -1, best_m = -1;
        int64_t remaining = (int64_t)nz * M;
        float T_prev = 0.f;

        while (remaining > 0) {
            // ---- choose the window threshold T
            float T;
            int cnt;
            if (remaining <= W) {
                T = INFINITY;
                cnt = (int)remaining;
            } else {
                // event rate near T_prev: sum of a_i over unfinished coordinates
                float rate = 0.f;
                for (int i = lane; i < D; i += 32)
                    if ((int)sm.cnt[i] < M) rate += sm.a[i] * inv_sc;
                rate = warp_sum(rate);
                float lo = T_prev, hi = INFINITY;
                int clo = 0, chi = (int)imin64(remaining, 0x7fffffff);
                const float target = 0.75f * (float)W;
                float guess = T_prev + target / fmaxf(rate, 1e-30f);
                T = lo;
                cnt = 0;
                for (int it = 0; it < 64; ++it) {
                    // odd steps bisect the float bit range, so the bracket halves at
                    // least every second step and 64 steps always suffice
                    if ((it & 1) || !(guess > lo && guess < hi)) {
                        // bisection on the float bit pattern (positive floats order as ints)
                        const uint32_t ul = __float_as_uint(lo);
                        const uint32_t uh = (hi == INFINITY) ? 0x7f800000u : __float_as_uint(hi);
                        if (uh <= ul + 1) break;
                        guess = __uint_as_float(ul + (uh - ul) / 2);
                    }
                    const int c = window_count(sm, D, M, guess, sc, inv_sc);
                    if (c <= W && c >= W / 4) { T = guess; cnt = c; clo = -1; break; }
                    if (c > W) { hi = guess; chi = c; }
                    else { lo = guess; clo = c; }
                    // interpolate between the bracket ends towards the target
                    if (hi != INFINITY) {
                        const float f = (target - (float)clo) / fmaxf((float)(chi - clo), 1.f);
                        guess = lo + (hi - lo) * fminf(fmaxf(f, 0.05f), 0.95f);
                    } else {
                        guess = T_prev + (lo - T_prev) * 2.f + 1e-30f;
                    }
                }
                if (clo != -1) {
                    // bracket collapsed: take lo if it makes progress, else hi
                    if (clo > 0) { T = lo; cnt = clo; }
                    else { T = hi; cnt = chi; }
                }
                if (cnt > W || cnt <= 0) {  // cannot happen for valid inputs
                    if (lane == 0) atomicOr(status, kStatusBounds);
                    break;
                }
            }
            // ---- gather the window's events
            int mine = 0;
            for (int i = lane; i < D; i += 32) mine += events_upto(T, sm.a[i], sc, inv_sc, M) - (int)sm.cnt[i];
            int pos = warp_incl_scan(mine) - mine;
            for (int i = lane; i < D; i += 32) {
                const float ai = sm.a[i];
                const int c0 = sm.cnt[i], c1 = events_upto(T, ai, sc, inv_sc, M);
                for (int k = c0; k < c1; ++k) {
                    const uint32_t kb = __float_as_uint(ev_key(k, ai, sc));
                    sm.keys[pos++] = ((uint64_t)kb << 32) | ((uint64_t)i << EV_MBITS) | (uint64_t)k;
                }
                sm.cnt[i] = (CntT)c1;
            }
            int np2 = 32;
            while (np2 < cnt) np2 <<= 1;
            for (int j = cnt + lane; j < np2; j += 32) sm.keys[j] = ~0ull;
            __syncwarp();
            // ---- warp bitonic sort of np2 keys
            for (int size = 2; size <= np2; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int p = lane; p < np2 / 2; p += 32) {
                        const int lo_i = 2 * p - (p & (stride - 1));
                        const int hi_i = lo_i + stride;
                        const bool up = (lo_i & size) == 0;
                        const uint64_t x = sm.keys[lo_i], y = sm.keys[hi_i];
                        if ((x > y) == up) { sm.keys[lo_i] = y; sm.keys[hi_i] = x; }
                    }
                    __syncwarp();
                }
            }
            // ---- exact order inside runs of equal FP32 keys: the lane at a run's
            // first position insertion-sorts the run (runs are disjoint, and the
            // FP32 key of every position is unchanged by sorting inside runs)
            for (int j = lane; j + 1 < cnt; j += 32) {
                const uint32_t kj = (uint32_t)(sm.keys[j] >> 32);
                if ((uint32_t)(sm.keys[j + 1] >> 32) != kj || (j > 0 && (uint32_t)(sm.keys[j - 1] >> 32) == kj))
                    continue;
                int e = j + 2;
                while (e < cnt && (uint32_t)(sm.keys[e] >> 32) == kj) ++e;
                for (int h = j + 1; h < e; ++h) {
                    const uint64_t x = sm.keys[h];
                    const int ix = ev_i(x), mx = ev_m(x);
                    int g = h - 1;
                    while (g >= j) {
                        const uint64_t y = sm.keys[g];
                        const int iy = ev_i(y), my = ev_m(y);
                        if (!ev_before(sm.a, ix, mx, iy, my)) break;
                        sm.keys[g + 1] = y;
                        --g;
                    }
                    sm.keys[g + 1] = x;
                }
            }
            __syncwarp();
            // ---- the window's states: <y, o'> after each event, 4 ||y||^2, and
            // the state of largest cosine (first one on ties)
            const int C = (cnt + 31) >> 5;                     // events per lane (contiguous chunk)
            const int c0 = min(cnt, lane * C), c1 = min(cnt, c0 + C);
            int64_t sumA = 0;
            int sumN = 0, gmin = 64;
            for (int j = c0; j < c1; ++j) {
                const uint64_t x = sm.keys[j];
                sumN += 8 * (ev_m(x) + 1);                  // 4 * ((m + 3/2)^2 - (m + 1/2)^2)
                if (in_range) {
                    const int64_t A = units_of(sm.a[ev_i(x)], ue);
                    sumA += A;
                    gmin = min(gmin, __ffsll(A) - 1);
                }
            }
            int64_t totA;
            const int64_t baseA = warp_excl_scan_i64(sumA, totA);
            const int baseN = warp_incl_scan(sumN) - sumN;
            const int totN = __shfl_sync(0xffffffffu, baseN + sumN, 31);
            bool fast = in_range;
            if (fast) {
                // no addition of the window rounds when the running sum and all
                // addends are multiples of 2^g and the final sum fits in 53 + g bits
                const int g = min(__reduce_min_sync(0xffffffffu, gmin), S_int > 0 ? __ffsll(S_int) - 1 : 64);
                const int64_t Pend = S_int + totA;
                fast = 64 - __clzll(Pend) <= 53 + g;
            }
            double bv = -1.0, bip = 0.0;                        // best cosine and its exact <y, o'>
            int bj = 0x7fffffff;
            uint32_t bn = 0;
            if (fast) {
                const float vmax_u = (float)ldexp(vmax, -ue);  // cosine bounds in units of u (scale-free)
                float lmax = 0.f;
                int64_t P = S_int + baseA;
                uint32_t N = n2q_run + (uint32_t)baseN;
                for (int j = c0; j < c1; ++j) {
                    const uint64_t x = sm.keys[j];
                    P += units_of(sm.a[ev_i(x)], ue);
                    N += 8 * (ev_m(x) + 1);
                    lmax = fmaxf(lmax, (float)P * rsqrtf(0.25f * (float)N));
                }
                const float thr = fmaxf(warp_max(lmax), vmax_u) * (1.0f - 1e-5f);
                P = S_int + baseA;
                N = n2q_run + baseN;
                for (int j = c0; j < c1; ++j) {
                    const uint64_t x = sm.keys[j];
                    P += units_of(sm.a[ev_i(x)], ue);
                    N += 8 * (ev_m(x) + 1);
                    if ((float)P * rsqrtf(0.25f * (float)N) >= thr) {
                        const double ipj = ldexp(__ll2double_rn(P), ue);   // exact: P has <= 53 significant bits
                        const double ve = __ddiv_rn(ipj, __dsqrt_rn(0.25 * (double)N));
                        if (ve > bv) { bv = ve; bip = ipj; bj = j; bn = N; }   // j ascending per lane: first max kept
                    }
                }
            } else if (lane == 0) {
                // serial FP64 walk, every addition rounded (two passes: bound, then exact check)
                float lmax = 0.f;
                double ip = ip_run;
                uint32_t N = n2q_run;
                for (int j = 0; j < cnt; ++j) {
                    const uint64_t x = sm.keys[j];
                    ip = __dadd_rn(ip, (double)sm.a[ev_i(x)]);
                    N += 8 * (ev_m(x) + 1);
                    lmax = fmaxf(lmax, (float)ip * rsqrtf(0.25f * (float)N));
                }
                const float thr = fmaxf(lmax, (float)vmax) * (1.0f - 1e-5f);
                ip = ip_run;
                N = n2q_run;
                for (int j = 0; j < cnt; ++j) {
                    const uint64_t x = sm.keys[j];
                    ip = __dadd_rn(ip, (double)sm.a[ev_i(x)]);
                    N += 8 * (ev_m(x) + 1);
                    if ((float)ip * rsqrtf(0.25f * (float)N) >= thr) {
                        const double ve = __ddiv_rn(ip, __dsqrt_rn(0.25 * (double)N));
                        if (ve > bv) { bv = ve; bip = ip; bj = j; bn = N; }
                    }
                }
                ip_run = ip;   // lane 0 only; broadcast below
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const double oip = __shfl_xor_sync(0xffffffffu, bip, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                const uint32_t on = __shfl_xor_sync(0xffffffffu, bn, o);
                if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bip = oip; bj = oj; bn = on; }
            }
            if (bv > vmax) {
                vmax = bv;
                const uint64_t x = sm.keys[bj];
                best_i = ev_i(x);
                best_m = ev_m(x);
                ip_best = bip;
                n2q_best = bn;
            }
            // advance the running state
            if (fast) {
                S_int += totA;
                ip_run = ldexp(__ll2double_rn(S_int), ue);
            } else {
                ip_run = __shfl_sync(0xffffffffu, ip_run, 0);
                if (in_range) S_int = __double2ll_rn(ldexp(ip_run, -ue));
            }
            n2q_run += totN;
            remaining -= cnt;
            T_prev = T;
            __syncwarp();
        }

        // ---- final state and code
        uint8_t* code = codes + v * D * code_bytes(B);
        const double abest = best_i >= 0 ? (double)sm.a[best_i] : 0.0;
        for (int i = lane; i < D; i += 32) {
            int mi = 0;
            const float ai = sm.a[i];
            if (best_i >= 0 && ai > 0.f) {
                const double rhs = (double)(best_m + 1) * (double)ai;
                auto qual = [&](int m) {  // event (i, m) precedes or equals (best_i, best_m)
                    const double lhs = (double)(m + 1) * abest;
                    return lhs < rhs || (lhs == rhs && i <= best_i);
                };
                double est = floor(rhs / abest);
                int j = est < 0.0 ? 0 : (est > (double)M ? M : (int)est);
                while (j < M && qual(j)) ++j;
                while (j > 0 && !qual(j - 1)) --j;
                mi = j;
            }
            const float x = r[i];
            const int u = x >= 0.f ? half + mi : half - 1 - mi;
            if (B > 8) reinterpret_cast<uint16_t*>(code)[i] = (uint16_t)u;
            else code[i] = (uint8_t)u;
        }
        if (lane == 0) {
            f_add[v] = __double2float_rn(nr2);
            f_res[v] = nr2 > 0.0 ? __double2float_rn(__ddiv_rn(-2.0 * nr2, ip_best)) : 0.f;
            if (stats) {
                stats[2 * v] = ip_best;
                stats[2 * v + 1] = 0.25 * (double)n2q_best;
            }
        }
        __syncwarp();
    }
}

static int enc_window(int D) {
    int W = 512;
    while (W < D) W <<= 1;
    return W;
}

template <typename CntT>
static cudaError_t launch_encode_t(const float* Rrot, int64_t n, int D, int B, uint8_t* codes, float* f_add,
                                   float* f_res, double* stats, uint32_t* status, cudaStream_t s) {
    const int W = enc_window(D);
    const size_t per_warp = ((size_t)W * 8 + (size_t)D * (4 + sizeof(CntT)) + 64 + 15) / 16 * 16;
    int warps = (int)((200 * 1024) / per_warp);
    warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
    const size_t smem = per_warp * warps;
    cudaError_t e = cudaFuncSetAttribute(encode_kernel<CntT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = ceil_div(n, warps);
    const int64_t cap = (int64_t)sms * 4;
    if (blocks > cap) blocks = cap;
    count_launch();
    encode_kernel<CntT><<<(unsigned)blocks, warps * 32, smem, s>>>(Rrot, n, D, B, W, codes, f_add, f_res, stats,
                                                                   status);
    return cudaGetLastError();
}

cudaError_t launch_encode(const float* Rrot, int64_t n, int D, int B, uint8_t* codes, float* f_add, float* f_res,
                          double* stats, uint32_t* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (B <= 9) return launch_encode_t<uint8_t>(Rrot, n, D, B, codes, f_add, f_res, stats, status, s);
    return launch_encode_t<uint16_t>(Rrot, n, D, B, codes, f_add, f_res, stats, status, s);
}

// ---------------------------------------------------------------------------
// g = f_add - f_res * <ybar, c'> per stored row (FP64 accumulation in ascending
// index, one rounding).  With it the estimate of Eq. 3.3 + Eq. (eq:dis to ip)
// against the *global* rotated query q' = P^T q_r becomes
//   est = ||q_r - c||^2 + g + f_res * <ybar, q'>,
// because P^T (q_r - c) = q' - c'.  One warp per row, lane 0 sums serially.
// ---------------------------------------------------------------------------
__global__ void gconst_kernel(const uint8_t* __restrict__ codes, const float* __restrict__ f_add,
                              const float* __restrict__ f_res, const float* __restrict__ Cp,
                              const int32_t* __restrict__ cl_of_row, int64_t n, int D, int B,
                              float* __restrict__ g_out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const float* c = Cp + (int64_t)cl_of_row[w] * D;
    const double off = 0.5 * (double)((1 << B) - 1);
    // lanes form exact products; lane 0 adds them in ascending order
    double acc = 0.0;
    for (int k0 = 0; k0 < D; k0 += 32) {
        const double prod = ((double)load_code(codes, B, w * D + k0 + lane) - off) * (double)c[k0 + lane];  // exact
        for (int j = 0; j < 32; ++j) {
            const double pj = __shfl_sync(0xffffffffu, prod, j);
            if (lane == 0) acc = __dadd_rn(acc, pj);
        }
    }
    if (lane == 0) g_out[w] = __double2float_rn(__dsub_rn((double)f_add[w], __dmul_rn((double)f_res[w], acc)));
}

cudaError_t launch_gconst(const uint8_t* codes, const float* f_add, const float* f_res, const float* Cp,
                          const int32_t* cl_of_row, int64_t n, int D, int B, float* g_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    gconst_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(codes, f_add, f_res, Cp, cl_of_row, n, D, B, g_out);
    return cudaGetLastError();
}

}  // namespace erq
