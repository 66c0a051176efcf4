// Search path kernels (Section 4.1 IVF search with the Section 3.2 estimator):
//   dqc      ||q_r - c||^2 for every probed (query, cluster) pair
//   plan     invert probe lists into per-cluster query lists and work items
//   scan     estimate every (query, candidate) pair of an item and keep the
//            item's top-k' per query (FP32 CUDA-core path)
//   merge    per query, the k' smallest estimates over all of its items
//   rerank   exact squared distances of the k' candidates, top-k
//   estimate estimates of explicit (query, id) pairs
//   backward gather of sum_j g_j f_res,j ybar_j and sum_j g_j c_j per query
//
// Estimator used by every GPU path (algebraically Eq. 3.3 + Eq. eq:dis to ip):
//   est = ||q_r - c||^2 + g + (f_res / 2) * <2 ybar, q'>,
//   q'  = P^T q_r (rotated once per query),  2 ybar = 2 ybar_u - (2^B - 1),
//   g   = f_add - f_res <ybar, c'>  (per row, index time),
// because P^T (q_r - c) = q' - c' and <ybar_u, x> - (2^B-1)/2 sum x = <ybar, x>.
#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_kernels.cuh"
#include "erq_search.cuh"
#include "warp_sort.cuh"

namespace erq {

// ---------------------------------------------------------------------------
// ||q_r - c||^2 (or, for the inner-product metric, -<q_r, c>) for every probed
// (query, cluster): one block per query, the query row in shared memory, one
// warp per probed cluster (looping when the query probes more clusters than
// the block has warps).  Each lane keeps up to eight 16-byte loads of the
// centroid row in flight (D <= 4096).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) dqc_kernel(const float* __restrict__ Q, const float* __restrict__ C,
                                                  const int32_t* __restrict__ probe, const int32_t* __restrict__ npr,
                                                  int64_t nq, int maxp, int D, int ip, float* __restrict__ dqc) {
    extern __shared__ float qs[];
    const int64_t q = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int np = npr[q];
    // the first centroid row's loads are issued before the query row is waited for
    constexpr int RU = 8;
    int slot = warp;
    float4 a[RU];
    auto issue = [&](int sl) {
        const int c = sl < np ? probe[q * maxp + sl] : -1;
        const float* y = C + (int64_t)(c < 0 ? 0 : c) * D;
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int t = 128 * u + lane * 4;
            if (t < D) a[u] = *reinterpret_cast<const float4*>(y + t);
        }
        return c;
    };
    int c = slot < np ? issue(slot) : -1;
    for (int k = threadIdx.x * 4; k < D; k += blockDim.x * 4)
        *reinterpret_cast<float4*>(qs + k) = *reinterpret_cast<const float4*>(Q + q * D + k);
    __syncthreads();
    for (; slot < np; slot += nw) {
        if (slot != warp) c = issue(slot);
        float s = 0.f;
        for (int t0 = 0; t0 < D; t0 += 128 * RU) {
            if (t0 > 0) {
                const float* y = C + (int64_t)(c < 0 ? 0 : c) * D;
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int t = t0 + 128 * u + lane * 4;
                    if (t < D) a[u] = *reinterpret_cast<const float4*>(y + t);
                }
            }
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int t = t0 + 128 * u + lane * 4;
                if (t < D) {
                    const float4 b = *reinterpret_cast<const float4*>(qs + t);
                    if (ip) {
                        s = fmaf(b.x, a[u].x, s);
                        s = fmaf(b.y, a[u].y, s);
                        s = fmaf(b.z, a[u].z, s);
                        s = fmaf(b.w, a[u].w, s);
                    } else {
                        const float d0 = b.x - a[u].x, d1 = b.y - a[u].y, d2 = b.z - a[u].z, d3 = b.w - a[u].w;
                        s = fmaf(d0, d0, s);
                        s = fmaf(d1, d1, s);
                        s = fmaf(d2, d2, s);
                        s = fmaf(d3, d3, s);
                    }
                }
            }
        }
        s = warp_sum(s);
        // invalid probe ids are reported through the status word
        if (lane == 0 && c >= 0) dqc[q * maxp + slot] = ip ? -s : s;
    }
}

// ---------------------------------------------------------------------------
// Planning.  Effective nprobe per query, validation, pair counts per cluster.
// ---------------------------------------------------------------------------
__global__ void plan_count_kernel(const int32_t* __restrict__ probe, int64_t probe_stride,
                                  const int32_t* __restrict__ npr_in, int npr_uniform, int64_t nq, int maxp,
                                  int nlist, const int64_t* __restrict__ list_off, int RR,
                                  int32_t* __restrict__ npr, int32_t* __restrict__ probe_c,
                                  int32_t* __restrict__ cnt_c, int32_t* __restrict__ touch_c,
                                  int32_t* __restrict__ slot_nr, const float* __restrict__ sqd,
                                  float* __restrict__ dqc, uint32_t* __restrict__ status,
                                  unsigned long long* __restrict__ stats, int two_phase) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long add_pairs = 0, add_rows = 0;
    if (t < nq * maxp) {
        const int64_t q = t / maxp;
        const int slot = (int)(t % maxp);
        int np = npr_in ? npr_in[q] : npr_uniform;
        if (np < 1 || np > maxp) {
            if (slot == 0) atomicOr(status, kStatusBounds);
            np = np < 1 ? 0 : maxp;
        }
        if (slot == 0) npr[q] = np;
        int nr = 0;
        int c = -1;
        if (slot < np) {
            c = probe[q * probe_stride + slot];
            if (c < 0 || c >= nlist) {
                atomicOr(status, kStatusBounds);
                c = -1;
            } else {
                const int64_t size = list_off[c + 1] - list_off[c];
                nr = (int)((size + RR - 1) / RR);
                // queries per (phase, cluster): with two phases, phase 0 holds each
                // query's first (nearest) probed cluster, phase 1 the others (ids nlist + c)
                atomicAdd(&cnt_c[(two_phase && slot > 0) ? nlist + c : c], 1);
                if (atomicAdd(&touch_c[c], 1) == 0) add_rows = (unsigned long long)size;
                add_pairs = (unsigned long long)size;
                if (sqd) dqc[t] = sqd[q * nlist + c];      // the probe's value of this pair
            }
        }
        probe_c[t] = c;
        slot_nr[t] = nr;
    }
    // one atomic per warp for the work counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        add_pairs += __shfl_xor_sync(0xffffffffu, add_pairs, o);
        add_rows += __shfl_xor_sync(0xffffffffu, add_rows, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (add_pairs) atomicAdd(&stats[0], add_pairs);
        if (add_rows) atomicAdd(&stats[1], add_rows);
    }
}

// per query: offsets of its (slot, range) lists, and their total
__global__ void plan_query_kernel(const int32_t* __restrict__ slot_nr, int64_t nq, int maxp,
                                  int32_t* __restrict__ slot_off, int64_t* __restrict__ qtot) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    int run = 0;
    for (int s = 0; s < maxp; ++s) {
        slot_off[q * maxp + s] = run;
        run += slot_nr[q * maxp + s];
    }
    qtot[q] = run;
}

// Exclusive scan of n int64 (out has n + 1 entries, out[n] = total), one
// block of 1024 threads per array (blockIdx.y selects a or b): chunks of
// 4096 values, four consecutive values per thread, warp shuffles then one
// pass over the 32 warp totals.
__global__ void __launch_bounds__(1024) excl_scan_i64_kernel(const int64_t* __restrict__ a, int64_t* __restrict__ out_a,
                                                             const int64_t* __restrict__ b, int64_t* __restrict__ out_b,
                                                             int64_t n) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry_s;
    const int64_t* in = blockIdx.y == 0 ? a : b;
    int64_t* out = blockIdx.y == 0 ? out_a : out_b;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += 4096) {
        const int64_t i0 = base + 4 * t;
        int64_t v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = i0 + j < n ? in[i0 + j] : 0;
        const int64_t own = v[0] + v[1] + v[2] + v[3];
        int64_t inc = own;                      // inclusive warp scan of the per-thread sums
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const int64_t w = wsum[lane];
            int64_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            wsum[lane] = wi - w;                // exclusive prefix of the warp totals
            if (lane == 31) carry_s = wi;       // chunk total
        }
        __syncthreads();
        int64_t run = carry + wsum[warp] + inc - own;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i0 + j < n) out[i0 + j] = run;
            run += v[j];
        }
        carry += carry_s;
        __syncthreads();                        // wsum / carry_s are rewritten by the next chunk
    }
    if (t == 0) out[n] = carry;
}

// Work items may come in two phases (PlanArgs::two_phase): phase 0 pairs every
// query with its first (nearest) probed cluster, phase 1 with the others, so
// that a query's candidate threshold is set by its nearest cluster before its
// other clusters are scanned (at the price of reading a cluster's codes once
// per phase).  Phase cluster ids: v = c (phase 0), nlist + c (phase 1); with
// one phase every pair is in phase 0.
// Rank rk in [0, 2 nlist): phase rk / nlist, clusters by decreasing size (`corder`).
__device__ __forceinline__ int phase_cluster(const int32_t* corder, int nlist, int rk) {
    const int r = rk % nlist;
    return (corder ? corder[r] : r) + (rk >= nlist ? nlist : 0);
}

// per phase cluster: pair count (int64) and, at its rank, its number of work items
__global__ void plan_cluster_kernel(const int32_t* __restrict__ cnt_c, const int64_t* __restrict__ list_off,
                                    const int32_t* __restrict__ corder, int nlist, int QT, int RR,
                                    int64_t* __restrict__ cnt64, int64_t* __restrict__ items_r) {
    const int rk = blockIdx.x * blockDim.x + threadIdx.x;
    if (rk >= 2 * nlist) return;
    const int v = phase_cluster(corder, nlist, rk), c = v % nlist;
    const int64_t size = list_off[c + 1] - list_off[c];
    const int64_t n = cnt_c[v];
    cnt64[v] = n;
    items_r[rk] = (n > 0 && size > 0) ? ((n + QT - 1) / QT) * ((size + RR - 1) / RR) : 0;
}

__global__ void plan_scatter_kernel(const int32_t* __restrict__ probe_c, int64_t nq, int maxp, int nlist, int two_phase,
                                    const int64_t* __restrict__ qoff, int32_t* __restrict__ pos_c,
                                    int64_t* __restrict__ qlist, DevChecks ck) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq * maxp) return;
    const int c = probe_c[t];
    if (c < 0) return;
    const int v = c + ((two_phase && t % maxp != 0) ? nlist : 0);
    const int p = atomicAdd(&pos_c[v], 1);
    if (ERQ_DCHECK(qoff[v] + p >= 0 && qoff[v] + p < ck.qlist, ck.status, 9)) qlist[qoff[v] + p] = t;  // t = q * maxp + slot
}

__global__ void plan_items_kernel(const int64_t* __restrict__ cnt64, const int64_t* __restrict__ list_off,
                                  const int64_t* __restrict__ item_off, const int32_t* __restrict__ corder,
                                  int nlist, int QT, int RR, int4* __restrict__ items, DevChecks ck) {
    const int rk = blockIdx.x * blockDim.x + threadIdx.x;
    if (rk >= 2 * nlist) return;
    const int v = phase_cluster(corder, nlist, rk), c = v % nlist;
    const int64_t b = item_off[rk], e = item_off[rk + 1];
    if (b == e) return;
    const int64_t size = list_off[c + 1] - list_off[c];
    const int nranges = (int)((size + RR - 1) / RR);
    int64_t w = b;
    const int nchunks = (int)((cnt64[v] + QT - 1) / QT);
    if (!ERQ_DCHECK(b >= 0 && e <= ck.items, ck.status, 10)) return;
    for (int r = 0; r < nranges; ++r)
        for (int ch = 0; ch < nchunks; ++ch) items[w++] = make_int4(v, ch, r, 0);
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core scan: Eq. 3.3's <2 ybar - (2^B - 1), q'> by FFMA.
// Item = (cluster c, query chunk, row range).  Tile: 64 queries x 128 rows,
// 128 threads with 8 x 8 outputs each (queries 4 tq .. 4 tq + 3 and 32 + 4 tq
// .. + 3, rows 4 tr .. + 3 and 64 + 4 tr .. + 3: four 16-byte shared loads per
// 64 FFMA; an item of at most 32 queries skips the upper half), K step 32.  The operands of step k + 1 are loaded from global
// memory into registers while step k is multiplied out of the other shared
// buffer (one barrier per step); codes are widened to 2 ybar - (2^B - 1) as
// they are stored.  After a tile the estimates go to shared memory (over the
// operand buffers) and 64 threads (one per query) push those that beat their
// heap's root through the query's max-heap of the k' best (estimate, id) keys.
// ---------------------------------------------------------------------------
constexpr int SC_QT = 64, SC_RB = 128, SC_BK = 32, SC_THREADS = 128;
constexpr int SC_QS = SC_QT + 4, SC_CS = SC_RB + 4;      // padded rows of the transposed operand tiles
constexpr int SC_OPS = 2 * SC_BK * (SC_QS + SC_CS) * 4;  // two buffers of both operands, bytes
constexpr int SC_EST = SC_QT * (SC_RB + 1) * 4;          // estimate tile (aliases the operand buffers)
static_assert(SC_EST <= SC_OPS, "estimate tile fits the operand buffers");

struct ScanArgs {
    const float* Qrot;          // [nq][D]
    const uint8_t* codes;       // [N][D]
    const float* g_const;       // [N]
    const float* f_res;         // [N]
    const int64_t* list_off;    // [nlist+1]
    const int64_t* list_ids;    // [N]
    const int64_t* qlist;       // per-cluster (q*maxp+slot) entries
    const int64_t* qoff;        // [nlist+1]
    const int4* items;
    const int64_t* n_items;     // device scalar
    const float* dqc;           // [nq][maxp]
    const int32_t* slot_off;    // [nq][maxp]
    const int64_t* qbase;       // [nq+1]
    uint64_t* inter;            // [L][kp]
    int32_t* inter_cnt;         // [L]
    int64_t nq, N;              // extents of Qrot and of the stored rows (device-side checks)
    unsigned int* work_ctr;     // items taken after the first grid-size ones (zero at launch)
    int maxp, D, B, kp, RR, nlist;
    int ip;                     // inner-product metric: est = -<c, q_r> + (f_res / 4) <2 ybar, q'>
    DevChecks ck;
};

// Register-staged operands of one K step: 16 query values of query (tid & 63)
// at k0 + 16 (tid >> 6), and the 32 codes of row tid at k0 (CB bytes each:
// 1 for B <= 8, 2 for B = 9).
template <int CB>
struct Fp32Stage {
    float4 q[4];
    uint4 c[2 * CB];
};

template <int CB>
__device__ __forceinline__ void fp32_load(Fp32Stage<CB>& st, const float* qrow, const uint8_t* crow, int k0, int tid) {
    const int kq = (tid >> 6) * 16;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        st.q[j] = qrow ? __ldg(reinterpret_cast<const float4*>(qrow + k0 + kq) + j) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 2 * CB; ++j)
        st.c[j] = crow ? __ldg(reinterpret_cast<const uint4*>(crow + (int64_t)k0 * CB) + j) : make_uint4(0u, 0u, 0u, 0u);
}

template <int CB>
__device__ __forceinline__ void fp32_store(const Fp32Stage<CB>& st, float* qs, float* cs, int tid, float off) {
    const int qi = tid & 63, kq = (tid >> 6) * 16;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        qs[(kq + 4 * j + 0) * SC_QS + qi] = st.q[j].x;
        qs[(kq + 4 * j + 1) * SC_QS + qi] = st.q[j].y;
        qs[(kq + 4 * j + 2) * SC_QS + qi] = st.q[j].z;
        qs[(kq + 4 * j + 3) * SC_QS + qi] = st.q[j].w;
    }
    if constexpr (CB == 1) {
        const uint32_t w[8] = {st.c[0].x, st.c[0].y, st.c[0].z, st.c[0].w, st.c[1].x, st.c[1].y, st.c[1].z, st.c[1].w};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int b = 0; b < 4; ++b) cs[(4 * j + b) * SC_CS + tid] = fmaf(2.f, (float)((w[j] >> (8 * b)) & 0xffu), -off);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t w[4] = {st.c[j].x, st.c[j].y, st.c[j].z, st.c[j].w};
#pragma unroll
            for (int h = 0; h < 4; ++h)
#pragma unroll
                for (int b = 0; b < 2; ++b)
                    cs[(8 * j + 2 * h + b) * SC_CS + tid] = fmaf(2.f, (float)((w[h] >> (16 * b)) & 0xffffu), -off);
        }
    }
}

// The next work item of a block: the first grid-size items go to the blocks
// in order, the rest to whichever block asks first (items come by decreasing
// list size, so this balances the tail).
__device__ __forceinline__ int64_t fp32_next_item(unsigned int* ctr, int64_t* s_next) {
    __syncthreads();                              // every thread has read the previous value
    if (threadIdx.x == 0) *s_next = (int64_t)gridDim.x + atomicAdd(ctr, 1u);
    __syncthreads();
    return *s_next;
}

template <int CB>
__global__ void __launch_bounds__(SC_THREADS) scan_fp32_kernel(ScanArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* ops = reinterpret_cast<float*>(smem);     // buffer b: queries at b * BK * (QS + CS), codes after them
    float (*E)[SC_RB + 1] = reinterpret_cast<float (*)[SC_RB + 1]>(smem);
    uint64_t* heap = reinterpret_cast<uint64_t*>(smem + SC_OPS + 16);                      // [kp][QT]
    __shared__ int64_t s_q[SC_QT];
    __shared__ int64_t s_list[SC_QT];
    __shared__ float s_dqc[SC_QT];
    __shared__ int s_hsize[SC_QT];
    __shared__ float s_g[SC_RB], s_fh[SC_RB];
    __shared__ uint32_t s_id[SC_RB];
    __shared__ int64_t s_next;

    const int tid = threadIdx.x;
    const int tq = tid & 7, tr = tid >> 3;
    const int D = a.D;
    const float off = (float)((1 << a.B) - 1);
    int64_t nitems = *a.n_items;
    if (!ERQ_DCHECK(nitems >= 0 && nitems <= a.ck.items, a.ck.status, 5)) nitems = 0;

    for (int64_t it = blockIdx.x; it < nitems; it = fp32_next_item(a.work_ctr, &s_next)) {
        const int4 item = a.items[it];
        if (!ERQ_DCHECK(item.x >= 0 && item.x < 2 * a.nlist, a.ck.status, 5)) continue;   // block-uniform
        const int v = item.x, c = v % a.nlist;                  // phase cluster -> cluster
        const int64_t qb = a.qoff[v] + (int64_t)item.y * SC_QT;
        const int nqi = (int)imin64(SC_QT, a.qoff[v + 1] - qb);
        const int64_t rb0 = a.list_off[c] + (int64_t)item.z * a.RR;
        const int64_t rb1 = imin64(a.list_off[c + 1], rb0 + a.RR);
        if (tid < SC_QT) {
            s_q[tid] = -1;
            if (tid < nqi && ERQ_DCHECK(qb + tid >= 0 && qb + tid < a.ck.qlist, a.ck.status, 5)) {
                const int64_t e = a.qlist[qb + tid];
                const int64_t q = e / a.maxp;
                if (ERQ_DCHECK(e >= 0 && e < a.ck.qlist && q < a.nq, a.ck.status, 5)) {
                    s_q[tid] = q;
                    s_dqc[tid] = a.dqc[e];
                    s_list[tid] = a.qbase[q] + a.slot_off[e] + item.z;
                }
            }
            s_hsize[tid] = 0;
        }
        __syncthreads();
        const int64_t qsel = s_q[tid & 63];
        const float* qrow = qsel >= 0 ? a.Qrot + qsel * D : nullptr;
        for (int64_t r0 = rb0; r0 < rb1; r0 += SC_RB) {
            const int nr = (int)imin64(SC_RB, rb1 - r0);
            const bool row_ok = tid < nr && ERQ_DCHECK(r0 + tid >= 0 && r0 + tid < a.N, a.ck.status, 5);
            if (row_ok) {
                s_g[tid] = a.ip ? 0.f : a.g_const[r0 + tid];
                s_fh[tid] = (a.ip ? 0.25f : 0.5f) * a.f_res[r0 + tid];
                s_id[tid] = (uint32_t)a.list_ids[r0 + tid];
            }
            const uint8_t* crow = row_ok ? a.codes + (r0 + tid) * D * CB : nullptr;
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            Fp32Stage<CB> st;
            fp32_load(st, qrow, crow, 0, tid);
            fp32_store(st, ops, ops + SC_BK * SC_QS, tid, off);
            __syncthreads();
            int buf = 0;
            for (int k0 = 0; k0 < D; k0 += SC_BK, buf ^= 1) {
                const bool more = k0 + SC_BK < D;
                if (more) fp32_load(st, qrow, crow, k0 + SC_BK, tid);
                const float* qs = ops + buf * SC_BK * (SC_QS + SC_CS);
                const float* cs = qs + SC_BK * SC_QS;
                if (nqi > 32) {
#pragma unroll 4
                    for (int kk = 0; kk < SC_BK; ++kk) {
                        const float4 q0 = *reinterpret_cast<const float4*>(qs + kk * SC_QS + tq * 4);
                        const float4 q1 = *reinterpret_cast<const float4*>(qs + kk * SC_QS + 32 + tq * 4);
                        const float4 c0 = *reinterpret_cast<const float4*>(cs + kk * SC_CS + tr * 4);
                        const float4 c1 = *reinterpret_cast<const float4*>(cs + kk * SC_CS + 64 + tr * 4);
                        const float qa[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                        const float ca[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                        for (int i = 0; i < 8; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(qa[i], ca[j], acc[i][j]);
                    }
                } else {                                   // queries 32..63 are padding: half the FMAs
#pragma unroll 4
                    for (int kk = 0; kk < SC_BK; ++kk) {
                        const float4 q0 = *reinterpret_cast<const float4*>(qs + kk * SC_QS + tq * 4);
                        const float4 c0 = *reinterpret_cast<const float4*>(cs + kk * SC_CS + tr * 4);
                        const float4 c1 = *reinterpret_cast<const float4*>(cs + kk * SC_CS + 64 + tr * 4);
                        const float qa[4] = {q0.x, q0.y, q0.z, q0.w};
                        const float ca[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(qa[i], ca[j], acc[i][j]);
                    }
                }
                if (more) {
                    float* nq = ops + (buf ^ 1) * SC_BK * (SC_QS + SC_CS);
                    fp32_store(st, nq, nq + SC_BK * SC_QS, tid, off);
                }
                __syncthreads();
            }
            // estimates to shared memory (the operand buffers are free: the
            // last step ended with a barrier)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int qi = (i < 4 ? 0 : 32) + tq * 4 + (i & 3), ri = (j < 4 ? 0 : 64) + tr * 4 + (j & 3);
                    float e = INFINITY;
                    if (qi < nqi && ri < nr) e = s_dqc[qi] + s_g[ri] + s_fh[ri] * acc[i][j];
                    E[qi][ri] = e;
                }
            __syncthreads();
            // heap update, one thread per query
            if (tid < nqi && s_q[tid] >= 0) {
                const int q = tid;
                int hs = s_hsize[q];
                const int kp = a.kp;
                uint64_t root = hs > 0 ? heap[q] : 0ull;
                for (int r = 0; r < nr; ++r) {
                    const uint64_t key = make_key(E[q][r], s_id[r]);
                    if (hs < kp) {  // sift up into a max-heap
                        int j = hs++;
                        while (j > 0) {
                            const int p = (j - 1) >> 1;
                            const uint64_t pk = heap[p * SC_QT + q];
                            if (pk >= key) break;
                            heap[j * SC_QT + q] = pk;
                            j = p;
                        }
                        heap[j * SC_QT + q] = key;
                        root = heap[q];
                    } else if (key < root) {  // replace the root, sift down
                        int j = 0;
                        for (;;) {
                            const int l = 2 * j + 1;
                            if (l >= kp) break;
                            int m = l;
                            uint64_t mk = heap[l * SC_QT + q];
                            if (l + 1 < kp) {
                                const uint64_t rk = heap[(l + 1) * SC_QT + q];
                                if (rk > mk) { m = l + 1; mk = rk; }
                            }
                            if (mk <= key) break;
                            heap[j * SC_QT + q] = mk;
                            j = m;
                        }
                        heap[j * SC_QT + q] = key;
                        root = heap[q];
                    }
                }
                s_hsize[q] = hs;
            }
            __syncthreads();
        }
        // write the item's lists
        if (tid < nqi && s_q[tid] >= 0 && ERQ_DCHECK(s_list[tid] >= 0 && s_list[tid] < a.ck.lists, a.ck.status, 4)) {
            const int hs = s_hsize[tid];
            const int64_t L = s_list[tid];
            uint64_t* dst = a.inter + L * a.kp;
            for (int j = 0; j < hs; ++j) dst[j] = heap[j * SC_QT + tid];
            a.inter_cnt[L] = hs;
        }
        __syncthreads();
    }
}

size_t scan_fp32_smem(int kp) { return (size_t)SC_OPS + 16 + (size_t)kp * SC_QT * 8; }

template <int CB>
static int fp32_blocks_per_sm(int kp) {
    int n = 1;
    const size_t smem = scan_fp32_smem(kp);
    if (cudaFuncSetAttribute(scan_fp32_kernel<CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, scan_fp32_kernel<CB>, SC_THREADS, smem) != cudaSuccess ||
        n < 1)
        return 1;
    return n;
}

int scan_fp32_blocks_per_sm(int kp, int B) { return B > 8 ? fp32_blocks_per_sm<2>(kp) : fp32_blocks_per_sm<1>(kp); }

// ---------------------------------------------------------------------------
// Merge: per query the k' smallest keys over its lists, ascending.
// Block of 256 threads; running best k' + a chunk, block bitonic sort.
// ---------------------------------------------------------------------------
__device__ void block_bitonic_u64(uint64_t* v, int n) {
    for (int size = 2; size <= n; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t x = v[lo], y = v[hi];
                if ((x > y) == up) { v[lo] = y; v[hi] = x; }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(256) merge_kernel(const uint64_t* __restrict__ inter,
                                                    const int32_t* __restrict__ inter_cnt,
                                                    const int64_t* __restrict__ qbase, int kp, int lstride,
                                                    int sortn, uint64_t* __restrict__ cand, DevChecks ck) {
    extern __shared__ uint64_t buf[];  // [sortn]
    __shared__ int s_fill;
    __shared__ uint64_t s_tau;         // entries >= s_tau cannot enter the top k'
    const int64_t q = blockIdx.x;
    const int64_t L0 = qbase[q], L1 = qbase[q + 1];
    for (int i = threadIdx.x; i < sortn; i += blockDim.x) buf[i] = kEmptyKey;
    if (threadIdx.x == 0) { s_fill = kp; s_tau = kEmptyKey; }
    __syncthreads();
    for (int64_t L = L0; L < L1; ++L) {
        if (!ERQ_DCHECK(L >= 0 && L < ck.lists, ck.status, 0)) break;
        int n = inter_cnt[L];
        if (!ERQ_DCHECK(n >= 0 && n <= lstride, ck.status, 0)) n = 0;
        if (s_fill + n > sortn) {          // uniform: s_fill is shared
            block_bitonic_u64(buf, sortn);
            for (int i = kp + threadIdx.x; i < sortn; i += blockDim.x) buf[i] = kEmptyKey;
            __syncthreads();
            if (threadIdx.x == 0) { s_fill = kp; s_tau = buf[kp - 1]; }
            __syncthreads();
        }
        const uint64_t tau = s_tau;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const uint64_t key = inter[L * lstride + j];
            if (key < tau) buf[atomicAdd(&s_fill, 1)] = key;
        }
        __syncthreads();
    }
    block_bitonic_u64(buf, sortn);
    for (int j = threadIdx.x; j < kp; j += blockDim.x) cand[q * kp + j] = buf[j];
}

// Merge for k' <= 32: one warp per query keeps the k' smallest keys in a
// sorted 32-entry list across the lanes; each list is read in 32-key chunks,
// and a chunk with a key below the current k'-th is sorted and merged in.
__global__ void __launch_bounds__(256) merge_warp_kernel(const uint64_t* __restrict__ inter,
                                                         const int32_t* __restrict__ inter_cnt,
                                                         const int64_t* __restrict__ qbase, int64_t nq, int kp,
                                                         int lstride, uint64_t* __restrict__ cand, DevChecks ck) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const int64_t L0 = qbase[q], L1 = qbase[q + 1];
    uint64_t list = kEmptyKey, th = kEmptyKey;
    for (int64_t Lb = L0; Lb < L1; Lb += 32) {
        if (!ERQ_DCHECK(Lb >= 0 && L1 <= ck.lists, ck.status, 1)) break;
        const int nl = (int)imin64(32, L1 - Lb);
        int myn = lane < nl ? inter_cnt[Lb + lane] : 0;           // counts of up to 32 lists at once
        if (!ERQ_DCHECK(myn >= 0 && myn <= lstride, ck.status, 1)) myn = 0;
        for (int i = 0; i < nl; ++i) {
            const int n = __shfl_sync(0xffffffffu, myn, i);
            const uint64_t* src = inter + (Lb + i) * lstride;
            for (int c0 = 0; c0 < n; c0 += 32) {
                const uint64_t key = c0 + lane < n ? src[c0 + lane] : kEmptyKey;
                const bool pass = key < th;
                if (!__any_sync(0xffffffffu, pass)) continue;
                list = ws_merge32(list, ws_sort32(pass ? key : kEmptyKey, lane), lane);
                th = ws_shfl(list, kp - 1);
            }
        }
    }
    if (lane < kp) cand[q * kp + lane] = list;
}

// ---------------------------------------------------------------------------
// Re-rank: exact squared distances (or inner products, ranked by -<o, q>) of
// the k' candidates (FP32), top-k; inner products are reported with their sign.
// Also writes cand_ids / cand_est when requested.  One block per query.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rerank_kernel(const uint64_t* __restrict__ cand, int kp, const float* __restrict__ X,
                                                     const float* __restrict__ Q, int D, int k, int do_rerank,
                                                     int ip, int sortn, int64_t* __restrict__ ids,
                                                     float* __restrict__ dists, int64_t* __restrict__ cand_ids,
                                                     float* __restrict__ cand_est, DevChecks ck) {
    const float sgn = ip ? -1.f : 1.f;       // keys hold -<o, q> for the inner-product metric
    extern __shared__ uint64_t keys[];  // [sortn]
    const int64_t q = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t* cq = cand + q * kp;
    if (cand_ids)
        for (int j = threadIdx.x; j < kp; j += blockDim.x) {
            const uint64_t kk = cq[j];
            cand_ids[q * kp + j] = kk == kEmptyKey ? -1 : (int64_t)key_id(kk);
            cand_est[q * kp + j] = sgn * (kk == kEmptyKey ? INFINITY : key_value(kk));
        }
    if (!do_rerank) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            const uint64_t kk = j < kp ? cq[j] : kEmptyKey;
            ids[q * k + j] = kk == kEmptyKey ? -1 : (int64_t)key_id(kk);
            dists[q * k + j] = sgn * (kk == kEmptyKey ? INFINITY : key_value(kk));
        }
        return;
    }
    for (int i = threadIdx.x; i < sortn; i += blockDim.x) keys[i] = kEmptyKey;
    __syncthreads();
    const float* qr = Q + q * D;
    for (int j = warp; j < kp; j += blockDim.x / 32) {
        const uint64_t kk = cq[j];
        if (kk == kEmptyKey) continue;
        const uint32_t id = key_id(kk);
        if (!ERQ_DCHECK((int64_t)id < ck.rows, ck.status, 2)) continue;
        const float* x = X + (int64_t)id * D;
        float s = 0.f;
        constexpr int RU = 8;                 // float4 loads per lane in flight
        for (int t0 = 0; t0 < D; t0 += 128 * RU) {
            float4 a[RU], b[RU];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int t = t0 + 128 * u + lane * 4;
                if (t < D) {
                    a[u] = *reinterpret_cast<const float4*>(x + t);
                    b[u] = *reinterpret_cast<const float4*>(qr + t);
                }
            }
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                if (t0 + 128 * u + lane * 4 < D) {
                    if (ip) {
                        s = fmaf(a[u].x, b[u].x, s);
                        s = fmaf(a[u].y, b[u].y, s);
                        s = fmaf(a[u].z, b[u].z, s);
                        s = fmaf(a[u].w, b[u].w, s);
                    } else {
                        const float d0 = a[u].x - b[u].x, d1 = a[u].y - b[u].y, d2 = a[u].z - b[u].z,
                                    d3 = a[u].w - b[u].w;
                        s = fmaf(d0, d0, s);
                        s = fmaf(d1, d1, s);
                        s = fmaf(d2, d2, s);
                        s = fmaf(d3, d3, s);
                    }
                }
            }
        }
        s = warp_sum(s);
        if (lane == 0) keys[j] = make_key(sgn * s, id);
    }
    __syncthreads();
    block_bitonic_u64(keys, sortn);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const uint64_t kk = keys[j];
        ids[q * k + j] = kk == kEmptyKey ? -1 : (int64_t)key_id(kk);
        dists[q * k + j] = sgn * (kk == kEmptyKey ? INFINITY : key_value(kk));
    }
}

// ---------------------------------------------------------------------------
// Estimates of explicit pairs, one warp per pair (FP32).
// ---------------------------------------------------------------------------
__global__ void estimate_kernel(const float* __restrict__ Q, const float* __restrict__ Qrot,
                                const int64_t* __restrict__ ids, int64_t nq, int nc, int64_t N,
                                const int64_t* __restrict__ row_of, const int32_t* __restrict__ cl_of_row,
                                const float* __restrict__ C, const uint8_t* __restrict__ codes,
                                const float* __restrict__ g_const, const float* __restrict__ f_res, int D, int B,
                                int ipm, float* __restrict__ est, uint32_t* __restrict__ status) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nq * nc) return;
    const int64_t q = w / nc;
    const int64_t id = ids[w];
    if (id < 0 || id >= N) {
        if (lane == 0) {
            est[w] = NAN;
            if (id >= N) atomicOr(status, kStatusBounds);
        }
        return;
    }
    const int64_t row = row_of[id];
    const float* c = C + (int64_t)cl_of_row[row] * D;
    const float* x = Q + q * D;
    const float* xr = Qrot + q * D;
    const float off = (float)((1 << B) - 1);
    float dq = 0.f, ip = 0.f;
    for (int k = lane; k < D; k += 32) {
        if (ipm) {
            dq = fmaf(c[k], x[k], dq);                     // <c, q_r>
        } else {
            const float d = x[k] - c[k];
            dq = fmaf(d, d, dq);
        }
        ip = fmaf(2.f * (float)load_code(codes, B, row * D + k) - off, xr[k], ip);
    }
    dq = warp_sum(dq);
    ip = warp_sum(ip);
    // squared distance ||q_r - c||^2 + g + (f_res/2) <2 ybar, q'>, or inner
    // product <c, q_r> - (f_res/4) <2 ybar, q'>
    if (lane == 0) est[w] = ipm ? dq - 0.25f * f_res[row] * ip : dq + g_const[row] + 0.5f * f_res[row] * ip;
}

// ---------------------------------------------------------------------------
// Backward gather: per query
//   V[q]  = sum_j g_j f_res,j ybar_j          (rotated space)
//   Wv[q] = 2 (G q_r - sum_j g_j c_j),  G = sum_j g_j
// then grad_Q = V P^T + Wv (one SGEMM).  One block per query, coordinates
// strided over threads, candidates in order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) backward_gather_kernel(const float* __restrict__ Q,
                                                              const int64_t* __restrict__ ids,
                                                              const float* __restrict__ gs, int nc, int64_t N,
                                                              const int64_t* __restrict__ row_of,
                                                              const int32_t* __restrict__ cl_of_row,
                                                              const float* __restrict__ C,
                                                              const uint8_t* __restrict__ codes,
                                                              const float* __restrict__ f_res, int D, int B,
                                                              int ipm, float* __restrict__ V, float* __restrict__ Wv,
                                                              uint32_t* __restrict__ status) {
    // squared distance: d est / d q_r = 2 (q_r - c) + f_res P ybar;
    // inner product:    d est / d q_r = c - (f_res / 2) P ybar
    const int64_t q = blockIdx.x;
    const float off = 0.5f * (float)((1 << B) - 1);
    const float fs = ipm ? -0.5f : 1.f;
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        float v = 0.f, wc = 0.f, G = 0.f;
        for (int j = 0; j < nc; ++j) {
            const int64_t id = ids[q * nc + j];
            if (id < 0) continue;
            if (id >= N) {
                if (k == 0) atomicOr(status, kStatusBounds);
                continue;
            }
            const float g = gs[q * nc + j];
            const int64_t row = row_of[id];
            const float yb = (float)load_code(codes, B, row * D + k) - off;
            v = fmaf(g * (fs * f_res[row]), yb, v);
            wc = fmaf(g, C[(int64_t)cl_of_row[row] * D + k], wc);
            G += g;
        }
        V[q * D + k] = v;
        Wv[q * D + k] = ipm ? wc : 2.f * (G * Q[q * D + k] - wc);
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------
cudaError_t launch_dqc(const float* Q, const float* C, const int32_t* probe, const int32_t* npr, int64_t nq, int maxp,
                       int D, int ip, float* dqc, cudaStream_t s) {
    if (nq <= 0 || maxp <= 0) return cudaSuccess;
    const size_t smem = (size_t)D * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(dqc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    dqc_kernel<<<(unsigned)nq, 32 * std::min(maxp, 16), smem, s>>>(Q, C, probe, npr, nq, maxp, D, ip, dqc);
    return cudaGetLastError();
}

cudaError_t launch_plan(const PlanArgs& p, cudaStream_t s) {
    const int64_t pairs = p.nq * p.maxp;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p.cnt_c, 0, sizeof(int32_t) * 2 * p.nlist, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.pos_c, 0, sizeof(int32_t) * 2 * p.nlist, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.touch_c, 0, sizeof(int32_t) * p.nlist, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.stats, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    count_launch();
    plan_count_kernel<<<(unsigned)ceil_div(pairs, 256), 256, 0, s>>>(
        p.probe, p.probe_stride, p.npr_in, p.npr_uniform, p.nq, p.maxp, p.nlist, p.list_off, p.RR, p.npr, p.probe_c,
        p.cnt_c, p.touch_c, p.slot_nr, p.sqd, p.dqc, p.status, p.stats, p.two_phase);
    count_launch();
    plan_query_kernel<<<(unsigned)ceil_div(p.nq, 256), 256, 0, s>>>(p.slot_nr, p.nq, p.maxp, p.slot_off, p.qtot);
    count_launch();
    excl_scan_i64_kernel<<<dim3(1, 1), 1024, 0, s>>>(p.qtot, p.qbase, nullptr, nullptr, p.nq);
    count_launch();
    plan_cluster_kernel<<<(unsigned)ceil_div(2 * p.nlist, 256), 256, 0, s>>>(p.cnt_c, p.list_off, p.corder, p.nlist,
                                                                              p.QT, p.RR, p.cnt64, p.items_c);
    count_launch();
    excl_scan_i64_kernel<<<dim3(1, 2), 1024, 0, s>>>(p.cnt64, p.qoff, p.items_c, p.item_off, 2 * p.nlist);
    count_launch();
    plan_scatter_kernel<<<(unsigned)ceil_div(pairs, 256), 256, 0, s>>>(p.probe_c, p.nq, p.maxp, p.nlist, p.two_phase,
                                                                       p.qoff, p.pos_c, p.qlist, p.ck);
    return cudaGetLastError();
}

cudaError_t launch_excl_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    count_launch();
    excl_scan_i64_kernel<<<dim3(1, 1), 1024, 0, s>>>(in, out, nullptr, nullptr, n);
    return cudaGetLastError();
}

cudaError_t launch_plan_items(const PlanArgs& p, int4* items, cudaStream_t s) {
    count_launch();
    plan_items_kernel<<<(unsigned)ceil_div(2 * p.nlist, 256), 256, 0, s>>>(p.cnt64, p.list_off, p.item_off,
                                                                           p.corder, p.nlist, p.QT, p.RR, items, p.ck);
    return cudaGetLastError();
}

cudaError_t launch_scan_fp32(const ScanLaunch& L, cudaStream_t s) {
    ScanArgs a;
    a.ck = L.ck;
    a.Qrot = L.Qrot; a.codes = L.codes; a.g_const = L.g_const; a.f_res = L.f_res; a.list_off = L.list_off;
    a.list_ids = L.list_ids; a.qlist = L.qlist; a.qoff = L.qoff; a.items = L.items; a.n_items = L.n_items;
    a.dqc = L.dqc; a.slot_off = L.slot_off; a.qbase = L.qbase; a.inter = L.inter; a.inter_cnt = L.inter_cnt;
    a.maxp = L.maxp; a.D = L.D; a.B = L.B; a.kp = L.kp; a.RR = L.RR; a.ip = L.ip; a.nlist = L.nlist;
    a.nq = L.nq; a.N = L.N; a.work_ctr = L.work_ctr;
    if (!a.work_ctr) return cudaErrorInvalidValue;
    const size_t smem = scan_fp32_smem(L.kp);
    const bool wide = L.B > 8;                    // 16-bit codes
    cudaError_t e = wide ? cudaFuncSetAttribute(scan_fp32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                         : cudaFuncSetAttribute(scan_fp32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (L.grid <= 0) return cudaSuccess;
    if (L.D % SC_BK != 0) return cudaErrorInvalidValue;
    count_launch();
    if (wide) scan_fp32_kernel<2><<<L.grid, SC_THREADS, smem, s>>>(a);
    else scan_fp32_kernel<1><<<L.grid, SC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// (id, value) pairs <-> candidate keys, for merging and re-ranking candidate
// lists given by the caller (e.g. the lists of several index shards).
// ---------------------------------------------------------------------------
// Empty key for ids < 0 or >= id_limit (id_limit > 0); the inner-product
// metric ranks by -value.  vals may be null (value 0: re-rank by id only).
__global__ void make_keys_kernel(const int64_t* __restrict__ ids, const float* __restrict__ vals, int64_t n,
                                 int64_t id_limit, int neg, uint64_t* __restrict__ keys) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t id = ids[t];
    const bool empty = id < 0 || id > 0xfffffffell || (id_limit > 0 && id >= id_limit);
    const float v = vals ? (neg ? -vals[t] : vals[t]) : 0.f;
    keys[t] = empty ? kEmptyKey : make_key(v, (uint32_t)id);
}

// Keys -> (id, value): empty keys give -1 and +inf (-inf for the inner-product metric).
__global__ void keys_to_pairs_kernel(const uint64_t* __restrict__ keys, int64_t n, int neg, int64_t* __restrict__ ids,
                                     float* __restrict__ vals) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint64_t k = keys[t];
    const float sgn = neg ? -1.f : 1.f;
    ids[t] = k == kEmptyKey ? -1 : (int64_t)key_id(k);
    vals[t] = sgn * (k == kEmptyKey ? INFINITY : key_value(k));
}

// One list per query: counts[q] = m, offsets[q] = q.
__global__ void one_list_per_query_kernel(int64_t nq, int m, int32_t* __restrict__ counts, int64_t* __restrict__ off) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= nq) off[t] = t;
    if (t < nq) counts[t] = m;
}

cudaError_t launch_make_keys(const int64_t* ids, const float* vals, int64_t n, int64_t id_limit, int neg,
                             uint64_t* keys, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    make_keys_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(ids, vals, n, id_limit, neg, keys);
    return cudaGetLastError();
}

cudaError_t launch_keys_to_pairs(const uint64_t* keys, int64_t n, int neg, int64_t* ids, float* vals, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    keys_to_pairs_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(keys, n, neg, ids, vals);
    return cudaGetLastError();
}

cudaError_t launch_one_list_per_query(int64_t nq, int m, int32_t* counts, int64_t* off, cudaStream_t s) {
    count_launch();
    one_list_per_query_kernel<<<(unsigned)ceil_div(nq + 1, 256), 256, 0, s>>>(nq, m, counts, off);
    return cudaGetLastError();
}

int merge_sortn(int kp, int lstride) {
    int sortn = 128;
    while (sortn < 4 * kp || sortn < kp + lstride + 32) sortn <<= 1;
    return sortn;
}

cudaError_t launch_merge(const uint64_t* inter, const int32_t* inter_cnt, const int64_t* qbase, int64_t nq, int kp,
                         int lstride, uint64_t* cand, const DevChecks& ck, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    if (kp <= 32) {
        count_launch();
        merge_warp_kernel<<<(unsigned)ceil_div(nq * 32, 256), 256, 0, s>>>(inter, inter_cnt, qbase, nq, kp, lstride,
                                                                          cand, ck);
        return cudaGetLastError();
    }
    const int sortn = merge_sortn(kp, lstride);
    cudaError_t e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sortn * 8);
    if (e != cudaSuccess) return e;
    count_launch();
    merge_kernel<<<(unsigned)nq, 256, sortn * 8, s>>>(inter, inter_cnt, qbase, kp, lstride, sortn, cand, ck);
    return cudaGetLastError();
}

// Exact re-rank for k' <= 32: one block of eight warps per query, the query
// row in shared memory; warp w computes ||x - q||^2 for candidates w, w + 8, ...
// with each lane keeping up to eight 16-byte loads of the row in flight (the
// first row's loads are issued before the query row is waited for), then warp
// 0 sorts the k' keys (distance, id) and writes the top k.
__global__ void __launch_bounds__(256, 4) rerank32_kernel(const uint64_t* __restrict__ cand, int kp,
                                                          const float* __restrict__ X, const float* __restrict__ Q,
                                                          int D, int k, int ip, int64_t* __restrict__ ids,
                                                          float* __restrict__ dists, int64_t* __restrict__ cand_ids,
                                                          float* __restrict__ cand_est, DevChecks ck) {
    const float sgn = ip ? -1.f : 1.f;       // keys hold -<o, q> for the inner-product metric
    extern __shared__ float qrow[];           // [D]
    __shared__ uint64_t keys[32];
    const int64_t q = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t* cq = cand + q * kp;
    constexpr int RU = 8;
    float4 a[RU];
    auto issue = [&](int j, int t0) {
        uint64_t kk = cq[j];
        if (kk != kEmptyKey && !ERQ_DCHECK((int64_t)key_id(kk) < ck.rows, ck.status, 3)) kk = kEmptyKey;
        const float* x = X + (int64_t)(kk == kEmptyKey ? 0u : key_id(kk)) * D;
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int t = t0 + 128 * u + lane * 4;
            if (t < D) a[u] = *reinterpret_cast<const float4*>(x + t);
        }
        return kk;
    };
    uint64_t kk = warp < kp ? issue(warp, 0) : kEmptyKey;
    for (int t = threadIdx.x * 4; t < D; t += blockDim.x * 4)
        *reinterpret_cast<float4*>(qrow + t) = *reinterpret_cast<const float4*>(Q + q * D + t);
    if (cand_ids && threadIdx.x < kp) {
        const uint64_t c = cq[threadIdx.x];
        cand_ids[q * kp + threadIdx.x] = c == kEmptyKey ? -1 : (int64_t)key_id(c);
        cand_est[q * kp + threadIdx.x] = sgn * (c == kEmptyKey ? INFINITY : key_value(c));
    }
    __syncthreads();
    for (int j = warp; j < kp; j += 8) {
        if (j != warp) kk = issue(j, 0);
        float s = 0.f;
        for (int t0 = 0; t0 < D; t0 += 128 * RU) {
            if (t0 > 0) issue(j, t0);
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int t = t0 + 128 * u + lane * 4;
                if (t < D) {
                    const float4 b = *reinterpret_cast<const float4*>(qrow + t);
                    if (ip) {
                        s = fmaf(a[u].x, b.x, s);
                        s = fmaf(a[u].y, b.y, s);
                        s = fmaf(a[u].z, b.z, s);
                        s = fmaf(a[u].w, b.w, s);
                    } else {
                        const float d0 = a[u].x - b.x, d1 = a[u].y - b.y, d2 = a[u].z - b.z, d3 = a[u].w - b.w;
                        s = fmaf(d0, d0, s);
                        s = fmaf(d1, d1, s);
                        s = fmaf(d2, d2, s);
                        s = fmaf(d3, d3, s);
                    }
                }
            }
        }
        s = warp_sum(s);
        if (lane == 0) keys[j] = kk == kEmptyKey ? kEmptyKey : make_key(sgn * s, key_id(kk));
    }
    __syncthreads();
    if (warp == 0) {
        const uint64_t v = ws_sort32(lane < kp ? keys[lane] : kEmptyKey, lane);
        if (lane < k) {
            ids[q * k + lane] = v == kEmptyKey ? -1 : (int64_t)key_id(v);
            dists[q * k + lane] = sgn * (v == kEmptyKey ? INFINITY : key_value(v));
        }
    }
}

cudaError_t launch_rerank(const uint64_t* cand, int64_t nq, int kp, const float* X, const float* Q, int D, int k,
                          int do_rerank, int ip, int64_t* ids, float* dists, int64_t* cand_ids, float* cand_est,
                          const DevChecks& ck, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    if (do_rerank && kp <= 32) {
        const size_t smem = (size_t)D * sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(rerank32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        count_launch();
        rerank32_kernel<<<(unsigned)nq, 256, smem, s>>>(cand, kp, X, Q, D, k, ip, ids, dists, cand_ids, cand_est, ck);
        return cudaGetLastError();
    }
    int sortn = 32;
    while (sortn < kp) sortn <<= 1;
    cudaError_t e = cudaFuncSetAttribute(rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sortn * 8);
    if (e != cudaSuccess) return e;
    count_launch();
    rerank_kernel<<<(unsigned)nq, 256, sortn * 8, s>>>(cand, kp, X, Q, D, k, do_rerank, ip, sortn, ids, dists,
                                                       cand_ids, cand_est, ck);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const float* Q, const float* Qrot, const int64_t* ids, int64_t nq, int nc,
                            const erq_index* ix, int ipm, float* est, cudaStream_t s) {
    const int64_t w = nq * nc;
    if (w <= 0) return cudaSuccess;
    count_launch();
    estimate_kernel<<<(unsigned)ceil_div(w * 32, 256), 256, 0, s>>>(Q, Qrot, ids, nq, nc, ix->N, ix->row_of,
                                                                    ix->cl_of_row, ix->C, ix->codes, ix->g_const,
                                                                    ix->f_res, ix->D, ix->B, ipm, est, ix->status);
    return cudaGetLastError();
}

cudaError_t launch_backward_gather(const float* Q, const int64_t* ids, const float* gs, int64_t nq, int nc,
                                   const erq_index* ix, int ipm, float* V, float* Wv, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    count_launch();
    backward_gather_kernel<<<(unsigned)nq, 256, 0, s>>>(Q, ids, gs, nc, ix->N, ix->row_of, ix->cl_of_row, ix->C,
                                                        ix->codes, ix->f_res, ix->D, ix->B, ipm, V, Wv, ix->status);
    return cudaGetLastError();
}

}  // namespace erq
