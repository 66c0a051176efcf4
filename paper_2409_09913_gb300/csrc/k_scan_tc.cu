// Tensor-core code scan (tcgen05, sm_103a): the contraction of Eq. 3.3,
// <2 ybar, q'> for every (query, candidate) pair of a work item, on the
// 5th-generation tensor cores with FP32 accumulation in tensor memory.
//
// A work item is (cluster, up to 64 of the queries that probe it, up to RR
// stored rows).  Operands of one MMA (kind::f16, M = 128, N = npad, K = 16):
//   A = 128 stored rows of the cluster, codes expanded to 2*ybar_u - (2^B-1),
//       odd integers in [-255, 255] and therefore exact in FP16, held in
//       tensor memory (row = lane, two FP16 values per column);
//   B = the item's queries (rotated q' in FP16), npad = the query count rounded
//       up to a multiple of 16, K-major.
// Codes are read from a packed, scan-specific copy: every inverted list padded
// to a multiple of 32 rows and stored as [tiles of 32 rows][K blocks of 64]
// [B words][32 rows] of 8 bytes, i.e. exactly B bits per coordinate (the
// layout is given at unpack_codes); the 128 rows of one stage and K block are
// four contiguous 256*B-byte pieces fetched by one 3-D TMA load.  Tensor
// memory: columns [0, 2 RP QN) hold two buffers of RP accumulators (QN columns
// each), the columns after them the expanded-code stages of RP x 32 columns.
// The accumulator holds row r in TMEM lane r and query j in column j; the
// estimate is est = ||q_r - c||^2 + g + (f_res / 2) * acc with g, f_res the
// stored per-row factors, or for the inner-product metric the ranking score
// -<c, q_r> + (f_res / 4) * acc = -(estimated <o_r, q_r>).  The product is
// exact up to the FP16 rounding of q' (relative 2^-11 per element);
// accumulation is FP32.
//
// Warp roles (27 warps = 864 threads with NG = 2, NFX = 10; one CTA per SM,
// persistent over work items):
//   warp 9     loader: per stage (128-row block, 64-wide K block) one TMA load
//              of the packed codes (L2 evict-first); per row block a bulk copy
//              of the rows' factors and ids; per item the queries'
//              ||q_r - c||^2 and output slots.  It runs up to LS stages ahead
//              of the tensor cores;
//   warps 10.. gatherers (NG warps): per stage, cp.async of the item's FP16 query rows
//              (L2 evict-last) into the 128B-swizzled B tile, completion
//              tracked on the stage's query barrier;
//   warps 4-7, converters, two sets that take alternate stages: one thread
//   and 23-26  per row unpacks the row's 64 B-bit codes of a stage (B 8-byte
//              words; a warp reads 256 contiguous bytes per word, conflict-
//              free) in registers and stores them as FP16 into the stage's
//              TMEM columns (warp w owns TMEM lanes 32 (w % 4) ..);
//   warp 8     MMA issuer of row block 0 (one elected thread) and TMEM owner;
//   warp 22    MMA issuer of row block 1.  Each issuer commits once per
//              stage to the stage's release barrier, which frees its codes,
//              query tile and TMEM code columns together;
//   warps 0-3  estimate tiles: warp w reads TMEM lanes 32w..32w+31 (its 32
//              rows for all queries) and stores g + (f_res/2)*acc into one of
//              EB query-major tiles in shared memory;
//   warps 12-21 filters (NFX warps, pipelined behind the tiles through
//              full/empty barriers): warp f filters the rows of the query
//              slots f + NFX j against per-query thresholds into per-query
//              candidate lists (warp ballots; when a list is full, a warp
//              bitonic sort keeps the k' smallest).  A query's threshold
//              starts at the smallest k'-th key published so far by its items
//              (an item publishes its list's k'-th key with atomicMin after
//              every compaction and at its end), which is never below the
//              query's final k'-th key, so each list stays a superset of what
//              the item contributes to the query's top-k'.
// A stage covers up to RP = 2 row blocks that share the stage's query tile and
// accumulate into separate TMEM accumulators, so two MMA dependency chains are
// in flight and the query gather is amortised over 256 rows.  Accumulators are
// double-buffered per stage group, so the epilogue of one group overlaps the
// MMAs of the next; two estimate tiles let the tile warps fill a block while
// the filter warps still work on the previous one.  Every mbarrier wait is
// bounded: on expiry the kernel records ERQ_ETIMEOUT in the status word, every
// role stops at its next wait (the abort flag), the copies and MMAs already
// issued are drained (bounded), TMEM is freed and the kernel returns.
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

constexpr int MR = 128;          // stored rows per MMA block (MMA M)
static_assert(MR == 128, "four 32-row groups per row block (TMEM lane quarters, filter masks)");
constexpr int KB = 64;           // FP16 elements per K block (one 128-byte swizzle row)
constexpr int MS = 4;            // row-factor buffers (one per row block)
constexpr int NMMA = 2;          // MMA issuing warps
constexpr int KCAP = 128;        // max k' of the tensor-core path
constexpr int NG = 2;            // query-gather warps (10 .. 10 + NG - 1)
constexpr int NFX = 10;          // filter warps (10 + NG ..)
constexpr int NEPI = 4 + NFX;    // epilogue warps: four estimate-tile warps and the filter warps
constexpr int MMA2 = 10 + NG + NFX;   // second MMA issuer (row block 1 of a stage group)
constexpr int NCV = 2;           // converter sets (warps 4-7, and CV2 .. CV2 + 3 when NCV = 2)
constexpr int CV2 = MMA2 + 1;
constexpr int THREADS = 32 * (CV2 + (NCV == 2 ? 4 : 0));
constexpr int TMEM_COLS = 512;     // accumulators 2 x RP x QN columns + LS x RP x 32 columns of codes

// Work-item shapes: QN queries per item (the MMA's N extent), KC-entry
// candidate lists, RP row blocks per stage, LS load stages, EB estimate tiles.
template <int QN_, int KC_, int RP_, int LS_, int EB_>
struct Cfg {
    static constexpr int QN = QN_;                 // queries per item (MMA N <= QN)
    static constexpr int KC = KC_;                 // per-query list capacity (list stride of the output)
    static constexpr int RP = RP_;                 // 128-row blocks per stage (independent accumulators)
    static constexpr int LS = LS_;                 // load stages (raw codes + query tile) in flight
    static constexpr int EB = EB_;                 // estimate tiles (2: filtering overlaps the next block)
    static constexpr int KS = KC_ <= 64 ? 64 : 256;   // sort width of a list compaction
    static constexpr int TILE_Q = QN * KB * 2;
    static constexpr int TILE_RAW = RP * MR * KB;  // packed codes of a stage (TMA staging; 128 * 8 B <= 8 KB per block)
    static constexpr int ACOL = 2 * RP * QN;       // first TMEM column of the expanded-code stages
    static_assert(ACOL + LS * RP * (KB / 2) <= TMEM_COLS, "tensor memory budget");
    static_assert(NCV == 1 || LS % 2 == 0, "the two converter sets take alternate stages and must see every use of theirs");
    static_assert(QN % (4 * NG) == 0 && QN % 32 == 0 && (QN + NFX - 1) / NFX <= 32, "query tile split");
    static_assert(RP >= 1 && RP <= NMMA && (EB == 1 || EB == 2), "stage shape");
    struct Smem {
        // offsets in bytes from a 1024-aligned base
        static constexpr int q = 0;                                // LS  x [QN queries][64] FP16, swizzled
        static constexpr int raw = q + LS * TILE_Q;                // LS  x RP x 8 KB: packed codes of 128 rows
        static constexpr int est = raw + LS * TILE_RAW;            // EB x [QN][MR] f32  g + (f_res/2) acc
        static constexpr int lists = est + EB * QN * MR * 4;       // [QN][KC] u64 candidate keys
        static constexpr int meta = lists + QN * KC * 8;           // MS x [MR] float4 {g, f_res/2, id, 0}
        static constexpr int iq = meta + MS * MR * 16;             // 2 x [QN] int4 {query row, dqc, slot lo, hi}
        static constexpr int idesc = iq + 2 * QN * 16;             // 2 x int4 {rb0 lo, rb0 hi, rows, queries}
        static constexpr int ids = idesc + 2 * 16;                 // EB x [MR] u32 ids of the row block
        static constexpr int cnt = ids + EB * MR * 4;              // [QN] int   list fill
        static constexpr int tau = cnt + QN * 4;                   // [QN] u64   admission threshold
        static constexpr int tq = tau + QN * 8;                    // 2 x [QN] u64 query-wide threshold at item start
        static constexpr int qsc = tq + 2 * QN * 8;                // 2 x [QN] f32 query scales (e4m3 path)
        static constexpr int bars = qsc + 2 * QN * 4;              // mbarriers (8 B each)
        static constexpr int nbars = 4 * LS + 4 + 2 * MS + 4 + 1 + 4;
        static constexpr int tmem_slot = bars + nbars * 8;
        static constexpr int abort_flag = tmem_slot + 4;
        static constexpr int total = abort_flag + 4 + 1024;        // + alignment slack
    };
    static_assert(Smem::total <= 227 * 1024, "scan_tc shared memory");
};
using CfgSmall = Cfg<64, 64, 2, 4, 2>;    // k' <= 32, up to 64 queries per item
using CfgLarge = Cfg<32, 160, 2, 4, 2>;   // k' <= 128, up to 32 queries per item
using CfgWide = Cfg<128, 64, 1, 2, 1>;    // k' <= 32, up to 128 queries per item (query-heavy lists)

// Packed codes of one stored row and one 64-coordinate K block -> 32 TMEM
// columns of FP16 pairs 2u - (2^B - 1) (column c holds coordinates 2c, 2c+1).
// The row's 8B bytes are B 8-byte words; word j of the 32 rows of a tile is a
// contiguous 256-byte run, so `base` points at word 0 of this row and word j
// is at base + 256 j.  With h the 32-bit half index (0..7 over words 0-3) and
// L a byte lane:
//   B >= 4: words 0-3 hold the low four bits of every code as nibbles, byte L
//           of half h = (u[8h + L] & 15) | (u[8h + 4 + L] & 15) << 4, and word
//           b (4 <= b < B) is bit plane b;
//   B < 4:  word b (b < B) is bit plane b;
//   bit plane b: bit 8L + (m & 7) of half (m >> 3) is bit b of u[4m + L].
// Four coordinates 4m..4m+3 are assembled in the byte lanes of one register
// (nibble: one shift and mask; each plane: one shift and one masked OR), as
// 2u for B <= 7 and u for B = 8.  A byte x placed under 0x64 is the FP16
// value 1024 + x (exact); 2u - off = (1024 + 2u) - (1024 + off) is then one
// exact subtraction (for B = 8: 2 (1024 + u) - 2048 - off, each step exact).
template <int B>
__device__ __forceinline__ void unpack_codes(const unsigned char* base, uint32_t (&w)[32]) {
    constexpr int T = B <= 7 ? 1 : 0;
    constexpr int BS = B >= 4 ? 4 : 0;
    uint2 W[B];
#pragma unroll
    for (int j = 0; j < B; ++j) W[j] = *reinterpret_cast<const uint2*>(base + 256 * j);
    const float off = (float)((1 << B) - 1);
    const __half2 c2 = __floats2half2_rn(1024.f + off, 1024.f + off);
    const __half2 off2 = __floats2half2_rn(off, off);
    const __half2 two = __floats2half2_rn(2.f, 2.f);
    const __half2 m2048 = __floats2half2_rn(-2048.f, -2048.f);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        uint32_t V = 0;
        if constexpr (B >= 4) {
            const int h = m >> 1;
            const uint32_t N = (h & 1) ? W[h >> 1].y : W[h >> 1].x;
            if constexpr (T == 1) V = (m & 1) ? (N >> 3) & 0x1E1E1E1Eu : (N << 1) & 0x1E1E1E1Eu;
            else V = (m & 1) ? (N >> 4) & 0x0F0F0F0Fu : N & 0x0F0F0F0Fu;
        }
#pragma unroll
        for (int b = BS; b < B; ++b) {
            const uint32_t P = m < 8 ? W[b].x : W[b].y;
            const int sh = b + T - (m & 7);
            const uint32_t x = sh >= 0 ? P << sh : P >> (-sh);
            V |= x & (0x01010101u << (b + T));
        }
        const uint32_t p0 = __byte_perm(V, 0x6464u, 0x4140u);   // {x0, 0x64, x1, 0x64}
        const uint32_t p1 = __byte_perm(V, 0x6464u, 0x4342u);   // {x2, 0x64, x3, 0x64}
        __half2 h0 = *reinterpret_cast<const __half2*>(&p0);
        __half2 h1 = *reinterpret_cast<const __half2*>(&p1);
        if constexpr (T == 1) {
            h0 = __hsub2(h0, c2);
            h1 = __hsub2(h1, c2);
        } else {
            h0 = __hsub2(__hfma2(h0, two, m2048), off2);
            h1 = __hsub2(__hfma2(h1, two, m2048), off2);
        }
        w[2 * m] = *reinterpret_cast<uint32_t*>(&h0);
        w[2 * m + 1] = *reinterpret_cast<uint32_t*>(&h1);
    }
}

__device__ __forceinline__ void unpack_codes_b(int B, const unsigned char* base, uint32_t (&w)[32]) {
    switch (B) {
        case 1: unpack_codes<1>(base, w); break;
        case 2: unpack_codes<2>(base, w); break;
        case 3: unpack_codes<3>(base, w); break;
        case 4: unpack_codes<4>(base, w); break;
        case 5: unpack_codes<5>(base, w); break;
        case 6: unpack_codes<6>(base, w); break;
        case 7: unpack_codes<7>(base, w); break;
        default: unpack_codes<8>(base, w); break;
    }
}

// Two FP16 values holding odd integers |x| <= 15 (exact in e4m3) -> their
// e4m3 encodings in bytes 0 and 2: the e4m3 exponent is the FP16 one minus 8
// (biases 15 and 7) and the three mantissa bits are the FP16 mantissa's top
// three (the lower seven are zero for these values).
__device__ __forceinline__ uint32_t half2_to_e4m3_pair(uint32_t w) {
    return (((w >> 7) & 0x00FF00FFu) - 0x00400040u) | ((w >> 8) & 0x00800080u);
}

struct Args {
    const unsigned char* Qb;      // [nq] rows of the query operand: FP16 (2D bytes) or e4m3 (qrow_bytes)
    int64_t qrow_bytes;
    const float* qscale;          // e4m3 path: per-query power-of-two scale of the e4m3 values
    const int4* itemd;            // [items] {rb0 lo, rb0 hi, rows, queries}
    const int4* itemq;            // [items][QN] {query row or -1, dqc bits, output list index lo, hi}
    const float4* rowmeta;        // [N] {g, f_res / 2, id bits, 0} in stored-row order
    const int64_t* n_items;
    uint64_t* inter;
    int32_t* inter_cnt;
    unsigned long long* tq;       // [nq] query-wide admission threshold (k'-th key of a finished item)
    uint32_t* status;
    int D, B, kp;
    int ip;                       // inner-product metric: est = -<c, q_r> + (f_res / 4) * acc
    DevChecks ck;
};

__device__ __forceinline__ int npad_of(int nqi) { return nqi <= 16 ? 16 : (nqi + 15) & ~15; }
__device__ __forceinline__ int64_t rb0_of(int4 d) { return (int64_t)(uint32_t)d.x | ((int64_t)d.y << 32); }

}  // namespace tc

using namespace tc;

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

// Ascending warp bitonic sort of N (a power of two >= 64) keys held as element
// e = i*32 + lane in v[i].
template <int N>
__device__ __forceinline__ void warp_sort(uint64_t (&v)[N / 32], int lane) {
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
#pragma unroll
            for (int i = 0; i < N / 32; ++i) {
                const int e = i * 32 + lane;
                const bool asc = (e & size) == 0 || size == N;
                if (d >= 32) {                     // partner in another register of this lane
                    const int j = i ^ (d / 32);
                    if (j > i) {
                        const uint64_t x = v[i], y = v[j];
                        v[i] = (x < y) == asc ? x : y;
                        v[j] = (x < y) == asc ? y : x;
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

// Keep the kp smallest keys of one query's list (cnt <= KS entries) in its
// first kp slots, sorted; returns the new admission threshold (the kp-th key).
template <int KS>
__device__ __noinline__ uint64_t compact_list(uint64_t* list, int cnt, int kp, int lane) {
    uint64_t v[KS / 32];
#pragma unroll
    for (int i = 0; i < KS / 32; ++i) {
        const int e = i * 32 + lane;
        v[i] = e < cnt ? list[e] : kEmptyKey;
    }
    warp_sort<KS>(v, lane);
    uint64_t th = kEmptyKey;
#pragma unroll
    for (int i = 0; i < KS / 32; ++i) {
        const int e = i * 32 + lane;
        if (e < kp) list[e] = v[i];
        const uint64_t t = shfl_u64(v[i], (kp - 1) & 31);
        if (i == (kp - 1) / 32) th = t;
    }
    __syncwarp();
    return th;
}

// F8: queries in e4m3 with a per-query scale, codes in e4m3 (B <= 4),
// tcgen05.mma kind::f8f6f4 (K = 32); a stage then covers 128 coordinates (two
// packed 64-coordinate blocks), which occupy the same 128 bytes per row in
// tensor memory and in the query tile as 64 FP16 coordinates.
template <class C, bool F8>
__global__ void __launch_bounds__(THREADS, 1) scan_tc_kernel(const __grid_constant__ CUtensorMap codes_map, tc::Args a) {
    constexpr int QN = C::QN, KC = C::KC, TILE_Q = C::TILE_Q, ACOL = C::ACOL;
    constexpr int RP = C::RP, LS = C::LS, EB = C::EB, TILE_RAW = C::TILE_RAW;
    using Smem = typename C::Smem;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Smem::bars);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Smem::tmem_slot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + Smem::abort_flag);
    int4* s_iq = reinterpret_cast<int4*>(sm + Smem::iq);
    int4* s_idesc = reinterpret_cast<int4*>(sm + Smem::idesc);
    const float4* s_meta = reinterpret_cast<const float4*>(sm + Smem::meta);
    // barrier addresses
    const uint32_t full_load0 = smem_u32(&bars[0]), empty_load0 = smem_u32(&bars[LS]);
    const uint32_t full_q0 = smem_u32(&bars[2 * LS]);
    const uint32_t full_a0 = smem_u32(&bars[3 * LS]);
    const uint32_t tfull0 = smem_u32(&bars[4 * LS]), tempty0 = smem_u32(&bars[4 * LS + 2]);
    const uint32_t full_meta0 = smem_u32(&bars[4 * LS + 4]);
    const uint32_t empty_meta0 = smem_u32(&bars[4 * LS + 4 + MS]);
    const uint32_t full_item0 = smem_u32(&bars[4 * LS + 4 + 2 * MS]);
    const uint32_t empty_item0 = smem_u32(&bars[4 * LS + 4 + 2 * MS + 2]);
    const uint32_t done_bar = smem_u32(&bars[4 * LS + 4 + 2 * MS + 4]);
    const uint32_t tile_full0 = smem_u32(&bars[4 * LS + 4 + 2 * MS + 5]);
    const uint32_t tile_empty0 = smem_u32(&bars[4 * LS + 4 + 2 * MS + 7]);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = a.D;
    const int nkb = F8 ? (D + 2 * KB - 1) / (2 * KB) : D / KB;   // stages per row group (128 bytes per row)
    int64_t nitems = *a.n_items;
    if (!ERQ_DCHECK(nitems >= 0 && nitems <= a.ck.items, a.ck.status, 7)) nitems = 0;   // uniform: every thread reads it

    if (tid == 0) {
        for (int s = 0; s < LS; ++s) {
            mbar_init(full_load0 + 8 * s, 1);      // the TMA expect_tx arrival
            mbar_init(empty_load0 + 8 * s, NMMA);  // one MMA commit per issuer: codes, queries and TMEM stage free
            mbar_init(full_q0 + 8 * s, 32 * NG);   // one cp.async arrival per gatherer lane
            mbar_init(full_a0 + 8 * s, 128);       // the converter set of the stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, NMMA);
            mbar_init(tempty0 + 8 * b, 128);
            mbar_init(full_item0 + 8 * b, 32);
            mbar_init(empty_item0 + 8 * b, 32 * NEPI);
        }
        for (int m = 0; m < MS; ++m) {
            mbar_init(full_meta0 + 8 * m, 1);
            mbar_init(empty_meta0 + 8 * m, 128);
        }
        mbar_init(done_bar, NMMA);
        for (int t = 0; t < 2; ++t) {
            mbar_init(tile_full0 + 8 * t, 128);        // the four estimate-tile warps
            mbar_init(tile_empty0 + 8 * t, 32 * NFX);  // the filter warps
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 9) {
        // ------------------------------------------------------------ loader
        uint32_t g = 0, rbg = 0, li = 0;
        bool ok = true;
        int64_t item = blockIdx.x;
        int4 dcur = make_int4(0, 0, 0, 0), qv[QN / 32];
#pragma unroll
        for (int j = 0; j < QN / 32; ++j) qv[j] = dcur;
        if (item < nitems) {
            dcur = a.itemd[item];
#pragma unroll
            for (int j = 0; j < QN / 32; ++j) qv[j] = a.itemq[item * QN + 32 * j + lane];
        }
        const uint64_t pol_codes = l2_evict_first();
        for (; item < nitems && ok; item += gridDim.x, ++li) {
            // next item's descriptors are fetched while this one streams
            const int64_t nxt = item + gridDim.x;
            int4 dn = make_int4(0, 0, 0, 0), nv[QN / 32];
#pragma unroll
            for (int j = 0; j < QN / 32; ++j) nv[j] = dn;
            if (nxt < nitems) {
                dn = a.itemd[nxt];
#pragma unroll
                for (int j = 0; j < QN / 32; ++j) nv[j] = a.itemq[nxt * QN + 32 * j + lane];
            }
            const int ib = li & 1;
            if (!mbar_wait_warp(empty_item0 + 8 * ib, ((li >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
            int4* iq = s_iq + ib * QN;
            unsigned long long* tqs = reinterpret_cast<unsigned long long*>(sm + Smem::tq) + ib * QN;
#pragma unroll
            for (int j = 0; j < QN / 32; ++j) {
                iq[32 * j + lane] = qv[j];
                tqs[32 * j + lane] = qv[j].x >= 0 ? __ldcg(a.tq + qv[j].x) : kEmptyKey;
                if (F8) reinterpret_cast<float*>(sm + Smem::qsc)[ib * QN + 32 * j + lane] = qv[j].x >= 0 ? a.qscale[qv[j].x] : 0.f;
            }
            if (lane == 0) s_idesc[ib] = dcur;
            mbar_arrive(full_item0 + 8 * ib);
            __syncwarp();
            const int64_t rb0 = rb0_of(dcur);                 // first padded row (multiple of 32)
            const int nrows = dcur.z;
            for (int r = 0; r < nrows && ok; r += RP * MR) {
                const int nb = min(RP, (nrows - r + MR - 1) / MR);     // 128-row blocks in this stage group
                for (int bb = 0; bb < nb && ok; ++bb, ++rbg) {
                    const int nr = min(MR, nrows - r - bb * MR);
                    const int m = rbg % MS;
                    if (!mbar_wait_warp(empty_meta0 + 8 * m, ((rbg / MS) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    if (lane == 0) {
                        mbar_arrive_expect_tx(full_meta0 + 8 * m, (uint32_t)nr * 16u);
                        bulk_load(smem_u32(sm + Smem::meta + m * MR * 16), a.rowmeta + rb0 + r + bb * MR,
                                  (uint32_t)nr * 16u, full_meta0 + 8 * m);
                    }
                }
                for (int kb = 0; kb < nkb && ok; ++kb, ++g) {
                    const int s = g % LS;
                    if (!mbar_wait_warp(empty_load0 + 8 * s, ((g / LS) & 1) ^ 1, abort_flag)) { ok = false; break; }
                    if (lane == 0) {
                        const uint32_t blk = (uint32_t)(MR / 32) * 256 * a.B;   // one packed block of 128 rows
                        mbar_arrive_expect_tx(full_load0 + 8 * s, (uint32_t)nb * blk * (F8 ? 2u : 1u));
                        for (int bb = 0; bb < nb; ++bb) {
                            const uint32_t dst = smem_u32(sm + Smem::raw + s * TILE_RAW + bb * MR * KB);
                            const int tile = (int)((rb0 + r + bb * MR) >> 5);
                            // (the second block of the last F8 stage may lie past D: the TMA fills zeros)
                            tma_load_3d_hint(dst, &codes_map, 0, F8 ? 2 * kb : kb, tile, full_load0 + 8 * s, pol_codes);
                            if (F8)
                                tma_load_3d_hint(dst + blk, &codes_map, 0, 2 * kb + 1, tile, full_load0 + 8 * s, pol_codes);
                        }
                    }
                    __syncwarp();
                }
            }
            dcur = dn;
#pragma unroll
            for (int j = 0; j < QN / 32; ++j) qv[j] = nv[j];
        }
        // drain: every copy this warp issued has landed before the CTA exits
        for (uint32_t k = 0; k < LS && k < g; ++k) {
            const uint32_t gg = g - 1 - k;
            mbar_wait_drain(full_load0 + 8 * (gg % LS), (gg / LS) & 1);
        }
        for (uint32_t k = 0; k < MS && k < rbg; ++k) {
            const uint32_t gg = rbg - 1 - k;
            mbar_wait_drain(full_meta0 + 8 * (gg % MS), (gg / MS) & 1);
        }
        __syncwarp();
    } else if (warp >= 10 && warp < 10 + NG) {
        // ------------------------------------------------------------ gatherers
        const uint64_t pol_q = l2_evict_last();
        const int ch = lane & 7, gi = warp - 10;
        uint32_t g = 0, li = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(full_item0 + 8 * ib, (li >> 1) & 1, abort_flag)) { ok = false; break; }
            const int4* iq = s_iq + ib * QN;
            const int4 d = s_idesc[ib];
            const int nq4 = npad_of(d.w) / 4;
            const int nsteps = ((d.z + RP * MR - 1) / (RP * MR)) * nkb;
            // this lane gathers 16-byte chunk ch of query rows (lane >> 3) + 4 (gi + NG i)
            const unsigned char* qp[QN / 4 / NG];
#pragma unroll
            for (int i = 0; i < QN / 4 / NG; ++i) {
                const int qrow = iq[(lane >> 3) + 4 * (gi + NG * i)].x;
                qp[i] = qrow >= 0 ? a.Qb + (int64_t)qrow * a.qrow_bytes + ch * 16 : nullptr;
            }
            for (int t = 0; t < nsteps; ++t, ++g) {
                const int s = g % LS, kb = t % nkb;
                if (!mbar_wait_warp(empty_load0 + 8 * s, ((g / LS) & 1) ^ 1, abort_flag)) { ok = false; break; }
                const uint32_t qs = smem_u32(sm + Smem::q + s * TILE_Q);
#pragma unroll
                for (int i = 0; i < QN / 4 / NG; ++i) {
                    if (gi + NG * i < nq4) {
                        const int qq = (lane >> 3) + 4 * (gi + NG * i);
                        const uint32_t dst = qs + qq * 128 + ((ch ^ (qq & 7)) << 4);
                        cp_async16_hint(dst, qp[i] ? (const void*)(qp[i] + kb * 128) : (const void*)a.Qb,
                                        qp[i] ? 16u : 0u, pol_q);
                    }
                }
                cp_async_mbar_arrive(full_q0 + 8 * s);
            }
        }
        cp_async_wait<0>();
        for (uint32_t k = 0; k < LS && k < g; ++k) {
            const uint32_t gg = g - 1 - k;
            mbar_wait_drain(full_q0 + 8 * (gg % LS), (gg / LS) & 1);
        }
        __syncwarp();
    } else if ((warp >= 4 && warp < 8) || warp >= CV2) {
        // ------------------------------------------------------------ converters
        // Two sets of four warps take alternate stages (set cs the stages g
        // with g % 2 == cs).  Converter thread = one row of the stage (TMEM
        // lane); warp w writes TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31.
        const int cs = warp >= CV2 ? 1 : 0;
        const int r = (warp & 3) * 32 + lane;
        const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
        const int B = a.B;
        const int roff = (r >> 5) * 256 * B + (r & 31) * 8;   // word 0 of row r in a 128-row block
        uint32_t g = 0, li = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(full_item0 + 8 * ib, (li >> 1) & 1, abort_flag)) { ok = false; break; }
            const int nrows = s_idesc[ib].z;
            const int nsteps = ((nrows + RP * MR - 1) / (RP * MR)) * nkb;
            for (int t = 0; t < nsteps; ++t, ++g) {
                if (NCV == 2 && (int)(g & 1) != cs) continue;
                const int s = g % LS;
                const int r0 = (t / nkb) * (RP * MR);
                const int nb = min(RP, (nrows - r0 + MR - 1) / MR);
                // the codes have landed; the stage's previous MMAs (which read its
                // TMEM columns) completed before the loader refilled it
                if (!mbar_wait_warp(full_load0 + 8 * s, (g / LS) & 1, abort_flag) ||
                    !mbar_wait_warp(empty_load0 + 8 * s, ((g / LS) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int bb = 0; bb < nb; ++bb) {                  // warp-uniform
                    uint32_t w[32];
                    const unsigned char* src = sm + Smem::raw + s * TILE_RAW + bb * MR * KB + roff;
                    if (F8) {
                        // two packed blocks -> 128 e4m3 codes, four per column
#pragma unroll
                        for (int hb = 0; hb < 2; ++hb) {
                            uint32_t h[32];
                            unpack_codes_b(B, src + hb * (MR / 32) * 256 * B, h);
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                w[16 * hb + c] = __byte_perm(half2_to_e4m3_pair(h[2 * c]),
                                                             half2_to_e4m3_pair(h[2 * c + 1]), 0x6420u);
                        }
                    } else {
                        unpack_codes_b(B, src, w);
                    }
                    ERQ_TMEM_ST32(tmem + lane_addr + ACOL + (s * RP + bb) * (KB / 2), w);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(full_a0 + 8 * s);
            }
        }
    } else if (warp == 8 || warp == MMA2) {
        // ------------------------------------------------------------ MMA issuers
        // Each issuer runs the accumulation chain of one row block of a stage
        // group (tcgen05.mma issue stalls the issuing thread, so two issuers
        // keep two chains in flight); both commit to the stage and tile barriers.
        const int mrb = warp == 8 ? 0 : 1;
        uint32_t g = 0, acc = 0, li = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(full_item0 + 8 * ib, (li >> 1) & 1, abort_flag)) { ok = false; break; }
            const int4 d = s_idesc[ib];
            const uint32_t idesc = idesc_f16(MR, npad_of(d.w));
            for (int r0 = 0; r0 < d.z && ok; r0 += RP * MR, ++acc) {   // acc counts stage groups
                const int nb = min(RP, (d.z - r0 + MR - 1) / MR);
                const int buf = acc & 1;
                if (!mbar_wait_warp(tempty0 + 8 * buf, ((acc >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tmem + buf * (RP * QN);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % LS;
                    if (!mbar_wait_warp(full_a0 + 8 * s, (g / LS) & 1, abort_flag) ||
                        !mbar_wait_warp(full_q0 + 8 * s, (g / LS) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();       // query tile written by cp.async (generic proxy)
                    tc_fence_after();
                    if (lane == 0) {
                        if (mrb < nb) {
                            const uint32_t ta = tmem + ACOL + (s * RP + mrb) * (KB / 2);
                            const uint32_t tq = smem_u32(sm + Smem::q + s * TILE_Q);
#pragma unroll
                            for (int k = 0; k < KB / 16; ++k) {         // 32 bytes of K per instruction
                                if (F8) mma_f8_ta(dt + mrb * QN, ta + k * 8, sdesc(tq + k * 32), idesc, (kb | k) != 0);
                                else mma_f16_ta(dt + mrb * QN, ta + k * 8, sdesc(tq + k * 32), idesc, (kb | k) != 0);
                            }
                        }
                        mma_commit(empty_load0 + 8 * s);     // codes, query tile and TMEM stage free
                        if (kb == nkb - 1) mma_commit(tfull0 + 8 * buf);
                    }
                    __syncwarp();
                }
            }
        }
        // all issued MMAs complete before TMEM is released
        if (lane == 0) mma_commit(done_bar);
        __syncwarp();
        mbar_wait_drain(done_bar, 0);
        __syncwarp();
    } else if (warp < 4) {
        // ------------------------------------------------------------ estimate tiles
        // Warp w moves TMEM lanes 32w..32w+31 (its 32 rows, all queries) of a
        // finished accumulator into a query-major estimate tile.
        float* s_est = reinterpret_cast<float*>(sm + Smem::est);
        uint32_t* s_ids = reinterpret_cast<uint32_t*>(sm + Smem::ids);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const int row = warp * 32 + lane;
        uint32_t blk = 0, pc = 0, rbg = 0, li = 0;     // row blocks, stage groups, meta slots, items
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(full_item0 + 8 * ib, (li >> 1) & 1, abort_flag)) { ok = false; break; }
            const int4 d = s_idesc[ib];
            const int nrows = d.z, npad = npad_of(d.w);
            for (int r = 0; r < nrows; r += MR, ++blk, ++rbg) {
                const int bb = (r / MR) % RP;                   // block within its stage group
                const int nb = min(RP, (nrows - (r - bb * MR) + MR - 1) / MR);
                const int buf = pc & 1, m = rbg % MS, t = blk % EB;
                if (!mbar_wait_warp(full_meta0 + 8 * m, (rbg / MS) & 1, abort_flag) ||
                    (bb == 0 && !mbar_wait_warp(tfull0 + 8 * buf, (pc >> 1) & 1, abort_flag)) ||
                    !mbar_wait_warp(tile_empty0 + 8 * t, ((blk / EB) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                float* est_t = s_est + t * (QN * MR);
                float4 mt = s_meta[m * MR + row];
                s_ids[t * MR + row] = __float_as_uint(mt.z);
                if (a.ip) {                                     // -<c, q_r> + (f_res / 4) acc: no g, half the factor
                    mt.x = 0.f;
                    mt.y *= 0.5f;
                }
#pragma unroll 1
                for (int cc = 0; cc < npad; cc += 32) {
                    uint32_t v[32];
                    ERQ_TMEM_LD32(tmem + lane_base + buf * (RP * QN) + bb * QN + cc, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (F8) {                                  // e4m3 queries carry a power-of-two scale (exact)
                        const float* sc = reinterpret_cast<const float*>(sm + Smem::qsc) + ib * QN + cc;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            est_t[(cc + i) * MR + row] = fmaf(mt.y, __uint_as_float(v[i]) * sc[i], mt.x);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) est_t[(cc + i) * MR + row] = fmaf(mt.y, __uint_as_float(v[i]), mt.x);
                    }
                }
                tc_fence_before();
                if (bb == nb - 1) {                             // the group's accumulators are free
                    mbar_arrive(tempty0 + 8 * buf);
                    ++pc;
                }
                mbar_arrive(empty_meta0 + 8 * m);
                mbar_arrive(tile_full0 + 8 * t);
            }
            if (!ok) break;
            mbar_arrive(empty_item0 + 8 * ib);
        }
    } else {
        // ------------------------------------------------------------ filters
        // NFX warps; warp f owns the query slots q = f + NFX j of every item.
        const float* s_est = reinterpret_cast<const float*>(sm + Smem::est);
        uint64_t* lists = reinterpret_cast<uint64_t*>(sm + Smem::lists);
        const uint32_t* s_ids = reinterpret_cast<const uint32_t*>(sm + Smem::ids);
        int* s_cnt = reinterpret_cast<int*>(sm + Smem::cnt);
        uint64_t* s_tau = reinterpret_cast<uint64_t*>(sm + Smem::tau);
        const int fw = warp - (10 + NG);
        const uint32_t below = (1u << lane) - 1u;
        const int kp = a.kp;
        uint32_t blk = 0, li = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(full_item0 + 8 * ib, (li >> 1) & 1, abort_flag)) { ok = false; break; }
            const int4 d = s_idesc[ib];
            const int nrows = d.z, nqi = d.w;
            const int4* iq = s_iq + ib * QN;
            if (lane < (QN + NFX - 1) / NFX) {
                const int q = fw + NFX * lane;
                if (q < nqi) {
                    s_cnt[q] = 0;
                    s_tau[q] = reinterpret_cast<const unsigned long long*>(sm + Smem::tq)[ib * QN + q];
                }
            }
            __syncwarp();
            for (int r = 0; r < nrows; r += MR, ++blk) {
                const int nr = min(MR, nrows - r);
                const int t = blk % EB;
                if (!mbar_wait_warp(tile_full0 + 8 * t, (blk / EB) & 1, abort_flag)) { ok = false; break; }
                const float* est_t = s_est + t * (QN * MR);
                const uint32_t* ids_t = s_ids + t * MR;
                // the 128 rows of each owned query; the four 32-row groups'
                // estimates are loaded together, compared as floats against
                // the threshold's estimate (a superset of the key test), and
                // only groups with a candidate form exact keys
                for (int q = fw; q < nqi; q += NFX) {
                    const float dq = __int_as_float(iq[q].y);
                    uint64_t tau = s_tau[q];
                    float tf = tau == kEmptyKey ? INFINITY : key_value(tau);
                    int cnt = s_cnt[q];
                    float e[MR / 32];
#pragma unroll
                    for (int j = 0; j < MR / 32; ++j) e[j] = dq + est_t[q * MR + j * 32 + lane];
#pragma unroll
                    for (int j = 0; j < MR / 32; ++j) {
                        const int rr = j * 32 + lane;
                        const bool pre = rr < nr && e[j] <= tf;
                        if (!__any_sync(0xffffffffu, pre)) continue;
                        const uint64_t key = make_key(e[j], ids_t[rr]);
                        bool pass = pre && key < tau;
                        uint32_t msk = __ballot_sync(0xffffffffu, pass);
                        if (msk == 0u) continue;
                        if (cnt + __popc(msk) > KC) {
                            // full: keep the k' smallest (KC - k' >= 32 leaves
                            // room for a group), then test the group again
                            tau = compact_list<C::KS>(lists + q * KC, cnt, kp, lane);
                            tf = key_value(tau);
                            cnt = kp;
                            // k' keys of this query are now <= tau and stay in
                            // its lists (a later compaction keeps the k'
                            // smallest), so tau bounds its other items too
                            if (lane == 0) atomicMin(a.tq + iq[q].x, (unsigned long long)tau);
                            pass = pass && key < tau;
                            msk = __ballot_sync(0xffffffffu, pass);
                            if (msk == 0u) continue;
                        }
                        if (pass) lists[q * KC + cnt + __popc(msk & below)] = key;
                        cnt += __popc(msk);
                        __syncwarp();
                    }
                    if (lane == 0) {
                        s_cnt[q] = cnt;
                        s_tau[q] = tau;
                    }
                    __syncwarp();
                }
                mbar_arrive(tile_empty0 + 8 * t);
            }
            if (!ok) break;
            for (int q = fw; q < nqi; q += NFX) {               // write this warp's lists
                int cnt = s_cnt[q];
                if (cnt >= kp) {                                 // keep the k' smallest; publish the k'-th
                    const uint64_t th = compact_list<C::KS>(lists + q * KC, cnt, kp, lane);
                    cnt = kp;
                    if (lane == 0) atomicMin(a.tq + iq[q].x, (unsigned long long)th);
                }
                const int64_t L = (int64_t)(uint32_t)iq[q].z | ((int64_t)iq[q].w << 32);
                if (!ERQ_DCHECK(L >= 0 && L < a.ck.lists && cnt >= 0 && cnt <= KC, a.ck.status, 6)) continue;
                uint64_t* dst = a.inter + L * KC;
                for (int e = lane; e < cnt; e += 32) dst[e] = lists[q * KC + e];
                if (lane == 0) a.inter_cnt[L] = cnt;
            }
            __syncwarp();
            mbar_arrive(empty_item0 + 8 * ib);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(a.status, kStatusTimeout);
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
    }
}

bool tc_available(int precision, int D, int kp) {
    return (precision == ERQ_PREC_FP16 || precision == ERQ_PREC_FP8) && D % KB == 0 && kp <= KCAP;
}

// Work-item query counts the tensor-core scan is built for, given k'.
bool scan_tc_shape_ok(int qn, int kp) {
    return (qn == CfgSmall::QN && kp <= 32) || (qn == CfgWide::QN && kp <= 32) || (qn == CfgLarge::QN && kp <= KCAP);
}

// Capacity (stride) of the per-(query, item) candidate lists written by the scan.
int scan_list_stride(int precision, int kp, int qn) {
    if (precision == ERQ_PREC_FP32) return kp;
    return qn == CfgLarge::QN ? CfgLarge::KC : CfgSmall::KC;   // CfgWide shares CfgSmall's list capacity
}

cudaError_t launch_to_half(const float* x, __half* y, int64_t n, cudaStream_t s);


// Per work item: {first padded row (lo, hi), rows, queries} and, per query slot,
// {query row or -1, ||q_r - c||^2 bits, output list index (lo, hi)}.  One warp per item.
__global__ void item_tables_kernel(const int4* __restrict__ items, const int64_t* __restrict__ n_items,
                                   const int64_t* __restrict__ list_off, const int64_t* __restrict__ poff,
                                   const int64_t* __restrict__ qoff, const int64_t* __restrict__ qlist,
                                   const float* __restrict__ dqc, const int64_t* __restrict__ qbase,
                                   const int32_t* __restrict__ slot_off, int maxp, int RR, int QN,
                                   int4* __restrict__ itemd, int4* __restrict__ itemq,
                                   unsigned long long* __restrict__ stats, DevChecks ck) {
    const int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= *n_items) return;
    if (!ERQ_DCHECK(it < ck.items, ck.status, 8)) return;
    const int4 w = items[it];
    const int c = w.x;
    const int64_t qb = qoff[c] + (int64_t)w.y * QN;
    const int nqi = (int)imin64(QN, qoff[c + 1] - qb);
    const int64_t size = list_off[c + 1] - list_off[c];
    const int64_t r0 = (int64_t)w.z * RR;
    const int64_t rb0 = poff[c] + r0;
    const int nrows = (int)(imin64(size, r0 + RR) - r0);
    if (lane == 0) {
        itemd[it] = make_int4((int)(uint32_t)rb0, (int)(rb0 >> 32), nrows, nqi);
        const unsigned long long nblk = (unsigned long long)((nrows + MR - 1) / MR);
        atomicAdd(&stats[2], nblk);
        atomicAdd(&stats[3], nblk * (unsigned long long)(nqi <= 16 ? 16 : (nqi + 15) & ~15));
    }
    for (int q = lane; q < QN; q += 32) {
        int4 v = make_int4(-1, 0, 0, 0);
        if (q < nqi && ERQ_DCHECK(qb + q >= 0 && qb + q < ck.qlist, ck.status, 8)) {
            const int64_t e = qlist[qb + q];
            const int64_t qr = e / maxp;
            const int64_t L = qbase[qr] + slot_off[e] + w.z;
            v = make_int4((int)qr, __float_as_int(dqc[e]), (int)(uint32_t)L, (int)(L >> 32));
        }
        itemq[it * QN + q] = v;
    }
}

cudaError_t launch_item_tables(const int4* items, const int64_t* n_items, int64_t items_bound, const int64_t* list_off,
                               const int64_t* poff, const int64_t* qoff, const int64_t* qlist, const float* dqc,
                               const int64_t* qbase, const int32_t* slot_off, int maxp, int RR, int qn, int4* itemd,
                               int4* itemq, unsigned long long* stats, const DevChecks& ck, cudaStream_t s) {
    if (items_bound <= 0) return cudaSuccess;
    count_launch();
    item_tables_kernel<<<(unsigned)ceil_div(items_bound, 8), 256, 0, s>>>(
        items, n_items, list_off, poff, qoff, qlist, dqc, qbase, slot_off, maxp, RR, qn, itemd, itemq, stats, ck);
    return cudaGetLastError();
}

// Packed scan layout of the index.  One thread per (tile t, K block kb, row r
// of the tile): padded row p = 32 t + r takes its cluster's stored row (or
// zeros past the cluster's end), packs the 64 codes of block kb into B 8-byte
// words (layout at unpack_codes) and writes word j to
// codes_p[((t * nkb + kb) * B + j) * 32 + r]; the kb = 0 thread also writes the
// row's {g, f_res / 2, id, 0} to rowmeta[p].
__global__ void scan_layout_kernel(const uint8_t* __restrict__ codes, const float* __restrict__ g,
                                   const float* __restrict__ f_res, const int64_t* __restrict__ ids,
                                   const int64_t* __restrict__ list_off, const int64_t* __restrict__ poff, int nlist,
                                   int64_t Np, int D, int B, uint64_t* __restrict__ codes_p,
                                   float4* __restrict__ rowmeta) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nkb = D / 64;
    const int r = (int)(tid & 31);
    const int64_t tk = tid >> 5;                 // t * nkb + kb
    const int64_t t = tk / nkb;
    const int kb = (int)(tk % nkb);
    const int64_t p = t * 32 + r;
    if (p >= Np) return;
    int lo = 0, hi = nlist;                      // cluster with poff[lo] <= p < poff[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (poff[mid] <= p) lo = mid;
        else hi = mid;
    }
    const int64_t j = p - poff[lo];
    const bool valid = j < list_off[lo + 1] - list_off[lo];
    const int64_t src = list_off[lo] + j;
    uint32_t u[16];                              // 64 codes, four per word (byte i of u[k] = code 4k + i)
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const uint4 v = valid ? reinterpret_cast<const uint4*>(codes + src * D + kb * 64)[x] : make_uint4(0u, 0u, 0u, 0u);
        u[4 * x] = v.x; u[4 * x + 1] = v.y; u[4 * x + 2] = v.z; u[4 * x + 3] = v.w;
    }
    uint64_t* dst = codes_p + (tk * B) * 32 + r;
    const int bs = B >= 4 ? 4 : 0;
    if (B >= 4) {
        // half h: byte L = (code 8h + L) & 15 | ((code 8h + 4 + L) & 15) << 4
        uint32_t N[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) N[h] = (u[2 * h] & 0x0F0F0F0Fu) | ((u[2 * h + 1] & 0x0F0F0F0Fu) << 4);
#pragma unroll
        for (int w = 0; w < 4; ++w) dst[w * 32] = (uint64_t)N[2 * w] | ((uint64_t)N[2 * w + 1] << 32);
    }
    for (int b = bs; b < B; ++b) {
        // bit 8L + (m & 7) of half (m >> 3) = bit b of code 4m + L
        uint32_t P[2] = {0u, 0u};
#pragma unroll
        for (int m = 0; m < 16; ++m)
            P[m >> 3] |= ((u[m] >> b) & 0x01010101u) << (m & 7);
        dst[b * 32] = (uint64_t)P[0] | ((uint64_t)P[1] << 32);
    }
    if (kb == 0)
        rowmeta[p] = valid ? make_float4(g[src], 0.5f * f_res[src], __uint_as_float((uint32_t)ids[src]), 0.f)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_scan_layout(const uint8_t* codes, const float* g, const float* f_res, const int64_t* ids,
                               const int64_t* list_off, const int64_t* poff, int nlist, int64_t Np, int D, int B,
                               uint64_t* codes_p, float4* rowmeta, cudaStream_t s) {
    if (Np <= 0) return cudaSuccess;
    count_launch();
    const int64_t n = ceil_div(Np, 32) * (D / 64) * 32;
    scan_layout_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(codes, g, f_res, ids, list_off, poff, nlist, Np, D,
                                                                  B, codes_p, rowmeta);
    return cudaGetLastError();
}

// 3-D view of the packed codes in 8-byte elements: (32 B words of a tile and
// K block, K block, tile); a box of (32 B, 1, 4) is the 128 rows x 8 B bytes
// of one stage, four contiguous tiles.
static bool make_codes_map(CUtensorMap* map, const uint64_t* codes_p, int64_t Np, int D, int B) {
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
    const int nkb = D / KB;
    const cuuint64_t dims[3] = {(cuuint64_t)(32 * B), (cuuint64_t)nkb, (cuuint64_t)((Np + 31) / 32)};
    const cuuint64_t strides[2] = {(cuuint64_t)256 * B, (cuuint64_t)256 * B * nkb};
    const cuuint32_t box[3] = {(cuuint32_t)(32 * B), 1, MR / 32};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)codes_p, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class C, bool F8>
static erq_status scan_tc_launch(const ScanLaunch& L, const tc::Args& a, cudaStream_t s) {
    const int smem = C::Smem::total;
    cudaError_t e = cudaFuncSetAttribute(scan_tc_kernel<C, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "scan_tc smem attribute");
    if (L.grid <= 0) return ERQ_OK;
    CUtensorMap map;
    if (!L.codes_p || ((uintptr_t)L.codes_p & 15) != 0 || (L.D % KB) != 0 || L.B < 1 || L.B > 8 ||
        !make_codes_map(&map, L.codes_p, L.Np, L.D, L.B))
        return fail(ERQ_ECUDA, "tensor-core scan: cuTensorMapEncodeTiled failed for the code array");
    count_launch();
    scan_tc_kernel<C, F8><<<L.grid, THREADS, smem, s>>>(map, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scan_tc launch");
    return ERQ_OK;
}

erq_status scan_tc(const ScanLaunch& L, int precision, cudaStream_t s) {
    if (!tc_available(precision, L.D, L.kp))
        return fail(ERQ_EUNSUPPORTED, "tensor-core scan: needs precision fp16 or fp8 and k' <= 128");
    const bool f8 = precision == ERQ_PREC_FP8;
    if (f8 && L.B > 4) return fail(ERQ_EUNSUPPORTED, "tensor-core scan: e4m3 holds the centred codes only for B <= 4");
    if (!(f8 ? (L.Q8 && L.qscale) : L.Qh != nullptr)) return fail(ERQ_EINVAL, "tensor-core scan: queries missing");
    if (!L.itemd || !L.itemq || !L.rowmeta || !L.tq) return fail(ERQ_EINVAL, "tensor-core scan: item tables missing");
    tc::Args a;
    a.ck = L.ck;
    a.Qb = f8 ? (const unsigned char*)L.Q8 : (const unsigned char*)L.Qh;
    a.qrow_bytes = f8 ? L.Dq : 2 * (int64_t)L.D;
    a.qscale = L.qscale;
    a.itemd = L.itemd; a.itemq = L.itemq; a.rowmeta = L.rowmeta; a.n_items = L.n_items;
    a.inter = L.inter; a.inter_cnt = L.inter_cnt; a.status = L.status; a.D = L.D; a.B = L.B; a.kp = L.kp;
    a.tq = L.tq;
    a.ip = L.ip;
    if (!scan_tc_shape_ok(L.qn, L.kp)) return fail(ERQ_EINVAL, "tensor-core scan: no kernel for this item shape");
    if (L.qn == CfgWide::QN) return f8 ? scan_tc_launch<CfgWide, true>(L, a, s) : scan_tc_launch<CfgWide, false>(L, a, s);
    if (L.qn == CfgSmall::QN)
        return f8 ? scan_tc_launch<CfgSmall, true>(L, a, s) : scan_tc_launch<CfgSmall, false>(L, a, s);
    return f8 ? scan_tc_launch<CfgLarge, true>(L, a, s) : scan_tc_launch<CfgLarge, false>(L, a, s);
}

// Rotated queries -> e4m3 for the kind::f8f6f4 scan.  Per query row a power of
// two s = 2^(floor(log2 max|q'|) - 7) puts the largest magnitude in [128, 256)
// (e4m3's largest finite value is 448); every q'_i / s (exact) is rounded to
// the nearest e4m3 value, ties to even, from its FP32 bits: for |y| >= 2^-6 the
// 23-bit mantissa keeps its top 3 bits (carry into the exponent on overflow),
// below it y is a multiple of 2^-9 after rounding |y| * 2^9 to an integer
// (8 then being the smallest normal's code).  Columns D .. Dq-1 are zero.
// One warp per query row.
__device__ __forceinline__ uint32_t e4m3_rn(float y) {
    const uint32_t bits = __float_as_uint(y);
    const uint32_t sign = (bits >> 31) << 7;
    const int ex = (int)((bits >> 23) & 0xffu) - 127;
    const uint32_t mant = bits & 0x7fffffu;
    uint32_t code;
    if (ex >= -6) {
        uint32_t r = mant >> 20;
        const uint32_t rem = mant & 0xfffffu;
        if (rem > 0x80000u || (rem == 0x80000u && (r & 1u))) ++r;
        int e4 = ex + 7;
        if (r == 8u) {
            r = 0u;
            ++e4;
        }
        code = ((uint32_t)e4 << 3) | r;
    } else if (ex >= -10) {
        const int sh = 14 - ex;                        // 21 .. 24
        const uint32_t full = mant | 0x800000u;
        uint32_t q = full >> sh;
        const uint32_t rem = full & ((1u << sh) - 1u), half = 1u << (sh - 1);
        if (rem > half || (rem == half && (q & 1u))) ++q;
        code = q;
    } else {
        code = 0u;                                     // below half of the smallest subnormal
    }
    return sign | code;
}

__global__ void quant_e4m3_kernel(const float* __restrict__ X, int64_t n, int D, int Dq, unsigned char* __restrict__ Y,
                                  float* __restrict__ scale) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float* x = X + r * D;
    float m = 0.f;
    for (int i = lane; i < D; i += 32) m = fmaxf(m, fabsf(x[i]));
    m = warp_max(m);
    int e = 0;
    if (m > 0.f) {
        frexpf(m, &e);                                 // m in [2^(e-1), 2^e)
        e -= 8;                                        // m / 2^e in [128, 256)
    }
    e = max(-126, min(127, e));
    const float inv = __int_as_float((127 - e) << 23), s = __int_as_float((127 + e) << 23);
    if (lane == 0) scale[r] = m > 0.f ? s : 1.f;
    unsigned char* y = Y + r * Dq;
    for (int i = lane * 4; i < Dq; i += 128) {
        uint32_t w = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (i + j < D) w |= e4m3_rn(x[i + j] * inv) << (8 * j);
        *reinterpret_cast<uint32_t*>(y + i) = w;
    }
}

cudaError_t launch_quant_e4m3(const float* x, int64_t n, int D, int Dq, unsigned char* y, float* scale, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    quant_e4m3_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(x, n, D, Dq, y, scale);
    return cudaGetLastError();
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
