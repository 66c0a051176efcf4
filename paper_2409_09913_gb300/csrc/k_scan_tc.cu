// Tensor-core code scan (tcgen05, sm_103a): the contraction of Eq. 3.3,
// <2 ybar, q'> for every (query, candidate) pair of a work item, on the
// 5th-generation tensor cores with FP32 accumulation in tensor memory.
//
// A work item is (cluster, up to QN of the queries that probe it, up to RR
// stored rows).  Operands of one MMA (kind::f16, M = 128, N = npad, K = 16):
//   A = 128 stored rows of the cluster, codes expanded to 2*ybar_u - (2^B-1),
//       odd integers in [-255, 255] and therefore exact in FP16, held in
//       tensor memory (row = lane, two FP16 values per column);
//   B = the item's queries (rotated q' in FP16), npad = the query count rounded
//       up to a multiple of 16, K-major, 128-byte swizzled rows gathered from
//       the query matrix by TMA (tile::gather4, four rows per copy).
// Codes are read from a packed, scan-specific copy: every inverted list padded
// to a multiple of 32 rows and stored as [tiles of 32 rows][K blocks of 64]
// [B words][32 rows] of 8 bytes, i.e. exactly B bits per coordinate (the
// layout is given at unpack_codes); the 128 rows of one row block and K block
// are four contiguous 256*B-byte pieces fetched by one 3-D TMA load.
//
// The estimate is est = ||q_r - c||^2 + g + (f_res / 2) * acc with g, f_res the
// stored per-row factors, or for the inner-product metric the ranking score
// -<c, q_r> + (f_res / 4) * acc = -(estimated <o_r, q_r>).  The product is
// exact up to the FP16 rounding of q' (relative 2^-11 per element);
// accumulation is FP32.
//
// One persistent CTA per SM takes work items from a global counter (items are
// ordered by decreasing cluster size).  A stage group is up to RP = 2 row
// blocks of 128 rows that share the stage's query tile; a stage is one
// 64-coordinate K block of the group.  Warp roles (27 warps):
//   warps 0-3    estimate tiles: warp w reads TMEM lanes 32w .. 32w + 31 (its
//                32 rows, all queries) of each finished row-block accumulator,
//                frees the accumulator as soon as its last columns are in
//                registers, and stores g + (f_res/2) acc into one of EB
//                query-major tiles in shared memory;
//   warps 4-11   converters, two sets of four that take alternate stages:
//                warp w unpacks the codes of rows 32 (w % 4) .. + 31 of both
//                row blocks of its stages from the raw stage in shared memory
//                into FP16 (or e4m3) values in the stage's TMEM columns;
//   warp 12      code loader: publishes the items, per row block a bulk copy of
//                the rows' factors and ids, per stage one TMA load of the packed
//                codes per row block into a raw ring that is released as soon as
//                the converters have read it (so loads run up to RS stages
//                ahead, independent of the tensor cores; RS is even, so that
//                each raw slot is always converted by the same converter set
//                and its phases are awaited in order);
//   warps 13-14  query loaders: per stage the item's query rows (128 bytes
//                each) by TMA gather4 into the stage's swizzled B tile, the
//                stages taken in turn by the two warps;
//   warps 15, 16 MMA issuers of row blocks 0 and 1 (one elected thread each;
//                warp 15 owns the tensor memory); each commits once per stage to
//                the stage's release barrier, which frees the query tile and the
//                stage's TMEM code columns;
//   warps 17-26  filters (NFX = 10), pipelined behind the tiles through full /
//                empty tile barriers: warp f owns the query slots f + NFX j and
//                filters their rows (float pre-filter against the threshold,
//                exact keys, ballots) into per-query candidate lists; a full
//                list is compacted by a warp bitonic sort to its k' smallest.
//                A query starts from the smallest k'-th key published so far by
//                its items, which is never below its final k'-th key, so each
//                list stays a superset of what the item contributes.
// Accumulators are double-buffered per row block, so the epilogue of one stage
// group overlaps the MMAs of the next.
// Every mbarrier wait is bounded (the limit is a kernel argument): on expiry
// the kernel records ERQ_ETIMEOUT in the status word, every role stops at its
// next wait (the abort flag), the copies and MMAs already issued are drained
// (bounded), TMEM is freed and the kernel returns.
#include <algorithm>
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

constexpr int MR = 128;          // stored rows per row block (MMA M = TMEM lanes)
static_assert(MR == 128, "four 32-row lane quarters per row block");
constexpr int KB = 64;           // FP16 elements per K block (one 128-byte swizzle row)
constexpr int RP = 2;            // row blocks per stage group (one accumulator and one issuer each)
constexpr int MS = 8;            // row-factor buffers
constexpr int RSMAX = 8;         // raw-code ring slots at most
constexpr int W_CV = 4;          // converter warps 4..11 (row block (w - 4) / 4, lane quarter w % 4)
constexpr int W_LD = 12;         // code loader and item publisher
constexpr int W_QL = 13;         // query-tile loaders 13 .. 13 + NQL - 1 (stage g: loader g % NQL)
constexpr int NQL = 2;
constexpr int W_MMA = W_QL + NQL;   // MMA issuers (row block 0, TMEM owner; row block 1)
constexpr int W_FX = W_MMA + 2;     // filter warps W_FX .. W_FX + NFX - 1
constexpr int NFX = 10;
constexpr int NWARP = W_FX + NFX;
constexpr int THREADS = 32 * NWARP;
constexpr int TMEM_COLS = 512;
constexpr int KCAP = 128;        // largest k' of the tensor-core path

// Work-item capacities: QN queries per item at most (the MMA's N extent), KC
// list entries per query, NBUF accumulator buffers per row block, LS stages of
// query tiles and TMEM code columns, EB estimate tiles (with two the filters
// work on one while the other fills), RAWK KB of raw-code ring, and LG: the
// per-query candidate lists live in the item's output list slots in global
// memory (LG = 1) instead of shared memory.
template <int QN_, int KC_, int NBUF_, int LS_, int EB_, int RAWK_, int LG_>
struct Cfg {
    static constexpr int QN = QN_, KC = KC_, NBUF = NBUF_, LS = LS_, EB = EB_, LG = LG_;
    static constexpr int RAW_BYTES = RAWK_ * 1024;
    static constexpr int KS = KC <= 64 ? 64 : 256;   // sort width of a list compaction
    static constexpr int TILE_Q = QN * 128;          // one stage's query tile: QN rows of 128 bytes
    static constexpr int ACOL = NBUF * RP * QN;      // first TMEM column of the code stages
    static_assert(ACOL + LS * RP * (KB / 2) <= TMEM_COLS, "tensor memory budget");
    static_assert(LS % 2 == 0, "the two converter sets take alternate stages and must own whole slots");
    static_assert(QN % 32 == 0 && KC >= 64 && (QN + NFX - 1) / NFX <= 32, "item shape");
    struct Smem {
        // offsets in bytes from a 1024-aligned base
        static constexpr int q = 0;                              // LS x [QN][128 B] query tiles, swizzled
        static constexpr int raw = q + LS * TILE_Q;              // raw-code ring (RS slots of RP x B KB)
        static constexpr int est = raw + RAW_BYTES;              // EB x [QN][MR] f32 g + (f_res/2) acc
        static constexpr int lists = est + EB * QN * MR * 4;     // [QN][KC] u64 candidate keys (LG = 0)
        static constexpr int meta = lists + (LG ? 0 : QN * KC * 8);   // MS x [MR] float4 {g, f_res/2, id, 0}
        static constexpr int iq = meta + MS * MR * 16;           // 2 x [QN] int4 {query row, dqc bits, list lo, hi}
        static constexpr int tq = iq + 2 * QN * 16;              // 2 x [QN] u64 query-wide threshold at publication
        static constexpr int qsc = tq + 2 * QN * 8;              // 2 x [QN] f32 query scale (e4m3 path)
        static constexpr int itd = qsc + 2 * QN * 4;             // 2 x int4 {rb0 lo, rb0 hi, rows, queries | -1}
        static constexpr int ids = itd + 2 * 16;                 // EB x [MR] u32 ids of the tile's rows
        static constexpr int bars = ids + EB * MR * 4;
        static constexpr int nbars = 2 * RSMAX + 2 * LS + LS * RP + 2 * NBUF * RP + 2 * MS + 4 + 2 + 2 * EB;
        static constexpr int tmem_slot = bars + nbars * 8;
        static constexpr int abort_flag = tmem_slot + 4;
        static constexpr int total = abort_flag + 4 + 1024;      // + alignment slack
    };
    static_assert(Smem::total <= 227 * 1024, "scan_tc shared memory");
    // barrier byte offsets from Smem::bars
    static constexpr int b_full_raw(int s) { return 8 * s; }
    static constexpr int b_empty_raw(int s) { return 8 * (RSMAX + s); }
    static constexpr int b_full_q(int s) { return 8 * (2 * RSMAX + s); }
    static constexpr int b_empty_st(int s) { return 8 * (2 * RSMAX + LS + s); }
    static constexpr int b_full_a(int s, int b) { return 8 * (2 * RSMAX + 2 * LS + s * RP + b); }
    static constexpr int b_tfull(int u, int b) { return 8 * (2 * RSMAX + 2 * LS + LS * RP + u * RP + b); }
    static constexpr int b_tempty(int u, int b) { return 8 * (2 * RSMAX + 2 * LS + LS * RP + NBUF * RP + u * RP + b); }
    static constexpr int B0 = 2 * RSMAX + 2 * LS + LS * RP + 2 * NBUF * RP;
    static constexpr int b_full_meta(int m) { return 8 * (B0 + m); }
    static constexpr int b_empty_meta(int m) { return 8 * (B0 + MS + m); }
    static constexpr int b_full_item(int i) { return 8 * (B0 + 2 * MS + i); }
    static constexpr int b_empty_item(int i) { return 8 * (B0 + 2 * MS + 2 + i); }
    static constexpr int b_done() { return 8 * (B0 + 2 * MS + 4); }
    // a barrier nothing arrives on (the test stall of the bounded-wait path)
    static constexpr int b_never() { return 8 * (B0 + 2 * MS + 5); }
    static constexpr int b_tile_full(int t) { return 8 * (B0 + 2 * MS + 6 + t); }
    static constexpr int b_tile_empty(int t) { return 8 * (B0 + 2 * MS + 6 + EB + t); }
};
using CfgA = Cfg<64, 64, 2, 4, 2, 64, 0>;    // k' <= 32, up to 64 queries per item
using CfgW = Cfg<128, 64, 1, 4, 1, 48, 1>;   // k' <= 32, up to 128 queries per item (twice the MMA width)
using CfgB = Cfg<32, 160, 2, 4, 2, 64, 0>;   // k' <= 128, up to 32 queries per item

// arrivals that complete a phase of the item-release barrier: every lane of the
// query loader, the converters, the two issuers, the tile warps and the filters
constexpr int kItemReleasers = 32 * (NQL + 8 + 2 + 4 + NFX);

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

// B = 9: bits 0-7 assembled in byte lanes as for B = 8 (nibble words 0-3,
// planes 4-7) and bit 8 from plane 8; placed under 0x64 with bit 8 in the high
// byte's lowest bit, each 16-bit lane is the FP16 value 1024 + u (u < 512,
// exact), and 2 (1024 + u) - 2048 - 511 = 2u - 511 (each step exact).
__device__ __forceinline__ void unpack_codes9(const unsigned char* base, uint32_t (&w)[32]) {
    uint2 W[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) W[j] = *reinterpret_cast<const uint2*>(base + 256 * j);
    const __half2 off2 = __floats2half2_rn(511.f, 511.f);
    const __half2 two = __floats2half2_rn(2.f, 2.f);
    const __half2 m2048 = __floats2half2_rn(-2048.f, -2048.f);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int h = m >> 1;
        const uint32_t N = (h & 1) ? W[h >> 1].y : W[h >> 1].x;
        uint32_t V = (m & 1) ? (N >> 4) & 0x0F0F0F0Fu : N & 0x0F0F0F0Fu;
#pragma unroll
        for (int b = 4; b < 8; ++b) {
            const uint32_t P = m < 8 ? W[b].x : W[b].y;
            const int sh = b - (m & 7);
            const uint32_t x = sh >= 0 ? P << sh : P >> (-sh);
            V |= x & (0x01010101u << b);
        }
        const uint32_t P8 = m < 8 ? W[8].x : W[8].y;
        const uint32_t H = ((P8 >> (m & 7)) & 0x01010101u) | 0x64646464u;   // 0x64 | bit 8, per byte lane
        const uint32_t p0 = __byte_perm(V, H, 0x5140u);   // {u0 lo, 0x64 | u0 bit 8, u1 lo, ...}
        const uint32_t p1 = __byte_perm(V, H, 0x7362u);
        __half2 h0 = *reinterpret_cast<const __half2*>(&p0);
        __half2 h1 = *reinterpret_cast<const __half2*>(&p1);
        h0 = __hsub2(__hfma2(h0, two, m2048), off2);
        h1 = __hsub2(__hfma2(h1, two, m2048), off2);
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
        case 8: unpack_codes<8>(base, w); break;
        default: unpack_codes9(base, w); break;
    }
}

// Two FP16 values holding odd integers |x| <= 15 (exact in e4m3) -> their
// e4m3 encodings in bytes 0 and 2: the e4m3 exponent is the FP16 one minus 8
// (biases 15 and 7) and the three mantissa bits are the FP16 mantissa's top
// three (the lower seven are zero for these values).  With X16 the encodings
// are those of 16 x (exponent + 4; at most 240, below e4m3's 448).
template <bool X16 = false>
__device__ __forceinline__ uint32_t half2_to_e4m3_pair(uint32_t w) {
    constexpr uint32_t sub = X16 ? 0x00200020u : 0x00400040u;
    return (((w >> 7) & 0x00FF00FFu) - sub) | ((w >> 8) & 0x00800080u);
}

// Four byte lanes holding 2x (x < 16) -> the e4m3 encodings of 2x - off
// (odd, |2x - off| <= 15), times 16 with X16, in byte lanes 0..3.
template <bool X16>
__device__ __forceinline__ uint32_t lanes_to_e4m3(uint32_t V, __half2 c) {
    const uint32_t p0 = __byte_perm(V, 0x6464u, 0x4140u);   // {x0, 0x64, x1, 0x64}: FP16 1024 + 2x
    const uint32_t p1 = __byte_perm(V, 0x6464u, 0x4342u);
    const __half2 h0 = __hsub2(*reinterpret_cast<const __half2*>(&p0), c);
    const __half2 h1 = __hsub2(*reinterpret_cast<const __half2*>(&p1), c);
    return __byte_perm(half2_to_e4m3_pair<X16>(*reinterpret_cast<const uint32_t*>(&h0)),
                       half2_to_e4m3_pair<X16>(*reinterpret_cast<const uint32_t*>(&h1)), 0x6420u);
}

// Split e4m3 form of B = 5..8 codes (Section 3.3 remarks that a B-bit code
// can be handled as parts of fewer bits).  With u = 16 h + l, l < 16,
//   2u - (2^B - 1) = 16 (2h - (2^(B-4) - 1)) + (2l - 15),
// and both brackets are odd integers of magnitude <= 15, so 16 hc and lc are
// exact in e4m3.  Output: 32 columns for one 64-coordinate block, w[m] the
// four values 16 hc of coordinates 4m..4m+3 and w[16 + m] their lc; the
// stage's query tile holds the block's e4m3 queries twice (bytes 0-63 and
// 64-127), so the four K = 32 MMAs of the stage sum 16 hc q + lc q exactly.
// Packed layout as at unpack_codes (B >= 4: nibble words 0-3, planes 4..B-1).
template <int B>
__device__ __forceinline__ void unpack_split(const unsigned char* base, uint32_t (&w)[32]) {
    static_assert(B >= 5 && B <= 8, "split form is for B = 5..8");
    uint2 W[B];
#pragma unroll
    for (int j = 0; j < B; ++j) W[j] = *reinterpret_cast<const uint2*>(base + 256 * j);
    const float offh = (float)((1 << (B - 4)) - 1);
    const __half2 ch = __floats2half2_rn(1024.f + offh, 1024.f + offh);
    const __half2 cl = __floats2half2_rn(1039.f, 1039.f);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int h = m >> 1;
        const uint32_t N = (h & 1) ? W[h >> 1].y : W[h >> 1].x;
        const uint32_t L = (m & 1) ? (N >> 3) & 0x1E1E1E1Eu : (N << 1) & 0x1E1E1E1Eu;   // 2l per byte lane
        uint32_t H = 0;                                                                 // 2h per byte lane
#pragma unroll
        for (int b = 4; b < B; ++b) {
            const uint32_t P = m < 8 ? W[b].x : W[b].y;
            const int sh = (b - 3) - (m & 7);
            const uint32_t x = sh >= 0 ? P << sh : P >> (-sh);
            H |= x & (0x01010101u << (b - 3));
        }
        w[m] = lanes_to_e4m3<true>(H, ch);
        w[16 + m] = lanes_to_e4m3<false>(L, cl);
    }
}

__device__ __forceinline__ void unpack_split_b(int B, const unsigned char* base, uint32_t (&w)[32]) {
    switch (B) {
        case 5: unpack_split<5>(base, w); break;
        case 6: unpack_split<6>(base, w); break;
        case 7: unpack_split<7>(base, w); break;
        default: unpack_split<8>(base, w); break;
    }
}

struct Args {
    const int4* itemd;            // [items] {rb0 lo, rb0 hi, rows, queries}
    const int4* itemq;            // [items][qn] {query row or -1, dqc bits, output list index lo, hi}
    int qn;                       // queries per item of the plan (row stride of itemq)
    const float4* rowmeta;        // [Np] {g, f_res / 2, id bits, 0} in padded stored-row order
    const int64_t* n_items;
    unsigned int* work_ctr;       // items taken after the first grid-size ones (zero at launch)
    uint64_t* inter;
    int32_t* inter_cnt;
    unsigned long long* tq;       // [nq] query-wide admission threshold (k'-th key of a finished item)
    const float* qscale;          // e4m3 path: per-query power-of-two scale of the e4m3 values
    uint32_t* status;
    int D, B, kp, nkb;            // nkb: stages per row group (64 FP16 or 128 e4m3 coordinates each)
    int ip;                       // inner-product metric: est = -<c, q_r> + (f_res / 4) * acc
    int codes_shared;             // items of one cluster share its rows (queries > QN): codes stay in L2 normally,
                                  // else they are loaded evict-first
    unsigned long long wait_ns;   // limit of every bounded wait
    long long stall_stage;        // >= 0: the first issuer waits at this stage on a barrier nothing arrives on
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

// A threshold on the estimate tile's values (g + (f_res/2) acc) that admits
// every value v with fl(dq + v) <= tf: tf - dq, raised by 2^-20 of
// |tf| + |dq| to cover the roundings of fl(dq + v) and of this expression
// (each within 2^-24 of the magnitudes involved) and by 2^-120 for the
// absolute error of subnormal results; +inf stays +inf.
__device__ __forceinline__ float relaxed_threshold(float tf, float dq) {
    return (tf - dq) + (0x1p-20f * (fabsf(tf) + fabsf(dq)) + 0x1p-120f);
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

// P selects the operand form: 0 FP16 codes and queries (kind::f16, K = 16);
// 1 e4m3 codes (B <= 4) and queries with a per-query scale (kind::f8f6f4,
// K = 32), a stage covering 128 coordinates (two packed 64-coordinate blocks)
// in the same 128 bytes per row of tensor memory and query tile as 64 FP16
// coordinates; 2 the split e4m3 form of B = 5..8 codes (unpack_split), a
// stage covering 64 coordinates whose query tile holds them twice.
template <class C, int P>
__global__ void __launch_bounds__(THREADS, 1)
    scan_tc_kernel(const __grid_constant__ CUtensorMap codes_map, const __grid_constant__ CUtensorMap codes_map1,
                   const __grid_constant__ CUtensorMap q_map, tc::Args a) {
    constexpr bool F8 = P != 0;       // e4m3 operands
    constexpr bool W2 = P == 1;       // two packed blocks per stage
    constexpr int QN = C::QN, KC = C::KC, LS = C::LS, NBUF = C::NBUF, TILE_Q = C::TILE_Q, ACOL = C::ACOL;
    constexpr int EB = C::EB, RAW_BYTES = C::RAW_BYTES;
    using Smem = typename C::Smem;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t bars = smem_u32(sm + Smem::bars);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Smem::tmem_slot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + Smem::abort_flag);
    int4* s_iq = reinterpret_cast<int4*>(sm + Smem::iq);
    int4* s_itd = reinterpret_cast<int4*>(sm + Smem::itd);
    unsigned long long* s_tq = reinterpret_cast<unsigned long long*>(sm + Smem::tq);
    float* s_qsc = reinterpret_cast<float*>(sm + Smem::qsc);
    const float4* s_meta = reinterpret_cast<const float4*>(sm + Smem::meta);
    const unsigned long long wlim = a.wait_ns;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = a.nkb;
    const uint32_t blk = (uint32_t)(MR / 32) * 256u * (uint32_t)a.B;    // packed codes of one 128-row K block
    const uint32_t slot_bytes = (uint32_t)RP * blk * (W2 ? 2u : 1u);
    // an even number of raw slots: stage g uses slot g % RS and converter set
    // g % 2, so every slot belongs to one set, which awaits its phases in order
    // (with an odd RS a set could test a slot's parity one phase early)
    const int RS = min(RSMAX, (int)(RAW_BYTES / slot_bytes)) & ~1;
    int64_t nitems = *a.n_items;
    if (!ERQ_DCHECK(nitems >= 0 && nitems <= a.ck.items, a.ck.status, 7)) nitems = 0;   // uniform: every thread reads it

    if (tid == 0) {
        for (int s = 0; s < RSMAX; ++s) {
            mbar_init(bars + C::b_full_raw(s), 1);
            mbar_init(bars + C::b_empty_raw(s), 128);     // the converter set of the stage
        }
        for (int s = 0; s < LS; ++s) {
            mbar_init(bars + C::b_full_q(s), 1);
            mbar_init(bars + C::b_empty_st(s), RP);
            for (int b = 0; b < RP; ++b) mbar_init(bars + C::b_full_a(s, b), 128);
        }
        for (int u = 0; u < NBUF; ++u)
            for (int b = 0; b < RP; ++b) {
                mbar_init(bars + C::b_tfull(u, b), 1);
                mbar_init(bars + C::b_tempty(u, b), 128);
            }
        for (int m = 0; m < MS; ++m) {
            mbar_init(bars + C::b_full_meta(m), 1);
            mbar_init(bars + C::b_empty_meta(m), 128);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bars + C::b_full_item(i), 32);
            mbar_init(bars + C::b_empty_item(i), kItemReleasers);
        }
        mbar_init(bars + C::b_done(), RP);
        mbar_init(bars + C::b_never(), 1);
        for (int t = 0; t < EB; ++t) {
            mbar_init(bars + C::b_tile_full(t), 128);       // the four estimate-tile warps
            mbar_init(bars + C::b_tile_empty(t), 32 * NFX); // the filter warps
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == W_LD) {
        // ------------------------------------------------------------ code loader, item publisher
        uint32_t g = 0, rbg = 0, li = 0;
        bool ok = true;
        int64_t item = blockIdx.x;
        const uint64_t pol_codes = a.codes_shared ? l2_evict_normal() : l2_evict_first();
        // the descriptor and query slots of the item published next, fetched
        // while the previous item streams (its thresholds are read when it is
        // published, so they are as tight as possible)
        constexpr int QPL = QN / 32;
        int4 pd = make_int4(0, 0, 0, -1), pv[QPL];
        auto prefetch = [&](int64_t it) {
            if (it >= nitems) return;
            pd = a.itemd[it];
#pragma unroll
            for (int k = 0; k < QPL; ++k) {
                const int q = lane + 32 * k;
                pv[k] = q < a.qn ? a.itemq[it * a.qn + q] : make_int4(-1, 0, 0, 0);
            }
        };
        prefetch(item);
        for (;; ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(bars + C::b_empty_item(ib), ((li >> 1) & 1) ^ 1, abort_flag, wlim)) {
                ok = false;
                break;
            }
            const bool have = item < nitems;
            int4 d = make_int4(0, 0, 0, -1);
            if (have) {
                d = pd;
#pragma unroll
                for (int k = 0; k < QPL; ++k) {
                    const int q = lane + 32 * k;
                    const int4 v = pv[k];
                    s_iq[ib * QN + q] = v;
                    s_tq[ib * QN + q] = v.x >= 0 ? __ldcg(a.tq + v.x) : kEmptyKey;
                    if (F8) s_qsc[ib * QN + q] = v.x >= 0 ? a.qscale[v.x] : 0.f;
                }
            }
            if (lane == 0) s_itd[ib] = d;
            __syncwarp();
            mbar_arrive(bars + C::b_full_item(ib));
            if (!have) break;
            const int64_t rb0 = rb0_of(d);                 // first padded row (multiple of 32)
            const int nrows = d.z;
            // the next item is claimed exactly once per published item: at the
            // start of this item's last stage group, so that its descriptor
            // arrives while the group streams (claiming no earlier keeps the
            // items of one list on several SMs at about the same time, sharing
            // its codes in L2), or below for an item without rows
            bool claimed = false;
            auto claim_next = [&]() {
                int nx = 0;
                if (lane == 0) nx = (int)atomicAdd(a.work_ctr, 1u);
                item = (int64_t)gridDim.x + __shfl_sync(0xffffffffu, nx, 0);
                prefetch(item);
                claimed = true;
            };
            for (int r = 0; r < nrows && ok; r += RP * MR) {
                if (r + RP * MR >= nrows) claim_next();
                const int nb = min(RP, (nrows - r + MR - 1) / MR);     // row blocks in this stage group
                for (int bb = 0; bb < nb && ok; ++bb, ++rbg) {
                    const int nr = min(MR, nrows - r - bb * MR);
                    const int m = rbg % MS;
                    if (!mbar_wait_warp(bars + C::b_empty_meta(m), ((rbg / MS) & 1) ^ 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        mbar_arrive_expect_tx(bars + C::b_full_meta(m), (uint32_t)nr * 16u);
                        bulk_load(smem_u32(sm + Smem::meta + m * MR * 16), a.rowmeta + rb0 + r + bb * MR,
                                  (uint32_t)nr * 16u, bars + C::b_full_meta(m));
                    }
                }
                for (int kb = 0; kb < nkb && ok; ++kb, ++g) {
                    const int s = g % RS;
                    if (!mbar_wait_warp(bars + C::b_empty_raw(s), ((g / RS) & 1) ^ 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        // whole 32-row tiles of the item's rows only: a block of
                        // fewer than 128 rows takes its tiles one by one (the rows
                        // past them are never admitted: the filters test rr < nr)
                        const int rem = nrows - r;
                        const uint32_t tiles = (uint32_t)min(RP * MR / 32, (rem + 31) >> 5);
                        mbar_arrive_expect_tx(bars + C::b_full_raw(s), tiles * 256u * (uint32_t)a.B * (W2 ? 2u : 1u));
                        for (int bb = 0; bb < nb; ++bb) {
                            const uint32_t dst = smem_u32(sm + Smem::raw + s * slot_bytes + bb * blk * (W2 ? 2 : 1));
                            const int tile = (int)((rb0 + r + bb * MR) >> 5);
                            const int nt = min(MR / 32, ((rem - bb * MR) + 31) >> 5);
                            // (the second block of the last P = 1 stage may lie past D: the TMA fills zeros)
                            for (int h = 0; h < (W2 ? 2 : 1); ++h) {
                                const int kk = W2 ? 2 * kb + h : kb;
                                if (nt == MR / 32) {
                                    tma_load_4d_hint(dst + h * blk, &codes_map, 0, 0, kk, tile,
                                                     bars + C::b_full_raw(s), pol_codes);
                                } else {
                                    for (int t = 0; t < nt; ++t)
                                        tma_load_4d_hint(dst + h * blk + t * 256u * (uint32_t)a.B, &codes_map1, 0, 0,
                                                         kk, tile + t, bars + C::b_full_raw(s), pol_codes);
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            if (!ok) break;
            if (!claimed) claim_next();
        }
        // drain: every copy this warp issued has landed before the CTA exits
        for (uint32_t k = 0; k < (uint32_t)RS && k < g; ++k) {
            const uint32_t gg = g - 1 - k;
            mbar_wait_drain(bars + C::b_full_raw(gg % RS), (gg / RS) & 1);
        }
        for (uint32_t k = 0; k < MS && k < rbg; ++k) {
            const uint32_t gg = rbg - 1 - k;
            mbar_wait_drain(bars + C::b_full_meta(gg % MS), (gg / MS) & 1);
        }
        __syncwarp();
    } else if (warp >= W_QL && warp < W_QL + NQL) {
        // ------------------------------------------------------------ query loaders (TMA gather4)
        // Loader j issues the query tiles of the stages g with g % NQL == j.
        const uint32_t qj = (uint32_t)(warp - W_QL);
        const uint64_t pol_q = l2_evict_last();           // the query rows are read by many items
        uint32_t g = 0;
        bool ok = true;
        for (uint32_t li = 0; ok; ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(bars + C::b_full_item(ib), (li >> 1) & 1, abort_flag, wlim)) break;
            const int4 d = s_itd[ib];
            if (d.w < 0) break;
            const int npad = npad_of(d.w);
            const int nsteps = ((d.z + RP * MR - 1) / (RP * MR)) * nkb;
            // lane i gathers query slots 4i .. 4i+3 (padding slots repeat slot 0's row)
            const int4* iq = s_iq + ib * QN;
            const int r0 = iq[0].x;
            int y[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int qs = 4 * lane + j;
                const int qr = qs < QN ? iq[qs].x : -1;
                y[j] = qr >= 0 ? qr : r0;
            }
            for (int t = 0; t < nsteps; ++t, ++g) {
                if (g % NQL != qj) continue;
                const int s = g % LS, kb = t % nkb;
                if (!mbar_wait_warp(bars + C::b_empty_st(s), ((g / LS) & 1) ^ 1, abort_flag, wlim)) {
                    ok = false;
                    break;
                }
                if (lane == 0) mbar_arrive_expect_tx(bars + C::b_full_q(s), (uint32_t)npad * 128u);
                __syncwarp();
                if (4 * lane < npad)
                    tma_gather4_hint(smem_u32(sm + Smem::q + s * TILE_Q + lane * 512), &q_map, kb * 128, y[0], y[1],
                                     y[2], y[3], bars + C::b_full_q(s), pol_q);
                __syncwarp();
            }
            if (!ok) break;
            mbar_arrive(bars + C::b_empty_item(ib));
        }
        for (uint32_t k = 0; k < LS && k < g; ++k) {     // (the stages this loader issued)
            const uint32_t gg = g - 1 - k;
            if (gg % NQL == qj) mbar_wait_drain(bars + C::b_full_q(gg % LS), (gg / LS) & 1);
        }
        __syncwarp();
    } else if (warp >= W_CV && warp < W_CV + 8) {
        // ------------------------------------------------------------ converters
        // Two sets of four warps take alternate stages (set cs the stages with
        // g % 2 == cs) and convert both row blocks of each: thread = one row of a
        // block (TMEM lane 32 (w % 4) + lane); the TMEM stores of the two blocks
        // are waited for once, while the other set converts the next stage.
        const int cs = (warp - W_CV) >> 2, qt = warp & 3;
        const int r = qt * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(qt * 32) << 16;
        const int B = a.B;
        const int roff = (r >> 5) * 256 * B + (r & 31) * 8;   // word 0 of row r in a 128-row block
        uint32_t g = 0;
        bool ok = true;
        for (uint32_t li = 0; ok; ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(bars + C::b_full_item(ib), (li >> 1) & 1, abort_flag, wlim)) break;
            const int4 d = s_itd[ib];
            if (d.w < 0) break;
            const int nrows = d.z;
            for (int r0 = 0; r0 < nrows && ok; r0 += RP * MR) {
                const int nb = min(RP, (nrows - r0 + MR - 1) / MR);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    if ((int)(g & 1) != cs) continue;
                    const int s = g % LS, rs = g % RS;
                    // the stage's TMEM columns are free (its previous MMAs completed)
                    // and its raw codes have landed
                    if (!mbar_wait_warp(bars + C::b_empty_st(s), ((g / LS) & 1) ^ 1, abort_flag, wlim) ||
                        !mbar_wait_warp(bars + C::b_full_raw(rs), (g / RS) & 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int bb = 0; bb < nb; ++bb) {                  // warp-uniform
                        uint32_t w[32];
                        const unsigned char* src = sm + Smem::raw + rs * slot_bytes + bb * blk * (W2 ? 2 : 1) + roff;
                        if (W2) {
                            // two packed blocks -> 128 e4m3 codes, four per column
#pragma unroll
                            for (int hb = 0; hb < 2; ++hb) {
                                uint32_t h[32];
                                unpack_codes_b(B, src + hb * blk, h);
#pragma unroll
                                for (int c = 0; c < 16; ++c)
                                    w[16 * hb + c] = __byte_perm(half2_to_e4m3_pair(h[2 * c]),
                                                                 half2_to_e4m3_pair(h[2 * c + 1]), 0x6420u);
                            }
                        } else if (P == 2) {
                            unpack_split_b(B, src, w);
                        } else {
                            unpack_codes_b(B, src, w);
                        }
                        ERQ_TMEM_ST32(tmem + lane_addr + ACOL + (s * RP + bb) * (KB / 2), w);
                    }
                    mbar_arrive(bars + C::b_empty_raw(rs));        // the raw slot may be refilled
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    tc_fence_before();
                    mbar_arrive(bars + C::b_full_a(s, 0));
                    mbar_arrive(bars + C::b_full_a(s, 1));
                }
            }
            if (!ok) break;
            mbar_arrive(bars + C::b_empty_item(ib));
        }
    } else if (warp == W_MMA || warp == W_MMA + 1) {
        // ------------------------------------------------------------ MMA issuers
        // Issuer b runs the accumulation chain of row block b of each stage group
        // (tcgen05.mma issue stalls the issuing thread, so two issuers keep two
        // chains in flight); both commit every stage to its release barrier.
        const int b = warp - W_MMA;
        uint32_t g = 0, u = 0;
        bool ok = true;
        for (uint32_t li = 0; ok; ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(bars + C::b_full_item(ib), (li >> 1) & 1, abort_flag, wlim)) break;
            const int4 d = s_itd[ib];
            if (d.w < 0) break;
            const uint32_t idesc = idesc_f16(MR, npad_of(d.w));
            for (int r0 = 0; r0 < d.z && ok; r0 += RP * MR) {
                const bool has = b < min(RP, (d.z - r0 + MR - 1) / MR);
                const int buf = u % NBUF;
                if (has) {
                    if (!mbar_wait_warp(bars + C::b_tempty(buf, b), ((u / NBUF) & 1) ^ 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                const uint32_t dt = tmem + (uint32_t)((buf * RP + b) * QN);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % LS;
                    if (b == 0 && (long long)g == a.stall_stage &&
                        !mbar_wait_warp(bars + C::b_never(), 0, abort_flag, wlim)) {
                        ok = false;                                // (always: nothing arrives on it)
                        break;
                    }
                    if (!mbar_wait_warp(bars + C::b_full_a(s, b), (g / LS) & 1, abort_flag, wlim) ||
                        !mbar_wait_warp(bars + C::b_full_q(s), (g / LS) & 1, abort_flag, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (lane == 0) {
                        if (has) {
                            const uint32_t ta = tmem + ACOL + (s * RP + b) * (KB / 2);
                            const uint32_t tq = smem_u32(sm + Smem::q + s * TILE_Q);
#pragma unroll
                            for (int k = 0; k < KB / 16; ++k) {         // 32 bytes of K per instruction
                                if (F8) mma_f8_ta(dt, ta + k * 8, sdesc(tq + k * 32), idesc, (kb | k) != 0);
                                else mma_f16_ta(dt, ta + k * 8, sdesc(tq + k * 32), idesc, (kb | k) != 0);
                            }
                        }
                        mma_commit(bars + C::b_empty_st(s));          // query tile and TMEM stage free
                        if (has && kb == nkb - 1) mma_commit(bars + C::b_tfull(buf, b));
                    }
                    __syncwarp();
                }
                if (has) ++u;
            }
            if (!ok) break;
            mbar_arrive(bars + C::b_empty_item(ib));
        }
        // all issued MMAs complete before TMEM is released
        if (lane == 0) mma_commit(bars + C::b_done());
        __syncwarp();
        mbar_wait_drain(bars + C::b_done(), 0);
        __syncwarp();
    } else if (warp < W_CV) {
        // ------------------------------------------------------------ estimate tiles
        // Warp w moves TMEM lanes 32w..32w+31 (its 32 rows, all queries) of each
        // finished row-block accumulator into a query-major estimate tile and
        // frees the accumulator.
        float* s_est = reinterpret_cast<float*>(sm + Smem::est);
        uint32_t* s_ids = reinterpret_cast<uint32_t*>(sm + Smem::ids);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const int row = warp * 32 + lane;
        uint32_t blk = 0, rbg = 0, u[RP] = {};
        bool ok = true;
        for (uint32_t li = 0; ok; ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(bars + C::b_full_item(ib), (li >> 1) & 1, abort_flag, wlim)) break;
            const int4 d = s_itd[ib];
            if (d.w < 0) break;
            const int nrows = d.z, npad = npad_of(d.w);
            for (int r0 = 0; r0 < nrows && ok; r0 += RP * MR) {
                const int nb = min(RP, (nrows - r0 + MR - 1) / MR);
                for (int rb = 0; rb < nb; ++rb, ++blk) {
                    const uint32_t mrb = rbg + rb;
                    const int m = mrb % MS, t = blk % EB, buf = u[rb] % NBUF;
                    if (!mbar_wait_warp(bars + C::b_full_meta(m), (mrb / MS) & 1, abort_flag, wlim) ||
                        !mbar_wait_warp(bars + C::b_tfull(buf, rb), (u[rb] / NBUF) & 1, abort_flag, wlim) ||
                        !mbar_wait_warp(bars + C::b_tile_empty(t), ((blk / EB) & 1) ^ 1, abort_flag, wlim)) {
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
                    if (row >= min(MR, nrows - r0 - rb * MR)) {    // past the block's rows: NaN, which no
                        mt.x = __int_as_float(0x7fc00000);         // threshold admits
                        mt.y = 0.f;
                    }
                    const uint32_t tacc = tmem + lane_base + (uint32_t)((buf * RP + rb) * QN);
#pragma unroll 1
                    for (int cc = 0; cc < npad; cc += 32) {
                        uint32_t v[32];
                        ERQ_TMEM_LD32(tacc + cc, v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (cc + 32 >= npad) {                     // the last columns are in registers:
                            tc_fence_before();                     // the accumulator is free
                            mbar_arrive(bars + C::b_tempty(buf, rb));
                        }
                        if (F8) {                                  // e4m3 queries carry a power-of-two scale (exact)
                            const float* sc = s_qsc + ib * QN + cc;
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                est_t[(cc + i) * MR + row] = fmaf(mt.y, __uint_as_float(v[i]) * sc[i], mt.x);
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i) est_t[(cc + i) * MR + row] = fmaf(mt.y, __uint_as_float(v[i]), mt.x);
                        }
                    }
                    ++u[rb];
                    mbar_arrive(bars + C::b_empty_meta(m));
                    mbar_arrive(bars + C::b_tile_full(t));
                }
                rbg += nb;
            }
            if (!ok) break;
            mbar_arrive(bars + C::b_empty_item(ib));
        }
    } else {
        // ------------------------------------------------------------ filters
        // NFX warps; warp f owns the query slots q = f + NFX j of every item and
        // filters their rows of each estimate tile (float pre-filter against the
        // threshold, exact keys, ballots) into per-query candidate lists; a full
        // list is compacted by a warp bitonic sort to its k' smallest.  A query
        // starts from the smallest k'-th key published so far by its items, which
        // is never below its final k'-th key, so each list stays a superset of
        // what the item contributes to the query's top-k'.
        const float* s_est = reinterpret_cast<const float*>(sm + Smem::est);
        uint64_t* lists_s = reinterpret_cast<uint64_t*>(sm + Smem::lists);
        // query q's candidate list: shared memory, or its output slot of the item
        auto list_of = [&](const int4* iq, int q) -> uint64_t* {
            if (C::LG) return a.inter + ((int64_t)(uint32_t)iq[q].z | ((int64_t)iq[q].w << 32)) * KC;
            return lists_s + q * KC;
        };
        const uint32_t* s_ids = reinterpret_cast<const uint32_t*>(sm + Smem::ids);
        const int fw = warp - W_FX;
        const uint32_t below = (1u << lane) - 1u;
        const int kp = a.kp;
        uint32_t blk = 0;
        bool ok = true;
        for (uint32_t li = 0; ok; ++li) {
            const int ib = li & 1;
            if (!mbar_wait_warp(bars + C::b_full_item(ib), (li >> 1) & 1, abort_flag, wlim)) break;
            const int4 d = s_itd[ib];
            if (d.w < 0) break;
            const int nrows = d.z, nqi = d.w;
            const int4* iq = s_iq + ib * QN;
            // lane j holds the state of the warp's j-th query slot q = fw + NFX j:
            // its distance term, admission threshold (key and float), list fill
            // and the threshold relaxed into the estimate tile's units
            const int nown = nqi > fw ? (nqi - fw + NFX - 1) / NFX : 0;
            float my_dq = 0.f, my_tf = -INFINITY, my_thr = -INFINITY;
            uint64_t my_tau = 0;
            int my_cnt = 0;
            if (lane < nown) {
                const int q = fw + NFX * lane;
                my_dq = __int_as_float(iq[q].y);
                my_tau = s_tq[ib * QN + q];
                my_tf = my_tau == kEmptyKey ? INFINITY : key_value(my_tau);
                my_thr = relaxed_threshold(my_tf, my_dq);
            }
            for (int r = 0; r < nrows; r += MR, ++blk) {
                const int nr = min(MR, nrows - r);
                const int t = blk % EB;
                if (!mbar_wait_warp(bars + C::b_tile_full(t), (blk / EB) & 1, abort_flag, wlim)) {
                    ok = false;
                    break;
                }
                const float* est_t = s_est + t * (QN * MR);
                const uint32_t* ids_t = s_ids + t * MR;
                // the 128 rows of each owned query, rows 4 lane .. 4 lane + 3 in
                // lane `lane` (rows past the block are NaN): one vote against the
                // relaxed threshold (a superset of the float test below, which is
                // a superset of the key test), then per row group the float
                // test and exact keys
                for (int jj = 0; jj < nown; ++jj) {
                    const int q = fw + NFX * jj;
                    const float thr = __shfl_sync(0xffffffffu, my_thr, jj);
                    const float4 v4 = *reinterpret_cast<const float4*>(est_t + q * MR + 4 * lane);
                    if (!__any_sync(0xffffffffu, v4.x <= thr || v4.y <= thr || v4.z <= thr || v4.w <= thr)) continue;
                    const float dq = __shfl_sync(0xffffffffu, my_dq, jj);
                    float tf = __shfl_sync(0xffffffffu, my_tf, jj);
                    uint64_t tau = shfl_u64(my_tau, jj);
                    int cnt = __shfl_sync(0xffffffffu, my_cnt, jj);
                    const float e[4] = {dq + v4.x, dq + v4.y, dq + v4.z, dq + v4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int rr = 4 * lane + j;
                        const bool pre = rr < nr && e[j] <= tf;
                        if (!__any_sync(0xffffffffu, pre)) continue;
                        const uint64_t key = make_key(e[j], ids_t[rr]);
                        bool pass = pre && key < tau;
                        uint32_t msk = __ballot_sync(0xffffffffu, pass);
                        if (msk == 0u) continue;
                        if (cnt + __popc(msk) > KC) {
                            // full: keep the k' smallest (KC - k' >= 32 leaves
                            // room for a group), then test the group again
                            tau = compact_list<C::KS>(list_of(iq, q), cnt, kp, lane);
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
                        if (pass) list_of(iq, q)[cnt + __popc(msk & below)] = key;
                        cnt += __popc(msk);
                        __syncwarp();
                    }
                    if (lane == jj) {
                        my_cnt = cnt;
                        my_tau = tau;
                        if (tf != my_tf) my_thr = relaxed_threshold(tf, dq);
                        my_tf = tf;
                    }
                }
                mbar_arrive(bars + C::b_tile_empty(t));
            }
            if (!ok) break;
            for (int jj = 0; jj < nown; ++jj) {                 // write this warp's lists
                const int q = fw + NFX * jj;
                int cnt = __shfl_sync(0xffffffffu, my_cnt, jj);
                if (cnt >= kp) {                                 // keep the k' smallest; publish the k'-th
                    const uint64_t th = compact_list<C::KS>(list_of(iq, q), cnt, kp, lane);
                    cnt = kp;
                    if (lane == 0) atomicMin(a.tq + iq[q].x, (unsigned long long)th);
                }
                const int64_t L = (int64_t)(uint32_t)iq[q].z | ((int64_t)iq[q].w << 32);
                if (!ERQ_DCHECK(L >= 0 && L < a.ck.lists && cnt >= 0 && cnt <= KC, a.ck.status, 6)) continue;
                uint64_t* dst = a.inter + L * KC;
                if (!C::LG)
                    for (int e = lane; e < cnt; e += 32) dst[e] = lists_s[q * KC + e];
                if (lane == 0) a.inter_cnt[L] = cnt;
            }
            __syncwarp();
            mbar_arrive(bars + C::b_empty_item(ib));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(a.status, kStatusTimeout);
    if (warp == W_MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
    }
}

bool tc_available(int precision, int D, int kp) {
    return (precision == ERQ_PREC_FP16 || precision == ERQ_PREC_FP8) && D % KB == 0 && kp <= KCAP;
}

// Work-item query counts the tensor-core scan is built for, given k'.
bool scan_tc_shape_ok(int qn, int kp) {
    return (kp <= 32 && (qn == 32 || qn == CfgA::QN || qn == CfgW::QN)) || (kp <= KCAP && qn == CfgB::QN);
}

// Capacity (stride) of the per-(query, item) candidate lists written by the scan.
int scan_list_stride(int precision, int kp, int qn) {
    (void)qn;
    if (precision == ERQ_PREC_FP32) return kp;
    return kp <= 32 ? CfgA::KC : CfgB::KC;
}

cudaError_t launch_to_half(const float* x, __half* y, int64_t n, cudaStream_t s);



// Per work item: {first padded row (lo, hi), rows, queries} and, per query slot,
// {query row or -1, ||q_r - c||^2 bits, output list index (lo, hi)}.  One warp per item.
__global__ void item_tables_kernel(const int4* __restrict__ items, const int64_t* __restrict__ n_items,
                                   const int64_t* __restrict__ list_off, const int64_t* __restrict__ poff,
                                   const int64_t* __restrict__ qoff, const int64_t* __restrict__ qlist,
                                   const float* __restrict__ dqc, const int64_t* __restrict__ qbase,
                                   const int32_t* __restrict__ slot_off, int maxp, int RR, int QN, int nlist,
                                   int4* __restrict__ itemd, int4* __restrict__ itemq,
                                   unsigned long long* __restrict__ stats, DevChecks ck) {
    const int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= *n_items) return;
    if (!ERQ_DCHECK(it < ck.items, ck.status, 8)) return;
    const int4 w = items[it];
    const int v = w.x, c = v % nlist;                   // phase cluster -> cluster
    const int64_t qb = qoff[v] + (int64_t)w.y * QN;
    const int nqi = (int)imin64(QN, qoff[v + 1] - qb);
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
                               const int64_t* qbase, const int32_t* slot_off, int maxp, int RR, int qn, int nlist,
                               int4* itemd, int4* itemq, unsigned long long* stats, const DevChecks& ck,
                               cudaStream_t s) {
    if (items_bound <= 0) return cudaSuccess;
    count_launch();
    item_tables_kernel<<<(unsigned)ceil_div(items_bound, 8), 256, 0, s>>>(
        items, n_items, list_off, poff, qoff, qlist, dqc, qbase, slot_off, maxp, RR, qn, nlist, itemd, itemq, stats,
        ck);
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
    uint32_t u[16];                              // 64 codes, four per word (byte i of u[k] = bits 0-7 of code 4k + i)
    uint32_t h8[16] = {};                        // B = 9: byte i of h8[k] = bit 8 of code 4k + i
    if (B <= 8) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const uint4 v = valid ? reinterpret_cast<const uint4*>(codes + src * D + kb * 64)[x] : make_uint4(0u, 0u, 0u, 0u);
            u[4 * x] = v.x; u[4 * x + 1] = v.y; u[4 * x + 2] = v.z; u[4 * x + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int x = 0; x < 8; ++x) {            // 16-bit codes: eight per uint4
            const uint4 v = valid ? reinterpret_cast<const uint4*>(codes + (src * D + kb * 64) * 2)[x]
                                  : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 2; ++h) {        // codes 8x + 4h .. + 3 -> word 2x + h
                const uint32_t a = w[2 * h], b = w[2 * h + 1];
                u[2 * x + h] = __byte_perm(a, b, 0x6420u);
                h8[2 * x + h] = __byte_perm(a, b, 0x7531u) & 0x01010101u;
            }
        }
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
            P[m >> 3] |= (b < 8 ? (u[m] >> b) & 0x01010101u : h8[m]) << (m & 7);
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
static bool make_codes_map(CUtensorMap* map, const uint64_t* codes_p, int64_t Np, int D, int B, int box_tiles) {
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
    // 4-D view [tiles][K blocks][B words][32 rows] of u64 (a box extent is at most 256 elements,
    // so the 32 B words of a tile and K block are two dimensions, not one of 32 B)
    const int nkb = D / KB;
    const cuuint64_t dims[4] = {32, (cuuint64_t)B, (cuuint64_t)nkb, (cuuint64_t)((Np + 31) / 32)};
    const cuuint64_t strides[3] = {256, (cuuint64_t)256 * B, (cuuint64_t)256 * B * nkb};
    const cuuint32_t box[4] = {32, (cuuint32_t)B, 1, (cuuint32_t)box_tiles};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, (void*)codes_p, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D view of the query operand (FP16 or e4m3 rows of row_bytes bytes) for
// tile::gather4: a box of one row of 128 bytes, 128-byte swizzle, so that four
// gathered rows land as consecutive 128-byte rows of the MMA's B tile.
static bool make_query_map(CUtensorMap* map, const void* base, int64_t nq, int64_t row_bytes) {
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
    const cuuint64_t dims[2] = {(cuuint64_t)row_bytes, (cuuint64_t)nq};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {128, 1};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class C, int P>
static erq_status scan_tc_launch(const ScanLaunch& L, const tc::Args& a, const void* qbase, int64_t qrow_bytes,
                                 cudaStream_t s) {
    const int smem = C::Smem::total;
    {   // the kernel's raw-code ring must hold an even number (>= 2) of stage slots
        const int64_t slot = (int64_t)RP * (MR / 32) * 256 * L.B * (P == 1 ? 2 : 1);
        if ((std::min<int64_t>(RSMAX, C::RAW_BYTES / slot) & ~1ll) < 2)
            return fail(ERQ_EUNSUPPORTED, "tensor-core scan: raw-code ring too small for this code width");
    }
    cudaError_t e = cudaFuncSetAttribute(scan_tc_kernel<C, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "scan_tc smem attribute");
    if (L.grid <= 0) return ERQ_OK;
    CUtensorMap cmap, cmap1, qmap;
    if (!L.codes_p || ((uintptr_t)L.codes_p & 15) != 0 || (L.D % KB) != 0 || L.B < 1 || L.B > 9 ||
        !make_codes_map(&cmap, L.codes_p, L.Np, L.D, L.B, MR / 32) ||
        !make_codes_map(&cmap1, L.codes_p, L.Np, L.D, L.B, 1))
        return fail(ERQ_ECUDA, "tensor-core scan: cuTensorMapEncodeTiled failed for the code array");
    if (!qbase || ((uintptr_t)qbase & 15) != 0 || qrow_bytes % 128 != 0 || L.nq < 1 ||
        !make_query_map(&qmap, qbase, L.nq, qrow_bytes))
        return fail(ERQ_ECUDA, "tensor-core scan: cuTensorMapEncodeTiled failed for the query array");
    count_launch();
    scan_tc_kernel<C, P><<<L.grid, THREADS, smem, s>>>(cmap, cmap1, qmap, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scan_tc launch");
    return ERQ_OK;
}

template <class C>
static erq_status scan_tc_form(int P, const ScanLaunch& L, const tc::Args& a, const void* qb, int64_t qrow,
                               cudaStream_t s) {
    if (P == 1) return scan_tc_launch<C, 1>(L, a, qb, qrow, s);
    if (P == 2) return scan_tc_launch<C, 2>(L, a, qb, qrow, s);
    return scan_tc_launch<C, 0>(L, a, qb, qrow, s);
}

erq_status scan_tc(const ScanLaunch& L, int precision, cudaStream_t s) {
    if (!tc_available(precision, L.D, L.kp))
        return fail(ERQ_EUNSUPPORTED, "tensor-core scan: needs precision fp16 or fp8 and k' <= 128");
    const bool f8 = precision == ERQ_PREC_FP8;
    const int P = f8 ? (L.B <= 4 ? 1 : 2) : 0;
    if (P == 2 && L.B > 8)
        return fail(ERQ_EUNSUPPORTED, "tensor-core scan: e4m3 holds the split code parts only for B <= 8");
    if (P == 2 && L.Dq != 2 * (int64_t)L.D) return fail(ERQ_EINVAL, "tensor-core scan: split e4m3 needs doubled query rows");
    if (!(f8 ? (L.Q8 && L.qscale) : L.Qh != nullptr)) return fail(ERQ_EINVAL, "tensor-core scan: queries missing");
    if (!L.itemd || !L.itemq || !L.rowmeta || !L.tq || !L.work_ctr)
        return fail(ERQ_EINVAL, "tensor-core scan: item tables missing");
    if (!scan_tc_shape_ok(L.qn, L.kp)) return fail(ERQ_EINVAL, "tensor-core scan: no kernel for this item shape");
    tc::Args a;
    a.ck = L.ck;
    a.itemd = L.itemd; a.itemq = L.itemq; a.qn = L.qn; a.rowmeta = L.rowmeta; a.n_items = L.n_items;
    a.work_ctr = L.work_ctr;
    a.inter = L.inter; a.inter_cnt = L.inter_cnt; a.tq = L.tq; a.qscale = L.qscale; a.status = L.status;
    a.D = L.D; a.B = L.B; a.kp = L.kp; a.ip = L.ip;
    a.nkb = P == 1 ? (int)(L.Dq / 128) : L.D / KB;
    a.wait_ns = L.wait_ns ? L.wait_ns : kWaitNs;
    // a cluster probed by more queries than one item holds is read by several
    // items at about the same time (items are ordered row range first)
    a.codes_shared = L.nq * (int64_t)L.maxp > (int64_t)L.qn * L.nlist ? 1 : 0;
    a.stall_stage = L.stall_stage;
    const void* qb = f8 ? L.Q8 : L.Qh;
    const int64_t qrow = f8 ? L.Dq : 2 * (int64_t)L.D;
    if (L.kp <= 32 && L.qn > CfgA::QN) return scan_tc_form<CfgW>(P, L, a, qb, qrow, s);
    if (L.kp <= 32) return scan_tc_form<CfgA>(P, L, a, qb, qrow, s);
    return scan_tc_form<CfgB>(P, L, a, qb, qrow, s);
}

// Rotated queries -> e4m3 for the kind::f8f6f4 scan.  Per query row a power of
// two s = 2^(floor(log2 max|q'|) - 7) puts the largest magnitude in [128, 256)
// (e4m3's largest finite value is 448); every q'_i / s (exact) is rounded to
// the nearest e4m3 value, ties to even, from its FP32 bits: for |y| >= 2^-6 the
// 23-bit mantissa keeps its top 3 bits (carry into the exponent on overflow),
// below it y is a multiple of 2^-9 after rounding |y| * 2^9 to an integer
// (8 then being the smallest normal's code).  Columns D .. Dq-1 are zero.
// With dup (the split form of B = 5..8 codes, Dq = 2 D) every 64-coordinate
// block is written twice: byte 128 j + t holds coordinate 64 j + (t mod 64).
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

__global__ void quant_e4m3_kernel(const float* __restrict__ X, int64_t n, int D, int Dq, int dup,
                                  unsigned char* __restrict__ Y, float* __restrict__ scale) {
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
        for (int j = 0; j < 4; ++j) {
            const int c = dup ? (((i + j) >> 7) << 6) | ((i + j) & 63) : i + j;
            if (c < D) w |= e4m3_rn(x[c] * inv) << (8 * j);
        }
        *reinterpret_cast<uint32_t*>(y + i) = w;
    }
}

cudaError_t launch_quant_e4m3(const float* x, int64_t n, int D, int Dq, int dup, unsigned char* y, float* scale,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (Dq % 4 != 0 || (dup && Dq != 2 * D) || (!dup && Dq < D)) return cudaErrorInvalidValue;
    count_launch();
    quant_e4m3_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(x, n, D, Dq, dup, y, scale);
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
