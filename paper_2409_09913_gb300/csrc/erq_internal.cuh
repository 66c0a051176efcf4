// Internal declarations shared by the CUDA translation units of liberq.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/erq.h"

namespace erq {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
erq_status fail(erq_status st, const std::string& msg);
erq_status cuda_fail(cudaError_t e, const char* what);

#define ERQ_CHECK_CUDA(expr)                                          \
    do {                                                              \
        cudaError_t _e = (expr);                                      \
        if (_e != cudaSuccess) return ::erq::cuda_fail(_e, #expr);    \
    } while (0)

#define ERQ_CHECK_LAUNCH(name)                                        \
    do {                                                              \
        cudaError_t _e = cudaGetLastError();                          \
        if (_e != cudaSuccess) return ::erq::cuda_fail(_e, name);     \
    } while (0)

#define ERQ_TRY(expr)                                                 \
    do {                                                              \
        erq_status _s = (expr);                                       \
        if (_s != ERQ_OK) return _s;                                  \
    } while (0)

// Device status word bits (written by kernels, read by erq_index_status).
enum : uint32_t { kStatusTimeout = 1u, kStatusBounds = 2u, kStatusRange = 4u };

// Checked build (-DERQ_CHECKS): bound checks on indices that kernels derive
// from device data.  A failed check sets kStatusBounds and bit 8 + site of the
// status word and the access is skipped (no trap); the next call that reads
// the status reports the sites.  In the normal build the checks compile away.
#ifdef ERQ_CHECKS
#define ERQ_DCHECK(cond, status, site) \
    ((cond) || (atomicOr((status), kStatusBounds | (1u << (8 + (site)))), false))
#else
#define ERQ_DCHECK(cond, status, site) true
#endif

// Limits the checked build compares device-derived indices against.
struct DevChecks {
    uint32_t* status = nullptr;
    int64_t lists = 0;       // candidate lists allocated (per-(query, item) lists)
    int64_t items = 0;       // work items allocated
    int64_t qlist = 0;       // entries of the per-cluster query lists
    int64_t rows = 0;        // stored rows N
    int nlist = 0;
};

// ---------------------------------------------------------------- keys
// Order-preserving map of an FP32 value to uint32 (NaN sorts last).
__host__ __device__ inline uint32_t float_to_ordered(float f) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float ordered_to_float(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
// Candidate key: (estimate, original id) in lexicographic order.
__host__ __device__ inline uint64_t make_key(float est, uint32_t id) {
    return ((uint64_t)float_to_ordered(est) << 32) | (uint64_t)id;
}
__host__ __device__ inline float key_value(uint64_t k) { return ordered_to_float((uint32_t)(k >> 32)); }
__host__ __device__ inline uint32_t key_id(uint64_t k) { return (uint32_t)(k & 0xffffffffu); }
constexpr uint64_t kEmptyKey = ~0ull;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Stored codes ybar_u: one byte per coordinate for B <= 8, a little-endian
// 16-bit word per coordinate for B = 9.
__host__ __device__ inline int code_bytes(int B) { return B > 8 ? 2 : 1; }
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t load_code(const uint8_t* codes, int B, int64_t i) {
    return B > 8 ? (uint32_t)reinterpret_cast<const uint16_t*>(codes)[i] : (uint32_t)codes[i];
}
#endif

// Process-wide count of kernel launches issued by the library.
void count_launch();

// ---------------------------------------------------------------- index
struct DeviceBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace erq

// The index object.  All pointers are device memory owned by the index.
struct erq_index {
    int64_t N = 0;
    int32_t D = 0, B = 0, nlist = 0, keep_raw = 0;
    int32_t normalized = 0;      // rows scaled to unit length at build (cosine metric)
    int64_t max_list = 0;
    float* P = nullptr;          // [D][D]
    float* PT = nullptr;         // [D][D] transpose of P (B operand of q' = P^T q)
    int32_t* eP = nullptr;       // [D] row exponents of P (tensor-core GEMM scaling)
    int32_t* ePT = nullptr;      // [D] row exponents of P^T
    int32_t* eC = nullptr;       // [nlist] row exponents of the centroids
    __half* PT_hi = nullptr;     // [D][D] P^T scaled by 2^-ePT, split into FP16 hi / lo parts
    __half* PT_lo = nullptr;
    __half* C_hi = nullptr;      // [nlist][D] centroids scaled by 2^-eC, FP16 hi / lo parts
    __half* C_lo = nullptr;
    float* C = nullptr;          // [nlist][D] centroids
    float* Cp = nullptr;         // [nlist][D] rotated centroids P^T c
    float* cnorm2 = nullptr;     // [nlist] ||c||^2 (FP32, for the probe)
    int64_t* list_off = nullptr; // [nlist+1]
    int64_t* list_ids = nullptr; // [N] original id of stored row
    int64_t* row_of = nullptr;   // [N] stored row of original id
    int32_t* cl_of_row = nullptr;// [N] cluster of stored row
    uint8_t* codes = nullptr;    // [N][D] ybar_u
    float* f_add = nullptr;      // [N]
    float* f_res = nullptr;      // [N]
    float* g_const = nullptr;    // [N] f_add - f_res * <ybar, c'>
    // tensor-core scan layout: every list padded to a multiple of 32 rows; codes
    // tiled as [Np/32 tiles][D/64 K blocks][32 rows][64 bytes]
    int64_t Np = 0;              // padded rows
    int64_t* poff = nullptr;     // [nlist+1] padded list offsets
    uint64_t* codes_p = nullptr; // [Np * D * B / 64] packed, tiled codes of the tensor-core scan
    float4* rowmeta = nullptr;   // [Np] {g, f_res/2, id, 0} per padded row (zeros for padding)
    float4* rowmeta1 = nullptr;  // [Np] {g1, f1/2, err1, 0}: 1-bit (MSB) factors of the two-stage search,
                                 //      computed at its first use from the raw rows
    float* X = nullptr;          // [N][D] raw rows, original order (keep_raw)
    uint32_t* status = nullptr;  // device status word
    std::vector<int64_t>* host_list_off = nullptr;  // host copy of list_off
    int32_t* corder = nullptr;   // [nlist] cluster ids by decreasing size (work-item order)
    // search workspace (grown on demand)
    void* ws = nullptr;          // phase-A / build workspace
    size_t ws_bytes = 0;
    void* ws_b = nullptr;        // phase-B workspace (data-dependent sizes)
    void* ws_ts = nullptr;       // two-stage search scratch (grown on demand, kept)
    size_t ws_ts_bytes = 0;
    size_t ws_b_bytes = 0;
    void* io = nullptr;          // device staging of erq_search_host
    size_t io_bytes = 0;
    void* pinned = nullptr;      // pinned host staging for erq_search_host
    static constexpr int kTimingRing = 512;   // timed searches whose phase events are kept
    cudaEvent_t* ev_ring = nullptr;  // [kTimingRing][7] phase boundaries of timed searches
    int64_t timing_seq = 0;      // timed searches so far
    int64_t timing_base = 0;     // first timed search not yet summed by erq_search_timing_total
    int timed = 0;               // 1 when the last search was timed
    int64_t last_stats[4] = {};  // pairs, distinct rows, work items, lists of the last search
    // scan work-item shape (queries per item qn, rows per item rr): forced by
    // erq_set_scan_config, else the autotuned entry of the k' class when its
    // queries x nprobe is within 4x of the search's, else a heuristic
    int force_qn = 0, force_rr = 0;
    struct ScanTune { int valid = 0; int64_t work = 0; int qn = 0, rr = 0; } tune[2];
    int last_qn = 0, last_rr = 0;
    unsigned int* dctr = nullptr;          // dynamic work-item counter of the tensor-core scan
    unsigned long long wait_ns = 0;        // limit of the scan's bounded waits (0 = the default 2 s)
    long long stall_stage = -1;            // test stall of the scan's bounded-wait path (-1 = none)
    unsigned long long* dstats = nullptr;  // [4] device counters of the last search: pairs, distinct rows,
                                           //     tensor-core row blocks, row blocks x padded queries
    size_t pinned_bytes = 0;
    int64_t device_bytes = 0;
};
