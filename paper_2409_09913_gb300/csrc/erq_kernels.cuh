// Device helpers and kernel launchers shared across translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <vector>

#include "erq_internal.cuh"

namespace erq {

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Inclusive prefix sum over the warp.
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---- k_linalg.cu
cudaError_t launch_rotate_fp64(const float* X, const int64_t* gather, const float* C, const int32_t* cl,
                               const float* P, float* out, int64_t n, int D, cudaStream_t s);
cudaError_t launch_sgemm(bool nt, const float* A, const float* B, float* C, int64_t M, int N, int K, float alpha,
                         const float* addend, cudaStream_t s);
cudaError_t launch_sqdist(const float* Q, const float* qn, const float* C, const float* cn, float* out, int64_t nq,
                          int nc, int D, cudaStream_t s);
cudaError_t launch_row_sqnorm(const float* X, int64_t n, int D, float* out, cudaStream_t s);
cudaError_t launch_normalize_rows(const float* X, int64_t n, int D, float* Y, cudaStream_t s);
cudaError_t launch_centroids(const float* X, const int64_t* list_off, const int64_t* list_ids, int nlist, int D,
                             float* C, int keep_empty, cudaStream_t s);
cudaError_t launch_group(const int32_t* assign, int64_t n, int nlist, int64_t* list_off, int64_t* list_ids,
                         int64_t* row_of, int32_t* cl_of_row, void* scratch, size_t scratch_bytes,
                         uint32_t* status, cudaStream_t s);
size_t group_scratch_bytes(int64_t n, int nlist);
cudaError_t launch_row_topk(const float* V, int64_t rows, int ncols, int64_t ld, int p, int32_t* out_idx,
                            float* out_val, int64_t ld_out, cudaStream_t s);
cudaError_t launch_row_topk_fast(const float* V, int64_t rows, int ncols, int64_t ld, int p, int32_t* out_idx,
                                 float* out_val, int64_t ld_out, cudaStream_t s);

// ---- k_gemm_tc.cu
cudaError_t launch_row_exp(const float* X, int64_t n, int K, int32_t* e, cudaStream_t s);
cudaError_t launch_split_hilo(const float* X, const int32_t* e, int64_t M, int K, __half* hi, __half* lo,
                              cudaStream_t s);
cudaError_t launch_query_prep(const float* X, int64_t M, int K, int32_t* e, float* sqn, __half* hi, __half* lo,
                              cudaStream_t s);
cudaError_t launch_gemm_tma(const __half* Ahi, const __half* Alo, const int32_t* eA, int64_t M, const __half* Bhi,
                            const __half* Blo, const int32_t* eB, int N, int K, float* C, int64_t ldc, int epi,
                            const float* rown, const float* coln, float* gmin, uint32_t* status, cudaStream_t s,
                            __half* Ch = nullptr);
cudaError_t launch_row_topk_groups(const float* V, const float* gmin, int64_t rows, int ncols, int64_t ld, int p,
                                   int32_t* out_idx, int64_t ld_out, cudaStream_t s);
cudaError_t launch_gemm_tc(const float* A, const int32_t* eA, int64_t M, const float* B, const int32_t* eB, int N,
                           int K, float* C, int64_t ldc, int epi, const float* addend, const float* rown,
                           const float* coln, uint32_t* status, cudaStream_t s);
cudaError_t launch_transpose(const float* X, int rows, int cols, float* out, cudaStream_t s);

// ---- k_encode.cu
cudaError_t launch_encode(const float* Rrot, int64_t n, int D, int B, uint8_t* codes, float* f_add, float* f_res,
                          double* stats, uint32_t* status, cudaStream_t s);
cudaError_t launch_gconst(const uint8_t* codes, const float* f_add, const float* f_res, const float* Cp,
                          const int32_t* cl_of_row, int64_t n, int D, int B, float* g_out, cudaStream_t s);

// ---- k_search.cu
struct SearchPlan;  // defined in k_search.cu

}  // namespace erq
