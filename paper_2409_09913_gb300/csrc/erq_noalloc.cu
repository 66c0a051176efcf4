// erq_search_backward_noalloc: the query gradient of erq_search_backward for
// callers that cannot allocate device memory while they run, for example
// hosts that hand all device memory out of their own pool.
//
// The intermediate matrices of the backward pass (V, Wv and V's row
// exponents) live in one statically sized array in device global memory,
// declared at file scope below.  Every GPU that loads liberq.so holds this
// array until the process exits.  All calls share it, so calls that may run
// at the same time on the GPU (two streams, two threads) race on it and must
// be serialised by the caller.  The contents left by the previous call are
// never read: every element used is written first.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "erq_kernels.cuh"
#include "erq_search.cuh"

namespace erq {

// Scratch array shared by every allocation-free call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ERQ_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch per device

// The host-side symbol is only a stand-in; the device address must be looked
// up with the device current.  Done once per device, on the first call.
erq_status scratch_address(void** out) {
    int dev = 0;
    ERQ_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(ERQ_EUNSUPPORTED, "erq_search_backward_noalloc: device id too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "erq_search_backward_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ERQ_OK;
}
}  // namespace

}  // namespace erq

using namespace erq;

extern "C" erq_status erq_search_backward_noalloc(erq_index* ix, const float* Q, int64_t nq, int32_t nc,
                                                   const int64_t* ids, const float* grad_scores, float* grad_Q,
                                                   void* stream) {
    if (!ix || nq < 0 || nc < 0) return fail(ERQ_EINVAL, "erq_search_backward_noalloc: bad arguments");
    if (nq == 0) return ERQ_OK;
    if (!Q || !grad_Q || (nc > 0 && (!ids || !grad_scores)))
        return fail(ERQ_EINVAL, "erq_search_backward_noalloc: null pointer");
    const size_t mat = (size_t)nq * ix->D;
    const size_t mat_pad = (mat + 63) / 64 * 64;
    const size_t need = 2 * mat_pad * sizeof(float) + (size_t)nq * sizeof(int32_t) + 512;
    if (need > (size_t)ERQ_NOALLOC_SCRATCH_BYTES)
        return fail(ERQ_EINVAL, "erq_search_backward_noalloc: nq * D too large for the fixed scratch array "
                                "(needs 8 * nq * D + 4 * nq + 512 <= ERQ_NOALLOC_SCRATCH_BYTES bytes)");
    void* base = nullptr;
    ERQ_TRY(scratch_address(&base));
    float* V = (float*)base;
    float* Wv = V + mat_pad;
    int32_t* eV = (int32_t*)(Wv + mat_pad);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = launch_backward_gather(Q, ids, grad_scores, nq, nc, ix, 0, V, Wv, s)) != cudaSuccess)
        return cuda_fail(e, "backward gather");
    if ((e = launch_row_exp(V, nq, ix->D, eV, s)) != cudaSuccess) return cuda_fail(e, "backward exponents");
    if ((e = launch_gemm_tc(V, eV, nq, ix->P, ix->eP, ix->D, ix->D, grad_Q, ix->D, 0, Wv, nullptr, nullptr, ix->status,
                            s)) != cudaSuccess)
        return cuda_fail(e, "backward gemm");
    return ERQ_OK;
}
