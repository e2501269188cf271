// chns_fma_peak: measured CUDA-core FMA throughput (FP32 or FP64) of the current GPU,
// the denominator of the ALU roofline of the element kernels.
//
// Every thread runs 8 independent chains of x <- fma(x, a, b) (enough independent work
// per warp to cover the FMA latency) over all SMs, 4 blocks of 256 threads per SM; one
// FMA counts as 2 flops.  The result is only written out so the chains are not removed.
#include <cuda_runtime.h>

#include "chns_internal.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_BLOCKS_PER_SM = 4;
constexpr int PK_CHAINS = 8;
constexpr int PK_UNROLL = 16;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }

template <class T>
__global__ void __launch_bounds__(PK_THREADS) fma_probe_kernel(T* __restrict__ out, int iters, T a, T b) {
    T x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PK_CHAINS; ++k) x[k] = fma_t(x[k], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
cudaError_t run_probe(void* scratch, int grid, int iters, cudaStream_t s) {
    // x -> a x + b converges to b / (1 - a) = 1: no overflow, no denormals
    fma_probe_kernel<T><<<grid, PK_THREADS, 0, s>>>(static_cast<T*>(scratch), iters, T(0.999999), T(1e-6));
    chns_count_launches(1);
    return cudaGetLastError();
}

}  // namespace

extern "C" chns_status chns_fma_peak(int32_t precision, int32_t iters, void* scratch, int64_t scratch_bytes,
                                     double* flops_per_s, void* stream) {
    if ((precision != 0 && precision != 1) || iters < 1 || !scratch || !flops_per_s) {
        chns_set_error("chns_fma_peak: precision must be 0 (FP64) or 1 (FP32), iters >= 1, pointers non-null");
        return CHNS_EINVAL;
    }
    const int grid = PK_BLOCKS_PER_SM * chns_num_sms();
    const int64_t need = (int64_t)grid * PK_THREADS * (precision == 0 ? 8 : 4);
    if (scratch_bytes < need) {
        chns_set_error("chns_fma_peak: scratch must hold " + std::to_string(need) + " bytes");
        return CHNS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CHNS_CUDA(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err == cudaSuccess) {
        // one untimed launch (module load, clocks up), then the timed one
        err = precision == 0 ? run_probe<double>(scratch, grid, iters, s) : run_probe<float>(scratch, grid, iters, s);
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        if (err == cudaSuccess)
            err = precision == 0 ? run_probe<double>(scratch, grid, iters, s) : run_probe<float>(scratch, grid, iters, s);
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    }
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return chns_cuda_status(err, "chns_fma_peak");
    const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * grid * PK_THREADS;
    *flops_per_s = flops / (ms * 1e-3);
    return CHNS_OK;
}
