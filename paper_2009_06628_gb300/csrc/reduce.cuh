// Block-level FP64 reduction helpers (deterministic order).
#pragma once

#include <cuda_runtime.h>

// Reduce K per-thread values over the block; thread 0 stores them to partials[blockIdx.x*K + k].
// Requires blockDim.x to be a multiple of 32 and at most 1024.
template <int K>
__device__ __forceinline__ void block_reduce_store(double* acc, double* partials) {
    __shared__ double sred[32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        acc[k] = v;
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sred[warp][k] = acc[k];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double v = lane < nw ? sred[lane][k] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) partials[(size_t)blockIdx.x * K + k] = v;
        }
    }
}

// One block of 256 threads sums nblocks partials of K components (fixed order).
__global__ void final_reduce_kernel(const double* __restrict__ partials, int nblocks, int K,
                                    double* __restrict__ out);
