// chns_mass_static: the integral of phi with no allocation at call time.
//
// Some callers cannot call cudaMalloc when they need this number: code that runs
// while a framework's caching allocator owns the device memory budget (a raw
// cudaMalloc would fail or fragment the pool), or code on a path where cudaMalloc's
// implicit device synchronisation is not allowed.  This entry point keeps its scratch
// (the per-block partial sums of the reduction) in a file-scope device array, so it
// allocates nothing; the caller passes the input field and a device output scalar.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "chns_internal.h"
#include "reduce.cuh"

namespace {

constexpr int MS_THREADS = 256;
constexpr int MS_CHUNK = 16;                              // elements per thread
constexpr int MS_MAX_BLOCKS = 16384;                      // scratch: 16384 doubles = 128 KiB
constexpr int64_t MS_MAX_ELEMENTS = (int64_t)MS_MAX_BLOCKS * MS_THREADS * MS_CHUNK;  // 67,108,864
constexpr int MS_MAX_DEVICES = 64;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) double g_mass_scratch[MS_MAX_BLOCKS];

constexpr double MS_GP = 0.78867513459481288225;  // (1 + 1/sqrt 3)/2
constexpr double MS_GM = 0.21132486540518711775;  // (1 - 1/sqrt 3)/2

// One element: |e| / 2^d ... evaluated as the Gauss sum of the Q1 interpolant of phi.
template <int D>
__device__ __forceinline__ double element_phi_integral(const DevMesh& m, const double* __restrict__ U, int64_t e) {
    constexpr int NC = 1 << D, NF = D + 3;
    const double h = ldexp(m.hi - m.lo, -(int)m.level[e]);
    const double detJ = (D == 2) ? 0.25 * h * h : 0.125 * h * h * h;
    double phi_c[NC];
    for (int a = 0; a < NC; ++a) {
        const int ent = m.e2n[e * NC + a];
        double s;
        if (ent >= 0) {
            s = U[(size_t)ent * NF + D + 1];
        } else {
            const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
            if (hp.z < 0) {
                s = 0.5 * U[(size_t)hp.x * NF + D + 1] + 0.5 * U[(size_t)hp.y * NF + D + 1];
            } else {
                s = 0.25 * U[(size_t)hp.x * NF + D + 1] + 0.25 * U[(size_t)hp.y * NF + D + 1] +
                    0.25 * U[(size_t)hp.z * NF + D + 1] + 0.25 * U[(size_t)hp.w * NF + D + 1];
            }
        }
        phi_c[a] = s;
    }
    double sum = 0.0;
    for (int q = 0; q < NC; ++q) {
        double val = 0.0;
        for (int a = 0; a < NC; ++a) {
            double N = 1.0;
            for (int k = 0; k < D; ++k) N *= (((a >> k) & 1) == ((q >> k) & 1)) ? MS_GP : MS_GM;
            val += N * phi_c[a];
        }
        sum += val;
    }
    return detJ * sum;
}

// Pass 1: block b sums elements [b*256*CHUNK, (b+1)*256*CHUNK) into scratch[b].
template <int D>
__global__ void mass_static_partial_kernel(DevMesh m, const double* __restrict__ U, double* __restrict__ scratch) {
    double acc[1] = {0.0};
    const int64_t base = (int64_t)blockIdx.x * MS_THREADS * MS_CHUNK;
    for (int k = 0; k < MS_CHUNK; ++k) {
        const int64_t e = base + (int64_t)k * MS_THREADS + threadIdx.x;
        if (e < m.E) acc[0] += element_phi_integral<D>(m, U, e);
    }
    block_reduce_store<1>(acc, scratch);
}

// Pass 2: one block sums the partials in a fixed order and writes the result.
__global__ void mass_static_final_kernel(const double* __restrict__ scratch, int nblocks, double* __restrict__ out) {
    __shared__ double sh[MS_THREADS];
    double v = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += MS_THREADS) v += scratch[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = MS_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// Device address of the scratch array, resolved once per device (with that device
// current).  In host code the symbol name is only a host-side stand-in.
std::mutex g_ms_mutex;
double* g_ms_addr[MS_MAX_DEVICES] = {};

chns_status scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return chns_cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= MS_MAX_DEVICES) {
        chns_set_error("chns_mass_static: device ordinal beyond 63");
        return CHNS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_ms_mutex);
    if (!g_ms_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return chns_cuda_status(e, "cudaGetSymbolAddress(g_mass_scratch)");
        g_ms_addr[dev] = static_cast<double*>(p);
    }
    *out = g_ms_addr[dev];
    return CHNS_OK;
}

}  // namespace

extern "C" chns_status chns_mass_static(const chns_mesh* m, const double* U, double* out, void* stream) {
    if (!m || !U || !out) {
        chns_set_error("chns_mass_static: null argument");
        return CHNS_EINVAL;
    }
    if (chns_require_q1(m, "chns_mass_static") != CHNS_OK) return CHNS_EINVAL;
    if (m->dm.E > MS_MAX_ELEMENTS) {
        chns_set_error("chns_mass_static: the mesh has more than 67,108,864 elements (the static scratch "
                       "holds 16,384 block sums of 4,096 elements); use chns_mass");
        return CHNS_EINVAL;
    }
    // the scratch address is resolved for the current device, and the kernels read the
    // mesh's arrays: both must be on the same GPU
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return chns_cuda_status(de, "cudaGetDevice");
    if (dev != m->device) {
        chns_set_error("chns_mass_static: the mesh was created on device " + std::to_string(m->device) +
                       " but device " + std::to_string(dev) + " is current; make the mesh's device current");
        return CHNS_EINVAL;
    }
    double* scratch = nullptr;
    chns_status st = scratch_for_current_device(&scratch);
    if (st != CHNS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t per_block = (int64_t)MS_THREADS * MS_CHUNK;
    const int nblocks = (int)((m->dm.E + per_block - 1) / per_block);
    if (m->dm.dim == 2) {
        mass_static_partial_kernel<2><<<nblocks, MS_THREADS, 0, s>>>(m->dm, U, scratch);
    } else {
        mass_static_partial_kernel<3><<<nblocks, MS_THREADS, 0, s>>>(m->dm, U, scratch);
    }
    chns_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return chns_cuda_status(e, "mass_static_partial_kernel");
    mass_static_final_kernel<<<1, MS_THREADS, 0, s>>>(scratch, nblocks, out);
    chns_count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return chns_cuda_status(e, "mass_static_final_kernel");
    return CHNS_OK;
}
