// Reductions of the hot path in FP64: mass (integral of phi, Proposition 1), the parts of
// the energy functional (Eq. energy_functional), and the BLAS-1 building blocks of the
// Krylov solver.  Every reduction is two-pass and deterministic: a fixed grid writes one
// partial per block (warp shuffles, then shared memory), one block sums the partials in
// a fixed order.
#include <cuda_runtime.h>

#include "chns_internal.h"
#include "reduce.cuh"

namespace {

constexpr double GP = 0.78867513459481288225;  // (1 + 1/sqrt 3)/2
constexpr double GM = 0.21132486540518711775;  // (1 - 1/sqrt 3)/2

// Corner values of one element for scalar or vector nodal data (with hanging weights).
template <int D>
__device__ __forceinline__ void corner_parents(const DevMesh& m, int ent, int p[4], int& n) {
    if (ent >= 0) {
        n = 1;
        p[0] = ent;
    } else {
        const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
        p[0] = hp.x;
        p[1] = hp.y;
        p[2] = hp.z;
        p[3] = hp.w;
        n = hp.z < 0 ? 2 : 4;
    }
}

// One thread per element; K partial sums per block.
template <int D, int K, class Body>
__device__ void element_sum(const DevMesh& m, double* partials, Body body) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m.E; e += (int64_t)gridDim.x * blockDim.x)
        body(e, acc);
    block_reduce_store<K>(acc, partials);
}

template <int D>
__global__ void mass_kernel(DevMesh m, const double* __restrict__ U, double* partials) {
    constexpr int NC = 1 << D, NF = D + 3;
    element_sum<D, 1>(m, partials, [&](int64_t e, double* acc) {
        const double h = ldexp(m.hi - m.lo, -(int)m.level[e]);
        const double detJ = (D == 2) ? 0.25 * h * h : 0.125 * h * h * h;
        double phi_c[NC];
        for (int a = 0; a < NC; ++a) {
            int p[4], n;
            corner_parents<D>(m, m.e2n[e * NC + a], p, n);
            const double w = n == 1 ? 1.0 : (n == 2 ? 0.5 : 0.25);
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += w * U[(size_t)p[j] * NF + D + 1];
            phi_c[a] = s;
        }
        double sum = 0.0;
        for (int q = 0; q < NC; ++q) {
            double val = 0.0;
            for (int a = 0; a < NC; ++a) {
                double N = 1.0;
                for (int k = 0; k < D; ++k) N *= (((a >> k) & 1) == ((q >> k) & 1)) ? GP : GM;
                val += N * phi_c[a];
            }
            sum += val;
        }
        acc[0] += detJ * sum;
    });
}

template <int D>
__global__ void energy_kernel(DevMesh m, double alpha, double beta, double Cn, double inv_CnWe, double inv_Fr,
                              const double* __restrict__ U, double* partials) {
    constexpr int NC = 1 << D, NF = D + 3;
    const double unit = (m.hi - m.lo) / (double)((int64_t)1 << m.max_level);
    element_sum<D, 3>(m, partials, [&](int64_t e, double* acc) {
        const double h = ldexp(m.hi - m.lo, -(int)m.level[e]);
        const double inv_h = 1.0 / h;
        const double detJ = (D == 2) ? 0.25 * h * h : 0.125 * h * h * h;
        const double z0 = m.lo + unit * (double)m.anchor[e * D + D - 1];
        double uc[NC][D + 2];  // v, phi, phi* (clip at independent nodes)
        for (int a = 0; a < NC; ++a) {
            int p[4], n;
            corner_parents<D>(m, m.e2n[e * NC + a], p, n);
            const double w = n == 1 ? 1.0 : (n == 2 ? 0.5 : 0.25);
            for (int f = 0; f < D + 2; ++f) uc[a][f] = 0.0;
            for (int j = 0; j < n; ++j) {
                const double* u = U + (size_t)p[j] * NF;
                for (int k = 0; k < D; ++k) uc[a][k] += w * u[k];
                const double phi = u[D + 1];
                uc[a][D] += w * phi;
                uc[a][D + 1] += w * fmin(1.0, fmax(-1.0, phi));
            }
        }
        double kin = 0.0, fre = 0.0, grav = 0.0;
        for (int q = 0; q < NC; ++q) {
            double v[D], phi = 0.0, ps = 0.0, gphi[D];
            for (int k = 0; k < D; ++k) v[k] = gphi[k] = 0.0;
            for (int a = 0; a < NC; ++a) {
                double f[D], s[D];
                for (int k = 0; k < D; ++k) {
                    f[k] = (((a >> k) & 1) == ((q >> k) & 1)) ? GP : GM;
                    s[k] = ((a >> k) & 1) ? inv_h : -inv_h;
                }
                double N = 1.0;
                for (int k = 0; k < D; ++k) N *= f[k];
                for (int k = 0; k < D; ++k) {
                    double dN = s[k];
                    for (int j = 0; j < D; ++j)
                        if (j != k) dN *= f[j];
                    gphi[k] += dN * uc[a][D];
                    v[k] += N * uc[a][k];
                }
                phi += N * uc[a][D];
                ps += N * uc[a][D + 1];
            }
            const double rho = alpha * ps + beta;
            double vv = 0.0, gg = 0.0;
            for (int k = 0; k < D; ++k) {
                vv += v[k] * v[k];
                gg += gphi[k] * gphi[k];
            }
            const double psi = 0.25 * (phi * phi - 1.0) * (phi * phi - 1.0);
            kin += 0.5 * rho * vv;
            fre += psi + 0.5 * Cn * Cn * gg;
            const double zq = z0 + h * (((q >> (D - 1)) & 1) ? GP : GM);
            grav += rho * zq;
        }
        acc[0] += detJ * kin;
        acc[1] += detJ * fre * inv_CnWe;
        acc[2] += detJ * grav * inv_Fr;
    });
}

template <int K>
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* partials) {
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += a[i] * b[i];
    block_reduce_store<1>(acc, partials);
}

// out[j] = V_j . w for j < k (V_j = V + j*ld), processed 8 vectors per pass.
__global__ void multidot8_kernel(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ w,
                                 int64_t n, double* partials) {
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < k) acc[j] += V[(size_t)j * ld + i] * wi;
    }
    block_reduce_store<8>(acc, partials);
}

int reduce_blocks(int64_t work) {
    int64_t b = (work + 255) / 256;
    const int64_t cap = 4 * (int64_t)chns_num_sms();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

__global__ void final_reduce_kernel(const double* __restrict__ partials, int nblocks, int K,
                                    double* __restrict__ out) {
    __shared__ double sh[256];
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v += partials[(size_t)i * K + k];
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

cudaError_t launch_mass(const chns_mesh* mm, const double* U, double* out_dev, cudaStream_t s) {
    const DevMesh& m = mm->dm;
    const int nb = reduce_blocks(m.E);
    if (m.dim == 2)
        { mass_kernel<2><<<nb, 256, 0, s>>>(m, U, mm->d_partials); chns_count_launches(1); }
    else
        { mass_kernel<3><<<nb, 256, 0, s>>>(m, U, mm->d_partials); chns_count_launches(1); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    { final_reduce_kernel<<<1, 256, 0, s>>>(mm->d_partials, nb, 1, out_dev); chns_count_launches(1); }
    return cudaGetLastError();
}

cudaError_t launch_energy(const chns_mesh* mm, const PhysConst& pc, const double* U, double* out_dev3,
                          cudaStream_t s) {
    const DevMesh& m = mm->dm;
    const int nb = reduce_blocks(m.E);
    const double inv_CnWe = 1.0 / (pc.Cn * pc.We);
    if (m.dim == 2)
        { energy_kernel<2><<<nb, 256, 0, s>>>(m, pc.alpha, pc.beta, pc.Cn, inv_CnWe, pc.inv_Fr, U, mm->d_partials); chns_count_launches(1); }
    else
        { energy_kernel<3><<<nb, 256, 0, s>>>(m, pc.alpha, pc.beta, pc.Cn, inv_CnWe, pc.inv_Fr, U, mm->d_partials); chns_count_launches(1); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    { final_reduce_kernel<<<1, 256, 0, s>>>(mm->d_partials, nb, 3, out_dev3); chns_count_launches(1); }
    return cudaGetLastError();
}

cudaError_t launch_dot(const chns_mesh* mm, const double* a, const double* b, int64_t n, double* out_dev,
                       cudaStream_t s) {
    const int nb = reduce_blocks(n);
    { dot_kernel<1><<<nb, 256, 0, s>>>(a, b, n, mm->d_partials); chns_count_launches(1); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    { final_reduce_kernel<<<1, 256, 0, s>>>(mm->d_partials, nb, 1, out_dev); chns_count_launches(1); }
    return cudaGetLastError();
}

cudaError_t launch_multidot(const chns_mesh* mm, const double* V, int64_t ld, int k, const double* w, int64_t n,
                            double* out_dev, cudaStream_t s) {
    const int nb = reduce_blocks(n);
    for (int j0 = 0; j0 < k; j0 += 8) {
        const int kk = (k - j0) < 8 ? (k - j0) : 8;
        { multidot8_kernel<<<nb, 256, 0, s>>>(V + (size_t)j0 * ld, ld, kk, w, n, mm->d_partials); chns_count_launches(1); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        { final_reduce_kernel<<<1, 256, 0, s>>>(mm->d_partials, nb, 8, out_dev + j0); chns_count_launches(1); }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
