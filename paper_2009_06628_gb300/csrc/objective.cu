// Derivatives of the quantities a rollout objective is built from:
//  * the free-energy part of E_tot (Eq. energy_functional),
//      F(phi; Cn) = 1/(Cn We) int psi(phi) + Cn/(2 We) int |grad phi|^2,
//    its gradient with respect to the nodal phi and its partial derivative in Cn;
//  * the reverse mode of the discrete potential right-hand side
//      b(phi; Cn)_a = (N_a, psi'(phi)) + Cn^2 (grad N_a, grad phi)
//    that defines mu^0 through M mu^0 = b (the potential equation of Definition 1 at
//    one time level): lambda^T db/dphi (a symmetric operator) and lambda^T db/dCn.
#include <cuda_runtime.h>

#include "chns_internal.h"
#include "reduce.cuh"

namespace {

constexpr double OGP = 0.78867513459481288225;  // (1 + 1/sqrt 3)/2
constexpr double OGM = 0.21132486540518711775;  // (1 - 1/sqrt 3)/2

template <int D>
__device__ __forceinline__ int corner_parents(const DevMesh& m, int64_t e, int a, int p[4]) {
    const int ent = m.e2n[e * (1 << D) + a];
    if (ent >= 0) {
        p[0] = ent;
        return 1;
    }
    const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
    p[0] = hp.x;
    p[1] = hp.y;
    p[2] = hp.z;
    p[3] = hp.w;
    return hp.z < 0 ? 2 : 4;
}

template <int D>
__device__ __forceinline__ void basis_at(int a, int q, double inv_h, double& N, double dN[D]) {
    double f[D], s[D];
    for (int k = 0; k < D; ++k) {
        f[k] = (((a >> k) & 1) == ((q >> k) & 1)) ? OGP : OGM;
        s[k] = ((a >> k) & 1) ? inv_h : -inv_h;
    }
    N = 1.0;
    for (int k = 0; k < D; ++k) N *= f[k];
    for (int k = 0; k < D; ++k) {
        double d = s[k];
        for (int j = 0; j < D; ++j)
            if (j != k) d *= f[j];
        dN[k] = d;
    }
}

// MODE 0: g_phi += dF/dphi (= b / (Cn We)), partials (int psi, int |grad phi|^2)
// MODE 1: y += (N psi''(phi) N + Cn^2 K) lambda, partial int grad lambda . grad phi
template <int D, int MODE>
__global__ void objective_kernel(DevMesh m, double Cn, double scale, const double* __restrict__ U,
                                 const double* __restrict__ lam, double* __restrict__ out, int out_stride,
                                 int out_field, double* partials) {
    constexpr int NC = 1 << D, NF = D + 3;
    double acc[2] = {0.0, 0.0};
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m.E; e += (int64_t)gridDim.x * blockDim.x) {
        const double h = ldexp(m.hi - m.lo, -(int)m.level[e]);
        const double inv_h = 1.0 / h, detJ = (D == 2) ? 0.25 * h * h : 0.125 * h * h * h;
        int par[NC][4], np[NC];
        double phi_c[NC], lam_c[NC];
        for (int a = 0; a < NC; ++a) {
            np[a] = corner_parents<D>(m, e, a, par[a]);
            const double w = np[a] == 1 ? 1.0 : (np[a] == 2 ? 0.5 : 0.25);
            double sp = 0.0, sl = 0.0;
            for (int j = 0; j < np[a]; ++j) {
                sp += w * U[(size_t)par[a][j] * NF + D + 1];
                if (MODE == 1) sl += w * lam[par[a][j]];
            }
            phi_c[a] = sp;
            lam_c[a] = sl;
        }
        double r[NC];
        for (int a = 0; a < NC; ++a) r[a] = 0.0;
        for (int q = 0; q < NC; ++q) {
            double phi = 0.0, lv = 0.0, gphi[D], glam[D];
            for (int k = 0; k < D; ++k) gphi[k] = glam[k] = 0.0;
            for (int a = 0; a < NC; ++a) {
                double N, dN[D];
                basis_at<D>(a, q, inv_h, N, dN);
                phi += N * phi_c[a];
                lv += N * lam_c[a];
                for (int k = 0; k < D; ++k) {
                    gphi[k] += dN[k] * phi_c[a];
                    glam[k] += dN[k] * lam_c[a];
                }
            }
            double gg = 0.0, gl = 0.0;
            for (int k = 0; k < D; ++k) {
                gg += gphi[k] * gphi[k];
                gl += glam[k] * gphi[k];
            }
            if (MODE == 0) {
                acc[0] += detJ * 0.25 * (phi * phi - 1.0) * (phi * phi - 1.0);
                acc[1] += detJ * gg;
            } else {
                acc[0] += detJ * gl;
            }
            for (int a = 0; a < NC; ++a) {
                double N, dN[D];
                basis_at<D>(a, q, inv_h, N, dN);
                double t;
                if (MODE == 0) {
                    t = N * (phi * phi * phi - phi);
                    for (int k = 0; k < D; ++k) t += Cn * Cn * dN[k] * gphi[k];
                } else {
                    t = N * (3.0 * phi * phi - 1.0) * lv;
                    for (int k = 0; k < D; ++k) t += Cn * Cn * dN[k] * glam[k];
                }
                r[a] += detJ * t;
            }
        }
        for (int a = 0; a < NC; ++a) {
            const double w = np[a] == 1 ? 1.0 : (np[a] == 2 ? 0.5 : 0.25);
            for (int j = 0; j < np[a]; ++j)
                atomicAdd(out + (size_t)par[a][j] * out_stride + out_field, scale * w * r[a]);
        }
    }
    block_reduce_store<2>(acc, partials);
}

int obj_blocks(int64_t E) {
    int64_t b = (E + 255) / 256;
    const int64_t cap = 4 * (int64_t)chns_num_sms();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

extern "C" chns_status chns_free_energy_grad(const chns_mesh* m, const chns_params* p, const double* U, double* g,
                                             double* dCn, void* stream) {
    if (chns_require_q1(m, "chns_free_energy_grad") != CHNS_OK) return CHNS_EINVAL;
    PhysConst pc;
    chns_status st = chns_check_params(m, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U || !g) { chns_set_error("null argument"); return CHNS_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const DevMesh& dm = m->dm;
    CHNS_CUDA(cudaMemsetAsync(g, 0, (size_t)dm.N * dm.nf * sizeof(double), s));
    const int nb = obj_blocks(dm.E);
    const double scale = 1.0 / (pc.Cn * pc.We);
    if (dm.dim == 2)
        objective_kernel<2, 0><<<nb, 256, 0, s>>>(dm, pc.Cn, scale, U, nullptr, g, dm.nf, dm.dim + 1, m->d_partials);
    else
        objective_kernel<3, 0><<<nb, 256, 0, s>>>(dm, pc.Cn, scale, U, nullptr, g, dm.nf, dm.dim + 1, m->d_partials);
    chns_count_launches(1);
    CHNS_CUDA(cudaGetLastError());
    double* res = m->d_partials + (size_t)m->n_partials * 8 - 16;
    final_reduce_kernel<<<1, 256, 0, s>>>(m->d_partials, nb, 2, res);
    chns_count_launches(1);
    CHNS_CUDA(cudaGetLastError());
    CHNS_CUDA(cudaMemcpyAsync(m->h_pinned, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHNS_CUDA(cudaStreamSynchronize(s));
    const double A = m->h_pinned[0], G = m->h_pinned[1];
    // dF/dCn = -A/(Cn^2 We) + G/(2 We)
    if (dCn) *dCn = -A / (pc.Cn * pc.Cn * pc.We) + G / (2.0 * pc.We);
    return CHNS_OK;
}

extern "C" chns_status chns_mu_rhs_vjp(const chns_mesh* m, const chns_params* p, const double* U, const double* lam,
                                       double* g_phi, double* dCn, void* stream) {
    if (chns_require_q1(m, "chns_mu_rhs_vjp") != CHNS_OK) return CHNS_EINVAL;
    PhysConst pc;
    chns_status st = chns_check_params(m, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U || !lam || !g_phi) { chns_set_error("null argument"); return CHNS_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const DevMesh& dm = m->dm;
    CHNS_CUDA(cudaMemsetAsync(g_phi, 0, (size_t)dm.N * sizeof(double), s));
    const int nb = obj_blocks(dm.E);
    if (dm.dim == 2)
        objective_kernel<2, 1><<<nb, 256, 0, s>>>(dm, pc.Cn, 1.0, U, lam, g_phi, 1, 0, m->d_partials);
    else
        objective_kernel<3, 1><<<nb, 256, 0, s>>>(dm, pc.Cn, 1.0, U, lam, g_phi, 1, 0, m->d_partials);
    chns_count_launches(1);
    CHNS_CUDA(cudaGetLastError());
    double* res = m->d_partials + (size_t)m->n_partials * 8 - 16;
    final_reduce_kernel<<<1, 256, 0, s>>>(m->d_partials, nb, 2, res);
    chns_count_launches(1);
    CHNS_CUDA(cudaGetLastError());
    CHNS_CUDA(cudaMemcpyAsync(m->h_pinned, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHNS_CUDA(cudaStreamSynchronize(s));
    // lambda^T db/dCn = 2 Cn int grad lambda . grad phi
    if (dCn) *dCn = 2.0 * pc.Cn * m->h_pinned[0];
    return CHNS_OK;
}
