// Newton's method of Section 3.4, matrix-free: each Newton iteration solves
// J dU = -R (Eq. newton_linear_system) with right-preconditioned restarted GMRES whose
// operator is the J x element kernel (FP32 in mixed mode, FP64 otherwise) and whose
// preconditioner is nodal block-Jacobi (plus the pressure Schur and Cahn-Hilliard
// blocks); orthogonalisation (classical Gram-Schmidt with selective re-orthogonalisation),
// dots, norms, the residual and the update stay FP64 on the device.  With the pressure
// level set by its mean (pin mode 2) J is singular (constant pressure); GMRES runs on
// J + u m_p^T / |Omega| instead, which is nonsingular and has the zero-mean solution of
// J dU = -R.  Gram-Schmidt (including the decision to re-orthogonalise) and the next
// Arnoldi vector stay on the device; the Hessenberg column goes to the host for the
// Givens update, and that read-back overlaps the next vector's operator application,
// which is queued before the host waits.  Also: the consistent initial chemical
// potential by CG.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

#include "chns_internal.h"
#include "pointwise.cuh"
#include "reduce.cuh"

struct SolverWS {
    int restart = 0;
    int64_t n = 0, N = 0;
    double* V = nullptr;     // (restart + 1) * n Arnoldi basis
    double* w = nullptr;     // n
    double* R = nullptr;     // n residual
    double* dU = nullptr;    // n Newton update
    double* z64 = nullptr;   // n
    double* t64 = nullptr;   // n
    double* S = nullptr;     // n row scaling 1/|diag J| of the current linearisation
    double* Sd = nullptr;    // n its inverse |diag J| (identity rows: 1)
    double* S0 = nullptr;    // n row scaling of the first Newton iterate (norm of the step)
    double* SR = nullptr;    // n scaled residual
    float* Uo32 = nullptr;   // n
    float* Us32 = nullptr;   // n
    float* z32 = nullptr;    // n
    float* y32 = nullptr;    // n
    float* Pblk32 = nullptr; // N * nf * nf block diagonal (FP32 build)
    double* Pblk64 = nullptr;
    float* Pinv32 = nullptr; // inverted blocks
    double* Pinv64 = nullptr;
    double* sc = nullptr;    // device scalars
    double* hsc = nullptr;   // pinned host scalars
    cudaEvent_t ev[16] = {};  // J x, preconditioner build / apply and Gram-Schmidt timing (two sets
                              // of J x / apply events alternate between Arnoldi steps)
    // pressure Schur-complement approximation (FP32)
    float* ce = nullptr;     // E element coefficients
    float* kdinv = nullptr;  // N inverse diagonal
    // CUDA graphs of the pressure Schur apply (2 + 2 (degree - 1) launches), captured on
    // a private stream per (input, output, output type) and Chebyshev set-up
    struct SchurGraph {
        cudaGraphExec_t exec = nullptr;
        const void* vin = nullptr;
        void* zout = nullptr;
        size_t to = 0;
        int gen = -1;
        int nk = 0;   // kernels in the graph (launch accounting)
    } sgraph[4];
    cudaStream_t cap = nullptr;
    int schur_gen = 0;
    bool no_graphs = false;
    // CUDA graphs of the Gram-Schmidt sequence of Arnoldi step j (its kernels take k = j + 1
    // and fixed workspace pointers), captured at first use
    cudaGraphExec_t orth_exec[257] = {};
    float* kbnd = nullptr;   // N bounds of the absolute row sums of the Schur Laplacian
    unsigned int* kmax = nullptr;  // max_p kbnd[p] / diag[p] (float bits)
    float* cr = nullptr;     // N Chebyshev work vectors
    float* cx = nullptr;
    float* cd = nullptr;
    float* cy = nullptr;
    double* part = nullptr;  // per-block partials of the fused orthogonalisation reductions
    // Cahn-Hilliard block (pc_type 2), FP32 nodal work arrays
    float* ch_dinv = nullptr;  // inverse diagonal of M + eps K
    float* ch_ml = nullptr;    // lumped mass (node integrals)
    float* ch_psi2 = nullptr;  // psi''(phi~) at the nodes
    float* ch_a = nullptr;
    float* ch_b = nullptr;
    float* ch_c = nullptr;
    float* ch_rm = nullptr;
    std::vector<float> ch_c1, ch_c2;
    float ch_inv_theta = 0.0f, ch_eps = 0.0f;
    std::vector<float> cheb_c1, cheb_c2;
    float cheb_inv_theta = 0.0f;
    int kref_dim = 0;
};

void chns_solver_ws_free(SolverWS* ws) {
    if (!ws) return;
    for (auto& g : ws->sgraph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& g : ws->orth_exec)
        if (g) cudaGraphExecDestroy(g);
    if (ws->cap) cudaStreamDestroy(ws->cap);
    cudaFree(ws->V);
    cudaFree(ws->w);
    cudaFree(ws->R);
    cudaFree(ws->dU);
    cudaFree(ws->z64);
    cudaFree(ws->t64);
    cudaFree(ws->S);
    cudaFree(ws->Sd);
    cudaFree(ws->S0);
    cudaFree(ws->SR);
    cudaFree(ws->Uo32);
    cudaFree(ws->Us32);
    cudaFree(ws->z32);
    cudaFree(ws->y32);
    cudaFree(ws->Pblk32);
    cudaFree(ws->Pblk64);
    cudaFree(ws->Pinv32);
    cudaFree(ws->Pinv64);
    cudaFree(ws->sc);
    cudaFree(ws->ce);
    cudaFree(ws->kdinv);
    cudaFree(ws->kbnd);
    cudaFree(ws->kmax);
    cudaFree(ws->cr);
    cudaFree(ws->cx);
    cudaFree(ws->cd);
    cudaFree(ws->cy);
    cudaFree(ws->part);
    cudaFree(ws->ch_dinv);
    cudaFree(ws->ch_ml);
    cudaFree(ws->ch_psi2);
    cudaFree(ws->ch_a);
    cudaFree(ws->ch_b);
    cudaFree(ws->ch_c);
    cudaFree(ws->ch_rm);
    if (ws->hsc) cudaFreeHost(ws->hsc);
    for (auto& e : ws->ev)
        if (e) cudaEventDestroy(e);
    delete ws;
}

namespace {

constexpr int MAXSC = 1024;
constexpr int ORTH_MAX_BX = 1024;   // row blocks of the fused orthogonalisation kernels

chns_status ensure_ws(chns_mesh* m, int restart) {
    SolverWS* ws = m->ws;
    if (ws && ws->restart >= restart) return CHNS_OK;
    if (ws) chns_solver_ws_free(ws);
    m->ws = nullptr;
    ws = new SolverWS();
    ws->restart = restart;
    ws->N = m->dm.N;
    ws->n = m->dm.N * m->dm.nf;
    const size_t n = (size_t)ws->n, nb = (size_t)m->dm.N * m->dm.nf * m->dm.nf;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    A((void**)&ws->V, (size_t)(restart + 1) * n * sizeof(double));
    A((void**)&ws->w, n * sizeof(double));
    A((void**)&ws->R, n * sizeof(double));
    A((void**)&ws->dU, n * sizeof(double));
    A((void**)&ws->z64, n * sizeof(double));
    A((void**)&ws->t64, n * sizeof(double));
    A((void**)&ws->S, n * sizeof(double));
    A((void**)&ws->Sd, n * sizeof(double));
    A((void**)&ws->S0, n * sizeof(double));
    A((void**)&ws->SR, n * sizeof(double));
    A((void**)&ws->Uo32, n * sizeof(float));
    A((void**)&ws->Us32, n * sizeof(float));
    A((void**)&ws->z32, n * sizeof(float));
    A((void**)&ws->y32, n * sizeof(float));
    A((void**)&ws->Pblk32, nb * sizeof(float));
    A((void**)&ws->Pblk64, nb * sizeof(double));
    A((void**)&ws->Pinv32, nb * sizeof(float));
    A((void**)&ws->Pinv64, nb * sizeof(double));
    A((void**)&ws->sc, MAXSC * sizeof(double));
    A((void**)&ws->ce, (size_t)m->dm.E * sizeof(float));
    A((void**)&ws->kdinv, (size_t)m->dm.N * sizeof(float));
    A((void**)&ws->kbnd, (size_t)m->dm.N * sizeof(float));
    A((void**)&ws->kmax, sizeof(unsigned int));
    A((void**)&ws->cr, (size_t)m->dm.N * sizeof(float));
    A((void**)&ws->cx, (size_t)m->dm.N * sizeof(float));
    A((void**)&ws->cd, (size_t)m->dm.N * sizeof(float));
    A((void**)&ws->cy, (size_t)m->dm.N * sizeof(float));
    A((void**)&ws->part, (size_t)ORTH_MAX_BX * (MAXSC / 32 + 1) * 9 * sizeof(double));
    for (float** p : {&ws->ch_dinv, &ws->ch_ml, &ws->ch_psi2, &ws->ch_a, &ws->ch_b, &ws->ch_c, &ws->ch_rm})
        A((void**)p, (size_t)m->dm.N * sizeof(float));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ws->hsc, MAXSC * sizeof(double));
    for (auto& ev : ws->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
        chns_solver_ws_free(ws);
        return chns_cuda_status(e, "cudaMalloc(solver workspace)");
    }
    m->ws = ws;
    return CHNS_OK;
}

// ---------------- BLAS-1 ----------------
__global__ void copy64_kernel(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}
__global__ void to32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
__global__ void to64_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}
// w -= sum_{j<k} h[j] V_j  (h in device memory)
__global__ void gs_update_kernel(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ h,
                                 double* __restrict__ w, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int j = 0; j < k; ++j) s -= h[j] * V[(size_t)j * ld + i];
        w[i] = s;
    }
}
// Fused h = V^T w for all k basis vectors (blockIdx.y picks 8 of them) and, in chunk 0,
// also w . w: partials[(chunk * gridDim.x + block) * 9 + j].  The 8 dot products of a
// warp are reduced by recursive halving (each exchange level hands half of the
// remaining values to the partner lane): 9 FP64 shuffle-adds per warp instead of 40,
// which matters because every FP64 add runs on the narrow FP64 pipe.
__global__ void orth_dots_kernel(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ w,
                                 int64_t n, double* __restrict__ partials, const double* __restrict__ pred) {
    if (pred && pred[0] == 0.0) return;   // second pass not needed (decided on the device)
    const int chunk = blockIdx.y;
    const int j0 = chunk * 8;
    const int kk = min(8, k - j0);
    double acc[8];
    double nrm = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    const double* Vc = V + (size_t)j0 * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < kk) acc[j] += Vc[(size_t)j * ld + i] * wi;
        if (chunk == 0) nrm += wi * wi;
    }
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // 8 -> 4 values (lane bit 4 keeps the upper half), 4 -> 2 (bit 3), 2 -> 1 (bit 2)
    double t4[4], t2[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const double keep = up ? acc[4 + t] : acc[t];
            const double give = up ? acc[t] : acc[4 + t];
            t4[t] = keep + __shfl_xor_sync(full, give, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const double keep = up ? t4[2 + t] : t4[t];
            const double give = up ? t4[t] : t4[2 + t];
            t2[t] = keep + __shfl_xor_sync(full, give, 8);
        }
    }
    const bool up4 = lane & 4;
    double t1 = (up4 ? t2[1] : t2[0]) + __shfl_xor_sync(full, up4 ? t2[0] : t2[1], 4);
    t1 += __shfl_xor_sync(full, t1, 2);
    t1 += __shfl_xor_sync(full, t1, 1);
    // lane holds the warp sum of value ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)
    __shared__ double sred[32][9];
    if ((lane & 3) == 0) sred[warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = t1;
    if (chunk == 0) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(full, nrm, off);
        if (lane == 0) sred[warp][8] = nrm;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        if (threadIdx.x < 8 || chunk == 0)
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) v += sred[w2][threadIdx.x];
        partials[((size_t)chunk * gridDim.x + blockIdx.x) * 9 + threadIdx.x] = v;
    }
}
// out[j] = sum over row blocks (one block per chunk, one warp per value), out_norm = w.w
__global__ void orth_dots_final_kernel(const double* __restrict__ partials, int nbx, int k, double* __restrict__ out,
                                       double* __restrict__ out_norm, const double* __restrict__ pred) {
    if (pred && pred[0] == 0.0) return;
    const int chunk = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // 9 warps
    const int j = warp;
    if (j >= 9) return;
    if (j < 8 && chunk * 8 + j >= k) return;
    if (j == 8 && chunk != 0) return;
    double v = 0.0;
    for (int b = lane; b < nbx; b += 32) v += partials[((size_t)chunk * nbx + b) * 9 + j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) {
        if (j < 8) out[chunk * 8 + j] = v;
        else out_norm[0] = v;
    }
}
// w -= sum_{j<k} h[j] V_j, and per-block partials of the new w . w
__global__ void gs_update_norm_kernel(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ h,
                                      double* __restrict__ w, int64_t n, double* __restrict__ partials,
                                      const double* __restrict__ pred) {
    if (pred && pred[0] == 0.0) return;
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int j = 0; j < k; ++j) s -= h[j] * V[(size_t)j * ld + i];
        w[i] = s;
        acc[0] += s * s;
    }
    block_reduce_store<1>(acc, partials);
}
// Second Gram-Schmidt pass only on severe cancellation (|w'|^2 < 0.01 |w|^2 after the
// first pass; on GB300 every pass is bound by the FP64 pipe): the flag goes to sc[605]
// for the predicated second-pass kernels; when the pass is skipped its coefficients
// sc[256..256+k) are zeroed and the norm sc[601] is carried to sc[603], so the host
// always reads h = h1 + h2 and the final |w|^2 from the same slots.
__global__ void reorth_decide_kernel(double* __restrict__ sc, int k) {
    const bool again = sc[601] < 0.01 * sc[600];
    if (!again)
        for (int i = threadIdx.x; i < k; i += blockDim.x) sc[256 + i] = 0.0;
    if (threadIdx.x == 0) {
        sc[605] = again ? 1.0 : 0.0;
        if (!again) sc[603] = sc[601];
    }
}
// final_reduce_kernel for one component (same fixed order), skipped when pred[0] == 0
__global__ void final_reduce1_pred_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out,
                                          const double* __restrict__ pred) {
    if (pred && pred[0] == 0.0) return;
    __shared__ double sh[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v += partials[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}
// next Arnoldi vector v = w / sqrt(nrm[0]) (zero on breakdown, which the host reports)
__global__ void scale_next_kernel(const double* __restrict__ w, double* __restrict__ v, int64_t n,
                                  const double* __restrict__ nrm) {
    const double a = nrm[0] > 0.0 ? 1.0 / sqrt(nrm[0]) : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = a * w[i];
}
// sum_n m_n (a + b - c)[n*NF + f] into per-block partials (the phi-mass change of a
// Newton update: a = U, b = dU, c = U^k)
__global__ void field_mass3_kernel(const double* __restrict__ m, const double* __restrict__ a,
                                   const double* __restrict__ b, const double* __restrict__ c, int NF, int f,
                                   int64_t N, double* partials) {
    double acc[1] = {0.0};
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const size_t i = (size_t)n * NF + f;
        acc[0] += m[n] * ((a[i] + b[i]) - c[i]);
    }
    block_reduce_store<1>(acc, partials);
}
// u = sum_{j<k} y[j] V_j (y host-provided via device scalars)
__global__ void combine_kernel(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ y,
                               double* __restrict__ u, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += y[j] * V[(size_t)j * ld + i];
        u[i] = s;
    }
}
// y = s .* x (FP32 or FP64 x)
template <class T>
__global__ void scale_vec_kernel(const T* x, const double* __restrict__ sv, double* y,
                                 int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = sv[i] * (double)x[i];
}
// y = x .* d (d = 1/S, stored, so no FP64 division)
__global__ void unscale_kernel(const double* __restrict__ x, const double* __restrict__ d, double* __restrict__ y,
                               int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * d[i];
}
__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}
// y = a*x + b*y
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = 8 * (int64_t)chns_num_sms();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ---------------- block-Jacobi preconditioner ----------------
// Diagonal n_f x n_f block of every independent node, from the element-corner self
// blocks d r_e[a] / d u_e[a] (forward mode with unit tangents).  Hanging corners are
// skipped: the preconditioner is approximate there (it only affects convergence).
template <int D, class T>
__global__ void __launch_bounds__(128) pc_build_kernel(DevMesh m, PCst<T> c, T inv_dt, const T* __restrict__ Uo,
                                                       const T* __restrict__ Un, T* __restrict__ blk,
                                                       float* __restrict__ ce, double ce_scale);

constexpr double GPc = 0.78867513459481288225, GMc = 0.21132486540518711775;

template <int D, class T>
struct PB {
    T N, dN[D], d2N[D == 2 ? 1 : 3];
};
template <int D, class T>
__device__ __forceinline__ PB<D, T> pbasis(int a, int q, T inv_h) {
    T f[D], s[D];
    for (int k = 0; k < D; ++k) {
        f[k] = (((a >> k) & 1) == ((q >> k) & 1)) ? T(GPc) : T(GMc);
        s[k] = ((a >> k) & 1) ? inv_h : -inv_h;
    }
    PB<D, T> b;
    if constexpr (D == 2) {
        b.N = f[0] * f[1];
        b.dN[0] = s[0] * f[1];
        b.dN[1] = f[0] * s[1];
        b.d2N[0] = s[0] * s[1];
    } else {
        b.N = f[0] * f[1] * f[2];
        b.dN[0] = s[0] * f[1] * f[2];
        b.dN[1] = f[0] * s[1] * f[2];
        b.dN[2] = f[0] * f[1] * s[2];
        b.d2N[0] = s[0] * s[1] * f[2];
        b.d2N[1] = s[0] * f[1] * s[2];
        b.d2N[2] = f[0] * s[1] * s[2];
    }
    return b;
}

template <int D, class T>
__global__ void __launch_bounds__(128) pc_build_kernel(DevMesh m, PCst<T> c, T inv_dt, const T* __restrict__ Uo,
                                                       const T* __restrict__ Un, T* __restrict__ blk,
                                                       float* __restrict__ ce, double ce_scale) {
    constexpr int NC = 1 << D, NF = D + 3, NH = (D == 2) ? 1 : 3, EPB = 128 / NC;
    __shared__ T s_ut[EPB][NC][NF], s_dd[EPB][NC][D + 1], s_ps[EPB][NC];
    __shared__ int s_node[EPB][NC];
    __shared__ unsigned char s_mask[EPB][NC];
    const int le = threadIdx.x / NC, t = threadIdx.x % NC;
    const int64_t e = (int64_t)blockIdx.x * EPB + le;
    const bool valid = e < m.E;
    T inv_h = T(1), detJ = T(0);
    if (valid) {
        const int ent = m.e2n[e * NC + t];
        int p[4] = {0, 0, 0, 0}, np = 1;
        if (ent >= 0) {
            p[0] = ent;
        } else {
            const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
            p[0] = hp.x;
            p[1] = hp.y;
            p[2] = hp.z;
            p[3] = hp.w;
            np = hp.z < 0 ? 2 : 4;
        }
        const T wt = np == 1 ? T(1) : (np == 2 ? T(0.5) : T(0.25));
        T so[NF], sn[NF], ps = T(0);
        unsigned mask = 0;
        for (int f = 0; f < NF; ++f) so[f] = sn[f] = T(0);
        for (int j = 0; j < np; ++j) {
            T o[NF], n[NF];
            for (int f = 0; f < NF; ++f) {
                o[f] = Uo[(size_t)p[j] * NF + f];
                n[f] = Un[(size_t)p[j] * NF + f];
                so[f] += wt * o[f];
                sn[f] += wt * n[f];
            }
            const T avg = T(0.5) * (o[D + 1] + n[D + 1]);
            if (avg <= T(1) && avg >= T(-1)) mask |= 1u << j;
            ps += wt * (avg > T(1) ? T(1) : (avg < T(-1) ? T(-1) : avg));
        }
        for (int f = 0; f < NF; ++f) s_ut[le][t][f] = T(0.5) * (so[f] + sn[f]);
        for (int i = 0; i < D; ++i) s_dd[le][t][i] = sn[i] - so[i];
        s_dd[le][t][D] = sn[D + 1] - so[D + 1];
        s_ps[le][t] = ps;
        s_node[le][t] = ent;
        s_mask[le][t] = (unsigned char)(mask & 1u);
        const T h = T(ldexp(m.hi - m.lo, -(int)m.level[e]));
        inv_h = T(1) / h;
        detJ = (D == 2) ? T(0.25) * h * h : T(0.125) * h * h * h;
    }
    __syncwarp();
    if (!valid) return;  // the remaining code uses only shuffles within the element's lanes
    const int q = t;
    const T g = T(4) * inv_h * inv_h;
    // primal inputs at Gauss point q
    QPIn<D, T> X;
    {
        X.p = X.phi = X.mu = X.phidt = X.divnew = X.ps = T(0);
        for (int k = 0; k < D; ++k) {
            X.v[k] = X.gp[k] = X.gphi[k] = X.gmu[k] = X.vdt[k] = X.gps[k] = T(0);
            for (int j = 0; j < D; ++j) X.gv[k][j] = T(0);
        }
        for (int k = 0; k < NH; ++k) X.H[k] = T(0);
        for (int a = 0; a < NC; ++a) {
            const PB<D, T> b = pbasis<D, T>(a, q, inv_h);
            const T* u = s_ut[le][a];
            for (int i = 0; i < D; ++i) {
                X.v[i] += b.N * u[i];
                for (int k = 0; k < D; ++k) X.gv[i][k] += b.dN[k] * u[i];
                X.vdt[i] += b.N * s_dd[le][a][i];
                X.divnew += b.dN[i] * (u[i] + T(0.5) * s_dd[le][a][i]);
            }
            X.p += b.N * u[D];
            X.phi += b.N * u[D + 1];
            X.mu += b.N * u[D + 2];
            for (int k = 0; k < D; ++k) {
                X.gp[k] += b.dN[k] * u[D];
                X.gphi[k] += b.dN[k] * u[D + 1];
                X.gmu[k] += b.dN[k] * u[D + 2];
                X.gps[k] += b.dN[k] * s_ps[le][a];
            }
            for (int k = 0; k < NH; ++k) X.H[k] += b.d2N[k] * u[D + 1];
            X.phidt += b.N * s_dd[le][a][D];
            X.ps += b.N * s_ps[le][a];
        }
        for (int i = 0; i < D; ++i) X.vdt[i] *= inv_dt;
        X.phidt *= inv_dt;
    }
    const unsigned lanes = ((1u << NC) - 1u) << ((threadIdx.x & 31) & ~(NC - 1));
    {
        // coefficient of the pressure Schur-complement approximation on this element:
        // dt/(2 We) times the mean of 1/rho(phi*) over the Gauss points
        T ir = T(1) / (c.alpha * X.ps + c.beta);
        for (int off = NC / 2; off > 0; off >>= 1) ir += __shfl_xor_sync(lanes, ir, off);
        if (q == 0) ce[e] = (float)(ce_scale * (double)ir / NC);
    }
    for (int a = 0; a < NC; ++a) {
        const int node = s_node[le][a];
        const PB<D, T> b = pbasis<D, T>(a, q, inv_h);
        for (int gf = 0; gf < NF; ++gf) {
            // unit tangent in field gf at corner a (averages move by 1/2, differences by 1)
            QPIn<D, Dual<T>> XD;
            const T hf = T(0.5);
            for (int i = 0; i < D; ++i) {
                XD.v[i] = Dual<T>(X.v[i], gf == i ? hf * b.N : T(0));
                for (int k = 0; k < D; ++k) XD.gv[i][k] = Dual<T>(X.gv[i][k], gf == i ? hf * b.dN[k] : T(0));
                XD.vdt[i] = Dual<T>(X.vdt[i], gf == i ? inv_dt * b.N : T(0));
                XD.gp[i] = Dual<T>(X.gp[i], gf == D ? hf * b.dN[i] : T(0));
                XD.gphi[i] = Dual<T>(X.gphi[i], gf == D + 1 ? hf * b.dN[i] : T(0));
                XD.gmu[i] = Dual<T>(X.gmu[i], gf == D + 2 ? hf * b.dN[i] : T(0));
                const T pst = (gf == D + 1 && s_mask[le][a]) ? hf * b.dN[i] : T(0);
                XD.gps[i] = Dual<T>(X.gps[i], pst);
            }
            XD.p = Dual<T>(X.p, gf == D ? hf * b.N : T(0));
            XD.phi = Dual<T>(X.phi, gf == D + 1 ? hf * b.N : T(0));
            XD.mu = Dual<T>(X.mu, gf == D + 2 ? hf * b.N : T(0));
            for (int k = 0; k < NH; ++k) XD.H[k] = Dual<T>(X.H[k], gf == D + 1 ? hf * b.d2N[k] : T(0));
            XD.phidt = Dual<T>(X.phidt, gf == D + 1 ? inv_dt * b.N : T(0));
            T dv = T(0);
            if (gf < D) dv = b.dN[gf];
            XD.divnew = Dual<T>(X.divnew, dv);
            XD.ps = Dual<T>(X.ps, (gf == D + 1 && s_mask[le][a]) ? hf * b.N : T(0));
            QPOut<D, Dual<T>> F;
            pointwise<D, Dual<T>, T>(XD, c, g, F);
            for (int f = 0; f < NF; ++f) {
                T v = b.N * F.f0[f].d;
                for (int k = 0; k < D; ++k) v += b.dN[k] * F.f1[f][k].d;
                v *= detJ;
                for (int off = NC / 2; off > 0; off >>= 1) v += __shfl_xor_sync(lanes, v, off);
                if (q == 0 && node >= 0) atomicAdd(blk + ((size_t)node * NF + f) * NF + gf, v);
            }
        }
    }
}

// Replace Dirichlet / pin rows by identity rows and invert every block (Gauss-Jordan
// with partial pivoting in FP64).
template <class TB, class TI>
__global__ void pc_invert_kernel(DevMesh m, const TB* __restrict__ blk, TI* __restrict__ inv, int pin,
                                 double* __restrict__ scale, double* __restrict__ unscale, int decouple_p) {
    const int NF = m.nf, D = m.dim;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= m.N) return;
    double A[6][12];
    for (int i = 0; i < NF; ++i)
        for (int j = 0; j < NF; ++j) {
            A[i][j] = (double)blk[((size_t)n * NF + i) * NF + j];
            A[i][NF + j] = (i == j) ? 1.0 : 0.0;
        }
    const unsigned fl = m.nflag[n];
    for (int i = 0; i < NF; ++i) {
        const bool idrow = (i < D && ((fl >> i) & 1u)) || (i == D && pin == 1 && n == 0);
        if (idrow)
            for (int j = 0; j < NF; ++j) A[i][j] = (i == j) ? 1.0 : 0.0;
    }
    // row equilibration 1/|J_ii| (identity rows: 1)
    for (int i = 0; i < NF; ++i) {
        const double a = fabs(A[i][i]);
        scale[(size_t)n * NF + i] = a > 1e-300 ? 1.0 / a : 1.0;
        if (unscale) unscale[(size_t)n * NF + i] = a > 1e-300 ? a : 1.0;
    }
    if (decouple_p & 1) {
        // the pressure is preconditioned separately (Schur-complement approximation)
        for (int j = 0; j < NF; ++j) A[D][j] = A[j][D] = (j == D) ? 1.0 : 0.0;
    }
    if (decouple_p & 2) {
        // phi and mu are preconditioned by the Cahn-Hilliard block solve
        for (int i = D + 1; i < NF; ++i)
            for (int j = 0; j < NF; ++j) A[i][j] = A[j][i] = (j == i) ? 1.0 : 0.0;
    }
    for (int col = 0; col < NF; ++col) {
        int piv = col;
        for (int r = col + 1; r < NF; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 2 * NF; ++j) {
                const double tmp = A[col][j];
                A[col][j] = A[piv][j];
                A[piv][j] = tmp;
            }
        double d = A[col][col];
        if (d == 0.0) d = 1e-300;
        const double inv_d = 1.0 / d;
        for (int j = 0; j < 2 * NF; ++j) A[col][j] *= inv_d;
        for (int r = 0; r < NF; ++r) {
            if (r == col) continue;
            const double f = A[r][col];
            if (f != 0.0)
                for (int j = 0; j < 2 * NF; ++j) A[r][j] -= f * A[col][j];
        }
    }
    for (int i = 0; i < NF; ++i)
        for (int j = 0; j < NF; ++j) inv[((size_t)n * NF + i) * NF + j] = (TI)A[i][NF + j];
}

// z = P^{-1} v per node (FP64 input; output type TO, arithmetic in the storage type's
// precision promoted to FP64 for the final update)
template <class TI, class TO>
__global__ void pc_apply_kernel(int64_t N, int NF, const TI* __restrict__ inv, const double* __restrict__ v,
                                TO* __restrict__ z) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    // arithmetic in the precision the blocks are stored in (FP32 for the mixed path)
    TI x[6];
    for (int j = 0; j < NF; ++j) x[j] = (TI)v[(size_t)n * NF + j];
    for (int i = 0; i < NF; ++i) {
        TI s = TI(0);
        for (int j = 0; j < NF; ++j) s += inv[((size_t)n * NF + i) * NF + j] * x[j];
        z[(size_t)n * NF + i] = (TO)s;
    }
}

// ---------------- initial chemical potential (mass-matrix CG) ----------------
// b_a = sum_q |J| (N_a psi'(phi_q) + Cn^2 grad N_a . grad phi_q)  and  y = M x, with the
// consistent Q1 mass matrix; hanging corners via their parents.
template <int D, int MODE>
__global__ void mu_kernel(DevMesh m, double Cn2, const double* __restrict__ U, const double* __restrict__ x,
                          double* __restrict__ y) {
    constexpr int NC = 1 << D, NF = D + 3;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const double h = ldexp(m.hi - m.lo, -(int)m.level[e]);
    const double inv_h = 1.0 / h, detJ = (D == 2) ? 0.25 * h * h : 0.125 * h * h * h;
    int par[NC][4], np[NC];
    double u[NC];
    for (int a = 0; a < NC; ++a) {
        const int ent = m.e2n[e * NC + a];
        if (ent >= 0) {
            np[a] = 1;
            par[a][0] = ent;
        } else {
            const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
            par[a][0] = hp.x;
            par[a][1] = hp.y;
            par[a][2] = hp.z;
            par[a][3] = hp.w;
            np[a] = hp.z < 0 ? 2 : 4;
        }
        const double w = np[a] == 1 ? 1.0 : (np[a] == 2 ? 0.5 : 0.25);
        double s = 0.0;
        for (int j = 0; j < np[a]; ++j)
            s += w * (MODE == 0 ? U[(size_t)par[a][j] * NF + D + 1] : x[par[a][j]]);
        u[a] = s;
    }
    double r[NC];
    for (int a = 0; a < NC; ++a) r[a] = 0.0;
    for (int q = 0; q < NC; ++q) {
        double val = 0.0, grad[D];
        for (int k = 0; k < D; ++k) grad[k] = 0.0;
        PB<D, double> B[NC];
        for (int a = 0; a < NC; ++a) {
            B[a] = pbasis<D, double>(a, q, inv_h);
            val += B[a].N * u[a];
            for (int k = 0; k < D; ++k) grad[k] += B[a].dN[k] * u[a];
        }
        for (int a = 0; a < NC; ++a) {
            double t;
            if (MODE == 0) {
                t = B[a].N * (val * val * val - val);
                for (int k = 0; k < D; ++k) t += Cn2 * B[a].dN[k] * grad[k];
            } else {
                t = B[a].N * val;
            }
            r[a] += detJ * t;
        }
    }
    for (int a = 0; a < NC; ++a) {
        const double w = np[a] == 1 ? 1.0 : (np[a] == 2 ? 0.5 : 0.25);
        for (int j = 0; j < np[a]; ++j) atomicAdd(y + par[a][j], w * r[a]);
    }
}

__global__ void insert_mu_kernel(const double* __restrict__ in, int NF, int f, int64_t N, double* __restrict__ U) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) U[(size_t)n * NF + f] = in[n];
}
// sum_n m_n v[n*NF + f] into per-block partials
template <class T>
__global__ void field_mass_kernel(const double* __restrict__ m, const T* __restrict__ v, int NF, int f,
                                  int64_t N, double* partials) {
    double acc[1] = {0.0};
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        acc[0] += m[n] * (double)v[(size_t)n * NF + f];
    block_reduce_store<1>(acc, partials);
}
// y = sv .* x + a * sc[0] on the rows of field f: the scaled operator of
// J' = J + u m_p^T / |Omega| (pin mode 2), u = |diag J| on the pressure rows, so S u = 1
// there.  The rank-one term moves the null mode of J (constant pressure) off zero.
template <class T>
__global__ void scale_vec_pmean_kernel(const T* x, const double* __restrict__ sv, double* y,
                                       int64_t n, int NF, int f, const double* __restrict__ sc, double a) {
    const double s = a * sc[0];
    const int64_t N = n / NF;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < N;
         node += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = node * NF;
        for (int g = 0; g < NF; ++g) y[i0 + g] = sv[i0 + g] * (double)x[i0 + g] + (g == f ? s : 0.0);
    }
}
// v[n*NF + f] -= sc[0] * inv_vol
__global__ void field_shift_kernel(double* __restrict__ v, int NF, int f, int64_t N, const double* __restrict__ sc,
                                   double inv_vol) {
    const double s = sc[0] * inv_vol;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        v[(size_t)n * NF + f] -= s;
}
__global__ void fill_kernel(double* __restrict__ x, double v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}
__global__ void jacobi_kernel(const double* __restrict__ d, const double* __restrict__ r, double* __restrict__ z,
                              int64_t N) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) z[n] = r[n] / d[n];
}

template <class R>
PCst<R> pcst_from(const PhysConst& pc) {
    PCst<R> c;
    c.alpha = R(pc.alpha);
    c.beta = R(pc.beta);
    c.gamma = R(pc.gamma);
    c.xi = R(pc.xi);
    c.Jc = R((pc.rho_minus - pc.rho_plus) / (2.0 * pc.rho_plus * pc.Cn));
    c.inv_Pe = R(pc.inv_Pe);
    c.inv_We = R(pc.inv_We);
    c.inv_Re = R(pc.inv_Re);
    c.inv_Fr = R(pc.inv_Fr);
    c.Cn_We = R(pc.Cn * pc.inv_We);
    c.inv_PeCn = R(1.0 / (pc.Pe * pc.Cn));
    c.Cn2 = R(pc.Cn * pc.Cn);
    c.Pe = R(pc.Pe);
    c.Re = R(pc.Re);
    c.four_over_dt2 = R(pc.four_over_dt2);
    c.C_I = R(pc.C_I);
    c.C_phi = R(pc.C_phi);
    return c;
}

struct Ctx {
    chns_mesh* m;
    SolverWS* ws;
    cudaStream_t s;
    int64_t n;
    int g;
};

// host read of k device scalars (synchronises)
chns_status read_sc(Ctx& c, const double* dev, int k, double* host) {
    CHNS_CUDA(cudaMemcpyAsync(c.ws->hsc, dev, k * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    CHNS_CUDA(cudaStreamSynchronize(c.s));
    std::memcpy(host, c.ws->hsc, k * sizeof(double));
    return CHNS_OK;
}

chns_status dot_host(Ctx& c, const double* a, const double* b, double* out) {
    CHNS_CUDA(launch_dot(c.m, a, b, c.n, c.ws->sc, c.s));
    return read_sc(c, c.ws->sc, 1, out);
}

template <int D, class T>
cudaError_t pc_build_launch(const chns_mesh* m, const PhysConst& pc, const T* Uo, const T* Un, T* blk,
                            float* ce, cudaStream_t s) {
    constexpr int NC = 1 << D, EPB = 128 / NC;
    cudaError_t e = cudaMemsetAsync(blk, 0, (size_t)m->dm.N * m->dm.nf * m->dm.nf * sizeof(T), s);
    if (e != cudaSuccess) return e;
    const double ce_scale = pc.dt / (2.0 * pc.We);
    { pc_build_kernel<D, T><<<(unsigned)((m->dm.E + EPB - 1) / EPB), 128, 0, s>>>(m->dm, pcst_from<T>(pc), T(pc.inv_dt), Uo, Un, blk, ce, ce_scale); chns_count_launches(1); }
    return cudaGetLastError();
}

// ---------------- pressure Schur-complement approximation ----------------
// Eliminating v^{k+1} from the momentum rows (dominated by rho M / dt at small dt)
// leaves, for p^{k+1}, approximately the Laplacian (grad q, dt/(2 rho We) grad p)
// (the Galerkin divergence and the stabilisation rows together).  Its inverse is
// approximated by a Jacobi-preconditioned Chebyshev iteration of fixed degree (a
// fixed polynomial, so GMRES sees a linear preconditioner).
__constant__ float c_Kref[64];   // Q1 stiffness of the unit element (2-point Gauss)

void kref_host(int D, float* K) {
    const int NC = 1 << D;
    const double gp = 0.78867513459481288225, gm = 0.21132486540518711775;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            double sum = 0.0;
            for (int q = 0; q < NC; ++q)
                for (int k = 0; k < D; ++k) {
                    double da = ((a >> k) & 1) ? 1.0 : -1.0, db = ((b >> k) & 1) ? 1.0 : -1.0;
                    for (int j = 0; j < D; ++j) {
                        if (j == k) continue;
                        da *= (((a >> j) & 1) == ((q >> j) & 1)) ? gp : gm;
                        db *= (((b >> j) & 1) == ((q >> j) & 1)) ? gp : gm;
                    }
                    sum += da * db;
                }
            K[a * NC + b] = (float)(sum / (double)NC);   // |det J| = (1/2)^d, unit Gauss weights
        }
}

template <int D>
__device__ __forceinline__ void schur_corners(const DevMesh& m, int64_t e, int par[][4], int np[]) {
    constexpr int NC = 1 << D;
    for (int a = 0; a < NC; ++a) {
        const int ent = m.e2n[e * NC + a];
        if (ent >= 0) {
            np[a] = 1;
            par[a][0] = ent;
        } else {
            const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
            par[a][0] = hp.x;
            par[a][1] = hp.y;
            par[a][2] = hp.z;
            par[a][3] = hp.w;
            np[a] = hp.z < 0 ? 2 : 4;
        }
    }
}

// Diagonal of the Schur Laplacian (constraint cross terms within a corner's parents
// are dropped: it only scales the Chebyshev iteration) and, per node p, a bound on the
// absolute row sum of the constrained operator: sum_q |K_pq| <= sum over the corners a
// that map to p of w_ap sum_b |K_e[a][b]| (the constraint weights of a corner sum to 1).
template <int D>
__global__ void schur_diag_kernel(DevMesh m, const float* __restrict__ ce, float* __restrict__ dg,
                                  float* __restrict__ bnd) {
    constexpr int NC = 1 << D;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const float h = (float)ldexp(m.hi - m.lo, -(int)m.level[e]);
    const float ch = ce[e] * (D == 2 ? 1.0f : h);
    int par[NC][4], np[NC];
    schur_corners<D>(m, e, par, np);
    for (int a = 0; a < NC; ++a) {
        const float w = np[a] == 1 ? 1.0f : (np[a] == 2 ? 0.5f : 0.25f);
        float rs = 0.0f;
        for (int b = 0; b < NC; ++b) rs += fabsf(c_Kref[a * NC + b]);
        for (int j = 0; j < np[a]; ++j) {
            atomicAdd(dg + par[a][j], w * w * ch * c_Kref[a * NC + a]);
            atomicAdd(bnd + par[a][j], w * ch * rs);
        }
    }
}

// out = max_n bnd[n] dinv[n] (non-negative floats compare like their bit patterns)
__global__ void gershgorin_max_kernel(const float* __restrict__ bnd, const float* __restrict__ dinv, int64_t N,
                                      unsigned int* __restrict__ out) {
    float v = 0.0f;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        v = fmaxf(v, bnd[n] * dinv[n]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(v));
}

// y += sgn K_c x  (y zeroed, or holding a right-hand side, by the caller)
template <int D>
__global__ void schur_matvec_kernel(DevMesh m, const float* __restrict__ ce, const float* __restrict__ x,
                                    float* __restrict__ y, float sgn = 1.0f) {
    constexpr int NC = 1 << D;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const float h = (float)ldexp(m.hi - m.lo, -(int)m.level[e]);
    const float ch = sgn * ce[e] * (D == 2 ? 1.0f : h);
    int par[NC][4], np[NC];
    schur_corners<D>(m, e, par, np);
    float xl[NC];
    for (int a = 0; a < NC; ++a) {
        const float w = np[a] == 1 ? 1.0f : (np[a] == 2 ? 0.5f : 0.25f);
        float s = 0.0f;
        for (int j = 0; j < np[a]; ++j) s += w * __ldg(x + par[a][j]);
        xl[a] = s;
    }
    for (int a = 0; a < NC; ++a) {
        float s = 0.0f;
#pragma unroll
        for (int b = 0; b < NC; ++b) s += c_Kref[a * NC + b] * xl[b];
        s *= ch;
        const float w = np[a] == 1 ? 1.0f : (np[a] == 2 ? 0.5f : 0.25f);
        for (int j = 0; j < np[a]; ++j) atomicAdd(y + par[a][j], w * s);
    }
}

__global__ void axpbyf_kernel(float a, float* __restrict__ x, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= a;
}
__constant__ float c_Mref[64];   // Q1 consistent mass of the unit element (2-point Gauss)

void mref_host(int D, float* Mr) {
    const int NC = 1 << D;
    const double gp = 0.78867513459481288225, gm = 0.21132486540518711775;
    for (int a = 0; a < NC; ++a)
        for (int b = 0; b < NC; ++b) {
            double sum = 0.0;
            for (int q = 0; q < NC; ++q) {
                double na = 1.0, nb = 1.0;
                for (int k = 0; k < D; ++k) {
                    na *= (((a >> k) & 1) == ((q >> k) & 1)) ? gp : gm;
                    nb *= (((b >> k) & 1) == ((q >> k) & 1)) ? gp : gm;
                }
                sum += na * nb;
            }
            Mr[a * NC + b] = (float)(sum / (double)NC);   // |det J| = (1/2)^d for h = 1
        }
}

// y += (alpha M + beta K) x, or its diagonal (DIAG), on the Q1 space with constraints;
// DIAG also accumulates into bnd the absolute-row-sum bounds used for the Gershgorin
// top of the spectrum (as for the pressure Schur Laplacian)
template <int D, bool DIAG>
__global__ void mk_kernel(DevMesh m, float span, float alpha, float beta, const float* __restrict__ x,
                          float* __restrict__ y, float* __restrict__ bnd = nullptr) {
    constexpr int NC = 1 << D;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const float h = ldexpf(span, -(int)m.level[e]);
    const float hd2 = (D == 2) ? 1.0f : h;            // h^(d-2)
    const float hd = hd2 * h * h;                      // h^d
    const float am = alpha * hd, bk = beta * hd2;
    int par[NC][4], np[NC];
    schur_corners<D>(m, e, par, np);
    if (DIAG) {
        for (int a = 0; a < NC; ++a) {
            const float w = np[a] == 1 ? 1.0f : (np[a] == 2 ? 0.5f : 0.25f);
            const float v = am * c_Mref[a * NC + a] + bk * c_Kref[a * NC + a];
            float rs = 0.0f;
            for (int b = 0; b < NC; ++b) rs += fabsf(am * c_Mref[a * NC + b] + bk * c_Kref[a * NC + b]);
            for (int j = 0; j < np[a]; ++j) {
                atomicAdd(y + par[a][j], w * w * v);
                if (bnd) atomicAdd(bnd + par[a][j], w * rs);
            }
        }
        return;
    }
    float xl[NC];
    for (int a = 0; a < NC; ++a) {
        const float w = np[a] == 1 ? 1.0f : (np[a] == 2 ? 0.5f : 0.25f);
        float sacc = 0.0f;
        for (int j = 0; j < np[a]; ++j) sacc += w * __ldg(x + par[a][j]);
        xl[a] = sacc;
    }
    for (int a = 0; a < NC; ++a) {
        float sacc = 0.0f;
#pragma unroll
        for (int b = 0; b < NC; ++b) sacc += (am * c_Mref[a * NC + b] + bk * c_Kref[a * NC + b]) * xl[b];
        const float w = np[a] == 1 ? 1.0f : (np[a] == 2 ? 0.5f : 0.25f);
        for (int j = 0; j < np[a]; ++j) atomicAdd(y + par[a][j], w * sacc);
    }
}

// nodal psi''(phi~) with phi~ the mid-point average, and the lumped mass (FP32)
template <class T>
__global__ void ch_nodal_kernel(int64_t N, int NF, int fphi, const T* __restrict__ Uo, const T* __restrict__ Un,
                                const double* __restrict__ nmass, float* __restrict__ psi2, float* __restrict__ ml) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float ph = 0.5f * ((float)Uo[(size_t)n * NF + fphi] + (float)Un[(size_t)n * NF + fphi]);
    psi2[n] = 3.0f * ph * ph - 1.0f;
    ml[n] = (float)nmass[n];
}

// rp = v_phi, rm = v_mu (strided FP64 input), a = rm / ml
__global__ void ch_load_kernel(int64_t N, int NF, int fphi, const double* __restrict__ v, float* __restrict__ rp,
                               float* __restrict__ rm, float* __restrict__ a, const float* __restrict__ ml) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    rp[n] = (float)v[(size_t)n * NF + fphi];
    const float r = (float)v[(size_t)n * NF + fphi + 1];
    rm[n] = r;
    a[n] = r / ml[n];
}
// t = rp + c * y
__global__ void ch_axpy_kernel(int64_t N, const float* __restrict__ rp, const float* __restrict__ y, float c,
                               float* __restrict__ t) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) t[n] = rp[n] + c * y[n];
}
// z_phi = x, z_mu = psi2 x + Cn^2 (K x) / ml - 2 rm / ml
template <class TO>
__global__ void ch_store_kernel(int64_t N, int NF, int fphi, const float* __restrict__ x, const float* __restrict__ kx,
                                const float* __restrict__ rm, const float* __restrict__ psi2,
                                const float* __restrict__ ml, float cn2, TO* __restrict__ z) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float xv = x[n], il = 1.0f / ml[n];
    z[(size_t)n * NF + fphi] = (TO)xv;
    z[(size_t)n * NF + fphi + 1] = (TO)(psi2[n] * xv + cn2 * kx[n] * il - 2.0f * rm[n] * il);
}

__global__ void recip_kernel(float* __restrict__ d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = d[i] > 0.0f ? 1.0f / d[i] : 0.0f;
}

// r = v_p (strided input), x = 0, d = dinv r / theta, y = 0 (the first matvec's output)
template <class TI>
__global__ void cheb_init_kernel(int64_t N, int NF, int f, const TI* __restrict__ v, const float* __restrict__ dinv,
                                 float* __restrict__ r, float* __restrict__ x, float* __restrict__ d, float* __restrict__ y,
                                 float inv_theta) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float rv = (float)v[(size_t)n * NF + f];
    r[n] = rv;
    x[n] = 0.0f;
    y[n] = 0.0f;
    d[n] = inv_theta * dinv[n] * rv;
}

// x += d; r -= y; d = c1 d + c2 dinv r; y = 0 (ready for the next accumulating matvec)
__global__ void cheb_step_kernel(int64_t N, const float* __restrict__ dinv, float* __restrict__ r, float* __restrict__ x,
                                 float* __restrict__ d, float* __restrict__ y, float c1, float c2) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    x[n] += d[n];
    const float rn = r[n] - y[n];
    y[n] = 0.0f;
    r[n] = rn;
    d[n] = c1 * d[n] + c2 * dinv[n] * rn;
}

template <class TO>
__global__ void cheb_final_kernel(int64_t N, int NF, int f, const float* __restrict__ x, const float* __restrict__ d,
                                  TO* __restrict__ z) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) z[(size_t)n * NF + f] = (TO)(x[n] + d[n]);
}


// ---------------- geometric multigrid for the pressure Schur Laplacian ----------------
// coarse element coefficients: the volume-weighted mean of the fine elements they hold
__global__ void mg_restrict_ce_kernel(int64_t Ef, int D, const int32_t* __restrict__ fmap,
                                      const int8_t* __restrict__ lev_f, const int8_t* __restrict__ lev_c,
                                      const float* __restrict__ ce_f, float* __restrict__ ce_c) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ef) return;
    const int c = fmap[e];
    atomicAdd(ce_c + c, ldexpf(ce_f[e], -D * ((int)lev_f[e] - (int)lev_c[c])));
}
__global__ void mg_copy_kernel(int64_t N, const float* __restrict__ a, float* __restrict__ b) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) b[n] = a[n];
}
template <class TI>
__global__ void mg_load_kernel(int64_t N, int NF, int f, const TI* __restrict__ v, float* __restrict__ b) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) b[n] = (float)v[(size_t)n * NF + f];
}
template <class TO>
__global__ void mg_store_kernel(int64_t N, int NF, int f, const float* __restrict__ x, TO* __restrict__ z) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) z[(size_t)n * NF + f] = (TO)x[n];
}
// out += x + d (a Chebyshev correction added to an existing iterate)
__global__ void cheb_final_add_kernel(int64_t N, const float* __restrict__ x, const float* __restrict__ d,
                                      float* __restrict__ out) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) out[n] += x[n] + d[n];
}

// Chebyshev coefficients of the three-term recurrence on [alpha, beta] (degree deg)
void cheb_coeffs(double alpha, double beta, int deg, std::vector<float>& c1, std::vector<float>& c2, float& inv_theta) {
    const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha), sigma = theta / delta;
    c1.assign(std::max(deg, 1), 0.0f);
    c2.assign(std::max(deg, 1), 0.0f);
    double rho = 1.0 / sigma;
    for (int k = 0; k + 1 < deg; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        c1[k] = (float)(rn * rho);
        c2[k] = (float)(2.0 * rn / delta);
        rho = rn;
    }
    inv_theta = (float)(1.0 / theta);
}

// One V-cycle for K x = b on level l (x overwritten), queued on stream st; returns the
// number of kernels queued.  Each level: Chebyshev pre-smoothing from x = 0, residual,
// restriction P^T, the coarser cycle, prolongation P added to x, residual, Chebyshev
// post-smoothing added to x; the coarsest level is one long Chebyshev sweep.
int mg_vcycle(MGHier* mg, int l, const float* ce0, cudaStream_t st) {
    MGLevel& L = mg->lv[(size_t)l];
    const float* ce = l == 0 ? ce0 : L.ce;
    const int D = L.dm.dim;
    const int gN = (int)((L.N + 255) / 256), gE = (int)((L.E + 255) / 256);
    int nk = 0;
    auto matvec = [&](const float* x, float* y, float sgn) {
        if (D == 2) schur_matvec_kernel<2><<<gE, 256, 0, st>>>(L.dm, ce, x, y, sgn);
        else schur_matvec_kernel<3><<<gE, 256, 0, st>>>(L.dm, ce, x, y, sgn);
        ++nk;
    };
    auto cheb = [&](const float* in, float* out, bool add) {
        cheb_init_kernel<float><<<gN, 256, 0, st>>>(L.N, 1, 0, in, L.dinv, L.cr, L.cx, L.cd, L.cy, L.inv_theta);
        ++nk;
        for (int k = 0; k + 1 < L.deg; ++k) {
            matvec(L.cd, L.cy, 1.0f);
            cheb_step_kernel<<<gN, 256, 0, st>>>(L.N, L.dinv, L.cr, L.cx, L.cd, L.cy, L.c1[(size_t)k], L.c2[(size_t)k]);
            ++nk;
        }
        if (add) cheb_final_add_kernel<<<gN, 256, 0, st>>>(L.N, L.cx, L.cd, out);
        else cheb_final_kernel<float><<<gN, 256, 0, st>>>(L.N, 1, 0, L.cx, L.cd, out);
        ++nk;
    };
    if (l + 1 == (int)mg->lv.size()) {
        cheb(L.b, L.x, false);
        return nk;
    }
    MGLevel& C = mg->lv[(size_t)l + 1];
    cheb(L.b, L.x, false);
    mg_copy_kernel<<<gN, 256, 0, st>>>(L.N, L.b, L.t);
    ++nk;
    matvec(L.x, L.t, -1.0f);
    transfer_apply_f32(C.P, true, false, L.t, C.b, st);
    ++nk;
    nk += mg_vcycle(mg, l + 1, ce0, st);
    transfer_apply_f32(C.P, false, true, C.x, L.x, st);
    ++nk;
    mg_copy_kernel<<<gN, 256, 0, st>>>(L.N, L.b, L.t);
    ++nk;
    matvec(L.x, L.t, -1.0f);
    cheb(L.t, L.x, true);
    return nk;
}

// Pressure Schur-complement preconditioner (pc_type >= 1), shared by the Newton step and
// the adjoint solve: set-up after the block-Jacobi build has written the element
// coefficients ws->ce, then applies z_p = (approximation of S^{-1}) v_p, either a
// Jacobi-Chebyshev polynomial of degree `degree` or one multigrid V-cycle (use_mg).
struct SchurPC {
    chns_mesh* m;
    SolverWS* ws;
    cudaStream_t s;
    int degree;
    bool use_mg;
    int D, NF, gE, gN1, g;
    SchurPC(chns_mesh* mm, SolverWS* w, cudaStream_t st, int deg, bool mg)
        : m(mm), ws(w), s(st), degree(deg), use_mg(mg), D(mm->dm.dim), NF(mm->dm.nf),
          gE((int)((mm->dm.E + 255) / 256)), gN1((int)((mm->dm.N + 255) / 256)), g(grid_for(w->n)) {}
    chns_status setup() { return use_mg ? mg_setup() : cheb_setup(); }
    chns_status cheb_setup() {
        if (ws->kref_dim != D) {
            float K[64], Mr[64];
            kref_host(D, K);
            mref_host(D, Mr);
            CHNS_CUDA(cudaMemcpyToSymbolAsync(c_Kref, K, sizeof(float) * (1 << D) * (1 << D), 0,
                                              cudaMemcpyHostToDevice, s));
            CHNS_CUDA(cudaMemcpyToSymbolAsync(c_Mref, Mr, sizeof(float) * (1 << D) * (1 << D), 0,
                                              cudaMemcpyHostToDevice, s));
            ws->kref_dim = D;
        }
        const int64_t N = m->dm.N;
        CHNS_CUDA(cudaMemsetAsync(ws->kdinv, 0, N * sizeof(float), s));
        CHNS_CUDA(cudaMemsetAsync(ws->kbnd, 0, N * sizeof(float), s));
        CHNS_CUDA(cudaMemsetAsync(ws->kmax, 0, sizeof(unsigned int), s));
        if (D == 2) { schur_diag_kernel<2><<<gE, 256, 0, s>>>(m->dm, ws->ce, ws->kdinv, ws->kbnd); chns_count_launches(1); }
        else { schur_diag_kernel<3><<<gE, 256, 0, s>>>(m->dm, ws->ce, ws->kdinv, ws->kbnd); chns_count_launches(1); }
        { recip_kernel<<<gN1, 256, 0, s>>>(ws->kdinv, N); chns_count_launches(1); }
        // The Chebyshev interval must not cut the top of the spectrum of D^{-1} K, where
        // the polynomial would amplify.  Gershgorin with the row-sum bounds gives it for
        // any positive D: 2 on a uniform mesh (off-diagonal stiffness entries are <= 0),
        // more where hanging constraints fold positive weights into a row.
        { gershgorin_max_kernel<<<g, 256, 0, s>>>(ws->kbnd, ws->kdinv, N, ws->kmax); chns_count_launches(1); }
        unsigned int kbits = 0;
        CHNS_CUDA(cudaMemcpyAsync(&ws->hsc[0], ws->kmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CHNS_CUDA(cudaStreamSynchronize(s));
        std::memcpy(&kbits, &ws->hsc[0], sizeof(unsigned int));
        float kb;
        std::memcpy(&kb, &kbits, sizeof(float));
        if (!(kb > 0.0f) || !std::isfinite(kb)) { chns_set_error("pressure Schur spectrum bound is not finite"); return CHNS_ENAN; }
        const double beta = 1.01 * (double)kb;
        const double nside = std::ldexp(1.0, m->max_level);
        const double ratio = std::max(16.0, nside * nside / 8.0);
        const double alpha = beta / ratio;
        const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha), sigma = theta / delta;
        const int deg = degree;
        ws->cheb_c1.assign(deg, 0.0f);
        ws->cheb_c2.assign(deg, 0.0f);
        double rho = 1.0 / sigma;
        for (int k = 0; k + 1 < deg; ++k) {
            const double rn = 1.0 / (2.0 * sigma - rho);
            ws->cheb_c1[k] = (float)(rn * rho);
            ws->cheb_c2[k] = (float)(2.0 * rn / delta);
            rho = rn;
        }
        ws->cheb_inv_theta = (float)(1.0 / theta);
        ws->schur_gen++;   // captured applies hold the old coefficients
        return CHNS_OK;
    }
    chns_status mg_setup() {
        if (ws->kref_dim != D) {
            float K[64], Mr[64];
            kref_host(D, K);
            mref_host(D, Mr);
            CHNS_CUDA(cudaMemcpyToSymbolAsync(c_Kref, K, sizeof(float) * (1 << D) * (1 << D), 0,
                                              cudaMemcpyHostToDevice, s));
            CHNS_CUDA(cudaMemcpyToSymbolAsync(c_Mref, Mr, sizeof(float) * (1 << D) * (1 << D), 0,
                                              cudaMemcpyHostToDevice, s));
            ws->kref_dim = D;
        }
        chns_status sb = mg_hier_build(m);
        if (sb != CHNS_OK) return sb;
        MGHier* mg = m->mg;
        const int nl = (int)mg->lv.size();
        for (int l = 1; l < nl; ++l) {
            MGLevel& C = mg->lv[(size_t)l];
            MGLevel& F = mg->lv[(size_t)l - 1];
            CHNS_CUDA(cudaMemsetAsync(C.ce, 0, C.E * sizeof(float), s));
            { mg_restrict_ce_kernel<<<(int)((F.E + 255) / 256), 256, 0, s>>>(F.E, D, C.fmap, F.dm.level, C.dm.level, l == 1 ? ws->ce : F.ce, C.ce); chns_count_launches(1); }
        }
        CHNS_CUDA(cudaMemsetAsync(mg->kmax, 0, nl * sizeof(unsigned int), s));
        for (int l = 0; l < nl; ++l) {
            MGLevel& L = mg->lv[(size_t)l];
            const float* cel = l == 0 ? ws->ce : L.ce;
            const int gEl = (int)((L.E + 255) / 256), gNl = (int)((L.N + 255) / 256);
            CHNS_CUDA(cudaMemsetAsync(L.dinv, 0, L.N * sizeof(float), s));
            CHNS_CUDA(cudaMemsetAsync(L.bnd, 0, L.N * sizeof(float), s));
            if (D == 2) { schur_diag_kernel<2><<<gEl, 256, 0, s>>>(L.dm, cel, L.dinv, L.bnd); chns_count_launches(1); }
            else { schur_diag_kernel<3><<<gEl, 256, 0, s>>>(L.dm, cel, L.dinv, L.bnd); chns_count_launches(1); }
            { recip_kernel<<<gNl, 256, 0, s>>>(L.dinv, L.N); chns_count_launches(1); }
            { gershgorin_max_kernel<<<grid_for(L.N), 256, 0, s>>>(L.bnd, L.dinv, L.N, mg->kmax + l); chns_count_launches(1); }
        }
        CHNS_CUDA(cudaGetLastError());
        CHNS_CUDA(cudaMemcpyAsync(ws->hsc, mg->kmax, nl * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CHNS_CUDA(cudaStreamSynchronize(s));
        for (int l = 0; l < nl; ++l) {
            MGLevel& L = mg->lv[(size_t)l];
            unsigned int kbits = 0;
            std::memcpy(&kbits, reinterpret_cast<const unsigned char*>(ws->hsc) + l * sizeof(unsigned int),
                        sizeof(unsigned int));
            float kb;
            std::memcpy(&kb, &kbits, sizeof(float));
            if (!(kb > 0.0f) || !std::isfinite(kb)) { chns_set_error("multigrid spectrum bound is not finite"); return CHNS_ENAN; }
            const double beta = 1.01 * (double)kb;
            if (l + 1 < nl) {
                // smoother: damp the upper part of the spectrum of D^{-1} K
                L.deg = degree;
                cheb_coeffs(beta / 10.0, beta, L.deg, L.c1, L.c2, L.inv_theta);
            } else {
                // coarsest level: one long sweep over the whole spectrum
                const double nside = std::ldexp(1.0, L.mesh ? L.mesh->max_level : m->max_level);
                L.deg = 16;
                cheb_coeffs(beta / std::max(16.0, nside * nside / 8.0), beta, L.deg, L.c1, L.c2, L.inv_theta);
            }
        }
        ws->schur_gen++;   // captured applies hold the old coefficients
        return CHNS_OK;
    }
    template <class TI, class TO>
    chns_status apply(const TI* vin, TO* zout) {
        const int64_t N = m->dm.N;
        // the apply is a sequence of short launches: replayed from a CUDA graph
        auto enqueue = [&](cudaStream_t st) -> int {
            if (use_mg) {
                MGHier* mg = m->mg;
                mg_load_kernel<TI><<<gN1, 256, 0, st>>>(N, NF, D, vin, mg->lv[0].b);
                const int nv = mg_vcycle(mg, 0, ws->ce, st);
                mg_store_kernel<TO><<<gN1, 256, 0, st>>>(N, NF, D, mg->lv[0].x, zout);
                return nv + 2;
            }
            cheb_init_kernel<TI><<<gN1, 256, 0, st>>>(N, NF, D, vin, ws->kdinv, ws->cr, ws->cx, ws->cd, ws->cy, ws->cheb_inv_theta);
            for (int k = 0; k + 1 < degree; ++k) {
                if (D == 2) schur_matvec_kernel<2><<<gE, 256, 0, st>>>(m->dm, ws->ce, ws->cd, ws->cy);
                else schur_matvec_kernel<3><<<gE, 256, 0, st>>>(m->dm, ws->ce, ws->cd, ws->cy);
                cheb_step_kernel<<<gN1, 256, 0, st>>>(N, ws->kdinv, ws->cr, ws->cx, ws->cd, ws->cy, ws->cheb_c1[k], ws->cheb_c2[k]);
            }
            cheb_final_kernel<TO><<<gN1, 256, 0, st>>>(N, NF, D, ws->cx, ws->cd, zout);
            return 2 + 2 * (degree - 1);
        };
        if (!ws->no_graphs) {
            SolverWS::SchurGraph* hit = nullptr;
            for (auto& g : ws->sgraph)
                if (g.exec && g.gen == ws->schur_gen && g.vin == (const void*)vin && g.zout == (void*)zout &&
                    g.to == sizeof(TO))
                    hit = &g;
            if (!hit) {
                SolverWS::SchurGraph* slot = &ws->sgraph[0];
                for (auto& g : ws->sgraph)
                    if (!g.exec || g.gen != ws->schur_gen) { slot = &g; break; }
                cudaGraphExec_t ex = nullptr;
                cudaGraph_t gr = nullptr;
                bool ok = ws->cap || cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking) == cudaSuccess;
                if (ok) ok = cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                int nk_cap = 0;
                if (ok) {
                    nk_cap = enqueue(ws->cap);
                    ok = cudaStreamEndCapture(ws->cap, &gr) == cudaSuccess && gr != nullptr;
                    if (ok) ok = cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
                    if (gr) cudaGraphDestroy(gr);
                }
                if (!ok) {
                    (void)cudaGetLastError();   // capture unavailable: launch directly from now on
                    ws->no_graphs = true;
                } else {
                    if (slot->exec) cudaGraphExecDestroy(slot->exec);
                    slot->exec = ex;
                    slot->vin = (const void*)vin;
                    slot->zout = (void*)zout;
                    slot->to = sizeof(TO);
                    slot->gen = ws->schur_gen;
                    slot->nk = nk_cap;
                    hit = slot;
                }
            }
            if (hit) {
                CHNS_CUDA(cudaGraphLaunch(hit->exec, s));
                chns_count_launches(hit->nk);
                return CHNS_OK;
            }
        }
        chns_count_launches(enqueue(s));
        CHNS_CUDA(cudaGetLastError());
        return CHNS_OK;
    }
};

}  // namespace

extern "C" chns_status chns_newton_step(const chns_mesh* mc, const chns_params* p, const chns_solver_opts* o,
                                        const double* U_old, double* U, chns_stats* stats, void* stream) {
    if (chns_require_q1(mc, "chns_newton_step") != CHNS_OK) return CHNS_EINVAL;
    chns_mesh* m = const_cast<chns_mesh*>(mc);
    PhysConst pc;
    chns_status st = chns_check_params(mc, p, &pc);
    if (st != CHNS_OK) return st;
    if (!o || !U_old || !U) { chns_set_error("null argument"); return CHNS_EINVAL; }
    if ((st = chns_check_rows(mc, U_old, 8)) != CHNS_OK || (st = chns_check_rows(mc, U, 8)) != CHNS_OK) return st;
    if (o->restart < 1 || o->restart > MAXSC / 4 || o->max_krylov < 1 || o->max_newton < 0 ||
        (o->precision != 0 && o->precision != 1) || (o->pc_type < 0 || o->pc_type > 4) ||
        (o->pc_type >= 1 && (o->pc_degree < 2 || o->pc_degree > 200)) ||
        !(o->ew_eta0 == 0.0 || (o->ew_eta0 > 0.0 && o->ew_eta0 < 1.0)) || (o->guess != 0 && o->guess != 1)) {
        chns_set_error("bad solver options (restart in [1, 256], max_krylov >= 1, precision 0/1, pc_type 0..4, "
                       "pc_degree in [2, 200], ew_eta0 0 or in (0, 1), guess 0/1)");
        return CHNS_EINVAL;
    }
    if ((st = ensure_ws(m, o->restart)) != CHNS_OK) return st;
    SolverWS* ws = m->ws;
    Ctx c{m, ws, (cudaStream_t)stream, ws->n, 0};
    c.g = grid_for(c.n);
    const int D = m->dm.dim, NF = m->dm.nf, mres = o->restart;
    const bool mixed = o->precision == 1;
    const int schur = o->pc_type >= 1 ? 1 : 0;
    const int chblk = (o->pc_type == 2 || o->pc_type == 4) ? 1 : 0;
    const bool use_mg = o->pc_type >= 3;   // pressure Schur by a multigrid V-cycle
    const int pcmask = schur | (chblk << 1);
    const int gE = (int)((m->dm.E + 255) / 256);
    const int gN1 = (int)((m->dm.N + 255) / 256);
    SchurPC spc(m, ws, c.s, o->pc_degree, use_mg);
    auto schur_apply_any = [&](auto vin, auto zout) -> chns_status { return spc.apply(vin, zout); };
    const int pin = p->pin_pressure;
    const int gN = (int)((m->dm.N + 127) / 128);
    chns_stats S;
    std::memset(&S, 0, sizeof(S));
    S.reason = CHNS_OK;

    CHNS_CUDA(cudaMemsetAsync(m->d_flags, 0, sizeof(unsigned int), c.s));
    if (o->guess == 0) { copy64_kernel<<<c.g, 256, 0, c.s>>>(U_old, U, c.n); chns_count_launches(1); }
    if (mixed) { to32_kernel<<<c.g, 256, 0, c.s>>>(U_old, ws->Uo32, c.n); chns_count_launches(1); }
    CHNS_CUDA(cudaGetLastError());

    std::vector<double> H((size_t)(mres + 1) * mres), cs(mres), sn(mres), gv(mres + 1), y(mres);
    double r0 = 0.0, rn = 0.0;
    chns_status result = CHNS_OK;
    // Cahn-Hilliard block: S_phi ~ (1/dt)(M + eps K) M^{-1} (M + eps K), eps^2 = dt Cn/(2 Pe)
    const float span = (float)(m->dm.hi - m->dm.lo);
    const int CH_DEG = 8;
    auto mk = [&](float alpha, float beta, const float* x, float* y) -> chns_status {
        CHNS_CUDA(cudaMemsetAsync(y, 0, m->dm.N * sizeof(float), c.s));
        if (D == 2) { mk_kernel<2, false><<<gE, 256, 0, c.s>>>(m->dm, span, alpha, beta, x, y); chns_count_launches(1); }
        else { mk_kernel<3, false><<<gE, 256, 0, c.s>>>(m->dm, span, alpha, beta, x, y); chns_count_launches(1); }
        return CHNS_OK;
    };
    auto ch_setup = [&](const void* Uo_any, const void* Un_any) -> chns_status {
        const int64_t N = m->dm.N;
        if (mixed) { ch_nodal_kernel<float><<<gN1, 256, 0, c.s>>>(N, NF, D + 1, (const float*)Uo_any, (const float*)Un_any, m->d_nmass, ws->ch_psi2, ws->ch_ml); chns_count_launches(1); }
        else { ch_nodal_kernel<double><<<gN1, 256, 0, c.s>>>(N, NF, D + 1, (const double*)Uo_any, (const double*)Un_any, m->d_nmass, ws->ch_psi2, ws->ch_ml); chns_count_launches(1); }
        ws->ch_eps = (float)std::sqrt(p->dt * p->Cn / (2.0 * p->Pe));
        CHNS_CUDA(cudaMemsetAsync(ws->ch_dinv, 0, N * sizeof(float), c.s));
        CHNS_CUDA(cudaMemsetAsync(ws->kbnd, 0, N * sizeof(float), c.s));
        CHNS_CUDA(cudaMemsetAsync(ws->kmax, 0, sizeof(unsigned int), c.s));
        if (D == 2) { mk_kernel<2, true><<<gE, 256, 0, c.s>>>(m->dm, span, 1.0f, ws->ch_eps, nullptr, ws->ch_dinv, ws->kbnd); chns_count_launches(1); }
        else { mk_kernel<3, true><<<gE, 256, 0, c.s>>>(m->dm, span, 1.0f, ws->ch_eps, nullptr, ws->ch_dinv, ws->kbnd); chns_count_launches(1); }
        { recip_kernel<<<gN1, 256, 0, c.s>>>(ws->ch_dinv, N); chns_count_launches(1); }
        // top of the spectrum of D^{-1}(M + eps K): Gershgorin with the row-sum bounds
        // (3.375 for the Q1 mass on a uniform 3D mesh, 2 for the stiffness)
        { gershgorin_max_kernel<<<c.g, 256, 0, c.s>>>(ws->kbnd, ws->ch_dinv, N, ws->kmax); chns_count_launches(1); }
        CHNS_CUDA(cudaGetLastError());
        unsigned int kbits = 0;
        CHNS_CUDA(cudaMemcpyAsync(&ws->hsc[0], ws->kmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, c.s));
        CHNS_CUDA(cudaStreamSynchronize(c.s));
        std::memcpy(&kbits, &ws->hsc[0], sizeof(unsigned int));
        float kb;
        std::memcpy(&kb, &kbits, sizeof(float));
        if (!(kb > 0.0f) || !std::isfinite(kb)) { chns_set_error("Cahn-Hilliard block spectrum bound is not finite"); return CHNS_ENAN; }
        const double beta = 1.01 * (double)kb, alpha = 0.05;
        const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha), sigma = theta / delta;
        ws->ch_c1.assign(CH_DEG, 0.0f);
        ws->ch_c2.assign(CH_DEG, 0.0f);
        double rho = 1.0 / sigma;
        for (int k = 0; k + 1 < CH_DEG; ++k) {
            const double rn = 1.0 / (2.0 * sigma - rho);
            ws->ch_c1[k] = (float)(rn * rho);
            ws->ch_c2[k] = (float)(2.0 * rn / delta);
            rho = rn;
        }
        ws->ch_inv_theta = (float)(1.0 / theta);
        return CHNS_OK;
    };
    // out = Chebyshev approximation of (M + eps K)^{-1} in (contiguous FP32)
    auto ch_cheb = [&](const float* in, float* out) -> chns_status {
        const int64_t N = m->dm.N;
        { cheb_init_kernel<float><<<gN1, 256, 0, c.s>>>(N, 1, 0, in, ws->ch_dinv, ws->cr, ws->cx, ws->cd, ws->cy, ws->ch_inv_theta); chns_count_launches(1); }
        for (int k = 0; k + 1 < CH_DEG; ++k) {
            chns_status s2 = mk(1.0f, ws->ch_eps, ws->cd, ws->cy);
            if (s2 != CHNS_OK) return s2;
            { cheb_step_kernel<<<gN1, 256, 0, c.s>>>(N, ws->ch_dinv, ws->cr, ws->cx, ws->cd, ws->cy, ws->ch_c1[k], ws->ch_c2[k]); chns_count_launches(1); }
        }
        { cheb_final_kernel<float><<<gN1, 256, 0, c.s>>>(N, 1, 0, ws->cx, ws->cd, out); chns_count_launches(1); }
        CHNS_CUDA(cudaGetLastError());
        return CHNS_OK;
    };
    auto ch_apply_any = [&](const double* v, auto zout) -> chns_status {
        using TO = std::remove_pointer_t<decltype(zout)>;
        const int64_t N = m->dm.N;
        chns_status s2;
        { ch_load_kernel<<<gN1, 256, 0, c.s>>>(N, NF, D + 1, v, ws->ch_b, ws->ch_rm, ws->ch_a, ws->ch_ml); chns_count_launches(1); }
        if ((s2 = mk(0.0f, 1.0f, ws->ch_a, ws->ch_c)) != CHNS_OK) return s2;                 // K M_L^{-1} r_mu
        { ch_axpy_kernel<<<gN1, 256, 0, c.s>>>(N, ws->ch_b, ws->ch_c, (float)(1.0 / (p->Pe * p->Cn)), ws->ch_b); chns_count_launches(1); }
        if ((s2 = ch_cheb(ws->ch_b, ws->ch_a)) != CHNS_OK) return s2;                      // (M + eps K)^{-1} t
        if ((s2 = mk(1.0f, 0.0f, ws->ch_a, ws->ch_c)) != CHNS_OK) return s2;                // M s
        { axpbyf_kernel<<<gN1, 256, 0, c.s>>>((float)p->dt, ws->ch_c, N); chns_count_launches(1); }
        if ((s2 = ch_cheb(ws->ch_c, ws->ch_a)) != CHNS_OK) return s2;                      // dphi
        if ((s2 = mk(0.0f, 1.0f, ws->ch_a, ws->ch_c)) != CHNS_OK) return s2;                // K dphi
        { ch_store_kernel<TO><<<gN1, 256, 0, c.s>>>(N, NF, D + 1, ws->ch_a, ws->ch_c, ws->ch_rm, ws->ch_psi2, ws->ch_ml, (float)(p->Cn * p->Cn), zout); chns_count_launches(1); }
        CHNS_CUDA(cudaGetLastError());
        return CHNS_OK;
    };
    // one classical Gram-Schmidt pass against V_0..V_{k-1}: h -> hdev[0..k), |w|^2 before
    // -> nrm_before, |w|^2 after -> nrm_after (all device scalars); with pred, every kernel
    // of the pass returns at once when pred[0] == 0
    auto orth_pass = [&](cudaStream_t st, int k, double* hdev, double* nrm_before, double* nrm_after,
                         const double* pred) {
        int nbx = c.g < ORTH_MAX_BX ? c.g : ORTH_MAX_BX;
        const int nch = (k + 7) / 8;
        orth_dots_kernel<<<dim3(nbx, nch), 256, 0, st>>>(ws->V, c.n, k, ws->w, c.n, ws->part, pred);
        orth_dots_final_kernel<<<nch, 288, 0, st>>>(ws->part, nbx, k, hdev, nrm_before, pred);
        gs_update_norm_kernel<<<nbx, 256, 0, st>>>(ws->V, c.n, k, hdev, ws->w, c.n, m->d_partials, pred);
        final_reduce1_pred_kernel<<<1, 256, 0, st>>>(m->d_partials, nbx, nrm_after, pred);
    };
    // Gram-Schmidt of Arnoldi step j with device-decided re-orthogonalisation, the next
    // Arnoldi vector and the read-back of the Hessenberg column: 10 kernels and a copy
    auto orth_enqueue = [&](cudaStream_t st, int j) {
        orth_pass(st, j + 1, ws->sc, ws->sc + 600, ws->sc + 601, nullptr);
        reorth_decide_kernel<<<1, 256, 0, st>>>(ws->sc, j + 1);
        orth_pass(st, j + 1, ws->sc + 256, ws->sc + 602, ws->sc + 603, ws->sc + 605);
        scale_next_kernel<<<c.g, 256, 0, st>>>(ws->w, ws->V + (size_t)(j + 1) * c.n, c.n, ws->sc + 603);
        cudaMemcpyAsync(ws->hsc, ws->sc, 606 * sizeof(double), cudaMemcpyDeviceToHost, st);
    };
    auto build_pc = [&]() -> chns_status {
        CHNS_CUDA(cudaEventRecord(ws->ev[2], c.s));
        if (mixed) {
            { to32_kernel<<<c.g, 256, 0, c.s>>>(U, ws->Us32, c.n); chns_count_launches(1); }
            cudaError_t e = (D == 2) ? pc_build_launch<2, float>(m, pc, ws->Uo32, ws->Us32, ws->Pblk32, ws->ce, c.s)
                                     : pc_build_launch<3, float>(m, pc, ws->Uo32, ws->Us32, ws->Pblk32, ws->ce, c.s);
            CHNS_CUDA(e);
            { pc_invert_kernel<float, float><<<gN, 128, 0, c.s>>>(m->dm, ws->Pblk32, ws->Pinv32, pin, ws->S, ws->Sd, pcmask); chns_count_launches(1); }
        } else {
            cudaError_t e = (D == 2) ? pc_build_launch<2, double>(m, pc, U_old, U, ws->Pblk64, ws->ce, c.s)
                                     : pc_build_launch<3, double>(m, pc, U_old, U, ws->Pblk64, ws->ce, c.s);
            CHNS_CUDA(e);
            { pc_invert_kernel<double, double><<<gN, 128, 0, c.s>>>(m->dm, ws->Pblk64, ws->Pinv64, pin, ws->S, ws->Sd, pcmask); chns_count_launches(1); }
        }
        CHNS_CUDA(cudaGetLastError());
        if (schur) {
            chns_status st3 = spc.setup();
            if (st3 != CHNS_OK) return st3;
        }
        if (chblk) {
            chns_status st3 = mixed ? ch_setup(ws->Uo32, ws->Us32) : ch_setup(U_old, U);
            if (st3 != CHNS_OK) return st3;
        }
        CHNS_CUDA(cudaEventRecord(ws->ev[3], c.s));
        return CHNS_OK;
    };
    // m_p^T v / |Omega| term of the pin-mode-2 operator: sum_n m_n v_p[n] into sc[610]
    const double inv_vol = 1.0 / m->volume;
    const int nbm = c.g < 1024 ? c.g : 1024;
    auto pmean = [&](const auto* v) {
        { field_mass_kernel<<<nbm, 256, 0, c.s>>>(m->d_nmass, v, NF, D, m->dm.N, m->d_partials); chns_count_launches(1); }
        { final_reduce_kernel<<<1, 256, 0, c.s>>>(m->d_partials, nbm, 1, ws->sc + 610); chns_count_launches(1); }
    };
    bool pc_pending = false;
    double eta_prev = 0.0, rn_prev = 0.0;   // previous forcing term and residual (Eisenstat-Walker)
    for (int it = 0;; ++it) {
        CHNS_CUDA(launch_residual(m, pc, U_old, U, ws->R, pin, c.s));
        if (it == 0) {
            // row equilibration of the step (1/|diag J| at U^0): the Newton test and the
            // Krylov residual weigh every field by its own scale (the pressure rows carry
            // coefficients ~ tau/We and would otherwise be invisible in ||R||)
            if ((st = build_pc()) != CHNS_OK) return st;
            pc_pending = true;
            { copy64_kernel<<<c.g, 256, 0, c.s>>>(ws->S, ws->S0, c.n); chns_count_launches(1); }
        }
        { scale_vec_kernel<double><<<c.g, 256, 0, c.s>>>(ws->R, ws->S0, ws->SR, c.n); chns_count_launches(1); }
        if ((st = dot_host(c, ws->SR, ws->SR, &rn)) != CHNS_OK) return st;
        unsigned int flag = 0;
        CHNS_CUDA(cudaMemcpy(&flag, m->d_flags, sizeof(unsigned int), cudaMemcpyDeviceToHost));
        rn = std::sqrt(rn);
        if (it == 0) r0 = rn;
        S.newton_its = it;
        if (it < CHNS_HIST) S.res_hist[it] = rn;
        S.res0 = r0;
        S.res_final = rn;
        if (flag & 1u) { chns_set_error("a tau_m radicand was not positive"); result = CHNS_ETAU; break; }
        if (!std::isfinite(rn)) { chns_set_error("non-finite residual norm"); result = CHNS_ENAN; break; }
        if (rn <= o->atol || rn <= o->rtol * r0) break;
        if (it >= o->max_newton) { chns_set_error("Newton did not converge"); result = CHNS_ENOCONV; break; }

        // linearisation state and preconditioner (already built for the first iterate)
        if (it > 0) {
            if ((st = build_pc()) != CHNS_OK) return st;
            pc_pending = true;
        }

        // GMRES(mres) on J dU = -R, right preconditioned, from dU = 0
        CHNS_CUDA(cudaMemsetAsync(ws->dU, 0, c.n * sizeof(double), c.s));
        double rnorm = rn;
        int kry = 0;
        // r = -S R (S: row equilibration of this linearisation)
        { scale_vec_kernel<double><<<c.g, 256, 0, c.s>>>(ws->R, ws->S, ws->w, c.n); chns_count_launches(1); }
        { axpby_kernel<<<c.g, 256, 0, c.s>>>(0.0, ws->w, -1.0, ws->w, c.n); chns_count_launches(1); }
        {
            double bb;
            if ((st = dot_host(c, ws->w, ws->w, &bb)) != CHNS_OK) return st;
            rnorm = std::sqrt(bb);
        }
        const double bnorm_s = rnorm;
        // forcing term: krylov_rtol (or the Eisenstat-Walker term with ew_eta0 > 0),
        // relaxed once the Newton target is near (a solve below a tenth of what the
        // target needs is wasted)
        const double target = std::max(o->atol, o->rtol * r0);
        double eta_k = o->krylov_rtol;
        if (o->ew_eta0 > 0.0) {
            // Eisenstat-Walker choice 2 (gamma 0.9, alpha 2) with their safeguard
            if (it == 0) {
                eta_k = o->ew_eta0;
            } else {
                const double ratio = rn / rn_prev;
                eta_k = 0.9 * ratio * ratio;
                const double guard = 0.9 * eta_prev * eta_prev;
                if (guard > 0.1) eta_k = std::max(eta_k, guard);
            }
            eta_k = std::min(0.9, std::max(o->krylov_rtol, eta_k));
        }
        const double eta = std::max(eta_k, std::min(0.5, 0.1 * target / rn));
        eta_prev = eta_k;
        rn_prev = rn;
        // w = S J M^{-1} S^{-1} V_j (similarity scaling: the eigenvalues are those of J M^{-1});
        // the J x / apply timing events come from set es (two sets alternate, so the next
        // vector's application can be queued before this one's events are read)
        auto apply_op = [&](int j, int es) -> chns_status {
            const double* Vj = ws->V + (size_t)j * c.n;
            cudaEvent_t* E = ws->ev + 8 * es;
            CHNS_CUDA(cudaEventRecord(E[4], c.s));
            { unscale_kernel<<<c.g, 256, 0, c.s>>>(Vj, ws->Sd, ws->SR, c.n); chns_count_launches(1); }
            if (mixed) {
                { pc_apply_kernel<float, float><<<gN, 128, 0, c.s>>>(m->dm.N, NF, ws->Pinv32, ws->SR, ws->z32); chns_count_launches(1); }
                if (schur && (st = schur_apply_any((const double*)ws->SR, ws->z32)) != CHNS_OK) return st;
                if (chblk && (st = ch_apply_any((const double*)ws->SR, ws->z32)) != CHNS_OK) return st;
                if (pin == 2) pmean(ws->z32);
                CHNS_CUDA(cudaEventRecord(E[5], c.s));
                CHNS_CUDA(cudaEventRecord(E[0], c.s));
                CHNS_CUDA(launch_jvp32(m, pc, ws->Uo32, ws->Us32, ws->z32, ws->y32, pin, c.s));
                CHNS_CUDA(cudaEventRecord(E[1], c.s));
                if (pin == 2)
                    { scale_vec_pmean_kernel<float><<<c.g, 256, 0, c.s>>>(ws->y32, ws->S, ws->w, c.n, NF, D, ws->sc + 610, inv_vol); chns_count_launches(1); }
                else
                    { scale_vec_kernel<float><<<c.g, 256, 0, c.s>>>(ws->y32, ws->S, ws->w, c.n); chns_count_launches(1); }
            } else {
                { pc_apply_kernel<double, double><<<gN, 128, 0, c.s>>>(m->dm.N, NF, ws->Pinv64, ws->SR, ws->z64); chns_count_launches(1); }
                if (schur && (st = schur_apply_any((const double*)ws->SR, ws->z64)) != CHNS_OK) return st;
                if (chblk && (st = ch_apply_any((const double*)ws->SR, ws->z64)) != CHNS_OK) return st;
                if (pin == 2) pmean(ws->z64);
                CHNS_CUDA(cudaEventRecord(E[5], c.s));
                CHNS_CUDA(cudaEventRecord(E[0], c.s));
                CHNS_CUDA(launch_jvp64(m, pc, U_old, U, ws->z64, ws->t64, pin, c.s));
                CHNS_CUDA(cudaEventRecord(E[1], c.s));
                if (pin == 2)
                    { scale_vec_pmean_kernel<double><<<c.g, 256, 0, c.s>>>(ws->t64, ws->S, ws->w, c.n, NF, D, ws->sc + 610, inv_vol); chns_count_launches(1); }
                else
                    { scale_vec_kernel<double><<<c.g, 256, 0, c.s>>>(ws->t64, ws->S, ws->w, c.n); chns_count_launches(1); }
            }
            CHNS_CUDA(cudaGetLastError());
            S.jvp_calls++;
            return CHNS_OK;
        };
        while (true) {
            // V0 = r / ||r||
            double beta = rnorm;
            { axpby_kernel<<<c.g, 256, 0, c.s>>>(1.0 / beta, ws->w, 0.0, ws->V, c.n); chns_count_launches(1); }
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            int j = 0;
            bool done = false;
            if ((st = apply_op(0, 0)) != CHNS_OK) return st;
            for (; j < mres && kry < o->max_krylov; ++j, ++kry) {
                const int es = j & 1;
                // classical Gram-Schmidt with selective re-orthogonalisation (decided on the
                // device) and the next Arnoldi vector, all queued without a host round trip
                CHNS_CUDA(cudaEventRecord(ws->ev[6], c.s));
                {
                    // replayed from a CUDA graph of this j once captured (the launches are short)
                    bool done_g = false;
                    if (!ws->no_graphs && j < 257) {
                        if (!ws->orth_exec[j]) {
                            cudaGraph_t gr = nullptr;
                            cudaGraphExec_t ex = nullptr;
                            bool ok = ws->cap || cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking) == cudaSuccess;
                            if (ok) ok = cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                            if (ok) {
                                orth_enqueue(ws->cap, j);
                                ok = cudaStreamEndCapture(ws->cap, &gr) == cudaSuccess && gr != nullptr;
                                if (ok) ok = cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
                                if (gr) cudaGraphDestroy(gr);
                            }
                            if (ok) ws->orth_exec[j] = ex;
                            else { (void)cudaGetLastError(); ws->no_graphs = true; }
                        }
                        if (ws->orth_exec[j]) {
                            CHNS_CUDA(cudaGraphLaunch(ws->orth_exec[j], c.s));
                            done_g = true;
                        }
                    }
                    if (!done_g) orth_enqueue(c.s, j);
                    chns_count_launches(10);
                    CHNS_CUDA(cudaGetLastError());
                }
                CHNS_CUDA(cudaEventRecord(ws->ev[7], c.s));
                CHNS_CUDA(cudaEventRecord(ws->ev[10], c.s));
                // queue the next vector's operator application before reading the scalars, so
                // the GPU works on it while the host updates the Hessenberg column; if this
                // iteration turns out to be the last one, that result is simply not used
                if (j + 1 < mres && kry + 1 < o->max_krylov)
                    if ((st = apply_op(j + 1, es ^ 1)) != CHNS_OK) return st;
                CHNS_CUDA(cudaEventSynchronize(ws->ev[10]));
                {
                    cudaEvent_t* E = ws->ev + 8 * es;
                    float ms = 0.0f;
                    CHNS_CUDA(cudaEventElapsedTime(&ms, E[0], E[1]));
                    S.jvp_ms += ms;
                    CHNS_CUDA(cudaEventElapsedTime(&ms, E[4], E[5]));
                    S.apply_ms += ms;
                    CHNS_CUDA(cudaEventElapsedTime(&ms, ws->ev[6], ws->ev[7]));
                    S.orth_ms += ms;
                    if (pc_pending) {
                        CHNS_CUDA(cudaEventElapsedTime(&ms, ws->ev[2], ws->ev[3]));
                        S.pc_ms += ms;
                        pc_pending = false;
                    }
                }
                const double hn = std::sqrt(ws->hsc[603]);
                for (int i = 0; i <= j; ++i) H[(size_t)i * mres + j] = ws->hsc[i] + ws->hsc[256 + i];
                H[(size_t)(j + 1) * mres + j] = hn;
                if (!std::isfinite(hn)) { chns_set_error("non-finite Arnoldi vector"); S.reason = CHNS_EBREAKDOWN; result = CHNS_EBREAKDOWN; break; }
                // Givens rotations
                for (int i = 0; i < j; ++i) {
                    const double a = H[(size_t)i * mres + j], b = H[(size_t)(i + 1) * mres + j];
                    H[(size_t)i * mres + j] = cs[i] * a + sn[i] * b;
                    H[(size_t)(i + 1) * mres + j] = -sn[i] * a + cs[i] * b;
                }
                const double a = H[(size_t)j * mres + j], b = H[(size_t)(j + 1) * mres + j];
                const double r = std::hypot(a, b);
                cs[j] = r > 0 ? a / r : 1.0;
                sn[j] = r > 0 ? b / r : 0.0;
                H[(size_t)j * mres + j] = r;
                H[(size_t)(j + 1) * mres + j] = 0.0;
                gv[j + 1] = -sn[j] * gv[j];
                gv[j] = cs[j] * gv[j];
                rnorm = std::fabs(gv[j + 1]);
                if (rnorm <= eta * bnorm_s || hn == 0.0) {
                    ++j;
                    ++kry;
                    done = true;
                    break;
                }
            }
            if (result != CHNS_OK) break;
            // y = H^{-1} g, dU += M^{-1} V y
            const int k = j;
            for (int i = k - 1; i >= 0; --i) {
                double s = gv[i];
                for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * mres + l] * y[l];
                y[i] = s / H[(size_t)i * mres + i];
            }
            std::memcpy(ws->hsc, y.data(), k * sizeof(double));
            CHNS_CUDA(cudaMemcpyAsync(ws->sc, ws->hsc, k * sizeof(double), cudaMemcpyHostToDevice, c.s));
            { combine_kernel<<<c.g, 256, 0, c.s>>>(ws->V, c.n, k, ws->sc, ws->t64, c.n); chns_count_launches(1); }
            { unscale_kernel<<<c.g, 256, 0, c.s>>>(ws->t64, ws->Sd, ws->SR, c.n); chns_count_launches(1); }
            if (mixed)
                { pc_apply_kernel<float, double><<<gN, 128, 0, c.s>>>(m->dm.N, NF, ws->Pinv32, ws->SR, ws->z64); chns_count_launches(1); }
            else
                { pc_apply_kernel<double, double><<<gN, 128, 0, c.s>>>(m->dm.N, NF, ws->Pinv64, ws->SR, ws->z64); chns_count_launches(1); }
            if (schur && (st = schur_apply_any((const double*)ws->SR, ws->z64)) != CHNS_OK) return st;
            if (chblk && (st = ch_apply_any((const double*)ws->SR, ws->z64)) != CHNS_OK) return st;
            { axpy_kernel<<<c.g, 256, 0, c.s>>>(1.0, ws->z64, ws->dU, c.n); chns_count_launches(1); }
            CHNS_CUDA(cudaGetLastError());
            if (done || kry >= o->max_krylov) break;
            // restart: r = -R - J dU (same operator as the Arnoldi process)
            if (mixed) {
                { to32_kernel<<<c.g, 256, 0, c.s>>>(ws->dU, ws->z32, c.n); chns_count_launches(1); }
                CHNS_CUDA(cudaEventRecord(ws->ev[0], c.s));
                CHNS_CUDA(launch_jvp32(m, pc, ws->Uo32, ws->Us32, ws->z32, ws->y32, pin, c.s));
                CHNS_CUDA(cudaEventRecord(ws->ev[1], c.s));
                { to64_kernel<<<c.g, 256, 0, c.s>>>(ws->y32, ws->w, c.n); chns_count_launches(1); }
            } else {
                CHNS_CUDA(cudaEventRecord(ws->ev[0], c.s));
                CHNS_CUDA(launch_jvp64(m, pc, U_old, U, ws->dU, ws->w, pin, c.s));
                CHNS_CUDA(cudaEventRecord(ws->ev[1], c.s));
            }
            S.jvp_calls++;
            { axpby_kernel<<<c.g, 256, 0, c.s>>>(-1.0, ws->R, -1.0, ws->w, c.n); chns_count_launches(1); }
            if (pin == 2) {
                pmean(ws->dU);
                { scale_vec_pmean_kernel<double><<<c.g, 256, 0, c.s>>>(ws->w, ws->S, ws->w, c.n, NF, D, ws->sc + 610, -inv_vol); chns_count_launches(1); }
            } else {
                { scale_vec_kernel<double><<<c.g, 256, 0, c.s>>>(ws->w, ws->S, ws->w, c.n); chns_count_launches(1); }
            }
            double rr;
            if ((st = dot_host(c, ws->w, ws->w, &rr)) != CHNS_OK) return st;
            rnorm = std::sqrt(rr);
            {
                float ms = 0.0f;
                CHNS_CUDA(cudaEventElapsedTime(&ms, ws->ev[0], ws->ev[1]));
                S.jvp_ms += ms;
            }
            if (rnorm <= eta * bnorm_s) break;
        }
        S.krylov_its += kry;
        if (it < CHNS_HIST) S.krylov_hist[it] = kry;
        if (result != CHNS_OK) break;
        if (pin == 2) {
            // keep int p^{k+1} = int p^k: remove the mean of the pressure update (the
            // constant pressure spans the null space of J when no row is pinned)
            const int nbk = c.g < 1024 ? c.g : 1024;
            { field_mass_kernel<<<nbk, 256, 0, c.s>>>(m->d_nmass, ws->dU, NF, D, m->dm.N, m->d_partials); chns_count_launches(1); }
            { final_reduce_kernel<<<1, 256, 0, c.s>>>(m->d_partials, nbk, 1, ws->sc + 600); chns_count_launches(1); }
            { field_shift_kernel<<<c.g, 256, 0, c.s>>>(ws->dU, NF, D, m->dm.N, ws->sc + 600, 1.0 / m->volume); chns_count_launches(1); }
            CHNS_CUDA(cudaGetLastError());
        }
        {
            // keep int phi^{k+1} = int phi^k (Proposition 1, exact for the solution of the
            // discrete system) for every inexact iterate too: shift the phi update by the
            // constant that removes the mass change (the nodal masses sum to |Omega|)
            const int nbk = c.g < 1024 ? c.g : 1024;
            { field_mass3_kernel<<<nbk, 256, 0, c.s>>>(m->d_nmass, U, ws->dU, U_old, NF, D + 1, m->dm.N, m->d_partials); chns_count_launches(1); }
            { final_reduce_kernel<<<1, 256, 0, c.s>>>(m->d_partials, nbk, 1, ws->sc + 606); chns_count_launches(1); }
            { field_shift_kernel<<<c.g, 256, 0, c.s>>>(ws->dU, NF, D + 1, m->dm.N, ws->sc + 606, 1.0 / m->volume); chns_count_launches(1); }
            CHNS_CUDA(cudaGetLastError());
        }
        { axpy_kernel<<<c.g, 256, 0, c.s>>>(1.0, ws->dU, U, c.n); chns_count_launches(1); }
        double du;
        if ((st = dot_host(c, ws->dU, ws->dU, &du)) != CHNS_OK) return st;
        S.du_norm = std::sqrt(du);
    }
    S.reason = result;
    if (stats) *stats = S;
    return result;
}

extern "C" chns_status chns_initial_mu(const chns_mesh* mc, const chns_params* p, double* U, void* stream) {
    if (chns_require_q1(mc, "chns_initial_mu") != CHNS_OK) return CHNS_EINVAL;
    chns_mesh* m = const_cast<chns_mesh*>(mc);
    PhysConst pc;
    chns_status st = chns_check_params(mc, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U) { chns_set_error("null argument"); return CHNS_EINVAL; }
    if ((st = ensure_ws(m, m->ws ? m->ws->restart : 1)) != CHNS_OK) return st;
    SolverWS* ws = m->ws;
    const int64_t N = m->dm.N;
    Ctx c{m, ws, (cudaStream_t)stream, N, grid_for(N)};
    const int D = m->dm.dim, NF = m->dm.nf;
    const int gE = (int)((m->dm.E + 127) / 128), gN = (int)((N + 255) / 256);
    // work vectors (each N doubles) carved from the Krylov workspace
    double* b = ws->w;
    double* x = ws->R;
    double* r = ws->dU;
    double* z = ws->z64;
    double* q = ws->t64;
    double* dg = ws->V;
    double* pvec = ws->V + N;
    const double Cn2 = p->Cn * p->Cn;
    cudaError_t e = cudaMemsetAsync(b, 0, N * sizeof(double), c.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dg, 0, N * sizeof(double), c.s);
    if (e != cudaSuccess) return chns_cuda_status(e, "cudaMemsetAsync");
    if (D == 2) {
        { mu_kernel<2, 0><<<gE, 128, 0, c.s>>>(m->dm, Cn2, U, nullptr, b); chns_count_launches(1); }
    } else {
        { mu_kernel<3, 0><<<gE, 128, 0, c.s>>>(m->dm, Cn2, U, nullptr, b); chns_count_launches(1); }
    }
    // Jacobi scaling by the row sums of M (the integral of each basis function, > 0)
    { fill_kernel<<<c.g, 256, 0, c.s>>>(q, 1.0, N); chns_count_launches(1); }
    if (D == 2)
        { mu_kernel<2, 1><<<gE, 128, 0, c.s>>>(m->dm, Cn2, U, q, dg); chns_count_launches(1); }
    else
        { mu_kernel<3, 1><<<gE, 128, 0, c.s>>>(m->dm, Cn2, U, q, dg); chns_count_launches(1); }
    CHNS_CUDA(cudaGetLastError());
    // CG from x = 0
    CHNS_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), c.s));
    { copy64_kernel<<<c.g, 256, 0, c.s>>>(b, r, N); chns_count_launches(1); }
    { jacobi_kernel<<<gN, 256, 0, c.s>>>(dg, r, z, N); chns_count_launches(1); }
    { copy64_kernel<<<c.g, 256, 0, c.s>>>(z, pvec, N); chns_count_launches(1); }
    double rz, bb;
    if ((st = dot_host(c, r, z, &rz)) != CHNS_OK) return st;
    if ((st = dot_host(c, b, b, &bb)) != CHNS_OK) return st;
    const double tol = 1e-14 * std::sqrt(bb);
    int it = 0;
    for (; it < 1000 && bb > 0.0; ++it) {
        CHNS_CUDA(cudaMemsetAsync(q, 0, N * sizeof(double), c.s));
        if (D == 2)
            { mu_kernel<2, 1><<<gE, 128, 0, c.s>>>(m->dm, Cn2, U, pvec, q); chns_count_launches(1); }
        else
            { mu_kernel<3, 1><<<gE, 128, 0, c.s>>>(m->dm, Cn2, U, pvec, q); chns_count_launches(1); }
        double pq, rr;
        if ((st = dot_host(c, pvec, q, &pq)) != CHNS_OK) return st;
        const double alpha = rz / pq;
        { axpy_kernel<<<c.g, 256, 0, c.s>>>(alpha, pvec, x, N); chns_count_launches(1); }
        { axpy_kernel<<<c.g, 256, 0, c.s>>>(-alpha, q, r, N); chns_count_launches(1); }
        if ((st = dot_host(c, r, r, &rr)) != CHNS_OK) return st;
        if (!std::isfinite(rr)) { chns_set_error("non-finite CG residual"); return CHNS_ENAN; }
        if (std::sqrt(rr) <= tol) break;
        { jacobi_kernel<<<gN, 256, 0, c.s>>>(dg, r, z, N); chns_count_launches(1); }
        double rz2;
        if ((st = dot_host(c, r, z, &rz2)) != CHNS_OK) return st;
        { axpby_kernel<<<c.g, 256, 0, c.s>>>(1.0, z, rz2 / rz, pvec, N); chns_count_launches(1); }
        rz = rz2;
    }
    { insert_mu_kernel<<<gN, 256, 0, c.s>>>(x, NF, D + 2, N, U); chns_count_launches(1); }
    CHNS_CUDA(cudaGetLastError());
    CHNS_CUDA(cudaStreamSynchronize(c.s));
    if (it >= 1000) { chns_set_error("mass-matrix CG did not converge"); return CHNS_ENOCONV; }
    return CHNS_OK;
}

// ---------------------------------------------------------------------------------
// Adjoint of one implicit step (reverse mode through Section 3.4's solve): with
// R(U^k, U^{k+1}; Cn) = 0, a cotangent g of U^{k+1} gives J^T lambda = P^T g
// (J = dR/dU^{k+1}; P the pressure-level normalisation of pin mode 2) and the
// cotangents -(dR/dU^k)^T lambda of U^k and -(dR/dCn)^T lambda of Cn.
// ---------------------------------------------------------------------------------
namespace {

template <class TI>
__global__ void pc_apply_T_kernel(int64_t N, int NF, const TI* __restrict__ inv, const double* __restrict__ v,
                                  double* __restrict__ z) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double x[6];
    for (int j = 0; j < NF; ++j) x[j] = v[(size_t)n * NF + j];
    for (int i = 0; i < NF; ++i) {
        double s = 0.0;
        for (int j = 0; j < NF; ++j) s += (double)inv[((size_t)n * NF + j) * NF + i] * x[j];
        z[(size_t)n * NF + i] = s;
    }
}

// unweighted sum of field f into per-block partials
__global__ void field_sum_kernel(const double* __restrict__ v, int NF, int f, int64_t N, double* partials) {
    double acc[1] = {0.0};
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        acc[0] += v[(size_t)n * NF + f];
    block_reduce_store<1>(acc, partials);
}
// sum_n wt[n*NF + f] v[n*NF + f] into per-block partials
__global__ void field_wdot_kernel(const double* __restrict__ wt, const double* __restrict__ v, int NF, int f,
                                  int64_t N, double* partials) {
    double acc[1] = {0.0};
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        acc[0] += wt[(size_t)n * NF + f] * v[(size_t)n * NF + f];
    block_reduce_store<1>(acc, partials);
}
// v[n*NF + f] += a * m[n] * sc[0]
__global__ void field_axpy_mass_kernel(double* __restrict__ v, int NF, int f, int64_t N, const double* __restrict__ m,
                                       const double* __restrict__ sc, double a) {
    const double s = a * sc[0];
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        v[(size_t)n * NF + f] += s * m[n];
}

}  // namespace

extern "C" chns_status chns_step_adjoint(const chns_mesh* mc, const chns_params* p, const chns_solver_opts* o,
                                         const double* U_old, const double* U_new, const double* g, double* lambda,
                                         double* gU_old, double* gCn, chns_stats* stats, void* stream) {
    if (chns_require_q1(mc, "chns_step_adjoint") != CHNS_OK) return CHNS_EINVAL;
    chns_mesh* m = const_cast<chns_mesh*>(mc);
    PhysConst pc;
    chns_status st = chns_check_params(mc, p, &pc);
    if (st != CHNS_OK) return st;
    if (!o || !U_old || !U_new || !g || !lambda || !gU_old) { chns_set_error("null argument"); return CHNS_EINVAL; }
    if ((st = chns_check_rows(mc, U_old, 8)) != CHNS_OK || (st = chns_check_rows(mc, U_new, 8)) != CHNS_OK) return st;
    if (o->restart < 1 || o->restart > MAXSC / 4 || o->max_krylov < 1 || o->pc_type < 0 || o->pc_type > 4 ||
        (o->pc_type >= 1 && (o->pc_degree < 2 || o->pc_degree > 200))) {
        chns_set_error("bad solver options (restart in [1, 256], max_krylov >= 1, pc_type 0..4, pc_degree in [2, 200])");
        return CHNS_EINVAL;
    }
    if ((st = ensure_ws(m, o->restart)) != CHNS_OK) return st;
    SolverWS* ws = m->ws;
    Ctx c{m, ws, (cudaStream_t)stream, ws->n, 0};
    c.g = grid_for(c.n);
    const int D = m->dm.dim, NF = m->dm.nf, mres = o->restart, pin = p->pin_pressure;
    // the pressure Schur approximation is symmetric, so J^T takes it as J does; the
    // Cahn-Hilliard block of pc_type 2 / 4 is not used here
    const bool schur = o->pc_type >= 1;
    SchurPC spc(m, ws, c.s, o->pc_degree, o->pc_type >= 3);
    const int gN = (int)((m->dm.N + 127) / 128);
    const int nbk = c.g < 1024 ? c.g : 1024;
    chns_stats S;
    std::memset(&S, 0, sizeof(S));

    // nodal blocks of J (FP64) at the converged state; J^T's blocks are their transposes
    cudaError_t ce = (D == 2) ? pc_build_launch<2, double>(m, pc, U_old, U_new, ws->Pblk64, ws->ce, c.s)
                              : pc_build_launch<3, double>(m, pc, U_old, U_new, ws->Pblk64, ws->ce, c.s);
    CHNS_CUDA(ce);
    { pc_invert_kernel<double, double><<<gN, 128, 0, c.s>>>(m->dm, ws->Pblk64, ws->Pinv64, pin, ws->S, ws->Sd, schur ? 1 : 0); chns_count_launches(1); }
    if (schur && (st = spc.setup()) != CHNS_OK) return st;
    // pin mode 2: J' = J + u m_p^T / |Omega| with u = |diag J| on the pressure rows is
    // nonsingular, and J'^T lambda = P^T g has the solution of J^T lambda = P^T g with
    // u^T lambda = 0 (GMRES on the singular J^T drifts along its null vector)
    const double inv_vol = 1.0 / m->volume;
    auto add_pmean_T = [&](const double* v, double* y) {
        { field_wdot_kernel<<<nbk, 256, 0, c.s>>>(ws->Sd, v, NF, D, m->dm.N, m->d_partials); chns_count_launches(1); }
        { final_reduce_kernel<<<1, 256, 0, c.s>>>(m->d_partials, nbk, 1, ws->sc + 820); chns_count_launches(1); }
        { field_axpy_mass_kernel<<<c.g, 256, 0, c.s>>>(y, NF, D, m->dm.N, m->d_nmass, ws->sc + 820, inv_vol); chns_count_launches(1); }
    };
    // b = P^T g: remove sum(g_p) * m / |Omega| from the pressure part (pin mode 2)
    double* b = ws->R;
    { copy64_kernel<<<c.g, 256, 0, c.s>>>(g, b, c.n); chns_count_launches(1); }
    if (pin == 2) {
        { field_sum_kernel<<<nbk, 256, 0, c.s>>>(g, NF, D, m->dm.N, m->d_partials); chns_count_launches(1); }
        { final_reduce_kernel<<<1, 256, 0, c.s>>>(m->d_partials, nbk, 1, ws->sc + 800); chns_count_launches(1); }
        { field_axpy_mass_kernel<<<c.g, 256, 0, c.s>>>(b, NF, D, m->dm.N, m->d_nmass, ws->sc + 800, -1.0 / m->volume); chns_count_launches(1); }
    }
    CHNS_CUDA(cudaGetLastError());
    double bb;
    if ((st = dot_host(c, b, b, &bb)) != CHNS_OK) return st;
    const double bnorm = std::sqrt(bb);
    CHNS_CUDA(cudaMemsetAsync(lambda, 0, c.n * sizeof(double), c.s));
    S.res0 = bnorm;
    chns_status result = CHNS_OK;
    if (bnorm > 0.0) {
        // right-preconditioned GMRES on J^T M^{-T} y = b, lambda = M^{-T} y
        std::vector<double> H((size_t)(mres + 1) * mres), cs(mres), sn(mres), gv(mres + 1), y(mres);
        double rnorm = bnorm;
        int kry = 0;
        { copy64_kernel<<<c.g, 256, 0, c.s>>>(b, ws->w, c.n); chns_count_launches(1); }
        while (true) {
            const double beta = rnorm;
            { axpby_kernel<<<c.g, 256, 0, c.s>>>(1.0 / beta, ws->w, 0.0, ws->V, c.n); chns_count_launches(1); }
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            int j = 0;
            bool done = false;
            for (; j < mres && kry < o->max_krylov; ++j, ++kry) {
                double* Vj = ws->V + (size_t)j * c.n;
                { pc_apply_T_kernel<double><<<gN, 128, 0, c.s>>>(m->dm.N, NF, ws->Pinv64, Vj, ws->z64); chns_count_launches(1); }
                if (schur && (st = spc.apply((const double*)Vj, ws->z64)) != CHNS_OK) return st;
                CHNS_CUDA(launch_vjp(m, pc, U_old, U_new, ws->z64, ws->w, nullptr, nullptr, pin, c.s));
                if (pin == 2) add_pmean_T(ws->z64, ws->w);
                S.jvp_calls++;
                CHNS_CUDA(launch_multidot(m, ws->V, c.n, j + 1, ws->w, c.n, ws->sc, c.s));
                { gs_update_kernel<<<c.g, 256, 0, c.s>>>(ws->V, c.n, j + 1, ws->sc, ws->w, c.n); chns_count_launches(1); }
                CHNS_CUDA(launch_multidot(m, ws->V, c.n, j + 1, ws->w, c.n, ws->sc + 256, c.s));
                { gs_update_kernel<<<c.g, 256, 0, c.s>>>(ws->V, c.n, j + 1, ws->sc + 256, ws->w, c.n); chns_count_launches(1); }
                CHNS_CUDA(launch_dot(m, ws->w, ws->w, c.n, ws->sc + 512, c.s));
                double hs[513];
                CHNS_CUDA(cudaMemcpyAsync(ws->hsc, ws->sc, 513 * sizeof(double), cudaMemcpyDeviceToHost, c.s));
                CHNS_CUDA(cudaStreamSynchronize(c.s));
                std::memcpy(hs, ws->hsc, 513 * sizeof(double));
                const double hn = std::sqrt(hs[512]);
                for (int i = 0; i <= j; ++i) H[(size_t)i * mres + j] = hs[i] + hs[256 + i];
                H[(size_t)(j + 1) * mres + j] = hn;
                if (!std::isfinite(hn)) { chns_set_error("non-finite Arnoldi vector"); result = CHNS_EBREAKDOWN; break; }
                for (int i = 0; i < j; ++i) {
                    const double a = H[(size_t)i * mres + j], bq = H[(size_t)(i + 1) * mres + j];
                    H[(size_t)i * mres + j] = cs[i] * a + sn[i] * bq;
                    H[(size_t)(i + 1) * mres + j] = -sn[i] * a + cs[i] * bq;
                }
                const double a = H[(size_t)j * mres + j], bq = H[(size_t)(j + 1) * mres + j];
                const double r = std::hypot(a, bq);
                cs[j] = r > 0 ? a / r : 1.0;
                sn[j] = r > 0 ? bq / r : 0.0;
                H[(size_t)j * mres + j] = r;
                H[(size_t)(j + 1) * mres + j] = 0.0;
                gv[j + 1] = -sn[j] * gv[j];
                gv[j] = cs[j] * gv[j];
                rnorm = std::fabs(gv[j + 1]);
                if (hn > 0.0)
                    { axpby_kernel<<<c.g, 256, 0, c.s>>>(1.0 / hn, ws->w, 0.0, ws->V + (size_t)(j + 1) * c.n, c.n); chns_count_launches(1); }
                if (rnorm <= o->krylov_rtol * bnorm || hn == 0.0) {
                    ++j;
                    ++kry;
                    done = true;
                    break;
                }
            }
            if (result != CHNS_OK) break;
            const int k = j;
            for (int i = k - 1; i >= 0; --i) {
                double sacc = gv[i];
                for (int l = i + 1; l < k; ++l) sacc -= H[(size_t)i * mres + l] * y[l];
                y[i] = sacc / H[(size_t)i * mres + i];
            }
            std::memcpy(ws->hsc, y.data(), k * sizeof(double));
            CHNS_CUDA(cudaMemcpyAsync(ws->sc, ws->hsc, k * sizeof(double), cudaMemcpyHostToDevice, c.s));
            { combine_kernel<<<c.g, 256, 0, c.s>>>(ws->V, c.n, k, ws->sc, ws->t64, c.n); chns_count_launches(1); }
            { pc_apply_T_kernel<double><<<gN, 128, 0, c.s>>>(m->dm.N, NF, ws->Pinv64, ws->t64, ws->z64); chns_count_launches(1); }
            if (schur && (st = spc.apply((const double*)ws->t64, ws->z64)) != CHNS_OK) return st;
            { axpy_kernel<<<c.g, 256, 0, c.s>>>(1.0, ws->z64, lambda, c.n); chns_count_launches(1); }
            CHNS_CUDA(cudaGetLastError());
            if (done || kry >= o->max_krylov) break;
            // restart: r = b - J^T lambda
            CHNS_CUDA(launch_vjp(m, pc, U_old, U_new, lambda, ws->w, nullptr, nullptr, pin, c.s));
            if (pin == 2) add_pmean_T(lambda, ws->w);
            S.jvp_calls++;
            { axpby_kernel<<<c.g, 256, 0, c.s>>>(1.0, b, -1.0, ws->w, c.n); chns_count_launches(1); }
            double rr;
            if ((st = dot_host(c, ws->w, ws->w, &rr)) != CHNS_OK) return st;
            rnorm = std::sqrt(rr);
            if (rnorm <= o->krylov_rtol * bnorm) break;
        }
        S.krylov_its = kry;
        S.res_final = rnorm;
        if (result == CHNS_OK && rnorm > o->krylov_rtol * bnorm * 1.0001) {
            chns_set_error("adjoint GMRES did not reach krylov_rtol within max_krylov");
            result = CHNS_ENOCONV;
        }
    }
    // cotangents of U^k and Cn: -(dR/dU^k)^T lambda, -(dR/dCn)^T lambda
    CHNS_CUDA(launch_vjp(m, pc, U_old, U_new, lambda, ws->t64, gU_old, gCn, pin, c.s));
    { axpby_kernel<<<c.g, 256, 0, c.s>>>(0.0, gU_old, -1.0, gU_old, c.n); chns_count_launches(1); }
    if (gCn) { axpby_kernel<<<1, 32, 0, c.s>>>(0.0, gCn, -1.0, gCn, 1); chns_count_launches(1); }
    if (pin == 2) {
        // the normalisation int p^{k+1} = int p^k passes sum(g_p) m / |Omega| to p^k
        { field_axpy_mass_kernel<<<c.g, 256, 0, c.s>>>(gU_old, NF, D, m->dm.N, m->d_nmass, ws->sc + 800, 1.0 / m->volume); chns_count_launches(1); }
    }
    CHNS_CUDA(cudaGetLastError());
    CHNS_CUDA(cudaStreamSynchronize(c.s));
    S.reason = result;
    if (stats) *stats = S;
    return result;
}

// M x = rhs with the consistent Q1 mass matrix (hanging constraints included), by
// Jacobi-preconditioned CG to a relative residual of 1e-14.  Used by the reverse mode
// of mu^0 (M is symmetric, so its adjoint is the same solve).
extern "C" chns_status chns_mass_solve(const chns_mesh* mc, const double* rhs, double* x, void* stream) {
    if (chns_require_q1(mc, "chns_mass_solve") != CHNS_OK) return CHNS_EINVAL;
    chns_mesh* m = const_cast<chns_mesh*>(mc);
    if (!m || !rhs || !x) { chns_set_error("null argument"); return CHNS_EINVAL; }
    chns_status st = ensure_ws(m, m->ws ? m->ws->restart : 1);
    if (st != CHNS_OK) return st;
    SolverWS* ws = m->ws;
    const int64_t N = m->dm.N;
    const int D = m->dm.dim;
    Ctx c{m, ws, (cudaStream_t)stream, N, grid_for(N)};
    const int gE = (int)((m->dm.E + 127) / 128), gN = (int)((N + 255) / 256);
    double* r = ws->dU;
    double* z = ws->z64;
    double* q = ws->t64;
    double* dg = ws->V;
    double* pvec = ws->V + N;
    CHNS_CUDA(cudaMemsetAsync(dg, 0, N * sizeof(double), c.s));
    { fill_kernel<<<c.g, 256, 0, c.s>>>(q, 1.0, N); chns_count_launches(1); }
    if (D == 2) { mu_kernel<2, 1><<<gE, 128, 0, c.s>>>(m->dm, 0.0, nullptr, q, dg); chns_count_launches(1); }
    else { mu_kernel<3, 1><<<gE, 128, 0, c.s>>>(m->dm, 0.0, nullptr, q, dg); chns_count_launches(1); }
    CHNS_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), c.s));
    { copy64_kernel<<<c.g, 256, 0, c.s>>>(rhs, r, N); chns_count_launches(1); }
    { jacobi_kernel<<<gN, 256, 0, c.s>>>(dg, r, z, N); chns_count_launches(1); }
    { copy64_kernel<<<c.g, 256, 0, c.s>>>(z, pvec, N); chns_count_launches(1); }
    CHNS_CUDA(cudaGetLastError());
    double rz, bb;
    if ((st = dot_host(c, r, z, &rz)) != CHNS_OK) return st;
    if ((st = dot_host(c, rhs, rhs, &bb)) != CHNS_OK) return st;
    const double tol = 1e-14 * std::sqrt(bb);
    int it = 0;
    for (; it < 1000 && bb > 0.0; ++it) {
        CHNS_CUDA(cudaMemsetAsync(q, 0, N * sizeof(double), c.s));
        if (D == 2) { mu_kernel<2, 1><<<gE, 128, 0, c.s>>>(m->dm, 0.0, nullptr, pvec, q); chns_count_launches(1); }
        else { mu_kernel<3, 1><<<gE, 128, 0, c.s>>>(m->dm, 0.0, nullptr, pvec, q); chns_count_launches(1); }
        double pq, rr;
        if ((st = dot_host(c, pvec, q, &pq)) != CHNS_OK) return st;
        const double alpha = rz / pq;
        { axpy_kernel<<<c.g, 256, 0, c.s>>>(alpha, pvec, x, N); chns_count_launches(1); }
        { axpy_kernel<<<c.g, 256, 0, c.s>>>(-alpha, q, r, N); chns_count_launches(1); }
        if ((st = dot_host(c, r, r, &rr)) != CHNS_OK) return st;
        if (!std::isfinite(rr)) { chns_set_error("non-finite CG residual"); return CHNS_ENAN; }
        if (std::sqrt(rr) <= tol) break;
        { jacobi_kernel<<<gN, 256, 0, c.s>>>(dg, r, z, N); chns_count_launches(1); }
        double rz2;
        if ((st = dot_host(c, r, z, &rz2)) != CHNS_OK) return st;
        { axpby_kernel<<<c.g, 256, 0, c.s>>>(1.0, z, rz2 / rz, pvec, N); chns_count_launches(1); }
        rz = rz2;
    }
    CHNS_CUDA(cudaGetLastError());
    CHNS_CUDA(cudaStreamSynchronize(c.s));
    if (it >= 1000) { chns_set_error("mass-matrix CG did not converge"); return CHNS_ENOCONV; }
    return CHNS_OK;
}
