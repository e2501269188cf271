// Triquadratic (Q2) elements (NEXT-4; the paper's manufactured-solution study, Section
// 5.1, uses quadratic elements): residual, J x (FP64 / FP32) and J^T w of Definition 2 on
// uniform octrees (no hanging nodes), with 3^d nodes per element and the 3-point Gauss
// rule per axis.
//
// Thread mapping: one group of 32 (3D) or 16 (2D) threads per element; during the gather
// lane a owns element node a, during the physics it owns Gauss point a, during the test
// contraction node a again (27 or 9 active lanes).  The basis values are products of the
// 1D quadratic Lagrange polynomials L_0 = xi (xi - 1)/2, L_1 = 1 - xi^2, L_2 = xi (xi + 1)/2
// at the Gauss points (0, +-sqrt(3/5)), evaluated on the fly.  Unlike Q1, the pure second
// derivatives do not vanish: the strong residuals take the full Hessian of phi and the
// Laplacians of v and mu (pointwise<..., Q2 = true>).
#include <cuda_runtime.h>

#include <type_traits>

#include "chns_internal.h"
#include "pointwise.cuh"

namespace {

template <int D>
struct Q2S {
    static constexpr int NN = D == 2 ? 9 : 27;    // nodes = Gauss points per element
    static constexpr int NF = D + 3;
    static constexpr int TPE = D == 2 ? 16 : 32;  // threads per element
    static constexpr int EPB = 128 / TPE;         // elements per block
    static constexpr int NH = D == 2 ? 1 : 3;
};

template <class T> struct G3;
template <> struct G3<double> {
    static __device__ __forceinline__ double pt(int i) { return i == 0 ? -0.77459666924148337704 : (i == 1 ? 0.0 : 0.77459666924148337704); }
    static __device__ __forceinline__ double wt(int i) { return i == 1 ? 0.88888888888888888889 : 0.55555555555555555556; }
};
template <> struct G3<float> {
    static __device__ __forceinline__ float pt(int i) { return i == 0 ? -0.77459666924148337704f : (i == 1 ? 0.0f : 0.77459666924148337704f); }
    static __device__ __forceinline__ float wt(int i) { return i == 1 ? 0.88888888888888888889f : 0.55555555555555555556f; }
};

template <class T>
__device__ __forceinline__ void lag1(int j, T t, T& L, T& dL, T& d2L) {
    if (j == 0) { L = T(0.5) * t * (t - T(1)); dL = t - T(0.5); d2L = T(1); }
    else if (j == 1) { L = T(1) - t * t; dL = T(-2) * t; d2L = T(-2); }
    else { L = T(0.5) * t * (t + T(1)); dL = t + T(0.5); d2L = T(1); }
}

// physical basis of node a at Gauss point q: value, gradient, Hessian (pure: hd[k]; mixed in
// the packed order xy, xz, yz), h: element size
template <int D, class T>
struct QB {
    T N, dN[D], hd[D], hm[Q2S<D>::NH];
};
template <int D, class T>
__device__ __forceinline__ QB<D, T> qbasis(int a, int q, T inv_h) {
    T L[D], dL[D], d2L[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        int ak = a, qk = q;
        for (int i = 0; i < k; ++i) { ak /= 3; qk /= 3; }
        lag1<T>(ak % 3, G3<T>::pt(qk % 3), L[k], dL[k], d2L[k]);
        const T s = T(2) * inv_h;            // d xi / d x
        dL[k] *= s;
        d2L[k] *= s * s;
    }
    QB<D, T> b;
    if constexpr (D == 2) {
        b.N = L[0] * L[1];
        b.dN[0] = dL[0] * L[1];
        b.dN[1] = L[0] * dL[1];
        b.hd[0] = d2L[0] * L[1];
        b.hd[1] = L[0] * d2L[1];
        b.hm[0] = dL[0] * dL[1];
    } else {
        b.N = L[0] * L[1] * L[2];
        b.dN[0] = dL[0] * L[1] * L[2];
        b.dN[1] = L[0] * dL[1] * L[2];
        b.dN[2] = L[0] * L[1] * dL[2];
        b.hd[0] = d2L[0] * L[1] * L[2];
        b.hd[1] = L[0] * d2L[1] * L[2];
        b.hd[2] = L[0] * L[1] * d2L[2];
        b.hm[0] = dL[0] * dL[1] * L[2];
        b.hm[1] = dL[0] * L[1] * dL[2];
        b.hm[2] = L[0] * dL[1] * dL[2];
    }
    return b;
}

template <int D, class T>
__device__ __forceinline__ T qweight(int q) {
    T w = T(1);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        w *= G3<T>::wt(q % 3);
        q /= 3;
    }
    return w;
}

template <class T>
__device__ __forceinline__ T clip1q(T x) { return x > T(1) ? T(1) : (x < T(-1) ? T(-1) : x); }

template <int D, class T, bool FLUX = true>
struct Q2Smem {
    T ut[Q2S<D>::NN][Q2S<D>::NF];
    T dd[Q2S<D>::NN][D + 1];
    T ps[Q2S<D>::NN];
    T x[Q2S<D>::NN][Q2S<D>::NF];     // tangent (J x) or adjoint seed (J^T w) rows
    T xps[Q2S<D>::NN];
    T f[FLUX ? Q2S<D>::NN : 1][Q2S<D>::NF * (D + 1)];
};

// primal (and tangent) interpolation at Gauss point q from the node data in shared memory
template <int D, class T, class S, bool FLUX>
__device__ __forceinline__ void q2_interp(const Q2Smem<D, T, FLUX>& M, int q, T inv_h, T inv_dt, QPIn<D, S>& X,
                                          bool tangent) {
    constexpr int NN = Q2S<D>::NN, NF = Q2S<D>::NF, NH = Q2S<D>::NH;
    T val[NF], grad[NF][D], lap[NF], hm[NH], hd[D], vd[D + 1], gdd[D], ps = T(0), gps[D];
    T tv[NF], tg[NF][D], tlap[NF], thm[NH], thd[D], tps = T(0), tgps[D];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        val[f] = lap[f] = tv[f] = tlap[f] = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) grad[f][k] = tg[f][k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < NH; ++k) hm[k] = thm[k] = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) hd[k] = thd[k] = gdd[k] = gps[k] = tgps[k] = T(0);
#pragma unroll
    for (int i = 0; i <= D; ++i) vd[i] = T(0);
    for (int a = 0; a < NN; ++a) {
        const QB<D, T> b = qbasis<D, T>(a, q, inv_h);
        T lapN = b.hd[0];
#pragma unroll
        for (int k = 1; k < D; ++k) lapN += b.hd[k];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T u = M.ut[a][f];
            val[f] += b.N * u;
#pragma unroll
            for (int k = 0; k < D; ++k) grad[f][k] += b.dN[k] * u;
            lap[f] += lapN * u;
        }
        const T uphi = M.ut[a][D + 1];
#pragma unroll
        for (int k = 0; k < NH; ++k) hm[k] += b.hm[k] * uphi;
#pragma unroll
        for (int k = 0; k < D; ++k) hd[k] += b.hd[k] * uphi;
#pragma unroll
        for (int i = 0; i <= D; ++i) vd[i] += b.N * M.dd[a][i];
#pragma unroll
        for (int k = 0; k < D; ++k) gdd[k] += b.dN[k] * M.dd[a][k];
        ps += b.N * M.ps[a];
#pragma unroll
        for (int k = 0; k < D; ++k) gps[k] += b.dN[k] * M.ps[a];
        if (tangent) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T u = M.x[a][f];
                tv[f] += b.N * u;
#pragma unroll
                for (int k = 0; k < D; ++k) tg[f][k] += b.dN[k] * u;
                tlap[f] += lapN * u;
            }
            const T xp = M.x[a][D + 1];
#pragma unroll
            for (int k = 0; k < NH; ++k) thm[k] += b.hm[k] * xp;
#pragma unroll
            for (int k = 0; k < D; ++k) thd[k] += b.hd[k] * xp;
            tps += b.N * M.xps[a];
#pragma unroll
            for (int k = 0; k < D; ++k) tgps[k] += b.dN[k] * M.xps[a];
        }
    }
    // assemble the quadrature-point input; tangents: averages move by x/2, differences by x
    auto mk = [&](T v, T d) -> S {
        if constexpr (std::is_same<S, T>::value) return v;
        else return S(v, d);
    };
    const T hf = T(0.5);
    T div = grad[0][0], tdiv = tg[0][0];
#pragma unroll
    for (int i = 1; i < D; ++i) { div += grad[i][i]; tdiv += tg[i][i]; }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        X.v[i] = mk(val[i], hf * tv[i]);
#pragma unroll
        for (int k = 0; k < D; ++k) X.gv[i][k] = mk(grad[i][k], hf * tg[i][k]);
        X.gp[i] = mk(grad[D][i], hf * tg[D][i]);
        X.gphi[i] = mk(grad[D + 1][i], hf * tg[D + 1][i]);
        X.gmu[i] = mk(grad[D + 2][i], hf * tg[D + 2][i]);
        X.vdt[i] = mk(vd[i] * inv_dt, inv_dt * tv[i]);
        X.gps[i] = mk(gps[i], tgps[i]);
        X.Hd[i] = mk(hd[i], hf * thd[i]);
        X.lapv[i] = mk(lap[i], hf * tlap[i]);
        div += hf * gdd[i];
    }
    X.p = mk(val[D], hf * tv[D]);
    X.phi = mk(val[D + 1], hf * tv[D + 1]);
    X.mu = mk(val[D + 2], hf * tv[D + 2]);
    X.lapmu = mk(lap[D + 2], hf * tlap[D + 2]);
#pragma unroll
    for (int k = 0; k < NH; ++k) X.H[k] = mk(hm[k], hf * thm[k]);
    X.phidt = mk(vd[D] * inv_dt, inv_dt * tv[D + 1]);
    X.divnew = mk(div, tdiv);
    X.ps = mk(ps, tps);
}

template <class R>
PCst<R> q2_pcst(const PhysConst& pc) {
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

enum { Q2_RES = 0, Q2_JVP = 1 };

template <int D, class T, int MODE>
__global__ void __launch_bounds__(128) q2_rj_kernel(DevMesh m, PCst<T> c, T inv_dt, T h, const T* __restrict__ Uo,
                                                    const T* __restrict__ Un, const T* __restrict__ xin,
                                                    T* __restrict__ out, unsigned int* __restrict__ flags) {
    constexpr int NN = Q2S<D>::NN, NF = Q2S<D>::NF, TPE = Q2S<D>::TPE, EPB = Q2S<D>::EPB;
    __shared__ Q2Smem<D, T> sm[EPB];
    const int le = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int64_t e = (int64_t)blockIdx.x * EPB + le;
    const bool valid = e < m.E && t < NN;
    Q2Smem<D, T>& S = sm[le];
    const T inv_h = T(1) / h;
    const T detJ = D == 2 ? T(0.25) * h * h : T(0.125) * h * h * h;
    int node = 0;
    if (valid) {
        node = m.e2n[e * NN + t];
        const T* po = Uo + (size_t)node * NF;
        const T* pn = Un + (size_t)node * NF;
        T o[NF], n[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            o[f] = po[f];
            n[f] = pn[f];
            S.ut[t][f] = T(0.5) * (o[f] + n[f]);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) S.dd[t][i] = n[i] - o[i];
        S.dd[t][D] = n[D + 1] - o[D + 1];
        const T avg = T(0.5) * (o[D + 1] + n[D + 1]);
        S.ps[t] = clip1q(avg);
        if (MODE == Q2_JVP) {
            const T* px = xin + (size_t)node * NF;
#pragma unroll
            for (int f = 0; f < NF; ++f) S.x[t][f] = px[f];
            S.xps[t] = (avg <= T(1) && avg >= T(-1)) ? T(0.5) * px[D + 1] : T(0);
        }
    }
    __syncwarp();
    if (valid) {
        const int q = t;
        const T g = T(4) * inv_h * inv_h;
        const T wq = detJ * qweight<D, T>(q);
        if (MODE == Q2_RES) {
            QPIn<D, T> X;
            q2_interp<D, T, T, true>(S, q, inv_h, inv_dt, X, false);
            QPOut<D, T> F;
            pointwise<D, T, T, true>(X, c, g, F);
            if (!(F.f1[D][0] == F.f1[D][0])) atomicOr(flags, 1u);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                S.f[q][f] = wq * F.f0[f];
#pragma unroll
                for (int k = 0; k < D; ++k) S.f[q][NF + f * D + k] = wq * F.f1[f][k];
            }
        } else {
            QPIn<D, Dual<T>> X;
            q2_interp<D, T, Dual<T>, true>(S, q, inv_h, inv_dt, X, true);
            QPOut<D, Dual<T>> F;
            pointwise<D, Dual<T>, T, true>(X, c, g, F);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                S.f[q][f] = wq * F.f0[f].d;
#pragma unroll
                for (int k = 0; k < D; ++k) S.f[q][NF + f * D + k] = wq * F.f1[f][k].d;
            }
        }
    }
    __syncwarp();
    if (valid) {
        const int a = t;
        T r[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) r[f] = T(0);
        for (int q = 0; q < NN; ++q) {
            const QB<D, T> b = qbasis<D, T>(a, q, inv_h);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T acc = b.N * S.f[q][f];
#pragma unroll
                for (int k = 0; k < D; ++k) acc += b.dN[k] * S.f[q][NF + f * D + k];
                r[f] += acc;
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) atomicAdd(out + (size_t)node * NF + f, r[f]);
    }
}

// J^T w on Q2 (FP64): the adjoint of the pointwise map at every Gauss point, then the
// transpose of the interpolation
template <int D>
__global__ void __launch_bounds__(D == 2 ? 128 : 64) q2_vjp_kernel(DevMesh m, PCst<double> c, double Cn, double inv_dt, double h,
                                                     const double* __restrict__ Uo, const double* __restrict__ Un,
                                                     const double* __restrict__ w, double* __restrict__ gn,
                                                     double* __restrict__ go, double* __restrict__ gCn) {
    constexpr int NN = Q2S<D>::NN, NF = Q2S<D>::NF, TPE = Q2S<D>::TPE, NH = Q2S<D>::NH;
    constexpr int EPB = (D == 2 ? 128 : 64) / TPE;
    // wb: seeds per node; xb: per Gauss point, the adjoints of the interpolated inputs
    constexpr int NXB = D + D * D + 1 + D + 1 + D + NH + 1 + D + D + 1 + 1 + 1 + D + D + D + 1;
    __shared__ Q2Smem<D, double, false> sm[EPB];
    __shared__ double sxb[EPB][NN][NXB];
    const int le = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int64_t e = (int64_t)blockIdx.x * EPB + le;
    const bool valid = e < m.E && t < NN;
    Q2Smem<D, double, false>& S = sm[le];
    const double inv_h = 1.0 / h;
    const double detJ = D == 2 ? 0.25 * h * h : 0.125 * h * h * h;
    int node = 0;
    bool inside = false;
    if (valid) {
        node = m.e2n[e * NN + t];
        double o[NF], n[NF];
        for (int f = 0; f < NF; ++f) {
            o[f] = Uo[(size_t)node * NF + f];
            n[f] = Un[(size_t)node * NF + f];
            S.ut[t][f] = 0.5 * (o[f] + n[f]);
        }
        for (int i = 0; i < D; ++i) S.dd[t][i] = n[i] - o[i];
        S.dd[t][D] = n[D + 1] - o[D + 1];
        const double avg = 0.5 * (o[D + 1] + n[D + 1]);
        inside = avg <= 1.0 && avg >= -1.0;
        S.ps[t] = clip1q(avg);
        // seeds: Dirichlet rows are replaced rows, their element contributions are discarded
        const unsigned fl = m.nflag[node];
        for (int f = 0; f < NF; ++f) {
            double wv = w[(size_t)node * NF + f];
            if (f < D && ((fl >> f) & 1u)) wv = 0.0;
            S.x[t][f] = wv;     // the seed rows reuse the tangent slots
        }
    }
    __syncwarp();
    double cnb = 0.0;
    if (valid) {
        const int q = t;
        const double g = 4.0 * inv_h * inv_h;
        const double wq = detJ * qweight<D, double>(q);
        QPIn<D, double> X;
        q2_interp<D, double, double, false>(S, q, inv_h, inv_dt, X, false);
        QPOut<D, double> Fb;
        for (int f = 0; f < NF; ++f) {
            Fb.f0[f] = 0.0;
            for (int k = 0; k < D; ++k) Fb.f1[f][k] = 0.0;
        }
        for (int a = 0; a < NN; ++a) {
            const QB<D, double> b = qbasis<D, double>(a, q, inv_h);
            for (int f = 0; f < NF; ++f) {
                const double wv = wq * S.x[a][f];
                Fb.f0[f] += b.N * wv;
                for (int k = 0; k < D; ++k) Fb.f1[f][k] += b.dN[k] * wv;
            }
        }
        QPIn<D, double> Xb;
        pointwise_adjoint<D, true>(X, c, Cn, g, Fb, Xb, cnb);
        double* o = sxb[le][q];
        int k = 0;
        for (int i = 0; i < D; ++i) o[k++] = Xb.v[i];
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) o[k++] = Xb.gv[i][j];
        o[k++] = Xb.p;
        for (int i = 0; i < D; ++i) o[k++] = Xb.gp[i];
        o[k++] = Xb.phi;
        for (int i = 0; i < D; ++i) o[k++] = Xb.gphi[i];
        for (int i = 0; i < NH; ++i) o[k++] = Xb.H[i];
        o[k++] = Xb.mu;
        for (int i = 0; i < D; ++i) o[k++] = Xb.gmu[i];
        for (int i = 0; i < D; ++i) o[k++] = Xb.vdt[i];
        o[k++] = Xb.phidt;
        o[k++] = Xb.divnew;
        o[k++] = Xb.ps;
        for (int i = 0; i < D; ++i) o[k++] = Xb.gps[i];
        for (int i = 0; i < D; ++i) o[k++] = Xb.Hd[i];
        for (int i = 0; i < D; ++i) o[k++] = Xb.lapv[i];
        o[k++] = Xb.lapmu;
    }
    __syncwarp();
    if (valid) {
        const int a = t;
        double ut[NF], ddv[D + 1], divb[D], psb = 0.0;
        for (int f = 0; f < NF; ++f) ut[f] = 0.0;
        for (int i = 0; i <= D; ++i) ddv[i] = 0.0;
        for (int i = 0; i < D; ++i) divb[i] = 0.0;
        for (int q = 0; q < NN; ++q) {
            const QB<D, double> b = qbasis<D, double>(a, q, inv_h);
            double lapN = b.hd[0];
            for (int kk = 1; kk < D; ++kk) lapN += b.hd[kk];
            const double* x = sxb[le][q];
            int k = 0;
            for (int i = 0; i < D; ++i) ut[i] += b.N * x[k++];
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) ut[i] += b.dN[j] * x[k++];
            ut[D] += b.N * x[k++];
            for (int i = 0; i < D; ++i) ut[D] += b.dN[i] * x[k++];
            ut[D + 1] += b.N * x[k++];
            for (int i = 0; i < D; ++i) ut[D + 1] += b.dN[i] * x[k++];
            for (int i = 0; i < NH; ++i) ut[D + 1] += b.hm[i] * x[k++];
            ut[D + 2] += b.N * x[k++];
            for (int i = 0; i < D; ++i) ut[D + 2] += b.dN[i] * x[k++];
            for (int i = 0; i < D; ++i) ddv[i] += b.N * x[k++];
            ddv[D] += b.N * x[k++];
            const double dvb = x[k++];
            for (int i = 0; i < D; ++i) divb[i] += b.dN[i] * dvb;
            psb += b.N * x[k++];
            for (int i = 0; i < D; ++i) psb += b.dN[i] * x[k++];
            for (int i = 0; i < D; ++i) ut[D + 1] += b.hd[i] * x[k++];
            for (int i = 0; i < D; ++i) ut[i] += lapN * x[k++];
            ut[D + 2] += lapN * x[k++];
        }
        double rn[NF], ro[NF];
        for (int f = 0; f < NF; ++f) rn[f] = ro[f] = 0.5 * ut[f];
        for (int i = 0; i < D; ++i) {
            rn[i] += inv_dt * ddv[i] + divb[i];
            ro[i] -= inv_dt * ddv[i];
        }
        rn[D + 1] += inv_dt * ddv[D];
        ro[D + 1] -= inv_dt * ddv[D];
        const double pst = inside ? 0.5 * psb : 0.0;
        for (int f = 0; f < NF; ++f) {
            const double extra = (f == D + 1) ? pst : 0.0;
            atomicAdd(gn + (size_t)node * NF + f, rn[f] + extra);
            if (go) atomicAdd(go + (size_t)node * NF + f, ro[f] + extra);
        }
    }
    if (gCn) {
        for (int off = 16; off > 0; off >>= 1) cnb += __shfl_xor_sync(0xffffffffu, cnb, off);
        if ((threadIdx.x & 31) == 0 && cnb != 0.0) atomicAdd(gCn, cnb);
    }
}

// Dirichlet velocity rows (as the Q1 path): residual v - g, J x identity, J^T w pass-through
template <int D, class T>
__global__ void q2_bc_kernel(DevMesh m, const T* __restrict__ a, T* __restrict__ out, bool residual) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.NB) return;
    const int64_t n = m.bnodes[i];
    const unsigned fl = m.nflag[n];
    for (int k = 0; k < D; ++k)
        if ((fl >> k) & 1u) {
            T v = a[n * (D + 3) + k];
            if (residual && m.bcval) v -= (T)m.bcval[n * D + k];
            out[n * (D + 3) + k] = v;
        }
}
template <int D>
__global__ void q2_bc_vjp_kernel(DevMesh m, const double* __restrict__ w, double* __restrict__ gn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.NB) return;
    const int64_t n = m.bnodes[i];
    const unsigned fl = m.nflag[n];
    for (int k = 0; k < D; ++k)
        if ((fl >> k) & 1u) gn[n * (D + 3) + k] += w[n * (D + 3) + k];
}

template <int D, class T, int MODE>
cudaError_t q2_launch_rj(const chns_mesh* mm, const PhysConst& pc, const T* Uo, const T* Un, const T* x, T* out,
                         cudaStream_t s) {
    const DevMesh& m = mm->dm;
    cudaError_t err = cudaMemsetAsync(out, 0, (size_t)m.N * (D + 3) * sizeof(T), s);
    if (err != cudaSuccess) return err;
    const T h = T(ldexp(m.hi - m.lo, -(int)mm->q2_level));
    const int EPB = Q2S<D>::EPB;
    q2_rj_kernel<D, T, MODE><<<(unsigned)((m.E + EPB - 1) / EPB), 128, 0, s>>>(m, q2_pcst<T>(pc), T(pc.inv_dt), h, Uo,
                                                                             Un, x, out, mm->d_flags);
    chns_count_launches(1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int64_t nb = m.NB > 0 ? m.NB : 1;
    q2_bc_kernel<D, T><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, MODE == Q2_RES ? Un : x, out, MODE == Q2_RES);
    chns_count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t q2_launch_residual(const chns_mesh* m, const PhysConst& pc, const double* Uo, const double* Un, double* R,
                               cudaStream_t s) {
    return m->dm.dim == 2 ? q2_launch_rj<2, double, Q2_RES>(m, pc, Uo, Un, nullptr, R, s)
                          : q2_launch_rj<3, double, Q2_RES>(m, pc, Uo, Un, nullptr, R, s);
}
cudaError_t q2_launch_jvp64(const chns_mesh* m, const PhysConst& pc, const double* Uo, const double* Un,
                            const double* x, double* y, cudaStream_t s) {
    return m->dm.dim == 2 ? q2_launch_rj<2, double, Q2_JVP>(m, pc, Uo, Un, x, y, s)
                          : q2_launch_rj<3, double, Q2_JVP>(m, pc, Uo, Un, x, y, s);
}
cudaError_t q2_launch_jvp32(const chns_mesh* m, const PhysConst& pc, const float* Uo, const float* Un, const float* x,
                            float* y, cudaStream_t s) {
    return m->dm.dim == 2 ? q2_launch_rj<2, float, Q2_JVP>(m, pc, Uo, Un, x, y, s)
                          : q2_launch_rj<3, float, Q2_JVP>(m, pc, Uo, Un, x, y, s);
}
cudaError_t q2_launch_vjp(const chns_mesh* mm, const PhysConst& pc, const double* Uo, const double* Un,
                          const double* w, double* gn, double* go, double* gCn, cudaStream_t s) {
    const DevMesh& m = mm->dm;
    const size_t bytes = (size_t)m.N * m.nf * sizeof(double);
    cudaError_t err = cudaMemsetAsync(gn, 0, bytes, s);
    if (err == cudaSuccess && go) err = cudaMemsetAsync(go, 0, bytes, s);
    if (err == cudaSuccess && gCn) err = cudaMemsetAsync(gCn, 0, sizeof(double), s);
    if (err != cudaSuccess) return err;
    const double h = ldexp(m.hi - m.lo, -(int)mm->q2_level);
    const int64_t nb = m.NB > 0 ? m.NB : 1;
    if (m.dim == 2) {
        q2_vjp_kernel<2><<<(unsigned)((m.E + 7) / 8), 128, 0, s>>>(
            m, q2_pcst<double>(pc), pc.Cn, pc.inv_dt, h, Uo, Un, w, gn, go, gCn);
        chns_count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        q2_bc_vjp_kernel<2><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, w, gn);
    } else {
        q2_vjp_kernel<3><<<(unsigned)((m.E + 1) / 2), 64, 0, s>>>(
            m, q2_pcst<double>(pc), pc.Cn, pc.inv_dt, h, Uo, Un, w, gn, go, gCn);
        chns_count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        q2_bc_vjp_kernel<3><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, w, gn);
    }
    chns_count_launches(1);
    return cudaGetLastError();
}
