// Pointwise Crank-Nicolson VMS physics at one quadrature point, its forward-mode
// tangent (through the Dual number type) and its hand-written reverse mode.
//
// Inputs at a Gauss point (all mid-point averages of Eq. averaging1 unless noted):
//   v, grad v (gv[i][j] = d_j v_i), p, grad p, phi, grad phi, the mixed second
//   derivatives of phi (the pure ones vanish on Q1), mu, grad mu,
//   vdt = (v^{k+1} - v^k)/dt, phidt = (phi^{k+1} - phi^k)/dt, divnew = div v^{k+1},
//   ps = phi* (the pull-back of the Remark on saturation, as a Q1 field) and grad phi*.
// Outputs: f0[f] multiplies the test value N_a, f1[f][k] multiplies d_k N_a, for the
// rows f = momentum_1..d, solenoidality, Cahn-Hilliard, potential (Definition 2).
#pragma once

#include <cuda_runtime.h>

template <class T>
struct Dual {
    T v, d;
    __host__ __device__ Dual() {}
    __host__ __device__ Dual(T a) : v(a), d(T(0)) {}
    __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
};

template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return {a + b.v, b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
    T q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <class T> __device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
    T q = a / b.v;
    return {q, -q * b.d / b.v};
}

// x^(-1/2) with its derivative -1/2 x^(-3/2) (CUDA's rsqrt: at most a few ulp off, far
// below the FP64 (1e-12) and FP32 (1e-5) parity bars)
__device__ __forceinline__ double inv_sqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
// 1/x with its derivative -x^(-2)
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }
template <class T> __device__ __forceinline__ Dual<T> recip(Dual<T> x) {
    T r = recip(x.v);
    return {r, -r * r * x.d};
}
template <class T> __device__ __forceinline__ Dual<T> inv_sqrt(Dual<T> x) {
    T r = inv_sqrt(x.v);
    return {r, T(-0.5) * r * r * r * x.d};
}
__device__ __forceinline__ double value_of(double x) { return x; }
__device__ __forceinline__ float value_of(float x) { return x; }
template <class T> __device__ __forceinline__ T value_of(Dual<T> x) { return x.v; }

// Index of the mixed second derivative (i != j) in the packed array
// (2D: xy; 3D: xy, xz, yz).
__device__ __forceinline__ constexpr int hidx(int i, int j) {
    return (i < j) ? (i == 0 ? j - 1 : 2) : (j == 0 ? i - 1 : 2);
}

template <int D, class S>
struct QPIn {
    S v[D], gv[D][D], p, gp[D], phi, gphi[D], H[D == 2 ? 1 : 3], mu, gmu[D], vdt[D], phidt, divnew,
        ps, gps[D];
    // second derivatives that vanish on Q1 and are read only by the Q2 instantiation:
    // pure second derivatives of phi, Laplacians of the velocity components and of mu
    S Hd[D], lapv[D], lapmu;
};

template <int D, class S>
struct QPOut {
    S f0[D + 3];
    S f1[D + 3][D];
};

// Constants of one time step in the working precision R.
template <class R>
struct PCst {
    R alpha, beta, gamma, xi;      // rho(phi) = alpha phi + beta, eta(phi) = gamma phi + xi
    R Jc;                          // (rho_- - rho_+)/(2 rho_+ Cn): J = Jc grad mu
    R inv_Pe, inv_We, inv_Re, inv_Fr, Cn_We, inv_PeCn, Cn2, Pe, Re;
    R four_over_dt2, C_I, C_phi;
};

// The pointwise map of Definition 2 (Crank-Nicolson substitution, Section 3.3 end).
// g = 4/h^2: the metric G = g I of the axis-aligned element (tr G = D g, G:G = D g^2).
// Q2: the strong residuals also carry the terms with pure second derivatives (they vanish
// on Q1): d_i phi d_ii phi + d_i phi lap phi in the capillary term, eta lap v_i in the
// viscous term, lap mu in R_phi.
template <int D, class S, class R, bool Q2 = false>
__device__ __forceinline__ void pointwise(const QPIn<D, S>& X, const PCst<R>& c, R g,
                                          QPOut<D, S>& F) {
    const S rho = c.alpha * X.ps + c.beta;
    const S eta = c.gamma * X.ps + c.xi;
    S J[D], conv[D], Jgv[D], Rm[D];
    S vv = X.v[0] * X.v[0], vJ;
#pragma unroll
    for (int k = 0; k < D; ++k) J[k] = c.Jc * X.gmu[k];
    vJ = X.v[0] * J[0];
#pragma unroll
    for (int k = 1; k < D; ++k) {
        vv = vv + X.v[k] * X.v[k];
        vJ = vJ + X.v[k] * J[k];
    }
    S Rc = X.gv[0][0];
#pragma unroll
    for (int k = 1; k < D; ++k) Rc = Rc + X.gv[k][k];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        S cv = X.v[0] * X.gv[i][0];
        S jg = J[0] * X.gv[i][0];
        S vs = (c.gamma * X.gps[0]) * X.gv[i][0];
#pragma unroll
        for (int j = 1; j < D; ++j) {
            cv = cv + X.v[j] * X.gv[i][j];
            jg = jg + J[j] * X.gv[i][j];
            vs = vs + (c.gamma * X.gps[j]) * X.gv[i][j];
        }
        S cap = S(R(0));
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (j != i) cap = cap + X.H[hidx(i, j)] * X.gphi[j];
        if constexpr (Q2) {
            S lapphi = X.Hd[0];
#pragma unroll
            for (int k = 1; k < D; ++k) lapphi = lapphi + X.Hd[k];
            cap = cap + X.gphi[i] * (X.Hd[i] + lapphi);
            vs = vs + eta * X.lapv[i];
        }
        conv[i] = cv;
        Jgv[i] = jg;
        S r = rho * (X.vdt[i] + cv) + c.inv_Pe * jg + c.Cn_We * cap + c.inv_We * X.gp[i] - c.inv_Re * vs;
        if (i == D - 1) r = r + c.inv_Fr * rho;
        Rm[i] = r;
    }
    S vg = X.v[0] * X.gphi[0];
#pragma unroll
    for (int k = 1; k < D; ++k) vg = vg + X.v[k] * X.gphi[k];
    S Rphi = X.phidt + X.phi * Rc + vg;
    if constexpr (Q2) Rphi = Rphi - c.inv_PeCn * X.lapmu;
    const S irho = recip(rho);
    const S er = c.inv_Re * (eta * irho);
    const S rad_m = c.four_over_dt2 + g * vv + (g * c.inv_Pe) * (vJ * irho) + (c.C_I * R(D) * g * g) * (er * er);
    const S tm = inv_sqrt(rad_m);
    // tau_c = 1/(tr G tau_m) = tau_m rad_m / (D g)
    const S tc = (tm * rad_m) * (R(1) / (R(D) * g));
    const S tp = inv_sqrt(c.four_over_dt2 + g * vv + (c.C_phi * R(D) * g * g) * (c.inv_PeCn * c.inv_PeCn));
    const S tm_rho = tm * irho;
    // momentum rows
    S a[D];
#pragma unroll
    for (int j = 0; j < D; ++j) a[j] = tm * X.v[j] - (tm * tm_rho) * Rm[j] + c.inv_Pe * tm_rho * J[j];
    const S diag = c.inv_We * (rho * tc * Rc - X.p);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        S rg = Rm[0] * X.gv[i][0];
#pragma unroll
        for (int j = 1; j < D; ++j) rg = rg + Rm[j] * X.gv[i][j];
        S f = rho * (X.vdt[i] + conv[i]) - tm * rg + c.inv_Pe * Jgv[i];
        if (i == D - 1) f = f + c.inv_Fr * rho;
        F.f0[i] = f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            S t = Rm[i] * a[j] - c.Cn_We * (X.gphi[i] * X.gphi[j]) + c.inv_Re * (eta * X.gv[i][j]);
            if (i == j) t = t + diag;
            F.f1[i][j] = t;
        }
    }
    // solenoidality
    F.f0[D] = X.divnew;
#pragma unroll
    for (int i = 0; i < D; ++i) F.f1[D][i] = tm_rho * Rm[i];
    // Cahn-Hilliard
    F.f0[D + 1] = X.phidt;
    const S tpR = tp * Rphi;
    const S tmphi = tm_rho * X.phi;
#pragma unroll
    for (int i = 0; i < D; ++i)
        F.f1[D + 1][i] = X.v[i] * (tpR - X.phi) + tmphi * Rm[i] + c.inv_PeCn * X.gmu[i];
    // potential
    F.f0[D + 2] = (X.phi * X.phi - R(1)) * X.phi - X.mu;
#pragma unroll
    for (int i = 0; i < D; ++i) F.f1[D + 2][i] = c.Cn2 * X.gphi[i];
}

// Reverse mode of `pointwise` in FP64: given the output adjoint Fb, return the input
// adjoint Xb and the adjoint of Cn (Cn enters through Jc, Cn/We, 1/(Pe Cn), Cn^2).
template <int D, bool Q2 = false>
__device__ __forceinline__ void pointwise_adjoint(const QPIn<D, double>& X, const PCst<double>& c,
                                                  double Cn, double g, const QPOut<D, double>& Fb,
                                                  QPIn<D, double>& Xb, double& Cnb) {
    // ---- forward sweep (intermediates kept) ----
    const double rho = c.alpha * X.ps + c.beta;
    const double eta = c.gamma * X.ps + c.xi;
    double J[D], conv[D], Jgv[D], Rm[D], cap[D], visc[D];
    double vv = 0.0, vJ = 0.0, Rc = 0.0, vg = 0.0, lapphi = 0.0;
    if (Q2)
        for (int k = 0; k < D; ++k) lapphi += X.Hd[k];
    for (int k = 0; k < D; ++k) {
        J[k] = c.Jc * X.gmu[k];
        vv += X.v[k] * X.v[k];
        vJ += X.v[k] * J[k];
        Rc += X.gv[k][k];
        vg += X.v[k] * X.gphi[k];
    }
    for (int i = 0; i < D; ++i) {
        double cv = 0, jg = 0, vs = 0, cp = 0;
        for (int j = 0; j < D; ++j) {
            cv += X.v[j] * X.gv[i][j];
            jg += J[j] * X.gv[i][j];
            vs += c.gamma * X.gps[j] * X.gv[i][j];
            if (j != i) cp += X.H[hidx(i, j)] * X.gphi[j];
        }
        if (Q2) {
            cp += X.gphi[i] * (X.Hd[i] + lapphi);
            vs += eta * X.lapv[i];
        }
        conv[i] = cv;
        Jgv[i] = jg;
        visc[i] = vs;
        cap[i] = cp;
        Rm[i] = rho * (X.vdt[i] + cv) + c.inv_Pe * jg + c.Cn_We * cp + c.inv_We * X.gp[i] - c.inv_Re * vs +
                (i == D - 1 ? c.inv_Fr * rho : 0.0);
    }
    const double Rphi = X.phidt + X.phi * Rc + vg - (Q2 ? c.inv_PeCn * X.lapmu : 0.0);
    const double irho = 1.0 / rho, irho2 = irho * irho;
    const double er = c.inv_Re * eta * irho;
    const double GG = double(D) * g * g;
    const double rad_m = c.four_over_dt2 + g * vv + (g * c.inv_Pe) * (vJ * irho) + c.C_I * GG * er * er;
    const double tm = rsqrt(rad_m);
    const double tc = tm * rad_m * (1.0 / (double(D) * g));
    const double rad_p = c.four_over_dt2 + g * vv + c.C_phi * GG * c.inv_PeCn * c.inv_PeCn;
    const double tp = rsqrt(rad_p);
    const double tm_rho = tm * irho;
    double a[D];
    for (int j = 0; j < D; ++j) a[j] = tm * X.v[j] - (tm * tm_rho) * Rm[j] + c.inv_Pe * tm_rho * J[j];

    // ---- reverse sweep ----
    double rhob = 0, etab = 0, tmb = 0, tcb = 0, tpb = 0, Rcb = 0, Rphib = 0, vvb = 0, vJb = 0;
    double Jb[D], Rmb[D], convb[D], Jgvb[D], capb[D], viscb[D], ab[D];
    for (int k = 0; k < D; ++k) {
        Jb[k] = Rmb[k] = convb[k] = Jgvb[k] = capb[k] = viscb[k] = ab[k] = 0.0;
        Xb.v[k] = Xb.gp[k] = Xb.gphi[k] = Xb.gmu[k] = Xb.vdt[k] = Xb.gps[k] = 0.0;
        for (int j = 0; j < D; ++j) Xb.gv[k][j] = 0.0;
    }
    for (int k = 0; k < (D == 2 ? 1 : 3); ++k) Xb.H[k] = 0.0;
    for (int k = 0; k < D; ++k) Xb.Hd[k] = Xb.lapv[k] = 0.0;
    Xb.p = Xb.phi = Xb.mu = Xb.phidt = Xb.divnew = Xb.ps = Xb.lapmu = 0.0;
    Cnb = 0.0;
    const double iCn = 1.0 / Cn;
    const double dJc = -c.Jc * iCn, dinvPeCn = -c.inv_PeCn * iCn, dCnWe = c.inv_We, dCn2 = 2.0 * Cn;

    // potential: f0 = phi^3 - phi - mu, f1_i = Cn^2 gphi_i
    Xb.mu -= Fb.f0[D + 2];
    Xb.phi += (3.0 * X.phi * X.phi - 1.0) * Fb.f0[D + 2];
    for (int i = 0; i < D; ++i) {
        Xb.gphi[i] += c.Cn2 * Fb.f1[D + 2][i];
        Cnb += dCn2 * X.gphi[i] * Fb.f1[D + 2][i];
    }
    // Cahn-Hilliard: f0 = phidt; f1_i = v_i (tp Rphi - phi) + (tm/rho) phi Rm_i + inv_PeCn gmu_i
    Xb.phidt += Fb.f0[D + 1];
    for (int i = 0; i < D; ++i) {
        const double fb = Fb.f1[D + 1][i];
        Xb.v[i] += (tp * Rphi - X.phi) * fb;
        tpb += X.v[i] * Rphi * fb;
        Rphib += X.v[i] * tp * fb;
        Xb.phi += (-X.v[i] + tm_rho * Rm[i]) * fb;
        tmb += (X.phi * irho) * Rm[i] * fb;
        rhob -= (tm * X.phi * irho2) * Rm[i] * fb;
        Rmb[i] += tm_rho * X.phi * fb;
        Xb.gmu[i] += c.inv_PeCn * fb;
        Cnb += dinvPeCn * X.gmu[i] * fb;
    }
    // solenoidality: f0 = divnew; f1_i = (tm/rho) Rm_i
    Xb.divnew += Fb.f0[D];
    for (int i = 0; i < D; ++i) {
        const double fb = Fb.f1[D][i];
        tmb += Rm[i] * irho * fb;
        rhob -= tm * Rm[i] * irho2 * fb;
        Rmb[i] += tm_rho * fb;
    }
    // momentum gradient part: f1_ij = Rm_i a_j - Cn_We gphi_i gphi_j + d_ij inv_We (rho tc Rc - p)
    //                                 + inv_Re eta gv_ij
    double trace = 0.0;
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) {
            const double fb = Fb.f1[i][j];
            Rmb[i] += a[j] * fb;
            ab[j] += Rm[i] * fb;
            Xb.gphi[i] -= c.Cn_We * X.gphi[j] * fb;
            Xb.gphi[j] -= c.Cn_We * X.gphi[i] * fb;
            Cnb -= dCnWe * X.gphi[i] * X.gphi[j] * fb;
            etab += c.inv_Re * X.gv[i][j] * fb;
            Xb.gv[i][j] += c.inv_Re * eta * fb;
        }
        trace += Fb.f1[i][i];
    }
    rhob += c.inv_We * tc * Rc * trace;
    tcb += c.inv_We * rho * Rc * trace;
    Rcb += c.inv_We * rho * tc * trace;
    Xb.p -= c.inv_We * trace;
    // a_j = tm v_j - (tm^2/rho) Rm_j + inv_Pe (tm/rho) J_j
    for (int j = 0; j < D; ++j) {
        tmb += ab[j] * (X.v[j] - 2.0 * tm_rho * Rm[j] + c.inv_Pe * J[j] * irho);
        Xb.v[j] += tm * ab[j];
        rhob += ab[j] * (tm * tm * Rm[j] - c.inv_Pe * tm * J[j]) * irho2;
        Rmb[j] -= (tm * tm_rho) * ab[j];
        Jb[j] += c.inv_Pe * tm_rho * ab[j];
    }
    // momentum value part: f0_i = rho (vdt_i + conv_i) - tm sum_j Rm_j gv_ij + inv_Pe Jgv_i
    //                             + [i == D-1] inv_Fr rho
    for (int i = 0; i < D; ++i) {
        const double fb = Fb.f0[i];
        rhob += (X.vdt[i] + conv[i]) * fb + (i == D - 1 ? c.inv_Fr * fb : 0.0);
        Xb.vdt[i] += rho * fb;
        convb[i] += rho * fb;
        Jgvb[i] += c.inv_Pe * fb;
        for (int j = 0; j < D; ++j) {
            tmb -= fb * Rm[j] * X.gv[i][j];
            Rmb[j] -= tm * fb * X.gv[i][j];
            Xb.gv[i][j] -= tm * fb * Rm[j];
        }
    }
    // tau_phi, tau_c, tau_m
    {
        const double radpb = -0.5 * tp * tp * tp * tpb;
        vvb += g * radpb;
        Cnb += radpb * c.C_phi * GG * 2.0 * c.inv_PeCn * dinvPeCn;
    }
    tmb -= tcb * tc * tm * rad_m;   // d(1/(D g tm))/dtm = -tc/tm, and 1/tm = tm rad_m
    {
        const double radmb = -0.5 * tm * tm * tm * tmb;
        vvb += g * radmb;
        vJb += (g * c.inv_Pe) * irho * radmb;
        rhob -= (g * c.inv_Pe) * vJ * irho2 * radmb;
        // C_I GG (eta/(rho Re))^2
        etab += 2.0 * c.C_I * GG * er * irho * c.inv_Re * radmb;
        rhob -= 2.0 * c.C_I * GG * er * er * irho * radmb;
    }
    // Rphi = phidt + phi Rc + v . gphi (- inv_PeCn lap mu on Q2)
    if (Q2) {
        Xb.lapmu -= c.inv_PeCn * Rphib;
        Cnb -= dinvPeCn * X.lapmu * Rphib;
    }
    Xb.phidt += Rphib;
    Xb.phi += Rc * Rphib;
    Rcb += X.phi * Rphib;
    for (int k = 0; k < D; ++k) {
        Xb.v[k] += X.gphi[k] * Rphib;
        Xb.gphi[k] += X.v[k] * Rphib;
    }
    // Rm_i = rho (vdt_i + conv_i) + inv_Pe Jgv_i + Cn_We cap_i + inv_We gp_i - inv_Re visc_i
    //        + [i == D-1] inv_Fr rho
    for (int i = 0; i < D; ++i) {
        const double rb = Rmb[i];
        rhob += (X.vdt[i] + conv[i]) * rb + (i == D - 1 ? c.inv_Fr * rb : 0.0);
        Xb.vdt[i] += rho * rb;
        convb[i] += rho * rb;
        Jgvb[i] += c.inv_Pe * rb;
        capb[i] += c.Cn_We * rb;
        Cnb += dCnWe * cap[i] * rb;
        Xb.gp[i] += c.inv_We * rb;
        viscb[i] -= c.inv_Re * rb;
    }
    // Rc = tr grad v
    for (int k = 0; k < D; ++k) Xb.gv[k][k] += Rcb;
    // visc_i = sum_k gamma gps_k gv_ik (+ eta lap v_i); cap_i = sum_{j != i} H_ij gphi_j
    // (+ gphi_i (Hd_i + lap phi)); Jgv_i = sum_j J_j gv_ij; conv_i = sum_j v_j gv_ij
    if (Q2) {
        double lapb = 0.0;
        for (int i = 0; i < D; ++i) {
            etab += X.lapv[i] * viscb[i];
            Xb.lapv[i] += eta * viscb[i];
            Xb.gphi[i] += (X.Hd[i] + lapphi) * capb[i];
            Xb.Hd[i] += X.gphi[i] * capb[i];
            lapb += X.gphi[i] * capb[i];
        }
        for (int k = 0; k < D; ++k) Xb.Hd[k] += lapb;
    }
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) {
            Xb.gps[j] += c.gamma * X.gv[i][j] * viscb[i];
            Xb.gv[i][j] += c.gamma * X.gps[j] * viscb[i] + J[j] * Jgvb[i] + X.v[j] * convb[i];
            Jb[j] += X.gv[i][j] * Jgvb[i];
            Xb.v[j] += X.gv[i][j] * convb[i];
            if (j != i) {
                Xb.H[hidx(i, j)] += X.gphi[j] * capb[i];
                Xb.gphi[j] += X.H[hidx(i, j)] * capb[i];
            }
        }
    }
    // vJ, vv
    for (int k = 0; k < D; ++k) {
        Xb.v[k] += J[k] * vJb + 2.0 * X.v[k] * vvb;
        Jb[k] += X.v[k] * vJb;
    }
    // J_k = Jc gmu_k
    for (int k = 0; k < D; ++k) {
        Xb.gmu[k] += c.Jc * Jb[k];
        Cnb += dJc * X.gmu[k] * Jb[k];
    }
    // eta = gamma ps + xi; rho = alpha ps + beta
    Xb.ps += c.gamma * etab + c.alpha * rhob;
}
