// Element kernels of the matrix-free hot path: residual (FP64), J x (FP64 / FP32,
// forward mode through Dual numbers) and J^T w (FP64, reverse mode).
//
// Thread mapping: 2^d threads per element; during the gather thread t owns element
// corner t, during the physics it owns Gauss point t, during the test contraction
// it owns corner t again.  An element's threads sit in one warp, so the exchanges go
// through shared memory with __syncwarp.  Elements are processed in their Morton
// order (consecutive elements share most nodes, which keeps gathers in L2/L1).
//
// Hanging corners (Section 4): a corner value is the mean of its 2 (edge) or 4 (face)
// parent nodes; the scatter applies the transpose (the same weights).
#include <cuda_runtime.h>

#include <type_traits>

#include "chns_internal.h"
#include "pointwise.cuh"

namespace {

template <int D>
struct Shape {
    static constexpr int NC = 1 << D;      // corners = Gauss points
    static constexpr int NF = D + 3;       // fields
    static constexpr int NH = (D == 2) ? 1 : 3;
    static constexpr int EPB = (D == 2) ? 32 : 16;  // elements per 128-thread block
};

template <class T> struct GaussC;
template <> struct GaussC<double> {
    static constexpr double cp = 0.78867513459481288225;  // (1 + 1/sqrt 3)/2
    static constexpr double cm = 0.21132486540518711775;  // (1 - 1/sqrt 3)/2
};
template <> struct GaussC<float> {
    static constexpr float cp = 0.78867513459481288225f;
    static constexpr float cm = 0.21132486540518711775f;
};

// Q1 basis of corner a at Gauss point q (both as bit patterns), physical derivatives.
template <int D, class T>
struct Basis {
    T N, dN[D], d2N[Shape<D>::NH];
};

template <int D, class T>
__device__ __forceinline__ Basis<D, T> basis(int a, int q, T inv_h) {
    T f[D], s[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const bool same = ((a >> k) & 1) == ((q >> k) & 1);
        f[k] = same ? GaussC<T>::cp : GaussC<T>::cm;
        s[k] = ((a >> k) & 1) ? inv_h : -inv_h;
    }
    Basis<D, T> b;
    if constexpr (D == 2) {
        b.N = f[0] * f[1];
        b.dN[0] = s[0] * f[1];
        b.dN[1] = f[0] * s[1];
        b.d2N[0] = s[0] * s[1];
    } else {
        b.N = f[0] * f[1] * f[D - 1];
        b.dN[0] = s[0] * f[1] * f[D - 1];
        b.dN[1] = f[0] * s[1] * f[D - 1];
        b.dN[D - 1] = f[0] * f[1] * s[D - 1];
        b.d2N[0] = s[0] * s[1] * f[D - 1];
        b.d2N[1 % Shape<D>::NH] = s[0] * f[1] * s[D - 1];
        b.d2N[2 % Shape<D>::NH] = f[0] * s[1] * s[D - 1];
    }
    return b;
}

template <class T>
__device__ __forceinline__ T clip1(T x) { return x > T(1) ? T(1) : (x < T(-1) ? T(-1) : x); }

// Shared-memory vector loads of the 3D corner / flux rows (fewer load instructions; the
// rows are laid out so every pair starts on an 8-byte (FP32) or 16-byte (FP64) boundary)
template <class T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };
template <class T>
__device__ __forceinline__ typename Pair<T>::type ld_pair(const T* p) {
    return *reinterpret_cast<const typename Pair<T>::type*>(p);
}

// A node row of NF values from global memory (read-only path).  In 3D a row is 24 B
// (FP32) or 48 B (FP64) at node * row, so it is read as three 8- or 16-byte pairs.
template <int D, class T>
__device__ __forceinline__ void ld_row(const T* __restrict__ p, T v[Shape<D>::NF]) {
    if constexpr (D == 3) {
        const typename Pair<T>::type* q = reinterpret_cast<const typename Pair<T>::type*>(p);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const typename Pair<T>::type t = __ldg(q + i);
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int f = 0; f < Shape<D>::NF; ++f) v[f] = __ldg(p + f);
    }
}

// element size (hi - lo) 2^-level, exact in the working precision (no FP64 work in
// the FP32 kernels: GB300's FP64 pipe is 1/64 of its FP32 rate)
__device__ __forceinline__ float scale_pow2(float span, int lev) { return ldexpf(span, -lev); }
__device__ __forceinline__ double scale_pow2(double span, int lev) { return ldexp(span, -lev); }

// Corner parents and weights of element corner entry `ent`.
struct Parents {
    int n;
    int p[4];
};

__device__ __forceinline__ Parents parents_of(const DevMesh& m, int ent) {
    Parents P;
    if (ent >= 0) {
        P.n = 1;
        P.p[0] = ent;
        P.p[1] = P.p[2] = P.p[3] = 0;
    } else {
        const int4 hp = reinterpret_cast<const int4*>(m.hang)[-ent - 1];
        P.p[0] = hp.x;
        P.p[1] = hp.y;
        P.p[2] = hp.z < 0 ? 0 : hp.z;
        P.p[3] = hp.w < 0 ? 0 : hp.w;
        P.n = hp.z < 0 ? 2 : 4;
    }
    return P;
}

// Primal corner data of one element in shared memory.
template <int D, class T>
struct __align__(16) CornerPrimal {
    T ut[Shape<D>::NC][Shape<D>::NF];   // mid-point average
    T dd[Shape<D>::NC][D + 1];          // (new - old) for v and phi
    T ps[Shape<D>::NC];                 // phi* (clip at independent nodes, interpolated)
};

// Gather of corner `a`: averages, differences and phi*; returns the clip masks of the
// parents (bit j set: parent j has |phi~| <= 1) for the tangent / adjoint.
template <int D, class T>
__device__ __forceinline__ unsigned gather_primal(const DevMesh& m, const Parents& P, const T* __restrict__ Uo,
                                                  const T* __restrict__ Un, CornerPrimal<D, T>& C, int a) {
    constexpr int NF = Shape<D>::NF;
    T so[NF], sn[NF];
    T ps = T(0);
    unsigned mask = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) so[f] = sn[f] = T(0);
    const T w = (P.n == 1) ? T(1) : (P.n == 2 ? T(0.5) : T(0.25));
    for (int j = 0; j < P.n; ++j) {
        const T* po = Uo + (size_t)P.p[j] * NF;
        const T* pn = Un + (size_t)P.p[j] * NF;
        T o[NF], n[NF];
        ld_row<D, T>(po, o);
        ld_row<D, T>(pn, n);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            so[f] += w * o[f];
            sn[f] += w * n[f];
        }
        const T avg = T(0.5) * (o[D + 1] + n[D + 1]);
        if (avg <= T(1) && avg >= T(-1)) mask |= 1u << j;
        ps += w * clip1(avg);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) C.ut[a][f] = T(0.5) * (so[f] + sn[f]);
#pragma unroll
    for (int i = 0; i < D; ++i) C.dd[a][i] = sn[i] - so[i];
    C.dd[a][D] = sn[D + 1] - so[D + 1];
    C.ps[a] = ps;
    return mask;
}

// Sum-factorised Q1 interpolation at one Gauss point: the corner values are reduced one
// axis at a time, u0 + w (u1 - u0) along each axis (w: weight of the corner with the axis
// bit set, (1 +- 1/sqrt 3)/2; the two 1D weights sum to 1), and the differences
// u1 - u0 give the derivative along that axis (times 1/h).  Same values as summing
// N_a u_a over the corners, without forming the basis products.
template <class T>
__device__ __forceinline__ void gauss_weights(int q, T w[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = ((q >> k) & 1) ? GaussC<T>::cp : GaussC<T>::cm;
}

// value only
template <int D, class T, class Get>
__device__ __forceinline__ T sf_value(const T w[3], Get u) {
    if constexpr (D == 2) {
        const T a0 = u(0) + w[0] * (u(1) - u(0));
        const T a1 = u(2) + w[0] * (u(3) - u(2));
        return a0 + w[1] * (a1 - a0);
    } else {
        T A[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) A[i] = u(2 * i) + w[0] * (u(2 * i + 1) - u(2 * i));
        const T a0 = A[0] + w[1] * (A[1] - A[0]);
        const T a1 = A[2] + w[1] * (A[3] - A[2]);
        return a0 + w[2] * (a1 - a0);
    }
}

// value, physical gradient and (if WANT_H) the mixed second derivatives
template <int D, bool WANT_H, class T, class Get>
__device__ __forceinline__ void sf_vgrad(const T w[3], T inv_h, Get u, T& val, T g[D], T* hm) {
    if constexpr (D == 2) {
        const T b0 = u(1) - u(0), b1 = u(3) - u(2);
        const T a0 = u(0) + w[0] * b0, a1 = u(2) + w[0] * b1;
        const T dy = a1 - a0, dby = b1 - b0;
        val = a0 + w[1] * dy;
        g[0] = (b0 + w[1] * dby) * inv_h;
        g[1] = dy * inv_h;
        if (WANT_H) hm[0] = dby * inv_h * inv_h;
    } else {
        T A[4], B[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            B[i] = u(2 * i + 1) - u(2 * i);
            A[i] = u(2 * i) + w[0] * B[i];
        }
        T AA[2], AB[2], BA[2], BB[2];
#pragma unroll
        for (int z = 0; z < 2; ++z) {
            AB[z] = A[2 * z + 1] - A[2 * z];
            AA[z] = A[2 * z] + w[1] * AB[z];
            BB[z] = B[2 * z + 1] - B[2 * z];
            BA[z] = B[2 * z] + w[1] * BB[z];
        }
        const T dz = AA[1] - AA[0], dABz = AB[1] - AB[0], dBAz = BA[1] - BA[0];
        val = AA[0] + w[2] * dz;
        g[0] = (BA[0] + w[2] * dBAz) * inv_h;
        g[1] = (AB[0] + w[2] * dABz) * inv_h;
        g[2] = dz * inv_h;
        if (WANT_H) {
            const T h2 = inv_h * inv_h;
            hm[0] = (BB[0] + w[2] * (BB[1] - BB[0])) * h2;   // xy
            hm[1] = dBAz * h2;                                // xz
            hm[2] = dABz * h2;                                // yz
        }
    }
}

// Interpolate the primal quadrature-point inputs at Gauss point q.
template <int D, class T>
__device__ __forceinline__ void interp_primal(const CornerPrimal<D, T>& C, int q, T inv_h, T inv_dt,
                                              QPIn<D, T>& X) {
    T w[3];
    gauss_weights<T>(q, w);
    T g[D], val;
    if constexpr (D == 3) {
        // 3D rows hold 6 fields and 4 differences: read them two at a time
        typename Pair<T>::type c[Shape<D>::NC];
#pragma unroll
        for (int a = 0; a < Shape<D>::NC; ++a) c[a] = ld_pair(&C.ut[a][0]);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].x; }, X.v[0], X.gv[0], nullptr);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].y; }, X.v[1], X.gv[1], nullptr);
#pragma unroll
        for (int a = 0; a < Shape<D>::NC; ++a) c[a] = ld_pair(&C.ut[a][2]);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].x; }, X.v[2], X.gv[2], nullptr);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].y; }, X.p, X.gp, nullptr);
#pragma unroll
        for (int a = 0; a < Shape<D>::NC; ++a) c[a] = ld_pair(&C.ut[a][4]);
        sf_vgrad<D, true, T>(w, inv_h, [&](int a) { return c[a].x; }, X.phi, X.gphi, X.H);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].y; }, X.mu, X.gmu, nullptr);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return C.ps[a]; }, X.ps, X.gps, nullptr);
        T div = X.gv[0][0] + X.gv[1][1] + X.gv[2][2];
#pragma unroll
        for (int a = 0; a < Shape<D>::NC; ++a) c[a] = ld_pair(&C.dd[a][0]);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].x; }, val, g, nullptr);
        X.vdt[0] = val * inv_dt;
        div += T(0.5) * g[0];
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].y; }, val, g, nullptr);
        X.vdt[1] = val * inv_dt;
        div += T(0.5) * g[1];
#pragma unroll
        for (int a = 0; a < Shape<D>::NC; ++a) c[a] = ld_pair(&C.dd[a][2]);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].x; }, val, g, nullptr);
        X.vdt[2] = val * inv_dt;
        div += T(0.5) * g[2];
        X.divnew = div;
        X.phidt = sf_value<D, T>(w, [&](int a) { return c[a].y; }) * inv_dt;
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return C.ut[a][i]; }, val, g, nullptr);
            X.v[i] = val;
#pragma unroll
            for (int k = 0; k < D; ++k) X.gv[i][k] = g[k];
        }
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return C.ut[a][D]; }, X.p, X.gp, nullptr);
        sf_vgrad<D, true, T>(w, inv_h, [&](int a) { return C.ut[a][D + 1]; }, X.phi, X.gphi, X.H);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return C.ut[a][D + 2]; }, X.mu, X.gmu, nullptr);
        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return C.ps[a]; }, X.ps, X.gps, nullptr);
        // div v^{k+1} = div v~ + (1/2) div (v^{k+1} - v^k)
        T div = X.gv[0][0];
#pragma unroll
        for (int i = 1; i < D; ++i) div += X.gv[i][i];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return C.dd[a][i]; }, val, g, nullptr);
            X.vdt[i] = val * inv_dt;
            div += T(0.5) * g[i];
        }
        X.divnew = div;
        X.phidt = sf_value<D, T>(w, [&](int a) { return C.dd[a][D]; }) * inv_dt;
    }
}

template <class R>
__host__ __device__ PCst<R> make_pcst(const PhysConst& pc) {
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

// Test-function contraction for corner a from the per-Gauss-point fluxes in shared
// memory (already scaled by |det J| w_q): r[f] = sum_q N_a f0 + grad N_a . f1.
template <int D, class T>
__device__ __forceinline__ void contract(const T (*sf)[Shape<D>::NF * (D + 1)], int a, T inv_h,
                                         T r[Shape<D>::NF]) {
    constexpr int NF = Shape<D>::NF, NS = NF * (D + 1);
#pragma unroll
    for (int f = 0; f < NF; ++f) r[f] = T(0);
#pragma unroll
    for (int q = 0; q < Shape<D>::NC; ++q) {
        const Basis<D, T> b = basis<D, T>(a, q, inv_h);
        T s[NS];
        if constexpr (D == 3) {
            // the 24 fluxes of a Gauss point in 16-byte shared loads (rows are 16-byte aligned)
            if constexpr (sizeof(T) == 4) {
                const float4* v = reinterpret_cast<const float4*>(sf[q]);
#pragma unroll
                for (int i = 0; i < NS / 4; ++i) {
                    const float4 t = v[i];
                    s[4 * i] = t.x;
                    s[4 * i + 1] = t.y;
                    s[4 * i + 2] = t.z;
                    s[4 * i + 3] = t.w;
                }
            } else {
                const double2* v = reinterpret_cast<const double2*>(sf[q]);
#pragma unroll
                for (int i = 0; i < NS / 2; ++i) {
                    const double2 t = v[i];
                    s[2 * i] = t.x;
                    s[2 * i + 1] = t.y;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) s[i] = sf[q][i];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T acc = b.N * s[f];
#pragma unroll
            for (int k = 0; k < D; ++k) acc += b.dN[k] * s[NF + f * D + k];
            r[f] += acc;
        }
    }
}

// Scatter strategies of the element kernels (chns_mesh_set_scatter):
//   SCAT_ATOMIC  one atomic add per corner row entry and parent (default);
//   SCAT_PLAIN   plain read-modify-write, for launches over one colour of an element
//                colouring (no two elements of a colour share a node): deterministic;
//   SCAT_WARPAGG the lanes of a warp that target the same node (found with
//                __match_any_sync) add their rows in shared memory first and one lane
//                issues the atomics.
enum { SCAT_ATOMIC = 0, SCAT_PLAIN = 1, SCAT_WARPAGG = 2 };

template <int D, class T, int SCAT>
__device__ __forceinline__ void scatter_add(T* __restrict__ out, const Parents& P, const T r[Shape<D>::NF]) {
    constexpr int NF = Shape<D>::NF;
    const T w = (P.n == 1) ? T(1) : (P.n == 2 ? T(0.5) : T(0.25));
    for (int j = 0; j < P.n; ++j) {
        T* o = out + (size_t)P.p[j] * NF;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (SCAT == SCAT_PLAIN)
                o[f] += w * r[f];
            else
                atomicAdd(o + f, w * r[f]);
        }
    }
}

// Warp-aggregated scatter: every lane of the warp calls it (valid == false: no rows).
// wbuf: this warp's 32 x NF shared staging rows.
template <int D, class T>
__device__ __forceinline__ void scatter_add_warpagg(T* __restrict__ out, const Parents& P, const T r[Shape<D>::NF],
                                                    bool valid, T (*wbuf)[Shape<D>::NF]) {
    constexpr int NF = Shape<D>::NF;
    const int lane = threadIdx.x & 31;
    const T w = (P.n == 1) ? T(1) : (P.n == 2 ? T(0.5) : T(0.25));
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        const int node = (valid && j < P.n) ? P.p[j] : -1;
        if (node >= 0) {
#pragma unroll
            for (int f = 0; f < NF; ++f) wbuf[lane][f] = w * r[f];
        }
        __syncwarp();
        const unsigned grp = __match_any_sync(0xffffffffu, node);
        if (node >= 0 && lane == __ffs(grp) - 1) {
            T acc[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f] = T(0);
            for (unsigned g = grp; g; g &= g - 1) {
                const int src = __ffs(g) - 1;
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f] += wbuf[src][f];
            }
            T* o = out + (size_t)node * NF;
#pragma unroll
            for (int f = 0; f < NF; ++f) atomicAdd(o + f, acc[f]);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------
// Residual (MODE_RES) and J x (MODE_JVP) share one kernel body.
// ---------------------------------------------------------------------------------
enum { MODE_RES = 0, MODE_JVP = 1 };

template <int D, class T, int MODE>
struct __align__(16) SmemRJ {
    CornerPrimal<D, T> cp;
    __align__(16) T x[MODE == MODE_JVP ? Shape<D>::NC : 1][Shape<D>::NF];   // tangent corner values
    T xps[MODE == MODE_JVP ? Shape<D>::NC : 1];                             // tangent of phi*
    __align__(16) T f[Shape<D>::NC][Shape<D>::NF * (D + 1)];                // fluxes per Gauss point
};

template <int D, class T, int MODE, int SCAT>
__global__ void __launch_bounds__(128, (MODE == MODE_JVP && sizeof(T) == 4) ? 5 : 1)
elem_rj_kernel(DevMesh m, PCst<T> c, T inv_dt, T span,
                                                      const T* __restrict__ Uo,
                                                      const T* __restrict__ Un,
                                                      const T* __restrict__ xin, T* __restrict__ out,
                                                      unsigned int* __restrict__ flags,
                                                      const int32_t* __restrict__ elist, int64_t ecount) {
    constexpr int NC = Shape<D>::NC, NF = Shape<D>::NF, EPB = Shape<D>::EPB;
    __shared__ __align__(16) SmemRJ<D, T, MODE> sm[EPB];
    __shared__ T wbuf[SCAT == SCAT_WARPAGG ? 4 : 1][32][NF];
    const int le = threadIdx.x / NC;
    const int t = threadIdx.x % NC;
    // element: the idx-th of the launch (elist: the listed elements of one colour)
    const int64_t idx = (int64_t)blockIdx.x * EPB + le;
    const bool valid = idx < ecount;
    const int64_t e = valid ? (elist ? (int64_t)elist[idx] : idx) : 0;
    SmemRJ<D, T, MODE>& S = sm[le];

    Parents P;
    P.n = 0;
    T inv_h = T(1), detJ = T(0);
    if (valid) {
        const int ent = m.e2n[e * NC + t];
        P = parents_of(m, ent);
        const unsigned mask = gather_primal<D, T>(m, P, Uo, Un, S.cp, t);
        const T h = scale_pow2(span, (int)m.level[e]);
        inv_h = T(1) / h;
        detJ = (D == 2) ? (T(0.25) * h * h) : (T(0.125) * h * h * h);
        if (MODE == MODE_JVP) {
            T sx[NF];
            T xps = T(0);
#pragma unroll
            for (int f = 0; f < NF; ++f) sx[f] = T(0);
            const T w = (P.n == 1) ? T(1) : (P.n == 2 ? T(0.5) : T(0.25));
            for (int j = 0; j < P.n; ++j) {
                T xr[NF];
                ld_row<D, T>(xin + (size_t)P.p[j] * NF, xr);
#pragma unroll
                for (int f = 0; f < NF; ++f) sx[f] += w * xr[f];
                if (mask & (1u << j)) xps += w * T(0.5) * xr[D + 1];
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) S.x[t][f] = sx[f];
            S.xps[t] = xps;
        }
    }
    __syncwarp();
    if (valid) {
        const int q = t;
        const T g = T(4) * inv_h * inv_h;
        QPIn<D, T> X;
        interp_primal<D, T>(S.cp, q, inv_h, inv_dt, X);
        if (MODE == MODE_RES) {
            QPOut<D, T> F;
            pointwise<D, T, T>(X, c, g, F);
            // non-positive tau_m radicand shows up as a non-finite tau
            if (!(F.f1[D][0] == F.f1[D][0])) atomicOr(flags, 1u);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                S.f[q][f] = detJ * F.f0[f];
#pragma unroll
                for (int k = 0; k < D; ++k) S.f[q][NF + f * D + k] = detJ * F.f1[f][k];
            }
        } else {
            // tangent inputs: averages move by x/2, differences by x
            QPIn<D, Dual<T>> XD;
            T xv[NF], xg[NF][D], xH[Shape<D>::NH], xdiv = T(0), xpsv = T(0), xpsg[D];
            {
                T w[3];
                gauss_weights<T>(q, w);
                if constexpr (D == 3) {
                    // tangent corner rows two fields at a time
                    typename Pair<T>::type c[NC];
#pragma unroll
                    for (int f = 0; f < NF; f += 2) {
#pragma unroll
                        for (int a = 0; a < NC; ++a) c[a] = ld_pair(&S.x[a][f]);
                        if (f == D + 1)
                            sf_vgrad<D, true, T>(w, inv_h, [&](int a) { return c[a].x; }, xv[f], xg[f], xH);
                        else
                            sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].x; }, xv[f], xg[f], nullptr);
                        sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return c[a].y; }, xv[f + 1], xg[f + 1], nullptr);
                    }
                } else {
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        if (f == D + 1)
                            sf_vgrad<D, true, T>(w, inv_h, [&](int a) { return S.x[a][f]; }, xv[f], xg[f], xH);
                        else
                            sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return S.x[a][f]; }, xv[f], xg[f], nullptr);
                    }
                }
                sf_vgrad<D, false, T>(w, inv_h, [&](int a) { return S.xps[a]; }, xpsv, xpsg, nullptr);
            }
#pragma unroll
            for (int i = 0; i < D; ++i) xdiv += xg[i][i];
            const T hf = T(0.5);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                XD.v[i] = Dual<T>(X.v[i], hf * xv[i]);
#pragma unroll
                for (int k = 0; k < D; ++k) XD.gv[i][k] = Dual<T>(X.gv[i][k], hf * xg[i][k]);
                XD.vdt[i] = Dual<T>(X.vdt[i], inv_dt * xv[i]);
                XD.gp[i] = Dual<T>(X.gp[i], hf * xg[D][i]);
                XD.gphi[i] = Dual<T>(X.gphi[i], hf * xg[D + 1][i]);
                XD.gmu[i] = Dual<T>(X.gmu[i], hf * xg[D + 2][i]);
                XD.gps[i] = Dual<T>(X.gps[i], xpsg[i]);
            }
            XD.p = Dual<T>(X.p, hf * xv[D]);
            XD.phi = Dual<T>(X.phi, hf * xv[D + 1]);
            XD.mu = Dual<T>(X.mu, hf * xv[D + 2]);
#pragma unroll
            for (int k = 0; k < Shape<D>::NH; ++k) XD.H[k] = Dual<T>(X.H[k], hf * xH[k]);
            XD.phidt = Dual<T>(X.phidt, inv_dt * xv[D + 1]);
            XD.divnew = Dual<T>(X.divnew, xdiv);
            XD.ps = Dual<T>(X.ps, xpsv);
            QPOut<D, Dual<T>> F;
            pointwise<D, Dual<T>, T>(XD, c, g, F);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                S.f[q][f] = detJ * F.f0[f].d;
#pragma unroll
                for (int k = 0; k < D; ++k) S.f[q][NF + f * D + k] = detJ * F.f1[f][k].d;
            }
        }
    }
    __syncwarp();
    if (SCAT == SCAT_WARPAGG) {
        T r[NF];
        if (valid) contract<D, T>(S.f, t, inv_h, r);
        scatter_add_warpagg<D, T>(out, P, r, valid, wbuf[(threadIdx.x >> 5) & 3]);
    } else if (SCAT == SCAT_PLAIN) {
        // corners of one element can share a parent node (hanging corners): they add one
        // after another, in corner order; elements of one colour share no node
        T r[NF];
        if (valid) contract<D, T>(S.f, t, inv_h, r);
#pragma unroll 1
        for (int a = 0; a < NC; ++a) {
            if (valid && t == a) scatter_add<D, T, SCAT_PLAIN>(out, P, r);
            __syncwarp();
        }
    } else if (valid) {
        T r[NF];
        contract<D, T>(S.f, t, inv_h, r);
        scatter_add<D, T, SCAT>(out, P, r);
    }
}

// Dirichlet velocity rows and the pressure pin.
//   residual: R = v^{k+1} - g on the Dirichlet rows (g: prescribed velocity, zero when the
//             mesh has none); R[0,p] = p^{k+1} - p^k
//   J x     : y = x on those rows
template <int D, class T>
__global__ void bc_rows_kernel(DevMesh m, const T* __restrict__ a, const T* __restrict__ b,
                               T* __restrict__ out, int pin, bool residual) {
    constexpr int NF = Shape<D>::NF;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.NB) {
        const int64_t n = m.bnodes[i];
        const unsigned fl = m.nflag[n];
#pragma unroll
        for (int k = 0; k < D; ++k)
            if ((fl >> k) & 1u) {
                T v = a[n * NF + k];
                if (residual && m.bcval) v -= (T)m.bcval[n * D + k];
                out[n * NF + k] = v;
            }
    }
    if (i == 0 && pin == 1) out[D] = b ? (a[D] - b[D]) : a[D];
}

// ---------------------------------------------------------------------------------
// J^T w (reverse mode, FP64)
// ---------------------------------------------------------------------------------
template <int D>
struct NXb {
    // packed adjoint of QPIn: v, gv, p, gp, phi, gphi, H, mu, gmu, vdt, phidt, divnew, ps, gps
    static constexpr int n = D + D * D + 1 + D + 1 + D + Shape<D>::NH + 1 + D + D + 1 + 1 + 1 + D;
};

template <int D>
struct SmemVJP {
    CornerPrimal<D, double> cp;
    double wb[Shape<D>::NC][Shape<D>::NF];
    double xb[Shape<D>::NC][NXb<D>::n];
};

template <int D, int SCAT>
__global__ void __launch_bounds__(64) elem_vjp_kernel(DevMesh m, PCst<double> c, double Cn, double inv_dt,
                                                      const double* __restrict__ Uo,
                                                      const double* __restrict__ Un,
                                                      const double* __restrict__ w, double* __restrict__ gn,
                                                      double* __restrict__ go, double* __restrict__ gCn, int pin,
                                                      const int32_t* __restrict__ elist, int64_t ecount) {
    constexpr int NC = Shape<D>::NC, NF = Shape<D>::NF, NH = Shape<D>::NH, EPB = 64 / NC;
    __shared__ SmemVJP<D> sm[EPB];
    const int le = threadIdx.x / NC;
    const int t = threadIdx.x % NC;
    const int64_t idx = (int64_t)blockIdx.x * EPB + le;
    const bool valid = idx < ecount;
    const int64_t e = valid ? (elist ? (int64_t)elist[idx] : idx) : 0;
    SmemVJP<D>& S = sm[le];
    Parents P;
    P.n = 0;
    unsigned mask = 0;
    double inv_h = 1.0, detJ = 0.0;
    if (valid) {
        P = parents_of(m, m.e2n[e * NC + t]);
        mask = gather_primal<D, double>(m, P, Uo, Un, S.cp, t);
        const double h = scale_pow2(m.hi - m.lo, (int)m.level[e]);
        inv_h = 1.0 / h;
        detJ = (D == 2) ? 0.25 * h * h : 0.125 * h * h * h;
        // adjoint seed: w on rows that the element contributes to (Dirichlet and pin
        // rows are replaced rows, their element contributions are discarded)
        double sw[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) sw[f] = 0.0;
        const double wt = (P.n == 1) ? 1.0 : (P.n == 2 ? 0.5 : 0.25);
        for (int j = 0; j < P.n; ++j) {
            const int n = P.p[j];
            const unsigned fl = m.nflag[n];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                double wv = __ldg(w + (size_t)n * NF + f);
                if (f < D && ((fl >> f) & 1u)) wv = 0.0;
                if (f == D && pin == 1 && n == 0) wv = 0.0;
                sw[f] += wt * wv;
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) S.wb[t][f] = sw[f];
    }
    __syncwarp();
    double cnb = 0.0;
    if (valid) {
        const int q = t;
        const double g = 4.0 * inv_h * inv_h;
        QPIn<D, double> X;
        interp_primal<D, double>(S.cp, q, inv_h, inv_dt, X);
        QPOut<D, double> Fb;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            Fb.f0[f] = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) Fb.f1[f][k] = 0.0;
        }
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const Basis<D, double> b = basis<D, double>(a, q, inv_h);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const double wv = detJ * S.wb[a][f];
                Fb.f0[f] += b.N * wv;
#pragma unroll
                for (int k = 0; k < D; ++k) Fb.f1[f][k] += b.dN[k] * wv;
            }
        }
        QPIn<D, double> Xb;
        pointwise_adjoint<D>(X, c, Cn, g, Fb, Xb, cnb);
        double* o = S.xb[q];
        int k = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) o[k++] = Xb.v[i];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) o[k++] = Xb.gv[i][j];
        o[k++] = Xb.p;
#pragma unroll
        for (int i = 0; i < D; ++i) o[k++] = Xb.gp[i];
        o[k++] = Xb.phi;
#pragma unroll
        for (int i = 0; i < D; ++i) o[k++] = Xb.gphi[i];
#pragma unroll
        for (int i = 0; i < NH; ++i) o[k++] = Xb.H[i];
        o[k++] = Xb.mu;
#pragma unroll
        for (int i = 0; i < D; ++i) o[k++] = Xb.gmu[i];
#pragma unroll
        for (int i = 0; i < D; ++i) o[k++] = Xb.vdt[i];
        o[k++] = Xb.phidt;
        o[k++] = Xb.divnew;
        o[k++] = Xb.ps;
#pragma unroll
        for (int i = 0; i < D; ++i) o[k++] = Xb.gps[i];
    }
    __syncwarp();
    double rn[NF], ro[NF], psb = 0.0;
    if (valid) {
        // transpose of the interpolation for corner a = t
        const int a = t;
        double ut[NF], ddv[D + 1], divb[D];
#pragma unroll
        for (int f = 0; f < NF; ++f) ut[f] = 0.0;
#pragma unroll
        for (int i = 0; i <= D; ++i) ddv[i] = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) divb[i] = 0.0;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const Basis<D, double> b = basis<D, double>(a, q, inv_h);
            const double* x = S.xb[q];
            int k = 0;
#pragma unroll
            for (int i = 0; i < D; ++i) ut[i] += b.N * x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) ut[i] += b.dN[j] * x[k++];
            ut[D] += b.N * x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i) ut[D] += b.dN[i] * x[k++];
            ut[D + 1] += b.N * x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i) ut[D + 1] += b.dN[i] * x[k++];
#pragma unroll
            for (int i = 0; i < NH; ++i) ut[D + 1] += b.d2N[i] * x[k++];
            ut[D + 2] += b.N * x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i) ut[D + 2] += b.dN[i] * x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i) ddv[i] += b.N * x[k++];
            ddv[D] += b.N * x[k++];
            const double dvb = x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i) divb[i] += b.dN[i] * dvb;
            psb += b.N * x[k++];
#pragma unroll
            for (int i = 0; i < D; ++i) psb += b.dN[i] * x[k++];
        }
        // corner adjoints of U^{k+1} and U^k: averages take 1/2 each, differences +-1/dt,
        // div v^{k+1} acts on the new level only
#pragma unroll
        for (int f = 0; f < NF; ++f) rn[f] = ro[f] = 0.5 * ut[f];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            rn[i] += inv_dt * ddv[i] + divb[i];
            ro[i] -= inv_dt * ddv[i];
        }
        rn[D + 1] += inv_dt * ddv[D];
        ro[D + 1] -= inv_dt * ddv[D];
    }
    {
        const double wt = (P.n == 1) ? 1.0 : (P.n == 2 ? 0.5 : 0.25);
        // plain adds (colouring): the corners of an element add one after another (two
        // corners can share a constraint parent); elements of one colour share no node
#pragma unroll 1
        for (int a = 0; a < (SCAT == SCAT_PLAIN ? NC : 1); ++a) {
            if (valid && (SCAT != SCAT_PLAIN || t == a)) {
                for (int j = 0; j < P.n; ++j) {
                    double* on = gn + (size_t)P.p[j] * NF;
                    double* oo = go ? go + (size_t)P.p[j] * NF : nullptr;
                    const double pst = (mask & (1u << j)) ? 0.5 * psb : 0.0;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const double extra = (f == D + 1) ? pst : 0.0;
                        if (SCAT == SCAT_PLAIN) {
                            on[f] += wt * (rn[f] + extra);
                            if (oo) oo[f] += wt * (ro[f] + extra);
                        } else {
                            atomicAdd(on + f, wt * (rn[f] + extra));
                            if (oo) atomicAdd(oo + f, wt * (ro[f] + extra));
                        }
                    }
                }
            }
            if (SCAT == SCAT_PLAIN) __syncwarp();
        }
    }
    if (gCn) {
        // block reduction of d/dCn (each Gauss point thread holds its share)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cnb += __shfl_xor_sync(0xffffffffu, cnb, off);
        if ((threadIdx.x & 31) == 0 && cnb != 0.0) atomicAdd(gCn, cnb);
    }
}

// Dirichlet/pin rows of J^T w: identity rows pass w through.
template <int D>
__global__ void bc_vjp_kernel(DevMesh m, const double* __restrict__ w, double* __restrict__ gn,
                              double* __restrict__ go, int pin) {
    constexpr int NF = Shape<D>::NF;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.NB) {
        const int64_t n = m.bnodes[i];
        const unsigned fl = m.nflag[n];
#pragma unroll
        for (int k = 0; k < D; ++k)
            if ((fl >> k) & 1u) gn[n * NF + k] += w[n * NF + k];
    }
    if (i == 0 && pin == 1) {
        gn[D] += w[D];
        if (go) go[D] -= w[D];
    }
}

template <int D, class T, int MODE>
cudaError_t launch_rj(const chns_mesh* mm, const PhysConst& pc, const T* Uo, const T* Un, const T* x,
                      T* out, int pin, cudaStream_t s) {
    const DevMesh& m = mm->dm;
    const size_t bytes = (size_t)m.N * Shape<D>::NF * sizeof(T);
    cudaError_t err = cudaMemsetAsync(out, 0, bytes, s);
    if (err != cudaSuccess) return err;
    const int EPB = Shape<D>::EPB;
    const PCst<T> c = make_pcst<T>(pc);
    if (mm->scatter == SCAT_PLAIN) {
        // one launch per colour of the element colouring, fixed order: deterministic sums
        for (size_t k = 0; k + 1 < mm->colour_off.size(); ++k) {
            const int64_t c0 = mm->colour_off[k], cnt = mm->colour_off[k + 1] - c0;
            if (cnt <= 0) continue;
            elem_rj_kernel<D, T, MODE, SCAT_PLAIN><<<(unsigned)((cnt + EPB - 1) / EPB), EPB * Shape<D>::NC, 0, s>>>(
                m, c, T(pc.inv_dt), T(m.hi - m.lo), Uo, Un, x, out, mm->d_flags, mm->d_elist + c0, cnt);
            chns_count_launches(1);
        }
    } else {
        const int64_t blocks = (m.E + EPB - 1) / EPB;
        if (mm->scatter == SCAT_WARPAGG)
            elem_rj_kernel<D, T, MODE, SCAT_WARPAGG><<<(unsigned)blocks, EPB * Shape<D>::NC, 0, s>>>(
                m, c, T(pc.inv_dt), T(m.hi - m.lo), Uo, Un, x, out, mm->d_flags, nullptr, m.E);
        else
            elem_rj_kernel<D, T, MODE, SCAT_ATOMIC><<<(unsigned)blocks, EPB * Shape<D>::NC, 0, s>>>(
                m, c, T(pc.inv_dt), T(m.hi - m.lo), Uo, Un, x, out, mm->d_flags, nullptr, m.E);
        chns_count_launches(1);
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int64_t nb = m.NB > 0 ? m.NB : 1;
    if (MODE == MODE_RES)
        { bc_rows_kernel<D, T><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, Un, Uo, out, pin, true); chns_count_launches(1); }
    else
        { bc_rows_kernel<D, T><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, x, nullptr, out, pin, false); chns_count_launches(1); }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_residual(const chns_mesh* m, const PhysConst& pc, const double* U_old, const double* U_new,
                            double* R, int pin, cudaStream_t s) {
    if (m->dm.dim == 2) return launch_rj<2, double, MODE_RES>(m, pc, U_old, U_new, nullptr, R, pin, s);
    return launch_rj<3, double, MODE_RES>(m, pc, U_old, U_new, nullptr, R, pin, s);
}

cudaError_t launch_jvp64(const chns_mesh* m, const PhysConst& pc, const double* U_old, const double* U_lin,
                         const double* x, double* y, int pin, cudaStream_t s) {
    if (m->dm.dim == 2) return launch_rj<2, double, MODE_JVP>(m, pc, U_old, U_lin, x, y, pin, s);
    return launch_rj<3, double, MODE_JVP>(m, pc, U_old, U_lin, x, y, pin, s);
}

cudaError_t launch_jvp32(const chns_mesh* m, const PhysConst& pc, const float* U_old, const float* U_lin,
                         const float* x, float* y, int pin, cudaStream_t s) {
    if (m->dm.dim == 2) return launch_rj<2, float, MODE_JVP>(m, pc, U_old, U_lin, x, y, pin, s);
    return launch_rj<3, float, MODE_JVP>(m, pc, U_old, U_lin, x, y, pin, s);
}

cudaError_t launch_vjp(const chns_mesh* mm, const PhysConst& pc, const double* U_old, const double* U_lin,
                       const double* w, double* gU_new, double* gU_old, double* gCn, int pin, cudaStream_t s) {
    const DevMesh& m = mm->dm;
    const int NF = m.nf;
    cudaError_t err = cudaMemsetAsync(gU_new, 0, (size_t)m.N * NF * sizeof(double), s);
    if (err == cudaSuccess && gU_old) err = cudaMemsetAsync(gU_old, 0, (size_t)m.N * NF * sizeof(double), s);
    if (err == cudaSuccess && gCn) err = cudaMemsetAsync(gCn, 0, sizeof(double), s);
    if (err != cudaSuccess) return err;
    const int64_t nb = m.NB > 0 ? m.NB : 1;
    const PCst<double> c = make_pcst<double>(pc);
    auto elems = [&](auto dimtag) {
        constexpr int D = decltype(dimtag)::value;
        constexpr int EPB = 64 / (1 << D);
        if (mm->scatter == SCAT_PLAIN) {
            for (size_t k = 0; k + 1 < mm->colour_off.size(); ++k) {
                const int64_t c0 = mm->colour_off[k], cnt = mm->colour_off[k + 1] - c0;
                if (cnt <= 0) continue;
                elem_vjp_kernel<D, SCAT_PLAIN><<<(unsigned)((cnt + EPB - 1) / EPB), 64, 0, s>>>(
                    m, c, pc.Cn, pc.inv_dt, U_old, U_lin, w, gU_new, gU_old, gCn, pin, mm->d_elist + c0, cnt);
                chns_count_launches(1);
            }
        } else {
            elem_vjp_kernel<D, SCAT_ATOMIC><<<(unsigned)((m.E + EPB - 1) / EPB), 64, 0, s>>>(
                m, c, pc.Cn, pc.inv_dt, U_old, U_lin, w, gU_new, gU_old, gCn, pin, nullptr, m.E);
            chns_count_launches(1);
        }
    };
    if (m.dim == 2) elems(std::integral_constant<int, 2>());
    else elems(std::integral_constant<int, 3>());
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (m.dim == 2)
        { bc_vjp_kernel<2><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, w, gU_new, gU_old, pin); chns_count_launches(1); }
    else
        { bc_vjp_kernel<3><<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(m, w, gU_new, gU_old, pin); chns_count_launches(1); }
    return cudaGetLastError();
}
