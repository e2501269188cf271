// C-ABI entry points, argument validation and error reporting.
#include <atomic>
#include <cmath>
#include <string>

#include "chns_internal.h"

namespace {
thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};
}

void chns_count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" int64_t chns_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void chns_set_error(const std::string& msg) { g_err = msg; }

chns_status chns_cuda_status(cudaError_t err, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(err);
    return CHNS_ECUDA;
}

extern "C" const char* chns_last_error(void) { return g_err.c_str(); }

int chns_num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    }
    return sms;
}

chns_status chns_require_q1(const chns_mesh* m, const char* what) {
    if (m && m->order != 1) {
        chns_set_error(std::string(what) + " is available for Q1 meshes only (Q2 meshes: residual, J x, J^T w)");
        return CHNS_EINVAL;
    }
    return CHNS_OK;
}

chns_status chns_check_rows(const chns_mesh* m, const void* p, int elem_bytes) {
    // 3D node rows (6 values) are read as pairs: the vector must start on 2 * elem_bytes
    if (m && m->dm.dim == 3 && p && ((uintptr_t)p % (uintptr_t)(2 * elem_bytes)) != 0) {
        chns_set_error("3D vectors must start on a " + std::to_string(2 * elem_bytes) + "-byte boundary");
        return CHNS_EINVAL;
    }
    return CHNS_OK;
}

chns_status chns_check_params(const chns_mesh* m, const chns_params* p, PhysConst* out) {
    if (!m || !p) { chns_set_error("null mesh or params"); return CHNS_EINVAL; }
    if (p->dim != m->dm.dim) { chns_set_error("params.dim differs from the mesh dimension"); return CHNS_EINVAL; }
    const double pos[] = {p->Re, p->We, p->Pe, p->Cn, p->dt, p->rho_ratio, p->eta_ratio};
    for (double v : pos)
        if (!(v > 0.0) || !std::isfinite(v)) {
            chns_set_error("Re, We, Pe, Cn, dt, rho_ratio, eta_ratio must be positive and finite");
            return CHNS_EINVAL;
        }
    if (!(p->C_I >= 0.0) || !(p->C_phi >= 0.0) || !std::isfinite(p->Fr)) {
        chns_set_error("C_I, C_phi must be >= 0 and Fr finite");
        return CHNS_EINVAL;
    }
    PhysConst& c = *out;
    c.dt = p->dt;
    c.inv_dt = 1.0 / p->dt;
    c.four_over_dt2 = 4.0 / (p->dt * p->dt);
    c.inv_Re = 1.0 / p->Re;
    c.inv_We = 1.0 / p->We;
    c.inv_Pe = 1.0 / p->Pe;
    c.inv_Fr = p->Fr > 0.0 ? 1.0 / p->Fr : 0.0;
    c.Cn = p->Cn;
    c.We = p->We;
    c.Pe = p->Pe;
    c.Re = p->Re;
    // Eq. (alpha_beta_defn) with rho_+ = eta_+ = 1 for the phi = +1 phase
    c.rho_plus = 1.0;
    c.rho_minus = 1.0 / p->rho_ratio;
    const double eta_plus = 1.0, eta_minus = 1.0 / p->eta_ratio;
    c.alpha = (c.rho_plus - c.rho_minus) / (2.0 * c.rho_plus);
    c.beta = (c.rho_plus + c.rho_minus) / (2.0 * c.rho_plus);
    c.gamma = (eta_plus - eta_minus) / (2.0 * eta_plus);
    c.xi = (eta_plus + eta_minus) / (2.0 * eta_plus);
    c.C_I = p->C_I;
    c.C_phi = p->C_phi;
    return CHNS_OK;
}

extern "C" chns_status chns_residual(const chns_mesh* m, const chns_params* p, const double* U_old,
                                     const double* U_new, double* R, void* stream) {
    PhysConst pc;
    chns_status st = chns_check_params(m, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U_old || !U_new || !R) { chns_set_error("null vector"); return CHNS_EINVAL; }
    if ((st = chns_check_rows(m, U_old, 8)) != CHNS_OK || (st = chns_check_rows(m, U_new, 8)) != CHNS_OK) return st;
    if (m->order == 2) {
        if (p->pin_pressure == 1) { chns_set_error("Q2 meshes take pin_pressure 0 or 2"); return CHNS_EINVAL; }
        CHNS_CUDA(q2_launch_residual(m, pc, U_old, U_new, R, (cudaStream_t)stream));
        return CHNS_OK;
    }
    CHNS_CUDA(launch_residual(m, pc, U_old, U_new, R, p->pin_pressure, (cudaStream_t)stream));
    return CHNS_OK;
}

extern "C" chns_status chns_jvp(const chns_mesh* m, const chns_params* p, const void* U_old, const void* U_lin,
                                const void* x, void* y, int32_t precision, void* stream) {
    PhysConst pc;
    chns_status st = chns_check_params(m, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U_old || !U_lin || !x || !y) { chns_set_error("null vector"); return CHNS_EINVAL; }
    if (precision == 0 || precision == 1) {
        const int eb = precision == 0 ? 8 : 4;
        if ((st = chns_check_rows(m, U_old, eb)) != CHNS_OK || (st = chns_check_rows(m, U_lin, eb)) != CHNS_OK ||
            (st = chns_check_rows(m, x, eb)) != CHNS_OK)
            return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (m->order == 2 && (precision == 0 || precision == 1)) {
        if (p->pin_pressure == 1) { chns_set_error("Q2 meshes take pin_pressure 0 or 2"); return CHNS_EINVAL; }
        if (precision == 0)
            CHNS_CUDA(q2_launch_jvp64(m, pc, (const double*)U_old, (const double*)U_lin, (const double*)x, (double*)y, s));
        else
            CHNS_CUDA(q2_launch_jvp32(m, pc, (const float*)U_old, (const float*)U_lin, (const float*)x, (float*)y, s));
        return CHNS_OK;
    }
    if (precision == 0) {
        CHNS_CUDA(launch_jvp64(m, pc, (const double*)U_old, (const double*)U_lin, (const double*)x, (double*)y,
                               p->pin_pressure, s));
    } else if (precision == 1) {
        CHNS_CUDA(launch_jvp32(m, pc, (const float*)U_old, (const float*)U_lin, (const float*)x, (float*)y,
                               p->pin_pressure, s));
    } else {
        chns_set_error("precision must be 0 (FP64) or 1 (FP32)");
        return CHNS_EINVAL;
    }
    return CHNS_OK;
}

extern "C" chns_status chns_vjp(const chns_mesh* m, const chns_params* p, const double* U_old, const double* U_lin,
                                const double* w, double* gU_new, double* gU_old, double* gCn, void* stream) {
    PhysConst pc;
    chns_status st = chns_check_params(m, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U_old || !U_lin || !w || !gU_new) { chns_set_error("null vector"); return CHNS_EINVAL; }
    if ((st = chns_check_rows(m, U_old, 8)) != CHNS_OK || (st = chns_check_rows(m, U_lin, 8)) != CHNS_OK) return st;
    if (m->order == 2) {
        if (p->pin_pressure == 1) { chns_set_error("Q2 meshes take pin_pressure 0 or 2"); return CHNS_EINVAL; }
        CHNS_CUDA(q2_launch_vjp(m, pc, U_old, U_lin, w, gU_new, gU_old, gCn, (cudaStream_t)stream));
        return CHNS_OK;
    }
    CHNS_CUDA(launch_vjp(m, pc, U_old, U_lin, w, gU_new, gU_old, gCn, p->pin_pressure, (cudaStream_t)stream));
    return CHNS_OK;
}

extern "C" chns_status chns_mass(const chns_mesh* m, const double* U, double* out, void* stream) {
    if (!m || !U || !out) { chns_set_error("null argument"); return CHNS_EINVAL; }
    if (chns_require_q1(m, "chns_mass") != CHNS_OK) return CHNS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CHNS_CUDA(launch_mass(m, U, m->d_partials + (size_t)m->n_partials * 8 - 8, s));
    CHNS_CUDA(cudaMemcpyAsync(m->h_pinned, m->d_partials + (size_t)m->n_partials * 8 - 8, sizeof(double),
                              cudaMemcpyDeviceToHost, s));
    CHNS_CUDA(cudaStreamSynchronize(s));
    *out = m->h_pinned[0];
    return CHNS_OK;
}

extern "C" chns_status chns_energy(const chns_mesh* m, const chns_params* p, const double* U, double* out,
                                   void* stream) {
    PhysConst pc;
    chns_status st = chns_check_params(m, p, &pc);
    if (st != CHNS_OK) return st;
    if (!U || !out) { chns_set_error("null argument"); return CHNS_EINVAL; }
    if ((st = chns_require_q1(m, "chns_energy")) != CHNS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double* dev_out = m->d_partials + (size_t)m->n_partials * 8 - 8;
    CHNS_CUDA(launch_energy(m, pc, U, dev_out, s));
    CHNS_CUDA(cudaMemcpyAsync(m->h_pinned, dev_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHNS_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < 3; ++i) out[i] = m->h_pinned[i];
    return CHNS_OK;
}
