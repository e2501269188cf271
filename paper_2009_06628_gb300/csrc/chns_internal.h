// Internal declarations shared by the translation units of libchns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "chns.h"

// Everything a kernel needs to know about the mesh (plain pointers into device memory).
struct DevMesh {
    int32_t dim, nc, nf;
    int64_t E, N, H, NB;
    const int32_t* e2n;     // E * nc: >= 0 independent node, < 0: -(hanging index + 1)
    const int32_t* hang;    // H * 4 parent node indices; -1 marks an unused slot (edge case)
    const int8_t* level;    // E element levels
    const uint8_t* nflag;   // N node flags, bit k < dim: velocity component k has a Dirichlet row
    const int32_t* bnodes;  // NB nodes with at least one Dirichlet velocity row
    const double* bcval;    // N * dim prescribed velocities of the Dirichlet rows (null: zero)
    const int32_t* anchor;  // E * dim element anchors (units of the finest cell)
    int32_t max_level;
    double lo, hi;
};

struct SolverWS;  // Newton-Krylov workspace (solver.cu)
struct MGHier;    // geometric multigrid hierarchy of the pressure Schur Laplacian (multigrid.cu)

struct chns_mesh {
    DevMesh dm;
    int32_t max_level;
    int32_t order = 1;                 // 1: Q1 on a 2:1 octree; 2: Q2 on a uniform octree
    int32_t q2_level = 0;              // Q2: the element level (max_level = q2_level + 1 then)
    int32_t device = 0;                // CUDA device ordinal that holds the mesh's arrays
    std::vector<int32_t> node_coords;  // host copy, N * dim
    // host copies of the element arrays (transfer operators, coarse meshes, remeshing)
    std::vector<int32_t> h_e2n;        // E * nc
    std::vector<int32_t> h_hang;       // max(H, 1) * 4
    std::vector<int32_t> h_anchor;     // E * dim
    std::vector<int8_t> h_level;       // E
    // owning device pointers
    int32_t* d_e2n = nullptr;
    int32_t* d_hang = nullptr;
    int8_t* d_level = nullptr;
    uint8_t* d_nflag = nullptr;
    int32_t* d_bnodes = nullptr;
    double* d_bcval = nullptr;       // prescribed Dirichlet velocities (null: homogeneous)
    int32_t* d_anchor = nullptr;
    double* d_nmass = nullptr;       // integral of each node's basis function
    double volume = 0.0;             // |Omega|
    // reduction workspace: per-block partial sums and a flag word
    double* d_partials = nullptr;
    int64_t n_partials = 0;
    double* h_pinned = nullptr;      // pinned host landing zone for scalar results
    unsigned int* d_flags = nullptr; // bit 0: a tau radicand was not positive
    SolverWS* ws = nullptr;
    MGHier* mg = nullptr;
    // scatter strategy of the element kernels (0 atomics, 1 colouring, 2 warp-aggregated)
    int32_t scatter = 0;
    int32_t* d_elist = nullptr;          // elements sorted by colour (Morton order within one)
    std::vector<int64_t> colour_off;     // colour k: d_elist[colour_off[k] .. colour_off[k + 1])
};

// Kernel-side parameter block derived from chns_params (all FP64; kernels cast).
struct PhysConst {
    double dt, inv_dt, four_over_dt2;
    double inv_Re, inv_We, inv_Pe, inv_Fr;  // inv_Fr = 0: no gravity
    double Cn, We, Pe, Re;
    double rho_plus, rho_minus;
    double alpha, beta, gamma, xi;
    double C_I, C_phi;
};

// error helpers (capi.cpp)
void chns_set_error(const std::string& msg);
chns_status chns_cuda_status(cudaError_t err, const char* where);
chns_status chns_check_params(const chns_mesh* mesh, const chns_params* p, PhysConst* out);
// 3D node rows are read in pairs: CHNS_EINVAL unless p is 2 * elem_bytes aligned
chns_status chns_check_rows(const chns_mesh* mesh, const void* p, int elem_bytes);

#define CHNS_CUDA(call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return chns_cuda_status(e_, #call);        \
    } while (0)

// kernel launchers (element_kernels.cu, reduce_kernels.cu)
cudaError_t launch_residual(const chns_mesh* m, const PhysConst& pc, const double* U_old,
                            const double* U_new, double* R, int pin, cudaStream_t s);
cudaError_t launch_jvp64(const chns_mesh* m, const PhysConst& pc, const double* U_old,
                         const double* U_lin, const double* x, double* y, int pin, cudaStream_t s);
cudaError_t launch_jvp32(const chns_mesh* m, const PhysConst& pc, const float* U_old,
                         const float* U_lin, const float* x, float* y, int pin, cudaStream_t s);
cudaError_t launch_vjp(const chns_mesh* m, const PhysConst& pc, const double* U_old,
                       const double* U_lin, const double* w, double* gU_new, double* gU_old,
                       double* gCn, int pin, cudaStream_t s);
cudaError_t launch_mass(const chns_mesh* m, const double* U, double* out_dev, cudaStream_t s);
cudaError_t launch_energy(const chns_mesh* m, const PhysConst& pc, const double* U,
                          double* out_dev3, cudaStream_t s);
// deterministic FP64 reductions into device scalars (solver.cu uses them)
cudaError_t launch_dot(const chns_mesh* m, const double* a, const double* b, int64_t n, double* out_dev,
                       cudaStream_t s);
cudaError_t launch_multidot(const chns_mesh* m, const double* V, int64_t ld, int k, const double* w, int64_t n,
                            double* out_dev, cudaStream_t s);

// ---------------------------------------------------------------------------------
// Transfer between the Q1 spaces of two meshes of the same domain (multigrid.cu):
// P u = the source field interpolated at the target's independent nodes (Q1 on the
// source element containing the node, source hanging constraints folded in), stored as
// CSR rows over target nodes, together with its transpose (rows over source nodes), in
// FP64 and FP32.  Exact (no loss) when the target mesh refines the source mesh.
struct TransferDev {
    int64_t n_src = 0, n_dst = 0, nnz = 0;
    int64_t* rp = nullptr;   // n_dst + 1
    int32_t* col = nullptr;  // nnz source nodes
    double* w = nullptr;
    float* wf = nullptr;
    int64_t* rpT = nullptr;  // n_src + 1
    int32_t* colT = nullptr; // nnz target nodes
    double* wT = nullptr;
    float* wTf = nullptr;
};
chns_status transfer_build(const chns_mesh* src, const chns_mesh* dst, TransferDev* T);
void transfer_free(TransferDev* T);
// out = P in (transpose = false; in: n_src x nf, out: n_dst x nf) or P^T in (transpose = true),
// FP64, overwriting out
cudaError_t transfer_apply_f64(const TransferDev& T, bool transpose, int nf, const double* in, double* out,
                               cudaStream_t s);
// scalar FP32 fields: out (+)= P in or P^T in
cudaError_t transfer_apply_f32(const TransferDev& T, bool transpose, bool add, const float* in, float* out,
                               cudaStream_t s);

// Geometric multigrid hierarchy of the pressure Schur Laplacian (multigrid.cu builds it,
// solver.cu sets it up and applies V-cycles).  Level 0 is the mesh itself; level l + 1 caps
// every leaf of level l at (deepest level of l) - 1, which keeps the octree complete and
// 2:1 balanced and makes its Q1 space a subspace of level l's.
struct MGLevel {
    chns_mesh* mesh = nullptr;  // owned coarse mesh (null for level 0)
    DevMesh dm;                 // the level's mesh as kernels see it
    int64_t N = 0, E = 0;
    TransferDev P;              // this level -> level - 1 (level >= 1)
    int32_t* fmap = nullptr;    // for every element of level - 1: its element on this level
    float* ce = nullptr;        // element coefficients of the Schur Laplacian
    float* dinv = nullptr;      // inverse diagonal
    float* bnd = nullptr;       // absolute-row-sum bounds (Gershgorin)
    float* b = nullptr;         // right-hand side, solution, residual
    float* x = nullptr;
    float* t = nullptr;
    float* cr = nullptr;        // Chebyshev work vectors
    float* cx = nullptr;
    float* cd = nullptr;
    float* cy = nullptr;
    std::vector<float> c1, c2;  // Chebyshev recurrence coefficients of this level
    float inv_theta = 0.0f;
    int deg = 0;
};
struct MGHier {
    std::vector<MGLevel> lv;
    unsigned int* kmax = nullptr;   // per-level Gershgorin bounds (float bits)
};
chns_status mg_hier_build(chns_mesh* m);   // no-op when m->mg exists
void chns_mg_free(MGHier* mg);

// Q2 element kernels (q2_kernels.cu)
cudaError_t q2_launch_residual(const chns_mesh* m, const PhysConst& pc, const double* Uo, const double* Un, double* R,
                               cudaStream_t s);
cudaError_t q2_launch_jvp64(const chns_mesh* m, const PhysConst& pc, const double* Uo, const double* Un,
                            const double* x, double* y, cudaStream_t s);
cudaError_t q2_launch_jvp32(const chns_mesh* m, const PhysConst& pc, const float* Uo, const float* Un, const float* x,
                            float* y, cudaStream_t s);
cudaError_t q2_launch_vjp(const chns_mesh* m, const PhysConst& pc, const double* Uo, const double* Un,
                          const double* w, double* gn, double* go, double* gCn, cudaStream_t s);
// CHNS_EINVAL (naming `what`) unless the mesh has Q1 elements
chns_status chns_require_q1(const chns_mesh* m, const char* what);

// launch accounting (capi.cpp)
void chns_count_launches(int n);

// grid sizing helper: SM count of the current device (cached)
int chns_num_sms();
