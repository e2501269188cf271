/*
 * chns.h -- C-ABI of the GB300 matrix-free CHNS hot path.
 *
 * Method: the fully-coupled, Crank-Nicolson, variational-multiscale (RBVMS)
 * Cahn-Hilliard Navier-Stokes scheme of Khanwale et al. (arXiv 2009.06628):
 * time scheme and weak form of Definition 1 (Section 3), the fully discrete VMS
 * form of Definition 2 with its stabilisation parameters and strong residuals
 * (Section 3.3), Newton's method of Section 3.4, on Q1 elements of a 2:1
 * balanced octree with hanging nodes (Section 4).
 *
 * Conventions shared by every call:
 *  - dim d in {2, 3}; n_f = d + 3 fields per node in the order v_1..v_d, p, phi, mu.
 *  - Vectors are caller-owned, contiguous, node-major and interleaved:
 *    U[node * n_f + field].  Pointers documented "device" must be CUDA device
 *    pointers (e.g. torch CUDA tensors); "host" pointers are ordinary memory.
 *  - In 3D, U-type vectors read by the element kernels (U_old, U_new / U_lin, x of J x)
 *    must start on a 16-byte (FP64) or 8-byte (FP32) boundary, as every cudaMalloc and
 *    torch allocation does: node rows are read in pairs.  Others give CHNS_EINVAL.
 *  - Independent nodes are numbered in Morton (Z) order of their integer
 *    coordinates (units of the finest cell, max_level + 1 bits per axis, x fastest).
 *  - Dirichlet rows: by default every velocity component of every node on the
 *    boundary of the domain cube has the row R = v^{k+1} (no-slip, Definition 1);
 *    chns_mesh_set_velocity_bc chooses, per face and component, Dirichlet rows
 *    R = v^{k+1} - g with prescribed values g, or the natural condition (no row
 *    replaced).  phi and mu always take the natural (no-flux) condition.
 *  - Pressure level (closed no-slip boxes determine p only up to a constant; the
 *    pressure rows sum to zero): params.pin_pressure = 0 keeps every row;
 *    1 replaces the pressure row of node 0 (the corner at lo^d) by p^{k+1} - p^k
 *    (a point value, which leaves J badly conditioned); 2 keeps every row (J has the
 *    constant pressure as null vector) and chns_newton_step keeps
 *    int p^{k+1} = int p^k by removing the mean of every pressure update.
 *  - Calls that take a `stream` (a cudaStream_t passed as void*, NULL = legacy
 *    default stream) are asynchronous on it, unless they return host scalars
 *    (mass, energy, Newton statistics, mu0), which synchronise that stream.
 *  - A mesh holds device workspace; one mesh may be used by one stream at a time.
 *  - On any error nothing of the caller's outputs is written before validation
 *    fails; a status other than CHNS_OK is returned and chns_last_error() gives
 *    a message (thread-local).
 */
#ifndef CHNS_H
#define CHNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CHNS_OK = 0,
    CHNS_EINVAL = 1,          /* bad argument (null pointer, dim, level, size, precision) */
    CHNS_ENOTSORTED = 2,      /* leaves not strictly increasing in Morton order */
    CHNS_ENOTCOMPLETE = 3,    /* leaves overlap, leave gaps, or are misaligned */
    CHNS_ENOTBALANCED = 4,    /* two leaves sharing a point differ by more than one level */
    CHNS_ENOMEM = 5,          /* host or device allocation failed */
    CHNS_ECUDA = 6,           /* a CUDA runtime call failed */
    CHNS_ENAN = 7,            /* a non-finite norm appeared in Newton/Krylov */
    CHNS_ENOCONV = 8,         /* Newton did not reach the tolerance within max_newton */
    CHNS_EBREAKDOWN = 9,      /* Krylov breakdown (zero or non-finite Arnoldi vector) */
    CHNS_ETAU = 10            /* a stabilisation radicand was not positive */
} chns_status;

/* Opaque mesh: immutable after creation, owns its device arrays and workspace. */
typedef struct chns_mesh chns_mesh;

/* One octree leaf: integer anchor in units of the finest cell (2^max_level cells
 * per axis; z = 0 in 2D) and its level.  16 bytes, matching an (n, 4) int32 array. */
typedef struct {
    int32_t x, y, z, level;
} chns_leaf;

/* Physical and numerical parameters of one time step (Section 2 groups).
 * rho_+ = eta_+ = 1 belong to the phi = +1 phase; rho_- = 1/rho_ratio,
 * eta_- = 1/eta_ratio (Eq. alpha_beta_defn).  Fr <= 0 disables gravity; gravity
 * points along -e_{d-1} (last axis).  C_I, C_phi: the constants of tau_m, tau_phi
 * (6 in the paper).  dt: the time step (also the Delta t inside tau). */
typedef struct {
    int32_t dim;
    int32_t pin_pressure;
    double Re, We, Pe, Cn, Fr;
    double rho_ratio, eta_ratio;
    double dt;
    double C_I, C_phi;
} chns_params;

/* Newton-Krylov options.  precision: 0 = FP64 everywhere; 1 = FP32 J.x and
 * preconditioner inside the Krylov solver, FP64 residual, orthogonalisation, dots,
 * norms and update (Newton acts as iterative refinement).  Norms are row-equilibrated:
 * S = 1/|diag J| at U^0 (every field weighed by its own scale; the pressure rows carry
 * coefficients of order tau/We).  Newton stops when ||S R||_2 <= rtol * ||S R(U^0)||_2 or
 * ||S R||_2 <= atol.  Krylov: GMRES(restart) on S J M^{-1} (M: nodal block-Jacobi,
 * right preconditioning) to relative tolerance eta = max(krylov_rtol, min(0.5,
 * 0.1 * target / ||S R||)) with target = max(atol, rtol ||S R(U^0)||) (the last linear
 * solve is not driven further than the Newton target needs), at most max_krylov
 * iterations per Newton iteration.  With ew_eta0 > 0 the fixed krylov_rtol in that
 * formula is replaced by the adaptive forcing term of Eisenstat and Walker (SIAM J. Sci.
 * Comput. 17, 1996, choice 2 with gamma = 0.9, alpha = 2 and their safeguard):
 * eta_0 = ew_eta0, eta_k = 0.9 (||S R_k|| / ||S R_{k-1}||)^2, raised to 0.9 eta_{k-1}^2
 * when that exceeds 0.1, and clamped to [krylov_rtol, 0.9]. */
typedef struct {
    double rtol, atol, krylov_rtol;
    int32_t max_newton, max_krylov, restart, precision;
    int32_t pc_type;     /* 0: nodal block-Jacobi; 1: block-Jacobi on v, phi, mu and a pressure
                            Schur-complement approximation (grad q, dt/(2 rho We) grad p)
                            inverted by a Jacobi-preconditioned Chebyshev polynomial (FP32);
                            2: as 1, with phi and mu preconditioned together by the
                            Cahn-Hilliard block: mu eliminated with the mass matrix and the
                            phi Schur complement approximated by (1/dt)(M + eps K) M^{-1}
                            (M + eps K), eps^2 = dt Cn/(2 Pe), two Chebyshev solves (FP32);
                            3: as 1, with the pressure Schur Laplacian inverted by one
                            geometric multigrid V-cycle on the octree's levels (each coarser
                            level caps the leaves one level shallower; Q1 prolongation, its
                            transpose as restriction, Jacobi-Chebyshev smoothing of degree
                            pc_degree, a degree-16 Chebyshev sweep on the coarsest level of at
                            most 300 nodes or level 1, FP32);
                            4: as 3, with the Cahn-Hilliard block of 2.  The hierarchy is built
                            (host work and device memory held by the mesh) on the first call
                            that asks for it. */
    int32_t pc_degree;   /* Chebyshev degree for pc_type 1/2 (whole apply) or 3/4 (smoother), in [2, 200] */
    double ew_eta0;      /* 0: fixed forcing term (krylov_rtol); in (0, 1): Eisenstat-Walker
                            forcing starting from this tolerance; anything else is CHNS_EINVAL.
                            The Newton step's first linear solve is then loose: at U^{k+1} = U^k
                            the residual is led by the pressure rows (the stabilisation term
                            carries the momentum imbalance before the time derivative has
                            responded), and the first Newton iteration is limited by the
                            nonlinearity rather than by the linear solve. */
    int32_t guess;       /* first Newton iterate of chns_newton_step: 0 = U_old (U_inout is
                            overwritten with it); 1 = U_inout as passed (the caller's guess,
                            e.g. the pressure p^{k-1}, which continues the previous step's
                            mid-point pressure: with p^0 = 0 the Crank-Nicolson pressure
                            p^{k+1} = 2 p~ - p^k alternates around p~, so U_old misses it).
                            The phi integral is still held at that of U_old; the pressure
                            mean is that of the first iterate.  Other values: CHNS_EINVAL. */
} chns_solver_opts;

#define CHNS_HIST 32

/* Statistics of one Newton step (filled also on CHNS_ENOCONV / ENAN / EBREAKDOWN);
 * res0 / res_final are row-equilibrated norms ||S R||_2. */
typedef struct {
    int32_t newton_its, krylov_its, jvp_calls, reason;
    double res0, res_final, du_norm;
    double jvp_ms;       /* device time of the J x launches (CUDA events on the stream) */
    double pc_ms;        /* device time of the preconditioner builds */
    double apply_ms;     /* device time of the preconditioner applications inside GMRES */
    double orth_ms;      /* device time of the Gram-Schmidt passes (dots, update, norms) */
    double res_hist[CHNS_HIST];     /* ||S R|| at Newton iterates 0 .. min(newton_its, CHNS_HIST - 1) */
    int32_t krylov_hist[CHNS_HIST]; /* GMRES iterations of linear solves 0 .. CHNS_HIST - 1 */
} chns_stats;

/* Build a mesh from a Morton-sorted, complete, 2:1 balanced leaf list (Section 4:
 * octant-to-node map, hanging-node virtualisation).  leaves: host array of n_leaves.
 * Domain: the cube [lo, hi]^dim.  Validates sortedness, completeness, alignment and
 * full (face/edge/vertex) 2:1 balance; enumerates independent nodes, element-to-
 * node map, hanging-node constraints (edge mid-point: 1/2 of 2 parents; face
 * centre: 1/4 of 4 parents) and the boundary nodes, then copies them to the
 * current CUDA device.  *out receives the mesh (library-owned; free with
 * chns_mesh_destroy).  Limits: 1 <= max_level <= 20. */
chns_status chns_mesh_create(int32_t dim, int32_t max_level, int64_t n_leaves,
                             const chns_leaf* leaves, double lo, double hi, chns_mesh** out);

/* Triquadratic (Q2) elements (Section 5.1 uses quadratic elements; NEXT-4) on the uniform
 * octree of one level: 3^d nodes per element on the lattice of half the element size, the
 * 3-point Gauss rule per axis, no hanging nodes.  Elements are in Morton order of their
 * anchors; nodes in Morton order of their integer coordinates, which are in units of
 * 2^-(level + 1) (chns_mesh_node_coords; the mesh's coordinate level is level + 1).  Element
 * node a = a_0 + 3 a_1 (+ 9 a_2) sits at 2 * anchor + a_k along axis k.  A Q2 mesh serves
 * chns_residual, chns_jvp (FP64 and FP32), chns_vjp and chns_mesh_set_velocity_bc; the
 * strong residuals then include the pure second derivatives (the full Hessian of phi, the
 * Laplacians of v and mu) that vanish on Q1.  Other calls return CHNS_EINVAL for it, and so
 * does pin_pressure = 1.  Limits: 1 <= level <= 8 (3D) or 11 (2D). */
chns_status chns_mesh_create_q2(int32_t dim, int32_t level, double lo, double hi, chns_mesh** out);
int32_t chns_mesh_order(const chns_mesh* mesh);   /* 1 (Q1) or 2 (Q2); -1 for NULL */

/* Free a mesh and its device memory (NULL is ignored). */
void chns_mesh_destroy(chns_mesh* mesh);

int64_t chns_mesh_num_nodes(const chns_mesh* mesh);     /* independent nodes N */
int64_t chns_mesh_num_elements(const chns_mesh* mesh);  /* leaves E */
int64_t chns_mesh_num_hanging(const chns_mesh* mesh);   /* distinct hanging points */
int32_t chns_mesh_dim(const chns_mesh* mesh);

/* Velocity boundary conditions of the mesh (Section 5 set-ups: the lid-driven cavity's
 * moving lid, the rising bubble's side walls with v_1 = 0 and d v_2 / d x = 0).
 * face_mask: host, 2 * dim bytes; face 2k is the face x_k = lo, face 2k + 1 the face
 * x_k = hi; bit c of a face's byte makes velocity component c a Dirichlet row on every
 * node of that face (a node on several faces takes the union); a component with no bit
 * keeps its weak-form row (natural condition).  values: device, N * dim doubles, the
 * prescribed g (read only where a Dirichlet row is set), copied into the mesh; NULL
 * means g = 0.  Replaces the default (all components of all boundary nodes, g = 0) for
 * every later call on the mesh.  With pin_pressure = 2 the prescribed velocities must
 * carry no net flux through the boundary (the pressure rows then still sum to zero). */
chns_status chns_mesh_set_velocity_bc(chns_mesh* mesh, const uint8_t* face_mask, const double* values);

/* Scatter strategy of the element kernels (residual, J x, J^T w) on this mesh: how element
 * rows are added into node rows (hanging corners folded into their parents).
 * mode 0: atomic adds (default); 1: element colouring -- elements are greedily coloured
 * (Morton order) so that no two elements of a colour share a node, one launch per colour
 * with plain adds: every node sums its contributions in a fixed order, so results are
 * bit-identical from run to run (the d/dCn scalar of chns_vjp still uses an atomic);
 * 2: warp-aggregated atomics (lanes of a warp that target one node add in shared memory
 * first; J^T w uses mode 0 there).  The colouring is built on the host at the first call
 * with mode 1.  CHNS_EINVAL for another mode. */
chns_status chns_mesh_set_scatter(chns_mesh* mesh, int32_t mode);
int32_t chns_mesh_num_colours(const chns_mesh* mesh);   /* 0 until mode 1 was set */

/* Copy the integer coordinates of the independent nodes (units of the finest
 * cell) to host memory coords[N * dim]. */
chns_status chns_mesh_node_coords(const chns_mesh* mesh, int32_t* coords);

/* Residual R(U^k, U^{k+1}) of Definition 2 with the Crank-Nicolson substitution of
 * Definition 1 (Section 3.3 end), FP64.  U_old = U^k, U_new = U^{k+1}, R: device
 * arrays of N * n_f doubles.  R is overwritten.  A non-positive tau radicand
 * produces non-finite entries (reported as CHNS_ETAU by chns_newton_step). */
chns_status chns_residual(const chns_mesh* mesh, const chns_params* params,
                          const double* U_old, const double* U_new, double* R, void* stream);

/* Newton Jacobian-vector product y = J x, J = dR/dU^{k+1} evaluated at
 * U^{k+1} = U_lin (Eq. newton_linear_system; analytic variations, Section 3.4),
 * computed by forward-mode differentiation of the element map.  precision 0: all
 * four arrays are double; precision 1: all four are float (FP32 arithmetic).
 * Dirichlet and pin rows of J are identity rows (y = x there).  y is overwritten. */
chns_status chns_jvp(const chns_mesh* mesh, const chns_params* params, const void* U_old,
                     const void* U_lin, const void* x, void* y, int32_t precision, void* stream);

/* Transpose product (reverse mode, FP64): gU_new = J^T w = w^T dR/dU^{k+1},
 * gU_old = w^T dR/dU^k, *gCn = w^T dR/dCn (a single device double), evaluated at
 * (U_old, U_lin).  All outputs are overwritten.  Any of gU_old / gCn may be NULL. */
chns_status chns_vjp(const chns_mesh* mesh, const chns_params* params, const double* U_old,
                     const double* U_lin, const double* w, double* gU_new, double* gU_old,
                     double* gCn, void* stream);

/* One implicit time step (Section 3.4): solve R(U_old, U) = 0 by inexact Newton from
 * U^{0} = U_old (U_inout is overwritten with U_old first), or from U_inout as passed
 * (opts->guess = 1), with matrix-free GMRES.  U_inout must not alias U_old.
 * With pin_pressure = 2, GMRES runs on J + u m_p^T / |Omega| (u = |diag J| on the
 * pressure rows, m_p the nodal masses): nonsingular, with the zero-mean-pressure
 * solution of J dU = -R.  U_old, U_inout: device, N * n_f doubles.  stats: host, may
 * be NULL.  Synchronises the stream (it reads scalars every GMRES iteration).  The
 * first call on a mesh allocates the Krylov workspace; the pressure-Schur apply is
 * captured into CUDA graphs on a private stream of the mesh and replayed on `stream`. */
chns_status chns_newton_step(const chns_mesh* mesh, const chns_params* params,
                             const chns_solver_opts* opts, const double* U_old, double* U_inout,
                             chns_stats* stats, void* stream);

/* Integral of phi over the domain (mass, Proposition 1), FP64, to host *out. */
chns_status chns_mass(const chns_mesh* mesh, const double* U, double* out, void* stream);

/* Parts of E_tot (Eq. energy_functional) at one time level, FP64, to host out[3]:
 * out[0] = 1/2 int rho(phi*) |v|^2, out[1] = 1/(Cn We) int psi(phi) + Cn^2/2 |grad phi|^2,
 * out[2] = 1/Fr int rho(phi*) x_{d-1} (0 without gravity). */
chns_status chns_energy(const chns_mesh* mesh, const chns_params* params, const double* U,
                        double* out, void* stream);

/* Consistent initial chemical potential: overwrite the mu field of U_inout (device)
 * with the solution of M mu = (N, psi'(phi)) + Cn^2 (grad N, grad phi), the potential
 * equation at one time level (Definition 1), by Jacobi-preconditioned CG to a
 * relative residual of 1e-14.  Synchronises the stream. */
chns_status chns_initial_mu(const chns_mesh* mesh, const chns_params* params, double* U_inout,
                            void* stream);

/* Reverse mode through one implicit step (the Newton solve of Section 3.4, Eq.
 * newton_linear_system, transposed): for a cotangent g of U^{k+1} = U_new solving
 * R(U_old, U_new; Cn) = 0, solve J^T lambda = P^T g by GMRES with the FP64 J^T w kernel
 * and the transposed nodal block-Jacobi (J = dR/dU^{k+1} at (U_old, U_new); P is the
 * pressure-level normalisation of pin mode 2), then write the cotangents
 * gU_old = -(dR/dU^k)^T lambda (+ the normalisation's share on p^k) and
 * *gCn = -(dR/dCn)^T lambda.  opts: restart, max_krylov, krylov_rtol and pc_type / pc_degree
 * are used, ew_eta0 is not (one linear solve) (pc_type >= 1 adds the pressure Schur approximation of the Newton step to the
 * transposed block-Jacobi -- it is symmetric -- as a Chebyshev polynomial (1, 2) or a
 * multigrid V-cycle (3, 4); the Cahn-Hilliard block of 2 / 4 is not used here).
 * U_old, U_new, g, lambda, gU_old: device N * n_f doubles; gCn: device double or NULL.
 * Synchronises the stream; CHNS_ENOCONV if GMRES stops short of krylov_rtol. */
chns_status chns_step_adjoint(const chns_mesh* mesh, const chns_params* params, const chns_solver_opts* opts,
                              const double* U_old, const double* U_new, const double* g, double* lambda,
                              double* gU_old, double* gCn, chns_stats* stats, void* stream);

/* Gradient of the free-energy part of E_tot (Eq. energy_functional) at one time level,
 * F = 1/(Cn We) int psi(phi) + Cn/(2 We) int |grad phi|^2: g (device, N * n_f, only the
 * phi field non-zero) = dF/dU, *dCn (host) = dF/dCn.  Synchronises the stream. */
chns_status chns_free_energy_grad(const chns_mesh* mesh, const chns_params* params, const double* U, double* g,
                                  double* dCn, void* stream);

/* Reverse mode of the potential right-hand side b(phi; Cn) = (N, psi'(phi)) +
 * Cn^2 (grad N, grad phi) that defines mu0 (chns_initial_mu): g_phi (device, N) =
 * (db/dphi)^T lam = (N, psi''(phi) lam) + Cn^2 (grad N, grad lam), *dCn (host) =
 * lam^T db/dCn.  U: device N * n_f (phi read), lam: device N.  Synchronises. */
chns_status chns_mu_rhs_vjp(const chns_mesh* mesh, const chns_params* params, const double* U, const double* lam,
                            double* g_phi, double* dCn, void* stream);

/* x = M^{-1} rhs with the consistent Q1 mass matrix (CG to 1e-14; M is symmetric, so
 * this is also its adjoint).  rhs, x: device N doubles.  Synchronises the stream. */
chns_status chns_mass_solve(const chns_mesh* mesh, const double* rhs, double* x, void* stream);

/* Integral of phi (as chns_mass) for callers that cannot allocate device memory when
 * they need it -- e.g. code running while a framework's caching allocator owns the free
 * device memory, or on a path where cudaMalloc's implicit device synchronisation is not
 * allowed.  The paper has no counterpart; it is a deployment variant of chns_mass.
 * It allocates nothing: its reduction scratch is a file-scope device array of 16,384
 * doubles (128 KiB, held by every GPU that loads the library until the process exits),
 * so meshes of more than 67,108,864 elements are rejected with CHNS_EINVAL, and so is a
 * call made while another device than the mesh's (the one current at chns_mesh_create)
 * is current, because the scratch address is the current device's.  U: device,
 * N * n_f doubles; out: one device double, written asynchronously on `stream` (no
 * host synchronisation).  The first call on a device resolves the scratch address for
 * that device (cudaGetSymbolAddress), so make it before any stream capture.  All calls
 * share the one scratch array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller. */
chns_status chns_mass_static(const chns_mesh* mesh, const double* U, double* out, void* stream);

/* Transfer between the Q1 spaces of two meshes of the same domain and dimension (Section 4:
 * parent-child interpolation on the octree, used for remeshing and by the multigrid
 * preconditioner).  P maps a field on `src` to the independent nodes of `dst`: each node
 * of dst takes the value of src's Q1 interpolant (hanging constraints of src included)
 * at its position, so P is exact when dst refines src and is injection when dst coarsens
 * src.  Built on the host from the meshes' leaf data; its rows and those of P^T are held
 * on the current device.  Free with chns_transfer_destroy. */
typedef struct chns_transfer chns_transfer;
chns_status chns_transfer_create(const chns_mesh* src, const chns_mesh* dst, chns_transfer** out);
void chns_transfer_destroy(chns_transfer* t);
int64_t chns_transfer_nnz(const chns_transfer* t);   /* stored weights of P (-1 for NULL) */
/* transpose = 0: out (dst nodes x nf) = P in (src nodes x nf); transpose = 1: out (src nodes
 * x nf) = P^T in (dst nodes x nf).  Node-major interleaved FP64 device vectors, nf in
 * [1, 16]; out is overwritten; asynchronous on `stream`. */
chns_status chns_transfer_apply(const chns_transfer* t, int32_t nf, int32_t transpose, const double* in,
                                double* out, void* stream);

/* Remeshing (Section 4, re-meshing and interpolation), one adaptation pass in three calls:
 * chns_adapt_flags (device) marks every element of `mesh`: +1 (refine) where some corner
 * value of phi (field d + 1 of U, hanging corners by their constraint means) has
 * |phi| < phi_threshold and the element's level is below max_level; -1 (coarsening
 * candidate) where every corner has |phi| >= phi_threshold and the level is above
 * min_level; 0 otherwise.  U: device, N * n_f doubles; flags: device, E int8 (overwritten);
 * asynchronous on `stream`. */
chns_status chns_adapt_flags(const chns_mesh* mesh, const double* U, double phi_threshold, int32_t min_level,
                             int32_t max_level, int8_t* flags, void* stream);

/* chns_adapt_leaves (host only): the new leaf list.  Complete families of 2^d sibling
 * leaves (consecutive in Morton order) whose members are all flagged -1 and deeper than
 * min_level become their parent; leaves flagged +1 below max_level_new split into their
 * 2^d children; then every leaf that touches (face, edge or vertex) a leaf more than one
 * level deeper is split until the tree is 2:1 balanced (refinement only).  leaves/flags:
 * host, n_leaves each, Morton-sorted, anchors in units of 2^-max_level.  out: host room for
 * `capacity` leaves, Morton-sorted, anchors in units of 2^-(*out_max_level) (the deepest
 * output level, at least 1).  *n_out receives the count; when it exceeds capacity nothing
 * is written to out and CHNS_EINVAL is returned (call again with room for *n_out).
 * The fields follow with chns_transfer_create(old mesh, new mesh) / chns_transfer_apply. */
chns_status chns_adapt_leaves(int32_t dim, int32_t max_level, int64_t n_leaves, const chns_leaf* leaves,
                              const int8_t* flags, int32_t min_level, int32_t max_level_new, chns_leaf* out,
                              int64_t capacity, int64_t* n_out, int32_t* out_max_level);

/* Host-only (no device work): the leaf list with every leaf deeper than `cap` replaced by
 * its ancestor at level `cap` (Morton order kept, duplicates merged), as the multigrid
 * hierarchy builds its coarse levels.  leaves: n_leaves Morton-sorted leaves with anchors in
 * units of 2^-max_level; out (host, room for n_leaves): the capped leaves with anchors in
 * units of 2^-cap; fmap (host, n_leaves, may be NULL): the output leaf of every input leaf;
 * *n_out: the output count.  A complete 2:1-balanced input gives a complete 2:1-balanced
 * output. */
chns_status chns_coarsen_leaves(int32_t dim, int32_t max_level, int64_t n_leaves, const chns_leaf* leaves,
                                int32_t cap, chns_leaf* out, int32_t* fmap, int64_t* n_out);

/* Measured CUDA-core FMA throughput of the current device, the ALU roofline of the
 * element kernels (a measurement aid; the paper has no counterpart): precision 1 = FP32
 * FFMA, 0 = FP64 DFMA.  Runs 8 independent fma chains per thread, 16-fold unrolled,
 * `iters` times, on 4 blocks of 256 threads per SM, once untimed and once between two CUDA
 * events on `stream`; *flops_per_s (host) = 2 flops per FMA / elapsed time.  scratch:
 * device buffer of at least 4 * SMs * 256 * (8 for FP64, 4 for FP32) bytes (receives the
 * chains' sums); CHNS_EINVAL if it is smaller.  Synchronises the stream. */
chns_status chns_fma_peak(int32_t precision, int32_t iters, void* scratch, int64_t scratch_bytes,
                          double* flops_per_s, void* stream);

/* Number of CUDA kernels this library has launched in this process (all meshes and
 * threads), for launch accounting by callers; kernels replayed from the library's CUDA
 * graphs count once per replay. */
int64_t chns_kernel_launches(void);

/* Message of the last error on this thread ("" if none). */
const char* chns_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHNS_H */
