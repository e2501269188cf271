"""Plain FP64 CPU oracle of the matrix-free CHNS hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.  It shares
no code with the CUDA path.

What it computes (paper: Section 3, Definition 1 with the averages of Eqs. for
the Crank-Nicolson mid-point, Definition 2 for the variational multiscale form,
the stabilisation parameters and strong residuals printed after Definition 2,
Section 3.4 for Newton):

  * ``residual``  R(U^k, U^{k+1}) of the fully discrete VMS weak form with the time
    derivative replaced by the Crank-Nicolson difference quotient; every spatial
    term is evaluated at the mid-point averages, except the Galerkin
    solenoidality term, which acts on v^{k+1} (Definition 1).
  * ``jvp``       J x with J = dR/dU^{k+1} (torch forward-mode autodiff).
  * ``vjp``       w^T dR/dU^{k+1}, w^T dR/dU^k, w^T dR/dCn (torch reverse mode).
  * ``jacobian``  the assembled dense J (small meshes).
  * ``newton_step`` Newton with a direct solve (Section 3.4).
  * ``mass``, ``energy``, ``initial_mu``.

Readings of the paper taken here (each also listed in the design notes):
  * Fields per node, in order: v_1..v_d, p, phi, mu.  rho_+ = eta_+ = 1 for the
    phi = +1 phase, rho_- = 1/rho_ratio, eta_- = 1/eta_ratio.
  * Mobility term of the Cahn-Hilliard row carries "+" (integration by parts of
    the strong form; Definition 1), not the "-" printed in Definition 2.
  * G_ij = sum_k d xi_k/dx_i d xi_k/dx_j for the map to [-1, 1]^d: (4/h^2) I.
  * phi* (the pull-back used only in rho and eta) is the clip to [-1, 1] of the
    nodal mid-point average at independent nodes, interpolated in the Q1 space
    ("its projection on the mesh").  Its derivative is 1 for |phi~| <= 1, else 0.
  * Second derivatives in the strong residuals are the exact element Hessians
    of the Q1 interpolants (the pure second derivatives vanish, mixed ones do not).
  * tau's are functions of the mid-point state and are differentiated exactly.
  * Quadrature: 2-point Gauss-Legendre per axis.
  * Gravity: g_hat = -e_{d-1} (last axis); Fr <= 0 means no gravity.
  * Dirichlet rows: by default every velocity component of every boundary node has
    the row R = v^{k+1} (no-slip); with ``bc`` chosen components of chosen faces have
    R = v^{k+1} - g and the others keep their weak-form rows (natural condition, as the
    bubble's side walls v_1 = 0, d v_2/dx = 0).  Pressure level (closed no-slip boxes leave p free up to a constant;
    the pressure rows sum to zero, so one of them is redundant): pin_pressure = 1
    replaces row p of node 0 by p^{k+1}_0 - p^k_0 (a point value: badly conditioned);
    pin_pressure = 2 keeps every row (J then has the constant pressure as its null
    vector) and Newton keeps int p^{k+1} = int p^k by removing the mean of each
    pressure update.
  * No subscale time derivative (quasi-static subscales, as in Definition 2).

Pins (tests/test_oracle_pins.py, tests/test_oracle_vms_pin.py) fix the Galerkin
terms (manufactured solution), the invariants (mass row-sum, pressure row-sum,
hydrostatic zero), tau_m, tau_phi and the stabilisation terms of the pressure and phi
rows (hand-evaluated spot values), and every term of Definition 2 -- the subgrid
momentum terms and tau_c included -- at an interior node, against a term-by-term
sympy evaluation of the printed weak form for a Q1 state in which every term is
non-zero.  The derivatives (jvp, vjp, jacobian) are pinned by central finite
differences and the adjoint identity; mass, energy and initial_mu by closed forms.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

DT = torch.float64


def _signs(dim):
    return np.array([[2 * ((a >> k) & 1) - 1 for k in range(dim)] for a in range(1 << dim)],
                    dtype=np.float64)


def basis_tables(dim):
    """Q1 basis on [-1,1]^d at the 2^d Gauss points (+-1/sqrt(3)).
    Returns N[q,a], dN[q,a,k] = dN_a/dxi_k, d2N[q,a,k,l] = d2N_a/dxi_k dxi_l."""
    s = _signs(dim)                      # corner signs (a, k)
    xq = s / math.sqrt(3.0)              # Gauss points in the same bit order (q, k)
    nq = nc = 1 << dim
    one_d = 0.5 * (1.0 + s[None, :, :] * xq[:, None, :])      # (q, a, k)
    d_one_d = 0.5 * s[None, :, :] * np.ones((nq, 1, 1))        # (q, a, k)
    N = np.prod(one_d, axis=2)
    dN = np.zeros((nq, nc, dim))
    d2N = np.zeros((nq, nc, dim, dim))
    for k in range(dim):
        f = d_one_d[:, :, k].copy()
        for j in range(dim):
            if j != k:
                f = f * one_d[:, :, j]
        dN[:, :, k] = f
        for l in range(dim):
            if l == k:
                continue  # each 1D factor is linear: d2/dxi_k^2 == 0
            g = d_one_d[:, :, k] * d_one_d[:, :, l]
            for j in range(dim):
                if j != k and j != l:
                    g = g * one_d[:, :, j]
            d2N[:, :, k, l] = g
    return torch.tensor(N, dtype=DT), torch.tensor(dN, dtype=DT), torch.tensor(d2N, dtype=DT), xq


def basis_tables_q2(dim):
    """Q2 (tensor-product quadratic Lagrange) basis on [-1,1]^d at the 3^d Gauss points
    (0, +-sqrt(3/5); weights 8/9, 5/9).  Node a = a_0 + 3 a_1 (+ 9 a_2) sits at
    xi_k = a_k - 1; Gauss point q likewise.  1D: L_0 = xi(xi-1)/2, L_1 = 1 - xi^2,
    L_2 = xi(xi+1)/2.  Returns N[q,a], dN[q,a,k], d2N[q,a,k,l], the points (q, d) and the
    weights w_q (product of the 1D weights)."""
    g = math.sqrt(0.6)
    pts1 = np.array([-g, 0.0, g])
    w1 = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])
    L = lambda j, t: (t * (t - 1.0) / 2.0, 1.0 - t * t, t * (t + 1.0) / 2.0)[j]
    dL = lambda j, t: (t - 0.5, -2.0 * t, t + 0.5)[j]
    d2L = lambda j, t: (1.0, -2.0, 1.0)[j]
    n = 3 ** dim
    idx = np.array([[(a // 3 ** k) % 3 for k in range(dim)] for a in range(n)])
    N = np.zeros((n, n))
    dN = np.zeros((n, n, dim))
    d2N = np.zeros((n, n, dim, dim))
    xq = pts1[idx]                                      # (q, d)
    wq = np.prod(w1[idx], axis=1)
    for q in range(n):
        t = xq[q]
        for a in range(n):
            f = [L(idx[a, k], t[k]) for k in range(dim)]
            df = [dL(idx[a, k], t[k]) for k in range(dim)]
            N[q, a] = np.prod(f)
            for k in range(dim):
                dN[q, a, k] = df[k] * np.prod([f[j] for j in range(dim) if j != k])
                for l in range(dim):
                    if l == k:
                        d2N[q, a, k, k] = d2L(idx[a, k], t[k]) * np.prod([f[j] for j in range(dim) if j != k])
                    else:
                        d2N[q, a, k, l] = df[k] * df[l] * np.prod([f[j] for j in range(dim) if j not in (k, l)])
    return (torch.tensor(N, dtype=DT), torch.tensor(dN, dtype=DT), torch.tensor(d2N, dtype=DT), xq,
            torch.tensor(wq, dtype=DT))


class Params:
    """Physical and numerical parameters of one time step."""

    def __init__(self, dim, Re, We, Pe, Cn, Fr, rho_ratio, eta_ratio, dt, C_I=6.0, C_phi=6.0,
                 pin_pressure=2, **_ignored):
        self.dim = int(dim)
        self.Re, self.We, self.Pe, self.Cn, self.Fr = float(Re), float(We), float(Pe), float(Cn), float(Fr)
        self.rho_ratio, self.eta_ratio = float(rho_ratio), float(eta_ratio)
        self.dt, self.C_I, self.C_phi = float(dt), float(C_I), float(C_phi)
        self.pin_pressure = int(pin_pressure)
        # Eq. (alpha_beta_defn) and the viscosity analogue, with rho_+ = eta_+ = 1
        rho_p, rho_m = 1.0, 1.0 / self.rho_ratio
        eta_p, eta_m = 1.0, 1.0 / self.eta_ratio
        self.rho_plus, self.rho_minus = rho_p, rho_m
        self.alpha = (rho_p - rho_m) / (2.0 * rho_p)
        self.beta = (rho_p + rho_m) / (2.0 * rho_p)
        self.gamma = (eta_p - eta_m) / (2.0 * eta_p)
        self.xi = (eta_p + eta_m) / (2.0 * eta_p)


class Oracle:
    """Element loops over a ``oracle.mesh.Mesh`` written with whole-array torch ops."""

    def __init__(self, mesh, elements=None, bc=None):
        """``elements`` (optional index array) restricts every element loop to a subset:
        rows of nodes whose whole support lies in the subset are then exact, which lets
        large meshes be checked on sampled nodes.  ``bc`` (optional) = (face_mask, g): the
        velocity Dirichlet rows per face and component (face 2k: x_k = lo, 2k + 1: x_k = hi,
        bit c: component c) and the prescribed values g (N, d) (None: zero); default: every
        component on every boundary node, g = 0 (no-slip)."""
        self.m = mesh
        d = mesh.dim
        self.d, self.nc, self.nf = d, mesh.nc, mesh.nf
        self.order = getattr(mesh, "order", 1)
        if self.order == 2:
            self.N, self.dN, self.d2N, self.xq_ref, self.wq = basis_tables_q2(d)
        else:
            self.N, self.dN, self.d2N, self.xq_ref = basis_tables(d)
            self.wq = None                                # unit Gauss weights
        sel = slice(None) if elements is None else np.asarray(elements)
        self.P = torch.tensor(mesh.parents[sel], dtype=torch.int64)
        self.W = torch.tensor(mesh.weights[sel], dtype=DT)
        self.h = torch.tensor(mesh.h[sel], dtype=DT)
        self.bnd = torch.tensor(np.nonzero(mesh.boundary)[0], dtype=torch.int64)
        d = mesh.dim
        n_side = 1 << mesh.max_level
        if bc is None:
            dmask = np.repeat(mesh.boundary[:, None], d, axis=1)
            g = np.zeros((mesh.N, d))
        else:
            face_mask, g = bc
            dmask = np.zeros((mesh.N, d), dtype=bool)
            for k in range(d):
                for side, at in ((0, 0), (1, n_side)):
                    on = mesh.nodes[:, k] == at
                    for c in range(d):
                        if (int(face_mask[2 * k + side]) >> c) & 1:
                            dmask[on, c] = True
            g = np.zeros((mesh.N, d)) if g is None else np.asarray(g, dtype=np.float64)
        self.dmask = torch.tensor(dmask)
        self.bc_g = torch.tensor(g, dtype=DT)
        # physical quadrature points (E, q, d)
        cx = torch.tensor(mesh.corner_x[sel], dtype=DT)
        self.xq = torch.einsum("qa,ead->eqd", self.N, cx)
        self.detJ = (0.5 * self.h) ** d           # times unit Gauss weights
        # integral of each independent node's basis function (hanging weights included)
        loc = self._wq(self.N).sum(0).reshape(1, -1) * self.detJ.reshape(-1, 1)        # (E, nc)
        self.node_mass = self.scatter(loc, mesh.N)
        self.volume = (mesh.hi - mesh.lo) ** d

    def _wq(self, a, axis=0):
        """a times the Gauss weights along its Gauss-point axis (Q1: unit weights, a unchanged)."""
        if self.wq is None:
            return a
        shape = [1] * a.dim()
        shape[axis] = -1
        return a * self.wq.reshape(shape)

    # -- gather / scatter with hanging-node constraints (Section 4) -------------
    def gather(self, U):
        """Element-corner values (E, nc, ...) of nodal data U (N, ...)."""
        vals = U[self.P]                                   # (E, nc, 4, ...)
        w = self.W.reshape(self.W.shape + (1,) * (U.dim() - 1))
        return (w * vals).sum(dim=2)

    def scatter(self, r_local, nnodes):
        """Transpose of ``gather``: sum element-corner contributions to nodes."""
        tail = r_local.shape[2:]
        w = self.W.reshape(self.W.shape + (1,) * len(tail))
        contrib = w * r_local.unsqueeze(2)                 # (E, nc, 4, ...)
        out = torch.zeros((nnodes,) + tuple(tail), dtype=DT)
        out.index_add_(0, self.P.reshape(-1), contrib.reshape((-1,) + tuple(tail)))
        return out

    # -- interpolation at quadrature points --------------------------------------
    def interp(self, ul):
        """Value, physical gradient and Hessian at the Gauss points of element-corner
        data ul (E, nc, ...): shapes (E, q, ...), (E, q, ..., d), (E, q, ..., d, d)."""
        h = self.h
        extra = ul.dim() - 2
        hs = h.reshape((-1, 1) + (1,) * extra)
        val = torch.einsum("qa,ea...->eq...", self.N, ul)
        grad = torch.einsum("qak,ea...->eq...k", self.dN, ul) * (2.0 / hs).unsqueeze(-1)
        hess = torch.einsum("qakl,ea...->eq...kl", self.d2N, ul) * (4.0 / hs ** 2).unsqueeze(-1).unsqueeze(-1)
        return val, grad, hess

    # -- the residual ------------------------------------------------------------
    def residual(self, prm, U_old, U_new, Cn=None, forcing=None, t_mid=None, check=True):
        """Residual R (N, nf) of Definition 2 with the time scheme of Definition 1.

        ``Cn`` may be a 0-d tensor (for d/dCn).  ``forcing`` (optional, for
        manufactured solutions) is a callable (xq, t) -> (f_mom (.., d), f_mu, f_phi)
        of body terms moved to the right-hand side of the momentum, potential and
        Cahn-Hilliard rows; they also enter the strong residuals."""
        d = self.d
        iv, ip, iphi, imu = slice(0, d), d, d + 1, d + 2
        if Cn is None:
            Cn = torch.tensor(prm.Cn, dtype=DT)
        Re, We, Pe, Fr, dt = prm.Re, prm.We, prm.Pe, prm.Fr, prm.dt
        al, be, ga, xi = prm.alpha, prm.beta, prm.gamma, prm.xi

        # time averages of Eq. (averaging1) at nodes, then element gathers
        Ut = 0.5 * (U_old + U_new)
        ut = self.gather(Ut)
        un = self.gather(U_new)
        uo = self.gather(U_old)
        # pull-back phi* (Remark on saturation): clip at independent nodes, Q1 projection
        phistar_nodes = torch.clamp(Ut[:, iphi], -1.0, 1.0)
        ps_l = self.gather(phistar_nodes)

        val_t, grad_t, hess_t = self.interp(ut)            # tilde fields
        val_n, grad_n, _ = self.interp(un)                 # level k+1
        val_o, _, _ = self.interp(uo)                      # level k
        ps, gps, _ = self.interp(ps_l)

        v = val_t[..., iv]                                 # (E,q,d)
        gv = grad_t[..., iv, :]                            # (E,q,i,j) = d_j v_i
        hv = hess_t[..., iv, :, :]                         # (E,q,i,k,l)
        p = val_t[..., ip]
        gp = grad_t[..., ip, :]
        phi = val_t[..., iphi]
        gphi = grad_t[..., iphi, :]
        hphi = hess_t[..., iphi, :, :]
        mu = val_t[..., imu]
        gmu = grad_t[..., imu, :]
        hmu = hess_t[..., imu, :, :]
        v_dt = (val_n[..., iv] - val_o[..., iv]) / dt
        phi_dt = (val_n[..., iphi] - val_o[..., iphi]) / dt
        div_vnew = torch.diagonal(grad_n[..., iv, :], dim1=-2, dim2=-1).sum(-1)

        rho = al * ps + be                                  # rho(phi*)
        eta = ga * ps + xi                                  # eta(phi*)
        geta = ga * gps                                     # grad eta(phi*)
        Jv = ((prm.rho_minus - prm.rho_plus) / (2.0 * prm.rho_plus * Cn)) * gmu   # thermo consistency
        psi_p = phi ** 3 - phi                              # Eq. (free_energy)

        # metric tensor of the map to [-1,1]^d
        hq = self.h.reshape(-1, 1)
        G = (4.0 / hq ** 2).unsqueeze(-1).unsqueeze(-1) * torch.eye(d, dtype=DT)    # (E,1,d,d)
        vGv = torch.einsum("eqi,eqij,eqj->eq", v, G.expand(-1, v.shape[1], -1, -1), v)
        vGJ = torch.einsum("eqi,eqij,eqj->eq", v, G.expand(-1, v.shape[1], -1, -1), Jv)
        GG = (G * G).sum((-1, -2))                          # (E,1)
        trG = torch.diagonal(G, dim1=-2, dim2=-1).sum(-1)   # (E,1)

        # gravity, g_hat = -e_{d-1}
        ghat = torch.zeros(d, dtype=DT)
        ghat[d - 1] = -1.0
        inv_Fr = (1.0 / Fr) if Fr > 0 else 0.0

        f_mom = f_mu = f_phi = 0.0
        if forcing is not None:
            f_mom, f_mu, f_phi = forcing(self.xq, t_mid)

        # strong residuals (printed after Definition 2), at the mid-point
        conv = torch.einsum("eqj,eqij->eqi", v, gv)               # v_j d_j v_i
        Jgv = torch.einsum("eqj,eqij->eqi", Jv, gv)               # J_j d_j v_i
        lap_phi = torch.diagonal(hphi, dim1=-2, dim2=-1).sum(-1)
        cap = torch.einsum("eqij,eqj->eqi", hphi, gphi) + gphi * lap_phi.unsqueeze(-1)  # d_j(d_i phi d_j phi)
        lap_v = torch.diagonal(hv, dim1=-2, dim2=-1).sum(-1)      # (E,q,i)
        visc = torch.einsum("eqk,eqik->eqi", geta, gv) + eta.unsqueeze(-1) * lap_v       # d_k(eta d_k v_i)
        grav = -rho.unsqueeze(-1) * ghat * inv_Fr                 # -rho g_i / Fr
        Rm = (rho.unsqueeze(-1) * v_dt + rho.unsqueeze(-1) * conv + Jgv / Pe + (Cn / We) * cap
              + gp / We - visc / Re + grav - f_mom)
        Rc = torch.diagonal(gv, dim1=-2, dim2=-1).sum(-1)
        lap_mu = torch.diagonal(hmu, dim1=-2, dim2=-1).sum(-1)
        Rphi = phi_dt + (phi * Rc + (v * gphi).sum(-1)) - lap_mu / (Pe * Cn) - f_phi

        # stabilisation parameters
        rad_m = 4.0 / dt ** 2 + vGv + vGJ / (rho * Pe) + prm.C_I * (eta / (rho * Re)) ** 2 * GG
        if check and torch.any(rad_m <= 0):
            raise FloatingPointError("tau_m radicand is not positive")
        tau_m = rad_m ** -0.5
        tau_c = 1.0 / (trG * tau_m)
        tau_phi = (4.0 / dt ** 2 + vGv + prm.C_phi * (1.0 / (Pe * Cn)) ** 2 * GG) ** -0.5

        nq = v.shape[1]
        E = v.shape[0]
        f0 = torch.zeros((E, nq, self.nf), dtype=DT)
        f1 = torch.zeros((E, nq, self.nf, d), dtype=DT)
        rho_ = rho.unsqueeze(-1)
        tm = tau_m.unsqueeze(-1)
        eye = torch.eye(d, dtype=DT)
        # momentum (test w_i): value part
        f0_mom = (rho_ * v_dt + rho_ * conv - tm * torch.einsum("eqj,eqij->eqi", Rm, gv)
                  + Jgv / Pe + grav - f_mom)
        # momentum: gradient part, index [i, j] multiplies d_j w_i
        f1_mom = (tm.unsqueeze(-1) * torch.einsum("eqj,eqi->eqij", v, Rm)
                  - (tau_m ** 2 / rho).unsqueeze(-1).unsqueeze(-1) * torch.einsum("eqj,eqi->eqij", Rm, Rm)
                  + (1.0 / Pe) * (tau_m / rho).unsqueeze(-1).unsqueeze(-1) * torch.einsum("eqj,eqi->eqij", Jv, Rm)
                  - (Cn / We) * torch.einsum("eqi,eqj->eqij", gphi, gphi)
                  - (p / We).unsqueeze(-1).unsqueeze(-1) * eye
                  + (rho * tau_c * Rc / We).unsqueeze(-1).unsqueeze(-1) * eye
                  + (1.0 / Re) * eta.unsqueeze(-1).unsqueeze(-1) * gv)
        f0[..., iv] = f0_mom
        f1[..., iv, :] = f1_mom
        # solenoidality (test q) with the PSPG-type term
        f0[..., ip] = div_vnew
        f1[..., ip, :] = (tau_m / rho).unsqueeze(-1) * Rm
        # Cahn-Hilliard (test q)
        f0[..., iphi] = phi_dt - f_phi
        f1[..., iphi, :] = (-v * phi.unsqueeze(-1)
                            + (tau_m / rho * phi).unsqueeze(-1) * Rm
                            + v * (tau_phi * Rphi).unsqueeze(-1)
                            + gmu / (Pe * Cn))
        # chemical potential (test q)
        f0[..., imu] = -mu + psi_p - f_mu
        f1[..., imu, :] = Cn ** 2 * gphi

        # test-function contraction: N_a f0 + dN_a/dx . f1, times |det J| w_q
        dNx = self.dN.unsqueeze(0) * (2.0 / self.h).reshape(-1, 1, 1, 1)    # (E,q,a,k)
        f0, f1 = self._wq(f0, 1), self._wq(f1, 1)
        r_loc = (torch.einsum("qa,eqf->eaf", self.N, f0)
                 + torch.einsum("eqak,eqfk->eaf", dNx, f1)) * self.detJ.reshape(-1, 1, 1)
        R = self.scatter(r_loc, U_new.shape[0])
        # Dirichlet rows (no-slip) and optional pressure pin
        R = R.clone()
        Rv = R[:, iv]
        R[:, iv] = torch.where(self.dmask, U_new[:, iv] - self.bc_g, Rv)
        if prm.pin_pressure == 1:
            R[0, ip] = U_new[0, ip] - U_old[0, ip]
        return R

    # -- derivatives (torch autodiff) --------------------------------------------
    def jvp(self, prm, U_old, U_lin, x, check=True):
        """J x, J = dR/dU^{k+1} at U^{k+1} = U_lin."""
        _, t = torch.func.jvp(lambda U: self.residual(prm, U_old, U, check=check), (U_lin,), (x,))
        return t

    def vjp(self, prm, U_old, U_lin, w):
        """(w^T dR/dU^{k+1}, w^T dR/dU^k, w^T dR/dCn) at (U_old, U_lin)."""
        Uo = U_old.clone().requires_grad_(True)
        Un = U_lin.clone().requires_grad_(True)
        Cn = torch.tensor(prm.Cn, dtype=DT, requires_grad=True)
        R = self.residual(prm, Uo, Un, Cn=Cn)
        gn, go, gc = torch.autograd.grad(R, (Un, Uo, Cn), grad_outputs=w)
        return gn, go, gc

    def jacobian(self, prm, U_old, U_lin, chunk=256):
        """Dense dR/dU^{k+1} (n_dof x n_dof), row/column index = node * nf + field."""
        n = U_lin.numel()
        J = torch.zeros((n, n), dtype=DT)
        self.residual(prm, U_old, U_lin)                   # raises if a tau radicand is <= 0
        f = lambda t: self.jvp(prm, U_old, U_lin, t.reshape(U_lin.shape), check=False).reshape(-1)
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            eye = torch.zeros((c1 - c0, n), dtype=DT)
            eye[torch.arange(c1 - c0), torch.arange(c0, c1)] = 1.0
            cols = torch.func.vmap(f)(eye)                 # (chunk, n)
            J[:, c0:c1] = cols.T
        return J

    def node_pairs(self):
        """All (row node, column node) pairs that share an element (with constraints)."""
        P = self.m.parents
        W = self.m.weights
        E, nc, _ = P.shape
        nodes = np.where(W > 0, P, -1).reshape(E, nc * 4)
        rows, cols = [], []
        for i in range(nc * 4):
            for j in range(nc * 4):
                ok = (nodes[:, i] >= 0) & (nodes[:, j] >= 0)
                rows.append(nodes[ok, i])
                cols.append(nodes[ok, j])
        pairs = np.unique(np.stack([np.concatenate(rows), np.concatenate(cols)], 1), axis=0)
        return pairs

    def node_colours(self, pairs):
        """Greedy distance-2 colouring of the node graph (edges = pairs): two nodes of the
        same colour never appear in one row of J."""
        n = self.m.N
        nbr = [[] for _ in range(n)]
        for a, b in pairs:
            nbr[a].append(b)
        colour = -np.ones(n, dtype=np.int64)
        for v in range(n):
            used = set()
            for u in nbr[v]:
                for w in nbr[u]:
                    if colour[w] >= 0:
                        used.add(colour[w])
            c = 0
            while c in used:
                c += 1
            colour[v] = c
        return colour

    def jacobian_sparse(self, prm, U_old, U_lin):
        """dR/dU^{k+1} as a scipy CSR matrix, recovered exactly from J x products with
        one probe per (node colour, field): columns of same-coloured nodes never share
        a row (Curtis-Powell-Reid)."""
        if not hasattr(self, "_pairs"):
            self._pairs = self.node_pairs()
            self._colour = self.node_colours(self._pairs)
        pairs, colour = self._pairs, self._colour
        nf = self.nf
        ncol = int(colour.max()) + 1
        probes = torch.zeros((ncol * nf,) + tuple(U_lin.shape), dtype=DT)
        for c in range(ncol):
            idx = torch.tensor(np.nonzero(colour == c)[0])
            for f in range(nf):
                probes[c * nf + f, idx, f] = 1.0
        self.residual(prm, U_old, U_lin)                   # raises if a tau radicand is <= 0
        Y = torch.func.vmap(lambda t: self.jvp(prm, U_old, U_lin, t, check=False))(probes)
        Y = Y.reshape(ncol, nf, -1, nf).numpy()            # (colour, col field, row node, row field)
        m_, n_ = pairs[:, 0], pairs[:, 1]
        rows, cols, vals = [], [], []
        for f in range(nf):
            for g in range(nf):
                rows.append(m_ * nf + g)
                cols.append(n_ * nf + f)
                vals.append(Y[colour[n_], f, m_, g])
        ndof = U_lin.numel()
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
        J = sp.csr_matrix((vals, (rows, cols)), shape=(ndof, ndof))
        J.eliminate_zeros()
        return J

    # -- Newton (Section 3.4) with a direct solve -----------------------------
    def newton_step(self, prm, U_old, rtol=1e-12, atol=1e-14, max_it=20, U0=None, forcing=None,
                    t_mid=None):
        """Solve R(U_old, U) = 0 from U^{0} = U_old: U <- U - J^{-1} R (sparse LU) until
        ||R||/||R(U^0)|| <= rtol or ||R|| <= atol.  Returns (U, history)."""
        U = (U_old if U0 is None else U0).clone()
        res = lambda V: self.residual(prm, U_old, V, forcing=forcing, t_mid=t_mid)
        R = res(U)
        r0 = float(torch.linalg.norm(R))
        hist = [r0]
        for _ in range(max_it):
            if hist[-1] <= atol or hist[-1] <= rtol * r0:
                break
            J = self.jacobian_sparse(prm, U_old, U)
            if prm.pin_pressure == 2:
                # bordered system: J dU + c lam = -R, c^T dU = 0 with c the pressure mean
                n = U.numel()
                c = np.zeros(n)
                c[self.d::self.nf] = self.node_mass.numpy() / self.volume
                K = sp.bmat([[J, sp.csr_matrix(c.reshape(-1, 1))], [sp.csr_matrix(c.reshape(1, -1)), None]])
                rhs = np.concatenate([-R.reshape(-1).numpy(), [0.0]])
                dU = spla.spsolve(K.tocsc(), rhs)[:n]
            else:
                dU = spla.spsolve(J.tocsc(), -R.reshape(-1).numpy())
            U = U + torch.tensor(dU, dtype=DT).reshape(U.shape)
            R = res(U)
            hist.append(float(torch.linalg.norm(R)))
        return U, hist

    # -- integrals -------------------------------------------------------------
    def mass(self, U):
        """Integral of phi over the domain."""
        phi_l = self.gather(U[:, self.d + 1])
        val, _, _ = self.interp(phi_l)
        return float((self._wq(val, 1) * self.detJ.reshape(-1, 1)).sum())

    def energy(self, prm, U, Cn=None):
        """(kinetic, free, gravitational) parts of E_tot (Eq. energy_functional):
        1/2 int rho(phi*) |v|^2,  1/(Cn We) int psi(phi) + Cn^2/2 |grad phi|^2,
        1/Fr int rho(phi*) x_{d-1}  (0 without gravity)."""
        d = self.d
        if Cn is None:
            Cn = prm.Cn
        ul = self.gather(U)
        val, grad, _ = self.interp(ul)
        ps, _, _ = self.interp(self.gather(torch.clamp(U[:, d + 1], -1.0, 1.0)))
        rho = prm.alpha * ps + prm.beta
        w = self._wq(self.detJ.reshape(-1, 1).expand(-1, self.N.shape[0]), 1)
        v = val[..., :d]
        phi = val[..., d + 1]
        gphi = grad[..., d + 1, :]
        kin = 0.5 * (rho * (v * v).sum(-1) * w).sum()
        psi = 0.25 * (phi ** 2 - 1.0) ** 2
        free = ((psi + 0.5 * Cn ** 2 * (gphi * gphi).sum(-1)) * w).sum() / (Cn * prm.We)
        grav = (rho * self.xq[..., d - 1] * w).sum() / prm.Fr if prm.Fr > 0 else torch.tensor(0.0, dtype=DT)
        return float(kin), float(free), float(grav)

    def mass_matrix(self):
        """Consistent Q1 mass matrix on independent nodes (scipy CSR)."""
        Me = torch.einsum("qa,qb->ab", self._wq(self.N), self.N)          # reference
        rows, cols, vals = [], [], []
        P = self.m.parents
        W = self.m.weights
        detJ = self.detJ.numpy()
        nc = self.nc
        for a in range(nc):
            for b in range(nc):
                for pa in range(4):
                    for pb in range(4):
                        w = W[:, a, pa] * W[:, b, pb] * detJ * float(Me[a, b])
                        keep = w != 0
                        rows.append(P[keep, a, pa])
                        cols.append(P[keep, b, pb])
                        vals.append(w[keep])
        n = self.m.N
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n))

    def mu_rhs(self, phi, Cn):
        """b_a = (N_a, psi'(phi)) + Cn^2 (grad N_a, grad phi) (discrete potential row
        at a single time level)."""
        pl = self.gather(phi)
        val, grad, _ = self.interp(pl)
        dNx = self.dN.unsqueeze(0) * (2.0 / self.h).reshape(-1, 1, 1, 1)
        w = self._wq(self.detJ.reshape(-1, 1).expand(-1, self.N.shape[0]), 1)
        r = (torch.einsum("qa,eq->ea", self.N, (val ** 3 - val) * w)
             + torch.einsum("eqak,eqk->ea", dNx, Cn ** 2 * grad * w.unsqueeze(-1)))
        return self.scatter(r, phi.shape[0])

    def initial_mu(self, prm, phi, Cn=None):
        """mu^0 from the discrete potential equation at one time level:
        M mu = (N, psi'(phi)) + Cn^2 K phi (direct sparse solve)."""
        if Cn is None:
            Cn = prm.Cn
        b = self.mu_rhs(phi, Cn).numpy()
        return torch.tensor(spla.spsolve(self.mass_matrix().tocsc(), b), dtype=DT)
