"""Pins of the CPU oracle against what the paper and the mathematics fix, without
the GPU.  Each test names the property it checks; together they are chosen so that
a dropped term, a wrong sign or a transposed index in the oracle fails one of them.
"""
import math

import numpy as np
import pytest
import sympy
import torch

import synth
from oracle import Mesh, Oracle, Params
from tests.helpers import drop_state, make_mesh, params

MESHES = [("uniform", 2, 3), ("adaptive", 2, 4), ("uniform", 3, 2), ("adaptive", 3, 3)]


def _ids(m):
    return f"{m[0]}{m[1]}d-L{m[2]}"


@pytest.mark.parametrize("case", MESHES, ids=_ids)
def test_patch_linear_fields_exact(case):
    """Hanging-node gather + Q1 interpolation reproduce any linear field and its
    gradient exactly at the Gauss points (Section 4, hanging-node virtualisation)."""
    _, m = make_mesh(*case)
    o = Oracle(m)
    d = m.dim
    a = np.array([0.3, -1.7, 0.9][:d])
    f = 0.25 + m.x @ a
    val, grad, hess = o.interp(o.gather(torch.tensor(f)))
    exact = 0.25 + o.xq.numpy() @ a
    assert np.abs(val.numpy() - exact).max() < 1e-13
    assert np.abs(grad.numpy() - a).max() < 1e-12
    assert np.abs(hess.numpy()).max() < 1e-10
    if case[0] == "adaptive":
        assert m.hanging.any()


@pytest.mark.parametrize("case", MESHES, ids=_ids)
def test_mass_row_sum_exact(case):
    """Sum over nodes of the Cahn-Hilliard rows equals (int phi^{k+1} - int phi^k)/dt
    for any state (test function q = 1; Proposition 1)."""
    _, m = make_mesh(*case)
    prm = params("drop3d" if m.dim == 3 else "drop2d")
    o, U, Un = drop_state(m, prm, perturb=1e-2)
    R = o.residual(prm, U, Un)
    lhs = float(R[:, m.dim + 1].sum())
    rhs = (o.mass(Un) - o.mass(U)) / prm.dt
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs))


@pytest.mark.parametrize("case", MESHES, ids=_ids)
def test_pressure_row_sum_zero(case):
    """Without the pin, the pressure rows sum to int div v^{k+1} = 0 when v^{k+1}
    vanishes on the boundary (partition of unity kills the stabilisation term)."""
    _, m = make_mesh(*case)
    prm = params("drop3d" if m.dim == 3 else "drop2d", pin_pressure=0)
    o, U, Un = drop_state(m, prm, perturb=1e-2)
    R = o.residual(prm, U, Un)
    scale = float(R[:, m.dim].abs().sum())
    assert abs(float(R[:, m.dim].sum())) <= 1e-12 * max(scale, 1.0)


def hydrostatic(m, prm, c=0.3):
    """v = 0, phi = c, mu = psi'(c), (1/We) grad p = rho(c) g_hat / Fr: a steady state
    of Eqs. (nav_stokes)-(phi_eqn) with psi of Eq. (free_energy)."""
    d = m.dim
    U = np.zeros((m.N, d + 3))
    rho_c = prm.alpha * c + prm.beta
    U[:, d] = -(prm.We * rho_c / prm.Fr) * m.x[:, d - 1] + 0.7
    U[:, d + 1] = c
    U[:, d + 2] = c ** 3 - c
    return torch.tensor(U)


@pytest.mark.parametrize("case", MESHES, ids=_ids)
@pytest.mark.parametrize("c", [0.3, -0.8])
def test_hydrostatic_state_is_exact_zero(case, c):
    """The hydrostatic state makes every row vanish to rounding, hanging nodes
    included: pins gravity, pressure, potential and the strong-residual assembly."""
    _, m = make_mesh(*case)
    prm = params("drop3d" if m.dim == 3 else "drop2d", Fr=1.0, rho_ratio=7.0, eta_ratio=3.0)
    o = Oracle(m)
    U = hydrostatic(m, prm, c)
    R = o.residual(prm, U, U)
    scale = prm.We * (prm.alpha * c + prm.beta) / prm.Fr * float(o.detJ.max()) / float(o.h.max())
    assert float(R.abs().max()) <= 1e-11 * max(scale, 1.0)


@pytest.mark.parametrize("case", MESHES, ids=_ids)
def test_potential_row_linear_patch(case):
    """At phi = 1/sqrt(3) (where psi'' = 0) the potential rows respond to a linear
    tangent in phi only through Cn^2 (grad q, grad phi), which vanishes at interior
    nodes for linear phi: a patch test of the gradient term through hanging nodes."""
    _, m = make_mesh(*case)
    d = m.dim
    prm = params("drop3d" if d == 3 else "drop2d")
    o = Oracle(m)
    U = torch.zeros((m.N, d + 3), dtype=torch.float64)
    U[:, d + 1] = 1.0 / math.sqrt(3.0)
    U[:, d + 2] = (1.0 / math.sqrt(3.0)) ** 3 - 1.0 / math.sqrt(3.0)
    x = torch.zeros_like(U)
    x[:, d + 1] = torch.tensor(m.x @ np.array([0.4, -1.1, 0.8][:d]))
    Jx = o.jvp(prm, U, U, x)
    interior = ~torch.tensor(m.boundary)
    ref = prm.Cn ** 2 * float(o.detJ.max()) / float(o.h.min()) ** 2
    assert float(Jx[interior, d + 2].abs().max()) <= 1e-10 * ref
    assert float(Jx[~interior, d + 2].abs().max()) > 1e-3 * ref     # boundary flux is not zero


@pytest.mark.parametrize("case", [("uniform", 2, 3), ("adaptive", 2, 3), ("uniform", 3, 2)], ids=_ids)
def test_jacobian_matches_central_differences(case):
    """J x (forward mode) against central differences with eps = 1e-6 on <= 64 elements."""
    _, m = make_mesh(*case)
    assert m.E <= 64
    prm = params("drop3d" if m.dim == 3 else "drop2d")
    o, U, Un = drop_state(m, prm, perturb=1e-2)
    x = torch.tensor(synth.random_vectors(U.numel(), 1, 5)[0]).reshape(U.shape)
    eps = 1e-6
    fd = (o.residual(prm, U, Un + eps * x) - o.residual(prm, U, Un - eps * x)) / (2 * eps)
    Jx = o.jvp(prm, U, Un, x)
    assert float((fd - Jx).norm() / Jx.norm()) < 1e-7
    # U^k and Cn derivatives of the reverse mode against differences too
    w = torch.tensor(synth.random_vectors(U.numel(), 1, 6)[0]).reshape(U.shape)
    gn, go, gc = o.vjp(prm, U, Un, w)
    fdo = (o.residual(prm, U + eps * x, Un) - o.residual(prm, U - eps * x, Un)) / (2 * eps)
    assert abs(float((w * fdo).sum()) - float((go * x).sum())) < 1e-6 * float(go.norm() * x.norm())
    epc = 1e-6 * prm.Cn
    rp = o.residual(prm, U, Un, Cn=torch.tensor(prm.Cn + epc, dtype=torch.float64))
    rm = o.residual(prm, U, Un, Cn=torch.tensor(prm.Cn - epc, dtype=torch.float64))
    fdc = float((w * (rp - rm)).sum()) / (2 * epc)
    assert abs(fdc - float(gc)) < 1e-6 * max(1.0, abs(fdc))


@pytest.mark.parametrize("case", [("adaptive", 2, 3), ("uniform", 3, 2)], ids=_ids)
def test_adjoint_identity_and_assembled_transpose(case):
    """<w, J x> = <J^T w, x>, and J^T w equals the transpose of the assembled J."""
    _, m = make_mesh(*case)
    prm = params("drop3d" if m.dim == 3 else "drop2d")
    o, U, Un = drop_state(m, prm, perturb=1e-2)
    x = torch.tensor(synth.random_vectors(U.numel(), 1, 8)[0]).reshape(U.shape)
    w = torch.tensor(synth.random_vectors(U.numel(), 1, 9)[0]).reshape(U.shape)
    Jx = o.jvp(prm, U, Un, x)
    gn, _, _ = o.vjp(prm, U, Un, w)
    a, b = float((w * Jx).sum()), float((gn * x).sum())
    assert abs(a - b) <= 1e-12 * float(w.norm() * Jx.norm())
    J = o.jacobian(prm, U, Un)
    assert float((J.T @ w.reshape(-1) - gn.reshape(-1)).norm() / gn.norm()) < 1e-13
    # Dirichlet and pin rows are identity rows of J
    d = m.dim
    bnd = np.nonzero(m.boundary)[0]
    for n in bnd[:5]:
        for i in range(d):
            r = n * (d + 3) + i
            row = J[r].clone()
            assert float(row[r]) == 1.0
            row[r] = 0.0
            assert float(row.abs().max()) == 0.0


def test_newton_conserves_mass_and_decreases_energy():
    """Converged steps conserve int phi to rounding (Proposition 1) and do not
    increase the total energy at a small time step (Theorem 1)."""
    _, m = make_mesh("uniform", 2, 3)
    prm = params("drop2d", dt=1e-3, We=1.0)
    o, U, _ = drop_state(m, prm, noise=0.05, vmax=0.2)
    m0 = o.mass(U)
    e_prev = sum(o.energy(prm, U))
    for _ in range(3):
        U, hist = o.newton_step(prm, U, rtol=1e-13, atol=1e-13)
        assert hist[-1] < 1e-11
        assert abs(o.mass(U) - m0) < 1e-12
        e = sum(o.energy(prm, U))
        assert e <= e_prev + 1e-12
        e_prev = e


def _mms_forcing(prm):
    """Body terms of the manufactured solution printed in Section 5.1, derived with
    sympy from the strong form Eqs. (nav_stokes), (mu_eqn), (phi_eqn)."""
    x1, x2, t = sympy.symbols("x1 x2 t")
    pi = sympy.pi
    v = [pi * sympy.sin(pi * x1) ** 2 * sympy.sin(2 * pi * x2) * sympy.sin(t),
         -pi * sympy.sin(2 * pi * x1) * sympy.sin(pi * x2) ** 2 * sympy.sin(t)]
    p = sympy.cos(pi * x1) * sympy.sin(pi * x2) * sympy.sin(t)
    phi = sympy.cos(pi * x1) * sympy.cos(pi * x2) * sympy.sin(t)
    mu = phi
    X = [x1, x2]
    rho = prm.alpha * phi + prm.beta
    eta = prm.gamma * phi + prm.xi
    J = [(prm.rho_minus - prm.rho_plus) / (2 * prm.rho_plus * prm.Cn) * sympy.diff(mu, xi) for xi in X]
    g = [0, -1]
    mom = []
    for i in range(2):
        e = rho * sympy.diff(v[i], t)
        e += sum(rho * v[j] * sympy.diff(v[i], X[j]) for j in range(2))
        e += sum(J[j] * sympy.diff(v[i], X[j]) for j in range(2)) / prm.Pe
        e += prm.Cn / prm.We * sum(sympy.diff(sympy.diff(phi, X[i]) * sympy.diff(phi, X[j]), X[j]) for j in range(2))
        e += sympy.diff(p, X[i]) / prm.We
        e -= sum(sympy.diff(eta * sympy.diff(v[i], X[j]), X[j]) for j in range(2)) / prm.Re
        e -= rho * g[i] / prm.Fr
        mom.append(e)
    lap = lambda f: sum(sympy.diff(f, xi, 2) for xi in X)
    f_mu = -mu + phi ** 3 - phi - prm.Cn ** 2 * lap(phi)
    f_phi = sympy.diff(phi, t) + sum(sympy.diff(v[i] * phi, X[i]) for i in range(2)) - lap(mu) / (prm.Pe * prm.Cn)
    fm = sympy.lambdify((x1, x2, t), mom, "numpy")
    fmu = sympy.lambdify((x1, x2, t), f_mu, "numpy")
    fph = sympy.lambdify((x1, x2, t), f_phi, "numpy")
    exact = sympy.lambdify((x1, x2, t), [v[0], v[1], p, phi, mu], "numpy")

    def forcing(xq, tm):
        a, b = xq[..., 0].numpy(), xq[..., 1].numpy()
        m0, m1 = fm(a, b, tm)
        fmom = torch.tensor(np.stack([np.broadcast_to(m0, a.shape), np.broadcast_to(m1, a.shape)], -1))
        return fmom, torch.tensor(np.broadcast_to(fmu(a, b, tm), a.shape)), torch.tensor(np.broadcast_to(fph(a, b, tm), a.shape))

    return forcing, exact


MMS_PARAMS = dict(dim=2, Re=10.0, We=1.0, Pe=3.0, Cn=1.0, Fr=1.0, rho_ratio=1.0, eta_ratio=1.0)


def test_temporal_self_convergence_order_two():
    """Crank-Nicolson is second order in time (Section 5.1): on the manufactured
    solution, with its body terms, differences of v and phi at a fixed time between
    runs with dt, dt/2, dt/4 shrink by ~4.  p and mu enter the scheme only through
    their mid-point averages, so their integer-level values are left out."""
    level = 4
    m = Mesh(2, level, synth.uniform_leaves(2, level))
    o = Oracle(m)
    t0, T = 0.5, 0.4
    sols = []
    for n in (4, 8, 16):
        prm = Params(dt=T / n, pin_pressure=1, **MMS_PARAMS)
        forcing, exact = _mms_forcing(prm)
        U = torch.tensor(np.stack(np.broadcast_arrays(*exact(m.x[:, 0], m.x[:, 1], t0)), -1))
        for k in range(n):
            U, hist = o.newton_step(prm, U, rtol=1e-13, atol=1e-13, forcing=forcing,
                                    t_mid=t0 + (k + 0.5) * prm.dt)
        sols.append(U)
    keep = [0, 1, 3]
    e1 = float((sols[0] - sols[1])[:, keep].norm())
    e2 = float((sols[1] - sols[2])[:, keep].norm())
    assert 3.5 < e1 / e2 < 4.5, (e1, e2)


def test_manufactured_solution_truncation_is_second_order():
    """The discrete residual of the interpolated manufactured solution of Section 5.1
    (Re=10, We=1, Cn=1, Pe=3, Fr=1, density ratio 1) with body terms from the strong
    form vanishes at second order as h -> h/2 (dt ~ h^2): this pins the Galerkin terms
    of every row, index order and signs included, against an independent derivation."""
    base = dict(pin_pressure=0, **MMS_PARAMS)
    errs = []
    for level in (4, 5, 6):
        h = 0.5 ** level
        prm = Params(dt=0.5 * h * h, **base)
        forcing, exact = _mms_forcing(prm)
        leaves = synth.uniform_leaves(2, level)
        m = Mesh(2, level, leaves)
        o = Oracle(m)
        t0 = 0.7
        Uo = torch.tensor(np.stack(np.broadcast_arrays(*exact(m.x[:, 0], m.x[:, 1], t0)), -1))
        Un = torch.tensor(np.stack(np.broadcast_arrays(*exact(m.x[:, 0], m.x[:, 1], t0 + prm.dt)), -1))
        R = o.residual(prm, Uo, Un, forcing=forcing, t_mid=t0 + 0.5 * prm.dt)
        interior = ~torch.tensor(m.boundary)
        scaled = R[interior] / (h ** 2)              # per unit area of the test function
        errs.append([float(scaled[:, f].abs().max()) for f in range(5)])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    # every row converges at second order (rate -> 2 from below)
    assert np.all(rates[-1] > 1.8), (errs, rates)
    assert np.all(rates[-1] < 2.2), (errs, rates)


@pytest.mark.parametrize("case", [("uniform", 2, 3), ("adaptive", 3, 3)], ids=_ids)
def test_integrals_closed_forms(case):
    """int 1 = |Omega|, int x = |Omega|/2; phi = 1, v = 0 has zero free energy and
    gravitational energy rho(1) * 1/2 / Fr; v = e_0 has kinetic energy rho/2."""
    _, m = make_mesh(*case)
    d = m.dim
    prm = params("drop3d" if d == 3 else "drop2d", Fr=2.0, rho_ratio=4.0)
    o = Oracle(m)
    U = torch.zeros((m.N, d + 3), dtype=torch.float64)
    U[:, d + 1] = 1.0
    assert abs(o.mass(U) - 1.0) < 1e-13
    kin, free, grav = o.energy(prm, U)
    assert abs(free) < 1e-14 and abs(kin) < 1e-14
    assert abs(grav - 1.0 * 0.5 / 2.0) < 1e-13
    U[:, d + 1] = torch.tensor(m.x[:, 0])
    assert abs(o.mass(U) - 0.5) < 1e-13
    U[:, d + 1] = -1.0
    U[:, 0] = 1.0
    kin, free, grav = o.energy(prm, U)
    assert abs(kin - 0.5 * (1.0 / 4.0)) < 1e-13


def test_equilibrium_profile_gives_small_mu():
    """phi = tanh(x/(sqrt(2) Cn)) solves psi'(phi) - Cn^2 phi'' = 0 (Eqs. mu_eqn,
    free_energy): the discrete mu^0 vanishes at second order under refinement."""
    Cn = 0.05
    prm = params("drop2d", Cn=Cn)
    errs = []
    for level in (5, 6, 7):
        leaves = synth.uniform_leaves(2, level)
        m = Mesh(2, level, leaves)
        o = Oracle(m)
        phi = torch.tensor(np.tanh((m.x[:, 0] - 0.5) / (math.sqrt(2.0) * Cn)))
        mu = o.initial_mu(prm, phi)
        errs.append(float(mu.abs().max()))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3, errs


def test_mirror_symmetry():
    """Mirroring x_0 -> 1 - x_0 with v_0 -> -v_0 maps the residual onto itself."""
    _, m = make_mesh("uniform", 2, 3)
    prm = params("drop2d", Fr=1.0, rho_ratio=3.0)
    o, U, Un = drop_state(m, prm, perturb=1e-2)
    key = {tuple(p): i for i, p in enumerate(m.nodes)}
    n_side = 1 << m.max_level
    perm = np.array([key[(n_side - p[0], p[1])] for p in m.nodes])
    flip = torch.ones(5, dtype=torch.float64)
    flip[0] = -1.0
    mir = lambda A: A[perm] * flip
    prm.pin_pressure = 0
    R = o.residual(prm, U, Un)
    Rm = o.residual(prm, mir(U), mir(Un))
    assert float((Rm - mir(R)).abs().max()) < 1e-11 * float(R.abs().max())


@pytest.mark.parametrize("dim,level", [(2, 3), (3, 2)])
def test_stabilisation_parameters_spot_values(dim, level):
    """Hand-evaluated tau_m and tau_phi (Definition 2 stabilisation parameters, G = (4/h^2) I
    on an axis-aligned cube) through the rows of a boundary node, for a state that is
    constant in space: v~ = v0 + a/2, phi jumps by b, mu = psi'(c), no gravity.  Then
    R_m = rho~ a / dt, R_c = 0 and R_phi = b / dt are constants, and for a node on the face
    x_0 = 0 (away from edges) the only surviving integral of a test gradient is
    int d_0 N_a = -h^(d-1):
      pressure row  = -(tau_m / rho~) rho~ a_0 / dt * h^(d-1)
      phi row       = -h^(d-1) (-v~_0 phi~ + tau_m a_0 phi~ / dt + v~_0 tau_phi b / dt) + (b / dt) h^d / 2.
    The velocity rows of that node are Dirichlet rows; the pressure and phi rows are not.
    (tau_c multiplies R_c = div v~ = 0 here and is not pinned by this state.)"""
    leaves = synth.uniform_leaves(dim, level)
    m = Mesh(dim, level, leaves)
    o = Oracle(m)
    cfg = synth.config_params("drop3d" if dim == 3 else "drop2d")
    cfg.update(Fr=0.0, rho_ratio=4.0, eta_ratio=3.0)
    prm = Params(**cfg)
    h = 1.0 / (1 << level)
    v0 = np.array([0.3, -0.2, 0.1][:dim])
    a = np.array([0.05, 0.02, -0.01][:dim])
    c, b = 0.4, 0.02
    U = np.zeros((m.N, dim + 3))
    U[:, :dim] = v0
    U[:, dim + 1] = c
    U[:, dim + 2] = c ** 3 - c
    Un = U.copy()
    Un[:, :dim] = v0 + a
    Un[:, dim + 1] = c + b
    Un[:, dim + 2] = U[:, dim + 2]
    R = o.residual(prm, torch.tensor(U), torch.tensor(Un)).numpy()
    # the node at x_0 = 0, every other coordinate at the middle of the domain
    target = np.array([0.0] + [0.5] * (dim - 1))
    node = int(np.argmin(np.abs(m.x - target).sum(axis=1)))
    assert np.abs(m.x[node] - target).max() < 1e-12
    vt = v0 + a / 2
    pt = c + b / 2
    rho = 0.5 * (1 + pt) * 1.0 + 0.5 * (1 - pt) / cfg["rho_ratio"]
    eta = 0.5 * (1 + pt) * 1.0 + 0.5 * (1 - pt) / cfg["eta_ratio"]
    dt = cfg["dt"]
    vGv = 4.0 / h ** 2 * float(vt @ vt)
    GG = 16.0 * dim / h ** 4
    tau_m = (4.0 / dt ** 2 + vGv + cfg["C_I"] * (eta / (rho * cfg["Re"])) ** 2 * GG) ** -0.5
    tau_phi = (4.0 / dt ** 2 + vGv + cfg["C_phi"] * (1.0 / (cfg["Pe"] * cfg["Cn"])) ** 2 * GG) ** -0.5
    face = h ** (dim - 1)
    p_row = -tau_m * a[0] / dt * face
    phi_row = -face * (-vt[0] * pt + tau_m * a[0] * pt / dt + vt[0] * tau_phi * b / dt) + (b / dt) * h ** dim / 2
    assert abs(R[node, dim] - p_row) <= 1e-12 * abs(p_row)
    assert abs(R[node, dim + 1] - phi_row) <= 1e-12 * abs(phi_row)
    # potential row: psi' at the mid-point average, -(q, mu~) + (q, psi'(phi~)), int N_a = h^d / 2
    mu_row = (pt ** 3 - pt - (c ** 3 - c)) * h ** dim / 2
    assert abs(R[node, dim + 2] - mu_row) <= 1e-12 * abs(mu_row)


def test_velocity_boundary_conditions_rows():
    """Mixed Dirichlet / natural velocity conditions (Section 5 set-ups): Dirichlet rows are
    exactly v^{k+1} - g, every other row equals the row of the residual with no Dirichlet
    row at all, and the default equals no-slip on every face."""
    leaves = synth.uniform_leaves(2, 3)
    m = Mesh(2, 3, leaves)
    prm = params("drop2d", Fr=1.0, rho_ratio=3.0, eta_ratio=2.0)
    o0, U, Un = drop_state(m, prm, perturb=1e-2)
    g = np.stack([np.sin(np.pi * m.x[:, 0]) ** 2, 0.3 * m.x[:, 1]], axis=1)
    # bubble side walls: v_0 Dirichlet on x = 0, 1; lid on y = 1 moving with g; y = 0 no-slip
    fm = [1, 1, 3, 3]
    ob = Oracle(m, bc=(fm, g))
    on = Oracle(m, bc=([0, 0, 0, 0], None))
    R = ob.residual(prm, U, Un).numpy()
    Rn = on.residual(prm, U, Un).numpy()
    mask = ob.dmask.numpy()
    assert mask[:, 0].sum() > mask[:, 1].sum() > 0
    vel = R[:, :2]
    assert np.array_equal(vel[mask], (Un.numpy()[:, :2] - g)[mask])
    assert np.array_equal(vel[~mask], Rn[:, :2][~mask])
    assert np.array_equal(R[:, 2:], Rn[:, 2:])
    Rd = Oracle(m, bc=([3, 3, 3, 3], None)).residual(prm, U, Un)
    assert torch.equal(Rd, o0.residual(prm, U, Un))
