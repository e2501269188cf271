"""Pin of every term of Definition 2 at one interior node, evaluated by hand.

The state is a set of multilinear polynomials (products of distinct coordinates:
1, x, y, xy, ... ), which the Q1 space of a uniform mesh reproduces exactly.  sympy
differentiates the continuous fields, forms the strong residuals R_m, R_c, R_phi, the
stabilisation parameters tau_m, tau_c, tau_phi (G = (4/h^2) I) and then every weak-form
term of Definition 2 (with the Crank-Nicolson substitution of Definition 1) separately,
tested against the hat function of the node and summed with the 2-point Gauss rule
over the 2^d elements around it.  Nothing here uses the oracle's basis tables, einsum
index strings or its grouping of terms into value and gradient fluxes: the hand sums
follow the term list of Definition 2, one term per line.

The node is interior, so no Dirichlet row replaces the momentum rows, and the state has
a velocity gradient that is not symmetric, a time jump in every field, a non-constant
chemical potential (J != 0), a bilinear phase field (mixed second derivatives, so the
capillary and variable-viscosity strong terms are non-zero) and a divergent velocity
(R_c != 0, so tau_c is visible).  Every term is checked to be large enough that flipping
its sign, or transposing its indices, would fail the comparison.
"""
import math

import numpy as np
import pytest
import sympy

import synth
from oracle import Mesh, MeshQ2, Oracle, Params


def _monomials(X, order=1):
    """Q1: the products of distinct coordinates (1, x, y, xy, ...), a basis of the Q1
    space.  Q2: the monomials of total degree <= 2 (1, x, y, x^2, xy, y^2, ...), which Q2
    elements reproduce exactly and which have non-zero pure and mixed second derivatives
    (the full Q2 basis would only make the symbolic expressions longer)."""
    d = len(X)
    out = []
    for s in range((order + 1) ** d):
        a = [(s // (order + 1) ** k) % (order + 1) for k in range(d)]
        if order == 2 and sum(a) > 2:
            continue
        m = sympy.Integer(1)
        for k in range(d):
            m = m * X[k] ** a[k]
        out.append(m)
    return out


def _physics(dim):
    """Parameters chosen so that no term of the momentum rows is negligible: a time step
    for which 4/dt^2 does not swamp the velocity and viscous parts of tau_m, unequal
    density and viscosity phases, gravity along -e_{d-1}."""
    return dict(dim=dim, Re=2.0, We=3.0, Pe=4.0, Cn=0.3, Fr=2.0, rho_ratio=4.0, eta_ratio=3.0,
                dt=0.02, C_I=6.0, C_phi=6.0, pin_pressure=0)


def hand_rows(dim, level=2, seed=11, order=1):
    """Returns (mesh, params, node, U_old, U_new, terms) where terms[row] is a dict
    {name: value} of the separate weak-form terms of that row of the interior node
    x_A = (1/2, ..., 1/2).  Every field is a multilinear polynomial plus a multiple of the
    hat function of x_A (itself multilinear on each element, so the field stays in the
    Q1 space, while its discrete Laplacian at x_A is not zero and the diffusion terms
    are visible).  order=2: Q2 elements (fields with squares of each coordinate, the
    quadratic hat of the vertex node, the 3-point Gauss rule), where the strong residuals
    also carry the pure second derivatives."""
    prm = _physics(dim)
    h = 1.0 / (1 << level)
    X = sympy.symbols(f"x0:{dim}", real=True)
    monos = _monomials(X, order)
    rng = np.random.default_rng(seed)
    xa = np.full(dim, 0.5)

    def q1(scale, base=0.0):
        coef = [scale * rng.uniform(-1.0, 1.0) for _ in monos]
        bump = scale * rng.uniform(0.5, 1.0)
        return (sympy.Float(base) + sum(sympy.Float(c) * m for c, m in zip(coef, monos)), bump)

    # (polynomial, bump height) of every field at both time levels
    vo = [q1(0.6, 0.3 * (k + 1)) for k in range(dim)]
    dv = [q1(0.05) for k in range(dim)]
    po, dp = q1(1.0), q1(0.3)
    phio, dphi = q1(0.08, 0.15), q1(0.01)
    muo, dmu = q1(0.6), q1(0.1)

    dt, Re, We, Pe, Cn, Fr = prm["dt"], prm["Re"], prm["We"], prm["Pe"], prm["Cn"], prm["Fr"]
    rho_p, rho_m = 1.0, 1.0 / prm["rho_ratio"]
    eta_p, eta_m = 1.0, 1.0 / prm["eta_ratio"]
    ghat = [0.0] * dim
    ghat[dim - 1] = -1.0
    g = 4.0 / h ** 2
    GG = dim * g * g
    trG = dim * g
    D = lambda f, k: sympy.diff(f, X[k])
    half = sympy.Rational(1, 2)
    Nsym = sympy.Symbol("N")
    dNs = sympy.symbols(f"dN0:{dim}")
    args = list(X) + [Nsym] + list(dNs)
    if order == 1:
        gp, gw = np.array([-1.0, 1.0]) / math.sqrt(3.0), np.array([1.0, 1.0])
    else:
        gp, gw = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)]), np.array([5.0, 8.0, 5.0]) / 9.0
    ng = gp.shape[0]
    wdet = (h / 2.0) ** dim

    terms = [dict() for _ in range(dim + 3)]
    radicands = []
    for side in range(1 << dim):
        s = [1 if (side >> k) & 1 else -1 for k in range(dim)]
        # basis function of x_A on this element: Q1 hat, or the quadratic Lagrange factor of
        # the element end at x_A (local xi = -1 on the element to the right of x_A, +1 on the
        # one to its left)
        hat = sympy.Integer(1)
        for k in range(dim):
            if order == 1:
                hat = hat * (1 - s[k] * (X[k] - float(xa[k])) / h)
            else:
                xi = 2 * (X[k] - float(xa[k] + s[k] * h / 2)) / h
                hat = hat * (xi * (xi - 1) / 2 if s[k] > 0 else xi * (xi + 1) / 2)
        F = lambda pb: pb[0] + sympy.Float(pb[1]) * hat
        vo_e = [F(vo[k]) for k in range(dim)]
        vn_e = [vo_e[k] + F(dv[k]) for k in range(dim)]
        po_e, pn_e = F(po), F(po) + F(dp)
        phio_e, phin_e = F(phio), F(phio) + F(dphi)
        muo_e, mun_e = F(muo), F(muo) + F(dmu)
        vt = [half * (vo_e[k] + vn_e[k]) for k in range(dim)]
        pt = half * (po_e + pn_e)
        phit = half * (phio_e + phin_e)
        mut = half * (muo_e + mun_e)
        # phi* = phi~ because |phi~| < 1 everywhere (checked at the nodes below)
        rho = (rho_p - rho_m) / (2 * rho_p) * phit + (rho_p + rho_m) / (2 * rho_p)
        eta = (eta_p - eta_m) / (2 * eta_p) * phit + (eta_p + eta_m) / (2 * eta_p)
        J = [(rho_m - rho_p) / (2 * rho_p * Cn) * D(mut, j) for j in range(dim)]

        # strong residuals at the mid-point (printed after Definition 2)
        Rm = []
        for i in range(dim):
            r = rho * (vn_e[i] - vo_e[i]) / dt
            r += sum(rho * vt[j] * D(vt[i], j) for j in range(dim))
            r += sum(J[j] * D(vt[i], j) for j in range(dim)) / Pe
            r += (Cn / We) * sum(D(D(phit, i) * D(phit, j), j) for j in range(dim))
            r += D(pt, i) / We
            r -= sum(D(eta * D(vt[i], k), k) for k in range(dim)) / Re
            r -= rho * ghat[i] / Fr
            Rm.append(r)
        Rc = sum(D(vt[i], i) for i in range(dim))
        Rphi = (phin_e - phio_e) / dt + sum(D(vt[i] * phit, i) for i in range(dim)) \
            - sum(D(D(mut, i), i) for i in range(dim)) / (Pe * Cn)
        vGv = g * sum(vt[k] * vt[k] for k in range(dim))
        vGJ = g * sum(vt[k] * J[k] for k in range(dim))
        rad_m = 4.0 / dt ** 2 + vGv + vGJ / (rho * Pe) + prm["C_I"] * (eta / (rho * Re)) ** 2 * GG
        tau_m = rad_m ** sympy.Rational(-1, 2)
        tau_c = 1 / (trG * tau_m)
        tau_phi = (4.0 / dt ** 2 + vGv + prm["C_phi"] * (1.0 / (Pe * Cn)) ** 2 * GG) ** sympy.Rational(-1, 2)

        # integrands, one per term of Definition 2; N / dN stand for the test function
        rows = []
        for i in range(dim):
            t = {
                "rho dv/dt": Nsym * rho * (vn_e[i] - vo_e[i]) / dt,
                "rho v.grad v": Nsym * sum(rho * vt[j] * D(vt[i], j) for j in range(dim)),
                "-tau_m Rm.grad v": -Nsym * sum(tau_m * Rm[j] * D(vt[i], j) for j in range(dim)),
                "(d_j w_i, v_j tau_m Rm_i)": sum(dNs[j] * vt[j] * tau_m * Rm[i] for j in range(dim)),
                "-(d_j w_i, tau_m^2/rho Rm_j Rm_i)": -sum(dNs[j] * tau_m ** 2 / rho * Rm[j] * Rm[i]
                                                          for j in range(dim)),
                "1/Pe (w_i, J_j d_j v_i)": Nsym * sum(J[j] * D(vt[i], j) for j in range(dim)) / Pe,
                "1/Pe (d_j w_i, J_j tau_m/rho Rm_i)": sum(dNs[j] * J[j] * tau_m / rho * Rm[i]
                                                          for j in range(dim)) / Pe,
                "-Cn/We (d_j w_i, d_i phi d_j phi)": -(Cn / We) * sum(dNs[j] * D(phit, i) * D(phit, j)
                                                                      for j in range(dim)),
                "-1/We (d_i w_i, p)": -dNs[i] * pt / We,
                "1/We (d_i w_i, rho tau_c Rc)": dNs[i] * rho * tau_c * Rc / We,
                "1/Re (d_k w_i, eta d_k v_i)": sum(dNs[k] * eta * D(vt[i], k) for k in range(dim)) / Re,
            }
            if ghat[i] != 0.0:
                t["-(w_i, rho g_i / Fr)"] = -Nsym * rho * ghat[i] / Fr
            rows.append(t)
        rows.append({
            "(q, div v^{k+1})": Nsym * sum(D(vn_e[i], i) for i in range(dim)),
            "(d_i q, tau_m/rho Rm_i)": sum(dNs[i] * tau_m / rho * Rm[i] for i in range(dim)),
        })
        rows.append({
            "(q, dphi/dt)": Nsym * (phin_e - phio_e) / dt,
            "-(d_i q, v_i phi)": -sum(dNs[i] * vt[i] * phit for i in range(dim)),
            "(d_i q, tau_m/rho Rm_i phi)": sum(dNs[i] * tau_m / rho * Rm[i] * phit for i in range(dim)),
            "(d_i q, v_i tau_phi Rphi)": sum(dNs[i] * vt[i] * tau_phi * Rphi for i in range(dim)),
            "1/(Pe Cn) (d_i q, d_i mu)": sum(dNs[i] * D(mut, i) for i in range(dim)) / (Pe * Cn),
        })
        rows.append({
            "-(q, mu)": -Nsym * mut,
            "(q, psi'(phi))": Nsym * (phit ** 3 - phit),
            "Cn^2 (d_i q, d_i phi)": Cn ** 2 * sum(dNs[i] * D(phit, i) for i in range(dim)),
        })

        # Gauss points of this element, their weights, the test function N_A and its gradient
        centre = xa + np.array(s) * h / 2.0
        qidx = [[(q // ng ** k) % ng for k in range(dim)] for q in range(ng ** dim)]
        pts = np.array([centre + np.array([gp[i[k]] for k in range(dim)]) * h / 2.0 for i in qidx])
        wts = np.array([np.prod([gw[i[k]] for k in range(dim)]) for i in qidx])
        fN = sympy.lambdify(X, hat, "numpy")
        fdN = [sympy.lambdify(X, sympy.diff(hat, X[k]), "numpy") for k in range(dim)]
        cols = [pts[:, k] for k in range(dim)]
        Nv = np.broadcast_to(fN(*cols), (pts.shape[0],)).astype(float)
        dNv = np.stack([np.broadcast_to(f(*cols), (pts.shape[0],)) for f in fdN], axis=1).astype(float)
        vals_in = cols + [Nv] + [dNv[:, k] for k in range(dim)]
        for r, row in enumerate(rows):
            for name, expr in row.items():
                vals = sympy.lambdify(args, expr, "numpy", cse=True)(*vals_in)
                terms[r][name] = terms[r].get(name, 0.0) + float(np.sum(np.broadcast_to(vals, Nv.shape) * wts)) * wdet
        radicands.append(np.asarray(sympy.lambdify(X, rad_m, "numpy")(*[pts[:, k] for k in range(dim)])))

    # radicands stay positive at every Gauss point
    assert all(np.all(r > 0) for r in radicands)
    # nodal values of the same fields on the uniform mesh (the hat is 1 at x_A, 0 elsewhere)
    m = Mesh(dim, level, synth.uniform_leaves(dim, level)) if order == 1 else MeshQ2(dim, level)
    node = int(np.argmin(np.abs(m.x - xa).sum(axis=1)))
    assert np.abs(m.x[node] - xa).max() < 1e-15 and not m.boundary[node]

    def nodal(pb):
        v = np.broadcast_to(sympy.lambdify(X, pb[0], "numpy")(*[m.x[:, k] for k in range(dim)]), (m.N,)).copy()
        v[node] += pb[1]
        return v

    U_old = np.stack([nodal(f) for f in vo + [po, phio, muo]], axis=1)
    U_new = U_old + np.stack([nodal(f) for f in dv + [dp, dphi, dmu]], axis=1)
    assert np.abs(0.5 * (U_old[:, dim + 1] + U_new[:, dim + 1])).max() < 1.0
    return m, Params(**prm), node, U_old, U_new, terms


def compare(oracle_cls, dim, order=1):
    """Largest |oracle row - sum of hand terms| relative to the sum of |terms|, over the
    d + 3 rows of the node, and the smallest |term| relative to the same scale."""
    import torch
    m, prm, node, U_old, U_new, terms = hand_rows(dim, order=order)
    o = oracle_cls(m)
    R = o.residual(prm, torch.tensor(U_old), torch.tensor(U_new)).numpy()
    err, small = 0.0, 1.0
    for f, t in enumerate(terms):
        scale = sum(abs(v) for v in t.values())
        ref = sum(t.values())
        err = max(err, abs(R[node, f] - ref) / scale)
        small = min(small, min(abs(v) for v in t.values()) / scale)
    return err, small


@pytest.mark.parametrize("dim", [2, 3])
def test_every_definition2_term_at_an_interior_node(dim):
    """Oracle rows of an interior node equal the term-by-term hand evaluation of
    Definition 2 (momentum with all VMS terms, tau_c; solenoidality with PSPG; Cahn-
    Hilliard with its stabilisation; potential) to rounding."""
    err, small = compare(Oracle, dim)
    assert err < 1e-12, err
    # every term is visible: a sign flip of any of them moves its row by 2|term|
    assert small > 1e-6, small


@pytest.mark.parametrize("dim", [2, 3])
def test_every_definition2_term_at_an_interior_node_q2(dim):
    """The same term-by-term evaluation on Q2 elements: the pure second derivatives of the
    strong residuals (eta lap v, d_i phi lap phi + d_i phi d_ii phi, lap mu) are non-zero."""
    err, small = compare(Oracle, dim, order=2)
    assert err < 1e-12, err
    assert small > 1e-7, small
