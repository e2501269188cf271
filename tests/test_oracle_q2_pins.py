"""Pins of the oracle's Q2 (triquadratic) elements, without the GPU: quadratic fields
and their derivatives are exact at the Gauss points; the 3-point rule integrates the
basis exactly (node masses); Proposition 1's mass row-sum, the pressure row-sum and the
hydrostatic zero hold on Q2 as on Q1; J x equals central finite differences; and the
residual of the interpolated manufactured solution of Section 5.1 vanishes at second
order in every row (dt ~ h^2)."""
import numpy as np
import pytest
import torch

from oracle import MeshQ2, Oracle, Params
from tests.helpers import params
from tests import test_oracle_pins as q1pins


@pytest.mark.parametrize("dim", [2, 3])
def test_q2_quadratic_patch(dim):
    m = MeshQ2(dim, 2)
    o = Oracle(m)
    rng = np.random.default_rng(0)
    A = rng.standard_normal((dim, dim))
    A = A + A.T
    b = rng.standard_normal(dim)
    f = lambda x: 0.3 + x @ b + 0.5 * np.einsum("ni,ij,nj->n", x, A, x)
    val, grad, hess = o.interp(o.gather(torch.tensor(f(m.x))))
    xq = o.xq.numpy()
    assert np.abs(val.numpy() - f(xq.reshape(-1, dim)).reshape(val.shape)).max() < 1e-14
    assert np.abs(grad.numpy() - (b + xq @ A)).max() < 1e-13
    assert np.abs(hess.numpy() - A).max() < 1e-12
    # node masses: int N_a over the domain sums to |Omega|; a vertex, edge and centre node of
    # one element carry (h/2)^d times products of 1/3 and 4/3
    assert abs(float(o.node_mass.sum()) - 1.0) < 1e-14


def _state(m, prm, seed=1, v_bnd_zero=True):
    d = m.dim
    rng = np.random.default_rng(seed)
    U = np.zeros((m.N, d + 3))
    r = np.sqrt(((m.x - 0.5) ** 2).sum(1))
    U[:, d + 1] = 0.8 * np.tanh((0.3 - r) / (np.sqrt(2) * 0.1))
    U[:, :d] = 0.1 * np.sin(np.pi * m.x) ** 2 * rng.standard_normal(d)
    U[:, d] = 0.05 * rng.standard_normal(m.N)
    U[:, d + 2] = 0.1 * rng.standard_normal(m.N)
    Un = U + 1e-2 * rng.standard_normal(U.shape)
    if v_bnd_zero:
        U[m.boundary, :d] = 0.0
        Un[m.boundary, :d] = 0.0
    return torch.tensor(U), torch.tensor(Un)


@pytest.mark.parametrize("dim,level", [(2, 3), (3, 2)])
def test_q2_row_sums_and_hydrostatic(dim, level):
    m = MeshQ2(dim, level)
    o = Oracle(m)
    prm = params("drop3d" if dim == 3 else "drop2d", pin_pressure=0, Fr=1.0, rho_ratio=4.0, eta_ratio=2.0)
    U, Un = _state(m, prm)
    R = o.residual(prm, U, Un)
    lhs = float(R[:, dim + 1].sum())
    rhs = (o.mass(Un) - o.mass(U)) / prm.dt
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs))
    scale = float(R[:, dim].abs().sum())
    assert abs(float(R[:, dim].sum())) <= 1e-12 * max(scale, 1.0)
    Uh = q1pins.hydrostatic(m, prm, c=0.3)
    assert float(o.residual(prm, Uh, Uh).abs().max()) < 1e-11


def test_q2_jacobian_matches_central_differences():
    m = MeshQ2(2, 2)
    o = Oracle(m)
    prm = params("drop2d", Fr=1.0, rho_ratio=3.0, eta_ratio=2.0)
    U, Un = _state(m, prm, seed=3)
    x = torch.tensor(np.random.default_rng(4).standard_normal(U.shape))
    Jx = o.jvp(prm, U, Un, x)
    eps = 1e-6
    fd = (o.residual(prm, U, Un + eps * x) - o.residual(prm, U, Un - eps * x)) / (2 * eps)
    assert float((Jx - fd).norm() / Jx.norm()) < 1e-8


def test_q2_manufactured_solution_truncation():
    base = dict(pin_pressure=0, **q1pins.MMS_PARAMS)
    errs = []
    for level in (3, 4, 5):
        h = 0.5 ** level
        prm = Params(dt=0.5 * h * h, **base)
        forcing, exact = q1pins._mms_forcing(prm)
        m = MeshQ2(2, level)
        o = Oracle(m)
        t0 = 0.7
        Uo = torch.tensor(np.stack(np.broadcast_arrays(*exact(m.x[:, 0], m.x[:, 1], t0)), -1))
        Un = torch.tensor(np.stack(np.broadcast_arrays(*exact(m.x[:, 0], m.x[:, 1], t0 + prm.dt)), -1))
        R = o.residual(prm, Uo, Un, forcing=forcing, t_mid=t0 + 0.5 * prm.dt)
        interior = ~torch.tensor(m.boundary)
        scaled = R[interior] / (0.5 * h) ** 2
        errs.append([float(scaled[:, f].abs().max()) for f in range(5)])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[-1] > 1.8), (errs, rates)
