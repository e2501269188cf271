"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, element by element
on the same seeded inputs: node numbering (bit-exact), residual, J x (FP64 and FP32),
J^T w with its U^k and Cn parts, mass, energy and mu^0.  Tolerances: relative L2
<= 1e-12 for FP64, <= 1e-5 for FP32 J x."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import Mesh as OMesh, Oracle, Params as OParams

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def chns():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2009_06628_gb300 as chns
    if not os.path.exists(chns.LIB_PATH):
        from paper_2009_06628_gb300 import build
        build.build()
    chns.load()
    return chns


# (name, dim, max_level, leaves-builder, params)
def _leaves(kind, dim, level):
    if kind == "uniform":
        return synth.uniform_leaves(dim, level)
    c = [0.45, 0.55, 0.5][:dim]
    return synth.sphere_band_leaves(dim, max(1, level - 3), level, [c], [0.3], 0.03)


CASES = [
    ("uniform", 2, 5, "drop2d", {}),                                   # 32 x 32 drop, no gravity
    ("adaptive", 2, 6, "drop2d", dict(Fr=1.0, rho_ratio=5.0, eta_ratio=3.0)),
    ("uniform", 3, 3, "drop3d", {}),
    ("adaptive", 3, 5, "drop3d", dict(rho_ratio=100.0, eta_ratio=50.0)),
    ("uniform", 3, 4, "drop3d", dict(pin_pressure=1)),                  # point-pinned pressure row
]


def _ids(c):
    return f"{c[0]}{c[1]}d-L{c[2]}" + ("-pin1" if c[4].get("pin_pressure") == 1 else "")


class Case:
    def __init__(self, chns, kind, dim, level, cfg_name, over, seed=1):
        self.leaves = _leaves(kind, dim, level)
        self.om = OMesh(dim, level, self.leaves)
        self.gm = chns.Mesh(dim, level, self.leaves)
        cfg = synth.config_params(cfg_name)
        cfg.update(over)
        self.cfg = cfg
        self.prm = chns.Params.make(**cfg)
        self.oprm = OParams(**cfg)
        self.o = Oracle(self.om)
        d = dim
        x = self.om.x
        U = np.zeros((self.om.N, d + 3))
        U[:, d + 1] = synth.drop_phi(x, [[0.5] * d], [0.25], cfg["Cn"], noise=1e-3, seed=seed)
        U[:, :d] = synth.fourier_velocity(x, 6, seed + 1, 0.1)
        U[:, d] = 0.05 * synth.random_vectors(self.om.N, 1, seed + 2)[0]
        U[:, d + 2] = 0.1 * synth.random_vectors(self.om.N, 1, seed + 3)[0]
        Un = U + 1e-3 * synth.random_vectors(U.size, 1, seed + 4)[0].reshape(U.shape)
        U[self.om.boundary, :d] = 0.0
        Un[self.om.boundary, :d] = 0.0
        self.U = torch.tensor(U)
        self.Un = torch.tensor(Un)
        self.dev = torch.device("cuda")
        self.Ud = self.U.to(self.dev)
        self.Und = self.Un.to(self.dev)


def rel(a, b):
    return float((a.cpu() - b).norm() / b.norm())


@pytest.fixture(scope="module", params=CASES, ids=_ids)
def case(request, chns):
    return Case(chns, *request.param)


def test_node_numbering_bit_exact(case):
    assert case.gm.N == case.om.N
    assert np.array_equal(case.gm.node_coords(), case.om.nodes.astype(np.int32))
    assert case.gm.H == len(np.unique(case.om.corner_x[case.om.hanging], axis=0))


def test_residual_fp64(chns, case):
    R = chns.residual(case.gm, case.prm, case.Ud, case.Und)
    Ro = case.o.residual(case.oprm, case.U, case.Un)
    assert rel(R, Ro) <= TOL64
    # Dirichlet rows are exact copies
    b = case.om.boundary
    d = case.om.dim
    assert torch.equal(R.cpu()[b, :d], case.Un[b, :d])


def test_jvp_fp64_many_directions(chns, case):
    X = synth.random_vectors(case.U.numel(), 16, 101)
    for i in range(16 if case.om.dim == 2 else 4):
        x = torch.tensor(X[i]).reshape(case.U.shape)
        y = chns.jvp(case.gm, case.prm, case.Ud, case.Und, x.to(case.dev))
        yo = case.o.jvp(case.oprm, case.U, case.Un, x)
        assert rel(y, yo) <= TOL64, i


def test_jvp_fp32(chns, case):
    x = torch.tensor(synth.random_vectors(case.U.numel(), 1, 201)[0]).reshape(case.U.shape)
    f = lambda t: t.to(case.dev, torch.float32)
    y = chns.jvp(case.gm, case.prm, f(case.U), f(case.Un), f(x))
    yo = case.o.jvp(case.oprm, case.U, case.Un, x)
    assert y.dtype == torch.float32
    assert rel(y.double(), yo) <= TOL32


def test_vjp_fp64(chns, case):
    w = torch.tensor(synth.random_vectors(case.U.numel(), 1, 301)[0]).reshape(case.U.shape)
    gn, go, gc = chns.vjp(case.gm, case.prm, case.Ud, case.Und, w.to(case.dev))
    gno, goo, gco = case.o.vjp(case.oprm, case.U, case.Un, w)
    assert rel(gn, gno) <= TOL64
    assert rel(go, goo) <= TOL64
    assert abs(float(gc.cpu()[0]) - float(gco)) <= TOL64 * max(1.0, abs(float(gco))) * 10


def test_adjoint_identity_gpu(chns, case):
    x = torch.tensor(synth.random_vectors(case.U.numel(), 1, 401)[0]).reshape(case.U.shape).to(case.dev)
    w = torch.tensor(synth.random_vectors(case.U.numel(), 1, 402)[0]).reshape(case.U.shape).to(case.dev)
    Jx = chns.jvp(case.gm, case.prm, case.Ud, case.Und, x)
    gn, _, _ = chns.vjp(case.gm, case.prm, case.Ud, case.Und, w, want_old=False, want_cn=False)
    a, b = float((w * Jx).sum()), float((gn * x).sum())
    assert abs(a - b) <= 1e-12 * float(w.norm() * Jx.norm())


def test_mass_and_energy(chns, case):
    m = chns.mass(case.gm, case.Und)
    mo = case.o.mass(case.Un)
    assert abs(m - mo) <= 1e-13 * max(1.0, abs(mo))
    e = chns.energy(case.gm, case.prm, case.Und)
    eo = case.o.energy(case.oprm, case.Un)
    for a, b in zip(e, eo):
        assert abs(a - b) <= 1e-12 * max(1e-12, abs(b)) + 1e-15


def test_initial_mu(chns, case):
    U = case.Und.clone()
    chns.initial_mu(case.gm, case.prm, U)
    mu_o = case.o.initial_mu(case.oprm, case.Un[:, case.om.dim + 1])
    d = case.om.dim
    assert rel(U[:, d + 2], mu_o) <= 1e-11
    # other fields untouched
    assert torch.equal(U[:, : d + 2], case.Und[:, : d + 2])
