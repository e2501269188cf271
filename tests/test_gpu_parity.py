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


def hanging_parent_rows(om):
    """Independent nodes that are constraint parents of some hanging corner."""
    return np.unique(om.parents[om.hanging][om.weights[om.hanging] > 0])


def max_abs_on_rows(a, b, rows):
    """max over the given rows of |a - b|, each field scaled by the largest |b| of that field
    over all rows (a relative-L2 check alone would dilute a few wrong rows)."""
    a, b = a.cpu().double(), b.double()
    scale = b.abs().amax(dim=0).clamp_min(1e-300)
    return float(((a[rows] - b[rows]).abs() / scale).max())


def test_node_numbering_bit_exact(case):
    assert case.gm.N == case.om.N
    assert np.array_equal(case.gm.node_coords(), case.om.nodes.astype(np.int32))
    assert case.gm.H == len(np.unique(case.om.corner_x[case.om.hanging], axis=0))


def test_residual_fp64(chns, case):
    R = chns.residual(case.gm, case.prm, case.Ud, case.Und)
    Ro = case.o.residual(case.oprm, case.U, case.Un)
    assert rel(R, Ro) <= TOL64
    rows = hanging_parent_rows(case.om)
    if rows.size:
        assert max_abs_on_rows(R, Ro, rows) <= 1e-11
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
        rows = hanging_parent_rows(case.om)
        if rows.size:
            assert max_abs_on_rows(y, yo, rows) <= 1e-11, i


def test_jvp_fp32(chns, case):
    x = torch.tensor(synth.random_vectors(case.U.numel(), 1, 201)[0]).reshape(case.U.shape)
    f = lambda t: t.to(case.dev, torch.float32)
    y = chns.jvp(case.gm, case.prm, f(case.U), f(case.Un), f(x))
    yo = case.o.jvp(case.oprm, case.U, case.Un, x)
    assert y.dtype == torch.float32
    assert rel(y.double(), yo) <= TOL32
    rows = hanging_parent_rows(case.om)
    if rows.size:
        assert max_abs_on_rows(y, yo, rows) <= 1e-5


def test_vjp_fp64(chns, case):
    w = torch.tensor(synth.random_vectors(case.U.numel(), 1, 301)[0]).reshape(case.U.shape)
    gn, go, gc = chns.vjp(case.gm, case.prm, case.Ud, case.Und, w.to(case.dev))
    gno, goo, gco = case.o.vjp(case.oprm, case.U, case.Un, w)
    assert rel(gn, gno) <= TOL64
    assert rel(go, goo) <= TOL64
    rows = hanging_parent_rows(case.om)
    if rows.size:
        assert max_abs_on_rows(gn, gno, rows) <= 1e-11
        assert max_abs_on_rows(go, goo, rows) <= 1e-11
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


def test_config2_full_vector_parity_64cubed(chns):
    """The 64^3 workload of the benchmark (uniform octree level 6, 274,625 nodes x 6 DOF, the
    tanh drop of radius 0.2 with Cn = 0.02, the 8-mode divergence-free velocity, density and
    viscosity ratios 10, gravity along -z): full-vector parity of the residual, FP64 J x (two
    directions), FP32 J x and J^T w (with its U^k and Cn parts) with the oracle."""
    import bench
    level = 6
    leaves = synth.uniform_leaves(3, level)
    om = OMesh(3, level, leaves)
    gm = chns.Mesh(3, level, leaves)
    cfg, U = bench.workload_state(om.x)
    o = Oracle(om)
    oprm = OParams(**cfg)
    prm = chns.Params.make(**cfg)
    U = torch.tensor(U)
    U[:, 5] = 0.1 * torch.tensor(synth.random_vectors(om.N, 1, 6)[0])
    Un = U + 1e-4 * torch.tensor(synth.random_vectors(U.numel(), 1, 7)[0]).reshape(U.shape)
    Un[torch.tensor(om.boundary), :3] = 0.0
    dev = torch.device("cuda")
    Ud, Und = U.to(dev), Un.to(dev)
    assert rel(chns.residual(gm, prm, Ud, Und), o.residual(oprm, U, Un)) <= TOL64
    X = synth.random_vectors(U.numel(), 2, 501)
    for i in range(2):
        x = torch.tensor(X[i]).reshape(U.shape)
        yo = o.jvp(oprm, U, Un, x)
        assert rel(chns.jvp(gm, prm, Ud, Und, x.to(dev)), yo) <= TOL64, i
        if i == 0:
            f = lambda t: t.to(dev, torch.float32)
            y32 = chns.jvp(gm, prm, f(U), f(Un), f(x))
            assert rel(y32.double(), yo) <= TOL32
    w = torch.tensor(synth.random_vectors(U.numel(), 1, 502)[0]).reshape(U.shape)
    gn, go, gc = chns.vjp(gm, prm, Ud, Und, w.to(dev))
    gno, goo, gco = o.vjp(oprm, U, Un, w)
    assert rel(gn, gno) <= TOL64
    assert rel(go, goo) <= TOL64
    assert abs(float(gc.cpu()[0]) - float(gco)) <= 1e-11 * max(1.0, abs(float(gco)))


def test_fma_peak_probe(chns):
    """The measured CUDA-core FMA rates behind the ALU rooflines are in the range the
    unit counts allow: FP32 at most 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s
    (above half of it), FP64 well below FP32."""
    f32 = chns.fma_peak(1, 20000)
    f64 = chns.fma_peak(0, 2000)
    assert 40e12 < f32 < 82e12, f32
    assert 0.1e12 < f64 < f32 / 8, (f64, f32)


def test_misaligned_3d_rows_are_rejected(chns):
    """3D node rows are read in pairs, so a vector that does not start on a 16-byte (FP64)
    or 8-byte (FP32) boundary is refused on the host before any kernel runs."""
    import ctypes
    level = 2
    gm = chns.Mesh(3, level, synth.uniform_leaves(3, level))
    prm = chns.Params.make(**synth.config_params("drop3d"))
    n = gm.N * 6
    buf = torch.zeros(2 * n + 4, dtype=torch.float64, device="cuda")
    good = ctypes.c_void_p(buf.data_ptr())
    bad = ctypes.c_void_p(buf.data_ptr() + 8)
    out = ctypes.c_void_p(buf.data_ptr() + 8 * (n + 2))
    lib = chns.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.chns_residual(gm.handle, ctypes.byref(prm), bad, good, out, s) == 1
    assert lib.chns_jvp(gm.handle, ctypes.byref(prm), good, bad, good, out, 0, s) == 1
    assert lib.chns_residual(gm.handle, ctypes.byref(prm), good, good, out, s) == 0
    torch.cuda.synchronize()
