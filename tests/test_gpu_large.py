"""Full-size adaptive workload (two drops, octree levels 4-9, refined within 3 Cn of the
interfaces, 2:1 balanced, ~2.5M elements with hanging nodes): node numbering bit-exact,
residual / J x / J^T w rows on seeded samples of nodes against the oracle restricted to
the elements around them, mass and energy against the oracle, and size-independent
properties (mass row-sum, hydrostatic zero) through the kernels alone."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import Mesh as OMesh, Oracle, Params as OParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2009_06628_gb300 as chns
    if not os.path.exists(chns.LIB_PATH):
        from paper_2009_06628_gb300 import build
        build.build()
    chns.load()
    cfg = synth.config_params("twodrops3d")
    centers, radii = synth.two_drops(3)
    leaves = synth.sphere_band_leaves(3, 4, 9, centers, radii, 3 * cfg["Cn"])
    gm = chns.Mesh(3, 9, leaves)
    om = OMesh(3, 9, leaves)
    x = om.x
    U = np.zeros((om.N, 6))
    U[:, 4] = synth.drop_phi(x, centers, radii, cfg["Cn"], noise=1e-3, seed=3)
    U[:, :3] = synth.fourier_velocity(x, 8, 4, 0.1)
    U[:, 3] = 0.05 * synth.random_vectors(om.N, 1, 5)[0]
    U[:, 5] = 0.1 * synth.random_vectors(om.N, 1, 6)[0]
    Un = U + 1e-3 * synth.random_vectors(U.size, 1, 7)[0].reshape(U.shape)
    U[om.boundary, :3] = 0.0
    Un[om.boundary, :3] = 0.0
    rng = np.random.default_rng(8)
    sample = np.sort(rng.choice(om.N, size=400, replace=False))
    touch = np.any(np.isin(om.parents, sample) & (om.weights > 0), axis=(1, 2))
    sub = Oracle(om, elements=np.nonzero(touch)[0])
    return dict(chns=chns, cfg=cfg, leaves=leaves, gm=gm, om=om, U=torch.tensor(U), Un=torch.tensor(Un),
                sample=torch.tensor(sample), sub=sub, prm=chns.Params.make(**cfg), oprm=OParams(**cfg))


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def test_mesh_is_large_adaptive_and_numbered_like_oracle(big):
    gm, om = big["gm"], big["om"]
    assert gm.E > 2_000_000 and gm.H > 0
    assert gm.N == om.N
    assert np.array_equal(gm.node_coords(), om.nodes.astype(np.int32))


def test_sampled_rows_residual_jvp_vjp(big):
    chns, gm, sub = big["chns"], big["gm"], big["sub"]
    U, Un, s = big["U"], big["Un"], big["sample"]
    prm, oprm = big["prm"], big["oprm"]
    Ud, Und = U.cuda(), Un.cuda()
    R = chns.residual(gm, prm, Ud, Und).cpu()
    Ro = sub.residual(oprm, U, Un)
    assert _rel(R[s], Ro[s]) <= 1e-12
    x = torch.tensor(synth.random_vectors(U.numel(), 1, 9)[0]).reshape(U.shape)
    y = chns.jvp(gm, prm, Ud, Und, x.cuda()).cpu()
    yo = sub.jvp(oprm, U, Un, x)
    assert _rel(y[s], yo[s]) <= 1e-12
    y32 = chns.jvp(gm, prm, Ud.float(), Und.float(), x.cuda().float()).cpu().double()
    assert _rel(y32[s], yo[s]) <= 1e-5
    gn, go, _ = chns.vjp(gm, prm, Ud, Und, x.cuda(), want_cn=False)
    gno, goo, _ = sub.vjp(oprm, U, Un, x)
    assert _rel(gn.cpu()[s], gno[s]) <= 1e-12
    assert _rel(go.cpu()[s], goo[s]) <= 1e-12


def test_mass_energy_and_invariants_at_full_size(big):
    chns, gm, om = big["chns"], big["gm"], big["om"]
    U, Un, prm, oprm = big["U"], big["Un"], big["prm"], big["oprm"]
    o = Oracle(om)
    Ud, Und = U.cuda(), Un.cuda()
    m_old, m_new = chns.mass(gm, Ud), chns.mass(gm, Und)
    assert abs(m_new - o.mass(Un)) <= 1e-12 * abs(o.mass(Un))
    e = chns.energy(gm, prm, Und)
    eo = o.energy(oprm, Un)
    for a, b in zip(e, eo):
        assert abs(a - b) <= 1e-11 * abs(b)
    # mass row-sum (Proposition 1) through the kernels alone
    R = chns.residual(gm, prm, Ud, Und)
    lhs = float(R[:, 4].sum())
    rhs = (m_new - m_old) / prm.dt
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))
    # hydrostatic state: every row vanishes
    c = 0.3
    H = torch.zeros_like(Ud)
    rho_c = oprm.alpha * c + oprm.beta
    H[:, 3] = torch.tensor(-(prm.We * rho_c / prm.Fr) * om.x[:, 2] + 0.7, device="cuda")
    H[:, 4] = c
    H[:, 5] = c ** 3 - c
    RH = chns.residual(gm, prm, H, H)
    hmax = 2.0 ** -4
    scale = prm.We * rho_c / prm.Fr * (0.5 * hmax) ** 3 / hmax
    assert float(RH.abs().max()) <= 1e-11 * scale


@pytest.fixture(scope="module")
def layer():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import bench
    import paper_2009_06628_gb300 as chns
    chns.load()
    leaves, level, cfg, phase = bench.layer_workload()
    gm = chns.Mesh(3, level, leaves)
    x = gm.node_x()
    U = np.zeros((gm.N, 6))
    U[:, 4] = synth.layer_phi(x, 0.5, 0.05, 1.0, phase, cfg["Cn"])
    U[:, :3] = synth.fourier_velocity(x, 8, 6, 0.05)
    U[np.any((x <= 0.0) | (x >= 1.0), axis=1), :3] = 0.0
    return dict(chns=chns, gm=gm, cfg=cfg, x=x, U=torch.tensor(U, device="cuda"))


def test_layer_mesh_invariants_at_26M_elements(layer):
    """The ~20M-element layer workload through the kernels alone: mass row-sum
    (Proposition 1), hydrostatic zero, and FP32 J x against FP64 J x."""
    chns, gm, cfg, x, U = layer["chns"], layer["gm"], layer["cfg"], layer["x"], layer["U"]
    assert gm.E > 20_000_000 and gm.H > 0
    prm = chns.Params.make(**cfg)
    gen = torch.Generator(device="cuda").manual_seed(11)
    Un = U + 1e-4 * torch.randn(U.shape, dtype=torch.float64, device="cuda", generator=gen)
    bnd = torch.tensor(np.any((x <= 0.0) | (x >= 1.0), axis=1), device="cuda")
    Un[bnd, :3] = 0.0
    R = chns.residual(gm, prm, U, Un)
    lhs = float(R[:, 4].sum())
    rhs = (chns.mass(gm, Un) - chns.mass(gm, U)) / prm.dt
    assert abs(lhs - rhs) <= 1e-8 * max(1.0, abs(rhs))
    xv = torch.randn(U.shape, dtype=torch.float64, device="cuda", generator=gen)
    y64 = chns.jvp(gm, prm, U, Un, xv)
    y32 = chns.jvp(gm, prm, U.float(), Un.float(), xv.float())
    assert float((y32.double() - y64).norm() / y64.norm()) <= 1e-5
    # hydrostatic state
    oprm = OParams(**cfg)
    c = -0.4
    rho_c = oprm.alpha * c + oprm.beta
    H = torch.zeros_like(U)
    H[:, 3] = torch.tensor(-(prm.We * rho_c / prm.Fr) * x[:, 2] + 0.7, device="cuda")
    H[:, 4] = c
    H[:, 5] = c ** 3 - c
    RH = chns.residual(gm, prm, H, H)
    hmax = 2.0 ** -5
    scale = prm.We * rho_c / prm.Fr * (0.5 * hmax) ** 3 / hmax
    assert float(RH.abs().max()) <= 1e-11 * scale
