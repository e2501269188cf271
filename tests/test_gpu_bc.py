"""Non-homogeneous and mixed velocity boundary conditions on the GPU (Section 5 set-ups):
a lid-driven cavity (moving top face, no-slip elsewhere) and the rising-bubble walls
(v_1 = 0 with d v_2/dx = 0 on the side walls, no-slip at top and bottom).  Residual,
FP64 / FP32 J x and J^T w against the oracle with the same conditions, and a Newton step
that lands on the prescribed velocities and matches FP64."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import Mesh as OMesh, Oracle, Params as OParams

pytestmark = pytest.mark.gpu


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


def lid_profile(x):
    """Regularised lid velocity 16 x^2 (1 - x)^2 (times the same in y in 3D): zero at the
    lid's edges, so no corner singularity."""
    d = x.shape[1]
    g = np.zeros_like(x)
    prof = 16.0 * x[:, 0] ** 2 * (1.0 - x[:, 0]) ** 2
    if d == 3:
        prof = prof * 16.0 * x[:, 1] ** 2 * (1.0 - x[:, 1]) ** 2
    g[:, 0] = prof
    return g


CASES = [
    # (dim, kind, level, face masks, use lid values)
    (2, "bubble", 5, [1, 1, 3, 3], False),
    (3, "lid", 4, [7, 7, 7, 7, 7, 7], True),
    (3, "bubble-adaptive", 5, [1, 1, 7, 7, 7, 7], False),
]


@pytest.mark.parametrize("dim,kind,level,fm,lid", CASES, ids=[c[1] + str(c[0]) for c in CASES])
def test_boundary_conditions_parity_and_newton(chns, dim, kind, level, fm, lid):
    if kind.endswith("adaptive"):
        leaves = synth.sphere_band_leaves(dim, 2, level, [[0.5] * dim], [0.25], 0.05)
    else:
        leaves = synth.uniform_leaves(dim, level)
    om = OMesh(dim, level, leaves)
    gm = chns.Mesh(dim, level, leaves)
    cfg = synth.config_params("drop3d" if dim == 3 else "drop2d")
    cfg.update(rho_ratio=5.0, eta_ratio=3.0, Fr=1.0)
    prm, oprm = chns.Params.make(**cfg), OParams(**cfg)
    g = lid_profile(om.x) if lid else np.zeros((om.N, dim))
    o = Oracle(om, bc=(fm, g))
    dev = torch.device("cuda")
    gm.set_velocity_bc(fm, torch.tensor(g, device=dev) if lid else None)
    U = np.zeros((om.N, dim + 3))
    U[:, dim + 1] = synth.drop_phi(om.x, [[0.5] * dim], [0.25], cfg["Cn"], noise=1e-3, seed=4)
    U[:, :dim] = synth.fourier_velocity(om.x, 4, 5, 0.1)
    U[:, dim] = 0.05 * synth.random_vectors(om.N, 1, 6)[0]
    Un = U + 1e-3 * synth.random_vectors(U.size, 1, 7)[0].reshape(U.shape)
    Ut, Unt = torch.tensor(U), torch.tensor(Un)
    Ud, Und = Ut.to(dev), Unt.to(dev)
    rel = lambda a, b: float((a.cpu() - b).norm() / b.norm())
    R = chns.residual(gm, prm, Ud, Und)
    Ro = o.residual(oprm, Ut, Unt)
    assert rel(R, Ro) <= 1e-12
    mask = o.dmask.numpy()
    assert np.array_equal(R.cpu().numpy()[:, :dim][mask], (Un[:, :dim] - g)[mask])
    x = torch.tensor(synth.random_vectors(U.size, 1, 8)[0]).reshape(U.shape)
    yo = o.jvp(oprm, Ut, Unt, x)
    assert rel(chns.jvp(gm, prm, Ud, Und, x.to(dev)), yo) <= 1e-12
    f = lambda t: t.to(dev, torch.float32)
    assert rel(chns.jvp(gm, prm, f(Ut), f(Unt), f(x)).double(), yo) <= 1e-5
    gn, go, gc = chns.vjp(gm, prm, Ud, Und, x.to(dev))
    gno, goo, gco = o.vjp(oprm, Ut, Unt, x)
    assert rel(gn, gno) <= 1e-12 and rel(go, goo) <= 1e-12
    # Newton: the step lands on the prescribed velocities and mixed matches FP64
    U0 = Ud.clone()
    U0[:, :dim] = 0.0
    chns.initial_mu(gm, prm, U0)
    kw = dict(rtol=1e-10, atol=1e-14, krylov_rtol=1e-4, restart=60, max_krylov=4000, pc_type=3, pc_degree=3)
    U32, s32 = chns.newton_step(gm, prm, chns.SolverOpts.make(precision=1, **kw), U0)
    U64, s64 = chns.newton_step(gm, prm, chns.SolverOpts.make(precision=0, **kw), U0)
    assert s32.reason == 0 and s64.reason == 0
    assert float((U32 - U64).norm() / U64.norm()) <= 1e-9
    v = U32.cpu().numpy()[:, :dim]
    assert np.abs(v[mask] - g[mask]).max() <= 1e-12
    # natural rows are free: the side-wall tangential velocity is not forced to zero
    if kind.startswith("bubble"):
        side = (om.nodes[:, 0] == 0) & ~np.any(om.nodes[:, 1:] == 0, axis=1) & ~np.any(om.nodes[:, 1:] == (1 << level), axis=1)
        assert np.abs(v[side, 1]).max() > 0.0
