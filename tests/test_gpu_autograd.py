"""Differentiation through the hot path (torch.autograd.Function wrappers over the C-ABI):
the residual's reverse and forward modes, the adjoint of an implicit step, and the
gradient of the free energy after a checkpointed rollout with respect to the initial
phi and Cn, checked against central finite differences; and J^T w against the oracle's
assembled Jacobian on a level-3 3D mesh."""
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


def small_problem(chns, dim=2, level=4, cfg_name="drop2d", seed=1, **over):
    """A drop whose phase field stays within [-0.8, 0.8]: the pull-back clip of phi at
    +-1 is a kink of the residual, where Newton and central differences both lose their
    smoothness, so the derivative checks keep clear of it."""
    leaves = synth.uniform_leaves(dim, level)
    gm = chns.Mesh(dim, level, leaves)
    cfg = synth.config_params(cfg_name)
    cfg.update(over)
    x = gm.node_x()
    U = np.zeros((gm.N, dim + 3))
    U[:, dim + 1] = 0.8 * synth.drop_phi(x, [[0.5] * dim], [0.25], cfg["Cn"] * 2, noise=1e-2, seed=seed)
    U[:, :dim] = synth.fourier_velocity(x, 4, seed + 1, 0.1)
    bnd = np.any((x <= 0.0) | (x >= 1.0), axis=1)
    U[bnd, :dim] = 0.0
    return gm, chns.Params.make(**cfg), cfg, torch.tensor(U, device="cuda")


def test_residual_function_modes(chns):
    from paper_2009_06628_gb300.autograd import Residual
    gm, prm, cfg, U = small_problem(chns)
    U_old = U.clone()
    chns.initial_mu(gm, prm, U_old)
    rnd = lambda seed: torch.tensor(synth.random_vectors(U_old.numel(), 1, seed)[0], device="cuda").reshape(U_old.shape)
    U_new = (U_old + 1e-3 * rnd(3)).contiguous()
    w = rnd(4)
    Cn = torch.tensor(cfg["Cn"], dtype=torch.float64, device="cuda", requires_grad=True)
    Uo = U_old.clone().requires_grad_(True)
    Un = U_new.clone().requires_grad_(True)
    R = Residual.apply(gm, prm, Uo, Un, Cn)
    (R * w).sum().backward()
    gn, go, gc = chns.vjp(gm, prm, U_old, U_new, w)
    # the kernels scatter with atomics, so two launches agree to rounding, not bitwise
    assert torch.allclose(Un.grad, gn, rtol=1e-12, atol=1e-14 * float(gn.abs().max()))
    assert torch.allclose(Uo.grad, go, rtol=1e-12, atol=1e-14 * float(go.abs().max()))
    assert abs(float(Cn.grad) - float(gc[0])) <= 1e-12 * abs(float(gc[0]))
    # forward-mode AD through the Function matches the J x kernel
    import torch.autograd.forward_ad as fwAD
    x = rnd(5)
    Cn0 = torch.tensor(cfg["Cn"], dtype=torch.float64, device="cuda")
    with fwAD.dual_level():
        R_dual = Residual.apply(gm, prm, U_old, fwAD.make_dual(U_new, x), Cn0)
        t = fwAD.unpack_dual(R_dual).tangent
    ref = chns.jvp(gm, prm, U_old, U_new, x)
    assert torch.allclose(t, ref, rtol=1e-12, atol=1e-14 * float(ref.abs().max()))


@pytest.mark.parametrize("dim,cfg_name,dt,n_dirs,eps", [(2, "drop2d", 2e-3, 8, 1e-5),
                                                       (3, "drop3d", 1e-3, 32, 1e-6)])
def test_rollout_gradient_matches_central_differences(chns, dim, cfg_name, dt, n_dirs, eps):
    from paper_2009_06628_gb300.autograd import rollout
    # level-3 meshes (9^d nodes): GMRES(256) with a 1e-12 Krylov tolerance nearly solves
    # each linearisation exactly, so every implicit step is converged far below the
    # finite-difference step and central differences see a smooth map
    gm, prm, cfg, U0 = small_problem(chns, dim=dim, level=3, cfg_name=cfg_name, dt=dt)
    opts = chns.SolverOpts.make(rtol=1e-12, atol=1e-13, krylov_rtol=1e-12, precision=0, restart=256,
                                max_krylov=4000, max_newton=20)
    adj = chns.SolverOpts.make(krylov_rtol=1e-12, restart=256, max_krylov=4000, precision=0)
    n_steps, every = 20, 5
    d = gm.dim

    def loss(phi0, cn, grad=False):
        U = U0.clone()
        U[:, d + 1] = phi0
        return rollout(gm, prm, opts, adj, U, cn, n_steps, every)

    phi0 = U0[:, d + 1].clone().requires_grad_(True)
    Cn = torch.tensor(cfg["Cn"], dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss(phi0, Cn)
    L.backward()
    g_phi, g_cn = phi0.grad.clone(), float(Cn.grad)
    # each step's relative residual is below 1e-12, so solver noise in a central
    # difference is ~1e-12 / eps and truncation ~eps^2, both below the 1e-4 bar
    dirs = synth.random_vectors(gm.N, n_dirs, 77)
    with torch.no_grad():
        for i in range(dirs.shape[0]):
            v = torch.tensor(dirs[i], device="cuda")
            lp = float(loss(phi0 + eps * v, Cn))
            lm = float(loss(phi0 - eps * v, Cn))
            fd = (lp - lm) / (2 * eps)
            ad = float((g_phi * v).sum())
            assert abs(fd - ad) <= 1e-4 * max(abs(fd), 1e-3), (i, fd, ad)
        ec = eps * cfg["Cn"]
        fd = (float(loss(phi0, Cn + ec)) - float(loss(phi0, Cn - ec))) / (2 * ec)
        assert abs(fd - g_cn) <= 1e-4 * max(abs(fd), 1e-3), (fd, g_cn)


def test_vjp_matches_assembled_oracle_jacobian_level3(chns):
    leaves = synth.uniform_leaves(3, 3)
    om = OMesh(3, 3, leaves)
    gm = chns.Mesh(3, 3, leaves)
    cfg = synth.config_params("drop3d")
    o = Oracle(om)
    oprm = OParams(**cfg)
    prm = chns.Params.make(**cfg)
    U = np.zeros((om.N, 6))
    U[:, 4] = synth.drop_phi(om.x, [[0.5, 0.5, 0.5]], [0.3], 0.1, noise=1e-3, seed=9)
    U[:, :3] = synth.fourier_velocity(om.x, 4, 10, 0.1)
    U[om.boundary, :3] = 0.0
    Ut = torch.tensor(U)
    Un = Ut + 1e-3 * torch.tensor(synth.random_vectors(U.size, 1, 11)[0]).reshape(U.shape)
    Un[torch.tensor(om.boundary), :3] = 0.0
    J = o.jacobian(oprm, Ut, Un)
    for seed in (12, 13):
        w = torch.tensor(synth.random_vectors(U.size, 1, seed)[0]).reshape(U.shape)
        gn, _, _ = chns.vjp(gm, prm, Ut.cuda(), Un.cuda(), w.cuda())
        ref = (J.T @ w.reshape(-1)).reshape(U.shape)
        assert float((gn.cpu() - ref).norm() / ref.norm()) <= 1e-12
