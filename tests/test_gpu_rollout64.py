"""Differentiation on the 64^3 mesh of the benchmark (uniform octree level 6, 274,625
nodes x 6 DOF), as the differentiation workload asks: the free energy after a 20-step
rollout (dt = 1e-3, checkpoints every 5 steps) differentiated with respect to the initial
phi field and Cn, against central finite differences (step 1e-6) on seeded directions.

The forward steps are mixed-precision Newton solves (FP32 J x inside GMRES, FP64
residual) driven to a relative residual of 1e-12, so the solver noise in a central
difference (~1e-12 / 1e-6) stays far below the 1e-4 bar; the adjoint solves run with the
FP64 J^T w kernel.  The drop profile is scaled to |phi| <= 0.8 so that the pull-back clip
at +-1 (a kink of the residual) is never active."""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

N_DIRS = 32


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


def test_rollout_gradient_64cubed(chns):
    import bench
    from paper_2009_06628_gb300.autograd import rollout
    level = 6
    gm = chns.Mesh(3, level, synth.uniform_leaves(3, level))
    cfg, U = bench.workload_state(gm.node_x())
    cfg["dt"] = 1e-3
    U[:, 4] *= 0.8
    prm = chns.Params.make(**cfg)
    U0 = torch.tensor(U, device="cuda")
    chns.initial_mu(gm, prm, U0)
    opts = chns.SolverOpts.make(rtol=1e-12, atol=1e-14, krylov_rtol=1e-6, precision=1, restart=60,
                                max_krylov=6000, max_newton=20, pc_type=1, pc_degree=16)
    adj = chns.SolverOpts.make(krylov_rtol=1e-11, restart=120, max_krylov=20000, precision=0)

    def loss(phi0, cn):
        Ux = U0.clone()
        Ux[:, 4] = phi0
        return rollout(gm, prm, opts, adj, Ux, cn, 20, 5)

    phi0 = U0[:, 4].clone().requires_grad_(True)
    Cn = torch.tensor(cfg["Cn"], dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss(phi0, Cn)
    L.backward()
    g_phi, g_cn = phi0.grad.clone(), float(Cn.grad)
    eps = 1e-6
    dirs = synth.random_vectors(gm.N, N_DIRS, 78)
    with torch.no_grad():
        for i in range(N_DIRS):
            v = torch.tensor(dirs[i], device="cuda")
            fd = (float(loss(phi0 + eps * v, Cn)) - float(loss(phi0 - eps * v, Cn))) / (2 * eps)
            ad = float((g_phi * v).sum())
            assert abs(fd - ad) <= 1e-4 * max(abs(fd), 1e-3), (i, fd, ad)
        ec = eps * cfg["Cn"]
        fd = (float(loss(phi0, Cn + ec)) - float(loss(phi0, Cn - ec))) / (2 * ec)
        assert abs(fd - g_cn) <= 1e-4 * max(abs(fd), 1e-3), (fd, g_cn)
