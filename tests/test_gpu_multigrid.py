"""Transfer operators and the multigrid-preconditioned Newton step on the GPU.

Transfer: the library's P (Q1 interpolation from one mesh to the nodes of another,
hanging constraints included) against the oracle's brute-force point interpolation, in
both directions between an adaptive mesh and its capped coarse level, and P^T against
the adjoint identity.  Newton: the multigrid pressure preconditioner (pc_type 3) only
changes how GMRES converges, so the mixed step must land on the FP64 step of the
Chebyshev preconditioner to 1e-9, conserve int phi and take fewer GMRES iterations."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import Mesh as OMesh

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


@pytest.mark.parametrize("dim,L", [(2, 6), (3, 5)])
def test_transfer_matches_oracle_interpolation(chns, dim, L):
    c = [0.45, 0.55, 0.5][:dim]
    fine = synth.sphere_band_leaves(dim, 2, L, [c], [0.3], 0.03)
    coarse, _ = chns.coarsen_leaves(dim, L, fine, L - 1)
    gf, gc = chns.Mesh(dim, L, fine), chns.Mesh(dim, L - 1, coarse)
    of, oc = OMesh(dim, L, fine), OMesh(dim, L - 1, coarse)
    assert of.hanging.any() and oc.hanging.any()
    rng = np.random.default_rng(5)
    uc = rng.standard_normal((gc.N, 3))
    uf = rng.standard_normal((gf.N, 3))
    dev = torch.device("cuda")
    up = chns.Transfer(gc, gf)                       # prolongation: coarse -> fine nodes
    down = chns.Transfer(gf, gc)                     # coarse nodes take the fine field's values
    got_up = up.apply(torch.tensor(uc, device=dev)).cpu().numpy()
    got_down = down.apply(torch.tensor(uf, device=dev)).cpu().numpy()
    assert np.abs(got_up - oc.interpolate_at(uc, of.x)).max() <= 1e-13
    assert np.abs(got_down - of.interpolate_at(uf, oc.x)).max() <= 1e-13
    # P^T: <P u, v> = <u, P^T v>
    v = torch.tensor(rng.standard_normal((gf.N, 3)), device=dev)
    u = torch.tensor(uc, device=dev)
    lhs = float((up.apply(u) * v).sum())
    rhs = float((u * up.apply(v, transpose=True)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # refining then coarsening a coarse field returns it (coarse nodes are fine nodes)
    assert np.abs(down.apply(up.apply(u)).cpu().numpy() - uc).max() <= 1e-14


def test_multigrid_newton_step(chns):
    """Reduced two-drop workload (levels 3-7, ratios 100/50): two mixed Newton steps with
    the multigrid pressure preconditioner against FP64 steps with the Chebyshev one."""
    import bench

    class Args:
        mesh, level = "twodrops_l7", 6

    gm, cfg, U = bench.workload_mesh(chns, Args)
    prm = chns.Params.make(**cfg)
    U0 = torch.tensor(U, device="cuda")
    chns.initial_mu(gm, prm, U0)
    kw = dict(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, restart=30, max_krylov=5000)
    omg = chns.SolverOpts.make(precision=1, pc_type=3, pc_degree=3, **kw)
    och = chns.SolverOpts.make(precision=1, pc_type=1, pc_degree=16, **kw)
    o64 = chns.SolverOpts.make(precision=0, pc_type=1, pc_degree=16, **kw)
    m0 = chns.mass(gm, U0)
    Umg, Uch, U64 = U0, U0, U0
    it_mg = it_ch = 0
    for _ in range(2):
        Umg, smg = chns.newton_step(gm, prm, omg, Umg)
        Uch, sch = chns.newton_step(gm, prm, och, Uch)
        U64, s64 = chns.newton_step(gm, prm, o64, U64)
        assert smg.reason == 0 and sch.reason == 0 and s64.reason == 0
        assert float((Umg - U64).norm() / U64.norm()) <= 1e-9
        assert abs(chns.mass(gm, Umg) - m0) <= 1e-12 * max(1.0, abs(m0))
        it_mg += smg.krylov_its
        it_ch += sch.krylov_its
    assert it_mg < it_ch, (it_mg, it_ch)
