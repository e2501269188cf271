"""Newton step (Section 3.4) on the GPU: FP64 against the oracle's direct-solve Newton
step, mixed precision (FP32 J x and preconditioner inside GMRES) against FP64 to
<= 1e-9 relative, mass conservation (Proposition 1), energy decay (Theorem 1) and the
host-side failure reports."""
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


def drop_problem(chns, dim, leaves, max_level, cfg_name, over=None, seed=1, vmax=0.1):
    cfg = synth.config_params(cfg_name)
    cfg.update(over or {})
    gm = chns.Mesh(dim, max_level, leaves)
    x = gm.node_x()
    U = np.zeros((gm.N, dim + 3))
    U[:, dim + 1] = synth.drop_phi(x, [[0.5] * dim], [0.25 if dim == 2 else 0.2], cfg["Cn"], noise=1e-3, seed=seed)
    U[:, :dim] = synth.fourier_velocity(x, 8, seed + 1, vmax)
    bnd = np.any((x <= 0.0) | (x >= 1.0), axis=1)
    U[bnd, :dim] = 0.0
    Ud = torch.tensor(U, device="cuda")
    prm = chns.Params.make(**cfg)
    chns.initial_mu(gm, prm, Ud)
    return gm, prm, cfg, Ud


def test_fp64_newton_matches_oracle(chns):
    leaves = synth.uniform_leaves(2, 5)
    gm, prm, cfg, U0 = drop_problem(chns, 2, leaves, 5, "drop2d")
    om = OMesh(2, 5, leaves)
    o = Oracle(om)
    opts = chns.SolverOpts.make(rtol=1e-12, atol=1e-16, krylov_rtol=1e-8, precision=0, restart=100,
                                max_krylov=4000)
    U1, st = chns.newton_step(gm, prm, opts, U0)
    Uo, hist = o.newton_step(OParams(**cfg), U0.cpu(), rtol=1e-12, atol=1e-16)
    err = float((U1.cpu() - Uo).norm() / Uo.norm())
    assert err <= 1e-9, (err, st.as_dict(), hist)
    assert st.reason == 0 and st.newton_its >= 1


@pytest.mark.parametrize("dim,level", [(2, 6), (3, 4)])
def test_mixed_matches_fp64(chns, dim, level):
    leaves = synth.uniform_leaves(dim, level)
    gm, prm, cfg, U0 = drop_problem(chns, dim, leaves, level, "drop2d" if dim == 2 else "drop3d")
    o64 = chns.SolverOpts.make(rtol=1e-11, atol=1e-16, krylov_rtol=1e-6, precision=0, restart=120,
                               max_krylov=20000)
    o32 = chns.SolverOpts.make(rtol=1e-11, atol=1e-16, krylov_rtol=1e-4, precision=1, restart=120,
                               max_krylov=20000)
    U64, s64 = chns.newton_step(gm, prm, o64, U0)
    U32, s32 = chns.newton_step(gm, prm, o32, U0)
    err = float((U32 - U64).norm() / U64.norm())
    assert err <= 1e-9, (err, s32.as_dict(), s64.as_dict())
    # the converged mixed step has an FP64-accurate residual
    R0 = float(chns.residual(gm, prm, U0, U0).norm())
    R = chns.residual(gm, prm, U0, U32)
    assert float(R.norm()) <= 1e-10 * R0


def test_adaptive_mixed_step_conserves_mass_and_energy(chns):
    leaves = synth.sphere_band_leaves(3, 2, 5, [[0.5, 0.5, 0.5]], [0.2], 0.06)
    gm, prm, cfg, U = drop_problem(chns, 3, leaves, 5, "drop3d", dict(rho_ratio=100.0, eta_ratio=50.0))
    assert gm.H > 0
    opts = chns.SolverOpts.make(rtol=1e-9, atol=1e-16, krylov_rtol=1e-4, precision=1, restart=120,
                                max_krylov=4000, max_newton=15, pc_type=2)
    m0 = chns.mass(gm, U)
    e_prev = sum(chns.energy(gm, prm, U))
    for _ in range(2):
        U, st = chns.newton_step(gm, prm, opts, U, check=False)
        assert st.reason == 0, st.as_dict()
        # Proposition 1: int phi is conserved (every Newton update keeps it, the drift is rounding)
        assert abs(chns.mass(gm, U) - m0) <= 1e-12 * max(1.0, abs(m0)), (chns.mass(gm, U) - m0, st.as_dict())
        e = sum(chns.energy(gm, prm, U))
        assert e <= e_prev + 1e-12
        e_prev = e


def test_adaptive_two_drop_steps_mixed_vs_fp64(chns):
    """Two implicit steps on the reduced two-drop workload (octree levels 3-7, 101,368
    elements, 25,744 hanging points, density / viscosity ratios 100 / 50), mixed and FP64
    along their own trajectories: every step converges, the two agree to 1e-9, the phi
    integral is conserved (Proposition 1) and the total energy does not increase."""
    import bench

    class Args:
        mesh, level = "twodrops_l7", 6

    gm, cfg, U = bench.workload_mesh(chns, Args)
    prm = chns.Params.make(**cfg)
    U0 = torch.tensor(U, device="cuda")
    chns.initial_mu(gm, prm, U0)
    kw = dict(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, restart=30, max_krylov=5000, pc_type=1, pc_degree=16)
    o32, o64 = chns.SolverOpts.make(precision=1, **kw), chns.SolverOpts.make(precision=0, **kw)
    m0 = chns.mass(gm, U0)
    E = [sum(chns.energy(gm, prm, U0))]
    Um, U64 = U0, U0
    for _ in range(2):
        Um, sm = chns.newton_step(gm, prm, o32, Um)
        U64, s64 = chns.newton_step(gm, prm, o64, U64)
        assert sm.reason == 0 and s64.reason == 0
        assert float((Um - U64).norm() / U64.norm()) <= 1e-9
        # Proposition 1: int phi is conserved to rounding along both trajectories
        assert abs(chns.mass(gm, Um) - m0) <= 1e-12 * max(1.0, abs(m0))
        assert abs(chns.mass(gm, U64) - m0) <= 1e-12 * max(1.0, abs(m0))
        E.append(sum(chns.energy(gm, prm, Um)))
    assert all(b <= a + 1e-12 for a, b in zip(E, E[1:])), E


def test_eisenstat_walker_forcing(chns):
    """The adaptive forcing term (ew_eta0 > 0) on the reduced two-drop workload with the
    multigrid pressure + Cahn-Hilliard preconditioner: the first linear solve stops at the
    loose first tolerance (fewer GMRES iterations than with the fixed forcing term), the
    step still reaches the Newton tolerance, the mixed and FP64 steps under the same
    forcing agree to 1e-9, phi is conserved (Proposition 1), and the state agrees with the
    fixed-forcing FP64 step to the accuracy the two stopping tests leave (both stop at a
    relative equilibrated residual of 1e-9)."""
    import bench

    class Args:
        mesh, level = "twodrops_l7", 6

    gm, cfg, U = bench.workload_mesh(chns, Args)
    prm = chns.Params.make(**cfg)
    U0 = torch.tensor(U, device="cuda")
    chns.initial_mu(gm, prm, U0)
    kw = dict(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, restart=30, max_krylov=3000, pc_type=4, pc_degree=2)
    Uf, sf = chns.newton_step(gm, prm, chns.SolverOpts.make(precision=0, **kw), U0)
    Um, sm = chns.newton_step(gm, prm, chns.SolverOpts.make(precision=1, ew_eta0=0.3, **kw), U0)
    Ue, se = chns.newton_step(gm, prm, chns.SolverOpts.make(precision=0, ew_eta0=0.3, **kw), U0)
    assert sf.reason == 0 and sm.reason == 0 and se.reason == 0
    assert se.res_final <= 1e-9 * se.res0 and sm.res_final <= 1e-9 * sm.res0
    assert se.krylov_hist[0] < sf.krylov_hist[0], (list(se.krylov_hist[:6]), list(sf.krylov_hist[:6]))
    assert float((Um - Ue).norm() / Ue.norm()) <= 1e-9
    m0 = chns.mass(gm, U0)
    assert abs(chns.mass(gm, Um) - m0) <= 1e-12 * max(1.0, abs(m0))
    assert abs(chns.mass(gm, Ue) - m0) <= 1e-12 * max(1.0, abs(m0))
    assert float((Ue - Uf).norm() / Uf.norm()) <= 1e-7


def test_newton_reports_failures_on_host(chns):
    leaves = synth.uniform_leaves(2, 4)
    gm, prm, cfg, U0 = drop_problem(chns, 2, leaves, 4, "drop2d")
    opts = chns.SolverOpts.make(max_newton=0, precision=1)
    U1, st = chns.newton_step(gm, prm, opts, U0, check=False)
    assert st.reason == 8                      # CHNS_ENOCONV, statistics still filled
    assert st.res0 > 0 and st.newton_its == 0
    for bad in (chns.SolverOpts.make(restart=0), chns.SolverOpts.make(ew_eta0=1.0),
                chns.SolverOpts.make(ew_eta0=-0.1)):
        with pytest.raises(chns.ChnsError) as e:
            chns.newton_step(gm, prm, bad, U0)
        assert e.value.name == "CHNS_EINVAL"
    Unan = U0.clone()
    Unan[3, 0] = float("nan")
    U2, st = chns.newton_step(gm, prm, chns.SolverOpts.make(), Unan, check=False)
    assert st.reason in (7, 10)                # CHNS_ENAN (or ETAU from the NaN radicand)
