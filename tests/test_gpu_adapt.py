"""Remeshing on the GPU (Section 4, re-meshing and interpolation): the device flags equal
the oracle's (bit-exact: the same FP64 corner means and comparisons), the fields move to
the new mesh as the oracle's Q1 interpolation at the new nodes, the phi integral is kept
exactly by refinement and to the interpolation error by coarsening, and a Newton step
on the adapted mesh converges."""
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


def _state(x, dim, centre, Cn):
    U = np.zeros((x.shape[0], dim + 3))
    U[:, dim + 1] = synth.drop_phi(x, [centre], [0.25], Cn)
    U[:, :dim] = synth.fourier_velocity(x, 4, 3, 0.1)
    U[np.any((x <= 0.0) | (x >= 1.0), axis=1), :dim] = 0.0
    return U


@pytest.mark.parametrize("dim,L", [(2, 7), (3, 5)])
def test_adapt_pass_matches_oracle(chns, dim, L):
    c0 = [0.45, 0.55, 0.5][:dim]
    leaves = synth.sphere_band_leaves(dim, 2, L - 1, [c0], [0.25], 0.05)
    gm = chns.Mesh(dim, L - 1, leaves)
    om = OMesh(dim, L - 1, leaves)
    cfg = synth.config_params("drop3d" if dim == 3 else "drop2d")
    # the drop sits off the refined band: the pass refines around it and coarsens the old band
    U = _state(om.x, dim, [0.55, 0.45, 0.5][:dim], 0.03)
    Ud = torch.tensor(U, device="cuda")
    flags = chns.adapt_flags(gm, Ud, 0.9, 2, L).cpu().numpy()
    assert np.array_equal(flags, om.adapt_flags(U[:, dim + 1], 0.9, 2, L))
    new, Un, _ = chns.adapt(gm, Ud, 0.9, 2, L)
    onew = OMesh(dim, new.max_level, new.leaves)
    assert np.array_equal(new.node_coords(), onew.nodes.astype(np.int32))
    ref = om.interpolate_at(U, onew.x)
    assert np.abs(Un.cpu().numpy() - ref).max() <= 1e-14
    # phi integral: exact where the pass only refines; coarsening moves it by the Q1
    # interpolation error of the tanh profile far from the interface (|phi| > 0.9 there)
    m_old, m_new = chns.mass(gm, Ud), chns.mass(new, Un)
    assert abs(m_new - m_old) <= 1e-3 * (1.0 if dim == 2 else 1.0)
    # refinement only (no coarsening: min_level at the current deepest level)
    new_r, Ur, _ = chns.adapt(gm, Ud, 0.9, L, L)
    assert abs(chns.mass(new_r, Ur) - m_old) <= 1e-14
    # the adapted state is a valid Newton starting point
    prm = chns.Params.make(**cfg)
    chns.initial_mu(new, prm, Un)
    opts = chns.SolverOpts.make(rtol=1e-9, atol=1e-14, krylov_rtol=1e-3, precision=1, restart=30, max_krylov=3000,
                                pc_type=3, pc_degree=3)
    U1, st = chns.newton_step(new, prm, opts, Un)
    assert st.reason == 0
    assert abs(chns.mass(new, U1) - chns.mass(new, Un)) <= 1e-12
