"""Host side of remeshing (no GPU): the adapted leaf list is complete and 2:1 balanced,
every leaf flagged for refinement is split, only complete families flagged for coarsening
merge, and repeated passes that re-evaluate the interface reach a fixed point with the
interface band at the finest level."""
import numpy as np
import pytest

import synth
from oracle import Mesh
from tests.test_multigrid_cpu import check_complete_balanced


@pytest.fixture(scope="module")
def chns():
    import os
    import paper_2009_06628_gb300 as chns
    if not os.path.exists(chns.LIB_PATH):
        from paper_2009_06628_gb300 import build
        build.build()
    chns.load()
    return chns


def _region_levels(leaves, dim, L):
    """Finest-grid array of the level of the leaf covering each finest cell."""
    n = 1 << L
    lev = np.full((n,) * dim, -1, dtype=np.int32)
    for x, y, z, l in leaves:
        s = 1 << (L - l)
        a = (x, y, z)[:dim]
        lev[tuple(slice(a[k], a[k] + s) for k in range(dim))] = l
    return lev


@pytest.mark.parametrize("dim,L", [(2, 6), (3, 5)])
def test_adaptation_pass(chns, dim, L):
    leaves = synth.sphere_band_leaves(dim, 2, L - 1, [[0.45, 0.55, 0.5][:dim]], [0.3], 0.05)
    m = Mesh(dim, L - 1, leaves)
    # the drop has moved: refine around the new interface, coarsen elsewhere
    phi = synth.drop_phi(m.x, [[0.55, 0.45, 0.5][:dim]], [0.25], 0.03)
    flags = m.adapt_flags(phi, 0.9, 2, L)
    assert (flags == 1).any() and (flags == -1).any()
    out, Lo = chns.adapt_leaves(dim, L - 1, leaves, flags, 2, L)
    assert Lo == L
    check_complete_balanced(out, dim, Lo)
    before = _region_levels(np.concatenate([leaves[:, :3] << 1, leaves[:, 3:]], axis=1), dim, L)
    after = _region_levels(out, dim, L)
    # every leaf flagged +1 is split; nothing is coarsened by more than one level, and only
    # where the whole family was flagged -1
    fl_region = np.zeros_like(before)
    for (x, y, z, l), f in zip(leaves, flags):
        s = 1 << (L - l)
        a = (2 * x, 2 * y, 2 * z)[:dim]
        fl_region[tuple(slice(a[k], a[k] + s) for k in range(dim))] = f
    assert np.all(after[fl_region == 1] > before[fl_region == 1])
    assert np.all(after >= before - 1)
    assert np.all((after >= before) | (fl_region == -1))


def test_repeated_passes_reach_the_target(chns):
    dim, L, lmin = 2, 7, 2
    leaves, Lc = synth.uniform_leaves(dim, 3), 3
    centre = [[0.52, 0.47]]
    for _ in range(10):
        m = Mesh(dim, Lc, leaves)
        phi = synth.drop_phi(m.x, centre, [0.25], 0.02)
        flags = m.adapt_flags(phi, 0.9, lmin, L)
        if not (flags == 1).any() and not (flags == -1).any():
            break
        leaves, Lc = chns.adapt_leaves(dim, Lc, leaves, flags, lmin, L)
    m = Mesh(dim, Lc, leaves)
    phi = synth.drop_phi(m.x, centre, [0.25], 0.02)
    flags = m.adapt_flags(phi, 0.9, lmin, L)
    near = np.zeros(m.E, dtype=bool)
    corner = (m.weights * phi[m.parents]).sum(-1)
    near = np.any(np.abs(corner) < 0.9, axis=1)
    assert Lc == L and np.all(m.level[near] == L)
    assert not (flags == 1).any()
    check_complete_balanced(leaves, dim, Lc)
