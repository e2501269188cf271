"""Host-side checks of the multigrid hierarchy and of the oracle's Q1 point interpolation
(no GPU): the capped leaf lists that define the coarse levels are complete, 2:1 balanced
and nested (every fine leaf lies inside its mapped coarse leaf), and the oracle's
interpolation, used to check the library's transfer operators, is exact on linear fields
and reproduces nodal values at the nodes."""
import itertools

import numpy as np
import pytest

import synth
from oracle import Mesh


@pytest.fixture(scope="module")
def chns():
    import os
    import paper_2009_06628_gb300 as chns
    if not os.path.exists(chns.LIB_PATH):
        from paper_2009_06628_gb300 import build
        build.build()
    chns.load()
    return chns


def _leaf_lookup(leaves):
    return {(int(l[0]), int(l[1]), int(l[2]), int(l[3])) for l in leaves}


def _containing(lookup, L, p, d):
    for lev in range(L, -1, -1):
        s = 1 << (L - lev)
        a = [(p[k] // s) * s for k in range(d)] + [0] * (3 - d)
        if (a[0], a[1], a[2], lev) in lookup:
            return lev
    return None


def check_complete_balanced(leaves, dim, L):
    """Every finest cell covered exactly once; two leaves that touch (face, edge or
    vertex) differ by at most one level.  Brute force over the finest grid."""
    n = 1 << L
    cover = np.zeros((n,) * dim, dtype=np.int32)
    for x, y, z, lev in leaves:
        s = 1 << (L - lev)
        a = (x, y, z)[:dim]
        cover[tuple(slice(a[k], a[k] + s) for k in range(dim))] += 1
    assert np.all(cover == 1)
    look = _leaf_lookup(leaves)
    for x, y, z, lev in leaves:
        s = 1 << (L - lev)
        a = (x, y, z)[:dim]
        for dv in itertools.product((-1, 0, 1), repeat=dim):
            if not any(dv):
                continue
            p = [a[k] - 1 if dv[k] < 0 else (a[k] + s if dv[k] > 0 else a[k]) for k in range(dim)]
            if any(c < 0 or c >= n for c in p):
                continue
            nl = _containing(look, L, p, dim)
            assert nl is not None and abs(nl - lev) <= 1, ((x, y, z, lev), p, nl)


@pytest.mark.parametrize("dim,L", [(2, 6), (3, 5)])
def test_capped_levels_complete_balanced_nested(chns, dim, L):
    c = [0.45, 0.55, 0.5][:dim]
    leaves = synth.sphere_band_leaves(dim, 1, L, [c], [0.3], 0.03)
    check_complete_balanced(leaves, dim, L)
    cur, cur_L = np.asarray(leaves), L
    while cur_L > 1:
        cap = int(cur[:, 3].max()) - 1
        out, fmap = chns.coarsen_leaves(dim, cur_L, cur, cap)
        assert out[:, 3].max() <= cap
        check_complete_balanced(out, dim, cap)
        # nested: each leaf lies inside the coarse leaf it maps to
        sh = cur_L - cap
        for e in range(0, cur.shape[0], max(1, cur.shape[0] // 500)):
            f, g = cur[e], out[fmap[e]]
            s_c = 1 << (cap - g[3])
            for k in range(dim):
                lo = g[k] << sh
                assert lo <= f[k] and f[k] + (1 << (cur_L - f[3])) <= lo + (s_c << sh)
        # Morton order kept: the map is non-decreasing and hits every coarse leaf
        assert np.all(np.diff(fmap) >= 0) and fmap[0] == 0 and fmap[-1] == out.shape[0] - 1
        cur, cur_L = out, cap


def test_oracle_point_interpolation_pins():
    """Q1 interpolation through hanging nodes is exact for linear fields at arbitrary
    points, and returns the nodal values at the nodes."""
    leaves = synth.sphere_band_leaves(3, 1, 4, [[0.45, 0.55, 0.5]], [0.3], 0.05)
    m = Mesh(3, 4, leaves)
    assert m.hanging.any()
    a = np.array([0.3, -1.1, 0.7])
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.0, 1.0, size=(200, 3))
    U = np.stack([0.2 + m.x @ a, -1.0 + 2.0 * m.x[:, 2]], axis=1)
    v = m.interpolate_at(U, pts)
    assert np.abs(v[:, 0] - (0.2 + pts @ a)).max() < 1e-14
    assert np.abs(v[:, 1] - (-1.0 + 2.0 * pts[:, 2])).max() < 1e-14
    Ur = rng.standard_normal((m.N, 2))
    idx = rng.choice(m.N, 100, replace=False)
    assert np.abs(m.interpolate_at(Ur, m.x[idx]) - Ur[idx]).max() < 1e-14
