"""Octree leaf lists for the synthetic workloads (Section 4: top-down refinement by a
user predicate, then 2:1 balancing).

A leaf is ``(x, y, z, level)``: the integer anchor of the octant in units of the
finest cell (``2**max_level`` cells per axis), and its level.  ``z`` is 0 in 2D.
Leaves are returned as an ``(n, 4)`` int32 array sorted in Morton (Z) order of
their anchors, which for a complete, non-overlapping octree is a total order.

Balancing enforces the full (face, edge and vertex) 2:1 condition: any two
leaves that share at least one point differ by at most one level.
"""
import numpy as np


def morton_encode(coords, bits):
    """Interleave the bits of integer coordinates ``coords`` (n, d); x varies fastest."""
    coords = np.asarray(coords, dtype=np.int64)
    n, d = coords.shape
    key = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        for k in range(d):
            key |= ((coords[:, k] >> b) & 1) << (b * d + k)
    return key


def leaves_to_array(anchors, levels, dim):
    anchors = np.asarray(anchors, dtype=np.int64)
    out = np.zeros((anchors.shape[0], 4), dtype=np.int32)
    out[:, :dim] = anchors[:, :dim]
    out[:, 3] = levels
    return out


def _sort_morton(anchors, levels, max_level):
    key = morton_encode(anchors, max_level)
    order = np.argsort(key, kind="stable")
    return anchors[order], levels[order]


def _children(anchors, levels, max_level, dim):
    size_child = (np.int64(1) << (max_level - levels - 1))
    out_a, out_l = [], []
    for c in range(1 << dim):
        off = np.array([(c >> k) & 1 for k in range(dim)], dtype=np.int64)
        out_a.append(anchors + off[None, :] * size_child[:, None])
        out_l.append(levels + 1)
    return np.concatenate(out_a), np.concatenate(out_l)


def uniform_leaves(dim, level):
    """All octants of one level, Morton-sorted; max_level == level."""
    n = 1 << level
    grids = np.meshgrid(*[np.arange(n, dtype=np.int64)] * dim, indexing="ij")
    anchors = np.stack([g.reshape(-1) for g in grids], axis=1)
    levels = np.full(anchors.shape[0], level, dtype=np.int64)
    anchors, levels = _sort_morton(anchors, levels, level)
    return leaves_to_array(anchors, levels, dim)


def refine_leaves(dim, min_level, max_level, predicate):
    """Top-down refinement: start from the uniform ``min_level`` grid and split every
    octant for which ``predicate(lo, hi, level)`` is true (``lo``, ``hi``: (n, d) physical
    corners in [0, 1]) until ``max_level``.  Returns Morton-sorted, *unbalanced* leaves."""
    n = 1 << min_level
    step = np.int64(1) << (max_level - min_level)
    grids = np.meshgrid(*[np.arange(n, dtype=np.int64) * step] * dim, indexing="ij")
    active_a = np.stack([g.reshape(-1) for g in grids], axis=1)
    active_l = np.full(active_a.shape[0], min_level, dtype=np.int64)
    done_a, done_l = [], []
    scale = 1.0 / float(1 << max_level)
    while active_a.shape[0]:
        size = (np.int64(1) << (max_level - active_l))
        lo = active_a * scale
        hi = (active_a + size[:, None]) * scale
        flag = (active_l < max_level) & np.asarray(predicate(lo, hi, active_l), dtype=bool)
        done_a.append(active_a[~flag])
        done_l.append(active_l[~flag])
        active_a, active_l = _children(active_a[flag], active_l[flag], max_level, dim)
    anchors = np.concatenate(done_a)
    levels = np.concatenate(done_l)
    anchors, levels = _sort_morton(anchors, levels, max_level)
    return leaves_to_array(anchors, levels, dim)


def balance_leaves(leaves, dim, max_level):
    """Enforce full 2:1 balance by repeatedly splitting any leaf that shares a point
    with a leaf more than one level finer.  Uses the fact that in a complete Morton-
    sorted octree the leaf containing point p is the last leaf whose anchor key is
    <= key(p)."""
    anchors = leaves[:, :dim].astype(np.int64)
    levels = leaves[:, 3].astype(np.int64)
    n_side = np.int64(1) << max_level
    dirs = np.array(np.meshgrid(*[[-1, 0, 1]] * dim, indexing="ij")).reshape(dim, -1).T
    dirs = dirs[np.any(dirs != 0, axis=1)]
    while True:
        keys = morton_encode(anchors, max_level)
        size = np.int64(1) << (max_level - levels)
        mark = np.zeros(anchors.shape[0], dtype=bool)
        for dvec in dirs:
            p = anchors.copy()
            for k in range(dim):
                if dvec[k] < 0:
                    p[:, k] = anchors[:, k] - 1
                elif dvec[k] > 0:
                    p[:, k] = anchors[:, k] + size
            ok = np.all((p >= 0) & (p < n_side), axis=1)
            if not np.any(ok):
                continue
            src = np.nonzero(ok)[0]
            idx = np.searchsorted(keys, morton_encode(p[src], max_level), side="right") - 1
            bad = levels[idx] < levels[src] - 1
            mark[idx[bad]] = True
        if not np.any(mark):
            break
        ca, cl = _children(anchors[mark], levels[mark], max_level, dim)
        anchors = np.concatenate([anchors[~mark], ca])
        levels = np.concatenate([levels[~mark], cl])
        anchors, levels = _sort_morton(anchors, levels, max_level)
    return leaves_to_array(anchors, levels, dim)


def sphere_band_leaves(dim, min_level, max_level, centers, radii, band):
    """Refine to ``max_level`` every octant that may meet the shell ``| |x-c| - R | <= band``
    of any sphere (circle in 2D), then 2:1-balance."""
    centers = np.asarray(centers, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)

    def pred(lo, hi, level):
        mid = 0.5 * (lo + hi)
        half_diag = 0.5 * np.sqrt(np.sum((hi - lo) ** 2, axis=1))
        hit = np.zeros(lo.shape[0], dtype=bool)
        for c, r in zip(centers, radii):
            dist = np.sqrt(np.sum((mid - c[None, :dim]) ** 2, axis=1))
            hit |= np.abs(dist - r) <= band + half_diag
        return hit

    return balance_leaves(refine_leaves(dim, min_level, max_level, pred), dim, max_level)


def plane_band_leaves(dim, min_level, max_level, z0, amplitude, wavelength, phase, band):
    """Refine to ``max_level`` every octant that may meet the band around the surface
    ``x_last = z0 + amplitude*cos(2*pi*x_0/wavelength + phase)``, then 2:1-balance."""
    slope = 2.0 * np.pi * abs(amplitude) / wavelength

    def pred(lo, hi, level):
        mid = 0.5 * (lo + hi)
        half_diag = 0.5 * np.sqrt(np.sum((hi - lo) ** 2, axis=1))
        zi = z0 + amplitude * np.cos(2.0 * np.pi * mid[:, 0] / wavelength + phase)
        return np.abs(mid[:, dim - 1] - zi) <= band + half_diag * (1.0 + slope)

    return balance_leaves(refine_leaves(dim, min_level, max_level, pred), dim, max_level)


def graded_band_leaves(dim, min_level, max_level, dist, band, grade=3.0):
    """Refine every octant of level l < max_level whose centre lies within
    ``band + grade * sqrt(dim) * size_l`` of a surface given by the distance function
    ``dist(points) -> |distance|``.  The margin growing with the octant size grades the
    refinement so that neighbouring leaves differ by at most one level for smooth
    surfaces (checked by the caller's mesh validation; ``balance_leaves`` repairs any
    remaining violation).  Returns Morton-sorted leaves."""
    def pred(lo, hi, level):
        mid = 0.5 * (lo + hi)
        size = hi[:, 0] - lo[:, 0]
        return dist(mid) <= band + grade * np.sqrt(dim) * size

    return refine_leaves(dim, min_level, max_level, pred)


def layer_distance(z0, amplitude, wavelength, phase, dim=3):
    """Approximate distance to x_last = z0 + amplitude cos(2 pi x_0/wavelength + phase)
    (vertical offset divided by the slope factor)."""
    k = 2.0 * np.pi / wavelength

    def dist(p):
        zi = z0 + amplitude * np.cos(k * p[:, 0] + phase)
        slope = amplitude * k * np.sin(k * p[:, 0] + phase)
        return np.abs(p[:, dim - 1] - zi) / np.sqrt(1.0 + slope * slope)

    return dist
