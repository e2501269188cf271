"""Oracle mesh: independent nodes and hanging-node constraints of a 2:1-balanced
octree (Section 4, "Handling hanging nodes").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package.

Conventions (shared with the CUDA path only through the documented C-ABI
behaviour, never through code):
  * Leaves are ``(x, y, z, level)`` integer anchors in units of the finest cell,
    sorted in Morton order; the domain is the cube [lo, hi]^d.
  * Element corner ``a`` (0 <= a < 2^d) sits at anchor + size * bit_k(a) along
    axis k (x is bit 0).
  * A corner is *hanging* when it lies at the midpoint of an edge (one "odd" axis)
    or the centre of a face (two "odd" axes, 3D) of a leaf one level coarser.  Its
    value is then the mean of the 2 (edge) or 4 (face) corners of that edge or face:
    the Q1 interpolant of the coarse side, which keeps the field continuous.
  * Independent nodes are all non-hanging corner points, numbered in Morton order of
    their integer coordinates (max_level + 1 bits per axis).
  * Boundary nodes are those with some coordinate equal to 0 or 2^max_level.
"""
import numpy as np


def _morton(coords, bits):
    coords = np.asarray(coords, dtype=np.int64)
    n, d = coords.shape
    key = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        for k in range(d):
            key |= ((coords[:, k] >> b) & 1) << (b * d + k)
    return key


class Mesh:
    """Plain numpy description of the finite-element mesh of a leaf list."""

    def __init__(self, dim, max_level, leaves, lo=0.0, hi=1.0):
        leaves = np.asarray(leaves, dtype=np.int64)
        self.dim = d = int(dim)
        self.max_level = L = int(max_level)
        self.lo, self.hi = float(lo), float(hi)
        self.nc = nc = 1 << d
        self.nf = d + 3
        anchors = leaves[:, :d]
        level = leaves[:, 3]
        size = np.int64(1) << (L - level)
        self.E = E = leaves.shape[0]
        self.anchors, self.level, self.size = anchors, level, size
        self.h = (self.hi - self.lo) * (0.5 ** level.astype(np.float64))

        bits = np.array([[(a >> k) & 1 for k in range(d)] for a in range(nc)], dtype=np.int64)
        corners = anchors[:, None, :] + bits[None, :, :] * size[:, None, None]  # (E, nc, d)
        cflat = corners.reshape(-1, d)
        sflat = np.repeat(size, nc)
        lflat = np.repeat(level, nc)

        # leaf lookup: key of (anchor, level)
        leaf_key = np.sort(_morton(anchors, L) * 64 + level)

        def is_leaf(anc, lev):
            k = _morton(anc, L) * 64 + lev
            i = np.searchsorted(leaf_key, k)
            i = np.minimum(i, leaf_key.shape[0] - 1)
            return leaf_key[i] == k

        odd = ((cflat // sflat[:, None]) & 1) == 1          # axes where the corner is mid-way
        nodd = odd.sum(axis=1)
        n_side = np.int64(1) << L
        hanging = np.zeros(cflat.shape[0], dtype=bool)
        cand = np.nonzero((nodd >= 1) & (nodd <= 2) & (nodd < d) & (lflat > 0))[0]
        if cand.size:
            c = cflat[cand]
            s = sflat[cand]
            o = odd[cand]
            nfree = d - nodd[cand]
            free_rank = np.cumsum(~o, axis=1) - 1          # rank of each non-odd axis
            # coarse leaves (size 2s) holding c on an edge/face: anchor = c - s on odd
            # axes, c - 2s or c on the other axes
            found = np.zeros(cand.size, dtype=bool)
            for combo in range(1 << (d - 1)):
                shift = ((combo >> np.maximum(free_rank, 0)) & 1).astype(bool) & ~o
                anc = np.where(o, c - s[:, None], np.where(shift, c - 2 * s[:, None], c))
                valid = (combo < (1 << nfree)) & np.all((anc >= 0) & (anc < n_side), axis=1)
                if np.any(valid):
                    idx = np.nonzero(valid)[0]
                    found[idx] |= is_leaf(anc[idx], lflat[cand][idx] - 1)
            hanging[cand[found]] = True

        # independent nodes: every non-hanging corner point
        nb = L + 1
        indep = cflat[~hanging]
        keys = np.unique(_morton(indep, nb))
        self.N = N = keys.shape[0]
        # decode node coordinates from keys
        nodes = np.zeros((N, d), dtype=np.int64)
        for b in range(nb):
            for k in range(d):
                nodes[:, k] |= ((keys >> (b * d + k)) & 1) << b
        self.nodes = nodes
        self.x = self.lo + (self.hi - self.lo) * nodes.astype(np.float64) / float(n_side)
        self.boundary = np.any((nodes == 0) | (nodes == n_side), axis=1)

        def node_index(pts):
            k = _morton(pts, nb)
            i = np.searchsorted(keys, k)
            i = np.minimum(i, N - 1)
            if not np.all(keys[i] == k):
                raise ValueError("constraint parent is not an independent node (mesh not 2:1 balanced)")
            return i

        parents = np.zeros((cflat.shape[0], 4), dtype=np.int64)
        weights = np.zeros((cflat.shape[0], 4), dtype=np.float64)
        nh = ~hanging
        parents[nh, 0] = node_index(cflat[nh])
        weights[nh, 0] = 1.0
        hi_idx = np.nonzero(hanging)[0]
        if hi_idx.size:
            c = cflat[hi_idx]
            s = sflat[hi_idx]
            o = odd[hi_idx]
            no = nodd[hi_idx]
            odd_rank = np.cumsum(o, axis=1) - 1
            for m in range(4):
                use = m < (1 << no)
                if not np.any(use):
                    continue
                up = ((m >> np.maximum(odd_rank, 0)) & 1).astype(bool)
                p = np.where(o, np.where(up, c + s[:, None], c - s[:, None]), c)
                sel = hi_idx[use]
                parents[sel, m] = node_index(p[use])
                weights[sel, m] = 1.0 / (1 << no[use])
        self.parents = parents.reshape(E, nc, 4)
        self.weights = weights.reshape(E, nc, 4)
        self.hanging = hanging.reshape(E, nc)
        # physical corner coordinates (E, nc, d)
        self.corner_x = self.lo + (self.hi - self.lo) * corners.astype(np.float64) / float(n_side)

    def interpolate_at(self, U, points):
        """Values at physical points (P, d) of the conforming Q1 field with nodal values U
        (N, ...): the leaf containing each point (the first one found, searched by brute
        force over all leaves), the point's local coordinates t in [0, 1]^d there, and the
        Q1 weights prod_k (t_k or 1 - t_k) of the leaf's corners, each corner taken through
        its hanging-node parents and weights.  A point on a face shared by two leaves gets
        the same value from either, because the field is continuous."""
        U = np.asarray(U, dtype=np.float64)
        pts = np.asarray(points, dtype=np.float64)
        d = self.dim
        lo = self.anchors.astype(np.float64) / float(1 << self.max_level)
        size = self.size.astype(np.float64) / float(1 << self.max_level)
        lo = self.lo + (self.hi - self.lo) * lo
        size = (self.hi - self.lo) * size
        out = np.zeros((pts.shape[0],) + U.shape[1:])
        for i, p in enumerate(pts):
            inside = np.all((p[None, :] >= lo - 1e-14) & (p[None, :] <= lo + size[:, None] + 1e-14), axis=1)
            e = int(np.nonzero(inside)[0][0])
            t = (p - lo[e]) / size[e]
            val = np.zeros(U.shape[1:])
            for a in range(self.nc):
                w = 1.0
                for k in range(d):
                    w *= t[k] if (a >> k) & 1 else 1.0 - t[k]
                for j in range(4):
                    if self.weights[e, a, j] > 0:
                        val = val + w * self.weights[e, a, j] * U[self.parents[e, a, j]]
            out[i] = val
        return out

    def adapt_flags(self, phi, thr, min_level, max_level):
        """Remeshing flags per element (+1 refine, -1 coarsening candidate, 0 keep): an
        element is near the interface when some corner value of phi (hanging corners: the
        mean of their 2 or 4 parents, summed pairwise) has |phi| < thr."""
        phi = np.asarray(phi, dtype=np.float64)
        P, W = self.parents, self.weights
        npar = (W > 0).sum(axis=2)                         # (E, nc): 1, 2 or 4
        v = phi[P]                                          # (E, nc, 4)
        corner = np.where(npar == 1, v[..., 0],
                          np.where(npar == 2, 0.5 * (v[..., 0] + v[..., 1]),
                                   0.25 * ((v[..., 0] + v[..., 1]) + (v[..., 2] + v[..., 3]))))
        near = np.any(np.abs(corner) < thr, axis=1)
        flags = np.zeros(self.E, dtype=np.int8)
        flags[near & (self.level < max_level)] = 1
        flags[~near & (self.level > min_level)] = -1
        return flags


class MeshQ2:
    """Triquadratic (Q2) elements on a uniform octree of one level (no hanging nodes):
    3^d nodes per element on the lattice of half the element size.  Node coordinates are
    integers in units of 2^-(level + 1); independent nodes are numbered in Morton order of
    those coordinates.  Element node a = a_0 + 3 a_1 (+ 9 a_2), a_k in {0, 1, 2}, sits at
    2 * anchor + a_k along axis k.  Exposes the attributes of ``Mesh`` that the oracle
    uses; every node is independent (weights 1 in slot 0)."""

    order = 2

    def __init__(self, dim, level, lo=0.0, hi=1.0):
        d = self.dim = int(dim)
        L = self.max_level = int(level)
        self.lo, self.hi = float(lo), float(hi)
        self.nc = 3 ** d
        self.nf = d + 3
        n = 1 << L
        grids = np.meshgrid(*[np.arange(n)] * d, indexing="ij")
        anchors = np.stack([g.reshape(-1) for g in grids], axis=1)           # units of 2^-L
        order = np.argsort(_morton(anchors, L))
        self.anchors = anchors[order]
        self.E = anchors.shape[0]
        self.level = np.full(self.E, L, dtype=np.int64)
        self.size = np.ones(self.E, dtype=np.int64)
        self.h = (self.hi - self.lo) * np.full(self.E, 0.5 ** L)
        loc = np.array([[(a // 3 ** k) % 3 for k in range(d)] for a in range(self.nc)], dtype=np.int64)
        pts = 2 * self.anchors[:, None, :] + loc[None, :, :]                  # units of 2^-(L+1)
        keys_all = _morton(pts.reshape(-1, d), L + 2)
        keys = np.unique(keys_all)
        self.N = keys.shape[0]
        nodes = np.zeros((self.N, d), dtype=np.int64)
        for b in range(L + 2):
            for k in range(d):
                nodes[:, k] |= ((keys >> (b * d + k)) & 1) << b
        self.nodes = nodes
        side = 2 * n
        self.x = self.lo + (self.hi - self.lo) * nodes.astype(np.float64) / float(side)
        self.boundary = np.any((nodes == 0) | (nodes == side), axis=1)
        idx = np.searchsorted(keys, keys_all).reshape(self.E, self.nc)
        self.parents = np.zeros((self.E, self.nc, 4), dtype=np.int64)
        self.parents[:, :, 0] = idx
        self.weights = np.zeros((self.E, self.nc, 4))
        self.weights[:, :, 0] = 1.0
        self.hanging = np.zeros((self.E, self.nc), dtype=bool)
        self.corner_x = self.lo + (self.hi - self.lo) * pts.astype(np.float64) / float(side)
