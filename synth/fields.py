"""Seeded nodal fields for the synthetic workloads.

Every generator takes the physical node coordinates ``x`` (N, d) that the caller
obtained from its own mesh, so the oracle and the CUDA path evaluate the same
formulas at the same points.  Random draws use numpy's PCG64 (``default_rng``)
with the seed recorded in the workload description.
"""
import math

import numpy as np


def drop_phi(x, centers, radii, Cn, noise=0.0, seed=None):
    """Phase field of one or more drops (phi = +1 inside): the 1D equilibrium profile
    tanh(s / (sqrt(2) Cn)) of the signed distance s = R - |x - c|, maximised over drops,
    plus optional seeded nodal noise uniform in [-noise, noise]."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    phi = np.full(x.shape[0], -np.inf)
    for c, r in zip(np.asarray(centers, dtype=np.float64), np.asarray(radii, dtype=np.float64)):
        dist = np.sqrt(np.sum((x - c[None, :d]) ** 2, axis=1))
        phi = np.maximum(phi, np.tanh((r - dist) / (math.sqrt(2.0) * Cn)))
    if noise:
        rng = np.random.default_rng(seed)
        phi = phi + rng.uniform(-noise, noise, size=phi.shape[0])
    return phi


def layer_phi(x, z0, amplitude, wavelength, phase, Cn):
    """Two-layer phase field, phi = +1 above the surface
    x_last = z0 + amplitude * cos(2 pi x_0 / wavelength + phase)."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    zi = z0 + amplitude * np.cos(2.0 * np.pi * x[:, 0] / wavelength + phase)
    return np.tanh((x[:, d - 1] - zi) / (math.sqrt(2.0) * Cn))


def fourier_velocity(x, n_modes, seed, vmax, kmax=3):
    """Divergence-free velocity that vanishes on the boundary of the unit box: a seeded
    sum of curls of a_m * psi_m * e_axis with psi_m = prod_k sin^2(pi k_mk x_k), k_mk in
    [1, kmax].  In 2D the stream function form v = (d psi/dy, -d psi/dx) is used.  The
    field is scaled so that max |v| over the given points equals ``vmax``."""
    x = np.asarray(x, dtype=np.float64)
    n, d = x.shape
    rng = np.random.default_rng(seed)
    v = np.zeros((n, d))
    for _ in range(n_modes):
        k = rng.integers(1, kmax + 1, size=d)
        a = rng.normal()
        axis = int(rng.integers(0, 3)) if d == 3 else 2
        s = np.sin(np.pi * k[None, :] * x) ** 2
        ds = 2.0 * np.pi * k[None, :] * np.sin(np.pi * k[None, :] * x) * np.cos(np.pi * k[None, :] * x)
        grad = np.empty((n, d))
        for j in range(d):
            g = ds[:, j].copy()
            for m in range(d):
                if m != j:
                    g *= s[:, m]
            grad[:, j] = g
        if d == 2:
            v[:, 0] += a * grad[:, 1]
            v[:, 1] -= a * grad[:, 0]
        else:
            # curl(psi e_axis) = grad(psi) x e_axis
            e = np.zeros(3)
            e[axis] = 1.0
            v += a * np.cross(grad, e[None, :])
    vm = np.max(np.sqrt(np.sum(v * v, axis=1)))
    if vm > 0:
        v *= vmax / vm
    return v


def two_drops(seed, radii=(0.12, 0.15), distance=0.35):
    """Centres and radii of the two-drop workload: the pair is centred in the unit box
    with a seeded random orientation of the line joining the centres."""
    rng = np.random.default_rng(seed)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    c1 = 0.5 - 0.5 * distance * u
    c2 = 0.5 + 0.5 * distance * u
    return np.stack([c1, c2]), np.array(radii, dtype=np.float64)


def random_vectors(n, count, seed):
    """``count`` seeded N(0, 1) vectors of length n, shape (count, n)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, n))


def config_params(name):
    """Physical parameters of the synthetic workloads (dimensionless groups, density and
    viscosity ratios rho+/rho-, eta+/eta-, time step).  ``Fr = 0`` means no gravity."""
    table = {
        # 2D drop, uniform level 5
        "drop2d": dict(dim=2, Re=100.0, We=10.0, Pe=100.0, Cn=0.05, Fr=0.0, rho_ratio=1.0,
                       eta_ratio=1.0, dt=1e-3),
        # 3D drop, uniform level 6, gravity along -z
        "drop3d": dict(dim=3, Re=100.0, We=10.0, Pe=100.0, Cn=0.02, Fr=1.0, rho_ratio=10.0,
                       eta_ratio=10.0, dt=5e-4),
        # 3D two drops on an adaptive octree
        "twodrops3d": dict(dim=3, Re=100.0, We=10.0, Pe=100.0, Cn=0.005, Fr=1.0,
                           rho_ratio=100.0, eta_ratio=50.0, dt=5e-4),
        # 3D two-layer (Rayleigh-Taylor-shaped) setup, heavy fluid on top
        "layer3d": dict(dim=3, Re=1000.0, We=1000.0, Pe=1000.0, Cn=0.0025, Fr=1.0,
                        rho_ratio=3.0, eta_ratio=1.0, dt=2e-4),
    }
    p = dict(table[name])
    p.setdefault("C_I", 6.0)
    p.setdefault("C_phi", 6.0)
    p.setdefault("pin_pressure", 2)
    return p
