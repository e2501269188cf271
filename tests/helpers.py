"""Shared test fixtures: small meshes (uniform and adaptive with hanging nodes) and
seeded states.  Imports the oracle and the synthetic-input generators only."""
import math

import numpy as np
import torch

import synth
from oracle import Mesh, Oracle, Params


def adaptive_leaves(dim, min_level, max_level, seed=7):
    """A small 2:1-balanced adaptive octree refined around a circle/sphere."""
    c = [0.45, 0.55, 0.5][:dim]
    return synth.sphere_band_leaves(dim, min_level, max_level, [c], [0.3], 0.02)


def make_mesh(kind, dim, level, min_level=None):
    if kind == "uniform":
        leaves = synth.uniform_leaves(dim, level)
    else:
        leaves = adaptive_leaves(dim, min_level if min_level is not None else max(1, level - 2), level)
    return leaves, Mesh(dim, level, leaves)


def drop_state(mesh, prm, seed=1, noise=1e-3, vmax=0.1, perturb=1e-3, mu_from_phi=True):
    """(U_old, U_new) near a drop: phi from a tanh profile + noise, divergence-free
    velocity vanishing on the boundary, mu from the discrete projection, and a
    seeded perturbation for the new level (boundary velocity kept zero)."""
    d = mesh.dim
    c = [0.5] * d
    U = np.zeros((mesh.N, d + 3))
    U[:, d + 1] = synth.drop_phi(mesh.x, [c], [0.25], prm.Cn, noise=noise, seed=seed)
    U[:, :d] = synth.fourier_velocity(mesh.x, 4, seed + 10, vmax)
    U[:, d] = 0.01 * synth.random_vectors(mesh.N, 1, seed + 20)[0]
    U = torch.tensor(U)
    o = Oracle(mesh)
    if mu_from_phi:
        U[:, d + 2] = o.initial_mu(prm, U[:, d + 1])
    rng = np.random.default_rng(seed + 30)
    Un = U + perturb * torch.tensor(rng.standard_normal(U.shape))
    Un[o.bnd, :d] = 0.0
    U[o.bnd, :d] = 0.0
    return o, U, Un


def params(name, **over):
    p = synth.config_params(name)
    p.update(over)
    return Params(**p)
