"""Scatter strategies of the element kernels: element colouring (deterministic: the same
bits on every run) and warp-aggregated atomics give the results of the default atomic
scatter to rounding, on uniform and hanging-node meshes."""
import os

import numpy as np
import pytest
import torch

import synth

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


@pytest.mark.parametrize("dim,kind,level", [(3, "uniform", 4), (3, "adaptive", 5), (2, "adaptive", 6)])
def test_scatter_modes_agree(chns, dim, kind, level):
    if kind == "uniform":
        leaves = synth.uniform_leaves(dim, level)
    else:
        leaves = synth.sphere_band_leaves(dim, 2, level, [[0.45, 0.55, 0.5][:dim]], [0.3], 0.03)
    gm = chns.Mesh(dim, level, leaves)
    cfg = synth.config_params("drop3d" if dim == 3 else "drop2d")
    cfg.update(rho_ratio=10.0, eta_ratio=5.0, Fr=1.0)
    prm = chns.Params.make(**cfg)
    x = gm.node_x()
    U = np.zeros((gm.N, dim + 3))
    U[:, dim + 1] = synth.drop_phi(x, [[0.5] * dim], [0.25], cfg["Cn"], noise=1e-3, seed=2)
    U[:, :dim] = synth.fourier_velocity(x, 4, 3, 0.1)
    U[:, dim] = 0.05 * synth.random_vectors(gm.N, 1, 4)[0]
    dev = torch.device("cuda")
    U0 = torch.tensor(U, device=dev)
    Un = U0 + 1e-3 * torch.tensor(synth.random_vectors(U.size, 1, 5)[0], device=dev).reshape(U.shape)
    X = torch.tensor(synth.random_vectors(U.size, 1, 6)[0], device=dev).reshape(U.shape)

    def run():
        return (chns.residual(gm, prm, U0, Un), chns.jvp(gm, prm, U0, Un, X),
                chns.jvp(gm, prm, U0.float(), Un.float(), X.float()), chns.vjp(gm, prm, U0, Un, X)[0])

    gm.set_scatter(0)
    ref = run()
    gm.set_scatter(1)
    assert gm.num_colours >= (1 << dim) and gm.num_colours <= 64
    if kind == "uniform":
        assert gm.num_colours == 1 << dim
    col1, col2 = run(), run()
    for a, b in zip(col1, col2):
        assert torch.equal(a, b)             # deterministic: identical bits run to run
    gm.set_scatter(2)
    agg = run()
    for i, (r, c, w) in enumerate(zip(ref, col1, agg)):
        tol = 1e-5 if r.dtype == torch.float32 else 1e-13
        for v in (c, w):
            assert float((v.double() - r.double()).norm() / r.double().norm()) <= tol, i
    gm.set_scatter(0)
