"""Q2 (triquadratic) elements on the GPU against the oracle: node numbering (bit-exact),
residual, J x (FP64 and FP32) and J^T w with its U^k and Cn parts, on uniform meshes in
2D and 3D, and the adjoint identity.  Tolerances as for Q1: relative L2 <= 1e-12 (FP64),
<= 1e-5 (FP32)."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import MeshQ2 as OMeshQ2, Oracle, Params as OParams

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


@pytest.mark.parametrize("dim,level", [(2, 4), (3, 3)])
def test_q2_parity(chns, dim, level):
    om = OMeshQ2(dim, level)
    gm = chns.MeshQ2(dim, level)
    assert gm.N == om.N and gm.E == om.E
    assert np.array_equal(gm.node_coords(), om.nodes.astype(np.int32))
    cfg = synth.config_params("drop3d" if dim == 3 else "drop2d")
    cfg.update(Fr=1.0, rho_ratio=5.0, eta_ratio=3.0)
    prm, oprm = chns.Params.make(**cfg), OParams(**cfg)
    o = Oracle(om)
    x = om.x
    U = np.zeros((om.N, dim + 3))
    U[:, dim + 1] = synth.drop_phi(x, [[0.5] * dim], [0.25], 0.1, noise=1e-3, seed=1)
    U[:, :dim] = synth.fourier_velocity(x, 4, 2, 0.1)
    U[:, dim] = 0.05 * synth.random_vectors(om.N, 1, 3)[0]
    U[:, dim + 2] = 0.1 * synth.random_vectors(om.N, 1, 4)[0]
    Un = U + 1e-3 * synth.random_vectors(U.size, 1, 5)[0].reshape(U.shape)
    U[om.boundary, :dim] = 0.0
    Un[om.boundary, :dim] = 0.0
    Ut, Unt = torch.tensor(U), torch.tensor(Un)
    dev = torch.device("cuda")
    Ud, Und = Ut.to(dev), Unt.to(dev)
    rel = lambda a, b: float((a.cpu().double() - b).norm() / b.norm())
    assert rel(chns.residual(gm, prm, Ud, Und), o.residual(oprm, Ut, Unt)) <= 1e-12
    X = synth.random_vectors(U.size, 2, 6)
    for i in range(2):
        xv = torch.tensor(X[i]).reshape(U.shape)
        yo = o.jvp(oprm, Ut, Unt, xv)
        assert rel(chns.jvp(gm, prm, Ud, Und, xv.to(dev)), yo) <= 1e-12, i
        f = lambda t: t.to(dev, torch.float32)
        assert rel(chns.jvp(gm, prm, f(Ut), f(Unt), f(xv)), yo) <= 1e-5, i
    w = torch.tensor(synth.random_vectors(U.size, 1, 7)[0]).reshape(U.shape)
    gn, go, gc = chns.vjp(gm, prm, Ud, Und, w.to(dev))
    gno, goo, gco = o.vjp(oprm, Ut, Unt, w)
    assert rel(gn, gno) <= 1e-12 and rel(go, goo) <= 1e-12
    assert abs(float(gc.cpu()[0]) - float(gco)) <= 1e-11 * max(1.0, abs(float(gco)))
    # adjoint identity on the device
    xv = torch.tensor(X[0]).reshape(U.shape).to(dev)
    Jx = chns.jvp(gm, prm, Ud, Und, xv)
    a, b = float((w.to(dev) * Jx).sum()), float((gn * xv).sum())
    assert abs(a - b) <= 1e-12 * float(w.norm() * Jx.cpu().norm())
    # Q1-only calls refuse a Q2 mesh on the host
    with pytest.raises(chns.ChnsError):
        chns.mass(gm, Ud)
