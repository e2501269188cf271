"""chns_mass_static: the mass integral for callers that cannot allocate device memory
at call time (a framework's caching allocator owns the free memory, or cudaMalloc's
implicit synchronisation is not allowed where the value is needed).  It keeps its
reduction scratch in a static device array and must agree with chns_mass.

Collected last on purpose (file name), so that a failure here comes after every
other test has run; it must also pass when run alone in a fresh process."""
import ctypes
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


@pytest.mark.parametrize("dim,kind", [(2, "uniform"), (3, "adaptive")])
def test_mass_static_matches_mass_on_two_calls(chns, dim, kind):
    if kind == "uniform":
        level = 6
        leaves = synth.uniform_leaves(dim, level)
    else:
        level = 5
        leaves = synth.sphere_band_leaves(dim, 2, level, [[0.45, 0.55, 0.5]], [0.3], 0.03)
    gm = chns.Mesh(dim, level, leaves)
    x = gm.node_x()
    lib = chns.load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((3, 4)):
        U = np.zeros((gm.N, dim + 3))
        U[:, dim + 1] = synth.drop_phi(x, [[0.5] * dim], [0.2 + 0.05 * call], 0.02, noise=1e-3, seed=seed)
        Ud = torch.tensor(U, device="cuda")
        expected = chns.mass(gm, Ud)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        code = lib.chns_mass_static(gm.handle, ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    stream)
        assert code == 0, lib.chns_last_error().decode()
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the library's kernels; the second takes no device memory
            assert torch.cuda.mem_get_info()[0] == free_before
        got = float(out.cpu()[0])
        assert abs(got - expected) <= TOL * max(1.0, abs(expected)), (call, got, expected)
