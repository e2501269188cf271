"""Host-side emulation of the partitioned (multi-GPU) operator application: the element
list split into contiguous Morton ranges, each range evaluated on its own and the
partial node vectors summed (the halo sum), equals the single-range result on every row
that is not a Dirichlet row (those are overwritten after the sum).  Checked with the
oracle for the residual and for J x, on 2:1-balanced meshes with hanging nodes."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from tests.helpers import drop_state, make_mesh, params


@pytest.mark.parametrize("dim,level,parts", [(2, 5, 2), (3, 3, 3)])
def test_partitioned_ranges_plus_halo_sum_equal_single_range(dim, level, parts):
    _, m = make_mesh("adaptive", dim, level)
    assert m.hanging.any()
    prm = params("drop3d" if dim == 3 else "drop2d")
    o, U, Un = drop_state(m, prm, perturb=1e-2)
    E = m.E
    cuts = np.linspace(0, E, parts + 1).astype(np.int64)
    x = torch.tensor(np.random.default_rng(3).standard_normal(U.shape))
    R_full = o.residual(prm, U, Un)
    y_full = o.jvp(prm, U, Un, x)
    R_sum = torch.zeros_like(R_full)
    y_sum = torch.zeros_like(y_full)
    for p in range(parts):
        sub = Oracle(m, elements=np.arange(cuts[p], cuts[p + 1]))
        R_sum += sub.residual(prm, U, Un)
        y_sum += sub.jvp(prm, U, Un, x)
    free = torch.ones(R_full.shape, dtype=torch.bool)
    free[torch.tensor(np.nonzero(m.boundary)[0]), :dim] = False
    for a, b in ((R_sum, R_full), (y_sum, y_full)):
        err = float((a[free] - b[free]).abs().max())
        assert err <= 1e-12 * float(b[free].abs().max())
