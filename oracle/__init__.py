"""CPU oracle of the CHNS hot path (plain FP64 numpy / PyTorch CPU).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
and reference legs of the benchmark may import it; the library never does.
"""
from .mesh import Mesh, MeshQ2
from .chns import Oracle, Params, basis_tables, basis_tables_q2

__all__ = ["Mesh", "MeshQ2", "Oracle", "Params", "basis_tables", "basis_tables_q2"]
