"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package only draws numbers: one-body and two-electron integrals shaped like
the workloads the solver is run on, and the random block entries of initial
iterates.  It contains none of the eigensolver's arithmetic, so both the product
path and the independent CPU oracle may import it.
"""

from .generators import (  # noqa: F401
    spinless_random_chain,
    hubbard_chain,
    molecule_like,
    coulomb_1d,
    random_block_values,
    Workload,
)
