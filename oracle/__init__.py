"""CPU oracle for the grey M1 radiation step — TEST INFRASTRUCTURE.

A plain, slow FP64 restatement of the discretisation of Bloch et al. (2021),
Sects. 2-3 and Appendices B-C, used to check the CUDA library. Only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it; the library never does, and the two share no code. Inputs come from
``seeded_inputs`` (data only).

Pinned by tests/test_oracle_*.py against closed forms, limits, invariants,
brute force and the values the paper prints. Parity unpinned beyond the oracle
itself: the whole implicit step at scale (no closed form exists; the pins cover
each ingredient).
"""
from .m1 import Closure, Scheme, eigenvalues  # noqa: F401
from .solvers import (block_jacobi, block_tridiagonal_part, dense_jacobian, dense_solve, gmres,  # noqa: F401
                      newton_solve)
