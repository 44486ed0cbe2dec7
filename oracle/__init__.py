"""CPU oracle for the grey M1 radiation step — TEST INFRASTRUCTURE.

A plain, slow FP64 restatement of the discretisation of Bloch et al. (2021),
Sects. 2-3 and Appendices B-C, used to check the CUDA library. Only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it; the library never does, and the two share no code. Inputs come from
``seeded_inputs`` (data only).

Pinned by tests/test_oracle_*.py against closed forms, limits, invariants,
brute force and the values the paper prints. The whole implicit step has no
closed form; it is pinned through its ingredients and in its diffusive limit
(one thick step against Eq. discreteDiffusionEqua; the Marshak wave of Sect. 5.1
against the diffusion reference of oracle/diffusion.py, AP 1.1 % and HLL 81 %
where the paper prints 1.1 % and 84 %; a Gaussian in a thick scattering medium
against the analytic solution of Eq. diffusionEqua under refinement). The
opacity-jump run of Sect. 5.2 reproduces the paper's > 20x flux peak with the
centred source and none with the well-balanced one. The admissibility fallback
(Scheme(fallback=...), newton_solve(realizability=True)) is pinned by its
reduction to HLL with fixed speeds and the centred source, the M1 flux-split
property that makes that scheme admissible, and admissible converged steps on
the beam and two-slab workloads where the AP + WB solution is not.
"""
from .m1 import Closure, Scheme, eigenvalues  # noqa: F401
from .solvers import (admissible_theta, block_jacobi, block_tridiagonal_part, dense_jacobian, dense_solve, gmres,  # noqa: F401
                      newton_solve)
