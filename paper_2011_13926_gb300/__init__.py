"""GB300 (sm_103a) implementation of the time-implicit grey M1 radiation step
(Bloch et al., A&A 2021): CUDA kernels behind the C ABI of include/m1.h, with a
thin ctypes binding (``paper_2011_13926_gb300.m1``)."""
from .m1 import (BC, MEM_DEVICE, MEM_HOST, PREC_FP64, PREC_MIXED, PRECOND_BJ, PRECOND_NONE,  # noqa: F401
                 Context, M1Error, context_from_problem, default_opts, grid_desc, load)
