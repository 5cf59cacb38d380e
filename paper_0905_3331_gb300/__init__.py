"""GB300 (sm_103a) library for the Wilson twisted-mass Dirac operator and its
even/odd-preconditioned CG solve (Jansen & Urbach, tmLQCD, arXiv:0905.3331).

The compute path is the CUDA library built from csrc/ (C ABI in include/tm.h);
``tm`` is its ctypes binding and ``inputs`` draws the seeded synthetic inputs.
"""
from . import build  # noqa: F401  (the module; build.build() compiles the library)
from .tm import (CG_FP64, CG_RELIABLE, CG_SQRT_EPS, DF64, F16, F32, F64, HOP_PAIRED, HOP_PIPELINED, LINK8,  # noqa: F401
                 LINK12, LINK18, Lattice, SolveInfo, TMError, launch_count, load, reset_launch_count,
                 correlator, solve_cg_batch)
