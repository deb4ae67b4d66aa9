"""GB300 (sm_103a) library for the hybrid Schwarz/multigrid spectral-element
Poisson solver of J. Stiller, "Nonuniformly weighted Schwarz smoothers for
spectral element multigrid".

The compute path is the C-ABI shared library built from csrc/ (declared in
include/sem_schwarz.h); this package only marshals arguments to it.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import EXPORTS, LIB_PATH, SemError, load_library, sem_config, sem_result  # noqa: F401
from .solver import Batch, Solver, Solver3, make_config  # noqa: F401
