"""GB300 (sm_103a) DGSEM library: semi-discrete operator of the compressible
Navier-Stokes equations with BR1 lifting, LSERK4(5) time stepping and its
discrete adjoint (Krais et al., FLEXI, Sec. 3.1 and 3.4), behind the C ABI of
include/flexi.h.  Importing the package does not load the shared library;
``paper_1910_02858_gb300.flexi.lib()`` does, and raises if it is missing.
"""
from .solver import Solver, SolverConfig  # noqa: F401
