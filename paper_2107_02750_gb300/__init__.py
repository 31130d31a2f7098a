"""GB300 (sm_103a) DG2 / multiwavelet-MRA flood solver.

Method: Sharifian & Kesserwani, "Benchmarking (multi)wavelet-based dynamic and
static non-uniform grid solvers for flood inundation modelling" (arXiv
2107.02750): the DG2 shallow-water step (Sect. 2.1.1, Eq. 1-4) on uniform,
static non-uniform (Sect. 2.2, 2.2.1) and adaptive MWDG2 (Sect. 2.3) grids,
with the multiwavelet MRA (Eq. 9-10) that builds them.

All computation runs in the CUDA library ``libmwdg`` (``csrc/``, C ABI in
``include/mwdg.h``); :mod:`.binding` marshals arguments to it.  There is no CPU
fallback: without the built library and a GPU the calls raise.
"""
from .binding import (Solver, Ensemble, MwdgError, fma_rate, lib, solver_from_problem, UNIFORM, STATIC, ADAPTIVE,
                      F64, F32, DG2, FV1, ACC, WALL, OPEN, WEST, EAST, SOUTH, NORTH)

__all__ = ["Solver", "Ensemble", "MwdgError", "fma_rate", "lib", "solver_from_problem", "UNIFORM", "STATIC", "ADAPTIVE",
           "F64", "F32", "DG2", "FV1", "ACC", "WALL", "OPEN", "WEST", "EAST", "SOUTH", "NORTH"]
