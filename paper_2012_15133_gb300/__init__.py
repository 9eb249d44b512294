"""GB300 (sm_103a) BDF2-SAV Fourier pseudo-spectral solver for the square
phase field crystal equation.

The compute path is the CUDA library ``libspfc.so`` behind the C interface
``include/spfc.h``; this package only marshals arguments to it (``spfc``
module) and builds it (``build`` module). There is no CPU fallback: using the
solver without the built library raises.
"""
from .spfc import (Solver, SPFCError, lib_path, load_library, FP64, FP32_BULK,
                   START_BDF1, START_GHOST, START_COPY, EXPORTED_SYMBOLS, field_energy_noalloc,
                   num_schedules, Batch, fp64_fma_rate)

__all__ = ["Solver", "SPFCError", "lib_path", "load_library", "FP64", "FP32_BULK",
           "START_BDF1", "START_GHOST", "START_COPY", "EXPORTED_SYMBOLS", "field_energy_noalloc",
           "num_schedules", "Batch", "fp64_fma_rate"]
