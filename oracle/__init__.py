"""FP64 CPU oracle for the SPFC BDF2-SAV scheme (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package; the CUDA product path never does.
"""
from .spfc_oracle import (Grid, Model, Oracle, A_inv, bdf1_sav_step, bdf2_sav_step, sav_r_update,
                          copy_start, ghost_start)

__all__ = ["Grid", "Model", "Oracle", "A_inv", "bdf1_sav_step", "bdf2_sav_step", "sav_r_update",
           "copy_start", "ghost_start"]
