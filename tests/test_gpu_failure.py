"""Failure detection without a GPU fault: the bounded device-side wait of the
grid barrier is made to run out on a counter that nothing advances; the
host reads the timeout status and the context stays usable."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SPFC_OK, SPFC_EINVAL, SPFC_ETIMEOUT = 0, 1, 5


def test_bounded_wait_expires_with_a_status_and_the_context_survives():
    from paper_2012_15133_gb300 import load_library, Solver
    from seeded_inputs import noisy_field
    lib = load_library()
    t0 = time.perf_counter()
    assert lib.spfc_wait_selftest(1, 1 << 16, None) == SPFC_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    assert lib.spfc_wait_selftest(0, 1 << 16, None) == SPFC_OK       # already satisfied
    assert lib.spfc_wait_selftest(1, -1, None) == SPFC_EINVAL
    assert lib.spfc_wait_selftest(1, 1 << 30, None) == SPFC_EINVAL
    s = Solver(2, 32, 16.0, 0.1, 1.0, 0.01, "fp64")
    s.init(noisy_field((32, 32), 0.2, 0.05, 5), "bdf1")
    s.step(5)
    e = s.energy()
    assert all(np.isfinite(e))
    assert s.sav_scalars()["nsteps"] == 6
