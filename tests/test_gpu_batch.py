"""Batched ensemble (uneven grid sizes and parameters) against single runs and
the oracle, through the C-ABI."""
import numpy as np
import pytest

from oracle import Oracle
from seeded_inputs import ensemble_run, noisy_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu tests")
    from paper_2012_15133_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _runs(sizes, count, dt=0.02):
    return [ensemble_run(i, sizes=sizes) for i in range(count)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_small_ensemble_matches_oracle(precision, tol):
    """Six runs over grids 16, 32, 64 (h = 0.5), drawn eps/beta/mean, 4 steps."""
    from paper_2012_15133_gb300 import Batch
    runs = _runs((16, 32, 64), 6)
    b = Batch(runs, 0.02, precision)
    for i, r in enumerate(runs):
        b.init(i, r["phi0"], "bdf1")
    b.step(4)
    for i, r in enumerate(runs):
        o = Oracle(2, r["n"], r["L"], r["eps"], r["beta"], r["dt"]).start(r["phi0"], "bdf1")
        o.step(4)
        assert rel_l2(b.get_field(i), o.phi) < 10 * tol, i
        sc = b.scalars(i)
        assert abs(sc["r"] - o.r) / o.r < 10 * tol
        assert sc["nsteps"] == 5  # the BDF1 start plus four steps


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_ensemble_sizes_per_step_match_oracle(precision, tol):
    """Per step from an identical state, at the scheme's gates (rel-L2 of
    phi^{n+1} and |r^{n+1} - r|/r at 1e-12 on the FP64 path, 1e-5 on the FP32
    bulk): one batch holding the ensemble workload's four grid classes 64^2,
    128^2, 256^2 and 512^2 (L = N/2, eps, beta and mean drawn per run, two
    runs per class), each run set to the oracle's state after its BDF1 start
    and two BDF2 steps. The first batched step runs after the preparing
    column pass, the second inside the replayed step (committed update in
    the column pass); the second is compared with the oracle advanced from
    the same state, so its error holds two steps of rounding."""
    from paper_2012_15133_gb300 import Batch
    runs = _runs((64, 128, 256, 512), 8)
    b = Batch(runs, 0.02, precision)
    oracles = []
    for i, r in enumerate(runs):
        o = Oracle(2, r["n"], r["L"], r["eps"], r["beta"], r["dt"], dft="numpy").start(r["phi0"], "bdf1")
        o.step(2)
        b.set_state(i, o.phi, o.phi_prev, o.r, o.r_prev)
        oracles.append(o)
    for k in range(2):
        b.step(1)
        for i, (r, o) in enumerate(zip(runs, oracles)):
            o.step(1)
            err = rel_l2(b.get_field(i), o.phi)
            assert err < tol, (k, i, r["n"], err)
            sc = b.scalars(i)
            assert abs(sc["r"] - o.r) / o.r < tol, (k, i, r["n"])
            assert abs(sc["E1"] - o.last_info["E1"]) / o.last_info["E1"] < tol, (k, i, r["n"])
            assert abs(sc["gamma"] - o.last_info["gamma"]) / abs(o.last_info["gamma"]) < tol, (k, i, r["n"])
            assert sc["status"] == 0


def test_ensemble_workload_sizes_match_single_runs():
    """Two runs of each of 64, 128, 256, 512 (the ensemble workload's sizes and
    parameter draws), FP32 bulk, against independent single-run solvers."""
    from paper_2012_15133_gb300 import Batch, Solver
    runs = _runs((64, 128, 256, 512), 8)
    b = Batch(runs, 0.02, "fp32")
    for i, r in enumerate(runs):
        b.init(i, r["phi0"], "bdf1")
    b.step(10)
    for i, r in enumerate(runs):
        s = Solver(2, r["n"], r["L"], r["eps"], r["beta"], r["dt"], "fp32").init(r["phi0"], "bdf1")
        s.step(10)
        assert rel_l2(b.get_field(i), s.get_field(0)) < 1e-5, i
        assert b.scalars(i)["mean"] == s.mass()[1]
        Eb, Es = b.energy(i)[1], s.energy()[1]
        assert abs(Eb - Es) / abs(Es) < 1e-6


def test_one_failing_run_does_not_stop_the_others():
    from paper_2012_15133_gb300 import Batch, SPFCError
    runs = _runs((32, 64), 4)
    b = Batch(runs, 0.02, "fp64")
    for i, r in enumerate(runs):
        phi = r["phi0"].copy()
        if i == 1:
            phi[2, 3] = np.inf  # failure injected on the host
            with pytest.raises(SPFCError) as ei:
                b.init(i, phi, "bdf1")
            assert ei.value.code == 4
        else:
            b.init(i, phi, "bdf1")
    b.step(3)
    b.sync()
    assert b.scalars(1)["status"] == 4
    for i in (0, 2, 3):
        sc = b.scalars(i)
        assert sc["status"] == 0 and sc["nsteps"] == 4
        assert np.all(np.isfinite(b.get_field(i)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("n", [128, 256, 512])
def test_every_batch_schedule_matches_the_oracle_per_step(precision, tol, n):
    """Each tile schedule a batch class can be built with (the autotuner's
    choices) takes the step of the oracle from an identical state."""
    from paper_2012_15133_gb300 import Batch
    from paper_2012_15133_gb300.autotune import batch_schedules
    runs = [ensemble_run(i, sizes=(n,)) for i in range(2)]
    states = []
    for r in runs:
        o = Oracle(2, r["n"], r["L"], r["eps"], r["beta"], r["dt"], dft="numpy").start(r["phi0"], "bdf1")
        o.step(2)
        states.append((o.phi.copy(), o.phi_prev.copy(), o.r, o.r_prev))
        o.step(1)
        states[-1] += (o.phi, o.r)
    for sch in batch_schedules(n):
        b = Batch(runs, 0.02, precision, schedule={n: sch})
        assert b.schedule(n) == sch
        for i, st in enumerate(states):
            b.set_state(i, st[0], st[1], st[2], st[3])
        b.step(1)
        for i, st in enumerate(states):
            assert rel_l2(b.get_field(i), st[4]) < tol, (sch, i)
            assert abs(b.scalars(i)["r"] - st[5]) / st[5] < tol, (sch, i)
        b.close()
