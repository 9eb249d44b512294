"""GPU parity of the 2D CUDA path against the FP64 oracle, through the C-ABI.

Tolerances: rel-L2 <= 1e-12 per step from an identical state on the FP64
path, <= 1e-5 on the FP32-bulk path (FFTs and pointwise work in float32,
reductions and scalars in float64); scalars at the same relative tolerance.
"""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from seeded_inputs import noisy_field, small_2d_case, crystal_2d_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu tests")
    from paper_2012_15133_gb300 import build
    build.build()


def _solver(case, precision="fp64", **kw):
    from paper_2012_15133_gb300 import Solver
    return Solver(case["d"], case["n"], case["L"], case["eps"], case["beta"], case["dt"], precision, **kw)


def _oracle(case):
    return Oracle(case["d"], case["n"], case["L"], case["eps"], case["beta"], case["dt"])


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_bdf1_start_small_case_fp64():
    c = small_2d_case()
    o = _oracle(c).start(c["phi0"], "bdf1")
    s = _solver(c).init(c["phi0"], "bdf1")
    assert rel_l2(s.get_field(0), o.phi) < 1e-12
    assert rel_l2(s.get_field(1), o.phi_prev) < 1e-12
    sc = s.sav_scalars()
    assert abs(sc["r"] - o.r) / o.r < 1e-12
    assert abs(sc["r_prev"] - o.r_prev) / o.r_prev < 1e-12


def test_small_case_trajectory_fp64_field_energy_mass_each_step():
    """64^2 on [0,32]^2, eps 0.1, dt 0.01, 200 steps, BDF1 start: field, modified
    energy and mass compared with the oracle at every step."""
    c = small_2d_case()
    o = _oracle(c).start(c["phi0"], "bdf1")
    s = _solver(c).init(c["phi0"], "bdf1")
    m0 = s.mass()[0]
    worst_phi = worst_E = worst_m = 0.0
    E_prev = None
    for n in range(200):
        o.step()
        s.step(1)
        phi = s.get_field(0)
        worst_phi = max(worst_phi, rel_l2(phi, o.phi))
        _, Em, _ = s.energy()
        Eo = o.modified_energy()
        worst_E = max(worst_E, abs(Em - Eo) / abs(Eo))
        m = s.mass()[0]
        assert m == m0                                  # zero mode kept exactly
        worst_m = max(worst_m, abs(m - o.mass()) / abs(o.mass()))
        if E_prev is not None:
            assert Em <= E_prev * (1 + 1e-13)           # Theorem: E_mod non-increasing
        E_prev = Em
    assert worst_phi < 1e-11, worst_phi
    assert worst_E < 1e-11, worst_E
    assert worst_m < 1e-13, worst_m


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L", [(16, (8.0, 8.0)), (32, (16.0, 11.0)), (128, (64.0, 64.0)), (512, (256.0, 256.0))])
def test_one_step_from_oracle_state(precision, n, L):
    """Per-step parity from an identical state, including the full 512^2 size of the
    crystallisation workload (eps 0.25, dt 0.05, 0.2 + 0.02 U noise) in both precisions."""
    c = crystal_2d_case(n)
    c["L"] = L
    o = _oracle(c).start(c["phi0"], "bdf1")
    o.step(2)
    s = _solver(c, precision).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    # the loaded state itself
    assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
    o.step()
    s.step(1)
    tol = TOL[precision]
    assert rel_l2(s.get_field(0), o.phi) < tol
    sc = s.sav_scalars()
    assert abs(sc["r"] - o.r) / o.r < tol
    assert abs(sc["E1"] - o.last_info["E1"]) / o.last_info["E1"] < tol
    g = o.last_info["gamma"]
    assert sc["gamma"] <= 0.0
    assert abs(sc["gamma"] - g) <= tol * max(abs(g), 1e-300) * 10


@pytest.mark.parametrize("mode", ["ghost", "copy"])
def test_ghost_and_copy_starts(mode):
    c = small_2d_case()
    # smooth trigonometric data: the explicit ghost point amplifies high modes by dt |k|^6
    k = 2 * math.pi / c["L"]
    x = np.arange(c["n"]) * c["L"] / c["n"]
    X, Y = np.meshgrid(x, x, indexing="xy")
    c["phi0"] = 0.2 + 0.1 * np.cos(3 * k * X) * np.sin(2 * k * Y) + 0.05 * np.cos(k * X + 4 * k * Y)
    o = _oracle(c).start(c["phi0"], mode)
    s = _solver(c).init(c["phi0"], mode)
    assert rel_l2(s.get_field(1), o.phi_prev) < 1e-12
    sc = s.sav_scalars()
    assert abs(sc["r"] - o.r) / o.r < 1e-12 and abs(sc["r_prev"] - o.r_prev) / o.r_prev < 1e-12
    o.step(5)
    s.step(5)
    assert rel_l2(s.get_field(0), o.phi) < 1e-12


def test_energies_against_oracle():
    c = small_2d_case()
    o = _oracle(c).start(c["phi0"], "bdf1")
    s = _solver(c).init(c["phi0"], "bdf1")
    o.step(10)
    s.step(10)
    Eo, Em, Eb = s.energy()
    assert abs(Eo - o.original_energy()) / abs(o.original_energy()) < 1e-11
    assert abs(Em - o.modified_energy()) / abs(o.modified_energy()) < 1e-11
    assert abs(Eb - o.breve_energy()) / abs(o.breve_energy()) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mass_is_conserved_exactly(precision):
    c = crystal_2d_case(128)
    s = _solver(c, precision).init(c["phi0"], "bdf1")
    m0, mean0 = s.mass()
    s.step(100)
    m1, mean1 = s.mass()
    assert m1 == m0 and mean1 == mean0
    assert abs(mean0 - float(np.mean(c["phi0"]))) < 1e-15


def test_fp32_bulk_trajectory_tracks_fp64():
    c = crystal_2d_case(256)
    a = _solver(c, "fp64").init(c["phi0"], "bdf1")
    b = _solver(c, "fp32").init(c["phi0"], "bdf1")
    a.step(50)
    b.step(50)
    assert rel_l2(b.get_field(0), a.get_field(0)) < 1e-5
    Ea, Eb = a.energy()[1], b.energy()[1]
    assert abs(Ea - Eb) / abs(Ea) < 1e-6


def test_checkpoint_resume_is_bit_identical(tmp_path):
    c = small_2d_case()
    a = _solver(c).init(c["phi0"], "bdf1")
    a.step(20)
    ref = a.get_field(0)
    b = _solver(c).init(c["phi0"], "bdf1")
    b.step(10)
    path = os.path.join(tmp_path, "ck.bin")
    b.save(path)
    b2 = _solver(c).load(path)
    b2.step(10)
    assert np.array_equal(b2.get_field(0), ref)
    assert b2.sav_scalars()["r"] == a.sav_scalars()["r"]


def test_dt_change_is_copy_restart():
    c = small_2d_case()
    o = _oracle(c).start(c["phi0"], "bdf1")
    s = _solver(c).init(c["phi0"], "bdf1")
    o.step(5)
    s.step(5)
    s.dt_change(0.02)
    o2 = Oracle(2, c["n"], c["L"], c["eps"], c["beta"], 0.02).start(o.phi, "copy")
    o2.step(5)
    s.step(5)
    assert rel_l2(s.get_field(0), o2.phi) < 1e-12


def test_device_pointer_io_matches_host_io():
    import torch
    c = crystal_2d_case(64)
    s1 = _solver(c).init(c["phi0"], "bdf1")
    dev = torch.tensor(c["phi0"], dtype=torch.float64, device="cuda")
    s2 = _solver(c).init(dev, "bdf1")
    s1.step(3)
    s2.step(3)
    out = torch.empty_like(dev)
    s2.get_field(0, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), s1.get_field(0))


@pytest.mark.parametrize("schedule,classes", [(0, {"row", "col_fused"}), (6, {"step"}), (7, {"step"})])
def test_timing_mode_matches_production_mode(schedule, classes):
    """Per-kernel timed launches (one step per launch, events around each)
    give the same steps as production launches: the graph-replayed two-kernel
    step (schedule 0) and the persistent step, whose production launch runs
    all seven steps in one kernel (schedules 6 and 7)."""
    c = crystal_2d_case(128)
    a = _solver(c, "fp32", schedule=schedule).init(c["phi0"], "bdf1")
    b = _solver(c, "fp32", schedule=schedule).init(c["phi0"], "bdf1")
    a.step(7)
    b.set_timing(True)
    b.step(7)
    kt = b.kernel_times()
    assert set(kt) == classes
    assert all(v[0] == 7 and v[1] > 0 for v in kt.values())
    assert np.array_equal(a.get_field(0), b.get_field(0))


def test_nonfinite_input_latches_device_status_and_context_survives():
    from paper_2012_15133_gb300 import SPFCError
    c = small_2d_case()
    bad = c["phi0"].copy()
    bad[3, 5] = np.nan                                # failure injected on the host
    s = _solver(c)
    with pytest.raises(SPFCError) as ei:
        s.init(bad, "bdf1")
        s.step(3)
        s.sync()
    assert ei.value.code == 4
    # the context stays usable: a fresh run on the same device works
    good = _solver(c).init(c["phi0"], "bdf1")
    good.step(2)
    assert np.all(np.isfinite(good.get_field(0)))


def test_errors_out_of_order_and_bad_sizes():
    from paper_2012_15133_gb300 import SPFCError, Solver
    c = small_2d_case()
    s = _solver(c)
    with pytest.raises(SPFCError) as ei:
        s.step(1)
    assert ei.value.code == 6
    with pytest.raises(SPFCError) as ei:
        Solver(2, 48, 24.0, 0.1, 1.0, 0.01)
    assert ei.value.code == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [128, 256, 512])
def test_every_launch_schedule_matches_the_oracle(precision, n):
    """All compiled tile schedules (the autotuner's choices) compute the same step."""
    from paper_2012_15133_gb300 import Solver, num_schedules
    c = crystal_2d_case(n)
    o = _oracle(c).start(c["phi0"], "bdf1")
    o.step(1)
    ref_state = (o.phi, o.phi_prev, o.r, o.r_prev)
    o.step(2)
    for sch in range(num_schedules(2, n)):
        s = Solver(2, n, c["L"], c["eps"], c["beta"], c["dt"], precision, schedule=sch)
        assert s.schedule == sch
        s.set_state(*ref_state)
        s.step(2)
        assert rel_l2(s.get_field(0), o.phi) < TOL[precision], sch
        assert abs(s.sav_scalars()["r"] - o.r) / o.r < TOL[precision], sch


def test_device_noise_start_equals_the_host_noise_field():
    """spfc_init_random draws the same SplitMix64 stream as the host inputs:
    starting from it or from the host field gives bit-identical runs."""
    from paper_2012_15133_gb300 import Solver
    from seeded_inputs import cube_3d_case
    for c, mean, amp, seed in ((crystal_2d_case(64), 0.2, 0.02, 1), (cube_3d_case(16), 0.15, 0.05, 2)):
        args = (c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], "fp64")
        a, b = Solver(*args), Solver(*args)
        a.init(c["phi0"], "bdf1")
        b.init_random(mean, amp, seed, "bdf1")
        assert np.array_equal(a.get_field(1), b.get_field(1))
        a.step(5)
        b.step(5)
        assert np.array_equal(a.get_field(0), b.get_field(0))


@pytest.mark.parametrize("schedule", [0, 6, 7])
def test_scalar_ring_records_every_step(schedule):
    """The device writes every committed step's scalars into a pinned host
    ring (no per-step synchronisation): after one sync the records equal the
    synchronising reads of an identical run, for the two-kernel and the
    persistent step, the BDF1 start included, with wrap-around."""
    import torch
    c = crystal_2d_case(128)
    cap = 4
    a = _solver(c, "fp32", schedule=schedule)
    ring = torch.full((cap, 8), -1.0, dtype=torch.float64).pin_memory()
    a.set_scalar_ring(ring)
    a.init(c["phi0"], "bdf1")
    a.step(6)
    a.sync()
    b = _solver(c, "fp32", schedule=schedule).init(c["phi0"], "bdf1")
    want = {}
    for _ in range(6):
        b.step(1)
        sc = b.sav_scalars(full=True)
        want[int(sc["nsteps"])] = sc
    rec = ring.numpy()
    for k in range(4, 8):  # the last `cap` steps (1 = the BDF1 start, 2..7 the steps)
        e = rec[k % cap]
        assert int(e[0]) == k
        sc = want[k]
        assert e[1] == sc["r"] and e[2] == sc["r_prev"] and e[3] == sc["xi"]
        assert e[4] == sc["gamma"] and e[5] == sc["E1"] and e[7] == 0.0
    assert np.array_equal(a.get_field(0), b.get_field(0))
    a.set_scalar_ring(None)


@pytest.mark.parametrize("schedule", [6, 7])
def test_persistent_step_failure_latches_status_and_context_survives(schedule):
    """A finite state whose step overflows (|grad phi|^4 beyond float32) makes
    the persistent step's scalar solve fail: every block takes the same
    decision and returns, the status word reports a non-finite value, a later
    launch on the failed handle returns at entry with the same error, and the
    context stays usable."""
    from paper_2012_15133_gb300 import SPFCError
    c = crystal_2d_case(128)
    s = _solver(c, "fp32", schedule=schedule).init(c["phi0"], "bdf1")
    big = c["phi0"] * 1e20
    s.set_state(big, big, 1.0, 1.0)
    with pytest.raises(SPFCError) as ei:
        s.step(3)
        s.sync()
    assert ei.value.code == 4
    with pytest.raises(SPFCError) as ei:
        s.step(1)
        s.sync()
    assert ei.value.code == 4
    good = _solver(c, "fp32", schedule=schedule).init(c["phi0"], "bdf1")
    good.step(4)
    assert np.all(np.isfinite(good.get_field(0)))
