"""GPU parity of the 3D CUDA path against the FP64 oracle, through the C-ABI
(same tolerances as 2D: rel-L2 <= 1e-12 float64, <= 1e-5 float32-bulk)."""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from seeded_inputs import cube_3d_case, noisy_field

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu tests")
    from paper_2012_15133_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _solver(c, precision="fp64"):
    from paper_2012_15133_gb300 import Solver
    return Solver(3, c["n"], c["L"], c["eps"], c["beta"], c["dt"], precision)


def _oracle(c, dft="naive"):
    return Oracle(3, c["n"], c["L"], c["eps"], c["beta"], c["dt"], dft=dft)


def test_bdf1_start_3d_fp64():
    c = cube_3d_case(16)
    o = _oracle(c).start(c["phi0"], "bdf1")
    s = _solver(c).init(c["phi0"], "bdf1")
    assert rel_l2(s.get_field(0), o.phi) < 1e-12
    assert rel_l2(s.get_field(1), o.phi_prev) < 1e-12
    sc = s.sav_scalars()
    assert abs(sc["r"] - o.r) / o.r < 1e-12 and abs(sc["r_prev"] - o.r_prev) / o.r_prev < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L", [(16, (8.0, 8.0, 8.0)), (32, (16.0, 12.0, 20.0)), (128, (64.0, 64.0, 64.0))])
def test_one_step_3d_from_oracle_state(precision, n, L):
    """Per-step parity from an identical state, up to the full 128^3 size of the 3D
    workload (eps 0.2, dt 0.02, 0.15 + 0.05 U noise)."""
    c = cube_3d_case(n)
    c["L"] = L
    o = _oracle(c, dft="numpy" if n >= 64 else "naive").start(c["phi0"], "bdf1")
    o.step(1)
    s = _solver(c, precision).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
    o.step()
    s.step(1)
    tol = TOL[precision]
    assert rel_l2(s.get_field(0), o.phi) < tol
    sc = s.sav_scalars()
    assert abs(sc["r"] - o.r) / o.r < tol
    assert abs(sc["E1"] - o.last_info["E1"]) / o.last_info["E1"] < tol
    assert sc["gamma"] <= 0.0


def test_trajectory_3d_fp64_field_energy_mass():
    c = cube_3d_case(32)
    o = _oracle(c).start(c["phi0"], "bdf1")
    s = _solver(c).init(c["phi0"], "bdf1")
    m0 = s.mass()[0]
    E_prev = None
    for _ in range(20):
        o.step()
        s.step(1)
        assert rel_l2(s.get_field(0), o.phi) < 1e-11
        _, Em, _ = s.energy()
        assert abs(Em - o.modified_energy()) / abs(o.modified_energy()) < 1e-11
        assert s.mass()[0] == m0
        if E_prev is not None:
            assert Em <= E_prev * (1 + 1e-13)
        E_prev = Em
    Eo, _, Eb = s.energy()
    assert abs(Eo - o.original_energy()) / abs(o.original_energy()) < 1e-11
    assert abs(Eb - o.breve_energy()) / abs(o.breve_energy()) < 1e-11


@pytest.mark.parametrize("mode", ["ghost", "copy"])
def test_ghost_and_copy_starts_3d(mode):
    c = cube_3d_case(16)
    k = 2 * math.pi / c["L"]
    x = np.arange(16) * c["L"] / 16
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    c["phi0"] = 0.15 + 0.1 * np.cos(2 * k * X) * np.sin(k * Y) + 0.05 * np.cos(k * Z + 2 * k * X)
    o = _oracle(c).start(c["phi0"], mode)
    s = _solver(c).init(c["phi0"], mode)
    assert rel_l2(s.get_field(1), o.phi_prev) < 1e-12
    o.step(3)
    s.step(3)
    assert rel_l2(s.get_field(0), o.phi) < 1e-12


def test_checkpoint_resume_3d_is_bit_identical(tmp_path):
    c = cube_3d_case(32)
    a = _solver(c, "fp32").init(c["phi0"], "bdf1")
    a.step(12)
    ref = a.get_field(0)
    b = _solver(c, "fp32").init(c["phi0"], "bdf1")
    b.step(6)
    path = os.path.join(tmp_path, "ck3.bin")
    b.save(path)
    b2 = _solver(c, "fp32").load(path)
    b2.step(6)
    assert np.array_equal(b2.get_field(0), ref)


def test_fp32_mass_exact_3d_and_tracks_fp64():
    c = cube_3d_case(64)
    a = _solver(c, "fp64").init(c["phi0"], "bdf1")
    b = _solver(c, "fp32").init(c["phi0"], "bdf1")
    m0 = b.mass()[0]
    a.step(20)
    b.step(20)
    assert b.mass()[0] == m0
    assert rel_l2(b.get_field(0), a.get_field(0)) < 1e-5
