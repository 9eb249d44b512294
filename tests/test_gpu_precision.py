"""The precision split of the FP32-bulk path (FFTs and pointwise work in
float32; E_1, the inner products, S, rho, LHS and r in float64), through the
C-ABI: the scalar solve is float64 on both paths, and the error of each result
of the FP32-bulk path against the FP64 oracle and the FP64 GPU path."""
import numpy as np
import pytest

from oracle import Oracle, sav_r_update
from seeded_inputs import crystal_2d_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu tests")
    from paper_2012_15133_gb300 import build
    build.build()


def _solver(c, precision):
    from paper_2012_15133_gb300 import Solver
    return Solver(2, c["n"], c["L"], c["eps"], c["beta"], c["dt"], precision)


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [128, 512])
def test_scalar_solve_is_float64_on_both_paths(precision, n):
    """Per step from the oracle's state: the device's r^{n+1} equals the
    scalar form of eqs. solver-2, -4 and -6 evaluated in float64 from the
    device's own E_1, gamma, eta, theta and r^n, r^{n-1} to 1e-13 on BOTH
    paths (a float-float or float32 solve would miss it by orders of
    magnitude), and those inputs match the oracle's at the path's gate."""
    c = crystal_2d_case(n)
    o = Oracle(2, n, c["L"], c["eps"], c["beta"], c["dt"], dft="numpy").start(c["phi0"], "bdf1")
    o.step(3)
    s = _solver(c, precision).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    r_n, r_nm1 = o.r, o.r_prev
    s.step(1)
    o.step(1)
    d = s.sav_scalars(full=True)
    r_host = sav_r_update(d["E1"], d["gamma"], d["eta"], d["theta"], r_n, r_nm1, c["dt"])
    assert abs(d["r"] - r_host) / abs(r_host) < 1e-13, (d["r"], r_host)
    tol = TOL[precision]
    for key in ("E1", "gamma", "eta", "theta"):
        ref = o.last_info[key]
        assert abs(d[key] - ref) <= tol * abs(ref), (key, d[key], ref)
    assert abs(d["r"] - o.r) / o.r < tol
    assert abs(d["denom"] - o.last_info["denom"]) / o.last_info["denom"] < tol
    assert rel_l2(s.get_field(0), o.phi) < tol


def test_fp32_bulk_error_per_result():
    """The 512^2 crystallisation workload from one BDF1 start, 100 steps on
    the FP32-bulk and the FP64 GPU paths: field, r, modified energy and mass
    of the former against the latter (mass exactly: the zero modes are float64
    on both paths), and both against the oracle after the first step."""
    c = crystal_2d_case(512)
    a = _solver(c, "fp64").init(c["phi0"], "bdf1")
    b = _solver(c, "fp32").init(c["phi0"], "bdf1")
    o = Oracle(2, 512, c["L"], c["eps"], c["beta"], c["dt"], dft="numpy").start(c["phi0"], "bdf1")
    assert rel_l2(a.get_field(0), o.phi) < 1e-12
    assert rel_l2(b.get_field(0), o.phi) < 1e-5
    assert abs(b.sav_scalars()["r"] - o.r) / o.r < 1e-6
    a.step(100)
    b.step(100)
    assert rel_l2(b.get_field(0), a.get_field(0)) < 1e-4
    ra, rb = a.sav_scalars()["r"], b.sav_scalars()["r"]
    assert abs(ra - rb) / ra < 1e-5
    Ea, Eb = a.energy()[1], b.energy()[1]
    assert abs(Ea - Eb) / abs(Ea) < 1e-5
    assert a.mass() == b.mass()
