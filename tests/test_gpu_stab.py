"""The stabilised scheme of Sec. 5.2 (- A dt Delta_N (phi^{n+1} - phi^n) on the
left of the dt-multiplied equation) on the GPU against the FP64 oracle, with
the tolerances of the plain scheme: rel-L2 <= 1e-12 per step from an
identical state on the FP64 path, <= 1e-5 on the FP32-bulk path."""
import numpy as np
import pytest

from oracle import Oracle
from seeded_inputs import crystal_2d_case, cube_3d_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
A = 3.0


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _pair(c, precision, stab=A):
    from paper_2012_15133_gb300 import Solver
    o = Oracle(c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], stab=stab)
    s = Solver(c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], precision)
    return o, s


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L", [(32, (16.0, 11.0)), (128, (64.0, 64.0))])
def test_stabilised_step_matches_the_oracle(precision, n, L):
    c = crystal_2d_case(n)
    c["L"] = L
    o, s = _pair(c, precision)
    o.start(c["phi0"], "bdf1").step(2)
    s.set_state(o.phi, o.phi_prev, o.r, o.r_prev).set_stabilization(A)
    for _ in range(3):
        o.step()
        s.step(1)
        assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
        assert abs(s.sav_scalars()["r"] - o.r) / o.r < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stabilised_start_and_3d_step(precision):
    # set before init: the first-order start is stabilised too
    c = crystal_2d_case(64)
    o, s = _pair(c, precision)
    s.set_stabilization(A)
    o.start(c["phi0"], "bdf1")
    s.init(c["phi0"], "bdf1")
    assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
    o.step(2)
    s.step(2)
    assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
    c3 = cube_3d_case(16)
    o3, s3 = _pair(c3, precision)
    o3.start(c3["phi0"], "bdf1").step(1)
    s3.set_state(o3.phi, o3.phi_prev, o3.r, o3.r_prev).set_stabilization(A)
    o3.step(2)
    s3.step(2)
    assert rel_l2(s3.get_field(0), o3.phi) < TOL[precision]


def test_zero_stabiliser_changes_nothing_and_checkpoints_record_it(tmp_path):
    from paper_2012_15133_gb300 import Solver, SPFCError
    c = crystal_2d_case(64)
    args = (c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], "fp64")
    a, b = Solver(*args), Solver(*args)
    a.init(c["phi0"], "bdf1").step(5)
    b.init(c["phi0"], "bdf1").set_stabilization(0.0).step(5)
    assert np.array_equal(a.get_field(0), b.get_field(0))
    b.set_stabilization(A).step(3)
    path = str(tmp_path / "stab.ckp")
    b.save(path)
    fresh = Solver(*args)
    fresh.init(c["phi0"], "bdf1")
    with pytest.raises(SPFCError):
        fresh.load(path)             # A = 0 here, 3 in the file
    fresh.set_stabilization(A).load(path)
    b.step(4)
    fresh.step(4)
    assert np.array_equal(b.get_field(0), fresh.get_field(0))
    with pytest.raises(SPFCError):
        b.set_stabilization(-1.0)


def _nucleation_run(stab, t_marks):
    """Sec. 5.2's rough-data case: a = 0.5 on [0, 100]^2, the 0.05 (2 r - 1)
    noise plus a nucleus of magnitude 10 at (50, 50) (read as a Gaussian of
    width 2), dt = 0.01, copy start; (t, xi, E_N, max |phi|) at t_marks."""
    from paper_2012_15133_gb300 import Solver
    from seeded_inputs import noisy_field
    n, L = 256, 100.0
    x = np.arange(n) * L / n
    X, Y = np.meshgrid(x, x)
    phi0 = noisy_field((n, n), 0.0, 0.05, 21) + 10.0 * np.exp(-((X - 50) ** 2 + (Y - 50) ** 2) / 8.0)
    s = Solver(2, n, L, 0.5, 1.0, 0.01, "fp64")
    s.set_stabilization(stab)
    s.init(phi0, "copy")
    out, t = [], 0.0
    for tm in t_marks:
        s.step(int(round((tm - t) / 0.01)))
        t = tm
        out.append((tm, s.sav_scalars()["xi"], s.energy()[0], float(np.abs(s.get_field(0)).max())))
    return out


def test_rough_nucleus_needs_the_stabiliser():
    """Plain SAV loses the auxiliary variable (r turns negative, E_N rises);
    the stabilised scheme with A = 100 keeps xi = r / sqrt(E_1) near 1, E_N
    decreasing and the nucleus relaxing."""
    plain = _nucleation_run(0.0, (0.1, 1.0, 5.0))
    assert min(xi for _, xi, _, _ in plain) < 0.5
    assert plain[-1][2] > plain[0][2]
    stab = _nucleation_run(100.0, (0.1, 1.0, 5.0, 20.0))
    assert all(0.8 < xi < 1.1 for _, xi, _, _ in stab), stab
    en = [e for _, _, e, _ in stab]
    assert all(b < a for a, b in zip(en, en[1:])), en
    assert stab[-1][3] < 0.5 * stab[0][3], stab
    print(f"\nnucleus: plain {plain}\nstabilised {stab}")
