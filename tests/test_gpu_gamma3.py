"""The optional phi^4 term on the GPU (2D single runs) against the FP64 oracle:
E_1 gains gamma3/4 ||phi||_4^4 and N gains gamma3 phi^3 with its mean removed,
the SAV scheme of Sec. 2.2-2.3 otherwise unchanged. Tolerances are those of the
plain scheme: rel-L2 <= 1e-12 per step from an identical state on the FP64
path, <= 1e-5 on the FP32-bulk path. The fields have a larger mean than the
crystal workload so that the cubic term is a sizeable part of N."""
import numpy as np
import pytest

from oracle import Oracle
from seeded_inputs import cube_3d_case, noisy_field

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
G3 = 1.0


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _case(n, L=None, seed=31):
    L = 0.5 * n if L is None else L
    return dict(d=2, n=n, L=L, eps=0.25, beta=1.0, dt=0.05, phi0=noisy_field((n, n), 0.4, 0.1, seed))


def _pair(c, precision, gamma3=G3):
    from paper_2012_15133_gb300 import Solver
    o = Oracle(c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], gamma3=gamma3)
    s = Solver(c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], precision)
    return o, s


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L", [(32, (16.0, 11.0)), (128, (64.0, 64.0))])
def test_gamma3_step_matches_the_oracle(precision, n, L):
    c = _case(n, L)
    o, s = _pair(c, precision)
    o.start(c["phi0"], "bdf1").step(2)
    s.set_gamma3(G3).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    plain = Oracle(2, n, L, c["eps"], c["beta"], c["dt"]).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    phi_start = o.phi.copy()
    for _ in range(3):
        o.step()
        plain.step()
        s.step(1)
        phi = s.get_field(0)
        assert rel_l2(phi, o.phi) < TOL[precision]
        assert abs(s.sav_scalars()["r"] - o.r) / o.r < TOL[precision]
        assert abs(s.sav_scalars()["E1"] - o.last_info["E1"]) / o.last_info["E1"] < TOL[precision]
    # the cubic term changes the three steps' increment by about 15 %
    assert rel_l2(o.phi - phi_start, plain.phi - phi_start) > 0.1


# The ghost point multiplies float32 rounding of the high modes by dt |k|^6
# (about 2.5e4 on this grid), so, as for the plain scheme, the ghost start is
# checked on the float64 path only.
@pytest.mark.parametrize("precision,mode", [("fp64", "bdf1"), ("fp32", "bdf1"), ("fp64", "ghost"),
                                            ("fp64", "copy"), ("fp32", "copy")])
def test_gamma3_starts_and_energies(precision, mode):
    # set before init: the start-up step (and r^0 = sqrt(E_1(phi^0))) take the term too
    c = _case(64)
    if mode == "ghost":
        # smooth data: the explicit ghost point amplifies high modes by dt |k|^6
        k = 2 * np.pi / c["L"]
        x = np.arange(64) * c["L"] / 64
        X, Y = np.meshgrid(x, x, indexing="xy")
        c["phi0"] = 0.4 + 0.1 * np.cos(3 * k * X) * np.sin(2 * k * Y) + 0.05 * np.cos(k * X + 4 * k * Y)
    o, s = _pair(c, precision)
    s.set_gamma3(G3)
    o.start(c["phi0"], mode)
    s.init(c["phi0"], mode)
    assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
    assert rel_l2(s.get_field(1), o.phi_prev) < TOL[precision]
    assert abs(s.sav_scalars()["r"] - o.r) / o.r < TOL[precision]
    o.step(4)
    s.step(4)
    assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
    e_orig, e_mod, _ = s.energy()
    assert abs(e_orig - o.original_energy()) / abs(o.original_energy()) < TOL[precision]
    assert abs(e_mod - o.modified_energy()) / abs(o.modified_energy()) < TOL[precision]


def test_gamma3_modified_energy_decays_and_mass_is_kept():
    """Theorem SPFC-energy stability needs only E_1 bounded below, which the
    phi^4 term keeps: the modified energy decreases step by step at a large dt
    and the mean of phi stays put."""
    from paper_2012_15133_gb300 import Solver
    c = _case(256, seed=32)
    s = Solver(2, 256, c["L"], c["eps"], c["beta"], 0.5, "fp64")
    s.set_gamma3(G3).init(c["phi0"], "bdf1")
    m0 = s.mass()[1]
    em = [s.energy()[1]]
    for _ in range(20):
        s.step(5)
        em.append(s.energy()[1])
    assert all(b <= a * (1 + 1e-12) for a, b in zip(em, em[1:])), em
    assert em[-1] < em[0]
    assert abs(s.mass()[1] - m0) < 1e-12 * abs(m0)


def test_gamma3_zero_is_the_plain_path_and_checkpoints_record_it(tmp_path):
    from paper_2012_15133_gb300 import Solver, SPFCError
    c = _case(64)
    args = (c["d"], c["n"], c["L"], c["eps"], c["beta"], c["dt"], "fp64")
    a, b = Solver(*args), Solver(*args)
    a.init(c["phi0"], "bdf1").step(5)
    b.set_gamma3(0.0).init(c["phi0"], "bdf1").step(5)
    assert np.array_equal(a.get_field(0), b.get_field(0))
    # switched on and off again mid-run: the plain kernels take over unchanged
    b.set_gamma3(G3).step(3).set_gamma3(0.0)
    a.set_state(b.get_field(0), b.get_field(1), b.sav_scalars()["r"], b.sav_scalars()["r_prev"])
    b.set_state(b.get_field(0), b.get_field(1), b.sav_scalars()["r"], b.sav_scalars()["r_prev"])
    a.step(4)
    b.step(4)
    assert np.array_equal(a.get_field(0), b.get_field(0))
    # checkpoints carry gamma3
    b.set_gamma3(G3).step(3)
    path = str(tmp_path / "g3.ckp")
    b.save(path)
    fresh = Solver(*args)
    fresh.init(c["phi0"], "bdf1")
    with pytest.raises(SPFCError):
        fresh.load(path)             # gamma3 = 0 here, 1 in the file
    fresh.set_gamma3(G3).load(path)
    b.step(4)
    fresh.step(4)
    assert np.array_equal(b.get_field(0), fresh.get_field(0))
    # per-kernel timing follows the three-pass form
    fresh.set_timing(True)
    fresh.step(2)
    kt = fresh.kernel_times()
    assert kt["col_inv+col_fwd"][0] == 4 and kt["row"][0] == 2, kt
    with pytest.raises(SPFCError):
        b.set_gamma3(-1.0)
    with pytest.raises(SPFCError):
        b.set_gamma3(float("nan"))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gamma3_3d_steps_starts_and_energies(precision):
    """3D on a box with three different side lengths: per step from an
    identical state, then the BDF1 start with the term set before init, E_N and
    the modified energy."""
    from paper_2012_15133_gb300 import Solver
    n, L = 16, (8.0, 6.0, 7.0)
    phi0 = noisy_field((n, n, n), 0.4, 0.1, 33)
    args = (3, n, L, 0.2, 1.0, 0.02)
    o = Oracle(*args, gamma3=G3).start(phi0, "bdf1").step(1)
    plain = Oracle(*args).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    s = Solver(*args, precision).set_gamma3(G3).set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    phi_start = o.phi.copy()
    for _ in range(3):
        o.step()
        plain.step()
        s.step(1)
        assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
        assert abs(s.sav_scalars()["r"] - o.r) / o.r < TOL[precision]
        assert abs(s.sav_scalars()["E1"] - o.last_info["E1"]) / o.last_info["E1"] < TOL[precision]
    assert rel_l2(o.phi - phi_start, plain.phi - phi_start) > 0.02  # about 5 % here
    o2 = Oracle(*args, gamma3=G3).start(phi0, "bdf1")
    s2 = Solver(*args, precision).set_gamma3(G3).init(phi0, "bdf1")
    assert rel_l2(s2.get_field(0), o2.phi) < TOL[precision]
    o2.step(2)
    s2.step(2)
    assert rel_l2(s2.get_field(0), o2.phi) < TOL[precision]
    e_orig, e_mod, _ = s2.energy()
    assert abs(e_orig - o2.original_energy()) / abs(o2.original_energy()) < TOL[precision]
    assert abs(e_mod - o2.modified_energy()) / abs(o2.modified_energy()) < TOL[precision]


def test_gamma3_3d_zero_is_the_plain_path():
    from paper_2012_15133_gb300 import Solver
    c3 = cube_3d_case(16)
    args = (3, 16, c3["L"], c3["eps"], c3["beta"], c3["dt"], "fp64")
    a, b = Solver(*args), Solver(*args)
    a.init(c3["phi0"], "bdf1").step(3)
    b.set_gamma3(G3).set_gamma3(0.0).init(c3["phi0"], "bdf1").step(3)
    assert np.array_equal(a.get_field(0), b.get_field(0))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gamma3_in_the_batched_ensemble(precision):
    """Three runs in two grid-size classes: gamma3 = 1 and gamma3 = 0 share the
    64^2 class (which then steps with the phi^4 passes), gamma3 = 0.5 alone at
    32^2. BDF1 start and four steps against the oracle, with E_N."""
    from paper_2012_15133_gb300 import Batch, SPFCError
    runs = [dict(n=n, L=0.5 * n, eps=0.25, beta=1.0, g3=g, phi0=noisy_field((n, n), 0.4, 0.1, 40 + i))
            for i, (n, g) in enumerate(((64, 1.0), (64, 0.0), (32, 0.5)))]
    b = Batch(runs, 0.05, precision)
    for i, r in enumerate(runs):
        b.set_gamma3(i, r["g3"]).init(i, r["phi0"], "bdf1")
    b.step(4)
    for i, r in enumerate(runs):
        o = Oracle(2, r["n"], r["L"], r["eps"], r["beta"], 0.05, gamma3=r["g3"]).start(r["phi0"], "bdf1").step(4)
        assert rel_l2(b.get_field(i, 0), o.phi) < TOL[precision], i
        e = b.energy(i)[0]
        assert abs(e - o.original_energy()) / abs(o.original_energy()) < TOL[precision], i
    with pytest.raises(SPFCError):
        b.set_gamma3(0, -1.0)
