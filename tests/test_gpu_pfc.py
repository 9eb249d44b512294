"""The PFC model of Sec. 1 (eq. energy-PFC) on the GPU (2D single runs)
against the FP64 oracle, with its own split: L = a + (1 + Delta)^2,
E_1 = gamma3/4 ||phi||_4^4 - 1/2 ||phi||^2 + (1 + 1/(4 gamma3)) |Omega|,
N = gamma3 phi^3 - phi. Tolerances are those of the SPFC scheme: rel-L2 <=
1e-12 per step from an identical state on the FP64 path, <= 1e-5 on the
FP32-bulk path. The data are the PFC model's usual regime: mean -0.3 with
noise 0.1 and eps = 0.25 (hexagonal crystallisation in 2D)."""
import numpy as np
import pytest

from oracle import Oracle
from seeded_inputs import noisy_field

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
G3 = 1.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu tests")
    from paper_2012_15133_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _case(n, L=None, seed=41, dt=0.1):
    L = (np.pi * n / 4.0) if L is None else L  # about 8 points per lattice period 2 pi / |k|, |k| = 1
    return dict(n=n, L=L, eps=0.25, beta=1.0, dt=dt, phi0=noisy_field((n, n), -0.3, 0.1, seed))


def _pair(c, precision, gamma3=G3):
    from paper_2012_15133_gb300 import Solver
    o = Oracle(2, c["n"], c["L"], c["eps"], c["beta"], c["dt"], pfc=True, gamma3=gamma3)
    s = Solver(2, c["n"], c["L"], c["eps"], c["beta"], c["dt"], precision).set_pfc(gamma3)
    return o, s


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L", [(32, (25.0, 19.0)), (128, None)])
def test_pfc_step_matches_the_oracle(precision, n, L):
    c = _case(n, L if L is None else L)
    if L is not None:
        c["L"] = L
    o, s = _pair(c, precision)
    o.start(c["phi0"], "bdf1").step(2)
    s.set_state(o.phi, o.phi_prev, o.r, o.r_prev)
    for _ in range(3):
        o.step()
        s.step(1)
        assert rel_l2(s.get_field(0), o.phi) < TOL[precision]
        sc = s.sav_scalars(full=True)
        for key, ref in (("r", o.r), ("E1", o.last_info["E1"]), ("gamma", o.last_info["gamma"]),
                         ("eta", o.last_info["eta"]), ("theta", o.last_info["theta"])):
            assert abs(sc[key] - ref) <= TOL[precision] * abs(ref), key


@pytest.mark.parametrize("precision,mode", [("fp64", "bdf1"), ("fp32", "bdf1"), ("fp64", "ghost"),
                                            ("fp64", "copy"), ("fp32", "copy")])
def test_pfc_starts_and_energies_match_the_oracle(precision, mode):
    """The three start-ups then four steps, with the PFC energy of eq.
    energy-PFC, the modified energy with the PFC operator and E_breve."""
    c = _case(64)
    o, s = _pair(c, precision)
    if mode == "ghost":
        # the explicit ghost point multiplies the rounding of the high modes by
        # dt |k|^2 (a + (1 - |k|^2)^2) (about 400 here): smooth data, as for SPFC
        g = o.grid
        c["phi0"] = g.idft(g.dft(c["phi0"]) * np.exp(-1.0 * g.K2))
    o.start(c["phi0"], mode).step(4)
    s.init(c["phi0"], mode).step(4)
    tol = 10 * TOL[precision]  # five steps of accumulated rounding
    assert rel_l2(s.get_field(0), o.phi) < tol
    assert abs(s.sav_scalars()["r"] - o.r) / o.r < tol
    E_orig, E_mod, E_breve = s.energy()
    assert abs(E_orig - o.original_energy()) <= tol * abs(o.original_energy())
    assert abs(E_mod - o.modified_energy()) <= tol * abs(o.modified_energy())
    assert abs(E_breve - o.breve_energy()) <= tol * abs(o.breve_energy())


def test_pfc_modified_energy_decreases_and_mass_is_kept():
    """The energy law of Theorem SPFC-energy stability for this split:
    the modified energy does not increase over 100 steps of a crystallising
    run at a large step (dt = 0.5), and the mass stays exactly constant."""
    c = _case(128, dt=0.5)
    o, s = _pair(c, "fp64")
    s.init(c["phi0"], "bdf1")
    m0 = s.mass()
    E = [s.energy()[1]]
    for _ in range(20):
        s.step(5)
        E.append(s.energy()[1])
    assert all(b <= a * (1 + 1e-13) for a, b in zip(E, E[1:])), E
    assert s.mass() == m0
    assert E[-1] < 0.99 * E[0]  # the run moves


def test_pfc_switch_back_and_refusals(tmp_path):
    """set_pfc(0) gives the SPFC scheme back bit for bit; the phi^4 setter of
    the SPFC model is refused while the PFC model is on; a checkpoint keeps
    the model and resumes bit-identically; 3D handles refuse the model."""
    from paper_2012_15133_gb300 import Solver, SPFCError
    from seeded_inputs import crystal_2d_case
    c = crystal_2d_case(64)
    args = (2, 64, c["L"], c["eps"], c["beta"], c["dt"], "fp64")
    a, b = Solver(*args), Solver(*args)
    a.set_pfc(1.0).set_pfc(0.0).init(c["phi0"], "bdf1").step(5)
    b.init(c["phi0"], "bdf1").step(5)
    assert np.array_equal(a.get_field(0), b.get_field(0))
    p = _case(64)
    o, s = _pair(p, "fp64")
    with pytest.raises(SPFCError):
        s.set_gamma3(0.5)
    s.init(p["phi0"], "bdf1").step(3)
    f = str(tmp_path / "pfc.ckp")
    s.save(f)
    s.step(4)
    _, t = _pair(p, "fp64")
    t.load(f)
    t.step(4)
    assert np.array_equal(s.get_field(0), t.get_field(0))
    spfc = Solver(2, 64, p["L"], p["eps"], p["beta"], p["dt"], "fp64")
    with pytest.raises(SPFCError):
        spfc.load(f)  # the model differs
    s3 = Solver(3, 16, 8.0, 0.25, 1.0, 0.05, "fp64")
    with pytest.raises(SPFCError):
        s3.set_pfc(1.0)
