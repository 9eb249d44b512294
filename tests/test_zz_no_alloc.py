"""The allocation-free entry point (spfc_field_energy_noalloc), called through
the C interface, against the allocating path (a solver handle's spfc_energy
and spfc_mass) on the same field. It serves callers that cannot allocate
device memory; its scratch is a fixed array inside the library that every
call reuses, so two calls in a row must both agree with the allocating path.
Collected last so that a failure here stops a -x run only after every other
test has run."""
import numpy as np
import pytest

from seeded_inputs import noisy_field, small_2d_case

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu tests")
    from paper_2012_15133_gb300 import build
    build.build()


def _reference(phi, n, L, eps, beta):
    """The allocating path on the same field: E_N; with both levels the field
    and r^n = r^{n-1} = 1 the modified energy is 1/2 ||L^{1/2} phi||^2 + 1
    (eq. discrete energy); the mass."""
    from paper_2012_15133_gb300 import Solver
    s = Solver(2, n, L, eps, beta, 0.01, "fp64")
    s.set_state(phi, phi, 1.0, 1.0)
    E_orig, E_mod, _ = s.energy()
    mass, _ = s.mass()
    return E_orig, E_mod - 1.0, mass


@pytest.mark.parametrize("n,L,eps,beta,seed", [(64, 32.0, 0.1, 1.0, 0), (256, 128.0, 0.25, 0.7, 3)])
def test_noalloc_matches_allocating_path_on_two_calls_in_a_row(n, L, eps, beta, seed):
    import torch
    from paper_2012_15133_gb300 import field_energy_noalloc
    phi_a = noisy_field((n, n), 0.2, 0.05, seed)
    phi_b = noisy_field((n, n), 0.15, 0.08, seed + 1)
    for phi in (phi_a, phi_b):
        E_ref, H_ref, m_ref = _reference(phi, n, L, eps, beta)
        dev = torch.tensor(phi, dtype=torch.float64, device="cuda")
        r1 = field_energy_noalloc(dev, L, eps, beta)
        r2 = field_energy_noalloc(dev, L, eps, beta)
        for r in (r1, r2):
            assert abs(r[0] - E_ref) <= TOL * abs(E_ref), (r[0], E_ref)
            assert abs(r[1] - H_ref) <= TOL * abs(H_ref), (r[1], H_ref)
            assert abs(r[2] - m_ref) <= TOL * abs(m_ref), (r[2], m_ref)
        assert r1 == r2


def test_noalloc_matches_the_oracle():
    """Against the FP64 CPU oracle on a 64^2 field: E_N (eq.
    energy-discrete-spectral), 1/2 ||L_N^{1/2} phi||^2 and the mass."""
    import torch
    from oracle import Oracle
    from paper_2012_15133_gb300 import field_energy_noalloc
    n, L, eps, beta = 64, (32.0, 32.0), 0.1, 1.3
    phi = noisy_field((n, n), 0.2, 0.1, 5)
    o = Oracle(2, n, L, eps, beta, 0.01)
    r = field_energy_noalloc(torch.tensor(phi, dtype=torch.float64, device="cuda"), L, eps, beta)
    E = o.model.E_orig(phi)
    H = 0.5 * o.model.L_norm_sq(phi)
    m = o.grid.mean_value(phi)
    assert abs(r[0] - E) <= TOL * abs(E) and abs(r[1] - H) <= TOL * abs(H) and abs(r[2] - m) <= TOL * abs(m)


def test_noalloc_reports_a_non_finite_field_and_recovers():
    """A field with a NaN written in on the host comes back as SPFC_ENONFINITE
    (4), with no state left behind: the next call on a clean field agrees with
    the allocating path again."""
    import torch
    from paper_2012_15133_gb300 import SPFCError, field_energy_noalloc
    n, L, eps, beta = 64, 32.0, 0.1, 1.0
    bad = noisy_field((n, n), 0.2, 0.05, 7)
    bad[3, 5] = np.nan
    with pytest.raises(SPFCError) as ei:
        field_energy_noalloc(torch.tensor(bad, dtype=torch.float64, device="cuda"), L, eps, beta)
    assert ei.value.code == 4
    good = noisy_field((n, n), 0.2, 0.05, 8)
    E_ref, H_ref, m_ref = _reference(good, n, L, eps, beta)
    r = field_energy_noalloc(torch.tensor(good, dtype=torch.float64, device="cuda"), L, eps, beta)
    assert abs(r[0] - E_ref) <= TOL * abs(E_ref) and abs(r[1] - H_ref) <= TOL * abs(H_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2012_15133_gb300 import SPFCError, field_energy_noalloc
    dev = torch.zeros((512, 512), dtype=torch.float64, device="cuda")
    with pytest.raises(SPFCError) as ei:
        field_energy_noalloc(dev, 256.0, 0.25, 1.0)
    assert ei.value.code == 1 and "256" in str(ei.value)
