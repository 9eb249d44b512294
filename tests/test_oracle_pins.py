"""The oracle pinned to closed forms, brute force and the paper's exact identities."""
import pytest

from seeded_inputs import splitmix64, uniform01
import oracle_pins as P


def test_splitmix64_published_values():
    # first outputs of SplitMix64 seeded with 0 and with 1234567 (reference implementation)
    assert [int(v) for v in splitmix64(0, 0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert int(splitmix64(1234567, 0, 1)[0]) == 6457827717110365317
    u = uniform01(5, 0, 10000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_dft_matches_defining_sum():
    assert P.pin_dft_bruteforce() < 1e-13


def test_dft_backends_agree():
    assert P.pin_backends() < 1e-13


def test_spectral_derivatives_trig_polynomials():
    assert P.pin_derivatives() < 1e-12


def test_nonlinear_potential_cosine_closed_form():
    assert P.pin_nonlinear_cosine() < 1e-12


def test_nonlinear_potential_against_symbolic_calculus():
    assert P.pin_nonlinear_sympy() < 1e-12


def test_summation_by_parts_odd_n():
    assert P.pin_sbp_odd() < 1e-12


def test_E1_lower_bound():
    assert P.min_E1_margin() >= -1e-14


def test_scheme_residual_2d():
    assert P.pin_residual(2) < 1e-12


def test_scheme_residual_3d():
    assert P.pin_residual(3) < 1e-12


def test_bdf1_start_residual():
    assert P.pin_bdf1_residual() < 1e-12


def test_exact_dissipation_identity():
    assert P.pin_dissipation() < 1e-9


def test_linear_part_closed_form():
    assert P.pin_linear_closed_form() < 1e-12


def test_mass_conservation():
    assert P.mass_drift() < 1e-13


def test_constant_state_is_steady():
    assert P.constant_state_error() < 1e-13


def test_ghost_point_closed_form():
    assert P.ghost_cosine_error() < 1e-12


def test_second_order_manufactured_solution():
    """The convergence test of Sec. 5.1 as the paper states it (tests/golden/
    sec5_1_convergence.json): the same exact solution, a and T, and the
    slope it reports, in both the l2 and the l-infinity norm."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "sec5_1_convergence.json")) as f:
        gold = json.load(f)
    for norm in ("l2", "linf"):
        slope = P.manufactured_slope(norm=norm, a=gold["a"], T=gold["T"])
        assert abs(slope - gold["slope"]) < gold["slope_tolerance"], (norm, slope)


def test_self_convergence_ratio():
    ratio = P.self_convergence_ratio()
    assert 3.6 < ratio < 4.4, ratio


def test_stabilised_scheme_residual():
    assert P.pin_stab_residual() < 1e-10


def test_stabilised_dissipation_identity():
    assert P.pin_stab_dissipation() < 1e-9


def test_stabilised_linear_part_closed_form():
    assert P.pin_stab_linear_closed_form() < 1e-12


def test_zero_stabiliser_is_the_plain_scheme():
    assert P.stab_zero_is_the_plain_scheme() == 0.0


def test_phi4_term_closed_form():
    assert P.pin_gamma3_cosine() < 1e-12


def test_potential_is_the_variational_derivative_of_E1():
    assert P.pin_gamma3_variational() < 1e-9


def test_scheme_residual_with_phi4_term():
    assert P.pin_residual(2, gamma3=0.8) < 1e-12


def test_energies_and_mass_closed_form():
    """E_N, the modified energy, E_breve and the mass of trigonometric
    polynomials against their closed forms (single modes along each axis of a
    non-square 2D and a non-cubic 3D box, and a 2D product mode)."""
    assert P.pin_energies_closed_form() < 1e-12


def test_scalar_form_of_the_solve():
    assert P.pin_scalar_form() < 1e-13


def test_pfc_split_closed_form():
    """The PFC model of Sec. 1: N, E_1, the operator and the energy of
    eq. energy-PFC in closed form, and the split identity E_N = 1/2 <phi, L phi>
    + E_1 - C |Omega|."""
    assert P.pin_pfc_closed_form() < 1e-12


def test_pfc_split_lower_bound():
    assert P.pfc_lower_bound_margin() >= -1e-14


def test_pfc_potential_is_the_variational_derivative():
    assert P.pin_pfc_variational() < 1e-9


def test_pfc_scheme_residual():
    # relative to the largest term of (a); the Swift-Hohenberg symbol's |k|^2 (1 - |k|^2)^2
    # amplifies the transforms' roundoff about as much as the stabilised scheme's does
    assert P.pin_residual(2, pfc=True) < 1e-10
    assert P.pin_residual(3, pfc=True) < 1e-10


def test_pfc_dissipation_identity():
    assert P.pin_dissipation(pfc=True) < 1e-9


def test_pfc_linear_part_closed_form():
    assert P.pin_linear_closed_form(pfc=True) < 1e-12
