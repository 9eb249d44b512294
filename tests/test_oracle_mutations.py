"""Plant plausible mistakes in the oracle (on the CPU) and check that at least
one pin catches each: a dropped term, a wrong sign or coefficient, a swapped
operand or axis, a wrong normalisation."""
import math

import numpy as np
import pytest

from oracle import spfc_oracle as so
import oracle_pins as P

PINS = [
    (P.pin_dft_bruteforce, lambda v: v < 1e-13),
    (P.pin_derivatives, lambda v: v < 1e-12),
    (P.pin_nonlinear_cosine, lambda v: v < 1e-12),
    (lambda: P.pin_residual(2), lambda v: v < 1e-12),
    (P.pin_bdf1_residual, lambda v: v < 1e-12),
    (P.pin_dissipation, lambda v: v < 1e-9),
    (P.pin_linear_closed_form, lambda v: v < 1e-12),
    (P.ghost_cosine_error, lambda v: v < 1e-12),
    (P.constant_state_error, lambda v: v < 1e-13),
    (P.min_E1_margin, lambda v: v >= -1e-14),
    (lambda: P.manufactured_slope((50, 100)), lambda v: -2.2 < v < -1.8),
    (P.pin_stab_residual, lambda v: v < 1e-10),
    (P.pin_stab_dissipation, lambda v: v < 1e-9),
    (P.pin_stab_linear_closed_form, lambda v: v < 1e-12),
    (P.pin_gamma3_cosine, lambda v: v < 1e-12),
    (P.pin_gamma3_variational, lambda v: v < 1e-9),
    (P.pin_energies_closed_form, lambda v: v < 1e-12),
    (P.pin_scalar_form, lambda v: v < 1e-13),
    (P.pin_pfc_closed_form, lambda v: v < 1e-12),
    (P.pfc_lower_bound_margin, lambda v: v >= -1e-14),
    (P.pin_pfc_variational, lambda v: v < 1e-9),
    (lambda: P.pin_residual(2, pfc=True), lambda v: v < 1e-10),
    (lambda: P.pin_dissipation(pfc=True), lambda v: v < 1e-9),
    (lambda: P.pin_linear_closed_form(pfc=True), lambda v: v < 1e-12),
]


def _some_pin_fails():
    for fn, ok in PINS:
        try:
            v = fn()
        except Exception:
            return True
        if not (isinstance(v, float) and math.isfinite(v) and ok(v)):
            return True
    return False


def _m_drop_laplacian_term(mp):
    def N_op(self, phi):
        g = self.g
        gr = g.grad(phi)
        s = sum(gc * gc for gc in gr)
        return -g.div([self.beta * s * gc for gc in gr])
    mp.setattr(so.Model, "N_op", N_op)


def _m_flip_quartic_sign(mp):
    def N_op(self, phi):
        g = self.g
        gr = g.grad(phi)
        s = sum(gc * gc for gc in gr)
        return g.div([self.beta * s * gc for gc in gr]) + 2.0 * g.div(gr)
    mp.setattr(so.Model, "N_op", N_op)


def _m_swap_derivative_axis(mp):
    def D(self, f, c):
        c2 = (c + 1) % self.d
        return self.idft(1j * self.kt[c2] * self.dft(f))
    mp.setattr(so.Grid, "D", D)


def _m_wrong_bdf2_operator(mp):
    orig = so.A_inv
    mp.setattr(so, "A_inv", lambda model, f, dt, c0: orig(model, f, dt, 1.0 if c0 == 1.5 else c0))


def _m_wrong_r_coefficient(mp):
    orig = so.bdf2_sav_step

    def step(model, dt, pn, pnm1, rn, rnm1, forcing=None):
        phi, r, info = orig(model, dt, pn, pnm1, rn, rnm1, forcing)
        ph = 2 * pn - pnm1
        Nh = model.N_op(ph)
        sq = math.sqrt(model.E1(ph))
        g = model.g
        D = 1.5 * phi - 2 * pn + 0.5 * pnm1
        # 1/(2 sqrt E1) in place of 1/(3 sqrt E1)
        r = 4 / 3 * rn - 1 / 3 * rnm1 + g.inner(Nh, D) / (2 * sq)
        return phi, r, info
    mp.setattr(so, "bdf2_sav_step", step)


def _m_E1_constant_ignores_beta(mp):
    orig = so.Model.__init__

    def init(self, grid, eps, beta=1.0, nonlinear=True):
        orig(self, grid, eps, beta, nonlinear)
        self.C = 2.0
    mp.setattr(so.Model, "__init__", init)


def _m_energy_quarter_dropped(mp):
    def E_mod(self, pn, po, rn, ro):
        psi = 2 * pn - po
        return 0.5 * (self.L_norm_sq(pn) + self.L_norm_sq(psi)) + 0.5 * (rn ** 2 + (2 * rn - ro) ** 2)
    mp.setattr(so.Model, "E_mod", E_mod)


def _m_first_order_extrapolation(mp):
    orig = so.bdf2_sav_step

    def step(model, dt, pn, pnm1, rn, rnm1, forcing=None):
        # evaluate E1 and N_N at phi^n instead of the extrapolation 2 phi^n - phi^{n-1}
        return _first_order(orig, model, dt, pn, pnm1, rn, rnm1, forcing)
    mp.setattr(so, "bdf2_sav_step", step)


def _first_order(orig, model, dt, pn, pnm1, rn, rnm1, forcing):
    real_E1, real_N = model.E1, model.N_op
    try:
        model.E1 = lambda phi: real_E1(pn)
        model.N_op = lambda phi: real_N(pn)
        return orig(model, dt, pn, pnm1, rn, rnm1, forcing)
    finally:
        del model.E1, model.N_op


def _m_dft_missing_normalisation(mp):
    orig = so.Grid.dft
    mp.setattr(so.Grid, "dft", lambda self, f: orig(self, f) * self.P)


def _m_linear_operator_sign(mp):
    def L_op(self, f):
        g = self.g
        return self.a * f - g.lap(g.lap(f))
    mp.setattr(so.Model, "L_op", L_op)


def _m_laplacian_drops_nyquist(mp):
    def lap(self, f):
        return self.idft(-sum(kt ** 2 for kt in self.kt) * self.dft(f))
    mp.setattr(so.Grid, "lap", lap)


def _m_stab_rhs_sign(mp):
    orig = so.stab_rhs
    mp.setattr(so, "stab_rhs", lambda model, dt, phi: -orig(model, dt, phi) if model.stab else 0.0)


def _m_stab_rhs_dropped(mp):
    mp.setattr(so, "stab_rhs", lambda model, dt, phi: 0.0)


def _m_stab_symbol_dropped(mp):
    def A_inv(model, f, dt, c0):
        g = model.g
        return g.idft(g.dft(f) / (c0 + dt * g.K2 * (model.a + g.K2 ** 2)))
    mp.setattr(so, "A_inv", A_inv)


def _m_stab_symbol_without_dt(mp):
    def A_inv(model, f, dt, c0):
        g = model.g
        return g.idft(g.dft(f) / (c0 + dt * g.K2 * (model.a + g.K2 ** 2) + model.stab * g.K2))
    mp.setattr(so, "A_inv", A_inv)


def _m_gamma3_dropped_from_N(mp):
    orig = so.Model.N_op

    def N_op(self, phi):
        g3, self.gamma3 = self.gamma3, 0.0
        try:
            return orig(self, phi)
        finally:
            self.gamma3 = g3
    mp.setattr(so.Model, "N_op", N_op)


def _m_gamma3_energy_factor(mp):
    orig = so.Model.E1

    def E1(self, phi):
        return orig(self, phi) + (self.gamma3 / 4.0) * self.g.hd * float(np.sum(phi ** 4))
    mp.setattr(so.Model, "E1", E1)


def _m_gamma3_mean_kept(mp):
    orig = so.Model.N_op

    def N_op(self, phi):
        n = orig(self, phi)
        return n + float(np.mean(self.gamma3 * phi ** 3)) if self.gamma3 else n
    mp.setattr(so.Model, "N_op", N_op)


def _m_original_energy_half_dropped(mp):
    def E_orig(self, phi):
        g = self.g
        s = self.grad_sq(phi)
        lp = g.lap(phi)
        return (self.beta / 4.0) * g.hd * float(np.sum(s * s)) + 0.5 * self.a * g.inner(phi, phi) \
            - g.hd * float(np.sum(s)) + g.inner(lp, lp) + (self.gamma3 / 4.0) * g.hd * float(np.sum(phi ** 4))
    mp.setattr(so.Model, "E_orig", E_orig)


def _m_original_energy_gamma3_dropped(mp):
    orig = so.Model.E_orig

    def E_orig(self, phi):
        return orig(self, phi) - (self.gamma3 / 4.0) * self.g.hd * float(np.sum(phi ** 4))
    mp.setattr(so.Model, "E_orig", E_orig)


def _m_breve_energy_without_a(mp):
    def E_breve(self, phi, r):
        g = self.g
        lp = g.lap(phi)
        return 0.5 * g.inner(phi, phi) + 0.5 * g.inner(lp, lp) + r * r
    mp.setattr(so.Model, "E_breve", E_breve)


def _m_modified_energy_swapped_levels(mp):
    def E_mod(self, pn, po, rn, ro):
        psi = 2 * po - pn
        return 0.25 * (self.L_norm_sq(pn) + self.L_norm_sq(psi)) + 0.5 * (rn ** 2 + (2 * rn - ro) ** 2)
    mp.setattr(so.Model, "E_mod", E_mod)


def _m_mass_without_cell_volume(mp):
    mp.setattr(so.Grid, "mean_value", lambda self, f: float(np.sum(f)))


def _m_scalar_form_rho_half(mp):
    orig = so.sav_r_update

    def upd(E1, gamma, eta, theta, r_n, r_nm1, dt, bdf1=False):
        # theta / (2 sqrt E1) in rho where the BDF2 form has theta / (3 sqrt E1)
        return orig(E1, gamma, eta, 1.5 * theta, r_n, r_nm1, dt, bdf1) if not bdf1 else \
            orig(E1, gamma, eta, theta, r_n, r_nm1, dt, bdf1)
    mp.setattr(so, "sav_r_update", upd)


def _m_pfc_symbol_sign(mp):
    orig = so.Model.L_symbol
    mp.setattr(so.Model, "L_symbol", lambda self, K2: self.a + (1.0 + K2) ** 2 if self.pfc else orig(self, K2))


def _m_pfc_operator_drops_laplacian(mp):
    orig = so.Model.L_op

    def L_op(self, f):
        if self.pfc:
            lf = self.g.lap(f)
            return (self.a + 1.0) * f + self.g.lap(lf)
        return orig(self, f)
    mp.setattr(so.Model, "L_op", L_op)


def _m_pfc_potential_keeps_linear_term_out(mp):
    orig = so.Model.N_op

    def N_op(self, phi):
        n = orig(self, phi)
        return n + (phi - float(np.mean(phi))) if self.pfc else n
    mp.setattr(so.Model, "N_op", N_op)


def _m_pfc_energy_constant(mp):
    orig = so.Model.use_pfc

    def use_pfc(self, gamma3=1.0):
        orig(self, gamma3)
        self.C = 1.0 + 1.0 / (2.0 * self.gamma3)
        return self
    mp.setattr(so.Model, "use_pfc", use_pfc)


MUTATIONS = [_m_drop_laplacian_term, _m_flip_quartic_sign, _m_swap_derivative_axis,
             _m_wrong_bdf2_operator, _m_wrong_r_coefficient, _m_E1_constant_ignores_beta,
             _m_energy_quarter_dropped, _m_first_order_extrapolation,
             _m_dft_missing_normalisation, _m_linear_operator_sign, _m_laplacian_drops_nyquist,
             _m_stab_rhs_sign, _m_stab_rhs_dropped, _m_stab_symbol_dropped, _m_stab_symbol_without_dt,
             _m_gamma3_dropped_from_N, _m_gamma3_energy_factor, _m_gamma3_mean_kept,
             _m_original_energy_half_dropped, _m_original_energy_gamma3_dropped, _m_breve_energy_without_a,
             _m_modified_energy_swapped_levels, _m_mass_without_cell_volume, _m_scalar_form_rho_half,
             _m_pfc_symbol_sign, _m_pfc_operator_drops_laplacian, _m_pfc_potential_keeps_linear_term_out,
             _m_pfc_energy_constant]


def test_pins_pass_unmutated():
    assert not _some_pin_fails()


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m.__name__[3:] for m in MUTATIONS])
def test_pins_catch_mutation(mutation, monkeypatch):
    mutation(monkeypatch)
    assert _some_pin_fails()
