"""Pins of the FP64 CPU reference of the surrogate network."""
import math

import numpy as np
import pytest

from oracle import fno_reference as F


def _cfg():
    return F.Config(n=16, width=4, m1=3, m2=2, layers=2, proj=5)


def test_truncated_dft_matches_numpy_fft():
    cfg = F.Config(n=32, width=2, m1=5, m2=4, layers=1, proj=2)
    v = np.random.default_rng(0).standard_normal((2, 3, 32, 32))
    vh = F.spec_forward(cfg, v)
    full = np.fft.fft2(v)                      # axes (y, x): full[..., ky, kx]
    ref = full[:, :, cfg.ky][:, :, :, cfg.kx]
    assert np.max(np.abs(vh - ref)) < 1e-10 * np.max(np.abs(ref))


def test_inverse_recovers_fields_within_the_retained_band():
    cfg = F.Config(n=32, width=2, m1=5, m2=4, layers=1, proj=2)
    n = 32
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    band = (np.cos(2 * math.pi * (3 * x + 2 * y) / n) + 0.5 * np.sin(2 * math.pi * (1 * x - 3 * y) / n)
            + 0.25 * np.cos(2 * math.pi * 2 * y / n) + 0.3)
    v = np.broadcast_to(band, (1, 1, n, n)).copy()
    back = F.spec_inverse(cfg, F.spec_forward(cfg, v))
    assert np.max(np.abs(back - v)) < 1e-12


def test_adjoints_by_dot_products():
    cfg = _cfg()
    rng = np.random.default_rng(2)
    v = rng.standard_normal((2, 3, 16, 16))
    gh = rng.standard_normal((2, 3, 4, 3)) + 1j * rng.standard_normal((2, 3, 4, 3))
    lhs = np.sum(np.real(F.spec_forward(cfg, v)) * gh.real + np.imag(F.spec_forward(cfg, v)) * gh.imag)
    rhs = np.sum(v * F.spec_forward_adjoint(cfg, gh))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    oh = rng.standard_normal((2, 3, 4, 3)) + 1j * rng.standard_normal((2, 3, 4, 3))
    g = rng.standard_normal((2, 3, 16, 16))
    lhs2 = np.sum(F.spec_inverse(cfg, oh) * g)
    adj = F.spec_inverse_adjoint(cfg, g)
    rhs2 = np.sum(oh.real * adj.real + oh.imag * adj.imag)
    assert abs(lhs2 - rhs2) < 1e-10 * abs(lhs2)


def test_gradient_against_finite_differences():
    cfg = _cfg()
    rng = np.random.default_rng(3)
    flat = F.init_params(cfg, seed=4) * 3.0 + 0.05 * rng.standard_normal(cfg.nparams())
    B, n = 2, 16
    phi_n = 0.2 + 0.05 * rng.standard_normal((B, n, n))
    phi_nm1 = phi_n + 0.01 * rng.standard_normal((B, n, n))
    target = phi_n + 0.02 * rng.standard_normal((B, n, n))
    eps, beta = np.array([0.1, 0.3]), np.array([0.8, 1.2])
    loss, grad = F.loss_and_grad(cfg, flat, phi_n, phi_nm1, eps, beta, target)
    idx = rng.choice(cfg.nparams(), size=60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = F.loss_and_grad(cfg, flat + e, phi_n, phi_nm1, eps, beta, target)
        lm, _ = F.loss_and_grad(cfg, flat - e, phi_n, phi_nm1, eps, beta, target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (i, fd, grad[i])


def test_prediction_keeps_the_mass():
    cfg = _cfg()
    rng = np.random.default_rng(5)
    flat = F.init_params(cfg, seed=6)
    phi_n = 0.2 + 0.05 * rng.standard_normal((2, 16, 16))
    out = F.predict(cfg, flat, phi_n, phi_n, np.array([0.1, 0.2]), np.array([1.0, 1.0]))
    assert np.max(np.abs(out.mean(axis=(1, 2)) - phi_n.mean(axis=(1, 2)))) < 1e-15
