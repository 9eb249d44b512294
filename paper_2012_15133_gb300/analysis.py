"""Host-side measures of a 2D density field (numpy), for the square-pattern
runs of Sec. 5.2: the dominant wave number of the structure factor and the
bond-orientational order of the density maxima."""
from __future__ import annotations

import numpy as np


def peak_wavenumber(phi, L):
    """|k| at the maximum of |FFT(phi - mean)|^2 on a square box of side L."""
    n = phi.shape[0]
    F = np.abs(np.fft.rfft2(phi - phi.mean())) ** 2
    ky = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    kx = 2 * np.pi * np.fft.rfftfreq(n, d=L / n)
    K = np.hypot(ky[:, None], kx[None, :])
    return float(K.flat[np.argmax(F)])


def bond_order(phi, L, orders=(4, 6)):
    """Mean |psi_m| over the local maxima of phi (periodic box of side L),
    psi_m = mean over the m nearest maxima of exp(i m theta): near 1 on a
    square lattice for m = 4, on a hexagonal one for m = 6. Returns
    ({m: mean |psi_m|}, number of maxima)."""
    n = phi.shape[0]
    h = L / n
    nb = [np.roll(np.roll(phi, dy, 0), dx, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0)]
    peak = np.all([phi > q for q in nb], axis=0) & (phi > phi.mean() + 0.5 * phi.std())
    ys, xs = np.nonzero(peak)
    pts = np.stack([xs * h, ys * h], 1)
    out = {}
    for m in orders:
        vals = []
        for p in pts:
            d = pts - p
            d -= L * np.round(d / L)
            r = np.hypot(d[:, 0], d[:, 1])
            idx = np.argsort(r)[1:m + 1]
            th = np.arctan2(d[idx, 1], d[idx, 0])
            vals.append(abs(np.mean(np.exp(1j * m * th))))
        out[m] = float(np.mean(vals)) if vals else 0.0
    return out, len(pts)
