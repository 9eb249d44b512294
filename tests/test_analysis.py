"""The pattern measures on synthetic lattices (CPU)."""
import numpy as np

from paper_2012_15133_gb300.analysis import bond_order, peak_wavenumber


def _lattice(kind, n=256, L=100.0):
    x = np.arange(n) * L / n
    X, Y = np.meshgrid(x, x)
    q = 2 * np.pi * 16 / L          # 16 periods across the box (|k| ~ 1.005)
    if kind == "square":
        return np.cos(q * X) + np.cos(q * Y), q
    # hexagonal: three waves 120 degrees apart, periodic on the box
    ks = [(q, 0.0), (-q / 2, q * np.sqrt(3) / 2), (-q / 2, -q * np.sqrt(3) / 2)]
    ks = [(2 * np.pi * round(kx * L / (2 * np.pi)) / L, 2 * np.pi * round(ky * L / (2 * np.pi)) / L) for kx, ky in ks]
    return sum(np.cos(kx * X + ky * Y) for kx, ky in ks), q


def test_peak_wavenumber_of_a_cosine():
    phi, q = _lattice("square")
    assert abs(peak_wavenumber(phi, 100.0) - q) < 1e-12


def test_bond_order_tells_square_from_hexagonal():
    sq, _ = _lattice("square")
    o, npk = bond_order(sq, 100.0)
    assert npk == 256 and o[4] > 0.99 and o[6] < 0.5
    hx, _ = _lattice("hex")
    o, npk = bond_order(hx, 100.0)
    assert o[6] > 0.8 and o[4] < 0.5
