"""Pins for the FP64 oracle: each function measures the oracle against
something other than itself (closed forms, brute force, the scheme's defining
equations, exact identities of the paper, textbook recurrences) and returns
the worst relative error. ``test_oracle_pins`` asserts the tolerances and
``test_oracle_mutations`` plants mistakes in the oracle to show that these
pins catch them.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from oracle import spfc_oracle as so
from seeded_inputs import noisy_field


def _rel(a, b, floor=1e-300):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), floor))


# --- P10 / DFT definition ----------------------------------------------------

def pin_dft_bruteforce() -> float:
    """Naive matrix DFT vs a pure-Python double/triple loop of the defining sum."""
    worst = 0.0
    for d, n, L in ((2, (5, 6), (1.0, 2.0)), (3, (3, 4, 5), (1.0, 1.5, 2.0))):
        g = so.Grid(d, n, L)
        rng = np.random.default_rng(7)
        f = rng.standard_normal(g.shape)
        fh = g.dft(f)
        ref = np.zeros(g.shape, dtype=np.complex128)
        for kidx in np.ndindex(*g.shape):
            acc = 0j
            for jidx in np.ndindex(*g.shape):
                ph = 0.0
                for ax in range(d):
                    N = g.shape[ax]
                    ph += kidx[ax] * jidx[ax] / N
                acc += f[jidx] * cmath.exp(-2j * math.pi * ph)
            ref[kidx] = acc / g.P
        worst = max(worst, float(np.max(np.abs(fh - ref))) / float(np.max(np.abs(ref))))
        back = g.idft(fh)
        worst = max(worst, _rel(back, f))
    return worst


def pin_backends() -> float:
    """Naive DFT vs numpy's FFT on 2D/3D, even and odd sizes (P10)."""
    worst = 0.0
    for d, n in ((2, 16), (2, (9, 12)), (3, 8), (3, (5, 6, 7))):
        gn = so.Grid(d, n, 3.0)
        gf = so.Grid(d, n, 3.0, dft="numpy")
        f = noisy_field(gn.shape, 0.1, 1.0, 11)
        a, b = gn.dft(f), gf.dft(f)
        worst = max(worst, float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
        worst = max(worst, _rel(gn.lap(f), gf.lap(f)))
    return worst


# --- P1: spectral derivatives on trigonometric polynomials ---------------------

def pin_derivatives() -> float:
    worst = 0.0
    for d, n, L in ((2, 16, 2.0), (2, (15, 12), (3.0, 1.0)), (3, (8, 10, 9), (1.0, 2.0, 4.0))):
        g = so.Grid(d, n, L)
        coords = np.meshgrid(*[np.arange(g.shape[ax]) * g.h[d - 1 - ax] for ax in range(d)],
                             indexing="ij")
        X = {c: coords[g.axis_of[c]] for c in range(d)}
        rng = np.random.default_rng(3)
        f = np.zeros(g.shape)
        df = [np.zeros(g.shape) for _ in range(d)]
        lapf = np.zeros(g.shape)
        for _ in range(4):
            # random mode with |l_c| < N_c/2 in each coordinate
            ls = [int(rng.integers(-((g.n[c] - 1) // 2), (g.n[c] - 1) // 2 + 1)) for c in range(d)]
            ks = [2 * math.pi * ls[c] / g.L[c] for c in range(d)]
            amp, ph = rng.standard_normal(), rng.uniform(0, 2 * math.pi)
            arg = sum(ks[c] * X[c] for c in range(d)) + ph
            f += amp * np.cos(arg)
            for c in range(d):
                df[c] += -amp * ks[c] * np.sin(arg)
            lapf += -amp * sum(kc * kc for kc in ks) * np.cos(arg)
        for c in range(d):
            worst = max(worst, _rel(g.D(f, c), df[c]))
        worst = max(worst, _rel(g.lap(f), lapf))
        worst = max(worst, _rel(g.div(g.grad(f)), lapf))
    return worst


# --- P2: nonlinear chemical potential and E1 in closed form --------------------

def pin_nonlinear_cosine() -> float:
    """phi = A cos(k x_c): N = 3/4 beta A^3 k^4 (cos kx - cos 3kx) - 2 A k^2 cos kx,
    E1 = |Omega| (beta/4 * 3/8 A^4 k^4 - 1/2 A^2 k^2) + C |Omega|."""
    worst = 0.0
    for d, n, L in ((2, 32, 16.0), (3, 16, 8.0)):
        for c in range(d):
            g = so.Grid(d, n, L)
            for beta in (1.0, 0.7):
                m = so.Model(g, eps=0.25, beta=beta)
                A = 0.8
                ell = 3 if 3 * 3 < g.n[c] // 2 else 2     # keep 3*ell below N/2 (no aliasing)
                k = 2 * math.pi * ell / g.L[c]
                coords = np.meshgrid(*[np.arange(g.shape[ax]) * g.h[d - 1 - ax] for ax in range(d)],
                                     indexing="ij")
                x = coords[g.axis_of[c]]
                phi = A * np.cos(k * x)
                Nref = 0.75 * beta * A ** 3 * k ** 4 * (np.cos(k * x) - np.cos(3 * k * x)) \
                    - 2 * A * k * k * np.cos(k * x)
                worst = max(worst, _rel(m.N_op(phi), Nref))
                E1ref = g.volume * (beta / 4 * 3 / 8 * A ** 4 * k ** 4 - 0.5 * A * A * k * k) \
                    + (1.0 + 1.0 / beta) * g.volume
                worst = max(worst, abs(m.E1(phi) - E1ref) / abs(E1ref))
    return worst


def pin_nonlinear_sympy() -> float:
    """Product modes: N_N and E_{1,N} against sympy's exact calculus (no aliasing:
    the cubic term's degree stays below N/2)."""
    import sympy as sp
    worst = 0.0
    beta_v, a_v = 1.3, 0.8
    x, y, z = sp.symbols("x y z", real=True)
    for d, n, L in ((2, 32, 10.0), (3, 16, 6.0)):
        g = so.Grid(d, n, L)
        m = so.Model(g, eps=1 - a_v, beta=beta_v)
        K = 2 * sp.pi / sp.Rational(int(L))
        if d == 2:
            phi = sp.Rational(3, 10) * sp.cos(2 * K * x) * sp.cos(K * y) + sp.Rational(1, 5) * sp.sin(3 * K * y + sp.Rational(1, 3))
            vars_ = (x, y)
        else:
            phi = sp.Rational(3, 10) * sp.cos(K * x) * sp.sin(2 * K * z) + sp.Rational(1, 4) * sp.cos(K * y + 2 * K * z)
            vars_ = (x, y, z)
        grads = [sp.diff(phi, v) for v in vars_]
        s = sum(gc ** 2 for gc in grads)
        Nexpr = -sum(sp.diff((beta_v * s - 2) * gc, v) for gc, v in zip(grads, vars_))
        lam = sp.lambdify(vars_, Nexpr, "numpy")
        lphi = sp.lambdify(vars_, phi, "numpy")
        mesh = np.meshgrid(*[np.arange(g.n[c]) * g.h[c] for c in range(d)], indexing="xy"
                           if d == 2 else "ij")
        if d == 2:
            X, Y = mesh
            args = (X, Y)
        else:
            # build [z, y, x] arrays explicitly
            zz, yy, xx = np.meshgrid(np.arange(g.n[2]) * g.h[2], np.arange(g.n[1]) * g.h[1],
                                     np.arange(g.n[0]) * g.h[0], indexing="ij")
            args = (xx, yy, zz)
        ph = np.broadcast_to(lphi(*args), g.shape).astype(np.float64)
        Nref = np.broadcast_to(lam(*args), g.shape).astype(np.float64)
        worst = max(worst, _rel(m.N_op(ph), Nref))
        # E1 reference: the analytic |grad phi|^2 summed on a 4x finer grid (the
        # trapezoid rule is exact for these trigonometric polynomials)
        ls = sp.lambdify(vars_, s, "numpy")
        M = 4 * n
        hf = L / M
        fine = np.meshgrid(*[np.arange(M) * hf for _ in range(d)], indexing="ij")
        sv = np.broadcast_to(ls(*fine), (M,) * d).astype(np.float64)
        E1ref = hf ** d * float(np.sum(beta_v / 4 * sv ** 2 - sv)) + m.C * g.volume
        worst = max(worst, abs(m.E1(ph) - E1ref) / abs(E1ref))
    return worst


# --- summation by parts and the lower bound ------------------------------------

def pin_sbp_odd() -> float:
    """<f, Delta g> = -<grad f, grad g>, <f, Delta^2 g> = <Delta f, Delta g>,
    grad.grad = Delta (odd N, eqs. spectral-coll-4-a and spectral-coll-inner product-3)."""
    worst = 0.0
    for d, n in ((2, 15), (3, 9)):
        g = so.Grid(d, n, 2.5)
        f = noisy_field(g.shape, 0.0, 1.0, 5)
        h = noisy_field(g.shape, 0.0, 1.0, 6)
        lhs = g.inner(f, g.lap(h))
        rhs = -sum(g.inner(a, b) for a, b in zip(g.grad(f), g.grad(h)))
        worst = max(worst, abs(lhs - rhs) / abs(rhs))
        lhs2 = g.inner(f, g.lap(g.lap(h)))
        rhs2 = g.inner(g.lap(f), g.lap(h))
        worst = max(worst, abs(lhs2 - rhs2) / abs(rhs2))
        worst = max(worst, _rel(g.div(g.grad(f)), g.lap(f)))
    return worst


def min_E1_margin() -> float:
    """min over random fields and beta of (E1 - |Omega|)/|Omega| (must be >= 0)."""
    lo = float("inf")
    for beta in (0.5, 1.0, 1.5):
        g = so.Grid(2, 16, 4.0)
        m = so.Model(g, 0.2, beta)
        for seed in range(4):
            phi = noisy_field(g.shape, 0.0, 3.0, 40 + seed)
            lo = min(lo, (m.E1(phi) - g.volume) / g.volume)
        # a field whose |grad phi|^2 sits near the minimiser 2/beta everywhere
        k = 2 * math.pi / g.L[0]
        x = np.arange(16) * g.h[0]
        phi = np.broadcast_to(math.sqrt(2 / beta) / k * np.sin(k * x), g.shape)
        lo = min(lo, (m.E1(phi) - g.volume) / g.volume)
    return lo


# --- the scheme -----------------------------------------------------------------

def _case(n=16, L=8.0, dt=0.05, eps=0.25, beta=1.0, amp=0.4, d=2, smooth=0.2, pfc=False):
    o = so.Oracle(d, n, L, eps, beta, dt)
    if pfc:
        o.model.use_pfc(pfc if isinstance(pfc, float) else 1.0)
    phi0 = noisy_field(o.grid.shape, 0.2, amp, 21)
    # smooth the random data a little so that the gradients stay moderate
    g = o.grid
    phi0 = g.idft(g.dft(phi0) * np.exp(-smooth * g.K2))
    return o, phi0


def pin_residual(d=2, gamma3=0.0, pfc=False) -> float:
    """Plug (phi^{n+1}, r^{n+1}) into eq. scheme-SAV-1 (a) and (b) directly."""
    o, phi0 = _case(d=d, n=16 if d == 2 else 8, L=8.0 if d == 2 else 5.0, pfc=pfc)
    if not pfc:
        o.model.gamma3 = gamma3
    o.start(phi0, "ghost")
    worst = 0.0
    m, g, dt = o.model, o.grid, o.dt
    for _ in range(3):
        pn, pnm1, rn, rnm1 = o.phi, o.phi_prev, o.r, o.r_prev
        o.step()
        pnp1, rnp1 = o.phi, o.r
        ph = 2 * pn - pnm1
        sq = math.sqrt(m.E1(ph))
        Nh = m.N_op(ph)
        D = 1.5 * pnp1 - 2 * pn + 0.5 * pnm1
        t_nl = g.lap(rnp1 / sq * Nh)
        t_lin = g.lap(m.L_op(pnp1))
        resa = D / dt - t_nl - t_lin
        # relative to the largest term of (a): the operator's |k|^6 amplifies roundoff
        scale = max(float(np.max(np.abs(t))) for t in (D / dt, t_nl, t_lin))
        worst = max(worst, float(np.max(np.abs(resa))) / scale)
        resb = (1.5 * rnp1 - 2 * rn + 0.5 * rnm1) / dt - g.inner(Nh, D / dt) / (2 * sq)
        worst = max(worst, abs(resb) / ((1.5 * abs(rnp1) + 2 * abs(rn) + 0.5 * abs(rnm1)) / dt))
    return worst


def pin_bdf1_residual() -> float:
    o, phi0 = _case()
    o.start(phi0, "bdf1")
    m, g, dt = o.model, o.grid, o.dt
    sq = math.sqrt(m.E1(phi0))
    Nh = m.N_op(phi0)
    D = o.phi - phi0
    t_nl = g.lap(o.r / sq * Nh)
    t_lin = g.lap(m.L_op(o.phi))
    resa = D / dt - t_nl - t_lin
    scale = max(float(np.max(np.abs(t))) for t in (D / dt, t_nl, t_lin))
    w = float(np.max(np.abs(resa))) / scale
    resb = (o.r - o.r_prev) / dt - g.inner(Nh, D / dt) / (2 * sq)
    return max(w, abs(resb) / ((abs(o.r) + abs(o.r_prev)) / dt), abs(o.r_prev - sq) / sq)


def pin_dissipation(pfc=False) -> float:
    """Exact identity eq. eng stab-5, with ||grad_N mu||^2 written as <-Delta_N mu, mu>.
    Returns the worst |identity residual| / |E^{n+1} - E^n|."""
    o, phi0 = _case(dt=0.1, pfc=pfc)
    o.start(phi0, "bdf1")
    m, g, dt = o.model, o.grid, o.dt
    worst = 0.0
    for _ in range(4):
        pn, pnm1, rn, rnm1 = o.phi, o.phi_prev, o.r, o.r_prev
        Eold = m.E_mod(pn, pnm1, rn, rnm1)
        ph = 2 * pn - pnm1
        sq = math.sqrt(m.E1(ph))
        Nh = m.N_op(ph)
        o.step()
        pnp1, rnp1 = o.phi, o.r
        Enew = m.E_mod(pnp1, pn, rnp1, rn)
        mu = m.L_op(pnp1) + rnp1 / sq * Nh
        dd = pnp1 - 2 * pn + pnm1
        rhs = -0.25 * m.L_norm_sq(dd) - 0.5 * (rnp1 - 2 * rn + rnm1) ** 2 \
            - dt * g.inner(-g.lap(mu), mu)
        worst = max(worst, abs((Enew - Eold) - rhs) / abs(Enew - Eold))
    return worst


def pin_linear_closed_form(pfc=False) -> float:
    """N_N switched off: each Fourier mode follows (3/2 + lam) x_{n+1} = 2 x_n - x_{n-1}/2,
    lam = dt |k|^2 (a + |k|^4) (PFC: dt |k|^2 (a + (1 - |k|^2)^2)), i.e. x_n = c1 z1^n +
    c2 z2^n with z the roots of (3/2 + lam) z^2 - 2 z + 1/2 = 0; r stays constant."""
    o = so.Oracle(2, 12, 6.0, 0.3, 1.0, 0.02, nonlinear=False)
    if pfc:
        o.model.use_pfc(1.0)
    g = o.grid
    phi0 = noisy_field(g.shape, 0.1, 0.5, 9)
    phim1 = noisy_field(g.shape, 0.1, 0.5, 10)
    o.set_state(phi0, phim1, 2.0, 2.0)
    nsteps = 25
    o.step(nsteps)
    x0, xm1 = g.dft(phi0), g.dft(phim1)
    lam = o.dt * g.K2 * ((o.model.a + (1.0 - g.K2) ** 2) if pfc else (o.model.a + g.K2 ** 2))
    worst = 0.0
    out = g.dft(o.phi)
    for idx in np.ndindex(*g.shape):
        lm = float(lam[idx])
        disc = cmath.sqrt(1 - 2 * lm)
        z1 = (2 + disc) / (3 + 2 * lm)
        z2 = (2 - disc) / (3 + 2 * lm)
        # x_0 = c1 + c2, x_{-1} = c1/z1 + c2/z2
        a11, a12, a21, a22 = 1, 1, 1 / z1, 1 / z2
        det = a11 * a22 - a12 * a21
        c1 = (x0[idx] * a22 - a12 * xm1[idx]) / det
        c2 = (a11 * xm1[idx] - a21 * x0[idx]) / det
        ref = c1 * z1 ** nsteps + c2 * z2 ** nsteps
        worst = max(worst, abs(out[idx] - ref) / max(abs(x0[idx]), 1e-12))
    worst = max(worst, abs(o.r - 2.0) / 2.0)
    return worst


def mass_drift(nsteps=40) -> float:
    o, phi0 = _case()
    o.start(phi0, "bdf1")
    m0 = o.grid.mean_value(phi0)
    worst = abs(o.mass() - m0)
    for _ in range(nsteps):
        o.step()
        worst = max(worst, abs(o.mass() - m0))
    return worst / abs(m0)


def constant_state_error() -> float:
    o = so.Oracle(2, 8, 4.0, 0.2, 1.0, 0.1)
    phi0 = np.full(o.grid.shape, 0.37)
    o.start(phi0, "bdf1")
    o.step(5)
    e = float(np.max(np.abs(o.phi - 0.37)))
    E1 = o.model.E1(o.phi)
    return max(e, abs(E1 - o.model.C * o.grid.volume) / E1, abs(o.r - math.sqrt(E1)) / o.r)


def ghost_cosine_error() -> float:
    """Ghost point for phi = A cos(kx): -Delta mu = k^2 mu for a single-x-mode mu,
    with mu = 3/4 b A^3 k^4 (cos - cos3) - 2 A k^2 cos + (a + k^4) A cos, so
    phi^{-1} = phi^0 + dt * (k^2 [..]_cos1 + 9 k^2 [..]_cos3)."""
    g = so.Grid(2, 32, 16.0)
    m = so.Model(g, eps=0.3, beta=1.2)
    A, ell, dt = 0.6, 2, 0.03
    k = 2 * math.pi * ell / g.L[0]
    x = np.broadcast_to(np.arange(32) * g.h[0], g.shape)
    phi = A * np.cos(k * x)
    c1 = 0.75 * m.beta * A ** 3 * k ** 4 - 2 * A * k * k + (m.a + k ** 4) * A
    c3 = -0.75 * m.beta * A ** 3 * k ** 4
    ref = phi + dt * (k * k * c1 * np.cos(k * x) + 9 * k * k * c3 * np.cos(3 * k * x))
    phim1, r0, rm1 = so.ghost_start(m, dt, phi)
    return max(_rel(phim1, ref), abs(r0 - math.sqrt(m.E1(phi))) / r0)


# --- P7: second order in time ----------------------------------------------------

def manufactured_errors(NTs=(50, 100, 200), n=16, a=0.975, T=1.0):
    """Sec. 5.1: phi_e = sin(2 pi x) cos(2 pi y) cos(t) / (2 pi) on (0,1)^2 with the
    paper's a = 0.975 and T = 1, forcing f = d_t phi_e - Delta_N mu_N(phi_e).
    Returns the discrete l2 and l-infinity errors at T, one of each per N_T."""
    l2, linf = [], []
    for NT in NTs:
        dt = T / NT
        o = so.Oracle(2, n, 1.0, 1.0 - a, 1.0, dt)
        g = o.grid
        X = np.broadcast_to(np.arange(n) * g.h[0], g.shape)
        Y = np.broadcast_to((np.arange(n) * g.h[1])[:, None], g.shape)
        base = np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y) / (2 * math.pi)

        def phe(t):
            return base * math.cos(t)

        def forcing(orc):
            t = (orc.nstep + 1) * dt
            return -base * math.sin(t) - g.lap(orc.model.mu(phe(t)))

        o.set_state(phe(0.0), phe(-dt), math.sqrt(o.model.E1(phe(0.0))),
                    math.sqrt(o.model.E1(phe(-dt))))
        o.step(NT, forcing=forcing)
        err = o.phi - phe(T)
        l2.append(math.sqrt(g.inner(err, err)))
        linf.append(float(np.max(np.abs(err))))
    return l2, linf


def manufactured_slope(NTs=(50, 100, 200), norm="l2", a=0.975, T=1.0) -> float:
    """Fitted slope of log(error) against log(N_T) for the Sec. 5.1 test."""
    l2, linf = manufactured_errors(NTs, a=a, T=T)
    errs = l2 if norm == "l2" else linf
    return float(np.polyfit(np.log(NTs), np.log(errs), 1)[0])


def self_convergence_ratio() -> float:
    """Small random-data case, BDF1 start, T fixed: ||u_dt - u_dt/2|| / ||u_dt/2 - u_dt/4||."""
    sols = []
    T = 0.8
    for nt in (32, 64, 128):
        o, phi0 = _case(n=16, L=8.0, dt=T / nt, smooth=1.0)
        o.start(phi0, "bdf1")
        o.step(nt - 1)
        sols.append(o.phi)
    a = np.linalg.norm(sols[0] - sols[1])
    b = np.linalg.norm(sols[1] - sols[2])
    return float(a / b)


# --- the stabilised scheme (Sec. 5.2: - A dt Delta_N (phi^{n+1} - phi^n)) ---------

STAB_A = 3.0


def pin_stab_residual() -> float:
    """Plug (phi^{n+1}, r^{n+1}) of the stabilised scheme into
    (3 phi^{n+1} - 4 phi^n + phi^{n-1})/(2 dt) - A Delta_N (phi^{n+1} - phi^n)
    = Delta_N mu^{n+1} and the unchanged r-equation (b), for the BDF1 start
    (first-order form) and three BDF2 steps."""
    o, phi0 = _case()
    o.model.stab = STAB_A
    m, g, dt = o.model, o.grid, o.dt
    o.start(phi0, "bdf1")
    sq = math.sqrt(m.E1(phi0))
    Nh = m.N_op(phi0)
    D = o.phi - phi0
    terms = (D / dt, STAB_A * g.lap(o.phi - phi0), g.lap(o.r / sq * Nh), g.lap(m.L_op(o.phi)))
    res = terms[0] - terms[1] - terms[2] - terms[3]
    worst = float(np.max(np.abs(res))) / max(float(np.max(np.abs(t))) for t in terms)
    for _ in range(3):
        pn, pnm1, rn, rnm1 = o.phi, o.phi_prev, o.r, o.r_prev
        o.step()
        pnp1, rnp1 = o.phi, o.r
        ph = 2 * pn - pnm1
        sq = math.sqrt(m.E1(ph))
        Nh = m.N_op(ph)
        D = 1.5 * pnp1 - 2 * pn + 0.5 * pnm1
        terms = (D / dt, STAB_A * g.lap(pnp1 - pn), g.lap(rnp1 / sq * Nh), g.lap(m.L_op(pnp1)))
        res = terms[0] - terms[1] - terms[2] - terms[3]
        worst = max(worst, float(np.max(np.abs(res))) / max(float(np.max(np.abs(t))) for t in terms))
        resb = (1.5 * rnp1 - 2 * rn + 0.5 * rnm1) / dt - g.inner(Nh, D / dt) / (2 * sq)
        worst = max(worst, abs(resb) / ((1.5 * abs(rnp1) + 2 * abs(rn) + 0.5 * abs(rnm1)) / dt))
    return worst


def pin_stab_dissipation() -> float:
    """The stabilised equation is (a) with mu~ = mu + A (phi^{n+1} - phi^n):
    testing it with mu~ gives the identity eq. eng stab-5 with -dt ||grad mu~||^2
    and the extra term - A <D, phi^{n+1} - phi^n>, D = 3/2 phi^{n+1} - 2 phi^n
    + 1/2 phi^{n-1}. Returns the worst |residual| / |E^{n+1} - E^n|."""
    o, phi0 = _case(dt=0.1)
    o.model.stab = STAB_A
    o.start(phi0, "bdf1")
    m, g, dt = o.model, o.grid, o.dt
    worst = 0.0
    for _ in range(4):
        pn, pnm1, rn, rnm1 = o.phi, o.phi_prev, o.r, o.r_prev
        Eold = m.E_mod(pn, pnm1, rn, rnm1)
        ph = 2 * pn - pnm1
        sq = math.sqrt(m.E1(ph))
        Nh = m.N_op(ph)
        o.step()
        pnp1, rnp1 = o.phi, o.r
        Enew = m.E_mod(pnp1, pn, rnp1, rn)
        mut = m.L_op(pnp1) + rnp1 / sq * Nh + STAB_A * (pnp1 - pn)
        dd = pnp1 - 2 * pn + pnm1
        D = 1.5 * pnp1 - 2 * pn + 0.5 * pnm1
        rhs = -0.25 * m.L_norm_sq(dd) - 0.5 * (rnp1 - 2 * rn + rnm1) ** 2 \
            - dt * g.inner(-g.lap(mut), mut) - STAB_A * g.inner(D, pnp1 - pn)
        worst = max(worst, abs((Enew - Eold) - rhs) / abs(Enew - Eold))
    return worst


def pin_stab_linear_closed_form() -> float:
    """N_N off, stabiliser on: each mode follows (3/2 + lam + s) x_{n+1} =
    (2 + s) x_n - x_{n-1}/2 with s = A dt |k|^2, solved by its two roots."""
    o = so.Oracle(2, 12, 6.0, 0.3, 1.0, 0.02, nonlinear=False, stab=STAB_A)
    g = o.grid
    phi0 = noisy_field(g.shape, 0.1, 0.5, 9)
    phim1 = noisy_field(g.shape, 0.1, 0.5, 10)
    o.set_state(phi0, phim1, 2.0, 2.0)
    nsteps = 25
    o.step(nsteps)
    x0, xm1 = g.dft(phi0), g.dft(phim1)
    lam = o.dt * g.K2 * (o.model.a + g.K2 ** 2)
    sk = STAB_A * o.dt * g.K2
    out = g.dft(o.phi)
    worst = 0.0
    for idx in np.ndindex(*g.shape):
        A2, B1 = 1.5 + float(lam[idx]) + float(sk[idx]), 2.0 + float(sk[idx])
        disc = cmath.sqrt(B1 * B1 - 2.0 * A2)
        z1, z2 = (B1 + disc) / (2 * A2), (B1 - disc) / (2 * A2)
        det = 1 / z2 - 1 / z1
        c1 = (x0[idx] / z2 - xm1[idx]) / det
        c2 = (xm1[idx] - x0[idx] / z1) / det
        ref = c1 * z1 ** nsteps + c2 * z2 ** nsteps
        worst = max(worst, abs(out[idx] - ref) / max(abs(x0[idx]), 1e-12))
    return worst


def stab_zero_is_the_plain_scheme() -> float:
    """stab = 0 reproduces the scheme of Sec. 2 bit for bit."""
    o1, phi0 = _case()
    o2, _ = _case()
    o2.model.stab = 0.0
    o1.start(phi0, "bdf1").step(3)
    o2.start(phi0, "bdf1").step(3)
    return float(np.max(np.abs(o1.phi - o2.phi)))



# --- the optional phi^4 term (gamma3/4 ||phi||_4^4 in E_1, gamma3 phi^3 in N) ---

def pin_gamma3_cosine() -> float:
    """phi = c0 + A cos(k x_c) with gamma3 on: N gains gamma3 (phi^3 - mean phi^3)
    = gamma3 (3 c0^2 A cos kx + 3/2 c0 A^2 cos 2kx + A^3/4 (3 cos kx + cos 3kx)), and
    E_1 gains gamma3/4 |Omega| (c0^4 + 3 c0^2 A^2 + 3/8 A^4)."""
    worst = 0.0
    for d, n, L in ((2, 32, 16.0), (3, 16, 8.0)):
        g = so.Grid(d, n, L)
        for c in range(d):
            for beta, g3 in ((1.0, 0.6), (0.7, 1.3)):
                m = so.Model(g, eps=0.25, beta=beta)
                m.gamma3 = g3
                A, c0 = 0.8, 0.3
                ell = 3 if 3 * 3 < g.n[c] // 2 else 2
                k = 2 * math.pi * ell / g.L[c]
                coords = np.meshgrid(*[np.arange(g.shape[ax]) * g.h[d - 1 - ax] for ax in range(d)],
                                     indexing="ij")
                x = coords[g.axis_of[c]]
                phi = c0 + A * np.cos(k * x)
                Nref = 0.75 * beta * A ** 3 * k ** 4 * (np.cos(k * x) - np.cos(3 * k * x)) \
                    - 2 * A * k * k * np.cos(k * x) \
                    + g3 * (3 * c0 * c0 * A * np.cos(k * x) + 1.5 * c0 * A * A * np.cos(2 * k * x)
                            + 0.25 * A ** 3 * (3 * np.cos(k * x) + np.cos(3 * k * x)))
                worst = max(worst, _rel(m.N_op(phi), Nref))
                E1ref = g.volume * (beta / 4 * 3 / 8 * A ** 4 * k ** 4 - 0.5 * A * A * k * k) \
                    + (1.0 + 1.0 / beta) * g.volume \
                    + g3 / 4 * g.volume * (c0 ** 4 + 3 * c0 * c0 * A * A + 3 / 8 * A ** 4)
                worst = max(worst, abs(m.E1(phi) - E1ref) / abs(E1ref))
    return worst


def pin_gamma3_variational() -> float:
    """N_N is the gradient of E_{1,N} along mass-preserving directions:
    (E1(phi + e psi) - E1(phi - e psi)) / (2 e) = <N_N(phi), psi> for mean-free psi
    (central differences with one Richardson step: error O(e^4)), with and without gamma3."""
    worst = 0.0
    for d, n, L in ((2, 16, 8.0), (3, 8, 5.0)):
        g = so.Grid(d, n, L)
        phi = noisy_field(g.shape, 0.25, 0.4, 31)
        phi = g.idft(g.dft(phi) * np.exp(-0.2 * g.K2))
        psi = noisy_field(g.shape, 0.0, 1.0, 32)
        psi = psi - psi.mean()
        for g3 in (0.0, 0.9):
            m = so.Model(g, eps=0.25, beta=1.1)
            m.gamma3 = g3
            cd = lambda e: (m.E1(phi + e * psi) - m.E1(phi - e * psi)) / (2 * e)
            fd = (4.0 * cd(5e-4) - cd(1e-3)) / 3.0      # Richardson: O(e^4)
            an = g.inner(m.N_op(phi), psi)
            worst = max(worst, abs(fd - an) / abs(an))
    return worst


# --- energies and mass of the diagnostics in closed form ----------------------

def _coords(g):
    d = g.d
    cs = np.meshgrid(*[np.arange(g.shape[ax]) * g.h[d - 1 - ax] for ax in range(d)], indexing="ij")
    return {c: cs[g.axis_of[c]] for c in range(d)}


def pin_energies_closed_form() -> float:
    """E_N (eq. energy-discrete-spectral), the modified energy of eq. discrete
    energy, E_breve (Sec. 5.2) and the mass <phi, 1> of trigonometric
    polynomials whose grid sums are exact (every harmonic of the quartic terms
    below N/2, so no aliasing):

    * phi = c0 + A cos(k x_c) along each coordinate c:
      ||phi||^2 = |Omega| (c0^2 + A^2/2), ||grad phi||^2 = |Omega| A^2 k^2 / 2,
      ||Delta_N phi||^2 = |Omega| A^2 k^4 / 2, ||grad phi||_4^4 = |Omega| 3/8 A^4 k^4,
      ||phi||_4^4 = |Omega| (c0^4 + 3 c0^2 A^2 + 3/8 A^4);
    * the 2D product mode phi = c0 + A cos(k1 x) cos(k2 y):
      ||phi||^2 = |Omega| (c0^2 + A^2/4), ||grad phi||^2 = |Omega| A^2 (k1^2 + k2^2)/4,
      ||Delta_N phi||^2 = |Omega| A^2 (k1^2 + k2^2)^2 / 4,
      ||grad phi||_4^4 = |Omega| A^4 (9/64 (k1^4 + k2^4) + 2/64 k1^2 k2^2),
      ||phi||_4^4 = |Omega| (c0^4 + 3/2 c0^2 A^2 + 9/64 A^4);
    then E_N = beta/4 G4 + a/2 P2 - G2 + 1/2 D2 + gamma3/4 Q4,
    ||L_N^{1/2} f||^2 = a P2(f) + D2(f), E_mod = 1/4 (||L^{1/2} phi^{n+1}||^2 +
    ||L^{1/2} (2 phi^{n+1} - phi^n)||^2) + 1/2 (r^{n+1 2} + (2 r^{n+1} - r^n)^2) and
    E_breve = a/2 P2 + 1/2 D2 + r^2 (r, r^n given numbers)."""
    worst = 0.0

    def energies(m, P2, G2, D2, G4, Q4):
        return (m.beta / 4 * G4 + 0.5 * m.a * P2 - G2 + 0.5 * D2 + m.gamma3 / 4 * Q4,
                0.5 * m.a * P2 + 0.5 * D2)

    for d, n, L in ((2, (32, 24), (16.0, 12.0)), (3, 16, (8.0, 6.0, 5.0))):
        g = so.Grid(d, n, L)
        X = _coords(g)
        V = g.volume
        for c in range(d):
            for eps, beta, g3 in ((0.25, 1.0, 0.0), (0.6, 0.7, 1.3)):
                m = so.Model(g, eps=eps, beta=beta)
                m.gamma3 = g3
                ell = 2 if 4 * 3 >= g.n[c] else 3              # 4 ell < N: no aliasing
                k = 2 * math.pi * ell / g.L[c]
                terms = {}
                for key, c0, A in (("new", 0.3, 0.8), ("old", -0.1, 0.5), ("psi", 0.7, 1.1)):
                    terms[key] = (V * (c0 ** 2 + A ** 2 / 2), V * A ** 2 * k ** 2 / 2, V * A ** 2 * k ** 4 / 2,
                                  V * 3 / 8 * A ** 4 * k ** 4, V * (c0 ** 4 + 3 * c0 ** 2 * A ** 2 + 3 / 8 * A ** 4))
                phi = 0.3 + 0.8 * np.cos(k * X[c])
                old = -0.1 + 0.5 * np.cos(k * X[c])           # 2 phi - old = 0.7 + 1.1 cos
                EN, EL = energies(m, *terms["new"])
                worst = max(worst, abs(m.E_orig(phi) - EN) / abs(EN))
                r, r_old = 1.7, 1.9
                worst = max(worst, abs(m.E_breve(phi, r) - (EL + r * r)) / (EL + r * r))
                Lnew = m.a * terms["new"][0] + terms["new"][2]
                Lpsi = m.a * terms["psi"][0] + terms["psi"][2]
                Emod = 0.25 * (Lnew + Lpsi) + 0.5 * (r * r + (2 * r - r_old) ** 2)
                worst = max(worst, abs(m.E_mod(phi, old, r, r_old) - Emod) / Emod)
                worst = max(worst, abs(g.mean_value(phi) - 0.3 * V) / (0.3 * V))
        if d == 2:
            for eps, beta, g3 in ((0.25, 1.0, 0.0), (0.4, 1.4, 0.9)):
                m = so.Model(g, eps=eps, beta=beta)
                m.gamma3 = g3
                k1, k2 = 2 * math.pi * 3 / g.L[0], 2 * math.pi * 2 / g.L[1]
                c0, A = 0.2, 0.9
                phi = c0 + A * np.cos(k1 * X[0]) * np.cos(k2 * X[1])
                KK = k1 * k1 + k2 * k2
                P2 = V * (c0 ** 2 + A ** 2 / 4)
                G2 = V * A ** 2 * KK / 4
                D2 = V * A ** 2 * KK ** 2 / 4
                G4 = V * A ** 4 * (9 / 64 * (k1 ** 4 + k2 ** 4) + 2 / 64 * k1 ** 2 * k2 ** 2)
                Q4 = V * (c0 ** 4 + 1.5 * c0 ** 2 * A ** 2 + 9 / 64 * A ** 4)
                EN, EL = energies(m, P2, G2, D2, G4, Q4)
                worst = max(worst, abs(m.E_orig(phi) - EN) / abs(EN))
                worst = max(worst, abs(m.E_breve(phi, 0.4) - (EL + 0.16)) / (EL + 0.16))
                worst = max(worst, abs(m.L_norm_sq(phi) - (m.a * P2 + D2)) / (m.a * P2 + D2))
                worst = max(worst, abs(g.mean_value(phi) - c0 * V) / (c0 * V))
    return worst


def pin_scalar_form() -> float:
    """The scalar form of the solve, r^{n+1} = rho + LHS / (2 sqrt(E1)) from
    (E1, gamma, eta, theta, r^n, r^{n-1}) alone, against r^{n+1} of the full
    elimination of Sec. 2.3 (eq. solver-2 evaluated with the new field), for
    BDF2 steps and the first-order start, plain and stabilised."""
    worst = 0.0
    for stab in (0.0, 3.0):
        o, phi0 = _case()
        o.model.stab = stab
        o.start(phi0, "bdf1")
        i = o.last_info
        worst = max(worst, abs(so.sav_r_update(i["E1"], i["gamma"], i["eta"], i["theta"], 0.0, 0.0, o.dt,
                                               bdf1=True) - o.r) / abs(o.r))
        for _ in range(3):
            r_n, r_nm1 = o.r, o.r_prev
            o.step()
            i = o.last_info
            worst = max(worst, abs(so.sav_r_update(i["E1"], i["gamma"], i["eta"], i["theta"], r_n, r_nm1,
                                                   o.dt) - o.r) / abs(o.r))
    return worst


# --- the PFC model of Sec. 1 (eq. energy-PFC) with its own split -------------

def pin_pfc_closed_form() -> float:
    """phi = c0 + A cos(k x_c) under the PFC model (gamma3 phi^4 / 4, beta = 0):
    N = gamma3 (3 c0^2 A cos kx + 3/2 c0 A^2 cos 2kx + A^3/4 (3 cos kx + cos 3kx)) - A cos kx
    (gamma3 phi^3 - phi with its mean removed);
    E_1 = |Omega| (gamma3/4 (c0^4 + 3 c0^2 A^2 + 3/8 A^4) - 1/2 (c0^2 + A^2/2) + 1 + 1/(4 gamma3));
    L phi = (a + 1) c0 + (a + (1 - k^2)^2) A cos kx (the Swift-Hohenberg operator a + (1 + Delta)^2);
    E_N = the PFC energy of eq. energy-PFC, |Omega| (gamma3/4 (c0^4 + 3 c0^2 A^2 + 3/8 A^4)
    + a/2 (c0^2 + A^2/2) - A^2 k^2 / 2 + A^2 k^4 / 4), and E_N = 1/2 <phi, L phi> + E_1 - C |Omega|."""
    worst = 0.0
    for d, n, L in ((2, (32, 24), (16.0, 12.0)), (3, 16, (8.0, 6.0, 5.0))):
        g = so.Grid(d, n, L)
        X = _coords(g)
        V = g.volume
        for c in range(d):
            for eps, g3 in ((0.25, 1.0), (0.6, 0.7)):
                m = so.Model(g, eps=eps).use_pfc(g3)
                a = m.a
                A, c0 = 0.8, 0.3
                ell = 3 if 3 * 3 < g.n[c] // 2 else 2
                k = 2 * math.pi * ell / g.L[c]
                x = X[c]
                phi = c0 + A * np.cos(k * x)
                Nref = g3 * (3 * c0 * c0 * A * np.cos(k * x) + 1.5 * c0 * A * A * np.cos(2 * k * x)
                             + 0.25 * A ** 3 * (3 * np.cos(k * x) + np.cos(3 * k * x))) - A * np.cos(k * x)
                worst = max(worst, _rel(m.N_op(phi), Nref))
                Q4 = c0 ** 4 + 3 * c0 * c0 * A * A + 3 / 8 * A ** 4
                P2 = c0 ** 2 + A ** 2 / 2
                E1ref = V * (g3 / 4 * Q4 - 0.5 * P2 + 1.0 + 1.0 / (4 * g3))
                worst = max(worst, abs(m.E1(phi) - E1ref) / E1ref)
                Lref = (a + 1.0) * c0 + (a + (1 - k * k) ** 2) * A * np.cos(k * x)
                worst = max(worst, _rel(m.L_op(phi), Lref))
                EN = V * (g3 / 4 * Q4 + a / 2 * P2 - A * A * k * k / 2 + A * A * k ** 4 / 4)
                worst = max(worst, abs(m.E_orig(phi) - EN) / abs(EN))
                split = 0.5 * m.L_norm_sq(phi) + m.E1(phi) - m.C * V
                worst = max(worst, abs(split - EN) / abs(EN))
    return worst


def pfc_lower_bound_margin() -> float:
    """E_1 >= |Omega| for the PFC split: equality at the constant states
    phi = +-1/sqrt(gamma3) (the minimum of gamma3/4 phi^4 - 1/2 phi^2), and
    above it on noisy fields. Returns the smallest (E_1 - |Omega|)/|Omega|
    seen, with the constant states' |E_1 - |Omega|| / |Omega| subtracted."""
    g = so.Grid(2, 16, 7.0)
    lo, eq = np.inf, 0.0
    for g3 in (1.0, 0.3, 2.5):
        m = so.Model(g, eps=0.2).use_pfc(g3)
        for sgn in (1.0, -1.0):
            v = np.full(g.shape, sgn / math.sqrt(g3))
            eq = max(eq, abs(m.E1(v) - g.volume) / g.volume)
        for seed in range(4):
            phi = noisy_field(g.shape, 0.0, 2.0 / math.sqrt(g3), 40 + seed)
            lo = min(lo, (m.E1(phi) - g.volume) / g.volume)
    return lo - eq


def pin_pfc_variational() -> float:
    """N_N of the PFC split is the gradient of E_{1,N} along mass-preserving
    directions (central differences with one Richardson step)."""
    worst = 0.0
    for d, n, L in ((2, 16, 8.0), (3, 8, 5.0)):
        g = so.Grid(d, n, L)
        phi = noisy_field(g.shape, 0.25, 0.6, 33)
        psi = noisy_field(g.shape, 0.0, 1.0, 34)
        psi = psi - psi.mean()
        for g3 in (1.0, 0.45):
            m = so.Model(g, eps=0.25).use_pfc(g3)
            cd = lambda e: (m.E1(phi + e * psi) - m.E1(phi - e * psi)) / (2 * e)
            fd = (4.0 * cd(5e-4) - cd(1e-3)) / 3.0
            an = g.inner(m.N_op(phi), psi)
            worst = max(worst, abs(fd - an) / abs(an))
    return worst
