"""FP64 CPU oracle for the BDF2 scalar-auxiliary-variable (SAV) Fourier
pseudo-spectral scheme for the square phase field crystal (SPFC) equation.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this module; only the test suite, the smoke check and the CPU
baseline leg of the benchmark use it. It shares no code with the CUDA path:
its only common dependency is ``seeded_inputs`` (random numbers, no method).

Everything here is plain and slow on purpose: real grid functions in float64,
a naive separable discrete Fourier transform built from explicit cos/sin
matrices (no FFT), and the scheme's solve taken in the order the paper's
Sec. 2.3 derives it (eqs. solver-1 .. solver-6), so that each line can be
checked against the paper by eye.

Readings where the paper is silent or leaves a choice (each listed in the
design notes of the repository):

* Domain ``[0, L]^d`` with ``N`` points per axis, ``h = L/N`` (the analysis
  uses ``(0,1)^d`` and odd N, Sec. 2.1; the experiments use ``(0, L)^2``,
  Sec. 5.2). Wave numbers ``k = 2 pi l / L`` with ``l`` in DFT order.
* Even N: first derivatives ``D_x, D_y, D_z`` use the symbol ``i k`` with the
  Nyquist wave number set to 0, so that they map real grid functions to real
  grid functions; the Laplacian ``Delta_N`` (eq. spectral-coll-3), ``L_N``
  and ``A_N`` keep the full ``|k|^2`` including Nyquist. Inside the nonlinear
  chemical potential the ``2 Delta phi`` term is evaluated as
  ``2 grad_N . grad_N phi``, which is the paper's identity
  eq. spectral-coll-4-a and makes ``N_N`` the exact variational derivative of
  ``E_{1,N}``. For odd N all of these coincide with the paper.
* A coefficient ``beta`` multiplies the ``1/4 |grad phi|^4`` term (the paper
  fixes it at 1, eq. energy-SPFC). The constant in ``E_1`` becomes
  ``C_beta = 1 + 1/beta`` so that ``E_{1,N} >= |Omega|`` still holds
  (eq. energy-SPFC-split-2-2); at beta = 1 it is the paper's 2.
* ``a = 1 - eps`` (Sec. 1).
* Startup: the paper's ghost point (eq. scheme-SAV-initial-1), the copy
  restart ``phi^{-1} = phi^0`` of Sec. 5.2, and a first-order SAV step
  (BDF1-SAV: the same construction with ``(phi^1 - phi^0)/dt``), which the
  paper does not print.
* The manufactured-solution forcing of Sec. 5.1, which the paper adds
  without writing it, is ``f = d_t phi_e - Delta_N mu_N(phi_e)`` on the grid,
  added to the right-hand side of eq. scheme-SAV-1 (a).
* The PFC model of Sec. 1 (eq. energy-PFC, phi^4 in place of |grad phi|^4),
  which the paper states but does not discretise, with gamma3 the phi^4
  coefficient (1 in the paper): the SPFC split cannot be reused (beta = 0
  leaves -||grad phi||^2 without a lower bound), so the concave term goes to
  the linear part as the Swift-Hohenberg operator: ``L = a + (1 + Delta)^2``
  (symbol ``a + (1 - |k|^2)^2 > 0``), which counts ``1/2 ||phi||^2`` more
  than the energy has, and ``E_1 = gamma3/4 ||phi||_4^4 - 1/2 ||phi||^2 +
  C |Omega|`` takes it back; ``C = 1 + 1/(4 gamma3)`` makes the integrand
  ``gamma3/4 (phi^2 - 1/gamma3)^2 + 1 >= 1``, so ``E_1 >= |Omega|`` as in
  eq. energy-SPFC-split-2-2. ``N = gamma3 phi^3 - phi`` (mean removed), and
  the SAV scheme of Sec. 2.2-2.3 is otherwise unchanged.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Grid, wave numbers and the naive discrete Fourier transform (Sec. 2.1)
# ---------------------------------------------------------------------------

class Grid:
    """Periodic grid on ``[0, L]^d`` with ``n`` points per axis.

    Arrays are indexed ``[y, x]`` in 2D and ``[z, y, x]`` in 3D (x fastest).
    ``axis_of[c]`` gives the numpy axis of coordinate ``c`` (0 = x, 1 = y,
    2 = z).
    """

    def __init__(self, d: int, n, L, dft: str = "naive"):
        if d not in (2, 3):
            raise ValueError("d must be 2 or 3")
        n = (int(n),) * d if np.isscalar(n) else tuple(int(v) for v in n)
        L = (float(L),) * d if np.isscalar(L) else tuple(float(v) for v in L)
        if len(n) != d or len(L) != d:
            raise ValueError("n and L need d entries (x first)")
        self.d = d
        self.n = n            # per coordinate: n[0] = Nx, n[1] = Ny, ...
        self.L = L
        self.shape = tuple(reversed(n))
        self.axis_of = [d - 1 - c for c in range(d)]
        self.h = tuple(L[c] / n[c] for c in range(d))
        self.hd = float(np.prod(self.h))          # h^d in <f,g> = h^d sum f g
        self.volume = float(np.prod(L))           # |Omega|
        self.P = int(np.prod(n))
        self.dft_kind = dft
        # integer modes l in DFT order, wave numbers k = 2 pi l / L
        self.k = []       # full wave numbers per coordinate (broadcastable)
        self.kt = []      # first-derivative wave numbers (Nyquist -> 0)
        self._F = []      # naive DFT matrices per coordinate
        for c in range(d):
            N = n[c]
            idx = np.arange(N)
            ell = np.where(idx <= (N - 1) // 2, idx, idx - N).astype(np.float64)
            kc = 2.0 * math.pi * ell / L[c]
            ktc = kc.copy()
            if N % 2 == 0:
                ktc[N // 2] = 0.0
            bshape = [1] * d
            bshape[self.axis_of[c]] = N
            self.k.append(kc.reshape(bshape))
            self.kt.append(ktc.reshape(bshape))
            # F[l, j] = exp(-2 pi i l j / N), angle reduced exactly mod N
            m = np.outer(idx, idx) % N
            ang = 2.0 * math.pi * m / N
            self._F.append(np.cos(ang) - 1j * np.sin(ang))
        self.K2 = sum(kc ** 2 for kc in self.k)   # |k|^2, Nyquist included

    # f_hat = (1/P) sum_j f_j exp(-i k . x_j)   (eq. spectral-coll-1 with
    # h^d -> 1/P on a general box)
    def dft(self, f: np.ndarray) -> np.ndarray:
        if self.dft_kind == "numpy":
            return np.fft.fftn(f) / self.P
        out = np.asarray(f, dtype=np.complex128)
        for c in range(self.d):
            ax = self.axis_of[c]
            out = np.moveaxis(np.tensordot(self._F[c], out, axes=([1], [ax])), 0, ax)
        return out / self.P

    # f_j = sum_k f_hat_k exp(+i k . x_j); the real part is returned and the
    # imaginary part is checked to be roundoff
    def idft(self, fh: np.ndarray) -> np.ndarray:
        if self.dft_kind == "numpy":
            out = np.fft.ifftn(fh) * self.P
        else:
            out = np.asarray(fh, dtype=np.complex128)
            for c in range(self.d):
                ax = self.axis_of[c]
                out = np.moveaxis(np.tensordot(np.conj(self._F[c]), out, axes=([1], [ax])), 0, ax)
        scale = max(1.0, float(np.max(np.abs(out.real))))
        if np.max(np.abs(out.imag)) > 1e-9 * scale:
            raise AssertionError("inverse DFT of a non-Hermitian spectrum")
        return out.real

    # --- operators of Sec. 2.1 ---------------------------------------------
    def D(self, f, c):
        """Collocation first derivative in coordinate c (eq. spectral-coll-2-1)."""
        return self.idft(1j * self.kt[c] * self.dft(f))

    def grad(self, f):
        """grad_N f (eq. spectral-coll-3)."""
        return [self.D(f, c) for c in range(self.d)]

    def div(self, vs):
        """grad_N . (v_1, .., v_d) (eq. spectral-coll-3)."""
        return sum(self.D(vs[c], c) for c in range(self.d))

    def lap(self, f):
        """Delta_N f = (D_x^2 + D_y^2 + D_z^2) f with symbol -|k|^2 (eq. spectral-coll-2-3)."""
        return self.idft(-self.K2 * self.dft(f))

    def inner(self, f, g) -> float:
        """<f, g> = h^d sum f g (eq. spectral-coll-inner product-1)."""
        return self.hd * float(np.sum(f * g))

    def mean_value(self, f) -> float:
        """<f, 1>, the quantity the paper calls the mean (Sec. 2.1)."""
        return self.hd * float(np.sum(f))


# ---------------------------------------------------------------------------
# Energies and chemical potentials (Sec. 2.2)
# ---------------------------------------------------------------------------

class Model:
    """SPFC parameters: a = 1 - eps, the |grad phi|^4 coefficient beta."""

    def __init__(self, grid: Grid, eps: float, beta: float = 1.0, nonlinear: bool = True):
        if not (0.0 < 1.0 - eps):
            raise ValueError("a = 1 - eps must be positive")
        self.g = grid
        self.a = 1.0 - eps
        self.beta = float(beta)
        self.C = 1.0 + 1.0 / self.beta       # C_beta; 2 at beta = 1
        self.nonlinear = nonlinear            # test switch: False sets N_N := 0
        self.stab = 0.0                       # A of the stabilised scheme (Sec. 5.2); 0: Sec. 2
        self.gamma3 = 0.0                     # optional gamma3/4 phi^4 in E_1 (the PFC term); 0: SPFC
        self.pfc = False                      # the PFC model of Sec. 1 with its own split

    def use_pfc(self, gamma3: float = 1.0):
        """Switch to the PFC model (eq. energy-PFC) with phi^4 coefficient gamma3 > 0:
        no |grad phi|^4 term (beta = 0), L = a + (1 + Delta)^2, E_1 = gamma3/4 ||phi||_4^4
        - 1/2 ||phi||^2 + (1 + 1/(4 gamma3)) |Omega|, N = gamma3 phi^3 - phi."""
        if not gamma3 > 0.0:
            raise ValueError("the PFC model needs gamma3 > 0")
        self.pfc = True
        self.gamma3 = float(gamma3)
        self.beta = 0.0
        self.C = 1.0 + 1.0 / (4.0 * self.gamma3)
        return self

    def L_symbol(self, K2):
        """Fourier symbol of L_N: a + |k|^4 (SPFC, Sec. 2.2) or a + (1 - |k|^2)^2 (PFC)."""
        return self.a + (1.0 - K2) ** 2 if self.pfc else self.a + K2 ** 2

    def L_op(self, f):
        """L_N f = a f + Delta_N^2 f (Sec. 2.1, before eq. spectral-coll-6); for the PFC
        model a f + (1 + Delta_N)^2 f = (a + 1) f + 2 Delta_N f + Delta_N^2 f."""
        g = self.g
        if self.pfc:
            lf = g.lap(f)
            return (self.a + 1.0) * f + 2.0 * lf + g.lap(lf)
        return self.a * f + g.lap(g.lap(f))

    def grad_sq(self, phi):
        """|grad_N phi|^2 pointwise."""
        return sum(gc * gc for gc in self.g.grad(phi))

    def E1(self, phi) -> float:
        """E_{1,N}(phi) = beta/4 ||grad_N phi||_4^4 - ||grad_N phi||_2^2 + C |Omega| (Sec. 2.2),
        plus gamma3/4 ||phi||_4^4 when the optional phi^4 term is on (E_1 >= |Omega| still)."""
        g = self.g
        if self.pfc:
            return (self.gamma3 / 4.0) * g.hd * float(np.sum(phi ** 4)) - 0.5 * g.hd * float(np.sum(phi * phi)) \
                + self.C * g.volume
        s = self.grad_sq(phi)
        e = (self.beta / 4.0) * g.hd * float(np.sum(s * s)) - g.hd * float(np.sum(s)) + self.C * g.volume
        if self.gamma3:
            e += (self.gamma3 / 4.0) * g.hd * float(np.sum(phi ** 4))
        return e

    def N_op(self, phi):
        """N_N(phi) = -grad_N . (beta |grad_N phi|^2 grad_N phi) + 2 grad_N . grad_N phi
        (eq. nonlinear chem pot-1 at the grid level, scheme-SAV-1)."""
        g = self.g
        if not self.nonlinear:
            return np.zeros(g.shape)
        if self.pfc:
            # the variational derivative of gamma3/4 ||phi||_4^4 - 1/2 ||phi||^2, mean removed
            n = self.gamma3 * phi ** 3 - phi
            return n - float(np.mean(n))
        gr = g.grad(phi)
        s = sum(gc * gc for gc in gr)
        n = -g.div([self.beta * s * gc for gc in gr]) + 2.0 * g.div(gr)
        if self.gamma3:
            # + gamma3 phi^3, the variational derivative of gamma3/4 ||phi||_4^4, with its
            # mean removed (N_hat_0 := 0: the divergence terms have none, and the zero mode
            # of N never enters the scheme, whose solution keeps the mass)
            c = self.gamma3 * phi ** 3
            n = n + c - float(np.mean(c))
        return n

    def mu(self, phi):
        """mu_N = N_N(phi) + L_N phi (eq. equation-SPFC at the grid level)."""
        return self.N_op(phi) + self.L_op(phi)

    def E_orig(self, phi) -> float:
        """E_N(phi) = beta/4 ||grad phi||_4^4 + a/2 ||phi||^2 - ||grad phi||^2 + 1/2 ||Delta_N phi||^2
        (eq. energy-discrete-spectral)."""
        g = self.g
        s = self.grad_sq(phi)
        lp = g.lap(phi)
        e = (self.beta / 4.0) * g.hd * float(np.sum(s * s)) + 0.5 * self.a * g.inner(phi, phi) \
            - g.hd * float(np.sum(s)) + 0.5 * g.inner(lp, lp)
        if self.gamma3:
            e += (self.gamma3 / 4.0) * g.hd * float(np.sum(phi ** 4))
        return e

    def L_norm_sq(self, f) -> float:
        """||L_N^{1/2} f||^2 = <f, L_N f> (eq. spectral-coll-inner product-4)."""
        return self.g.inner(f, self.L_op(f))

    def E_mod(self, phi_new, phi_old, r_new, r_old) -> float:
        """Modified energy of Theorem SPFC-energy stability (eq. discrete energy)."""
        psi = 2.0 * phi_new - phi_old
        return 0.25 * (self.L_norm_sq(phi_new) + self.L_norm_sq(psi)) \
            + 0.5 * (r_new ** 2 + (2.0 * r_new - r_old) ** 2)

    def E_breve(self, phi, r) -> float:
        """a/2 ||phi||^2 + 1/2 ||Delta_N phi||^2 + |r|^2, the SAV energy plotted in Sec. 5.2."""
        g = self.g
        if self.pfc:  # 1/2 <phi, L_N phi> + r^2 with the PFC operator
            return 0.5 * self.L_norm_sq(phi) + r * r
        lp = g.lap(phi)
        return 0.5 * self.a * g.inner(phi, phi) + 0.5 * g.inner(lp, lp) + r * r


# ---------------------------------------------------------------------------
# The scheme (Sec. 2.2 / 2.3)
# ---------------------------------------------------------------------------

def A_inv(model: Model, f, dt: float, c0: float):
    """Solve (c0 I - dt Delta_N L_N - A dt Delta_N) u = f by division in
    Fourier space (A = model.stab, 0 for the scheme of Sec. 2).

    c0 = 3/2 gives A_N of eq. solver-1; c0 = 1 the first-order operator.
    The symbol is c0 + dt |k|^2 (a + |k|^4) + A dt |k|^2 > 0 (for the PFC model
    a + (1 - |k|^2)^2 in place of a + |k|^4).
    """
    g = model.g
    sym = c0 + dt * g.K2 * model.L_symbol(g.K2) + model.stab * dt * g.K2
    return g.idft(g.dft(f) / sym)


def stab_rhs(model: Model, dt: float, phi_n):
    """Right-hand-side part of the stabiliser of Sec. 5.2: the left side of (a)
    times dt gains - A dt Delta_N (phi^{n+1} - phi^n), whose phi^n part moves to
    the right as - A dt Delta_N phi^n (zero for the scheme of Sec. 2)."""
    if not model.stab:
        return 0.0
    return -model.stab * dt * model.g.lap(phi_n)


def bdf2_sav_step(model: Model, dt: float, phi_n, phi_nm1, r_n: float, r_nm1: float,
                  forcing=None):
    """One step of eq. scheme-SAV-1, solved as in Sec. 2.3.

    ``forcing`` (grid function or None) is added to the right-hand side of
    (a) (used by the manufactured-solution test of Sec. 5.1).
    Returns (phi_{n+1}, r_{n+1}, info).
    """
    g = model.g
    phi_hat = 2.0 * phi_n - phi_nm1                 # explicit extrapolation
    E1 = model.E1(phi_hat)
    sqE1 = math.sqrt(E1)
    Nh = model.N_op(phi_hat)
    lapN = g.lap(Nh)
    # right-hand side g_N^n after substituting eq. solver-2 into eq. solver-1
    base = 2.0 * phi_n - 0.5 * phi_nm1 + stab_rhs(model, dt, phi_n)
    if forcing is not None:
        base = base + dt * forcing
    coef = (4.0 / 3.0) * r_n - (1.0 / 3.0) * r_nm1 \
        + g.inner(Nh, -2.0 * phi_n + 0.5 * phi_nm1) / (3.0 * sqE1)
    gN = (dt / sqE1) * coef * lapN + base
    Ainv_g = A_inv(model, gN, dt, 1.5)
    Ainv_lapN = A_inv(model, lapN, dt, 1.5)
    gam = g.inner(Nh, Ainv_lapN)                                   # eq. solver-5: <= 0
    denom = 1.0 - dt / (2.0 * E1) * gam
    LHS = g.inner(Nh, Ainv_g) / denom                              # eq. solver-4
    phi_np1 = (dt / (2.0 * E1)) * LHS * Ainv_lapN + Ainv_g         # eq. solver-6
    r_np1 = (4.0 / 3.0) * r_n - (1.0 / 3.0) * r_nm1 \
        + g.inner(Nh, 1.5 * phi_np1 - 2.0 * phi_n + 0.5 * phi_nm1) / (3.0 * sqE1)  # eq. solver-2
    # the two remaining inner products of the scalar form of the solve (diagnostics):
    # eta = <N, A^{-1} (2 phi^n - phi^{n-1}/2 + stabiliser)>, theta = <N, 2 phi^n - phi^{n-1}/2>
    eta = g.inner(Nh, A_inv(model, 2.0 * phi_n - 0.5 * phi_nm1 + stab_rhs(model, dt, phi_n), dt, 1.5))
    theta = g.inner(Nh, 2.0 * phi_n - 0.5 * phi_nm1)
    info = dict(E1=E1, sqrtE1=sqE1, gamma=gam, denom=denom, LHS=LHS, xi=r_np1 / sqE1, eta=eta, theta=theta)
    return phi_np1, r_np1, info


def sav_r_update(E1: float, gamma: float, eta: float, theta: float, r_n: float, r_nm1: float, dt: float,
                 bdf1: bool = False) -> float:
    """r^{n+1} from the step's scalars alone: eq. solver-2 with <N, phi^{n+1}> = LHS
    (eq. solver-4 and eq. solver-6), i.e.
    rho = 4/3 r^n - 1/3 r^{n-1} - theta / (3 sqrt(E1)),
    LHS = (dt rho gamma / sqrt(E1) + eta) / (1 - dt gamma / (2 E1)),
    r^{n+1} = rho + LHS / (2 sqrt(E1)).
    The first-order start has rho = r^0 - theta / (2 sqrt(E1)) with r^0 = sqrt(E1)."""
    S = math.sqrt(E1)
    rho = (S - theta / (2.0 * S)) if bdf1 else (4.0 * r_n - r_nm1 - theta / S) / 3.0
    LHS = (dt * rho * gamma / S + eta) / (1.0 - dt * gamma / (2.0 * E1))
    return rho + LHS / (2.0 * S)


def bdf1_sav_step(model: Model, dt: float, phi0, forcing=None):
    """First-order SAV start (not printed in the paper):
    (phi^1 - phi^0)/dt = Delta_N (r^1/sqrt(E1) N_N(phi^0) + L_N phi^1),
    (r^1 - r^0)/dt = <N_N(phi^0), (phi^1 - phi^0)/dt> / (2 sqrt(E1)),
    with r^0 = sqrt(E_{1,N}(phi^0)), solved by the same elimination as Sec. 2.3.
    Returns (phi^1, r^1, r^0, info)."""
    g = model.g
    E1 = model.E1(phi0)
    sqE1 = math.sqrt(E1)
    r0 = sqE1
    Nh = model.N_op(phi0)
    lapN = g.lap(Nh)
    base = (phi0 if forcing is None else phi0 + dt * forcing) + stab_rhs(model, dt, phi0)
    coef = r0 - g.inner(Nh, phi0) / (2.0 * sqE1)
    gN = (dt / sqE1) * coef * lapN + base
    Ainv_g = A_inv(model, gN, dt, 1.0)
    Ainv_lapN = A_inv(model, lapN, dt, 1.0)
    gam = g.inner(Nh, Ainv_lapN)
    denom = 1.0 - dt / (2.0 * E1) * gam
    LHS = g.inner(Nh, Ainv_g) / denom
    phi1 = (dt / (2.0 * E1)) * LHS * Ainv_lapN + Ainv_g
    r1 = r0 + g.inner(Nh, phi1 - phi0) / (2.0 * sqE1)
    eta = g.inner(Nh, A_inv(model, phi0 + stab_rhs(model, dt, phi0), dt, 1.0))
    theta = g.inner(Nh, phi0)
    info = dict(E1=E1, sqrtE1=sqE1, gamma=gam, denom=denom, LHS=LHS, xi=r1 / sqE1, eta=eta, theta=theta)
    return phi1, r1, r0, info


def ghost_start(model: Model, dt: float, phi0):
    """phi^{-1} = phi^0 - dt Delta_N mu^0, r^0 = sqrt(E1(phi^0)), r^{-1} = sqrt(E1(phi^{-1}))
    (eq. scheme-SAV-initial-1 and the line after eq. scheme-SAV-initial-2)."""
    g = model.g
    phim1 = phi0 - dt * g.lap(model.mu(phi0))
    return phim1, math.sqrt(model.E1(phi0)), math.sqrt(model.E1(phim1))


def copy_start(model: Model, phi0):
    """phi^{-1} = phi^0 (the restart rule of Sec. 5.2), r^{-1} = r^0 = sqrt(E1(phi^0))."""
    r0 = math.sqrt(model.E1(phi0))
    return phi0.copy(), r0, r0


# ---------------------------------------------------------------------------
# Driver
# ---------------------------------------------------------------------------

class Oracle:
    """State (phi^n, phi^{n-1}, r^n, r^{n-1}) advanced by bdf2_sav_step."""

    def __init__(self, d, n, L, eps, beta, dt, nonlinear=True, dft="naive", stab=0.0, gamma3=0.0, pfc=False):
        self.grid = Grid(d, n, L, dft=dft)
        self.model = Model(self.grid, eps, beta if beta > 0 else 1.0, nonlinear=nonlinear)
        self.model.stab = float(stab)
        self.model.gamma3 = float(gamma3)
        if pfc:
            self.model.use_pfc(gamma3)
        self.dt = float(dt)
        self.phi = self.phi_prev = None
        self.r = self.r_prev = None
        self.nstep = 0
        self.last_info = None

    def start(self, phi0, mode: str = "bdf1", forcing=None):
        phi0 = np.array(phi0, dtype=np.float64).reshape(self.grid.shape)
        if mode == "bdf1":
            phi1, r1, r0, info = bdf1_sav_step(self.model, self.dt, phi0, forcing)
            self.phi, self.phi_prev, self.r, self.r_prev = phi1, phi0, r1, r0
            self.last_info = info
        elif mode == "ghost":
            phim1, r0, rm1 = ghost_start(self.model, self.dt, phi0)
            self.phi, self.phi_prev, self.r, self.r_prev = phi0, phim1, r0, rm1
        elif mode == "copy":
            phim1, r0, rm1 = copy_start(self.model, phi0)
            self.phi, self.phi_prev, self.r, self.r_prev = phi0, phim1, r0, rm1
        else:
            raise ValueError(mode)
        self.nstep = 0
        return self

    def set_state(self, phi, phi_prev, r, r_prev):
        self.phi = np.array(phi, dtype=np.float64).reshape(self.grid.shape)
        self.phi_prev = np.array(phi_prev, dtype=np.float64).reshape(self.grid.shape)
        self.r, self.r_prev = float(r), float(r_prev)
        return self

    def step(self, nsteps: int = 1, forcing=None):
        for _ in range(nsteps):
            f = forcing(self) if callable(forcing) else forcing
            phi_np1, r_np1, info = bdf2_sav_step(self.model, self.dt, self.phi, self.phi_prev,
                                                 self.r, self.r_prev, f)
            self.phi_prev, self.phi = self.phi, phi_np1
            self.r_prev, self.r = self.r, r_np1
            self.last_info = info
            self.nstep += 1
        return self

    def modified_energy(self) -> float:
        return self.model.E_mod(self.phi, self.phi_prev, self.r, self.r_prev)

    def original_energy(self) -> float:
        return self.model.E_orig(self.phi)

    def breve_energy(self) -> float:
        return self.model.E_breve(self.phi, self.r)

    def mass(self) -> float:
        return self.grid.mean_value(self.phi)
