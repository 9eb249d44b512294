"""FP64 CPU reference of the spectral-convolution surrogate network (a Fourier
neural operator, Li et al., "Fourier Neural Operator for Parametric Partial
Differential Equations", 2020) that advances the SPFC state K steps at once.

TEST INFRASTRUCTURE ONLY: the tests use it to check the GPU network's forward
pass and gradients. It shares no code with the CUDA path.

Network (all sizes are arguments; the production one has width 32, 16 x 32
retained modes, 4 layers, projection width 64):
  input per grid point   a = ((phi^n - m)/s, (phi^{n-1} - m)/s, eps, beta),
                         m = mean of phi^n, s = 0.1
  lift                   v = L a + lb                         (width channels)
  layer l = 0..nl-1      u = SpecConv_l(v) + W_l v + b_l, v = gelu(u) (no gelu on the last)
  SpecConv               v_hat = DFT of v restricted to kx in [0, m1), ky in
                         {0..m2-1} U {n-m2..n-1}; o_hat = R_l v_hat per mode
                         (complex width x width matrix); back to the grid by
                         the inverse real transform of the truncated spectrum,
                         (1/n^2) sum_kx w_kx Re(sum_ky o_hat e^{i(kx x + ky y) 2pi/n}),
                         w_0 = 1, w_kx = 2 otherwise
  projection             q = gelu(Q1 v + q1b), d = Q2 q + q2b   (one channel)
  output                 phi^{n+K} = phi^n + s (d - mean(d))    (mass kept exactly)
Loss: mean over samples and points of (d - mean(d) - (phi_target - phi^n)/s)^2.
gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SCALE = 0.1


class Config:
    def __init__(self, n=256, width=32, m1=16, m2=16, layers=4, proj=64):
        if 2 * m2 > n or m1 > n // 2:
            raise ValueError("too many modes for the grid")
        self.n, self.width, self.m1, self.m2, self.layers, self.proj = n, width, m1, m2, layers, proj
        self.ky = np.concatenate([np.arange(m2), np.arange(n - m2, n)])   # retained ky (2 m2 values)
        self.kx = np.arange(m1)

    def param_shapes(self):
        W, M = self.width, (2 * self.m2, self.m1)
        shapes = [("lift_w", (W, 4)), ("lift_b", (W,))]
        for l in range(self.layers):
            shapes += [(f"Rr{l}", (W, W) + M), (f"Ri{l}", (W, W) + M), (f"W{l}", (W, W)), (f"b{l}", (W,))]
        shapes += [("q1_w", (self.proj, W)), ("q1_b", (self.proj,)), ("q2_w", (1, self.proj)), ("q2_b", (1,))]
        return shapes

    def nparams(self):
        return int(sum(np.prod(s) for _, s in self.param_shapes()))


def unpack(cfg: Config, flat):
    out, o = {}, 0
    for name, shape in cfg.param_shapes():
        k = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(cfg: Config, d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in cfg.param_shapes()])


def init_params(cfg: Config, seed=0):
    """Uniform fan-in initialisation (spectral weights scaled by 1/width^2)."""
    rng = np.random.default_rng(seed)
    d = {}
    W = cfg.width
    for name, shape in cfg.param_shapes():
        if name.startswith("R"):
            d[name] = rng.uniform(0, 1, shape) / (W * W)
        elif name.endswith("_b") or (name.startswith("b") and name[1:].isdigit()):
            d[name] = np.zeros(shape)
        else:
            fan_in = shape[-1]
            lim = 1.0 / math.sqrt(fan_in)
            d[name] = rng.uniform(-lim, lim, shape)
    return pack(cfg, d)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _dft_mats(cfg: Config):
    n = cfg.n
    x = np.arange(n)
    Ex = np.exp(-2j * math.pi * np.outer(x, cfg.kx) / n)        # (n, m1): e^{-i kx x}
    Ey = np.exp(-2j * math.pi * np.outer(cfg.ky, x) / n)        # (2 m2, n): e^{-i ky y}
    wx = np.where(cfg.kx == 0, 1.0, 2.0)
    return Ex, Ey, wx


def spec_forward(cfg, v):
    """v (B, C, n, n) [y, x] -> truncated spectrum (B, C, 2 m2, m1)."""
    Ex, Ey, _ = _dft_mats(cfg)
    X = v @ Ex                                   # (B, C, n(y), m1)
    return np.einsum("ky,bcyx->bckx", Ey, X)      # (B, C, 2m2, m1)


def spec_inverse(cfg, oh):
    """truncated spectrum (B, C, 2 m2, m1) -> real grid (B, C, n, n)."""
    n = cfg.n
    Ex, Ey, wx = _dft_mats(cfg)
    Z = np.einsum("ky,bckx->bcyx", np.conj(Ey), oh)     # sum_ky oh e^{+i ky y}: (B, C, n, m1)
    out = np.real((Z * wx) @ np.conj(Ex).T)             # sum_kx w Re(Z e^{+i kx x})
    return out / (n * n)


def spec_inverse_adjoint(cfg, g):
    """Adjoint of spec_inverse w.r.t. the real pair (Re oh, Im oh), returned as a
    complex array whose real/imag parts are d/dRe, d/dIm."""
    n = cfg.n
    Ex, Ey, wx = _dft_mats(cfg)
    # out = Re( sum_ky sum_kx w oh e^{i th} ) / n^2, th = kx x + ky y (times 2 pi / n):
    # d out / d Re(oh) = w cos(th) / n^2, d out / d Im(oh) = -w sin(th) / n^2, so
    # dL/dRe + i dL/dIm = (w / n^2) sum g e^{-i th}
    G = (g / (n * n)) @ Ex                      # sum_x g e^{-i kx x}: (B,C,n,m1)
    H = np.einsum("ky,bcyx->bckx", Ey, G)        # sum_y e^{-i ky y}: (B,C,2m2,m1)
    return H * wx


def spec_forward_adjoint(cfg, gh):
    """Adjoint of spec_forward for a real input: given dL/dRe(vh) + i dL/dIm(vh)
    (complex gh), return dL/dv (real)."""
    Ex, Ey, _ = _dft_mats(cfg)
    # vh = sum_{x,y} v e^{-i th}: dL/dv[y,x] = sum_k [gr Re(e^{-i th}) + gi Im(e^{-i th})]
    #                                       = Re( sum_k conj(gh) e^{-i th} )
    Z = np.einsum("ky,bckx->bcyx", Ey, np.conj(gh))      # sum_ky conj(gh) e^{-i ky y}
    return np.real(Z @ Ex.T)                              # sum_kx (...) e^{-i kx x}


def forward(cfg: Config, flat, phi_n, phi_nm1, eps, beta, keep=False):
    """phi_n, phi_nm1: (B, n, n); eps, beta: (B,). Returns d (B, n, n) (before the
    mean removal) and, if keep, the intermediates for backward."""
    p = unpack(cfg, flat)
    B = phi_n.shape[0]
    m = phi_n.reshape(B, -1).mean(axis=1)[:, None, None]
    a = np.stack([(phi_n - m) / SCALE, (phi_nm1 - m) / SCALE,
                  np.broadcast_to(eps[:, None, None], phi_n.shape),
                  np.broadcast_to(beta[:, None, None], phi_n.shape)], axis=1)       # (B, 4, n, n)
    v = np.einsum("cj,bjyx->bcyx", p["lift_w"], a) + p["lift_b"][None, :, None, None]
    cache = {"a": a, "v": [v], "u": [], "vh": []}
    for l in range(cfg.layers):
        vh = spec_forward(cfg, v)
        R = p[f"Rr{l}"] + 1j * p[f"Ri{l}"]
        oh = np.einsum("iokx,bikx->bokx", R, vh)
        u = spec_inverse(cfg, oh) + np.einsum("oi,biyx->boyx", p[f"W{l}"], v) + p[f"b{l}"][None, :, None, None]
        v = gelu(u) if l < cfg.layers - 1 else u
        cache["vh"].append(vh)
        cache["u"].append(u)
        cache["v"].append(v)
    z = np.einsum("qc,bcyx->bqyx", p["q1_w"], v) + p["q1_b"][None, :, None, None]
    q = gelu(z)
    d = np.einsum("oq,bqyx->boyx", p["q2_w"], q)[:, 0] + p["q2_b"][0]
    cache.update(z=z, q=q)
    return (d, cache) if keep else d


def predict(cfg, flat, phi_n, phi_nm1, eps, beta):
    d = forward(cfg, flat, phi_n, phi_nm1, eps, beta)
    B = d.shape[0]
    return phi_n + SCALE * (d - d.reshape(B, -1).mean(axis=1)[:, None, None])


def loss_and_grad(cfg: Config, flat, phi_n, phi_nm1, eps, beta, phi_target):
    p = unpack(cfg, flat)
    d, c = forward(cfg, flat, phi_n, phi_nm1, eps, beta, keep=True)
    B, n = d.shape[0], cfg.n
    dc = d - d.reshape(B, -1).mean(axis=1)[:, None, None]
    t = (phi_target - phi_n) / SCALE
    res = dc - t
    cnt = B * n * n
    loss = float(np.sum(res * res) / cnt)
    gdc = 2.0 * res / cnt
    gd = gdc - gdc.reshape(B, -1).mean(axis=1)[:, None, None]      # through the mean removal
    g = {k: np.zeros_like(v) for k, v in p.items()}
    # projection
    g["q2_b"][0] = gd.sum()
    g["q2_w"][0] = np.einsum("byx,bqyx->q", gd, c["q"])
    gq = p["q2_w"][0][None, :, None, None] * gd[:, None]
    gz = gq * gelu_grad(c["z"])
    g["q1_b"] = gz.sum(axis=(0, 2, 3))
    v = c["v"][-1]
    g["q1_w"] = np.einsum("bqyx,bcyx->qc", gz, v)
    gv = np.einsum("qc,bqyx->bcyx", p["q1_w"], gz)
    for l in reversed(range(cfg.layers)):
        u = c["u"][l]
        gu = gv * gelu_grad(u) if l < cfg.layers - 1 else gv
        vin = c["v"][l]
        g[f"b{l}"] = gu.sum(axis=(0, 2, 3))
        g[f"W{l}"] = np.einsum("boyx,biyx->oi", gu, vin)
        gv_in = np.einsum("oi,boyx->biyx", p[f"W{l}"], gu)
        goh = spec_inverse_adjoint(cfg, gu)                        # dL/dRe(oh) + i dL/dIm(oh)
        vh = c["vh"][l]
        # oh = R vh: d/dRr = Re(goh conj(vh))... written out in real form
        gr, gi = goh.real, goh.imag
        vr, vi = vh.real, vh.imag
        g[f"Rr{l}"] = np.einsum("bokx,bikx->iokx", gr, vr) + np.einsum("bokx,bikx->iokx", gi, vi)
        g[f"Ri{l}"] = np.einsum("bokx,bikx->iokx", gi, vr) - np.einsum("bokx,bikx->iokx", gr, vi)
        Rr, Ri = p[f"Rr{l}"], p[f"Ri{l}"]
        gvr = np.einsum("iokx,bokx->bikx", Rr, gr) + np.einsum("iokx,bokx->bikx", Ri, gi)
        gvi = -np.einsum("iokx,bokx->bikx", Ri, gr) + np.einsum("iokx,bokx->bikx", Rr, gi)
        gv = gv_in + spec_forward_adjoint(cfg, gvr + 1j * gvi)
    a = c["a"]
    g["lift_b"] = gv.sum(axis=(0, 2, 3))
    g["lift_w"] = np.einsum("bcyx,bjyx->cj", gv, a)
    return loss, pack(cfg, g)
