"""Learned surrogate of K SAV steps, with the plain SAV step as its fallback
and judge.

The network (a Fourier neural operator, declared in include/spfc.h) runs in
this library's CUDA kernels (BF16 tensor-core GEMMs, FP32 accumulation):
forward, backward and Adam, and so does the jump-and-check loop
(spfc_surrogate_advance). This module marshals arguments and drives
training on trajectories of the batched solver. The loop:

* a jump maps (phi^{n-1}, phi^n, eps, beta) to a prediction of phi^{n+K};
* after an accepted jump the two-level scheme restarts with the copy
  convention phi^{n+K-1} := phi^{n+K}, r = sqrt(E_1) (the paper's restart
  after a time-step change, Sec. 5);
* the jump is rejected, and K plain SAV steps taken instead, if the modified
  energy (the paper's discrete energy) of the restarted prediction exceeds
  that of the live two-level state (phi^n, phi^{n-1}, r^n, r^{n-1}). With
  r = sqrt(E_1) the modified energy of a copy-restarted field is
  E_N(phi) + C_beta |Omega|, E_N with the run's phi^4 term;
* every ``check_every`` jumps, K plain steps from the same state judge the
  jump: rel-L2 above ``tol`` rejects it (and the plain result is kept).
"""
from __future__ import annotations

import ctypes as ct
import time

import numpy as np

from .spfc import SPFCError, Solver, Batch, load_library, _current_stream_ptr, field_energy_noalloc

_FP = ct.POINTER(ct.c_float)

# the network of the surrogate workload: 4 layers, width 32, 16 retained
# modes per axis (kx < 16, |ky| <= 16 in the half spectrum), projection 64
DEFAULT_NET = dict(width=32, modes1=16, modes2=16, layers=4, proj=64)


class FNO:
    """The surrogate network on the current CUDA device."""

    def __init__(self, n=256, width=32, modes1=16, modes2=16, layers=4, proj=64, max_batch=16):
        self._lib = load_library()
        self.n, self.width, self.modes1, self.modes2 = n, width, modes1, modes2
        self.layers, self.proj, self.max_batch = layers, proj, max_batch
        h = ct.c_void_p()
        rc = self._lib.spfc_fno_create(n, width, modes1, modes2, layers, proj, max_batch, _current_stream_ptr(),
                                       ct.byref(h))
        if rc != 0:
            raise SPFCError(rc, self._lib.spfc_fno_last_error(None).decode())
        self._h = h
        self.nparams = int(self._lib.spfc_fno_num_params(h))

    def _check(self, rc):
        if rc != 0:
            raise SPFCError(rc, self._lib.spfc_fno_last_error(self._h).decode())

    def set_params(self, flat):
        arr = np.ascontiguousarray(flat, dtype=np.float32)
        if arr.size != self.nparams:
            raise ValueError("wrong number of parameters")
        self._check(self._lib.spfc_fno_set_params(self._h, arr.ctypes.data_as(_FP)))

    def get_params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        self._check(self._lib.spfc_fno_get_params(self._h, out.ctypes.data_as(_FP)))
        return out

    @staticmethod
    def _dev(t):
        import torch
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("fields must be contiguous float32 CUDA tensors [batch, n, n]")
        return ct.c_void_p(t.data_ptr())

    @staticmethod
    def _params(eps, beta, B):
        e = (ct.c_double * B)(*[float(x) for x in eps])
        b = (ct.c_double * B)(*[float(x) for x in beta])
        return e, b

    def predict(self, phi_n, phi_nm1, eps, beta, out=None):
        """phi^{n+K} for a batch of float32 CUDA fields [B, n, n]."""
        import torch
        B = phi_n.shape[0]
        if out is None:
            out = torch.empty_like(phi_n)
        e, b = self._params(eps, beta, B)
        self._check(self._lib.spfc_fno_predict(self._h, B, self._dev(phi_n), self._dev(phi_nm1), e, b,
                                               self._dev(out)))
        return out

    def loss_grad(self, phi_n, phi_nm1, eps, beta, target, want_grad=False):
        """Mean-square loss of the scaled increment; the gradient stays on the
        device for adam_step (and is returned when want_grad)."""
        B = phi_n.shape[0]
        e, b = self._params(eps, beta, B)
        loss = ct.c_double()
        g = np.empty(self.nparams, dtype=np.float32) if want_grad else None
        self._check(self._lib.spfc_fno_loss_grad(self._h, B, self._dev(phi_n), self._dev(phi_nm1), e, b,
                                                 self._dev(target), ct.byref(loss),
                                                 g.ctypes.data_as(_FP) if want_grad else None))
        return (loss.value, g) if want_grad else loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self._check(self._lib.spfc_fno_adam_step(self._h, lr, beta1, beta2, eps, weight_decay))

    def save(self, path):
        """Write the weights (with the network's shape) to a file."""
        import os
        self._check(self._lib.spfc_fno_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Read weights written by save() into a network of the same shape."""
        import os
        self._check(self._lib.spfc_fno_load(self._h, os.fsencode(path)))
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.spfc_fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def init_params(fno: FNO, seed=0):
    """Uniform fan-in initialisation in the library's parameter order (lift,
    per layer Rr, Ri, W, b, then the projection); spectral weights are scaled
    by 1/width^2, biases start at zero."""
    rng = np.random.default_rng(seed)
    W, M = fno.width, 2 * fno.modes2 * fno.modes1
    parts = [rng.uniform(-0.5, 0.5, W * 4), np.zeros(W)]
    for _ in range(fno.layers):
        parts += [rng.uniform(0, 1, W * W * M) / (W * W), rng.uniform(0, 1, W * W * M) / (W * W),
                  rng.uniform(-1, 1, W * W) / np.sqrt(W), np.zeros(W)]
    parts += [rng.uniform(-1, 1, fno.proj * W) / np.sqrt(W), np.zeros(fno.proj),
              rng.uniform(-1, 1, fno.proj) / np.sqrt(fno.proj), np.zeros(1)]
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == fno.nparams
    return flat


def trajectory_pairs(runs, dt, K, snapshots, spacing, warm, precision="fp32"):
    """Training triples from trajectories of the batched solver.

    runs: dicts with n, L, eps, beta, phi0 (all of one grid size). After
    `warm` steps, `snapshots` times: record (phi^{t-1}, phi^t), step K, record
    phi^{t+K}, then step `spacing` - K more. Returns float32 CUDA tensors
    (phi_n, phi_nm1, target) of shape [runs * snapshots, n, n] and numpy eps,
    beta per sample."""
    import torch
    b = Batch(runs, dt, precision)
    for i, r in enumerate(runs):
        b.init(i, r["phi0"], "bdf1")
    if warm:
        b.step(warm)
    n = int(runs[0]["n"])
    total = len(runs) * snapshots
    X1, X0, Y = (torch.empty((total, n, n), dtype=torch.float32, device="cuda") for _ in range(3))
    dev = lambda a: torch.from_numpy(a.astype(np.float32))
    for s in range(snapshots):
        o = s * len(runs)
        for i in range(len(runs)):
            X1[o + i].copy_(dev(b.get_field(i, 0)))
            X0[o + i].copy_(dev(b.get_field(i, 1)))
        b.step(K)
        for i in range(len(runs)):
            Y[o + i].copy_(dev(b.get_field(i, 0)))
        if spacing > K and s + 1 < snapshots:
            b.step(spacing - K)
    b.close()
    eps = np.array([r["eps"] for r in runs] * snapshots)
    beta = np.array([r["beta"] for r in runs] * snapshots)
    # sample i * len(runs) + j is run j at snapshot i
    return {"phi_n": X1, "phi_nm1": X0, "target": Y, "eps": eps, "beta": beta}


def train(fno: FNO, data, iters, batch, lr=1e-3, seed=0, weight_decay=0.0):
    """Adam with a cosine learning-rate schedule on random mini-batches;
    returns the per-iteration losses."""
    import torch
    rng = np.random.default_rng(seed)
    nsamp = data["phi_n"].shape[0]
    losses = []
    for it in range(iters):
        idx = np.sort(rng.choice(nsamp, size=min(batch, nsamp), replace=False))
        ti = torch.as_tensor(idx, device="cuda")
        loss = fno.loss_grad(data["phi_n"][ti].contiguous(), data["phi_nm1"][ti].contiguous(), data["eps"][idx],
                             data["beta"][idx], data["target"][ti].contiguous())
        fno.adam_step(lr=lr * 0.5 * (1.0 + np.cos(np.pi * it / max(1, iters))), weight_decay=weight_decay)
        losses.append(loss)
    return losses


def identity_loss(data):
    """Loss of a network that predicts no change (d = 0): the scale against
    which a trained loss is read."""
    inc = (data["target"] - data["phi_n"]).double() / 0.1
    inc = inc - inc.mean(dim=(1, 2), keepdim=True)
    return float((inc * inc).mean())


class JumpLog:
    def __init__(self):
        self.jumps = self.accepted = self.rejected_energy = self.rejected_check = self.checks = 0
        self.check_errors = []
        self.decisions = []   # (jump, run, "accept" | "energy" | "check")

    def as_dict(self):
        return {"jumps": self.jumps, "accepted": self.accepted, "rejected_energy": self.rejected_energy,
                "rejected_check": self.rejected_check, "checks": self.checks,
                "fallback_rate": 1.0 - self.accepted / max(1, self.jumps),
                "max_check_rel_l2": max(self.check_errors) if self.check_errors else None}


def _twin(s):
    """A solver with the run's grid, parameters and precision (stabiliser and
    phi^4 term included), for the periodic plain-step check."""
    t = Solver(2, s.n[0], s.L[0], s.eps, s.beta, s.dt, "fp64" if s.precision == 0 else "fp32")
    if s.stab:
        t.set_stabilization(s.stab)
    if s.gamma3:
        t.set_gamma3(s.gamma3)
    return t


def judges_for(solvers):
    """One twin solver per run, for the periodic plain-step check of advance();
    creating them up front keeps their set-up out of a timed advance."""
    return {i: _twin(s) for i, s in enumerate(solvers)}


_KINDS = ("accept", "energy", "check")


def advance(solvers, fno: FNO, K, jumps, check_every=5, tol=1e-3, log=None, judges=None):
    """Advance 2D square runs (Solver objects of one grid size n <= 256) by
    jumps x K steps with the surrogate, falling back to K plain SAV steps per
    rejected jump (the loop runs in the library: spfc_surrogate_advance). One
    network call predicts all runs of a jump round.
    judges: twins from judges_for(solvers), kept by the caller (else made
    here, when checks are on, and closed on return)."""
    if log is None:
        log = JumpLog()
    R = len(solvers)
    n = solvers[0].n[0]
    if any(s.d != 2 or s.n != [n, n] or s.L[0] != s.L[1] for s in solvers):
        raise ValueError("the surrogate takes square 2D runs of one grid size")
    if R > fno.max_batch or n != fno.n:
        raise ValueError("runs do not fit the network (grid size or batch)")
    own = judges is None and check_every > 0
    judge = judges_for(solvers) if own else judges
    runs = (ct.c_void_p * R)(*[s._h.value for s in solvers])
    twins = (ct.c_void_p * R)(*[judge[i]._h.value for i in range(R)]) if check_every > 0 else None
    counts = (ct.c_int64 * 5)()
    dec = (ct.c_int8 * max(1, jumps * R))()
    errs = (ct.c_double * max(1, jumps * R))()
    try:
        rc = fno._lib.spfc_surrogate_advance(fno._h, runs, twins, R, int(K), int(jumps), int(check_every),
                                             float(tol), counts, dec, errs)
    finally:
        if own:
            for t in judge.values():
                t.close()
    if rc != 0:
        raise SPFCError(rc, fno._lib.spfc_surrogate_last_error().decode())
    log.jumps += counts[0]
    log.accepted += counts[1]
    log.rejected_energy += counts[2]
    log.rejected_check += counts[3]
    log.checks += counts[4]
    for j in range(jumps):
        for i in range(R):
            log.decisions.append((j, i, _KINDS[dec[j * R + i]]))
            e = errs[j * R + i]
            if e == e:  # checked (NaN otherwise)
                log.check_errors.append(e)
    return log


def timed(fn, *args, **kw):
    """(result, seconds) of fn with the device synchronised on both sides."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn(*args, **kw)
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0
