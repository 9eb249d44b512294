"""ctypes binding of ``libspfc.so`` (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python
arguments (numpy arrays for host data, torch CUDA tensors for device data,
torch streams) into the plain pointers and sizes of ``include/spfc.h``.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from .build import LIB

FP64, FP32_BULK = 0, 1
START_BDF1, START_GHOST, START_COPY = 0, 1, 2
_PREC = {"fp64": FP64, "f64": FP64, FP64: FP64, "fp32": FP32_BULK, "f32": FP32_BULK,
         "fp32_bulk": FP32_BULK, FP32_BULK: FP32_BULK}
_START = {"bdf1": START_BDF1, "ghost": START_GHOST, "copy": START_COPY,
          START_BDF1: START_BDF1, START_GHOST: START_GHOST, START_COPY: START_COPY}

_P = ct.c_void_p
_D = ct.c_double
_I = ct.c_int
_DP = ct.POINTER(ct.c_double)
_F = ct.c_float
_FP = ct.POINTER(ct.c_float)

# name -> (restype, argtypes), one entry per function of include/spfc.h
_SIGS = {
    "spfc_create": (_I, [_I, ct.POINTER(_I), _DP, _D, _D, _D, _I, _P, ct.POINTER(_P)]),
    "spfc_num_schedules": (_I, [_I, _I]),
    "spfc_create_scheduled": (_I, [_I, ct.POINTER(_I), _DP, _D, _D, _D, _I, _P, _I, ct.POINTER(_P)]),
    "spfc_schedule": (_I, [_P]),
    "spfc_init": (_I, [_P, _P, _I, _I]),
    "spfc_init_random": (_I, [_P, _D, _D, ct.c_uint64, _I]),
    "spfc_set_state": (_I, [_P, _P, _P, _D, _D, _I]),
    "spfc_step": (_I, [_P, ct.c_int64]),
    "spfc_energy": (_I, [_P, _DP, _DP, _DP]),
    "spfc_mass": (_I, [_P, _DP, _DP]),
    "spfc_sav_scalars": (_I, [_P, _DP, _I]),
    "spfc_get_field": (_I, [_P, _P, _I, _I]),
    "spfc_dt_change": (_I, [_P, _D]),
    "spfc_set_stabilization": (_I, [_P, _D]),
    "spfc_set_gamma3": (_I, [_P, _D]),
    "spfc_set_pfc": (_I, [_P, _D]),
    "spfc_save": (_I, [_P, ct.c_char_p]),
    "spfc_load": (_I, [_P, ct.c_char_p]),
    "spfc_set_scalar_ring": (_I, [_P, _P, ct.c_int64]),
    "spfc_sync": (_I, [_P]),
    "spfc_set_timing": (_I, [_P, _I]),
    "spfc_kernel_times": (_I, [_P, _I, ct.POINTER(ct.c_char_p), ct.POINTER(ct.c_int64), _DP]),
    "spfc_device_bytes": (ct.c_int64, [_P]),
    "spfc_wait_selftest": (_I, [ct.c_ulonglong, ct.c_longlong, _P]),
    "spfc_fp64_fma_rate": (_I, [_DP, _P]),
    "spfc_destroy": (None, [_P]),
    "spfc_last_error": (ct.c_char_p, [_P]),
    "spfc_batch_create": (_I, [_I, ct.POINTER(_I), _DP, _DP, _DP, _D, _I, _P, ct.POINTER(_P)]),
    "spfc_batch_create_scheduled": (_I, [_I, ct.POINTER(_I), _DP, _DP, _DP, _D, _I, _P, ct.POINTER(_I),
                                         ct.POINTER(_P)]),
    "spfc_batch_schedule_valid": (_I, [_I, _I]),
    "spfc_batch_schedule": (_I, [_P, _I]),
    "spfc_batch_init": (_I, [_P, _I, _P, _I]),
    "spfc_batch_set_state": (_I, [_P, _I, _P, _P, _D, _D]),
    "spfc_batch_set_gamma3": (_I, [_P, _I, _D]),
    "spfc_batch_step": (_I, [_P, ct.c_int64]),
    "spfc_batch_sync": (_I, [_P]),
    "spfc_batch_get_field": (_I, [_P, _I, _P, _I]),
    "spfc_batch_scalars": (_I, [_P, _I, _DP, _I]),
    "spfc_batch_energy": (_I, [_P, _I, _DP]),
    "spfc_batch_points": (ct.c_int64, [_P]),
    "spfc_batch_destroy": (None, [_P]),
    "spfc_batch_last_error": (ct.c_char_p, [_P]),
    "spfc_field_energy_noalloc": (_I, [_I, _DP, _D, _D, _P, _DP, _P]),
    "spfc_noalloc_last_error": (ct.c_char_p, []),
    "spfc_fno_create": (_I, [_I, _I, _I, _I, _I, _I, _I, _P, ct.POINTER(_P)]),
    "spfc_fno_num_params": (ct.c_int64, [_P]),
    "spfc_fno_set_params": (_I, [_P, _FP]),
    "spfc_fno_get_params": (_I, [_P, _FP]),
    "spfc_fno_predict": (_I, [_P, _I, _P, _P, _DP, _DP, _P]),
    "spfc_fno_loss_grad": (_I, [_P, _I, _P, _P, _DP, _DP, _P, _DP, _FP]),
    "spfc_fno_adam_step": (_I, [_P, _F, _F, _F, _F, _F]),
    "spfc_fno_destroy": (None, [_P]),
    "spfc_fno_last_error": (ct.c_char_p, [_P]),
    "spfc_gemm_selftest": (_I, [_I, _I, _I, _I, _I, _I, _P, _P, _P, _P]),
    "spfc_fno_save": (_I, [_P, ct.c_char_p]),
    "spfc_fno_load": (_I, [_P, ct.c_char_p]),
    "spfc_surrogate_advance": (_I, [_P, ct.POINTER(_P), ct.POINTER(_P), _I, _I, _I, _I, _D,
                                    ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int8), _DP]),
    "spfc_surrogate_last_error": (ct.c_char_p, []),
}
EXPORTED_SYMBOLS = tuple(_SIGS)

_lib = None


def lib_path() -> str:
    return LIB


def load_library(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2012_15133_gb300.build.build(); "
                           "the solver has no CPU fallback")
    lib = ct.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class SPFCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"spfc error {code}: {msg}")
        self.code = code


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _current_stream_ptr():
    import torch
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def field_energy_noalloc(phi, L, eps, beta, stream=None):
    """Energy diagnostics of one 2D float64 CUDA field through the allocation-free
    entry point (see include/spfc.h): returns (E_N, 1/2 ||L^{1/2} phi||^2, mass)."""
    import torch
    lib = load_library()
    if not (phi.is_cuda and phi.dtype == torch.float64 and phi.is_contiguous() and phi.dim() == 2
            and phi.shape[0] == phi.shape[1]):
        raise ValueError("phi must be a square, contiguous float64 CUDA tensor")
    if phi.device.index != torch.cuda.current_device():
        raise ValueError("phi must live on the current CUDA device (the entry point runs there)")
    Ls = [float(L)] * 2 if np.isscalar(L) else [float(v) for v in L]
    out = (ct.c_double * 3)()
    sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream)
    rc = lib.spfc_field_energy_noalloc(int(phi.shape[0]), (ct.c_double * 2)(*Ls), float(eps), float(beta),
                                       ct.c_void_p(phi.data_ptr()), out, sp)
    if rc != 0:
        raise SPFCError(rc, lib.spfc_noalloc_last_error().decode())
    return out[0], out[1], out[2]


def fp64_fma_rate(stream=None):
    """Measured float64 FMA throughput of the current GPU in GFLOP/s (the
    arithmetic roofline of the float64 step)."""
    lib = load_library()
    out = ct.c_double()
    sp = _current_stream_ptr() if stream is None else ct.c_void_p(
        stream if isinstance(stream, int) else stream.cuda_stream)
    rc = lib.spfc_fp64_fma_rate(ct.byref(out), sp)
    if rc != 0:
        raise SPFCError(rc, "FP64 FMA rate measurement failed")
    return out.value


def gemm_selftest(A, B, splits=1, flags=0, stream=None):
    """C = A @ B through the surrogate network's tensor-core product (operands
    rounded to bfloat16, float32 accumulation). A: (batch, M, K), B: (batch,
    K, N) float32 host arrays; flags select the device storage of A and B
    (see include/spfc.h). Returns C as a (batch, M, N) float32 array."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    if A.ndim != 3 or B.ndim != 3 or A.shape[0] != B.shape[0] or A.shape[2] != B.shape[1]:
        raise ValueError("A must be (batch, M, K) and B (batch, K, N)")
    bt, M, K = A.shape
    N = B.shape[2]
    C = np.empty((bt, M, N), dtype=np.float32)
    lib = load_library()
    sp = _current_stream_ptr() if stream is None else ct.c_void_p(
        stream if isinstance(stream, int) else stream.cuda_stream)
    rc = lib.spfc_gemm_selftest(M, N, K, bt, int(splits), int(flags), A.ctypes.data_as(_P),
                                B.ctypes.data_as(_P), C.ctypes.data_as(_P), sp)
    if rc != 0:
        raise SPFCError(rc, "tensor-core GEMM self-test failed")
    return C


def num_schedules(d, n):
    return int(load_library().spfc_num_schedules(int(d), int(n)))


class Solver:
    """One SPFC run on the current CUDA device (see include/spfc.h).

    Host arrays are numpy float64 arrays of shape (N,)*d (x fastest = last
    axis); device arrays are contiguous float64 torch CUDA tensors.
    """

    def __init__(self, d, n, L, eps, beta, dt, precision="fp64", stream=None, schedule=None):
        self._lib = load_library()
        self.d = int(d)
        n = [int(n)] * self.d if np.isscalar(n) else [int(v) for v in n]
        L = [float(L)] * self.d if np.isscalar(L) else [float(v) for v in L]
        self.n, self.L = n, L
        self.eps, self.beta, self.dt = float(eps), float(beta), float(dt)
        self.stab = self.gamma3 = 0.0
        self.shape = tuple(reversed(n))
        self.precision = _PREC[precision]
        if stream is None:
            sp = _current_stream_ptr()
        elif isinstance(stream, int):
            sp = ct.c_void_p(stream)
        else:
            sp = ct.c_void_p(stream.cuda_stream)
        self._stream = sp
        h = ct.c_void_p()
        if schedule == "auto":
            from .autotune import lookup
            schedule = lookup(self.d, n[0], self.precision)
        rc = self._lib.spfc_create_scheduled(self.d, (ct.c_int * self.d)(*n), (ct.c_double * self.d)(*L),
                                             float(eps), float(beta), float(dt), self.precision, sp,
                                             -1 if schedule is None else int(schedule), ct.byref(h))
        if rc != 0:
            raise SPFCError(rc, self._lib.spfc_last_error(None).decode())
        self._h = h

    # -- helpers ---------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise SPFCError(rc, self._lib.spfc_last_error(self._h).decode())

    def _field_arg(self, a):
        """Return (pointer, on_device, keepalive) for an input field."""
        if _is_torch(a):
            import torch
            if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
                raise ValueError("device fields must be contiguous float64 CUDA tensors")
            if tuple(a.shape) != self.shape and a.numel() != int(np.prod(self.shape)):
                raise ValueError("field has the wrong size")
            return ct.c_void_p(a.data_ptr()), 1, a
        arr = np.ascontiguousarray(a, dtype=np.float64)
        if arr.size != int(np.prod(self.shape)):
            raise ValueError("field has the wrong size")
        return arr.ctypes.data_as(ct.c_void_p), 0, arr

    # -- API -------------------------------------------------------------------
    def init(self, phi0, mode="bdf1"):
        ptr, dev, keep = self._field_arg(phi0)
        self._check(self._lib.spfc_init(self._h, ptr, dev, _START[mode]))
        return self

    def init_random(self, mean, amp, seed, mode="bdf1"):
        """Start from mean + amp U(-1, 1), the noise drawn on the device from
        SplitMix64 (the same stream as seeded_inputs.noisy_field)."""
        self._check(self._lib.spfc_init_random(self._h, float(mean), float(amp), int(seed), _START[mode]))
        return self

    def set_state(self, phi, phi_prev, r, r_prev):
        p1, d1, k1 = self._field_arg(phi)
        p2, d2, k2 = self._field_arg(phi_prev)
        if d1 != d2:
            raise ValueError("both fields must be on the host or both on the device")
        self._check(self._lib.spfc_set_state(self._h, p1, p2, float(r), float(r_prev), d1))
        return self

    def step(self, nsteps=1):
        self._check(self._lib.spfc_step(self._h, int(nsteps)))
        return self

    def energy(self):
        """(E_orig, E_mod, E_breve)"""
        a, b, c = ct.c_double(), ct.c_double(), ct.c_double()
        self._check(self._lib.spfc_energy(self._h, ct.byref(a), ct.byref(b), ct.byref(c)))
        return a.value, b.value, c.value

    def mass(self):
        """(mass, mean)"""
        a, b = ct.c_double(), ct.c_double()
        self._check(self._lib.spfc_mass(self._h, ct.byref(a), ct.byref(b)))
        return a.value, b.value

    def set_scalar_ring(self, ring):
        """Per-step records written by the device into page-locked host memory:
        ring is a pinned torch float64 tensor of shape (capacity, 8) (None
        removes it). Record steps % capacity of every committed step holds
        (steps, r^{n+1}, r^n, xi, gamma, E_1, alpha, status); complete after
        the stream is synchronised."""
        if ring is None:
            self._check(self._lib.spfc_set_scalar_ring(self._h, None, 0))
            self._ring = None
            return self
        if ring.dtype.itemsize != 8 or ring.dim() != 2 or ring.shape[1] != 8 or not ring.is_contiguous():
            raise ValueError("the ring is a contiguous float64 tensor of shape (capacity, 8)")
        if not ring.is_pinned():
            raise ValueError("the ring must be page-locked (pin_memory())")
        self._check(self._lib.spfc_set_scalar_ring(self._h, ct.c_void_p(ring.data_ptr()), int(ring.shape[0])))
        self._ring = ring  # kept alive with the handle
        return self

    def sav_scalars(self, full=False):
        """r^n, r^{n-1}, xi, gamma, E_1, steps; with full=True also eta, theta,
        the denominator 1 - dt gamma/(2 E_1) and LHS of the last solve."""
        k = 10 if full else 6
        out = (ct.c_double * k)()
        self._check(self._lib.spfc_sav_scalars(self._h, out, k))
        keys = ("r", "r_prev", "xi", "gamma", "E1", "nsteps", "eta", "theta", "denom", "LHS")
        return dict(zip(keys, list(out)))

    def get_field(self, which=0, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        ptr, dev, keep = self._field_arg(out)
        self._check(self._lib.spfc_get_field(self._h, ptr, dev, int(which)))
        return out

    def dt_change(self, dt):
        self._check(self._lib.spfc_dt_change(self._h, float(dt)))
        self.dt = float(dt)
        return self

    def set_stabilization(self, A):
        """The stabilised scheme of Sec. 5.2 with constant A >= 0 (0: plain)."""
        self._check(self._lib.spfc_set_stabilization(self._h, float(A)))
        self.stab = float(A)
        return self

    def set_pfc(self, gamma3=1.0):
        """Switch to the PFC model of Sec. 1 with phi^4 coefficient gamma3 > 0
        (its own split: L = a + (1 + Delta)^2, E_1 = gamma3/4 ||phi||_4^4 -
        1/2 ||phi||^2 + C |Omega|); gamma3 = 0 switches back to SPFC."""
        self._check(self._lib.spfc_set_pfc(self._h, float(gamma3)))
        return self

    def set_gamma3(self, gamma3):
        """The optional phi^4 term: E_1 gains gamma3/4 ||phi||_4^4 and N gains
        gamma3 phi^3 with its mean removed (0: SPFC)."""
        self._check(self._lib.spfc_set_gamma3(self._h, float(gamma3)))
        self.gamma3 = float(gamma3)
        return self

    def save(self, path):
        self._check(self._lib.spfc_save(self._h, os.fsencode(path)))

    def load(self, path):
        self._check(self._lib.spfc_load(self._h, os.fsencode(path)))
        return self

    def sync(self):
        self._check(self._lib.spfc_sync(self._h))

    def set_timing(self, on=True):
        self._check(self._lib.spfc_set_timing(self._h, 1 if on else 0))

    def kernel_times(self):
        names = (ct.c_char_p * 16)()
        launches = (ct.c_int64 * 16)()
        ms = (ct.c_double * 16)()
        n = self._lib.spfc_kernel_times(self._h, 16, names, launches, ms)
        if n < 0:
            self._check(n)
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(n)}

    @property
    def schedule(self):
        return int(self._lib.spfc_schedule(self._h))

    def device_bytes(self):
        return int(self._lib.spfc_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.spfc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched ensemble of independent 2D runs (see include/spfc.h).

    runs: sequence of dicts with keys n, L, eps, beta (square boxes).
    schedule: None (each grid size's default), "auto" (the autotuner's table
    for this GPU, the default where it has no entry), an int for every class
    of N >= 128, or a dict {n: schedule}."""

    def __init__(self, runs, dt, precision="fp32", stream=None, schedule=None):
        self._lib = load_library()
        self.runs = [dict(r) for r in runs]
        k = len(self.runs)
        ns = (ct.c_int * k)(*[int(r["n"]) for r in self.runs])
        Ls = (ct.c_double * k)(*[float(r["L"]) for r in self.runs])
        es = (ct.c_double * k)(*[float(r["eps"]) for r in self.runs])
        bs = (ct.c_double * k)(*[float(r["beta"]) for r in self.runs])
        sp = _current_stream_ptr() if stream is None else ct.c_void_p(
            stream if isinstance(stream, int) else stream.cuda_stream)
        scheds = None
        if schedule is not None:
            def pick(n):
                if schedule == "auto":
                    from .autotune import lookup_batch
                    return lookup_batch(n, precision)
                if isinstance(schedule, dict):
                    return int(schedule.get(n, -1))
                return int(schedule) if n >= 128 else -1
            scheds = (ct.c_int * k)(*[pick(int(r["n"])) for r in self.runs])
        h = ct.c_void_p()
        rc = self._lib.spfc_batch_create_scheduled(k, ns, Ls, es, bs, float(dt), _PREC[precision], sp, scheds,
                                                   ct.byref(h))
        if rc != 0:
            raise SPFCError(rc, self._lib.spfc_batch_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != 0:
            raise SPFCError(rc, self._lib.spfc_batch_last_error(self._h).decode())

    def init(self, run, phi0, mode="bdf1"):
        arr = np.ascontiguousarray(phi0, dtype=np.float64)
        n = int(self.runs[run]["n"])
        if arr.size != n * n:
            raise ValueError("field has the wrong size")
        self._check(self._lib.spfc_batch_init(self._h, int(run), arr.ctypes.data_as(ct.c_void_p), _START[mode]))
        return self

    def set_state(self, run, phi, phi_prev, r, r_prev):
        """Both time levels (host arrays) and r^n, r^{n-1} of one run."""
        n = int(self.runs[run]["n"])
        a = np.ascontiguousarray(phi, dtype=np.float64)
        b = np.ascontiguousarray(phi_prev, dtype=np.float64)
        if a.size != n * n or b.size != n * n:
            raise ValueError("field has the wrong size")
        self._check(self._lib.spfc_batch_set_state(self._h, int(run), a.ctypes.data_as(ct.c_void_p),
                                                   b.ctypes.data_as(ct.c_void_p), float(r), float(r_prev)))
        return self

    def step(self, nsteps=1):
        self._check(self._lib.spfc_batch_step(self._h, int(nsteps)))
        return self

    def sync(self):
        self._check(self._lib.spfc_batch_sync(self._h))

    def get_field(self, run, which=0):
        n = int(self.runs[run]["n"])
        out = np.empty((n, n), dtype=np.float64)
        self._check(self._lib.spfc_batch_get_field(self._h, int(run), out.ctypes.data_as(ct.c_void_p), int(which)))
        return out

    def scalars(self, run):
        out = (ct.c_double * 8)()
        rc = self._lib.spfc_batch_scalars(self._h, int(run), out, 8)
        keys = ("r", "r_prev", "xi", "gamma", "E1", "nsteps", "mean", "status")
        d = dict(zip(keys, list(out)))
        if rc != 0 and d["status"] == 0:
            self._check(rc)
        return d

    def energy(self, run):
        out = (ct.c_double * 3)()
        self._check(self._lib.spfc_batch_energy(self._h, int(run), out))
        return out[0], out[1], out[2]

    def set_gamma3(self, run, gamma3):
        """The optional phi^4 term of one run (see Solver.set_gamma3)."""
        self._check(self._lib.spfc_batch_set_gamma3(self._h, int(run), float(gamma3)))
        return self

    @property
    def points(self):
        return int(self._lib.spfc_batch_points(self._h))

    def schedule(self, n):
        """The tile schedule of the class of grid size n (-1: none)."""
        return int(self._lib.spfc_batch_schedule(self._h, int(n)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.spfc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
