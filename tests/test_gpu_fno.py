"""GPU surrogate network against the float64 CPU reference of the same network.

The GPU multiplies in BF16 (weights and activations rounded to bfloat16,
float32 accumulation); the reference runs in float64 on the bf16-rounded
weights, so what remains is the rounding of activations and DFT tables to
bfloat16. Tolerances: a few parts in a hundred on the predicted increment and
on the gradient (several BF16 roundings of about 2^-9 each compound over the
layers), exact float32 behaviour where no BF16 product is involved (mass,
Adam)."""
import numpy as np
import pytest

from oracle import fno_reference as F

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _bf16(x):
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _bf16_params(cfg, flat):
    """Round the parameters the GPU reads as bfloat16 (all but the layer and
    projection biases, which it adds in float32)."""
    d = F.unpack(cfg, flat)
    out = {}
    for name, v in d.items():
        keep32 = (name.startswith("b") and name[1:].isdigit()) or name in ("q1_b", "q2_b")
        out[name] = np.asarray(v, dtype=np.float32).astype(np.float64) if keep32 else _bf16(v)
    return F.pack(cfg, out)


def _case(cfg, B, seed):
    rng = np.random.default_rng(seed)
    n = cfg.n
    flat = F.init_params(cfg, seed=seed) * 2.0 + 0.02 * rng.standard_normal(cfg.nparams())
    flat = flat.astype(np.float32).astype(np.float64)
    phi_n = 0.2 + 0.3 * np.cos(2 * np.pi * (3 * np.arange(n)[None, :] + np.arange(n)[:, None]) / n)[None] \
        + 0.05 * rng.standard_normal((B, n, n))
    phi_nm1 = phi_n + 0.01 * rng.standard_normal((B, n, n))
    target = phi_n + 0.02 * rng.standard_normal((B, n, n))
    eps = rng.uniform(0.05, 0.35, B)
    beta = rng.uniform(0.5, 1.5, B)
    return flat, phi_n, phi_nm1, target, eps, beta


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda").contiguous()


def _net(cfg, B):
    from paper_2012_15133_gb300.surrogate import FNO
    return FNO(n=cfg.n, width=cfg.width, modes1=cfg.m1, modes2=cfg.m2, layers=cfg.layers, proj=cfg.proj, max_batch=B)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


CONFIGS = [
    (F.Config(n=32, width=8, m1=4, m2=4, layers=2, proj=16), 3),
    (F.Config(n=64, width=16, m1=8, m2=6, layers=3, proj=24), 2),
]


@pytest.mark.parametrize("cfg,B", CONFIGS, ids=["n32w8", "n64w16"])
def test_forward_matches_the_reference(cfg, B):
    flat, phi_n, phi_nm1, _, eps, beta = _case(cfg, B, 11)
    net = _net(cfg, B)
    net.set_params(flat)
    out = net.predict(_dev(phi_n), _dev(phi_nm1), eps, beta).double().cpu().numpy()
    phi32 = np.asarray(phi_n, dtype=np.float32).astype(np.float64)
    ref = F.predict(cfg, _bf16_params(cfg, flat), phi32, np.asarray(phi_nm1, np.float32).astype(np.float64), eps, beta)
    inc_err = _rel(out - phi32, ref - phi32)
    assert inc_err < 3e-2, inc_err
    # the mean of the increment is removed: mass is kept to float32 rounding
    for b in range(B):
        assert abs(out[b].mean() - phi32[b].mean()) < 1e-6


@pytest.mark.parametrize("cfg,B", CONFIGS, ids=["n32w8", "n64w16"])
def test_loss_and_gradient_match_the_reference(cfg, B):
    flat, phi_n, phi_nm1, target, eps, beta = _case(cfg, B, 12)
    net = _net(cfg, B)
    net.set_params(flat)
    loss, g = net.loss_grad(_dev(phi_n), _dev(phi_nm1), eps, beta, _dev(target), want_grad=True)
    f32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
    lref, gref = F.loss_and_grad(cfg, _bf16_params(cfg, flat), f32(phi_n), f32(phi_nm1), eps, beta, f32(target))
    assert abs(loss - lref) < 2e-2 * lref, (loss, lref)
    assert _rel(g, gref) < 5e-2, _rel(g, gref)
    # every parameter group separately (a transposed or misplaced block would
    # hide in the total)
    o = 0
    for name, shape in cfg.param_shapes():
        k = int(np.prod(shape))
        gg, rr = g[o:o + k], gref[o:o + k]
        o += k
        if np.linalg.norm(rr) > 1e-6 * np.linalg.norm(gref):
            assert _rel(gg, rr) < 1e-1, (name, _rel(gg, rr))


def test_production_network_at_256_matches_the_reference():
    cfg = F.Config(n=256, width=32, m1=16, m2=16, layers=4, proj=64)
    B = 2
    flat, phi_n, phi_nm1, target, eps, beta = _case(cfg, B, 13)
    net = _net(cfg, B)
    net.set_params(flat)
    f32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
    out = net.predict(_dev(phi_n), _dev(phi_nm1), eps, beta).double().cpu().numpy()
    pb = _bf16_params(cfg, flat)
    ref = F.predict(cfg, pb, f32(phi_n), f32(phi_nm1), eps, beta)
    assert _rel(out - f32(phi_n), ref - f32(phi_n)) < 3e-2
    loss, g = net.loss_grad(_dev(phi_n), _dev(phi_nm1), eps, beta, _dev(target), want_grad=True)
    lref, gref = F.loss_and_grad(cfg, pb, f32(phi_n), f32(phi_nm1), eps, beta, f32(target))
    assert abs(loss - lref) < 2e-2 * lref
    assert _rel(g, gref) < 5e-2


def test_adam_step_follows_its_definition():
    cfg, B = CONFIGS[0]
    flat, phi_n, phi_nm1, target, eps, beta = _case(cfg, B, 14)
    net = _net(cfg, B)
    net.set_params(flat)
    w = net.get_params().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    lr, b1, b2, e, wd = 1e-3, 0.9, 0.999, 1e-8, 1e-4
    for t in range(1, 4):
        _, g = net.loss_grad(_dev(phi_n), _dev(phi_nm1), eps, beta, _dev(target), want_grad=True)
        net.adam_step(lr, b1, b2, e, wd)
        gi = g.astype(np.float64) + wd * w
        m = b1 * m + (1 - b1) * gi
        v = b2 * v + (1 - b2) * gi * gi
        w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + e)
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - w)) < 1e-6 * max(1.0, np.max(np.abs(w)))
        w = got


def test_invalid_sizes_are_rejected():
    from paper_2012_15133_gb300.surrogate import FNO
    from paper_2012_15133_gb300 import SPFCError
    with pytest.raises(SPFCError):
        FNO(n=48)
    with pytest.raises(SPFCError):
        FNO(n=64, modes1=40)
    net = FNO(n=32, width=4, modes1=2, modes2=2, layers=1, proj=4, max_batch=2)
    x = torch.zeros((3, 32, 32), device="cuda")
    with pytest.raises(SPFCError):
        net.predict(x, x, [0.1] * 3, [1.0] * 3)


def _round_bf16(x):
    """float32 -> bfloat16 -> float32, round to nearest even (bit arithmetic)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


# (batch, M, N, K, splits, flags): ragged tiles in every dimension; the tile's
# rows on M or on N (N > M); 16-, 32- and 64-column tiles; K below one stage,
# not a multiple of 8, and many stages; split-K with empty splits; each device
# storage (A as bfloat16, A or B column-major: strided and contiguous gathers,
# aligned and unaligned).
GEMM_CASES = [
    (1, 200, 64, 70, 1, 0),
    (2, 33, 300, 45, 1, 0),
    (3, 128, 16, 256, 1, 1),
    (1, 64, 5, 513, 1, 2),
    (1, 1, 1000, 40, 1, 4),
    (1, 40, 24, 1000, 4, 0),
    (1, 17, 29, 100, 8, 3),
    (2, 130, 100, 32, 1, 6),
    (1, 8, 1, 7, 1, 7),
    (4, 300, 48, 96, 1, 5),
]


@pytest.mark.parametrize("bt,M,N,K,splits,flags", GEMM_CASES)
def test_tensor_core_gemm_matches_the_bf16_product(bt, M, N, K, splits, flags):
    """The tcgen05 product equals the float64 product of the bf16-rounded
    operands to float32 accumulation: |C - ref| <= 4 K 2^-24 (|A| |B|)."""
    from paper_2012_15133_gb300 import spfc
    rng = np.random.default_rng(1000 + M + 7 * N + 13 * K + flags)
    A = rng.standard_normal((bt, M, K)).astype(np.float32)
    B = rng.standard_normal((bt, K, N)).astype(np.float32)
    C = spfc.gemm_selftest(A, B, splits=splits, flags=flags)
    Ab = _round_bf16(A).astype(np.float64)
    Bb = _round_bf16(B).astype(np.float64)
    ref = Ab @ Bb
    bound = 4 * K * 2.0 ** -24 * (np.abs(Ab) @ np.abs(Bb)) + 1e-30
    err = np.abs(C.astype(np.float64) - ref)
    assert np.all(err <= bound), (float(np.max(err / bound)), np.unravel_index(np.argmax(err / bound), err.shape))


def test_tensor_core_gemm_is_deterministic():
    from paper_2012_15133_gb300 import spfc
    rng = np.random.default_rng(5)
    A = rng.standard_normal((2, 150, 300)).astype(np.float32)
    B = rng.standard_normal((2, 300, 40)).astype(np.float32)
    C1 = spfc.gemm_selftest(A, B, splits=3)
    C2 = spfc.gemm_selftest(A, B, splits=3)
    assert np.array_equal(C1, C2)


def test_tensor_core_gemm_wait_bound_latches_timeout_and_context_survives():
    """A wait that nothing completes (the self-test's flag 8) ends by its
    bound (about a second), the call reports SPFC_ETIMEOUT, and the next
    product on the same context is exact again."""
    import time
    from paper_2012_15133_gb300 import spfc, SPFCError
    rng = np.random.default_rng(9)
    A = rng.standard_normal((1, 100, 64)).astype(np.float32)
    B = rng.standard_normal((1, 64, 16)).astype(np.float32)
    t0 = time.perf_counter()
    with pytest.raises(SPFCError) as ei:
        spfc.gemm_selftest(A, B, flags=8)
    assert ei.value.code == 5  # SPFC_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    C = spfc.gemm_selftest(A, B)
    ref = _round_bf16(A).astype(np.float64) @ _round_bf16(B).astype(np.float64)
    bound = 4 * 64 * 2.0 ** -24 * (np.abs(_round_bf16(A)).astype(np.float64) @ np.abs(_round_bf16(B)).astype(np.float64))
    assert np.all(np.abs(C - ref) <= bound)
