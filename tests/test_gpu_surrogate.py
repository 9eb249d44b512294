"""The learned surrogate trained on the solver's own trajectories, and its
fallback to the plain SAV step.

A network of the production shape (4 layers, width 32, 16 x 32 retained
modes, projection 64) is trained on a 64^2 ensemble (L = 32; the square
lattice's wave number then sits at mode index about 5, inside the retained
band) with the library's backward and Adam kernels. The tests check that:
training lowers the loss far below that of predicting no change, also on
held-out seeds; an accepted jump never raises E_N and restarts the two-level
scheme from the prediction; a rejected jump is exactly K plain steps; and
the trained network predicts K steps much closer to the plain scheme than
the untrained one. The throughput with and without the network is printed.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, K = 64, 20


def _runs(count, held_out=False):
    from seeded_inputs import surrogate_run
    return [surrogate_run(i, n=N, held_out=held_out) for i in range(count)]


@pytest.fixture(scope="module")
def trained():
    from paper_2012_15133_gb300 import surrogate as S
    data = S.trajectory_pairs(_runs(32), 0.02, K, 8, 100, 50)
    net = S.FNO(n=N, width=32, modes1=16, modes2=16, layers=4, proj=64, max_batch=16)
    init = S.init_params(net, 0)
    net.set_params(init)
    losses = S.train(net, data, 400, 16, lr=2e-3)
    return net, data, losses, init


def _solvers(count, warm=50):
    from paper_2012_15133_gb300 import Solver
    out = []
    for r in _runs(count, held_out=True):
        s = Solver(2, N, r["L"], r["eps"], r["beta"], r["dt"], "fp32")
        s.init(r["phi0"], "bdf1")
        s.step(warm)
        out.append(s)
    return out


def test_training_lowers_the_loss_on_training_and_held_out_trajectories(trained):
    from paper_2012_15133_gb300 import surrogate as S
    net, data, losses, _ = trained
    assert all(np.isfinite(losses))
    idl = S.identity_loss(data)
    assert np.mean(losses[-20:]) < 0.1 * idl, (np.mean(losses[-20:]), idl)
    # held-out seeds, sampled at the same times as the training pairs
    held = S.trajectory_pairs(_runs(4, held_out=True), 0.02, K, 8, 100, 50)
    hl = np.mean([net.loss_grad(held["phi_n"][i:i + 16].contiguous(), held["phi_nm1"][i:i + 16].contiguous(),
                                held["eps"][i:i + 16], held["beta"][i:i + 16], held["target"][i:i + 16].contiguous())
                  for i in (0, 16)])
    assert hl < 0.2 * S.identity_loss(held), (hl, S.identity_loss(held))


def _restarted_energy(pred, s, gamma3=0.0):
    """The modified energy of a field after the copy restart, r = sqrt(E_1):
    E_N(field) + C_beta |Omega|, E_N with the phi^4 term."""
    from paper_2012_15133_gb300 import field_energy_noalloc
    h2 = (s.L[0] / s.n[0]) * (s.L[1] / s.n[1])
    e = field_energy_noalloc(pred, s.L[0], s.eps, s.beta)[0]
    return e + 0.25 * gamma3 * h2 * float(torch.sum(pred ** 4)) + (1.0 + 1.0 / s.beta) * s.L[0] * s.L[1]


def test_accepted_jumps_keep_energy_and_restart_from_the_prediction(trained):
    from paper_2012_15133_gb300 import surrogate as S
    net = trained[0]
    sol = _solvers(4)
    accepted = 0
    for j in range(4):
        before = [s.get_field(0) for s in sol]
        e_before = [s.energy()[1] for s in sol]  # the modified energy of the live state
        cur = torch.tensor(np.stack(before), dtype=torch.float32, device="cuda")
        prev = torch.tensor(np.stack([s.get_field(1) for s in sol]), dtype=torch.float32, device="cuda")
        pred = net.predict(cur, prev, [s.eps for s in sol], [s.beta for s in sol]).double().cpu().numpy()
        log = S.advance(sol, net, K, 1, check_every=0)
        for (_, i, what) in log.decisions:
            s = sol[i]
            after = s.get_field(0)
            if what == "accept":
                accepted += 1
                # the copy restart: both levels hold the prediction
                assert np.max(np.abs(after - pred[i])) < 1e-6 * np.max(np.abs(pred[i]))
                assert np.array_equal(s.get_field(1), after)
                e_after = s.energy()[1]  # the modified energy of the copy-restarted state
                assert e_after <= e_before[i] * (1 + 1e-12)
                assert abs(e_after - _restarted_energy(torch.tensor(after, device="cuda"), s)) < 1e-9 * e_after
            else:
                assert what == "energy"
    assert accepted > 0


def test_rejected_jumps_are_exactly_the_plain_steps():
    from paper_2012_15133_gb300 import surrogate as S
    # a network with inflated weights predicts rough fields whose energy rises
    net = S.FNO(n=N, width=8, modes1=4, modes2=4, layers=1, proj=8, max_batch=4)
    net.set_params(S.init_params(net, 3) * 40.0)
    a, b = _solvers(3), _solvers(3)
    log = S.advance(a, net, K, 3, check_every=0)
    assert log.rejected_energy == log.jumps == 9
    for s in b:
        s.step(3 * K)
    for sa, sb in zip(a, b):
        assert np.array_equal(sa.get_field(0), sb.get_field(0))
        assert sa.sav_scalars()["r"] == sb.sav_scalars()["r"]


def _reference_advance(solvers, net, K, jumps, check_every, tol):
    """The jump loop composed in Python from the binding's single calls: the
    decisions the library's native loop must reproduce."""
    from paper_2012_15133_gb300 import Solver
    R, n = len(solvers), solvers[0].n[0]
    cur = torch.empty((R, n, n), dtype=torch.float64, device="cuda")
    prev = torch.empty_like(cur)
    twins = [Solver(2, n, s.L[0], s.eps, s.beta, s.dt, "fp32") for s in solvers]
    decisions, errs = [], []
    for j in range(jumps):
        for i, s in enumerate(solvers):
            s.get_field(0, out=cur[i])
            s.get_field(1, out=prev[i])
        pred = net.predict(cur.float(), prev.float(), [s.eps for s in solvers], [s.beta for s in solvers]).double()
        check = check_every > 0 and j % check_every == 0
        for i, s in enumerate(solvers):
            e_now = s.energy()[1]
            e_new = _restarted_energy(pred[i], s, getattr(s, "gamma3", 0.0))
            if e_new > e_now:
                decisions.append((j, i, "energy"))
                s.step(K)
                continue
            if check:
                sc, t = s.sav_scalars(), twins[i]
                t.set_state(cur[i], prev[i], sc["r"], sc["r_prev"])
                t.step(K)
                plain = t.get_field(0, out=torch.empty_like(cur[i]))
                err = float(torch.linalg.vector_norm(pred[i] - plain) / torch.linalg.vector_norm(plain))
                errs.append(err)
                if err > tol:
                    decisions.append((j, i, "check"))
                    ts = t.sav_scalars()
                    s.set_state(plain, t.get_field(1, out=torch.empty_like(cur[i])), ts["r"], ts["r_prev"])
                    continue
            decisions.append((j, i, "accept"))
            s.init(pred[i].contiguous(), "copy")
    for t in twins:
        t.close()
    return decisions, errs


@pytest.mark.parametrize("check_every,tol", [(0, 1e-3), (1, 1e-3), (2, 10.0)])
def test_the_native_loop_makes_the_decisions_of_its_composition(trained, check_every, tol):
    """spfc_surrogate_advance against the same loop composed from single calls:
    the same decisions and check errors, and bit-identical runs afterwards."""
    from paper_2012_15133_gb300 import surrogate as S
    net = trained[0]
    a, b = _solvers(4), _solvers(4)
    log = S.advance(a, net, K, 4, check_every=check_every, tol=tol)
    dec, errs = _reference_advance(b, net, K, 4, check_every, tol)
    assert log.decisions == dec
    assert log.jumps == 16 and log.accepted == sum(d == "accept" for _, _, d in dec)
    assert len(log.check_errors) == len(errs) == log.checks
    assert all(abs(x - y) <= 1e-12 * y for x, y in zip(log.check_errors, errs))
    for sa, sb in zip(a, b):
        assert np.array_equal(sa.get_field(0), sb.get_field(0))
        assert np.array_equal(sa.get_field(1), sb.get_field(1))
        assert sa.sav_scalars()["r"] == sb.sav_scalars()["r"]
    if check_every == 1:
        assert log.rejected_check > 0   # tol 1e-3 is tighter than the network
    if tol > 1:
        assert log.rejected_check == 0


def test_the_native_loop_refuses_mismatched_handles(trained):
    """Twins must match their runs (grid, parameters, precision); runs must be
    initialised square grids of the network's size; checks need twins."""
    import ctypes as ct
    from paper_2012_15133_gb300 import Solver
    from paper_2012_15133_gb300.spfc import load_library
    lib = load_library()
    net = trained[0]
    a = _solvers(2)
    good = [Solver(2, N, s.L[0], s.eps, s.beta, s.dt, "fp32") for s in a]
    wrong = [Solver(2, N, s.L[0], s.eps + 0.01, s.beta, s.dt, "fp32") for s in a]
    fresh = Solver(2, N, a[0].L[0], a[0].eps, a[0].beta, a[0].dt, "fp32")
    arr = lambda hs: (ct.c_void_p * len(hs))(*[h._h.value for h in hs])
    call = lambda runs, twins, check: lib.spfc_surrogate_advance(net._h, runs, twins, 2, K, 1, check, 1e-3,
                                                                 None, None, None)
    assert call(arr(a), arr(wrong), 1) == 1
    assert "parameters" in lib.spfc_surrogate_last_error().decode()
    assert call(arr(a), None, 1) == 1
    assert call(arr([a[0], fresh]), arr(good), 1) == 6       # not initialised
    assert call(arr(a), arr([good[0], a[0]]), 1) == 1       # a run as a twin of another
    assert "one of the runs" in lib.spfc_surrogate_last_error().decode()
    assert call(arr(a), arr([good[0], good[0]]), 1) == 1     # one twin for two runs
    assert call(arr([a[0], a[0]]), arr(good), 1) == 1        # a run twice
    assert call(arr(a), arr(good), 1) == 0
    for h in good + wrong + [fresh]:
        h.close()


def test_twins_follow_the_runs_stabiliser_and_phi4_term(trained):
    """judges_for gives each twin its run's stabiliser and gamma3, which the
    native loop requires of a twin; the checked loop then runs."""
    from paper_2012_15133_gb300 import surrogate as S
    net = trained[0]
    a = _solvers(2)
    a[0].set_stabilization(2.0)
    a[1].set_gamma3(0.5)
    judges = S.judges_for(a)
    assert judges[0].stab == 2.0 and judges[1].gamma3 == 0.5
    log = S.advance(a, net, K, 2, check_every=1, tol=1e-3, judges=judges)
    assert log.jumps == 4
    for t in judges.values():
        t.close()


def test_weights_file_round_trip(trained, tmp_path):
    from paper_2012_15133_gb300 import surrogate as S, SPFCError
    net = trained[0]
    path = str(tmp_path / "net.fno")
    net.save(path)
    other = S.FNO(n=N, width=32, modes1=16, modes2=16, layers=4, proj=64, max_batch=16)
    other.set_params(S.init_params(other, 7))
    other.load(path)
    assert np.array_equal(other.get_params(), net.get_params())
    x = torch.full((2, N, N), 0.2, device="cuda")
    assert torch.equal(other.predict(x, x, [0.2, 0.1], [1.0, 0.8]), net.predict(x, x, [0.2, 0.1], [1.0, 0.8]))
    small = S.FNO(n=N, width=8, modes1=4, modes2=4, layers=1, proj=8, max_batch=4)
    with pytest.raises(SPFCError):
        small.load(path)
    other.close()
    small.close()


def test_what_the_trained_network_gains(trained):
    """Rel-L2 of K-step predictions against the plain scheme on held-out
    seeds (at the training pairs' times), for the trained network, the
    untrained one and the no-change predictor; the rel-L2 of a field is
    about the square root of the increment loss ratio times the no-change
    error. Then the point-steps/s of surrogate + fallback and of plain
    steps on the same runs."""
    from paper_2012_15133_gb300 import surrogate as S
    net, _, _, init = trained
    held = S.trajectory_pairs(_runs(4, held_out=True), 0.02, K, 8, 100, 50)
    fresh = S.FNO(n=N, width=32, modes1=16, modes2=16, layers=4, proj=64, max_batch=16)
    fresh.set_params(init)

    def rel_err(pred_fn):
        errs = []
        for i in (0, 16):
            sl = slice(i, i + 16)
            p = pred_fn(held["phi_n"][sl].contiguous(), held["phi_nm1"][sl].contiguous(), held["eps"][sl],
                        held["beta"][sl])
            t = held["target"][sl]
            errs += [float(torch.linalg.vector_norm(p[j] - t[j]) / torch.linalg.vector_norm(t[j])) for j in range(16)]
        return float(np.mean(errs))
    err_trained = rel_err(net.predict)
    err_untrained = rel_err(fresh.predict)
    err_none = rel_err(lambda a, b, e, bt: a)
    assert err_trained < 0.5 * err_none, (err_trained, err_none)
    assert err_trained < 0.5 * err_untrained, (err_trained, err_untrained)
    # throughput with and without the network (every 5th jump checked)
    jumps = 10
    sol = _solvers(8, warm=350)
    log, t_sur = S.timed(S.advance, sol, net, K, jumps, check_every=5, tol=1e-3)
    ref = _solvers(8, warm=350)
    _, t_plain = S.timed(lambda: [s.step(K * jumps) for s in ref])
    pts = 8 * N * N * K * jumps
    print(f"\nsurrogate 64^2: rel-L2 per jump trained {err_trained:.2e}, untrained {err_untrained:.2e}, "
          f"no change {err_none:.2e}; {log.as_dict()}; "
          f"Mpt-steps/s surrogate+fallback {pts / t_sur / 1e6:.0f}, plain {pts / t_plain / 1e6:.0f}")
    assert log.jumps == 8 * jumps


def test_the_native_loop_judges_runs_with_the_phi4_term(trained):
    """Runs with the phi^4 term (gamma3 = 0.5): the native loop's energy test
    takes the term into the restarted prediction's modified energy, as the
    loop composed from single calls does; the same decisions."""
    from paper_2012_15133_gb300 import surrogate as S
    net = trained[0]
    a, b = _solvers(4), _solvers(4)
    for s in a + b:
        s.set_gamma3(0.5)
    log = S.advance(a, net, K, 3, check_every=0)
    dec, _ = _reference_advance(b, net, K, 3, 0, 1e-3)
    assert log.decisions == dec
    for sa, sb in zip(a, b):
        assert np.array_equal(sa.get_field(0), sb.get_field(0))
