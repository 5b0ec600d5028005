"""The learned warm start on the GPU: network forward pass and gradients against the CPU oracle
(which emulates the kernels' bfloat16 roundings), training lowering the loss, and the guessed
step: it reaches the oracle's solution whatever the guess, uses a good guess and falls back from a
bad one.  The network predicts a learned second-order extrapolation s + d + theta * D from the
last three states (d the change, D the second difference, theta = y * out_scale)."""
import math

import numpy as np
import pytest
import torch

from oracle import ch_oracle as o
from oracle import warmstart_oracle as wo
from paper_2204_03575_gb300 import inputs

pytestmark = pytest.mark.gpu


def small_theta(rng, scale=0.25):
    return (rng.standard_normal(wo.NPARAM) * scale).astype(np.float32)


def _history(rng, P, B=None, dtype=np.float64):
    """Consecutive states s_{k-2}, s_{k-1}, s_k, s_{k+1} (P x 4, or B x P x 4)."""
    shape = (P, 4) if B is None else (B, P, 4)
    q2 = rng.standard_normal(shape)
    q = q2 + 0.05 * rng.standard_normal(shape)
    s = q + 0.05 * rng.standard_normal(shape)
    n = s + (s - q) + 0.8 * (s - 2 * q + q2) + 1e-3 * rng.standard_normal(shape)
    return [a.astype(dtype) for a in (q2, q, s, n)]


# small images, and the 129 x 129 and 257 x 257 images of the benchmark's meshes (many tiles per
# row and many rows of blocks: the multi-block tiling at full size)
@pytest.mark.parametrize("engine", [0, 1])  # mma.sync, tcgen05
@pytest.mark.parametrize("H,W", [(12, 20), (17, 9), (129, 129), (257, 257)])
def test_forward_matches_oracle(lib, H, W, engine):
    rng = np.random.default_rng(0)
    net = lib.WarmStartNet(H, W, max_batch=2)
    net.set_engine(engine)
    theta = small_theta(rng)
    net.set_params(theta)
    mean, inv_std, scale = rng.standard_normal(8) * 0.1, rng.uniform(0.5, 2.0, 8), rng.uniform(0.5, 2.0, 4)
    net.set_norm(mean, inv_std, scale)
    q2, q, s, _ = _history(rng, H * W)
    pred = net.predict(*(torch.from_numpy(a).cuda() for a in (s, q, q2))).cpu().numpy()
    img = lambda a: a.reshape(H, W, 4)
    ref = wo.predict(wo.unpack(theta.astype(np.float64)), img(s), img(q), img(q2), (mean, inv_std, scale), bf=True)
    # the network's part theta * D of the prediction
    c = pred.reshape(H, W, 4) - img(s) - (img(s) - img(q))
    c_ref = ref - img(s) - (img(s) - img(q))
    assert np.linalg.norm(c - c_ref) <= 5e-3 * np.linalg.norm(c_ref)
    assert np.abs(c - c_ref).max() <= 3e-2 * np.abs(c_ref).max()


def test_zero_and_unit_networks_are_linear_and_quadratic_extrapolation(lib):
    from paper_2204_03575_gb300 import warmstart as ws
    H, W = 9, 11
    rng = np.random.default_rng(7)
    q2, q, s, _ = (torch.from_numpy(a).cuda() for a in _history(rng, H * W))
    zero = ws.zero_net(W - 1, H - 1)
    zero.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    np.testing.assert_array_equal(zero.predict(s, q, q2).cpu().numpy(), (s + (s - q)).cpu().numpy())
    quad = ws.quadratic_net(W - 1, H - 1)
    np.testing.assert_allclose(quad.predict(s, q, q2).cpu().numpy(), (3 * s - 3 * q + q2).cpu().numpy(),
                               rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("engine", [0, 1])  # mma.sync, tcgen05
@pytest.mark.parametrize("lap,H,W", [(0.0, 12, 20), (0.5, 12, 20), (0.0, 129, 129), (0.5, 129, 131)])
def test_gradients_match_oracle(lib, lap, H, W, engine):
    rng = np.random.default_rng(1)
    B = 2
    net = lib.WarmStartNet(H, W, max_batch=B)
    net.set_engine(engine)
    theta = small_theta(rng)
    net.set_params(theta)
    norm = (rng.standard_normal(8) * 0.05, rng.uniform(0.5, 2.0, 8), np.array([0.7, 1.2, 0.5, 0.9]))
    net.set_norm(*norm)
    q2, q, x, n = _history(rng, H * W, B, np.float32)
    loss = net.train_step(*(torch.from_numpy(a).cuda() for a in (x, q, q2, n)), 0.0, lap=lap)
    _, g = net.get_params()
    img = lambda a: a.astype(np.float64).reshape(B, H, W, 4)
    L_ref, g_ref = wo.loss_and_grads(theta.astype(np.float64), img(x), img(q), img(q2), img(n), norm, bf=True, lap=lap)
    assert math.isclose(loss, L_ref, rel_tol=1e-3), (loss, L_ref)
    # per layer (padded entries are zero on both sides)
    sizes = [9 * 16 * 32, 32, 9 * 32 * 32, 32, 9 * 32 * 8, 8]
    k = 0
    for m in sizes:
        a, b = g[k:k + m], g_ref[k:k + m]
        assert np.linalg.norm(a - b) <= 2e-2 * max(np.linalg.norm(b), 1e-12), (k, m)
        k += m
    # lr = 0 left the parameters unchanged
    p, _ = net.get_params()
    np.testing.assert_array_equal(p, theta)


def test_training_lowers_the_loss(lib):
    """Fit a smooth field of second-order coefficients; Adam steps through the library drive the
    state-space loss down."""
    rng = np.random.default_rng(2)
    B, H, W = 4, 24, 24
    net = lib.WarmStartNet(H, W, max_batch=B)
    from paper_2204_03575_gb300 import warmstart as ws
    net.set_params(ws.init_params(net.nparams, 0))
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, W), indexing="ij")
    xs, qs, q2s, ns = [], [], [], []
    for b in range(B):
        f = np.stack([np.sin(3 * xx + b), np.cos(2 * yy - b), xx * yy, xx - yy], -1).reshape(-1, 4)
        d1, d2 = 0.01 * np.cos(f), 0.01 * np.cos(f) - 0.002 * np.sin(2 * f)
        th = (0.5 + 0.4 * np.tanh(f))  # the coefficient of the second difference, smooth in the fields
        q2s.append(f - d1 - d2)
        qs.append(f - d1)
        xs.append(f)
        ns.append(f + d1 + th * (d1 - d2))
    T = lambda a: torch.tensor(np.array(a), dtype=torch.float32, device="cuda")
    X, Q, Q2, Nx = T(xs), T(qs), T(q2s), T(ns)
    first = net.train_step(X, Q, Q2, Nx, 0.0)
    for _ in range(300):
        last = net.train_step(X, Q, Q2, Nx, 3e-3)
    assert last < 0.05 * first, (first, last)


def _state_pair(lib, nx, ny, rtol):
    p = lib.Params(nx=nx, ny=ny, rtol=rtol)
    system = lib.System(lib.Mesh(p), p)
    return lib.State(system, lib.Precond(system)), system


def test_guess_step_reaches_the_oracle_solution(lib):
    """Whatever the guess -- a good one, a poor one -- the step is the oracle's step."""
    nx, ny = 24, 20
    s = o.Solver(o.Params(nx=nx, ny=ny))
    pp, pn = inputs.initial_state(s.N, 0.33, 0.31, 0.01, seed=9)
    ref = s.step(o.initial(s.N, pp, pn))
    good = torch.tensor(np.stack([ref.phi_p, ref.phi_nfa, ref.mu_p, ref.mu_nfa], 1) * (1 + 1e-7),
                        device="cuda")
    bad = torch.full((s.N, 4), 7.0, dtype=torch.float64, device="cuda")
    for guess, expect_warm in ((good, [1, 1]), (bad, [0, 0])):
        state, _ = _state_pair(lib, nx, ny, 1e-13)
        state.set(torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda())
        st = state.step_guess(guess)
        assert st["warm"] == expect_warm
        g = {k: v.cpu().numpy() for k, v in state.get().items()}
        for k in ("phi_p", "phi_nfa", "mu_p", "mu_nfa"):
            assert np.abs(g[k] - getattr(ref, k)).max() <= 1e-10 * np.abs(getattr(ref, k)).max(), k
    # the good guess saves iterations
    st_plain_state, _ = _state_pair(lib, nx, ny, 1e-13)
    st_plain_state.set(torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda())
    plain = st_plain_state.step()
    state, _ = _state_pair(lib, nx, ny, 1e-13)
    state.set(torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda())
    warm = state.step_guess(good)
    assert max(warm["iters"]) < max(plain["iters"])


def _oracle_operator(solver):
    """The saddle operator of the oracle's step on H x W x 4 node images, and the rhs builder."""
    A = o.saddle_matrix(solver.M, solver.K, solver.p)
    N = solver.N

    def apply(img):
        flat = img.reshape(N, 4)
        out = np.empty_like(flat)
        for sp in (0, 1):
            v = A @ np.concatenate([flat[:, sp], flat[:, sp + 2]])
            out[:, sp], out[:, sp + 2] = v[:N], v[N:]
        return out.reshape(img.shape)

    def rhs(state4):
        st = o.State(state4[:, 0], state4[:, 1], state4[:, 2], state4[:, 3])
        bp, bn = solver.rhs_pair(st)
        return np.stack([bp[:N], bn[:N], bp[N:], bn[N:]], 1)
    return apply, rhs


def _trajectory(solver, nsteps, seed):
    pp, pn = inputs.initial_state(solver.N, 0.33, 0.31, 0.01, seed=seed)
    s = o.initial(solver.N, pp, pn)
    out = [np.stack([s.phi_p, s.phi_nfa, s.mu_p, s.mu_nfa], 1)]
    for _ in range(nsteps):
        s = solver.step(s)
        out.append(np.stack([s.phi_p, s.phi_nfa, s.mu_p, s.mu_nfa], 1))
    return out


@pytest.mark.parametrize("precond", [False, True])
def test_residual_training_matches_oracle(lib, precond):
    """Loss and gradients of the residual-loss step against the oracle's, on states of the
    oracle's own trajectory (the zero network gives loss 0 exactly: ln 1).  The mesh has fewer nodes
    than the coarsest AMG level holds, so the library's Algorithm 1 is exact, as the oracle's."""
    nx, ny = 12, 8
    H, W = ny + 1, nx + 1
    solver = o.Solver(o.Params(nx=nx, ny=ny))
    traj = _trajectory(solver, 5, seed=3)
    X = np.stack([traj[3], traj[4]])
    Q = np.stack([traj[2], traj[3]])
    Q2 = np.stack([traj[1], traj[2]])
    p = lib.Params(nx=nx, ny=ny)
    system = lib.System(lib.Mesh(p), p)
    net = lib.WarmStartNet(H, W, max_batch=2)
    rng = np.random.default_rng(12)
    norm = (rng.standard_normal(8) * 0.05, rng.uniform(0.5, 2.0, 8), np.array([0.8, 1.1, 0.6, 1.3]))
    net.set_norm(*norm)
    Xd, Qd, Q2d = (torch.from_numpy(a).cuda() for a in (X, Q, Q2))
    pc = lib.Precond(system) if precond else None
    net.set_params(np.zeros(net.nparams, np.float32))
    assert net.train_residual(system, Xd, Qd, Q2d, 0.0, precond=pc) == 0.0
    theta = small_theta(rng, 0.2)
    net.set_params(theta)
    loss = net.train_residual(system, Xd, Qd, Q2d, 0.0, precond=pc)
    _, g = net.get_params()
    apply, rhs = _oracle_operator(solver)
    img = lambda a: a.reshape(H, W, 4)
    Pinv = None
    if precond:
        def Pinv(v):
            flat = v.reshape(-1, 4)
            w1, w2 = o.algorithm1_exact(solver.M, solver.K, solver.p, flat[:, :2], flat[:, 2:])
            return np.concatenate([w1, w2], 1).reshape(v.shape)
    L_ref, g_ref = wo.residual_loss_and_grads(theta.astype(np.float64), [img(x) for x in X], [img(q) for q in Q],
                                              [img(q) for q in Q2], [img(rhs(x)) for x in X], apply, norm, bf=True,
                                              apply_Pinv=Pinv)
    assert math.isclose(loss, L_ref, rel_tol=2e-3, abs_tol=2e-3), (loss, L_ref)
    sizes = [9 * 16 * 32, 32, 9 * 32 * 32, 32, 9 * 32 * 8, 8]
    k = 0
    for n in sizes:
        a, b = g[k:k + n], g_ref[k:k + n]
        assert np.linalg.norm(a - b) <= 2e-2 * max(np.linalg.norm(b), 1e-30), (k, n)
        k += n


def test_residual_training_rejects_a_mismatched_system(lib):
    p = lib.Params(nx=12, ny=8)
    system = lib.System(lib.Mesh(p), p)
    net = lib.WarmStartNet(10, 13, max_batch=1)
    x = torch.zeros((1, 13 * 10, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.ChError):
        net.train_residual(system, x, x.clone(), x.clone(), 0.0)


def test_learned_warm_start_saves_iterations(lib):
    """Trained on the solver's own trajectories against the step residual, the network's guess
    takes fewer FGMRES iterations on a held-out run than the previous-state guess and than linear
    extrapolation (the zero network), and about as few as quadratic extrapolation (theta = 1), the
    held-out selection's fallback."""
    from paper_2204_03575_gb300 import warmstart as ws
    nx = 128
    data = ws.generate_pairs(nx, nx, seeds=range(8), steps=50, dtype=torch.float64)
    system = ws.make_system(nx, nx)
    net = lib.WarmStartNet(nx + 1, nx + 1, max_batch=8)
    net, info = ws.train_residual(data, net, system, epochs=8, batch=8, lr=2e-3)
    del data
    assert info["loss_per_epoch"][-1] < 0.0  # beats linear extrapolation on the training set
    plain = ws.run_steps(nx, nx, 1000, 25)
    learned = ws.run_steps(nx, nx, 1000, 25, net=net)
    linear = ws.run_steps(nx, nx, 1000, 25, extrapolate=True)
    quad = ws.run_steps(nx, nx, 1000, 25, net=ws.quadratic_net(nx, nx))
    its = lambda st: float(np.mean([max(s["iters"]) for s in st[3:]]))
    print({"previous": its(plain), "linear": its(linear), "quadratic": its(quad), "learned": its(learned)})
    assert its(learned) < 0.97 * its(plain), (its(learned), its(plain))
    assert its(learned) < its(linear), (its(learned), its(linear))
    # selection by the iterations of a validation run (seed 999) among theta = 1 (quadratic
    # extrapolation), per-field constants fitted on that run, and the epochs: the kept network is no
    # worse than theta = 1 there, and on this run within 5 % of it
    sc, const = info["selection_scores_quadratic_then_epochs"], info["constant_theta"]
    assert info["held_out_pairs"] > 0 and len(info["held_out_loss_per_epoch"]) == 8 and len(sc) == 9
    sel = info["selected"]
    kept = sc[0] if sel == "quadratic" else const["iterations"] if sel == "constant theta" else sc[int(sel.split()[1])]
    assert kept == min([sc[0], const["iterations"]] + sc[1:])  # the kept candidate has the fewest
    assert its(learned) <= 1.05 * its(quad), (its(learned), its(quad))
    # the guess was taken, and every step still met the tolerance
    assert np.mean([sum(s["warm"]) for s in learned[3:]]) > 1.0
    assert all(max(s["relres"]) <= 1e-8 for s in learned)


def test_step_learned_with_zero_network_is_extrapolation(lib):
    """ch_step_learned keeps two predecessors on the device: with the zero network its guess is
    s_k + (s_k - s_{k-1}), and the steps are bitwise those of ch_step_guess given that guess.
    The first three steps after the state is set start from the previous state."""
    from paper_2204_03575_gb300 import warmstart as ws
    nx, ny = 24, 20
    zero = ws.zero_net(nx, ny)
    a = ws.make_state(nx, ny)
    b = ws.make_state(nx, ny)
    for s in (a, b):
        s.init_seeded(0.33, 0.31, 0.01, seed=5)
    st_a = [a.step_learned(zero) for _ in range(6)]
    assert all(s["warm"] == [0, 0] for s in st_a[:3])
    prev = None
    for k in range(6):
        cur = b.state4()
        if k < 3:
            b.step()
        else:
            b.step_guess((cur + (cur - prev)).contiguous())
        prev = cur
    ga, gb = a.state4(), b.state4()
    assert torch.equal(ga, gb)
    assert sum(sum(s["warm"]) for s in st_a[3:]) >= 1


def test_step_learned_rejects_a_network_of_another_size(lib):
    from paper_2204_03575_gb300 import warmstart as ws
    s = ws.make_state(24, 20)
    s.init_seeded(0.33, 0.31, 0.01, seed=5)
    with pytest.raises(lib.ChError):
        s.step_learned(ws.zero_net(20, 24))


@pytest.mark.parametrize("fp32", [False, True])
def test_fit_norm_matches_its_definition(lib, fp32):
    """ch_ws_fit_norm: field means and 1/std over the set (n - 1 divisor), change channels (0, 1),
    out_scale 1, against numpy in float64; the statistics are set on the network (a bias-only last
    layer makes the prediction s + d + b3 * D, and the field statistics enter the input)."""
    rng = np.random.default_rng(8)
    S, H, W = 5, 9, 13
    q2, q, x, _ = _history(rng, H * W, S)
    x = x * [1.0, 2.0, 0.5, 3.0] + [0.3, -0.2, 1.0, 0.0]
    dt = np.float32 if fp32 else np.float64
    X = x.astype(dt)
    net = lib.WarmStartNet(H, W, max_batch=1)
    mean, inv_std, out = net.fit_norm(torch.from_numpy(X).cuda())
    xd = X.astype(np.float64)
    np.testing.assert_allclose(mean[:4], xd.reshape(-1, 4).mean(0), rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(mean[4:], 0.0)
    np.testing.assert_allclose(inv_std[:4], 1.0 / xd.reshape(-1, 4).std(0, ddof=1), rtol=1e-12)
    np.testing.assert_array_equal(inv_std[4:], 1.0)
    np.testing.assert_array_equal(out, 1.0)
    theta = np.zeros(net.nparams, np.float32)
    theta[-8:-4] = [0.5, -1.0, 2.0, 0.25]  # b3 (first four output channels)
    net.set_params(theta)
    s0, q0, q20 = xd[0], q[0], q2[0]
    pred = net.predict(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s0, q0, q20))).cpu().numpy()
    want = s0 + (s0 - q0) + theta[-8:-4].astype(np.float64) * (s0 - 2 * q0 + q20)
    np.testing.assert_allclose(pred, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # a network reading the fields: its output, and so the prediction, depends on the statistics set
    theta = small_theta(rng, 0.3)
    net.set_params(theta)
    a = net.predict(*(torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (s0, q0, q20))).cpu().numpy()
    ref = wo.predict(wo.unpack(theta.astype(np.float64)), s0.reshape(H, W, 4), q0.reshape(H, W, 4),
                     q20.reshape(H, W, 4), (mean, inv_std, out), bf=True)
    c, cr = a.reshape(H, W, 4) - 2 * s0.reshape(H, W, 4) + q0.reshape(H, W, 4), ref - 2 * s0.reshape(H, W, 4) + q0.reshape(H, W, 4)
    assert np.linalg.norm(c - cr) <= 5e-3 * np.linalg.norm(cr)


def test_engines_agree_and_bad_engine_is_refused(lib):
    """The tcgen05 and mma.sync convolutions give the same predictions up to FP32 accumulation
    order (then one BF16 rounding of the activations); an unknown engine is refused."""
    H, W = 65, 97
    rng = np.random.default_rng(3)
    theta = small_theta(rng)
    q2, q, s, _ = (torch.from_numpy(a).cuda() for a in _history(rng, H * W))
    preds = []
    for engine in (0, 1):
        net = lib.WarmStartNet(H, W, max_batch=1)
        net.set_engine(engine)
        net.set_params(theta)
        net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
        preds.append(net.predict(s, q, q2).cpu().numpy() - (2 * s - q).cpu().numpy())
    a, b = preds
    assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b)
    with pytest.raises(lib.ChError) as e:
        net.set_engine(2)
    assert e.value.status == lib.ERR_ARG


def test_tcgen05_wait_timeout_is_reported_and_the_context_stays_usable(lib):
    """The tcgen05 convolutions' only wait (on the mbarrier their MMAs commit to) is bounded: with
    the MMAs withheld (ch_ws_inject_mma_timeout) every block's wait runs out, the blocks free their
    tensor memory and return, and the synchronising training call reports CH_ERR_INTERNAL once; the
    device context stays usable and the same step then reproduces its loss bitwise."""
    H, W, B = 33, 41, 2
    rng = np.random.default_rng(11)
    net = lib.WarmStartNet(H, W, max_batch=B)
    net.set_engine(1)
    net.set_params(small_theta(rng))
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    q2, q, x, n = (torch.from_numpy(a).cuda() for a in _history(rng, H * W, B, np.float32))
    ref = net.train_step(x, q, q2, n, 0.0)
    net.inject_mma_timeout(True)
    with pytest.raises(lib.ChError) as e:
        net.train_step(x, q, q2, n, 0.0)
    assert e.value.status == lib.ERR_INTERNAL
    net.inject_mma_timeout(False)
    assert net.train_step(x, q, q2, n, 0.0) == ref
