"""The learned warm start on the GPU: network forward pass and gradients against the CPU oracle
(which emulates the kernels' bfloat16 roundings), training lowering the loss, and the guessed
step: it reaches the oracle's solution whatever the guess, uses a good guess and falls back from a
bad one."""
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


# small images, and the 129 x 129 and 257 x 257 images of the benchmark's meshes (many tiles per
# row and many rows of blocks: the multi-block tiling at full size)
@pytest.mark.parametrize("H,W", [(12, 20), (17, 9), (129, 129), (257, 257)])
def test_forward_matches_oracle(lib, H, W):
    rng = np.random.default_rng(0)
    net = lib.WarmStartNet(H, W, max_batch=2)
    theta = small_theta(rng)
    net.set_params(theta)
    mean, inv_std, scale = rng.standard_normal(8) * 0.1, rng.uniform(0.5, 2.0, 8), rng.uniform(0.5, 2.0, 4)
    net.set_norm(mean, inv_std, scale)
    state, prev = rng.standard_normal((H * W, 4)), rng.standard_normal((H * W, 4))
    pred = net.predict(torch.from_numpy(state).cuda(), torch.from_numpy(prev).cuda()).cpu().numpy()
    s, q = state.reshape(H, W, 4), prev.reshape(H, W, 4)
    y_ref, _ = wo.forward(wo.unpack(theta.astype(np.float64)), wo.inputs(s, q, mean, inv_std), bf=True)
    y = ((pred - state - (state - prev)) / (scale * wo.change_scale(s, q))).reshape(H, W, 4)
    assert np.linalg.norm(y - y_ref) <= 5e-3 * np.linalg.norm(y_ref)
    assert np.abs(y - y_ref).max() <= 3e-2 * np.abs(y_ref).max()
    # the oracle's whole prediction agrees too
    full = wo.predict(wo.unpack(theta.astype(np.float64)), s, q, (mean, inv_std, scale), bf=True)
    assert np.abs(pred.reshape(H, W, 4) - full).max() <= 3e-2 * np.abs(y_ref * scale * wo.change_scale(s, q)).max()


def test_zero_network_is_linear_extrapolation(lib):
    H, W = 9, 11
    net = lib.WarmStartNet(H, W, max_batch=1)
    net.set_params(np.zeros(net.nparams, np.float32))
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    rng = np.random.default_rng(7)
    s, q = rng.standard_normal((H * W, 4)), rng.standard_normal((H * W, 4))
    pred = net.predict(torch.from_numpy(s).cuda(), torch.from_numpy(q).cuda()).cpu().numpy()
    np.testing.assert_array_equal(pred, s + (s - q))


@pytest.mark.parametrize("lap,H,W", [(0.0, 12, 20), (0.5, 12, 20), (0.0, 129, 129), (0.5, 129, 131)])
def test_gradients_match_oracle(lib, lap, H, W):
    rng = np.random.default_rng(1)
    B = 2
    net = lib.WarmStartNet(H, W, max_batch=B)
    theta = small_theta(rng)
    net.set_params(theta)
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    x = rng.standard_normal((B, H * W, 4)).astype(np.float32)
    q = (x - 0.01 * rng.standard_normal((B, H * W, 4))).astype(np.float32)
    n = (2 * x.astype(np.float64) - q + 1e-3 * rng.standard_normal((B, H * W, 4))).astype(np.float32)
    loss = net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), torch.from_numpy(n).cuda(), 0.0,
                          lap=lap)
    _, g = net.get_params()
    img = lambda a, b: a[b].astype(np.float64).reshape(H, W, 4)
    xin = np.stack([wo.inputs(img(x, b), img(q, b)) for b in range(B)])
    tin = np.stack([wo.targets(img(x, b), img(q, b), img(n, b), np.ones(4)) for b in range(B)])
    L_ref, g_ref = wo.loss_and_grads(theta.astype(np.float64), xin, tin, bf=True, lap=lap)
    assert math.isclose(loss, L_ref, rel_tol=1e-3)
    # per layer (padded entries are zero on both sides)
    sizes = [9 * 16 * 32, 32, 9 * 32 * 32, 32, 9 * 32 * 8, 8]
    k = 0
    for n in sizes:
        a, b = g[k:k + n], g_ref[k:k + n]
        assert np.linalg.norm(a - b) <= 2e-2 * max(np.linalg.norm(b), 1e-12), (k, n)
        k += n
    # lr = 0 left the parameters unchanged
    p, _ = net.get_params()
    np.testing.assert_array_equal(p, theta)


def test_training_lowers_the_loss(lib):
    """Fit a smooth linear target map; Adam steps through the library drive the loss down."""
    rng = np.random.default_rng(2)
    B, H, W = 4, 24, 24
    net = lib.WarmStartNet(H, W, max_batch=B)
    from paper_2204_03575_gb300 import warmstart
    net.set_params(warmstart.init_params(net.nparams, 0))
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, W), indexing="ij")
    xs, qs, ns = [], [], []
    for b in range(B):
        f = np.stack([np.sin(3 * xx + b), np.cos(2 * yy - b), xx * yy, xx - yy], -1).reshape(-1, 4)
        d = 0.01 * np.cos(f)
        xs.append(f)
        qs.append(f - d)
        ns.append(f + d + 1e-3 * (0.5 * f[:, ::-1] - 0.2 * f))  # a smooth correction of the extrapolation
    X = torch.tensor(np.array(xs), dtype=torch.float32, device="cuda")
    Q = torch.tensor(np.array(qs), dtype=torch.float32, device="cuda")
    Nx = torch.tensor(np.array(ns), dtype=torch.float32, device="cuda")
    first = net.train_step(X, Q, Nx, 0.0)
    for _ in range(300):
        last = net.train_step(X, Q, Nx, 3e-3)
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
    oracle's own trajectory (the zero network gives loss 1 exactly).  The mesh has fewer nodes
    than the coarsest AMG level holds, so the library's Algorithm 1 is exact, as the oracle's."""
    nx, ny = 12, 8
    H, W = ny + 1, nx + 1
    solver = o.Solver(o.Params(nx=nx, ny=ny))
    traj = _trajectory(solver, 4, seed=3)
    X = np.stack([traj[2], traj[3]])
    Q = np.stack([traj[1], traj[2]])
    p = lib.Params(nx=nx, ny=ny)
    system = lib.System(lib.Mesh(p), p)
    net = lib.WarmStartNet(H, W, max_batch=2)
    rng = np.random.default_rng(12)
    norm = (rng.standard_normal(8) * 0.05, rng.uniform(0.5, 2.0, 8), np.array([0.3, 0.3, 0.2, 0.2]))
    net.set_norm(*norm)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    pc = lib.Precond(system) if precond else None
    net.set_params(np.zeros(net.nparams, np.float32))
    assert net.train_residual(system, Xd, Qd, 0.0, precond=pc) == 1.0
    theta = small_theta(rng, 0.2)
    net.set_params(theta)
    loss = net.train_residual(system, Xd, Qd, 0.0, precond=pc)
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
                                              [img(rhs(x)) for x in X], apply, norm, bf=True, apply_Pinv=Pinv)
    assert math.isclose(loss, L_ref, rel_tol=2e-3), (loss, L_ref)
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
        net.train_residual(system, x, x.clone(), 0.0)


def test_learned_warm_start_saves_iterations(lib):
    """Trained on the solver's own trajectories against the step residual, the network's guess
    takes fewer FGMRES iterations than the previous-state guess on a held-out run."""
    from paper_2204_03575_gb300 import warmstart as ws
    nx = 128
    data = ws.generate_pairs(nx, nx, seeds=range(8), steps=50, dtype=torch.float64)
    system = ws.make_system(nx, nx)
    net = lib.WarmStartNet(nx + 1, nx + 1, max_batch=8)
    net, info = ws.train_residual(data, net, system, epochs=8, batch=8, lr=2e-3)
    assert info["loss_per_epoch"][-1] < 0.8 * info["loss_per_epoch"][0]
    plain = ws.run_steps(nx, nx, 1000, 25)
    learned = ws.run_steps(nx, nx, 1000, 25, net=net)
    its = lambda st: float(np.mean([max(s["iters"]) for s in st[2:]]))
    # >= 3 % fewer iterations (measured 4.8 % with the default smoother: 12.09 vs 12.70 per step)
    assert its(learned) < 0.97 * its(plain), (its(learned), its(plain))
    # the guess was taken, and every step still met the tolerance
    assert np.mean([sum(s["warm"]) for s in learned[2:]]) > 1.0
    assert all(max(s["relres"]) <= 1e-8 for s in learned)


def test_step_learned_with_zero_network_is_extrapolation(lib):
    """ch_step_learned keeps the predecessor on the device: with the zero network its guess is
    s_k + (s_k - s_{k-1}), and the steps are bitwise those of ch_step_guess given that guess.
    The first two steps after the state is set start from the previous state."""
    from paper_2204_03575_gb300 import warmstart as ws
    nx, ny = 24, 20
    zero = ws.zero_net(nx, ny)
    a = ws.make_state(nx, ny)
    b = ws.make_state(nx, ny)
    for s in (a, b):
        s.init_seeded(0.33, 0.31, 0.01, seed=5)
    st_a = [a.step_learned(zero) for _ in range(5)]
    assert st_a[0]["warm"] == [0, 0] and st_a[1]["warm"] == [0, 0]
    prev = None
    for k in range(5):
        cur = b.state4()
        if k < 2:
            b.step()
        else:
            b.step_guess((cur + (cur - prev)).contiguous())
        prev = cur
    ga, gb = a.state4(), b.state4()
    assert torch.equal(ga, gb)
    assert sum(sum(s["warm"]) for s in st_a[2:]) >= 1


def test_step_learned_rejects_a_network_of_another_size(lib):
    from paper_2204_03575_gb300 import warmstart as ws
    s = ws.make_state(24, 20)
    s.init_seeded(0.33, 0.31, 0.01, seed=5)
    with pytest.raises(lib.ChError):
        s.step_learned(ws.zero_net(20, 24))


@pytest.mark.parametrize("fp32", [False, True])
def test_fit_norm_matches_its_definition(lib, fp32):
    """ch_ws_fit_norm: field means and 1/std over the set, change channels (0, 1), and the std of
    the extrapolation's correction in units of the per-sample RMS of the change (n - 1 divisors),
    against numpy in float64; the statistics are set on the network (a bias-only last layer makes
    the prediction s + d + b3 * out_scale * r)."""
    rng = np.random.default_rng(8)
    S, H, W = 5, 9, 13
    X = rng.standard_normal((S, H * W, 4)) * [1.0, 2.0, 0.5, 3.0] + [0.3, -0.2, 1.0, 0.0]
    Q = X - 0.01 * rng.standard_normal(X.shape)
    Y = 2 * X - Q + 1e-3 * rng.standard_normal(X.shape)
    dt = np.float32 if fp32 else np.float64
    X, Q, Y = (a.astype(dt) for a in (X, Q, Y))
    net = lib.WarmStartNet(H, W, max_batch=1)
    mean, inv_std, out = net.fit_norm(*(torch.from_numpy(a).cuda() for a in (Q, X, Y)))
    x, q, y = (a.astype(np.float64) for a in (X, Q, Y))
    d = x - q
    r = np.maximum(np.sqrt((d ** 2).mean(1, keepdims=True)), 1e-30)
    e = ((y - x) - d) / r
    np.testing.assert_allclose(mean[:4], x.reshape(-1, 4).mean(0), rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(mean[4:], 0.0)
    np.testing.assert_allclose(inv_std[:4], 1.0 / x.reshape(-1, 4).std(0, ddof=1), rtol=1e-12)
    np.testing.assert_array_equal(inv_std[4:], 1.0)
    np.testing.assert_allclose(out, e.reshape(-1, 4).std(0, ddof=1), rtol=1e-11)
    theta = np.zeros(net.nparams, np.float32)
    theta[-8:-4] = [0.5, -1.0, 2.0, 0.25]  # b3 (first four output channels)
    net.set_params(theta)
    s0, q0 = x[0], q[0]
    pred = net.predict(torch.from_numpy(s0).cuda(), torch.from_numpy(q0).cuda()).cpu().numpy()
    rr = wo.change_scale(s0.reshape(H, W, 4), q0.reshape(H, W, 4))
    want = s0 + (s0 - q0) + theta[-8:-4].astype(np.float64) * out.astype(np.float32) * rr
    np.testing.assert_allclose(pred, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
