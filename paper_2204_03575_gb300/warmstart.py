"""Learned warm start: training data from the solver, training and use of the network.

The network (``ch.WarmStartNet``, kernels in ``csrc/warmstart.cu``) predicts the state at step k+1
from the states at steps k, k-1 and k-2 on the nodal image of a 2D structured mesh as a learned
second-order extrapolation s_k + d + theta * D (d the last change, D the second difference, theta
the network's output scaled per channel); ``ch_step_guess`` takes the prediction as FGMRES's
initial iterate wherever its true FP64 residual beats that of the previous state, so the FP64
residual decides between it and the previous step, which stays the fallback.

    data = generate_pairs(nx, ny, seeds=range(20), steps=100, dtype=torch.float64)  # plain solver
    net = ch.WarmStartNet(ny + 1, nx + 1, 8)
    net, info = train_residual(data, net, make_system(nx, ny))   # library kernels, Adam
    stats = run_steps(nx, ny, seed, 20, net=net)                  # ch_step_learned per step

PyTorch holds the tensors (state stacks, shuffling indices); the normalisation statistics, every
layer, loss, gradient and optimiser update, and every prediction during stepping run in the
library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ch, inputs


def seed_bases(seed: int, lo: float = 0.20, hi: float = 0.45):
    """Initial bases (phi_p0, phi_nfa0) of a training run, uniform in [lo, hi) from SplitMix64."""
    u = (inputs.splitmix64(np.uint64(seed) ^ (np.uint64(0x5EED) << np.uint64(40)) ^ np.arange(2, dtype=np.uint64))
         >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return lo + (hi - lo) * u[0], lo + (hi - lo) * u[1]


def make_state(nx: int, ny: int, precision: int = 0, **kw):
    p = ch.Params(nx=nx, ny=ny, precision=precision, **kw)
    system = ch.System(ch.Mesh(p), p)
    return ch.State(system, ch.Precond(system))


def make_system(nx: int, ny: int, **kw):
    """The time-step system of the nx x ny mesh (for the residual loss)."""
    p = ch.Params(nx=nx, ny=ny, **kw)
    return ch.System(ch.Mesh(p), p)


def generate_pairs(nx: int, ny: int, seeds, steps: int, precision: int = 0, burn_in: int = 1,
                   dtype=torch.float32):
    """(Q2, Q, X, Y): CUDA tensors (S, N, 4) of `dtype` holding consecutive states s_{k-2}, s_{k-1},
    s_k, s_{k+1} along the solver's own trajectories, `steps` quadruples per seed.  The first
    quadruple starts `burn_in` steps after the initial state (whose chemical potentials the first
    step sets up)."""
    q2s, qs, xs, ys = [], [], [], []
    state = make_state(nx, ny, precision)
    for seed in seeds:
        b0, b1 = seed_bases(seed)
        state.init_seeded(b0, b1, 0.01, seed=int(seed))
        for _ in range(burn_in):
            state.step()
        hist = [state.state4()]
        for _ in range(2):
            state.step()
            hist.append(state.state4())
        for _ in range(steps):
            state.step()
            nxt = state.state4()
            q2s.append(hist[-3].to(dtype))
            qs.append(hist[-2].to(dtype))
            xs.append(hist[-1].to(dtype))
            ys.append(nxt.to(dtype))
            hist = hist[-2:] + [nxt]
    return torch.stack(q2s), torch.stack(qs), torch.stack(xs), torch.stack(ys)


def init_params(nparams: int, seed: int = 0):
    """He-uniform initial weights in the library's parameter layout, zero biases but for the output
    bias of the four used channels, 1: with out_scale 1 the network starts close to theta = 1,
    quadratic extrapolation."""
    rng = np.random.default_rng(seed)
    layers = [(9 * 16 * 32, 9 * 12, 32), (9 * 32 * 32, 9 * 32, 32), (9 * 32 * 8, 9 * 32, 8)]
    out = []
    for i, (n, fan_in, nb) in enumerate(layers):
        lim = np.sqrt(6.0 / fan_in) * (0.1 if i == 2 else 1.0)  # start close to theta = 1
        out.append(rng.uniform(-lim, lim, n))
        out.append(np.zeros(nb))
    out[-1][:4] = 1.0
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == nparams
    return theta


def train(data, net, epochs: int = 8, batch: int = 8, lr: float = 2e-3, seed: int = 0,
          use_fields: bool = True, lap: float = 0.0):
    """Fit `net` (a ch.WarmStartNet sized for the mesh) to the next states in state space on
    `data` = (Q2, Q, X, Y) from generate_pairs.  With use_fields=False the field channels are
    switched off (scale 0) and the network sees only the change and the second difference; `lap`
    weighs the grid-Laplacian term of the loss.  Returns (net, info)."""
    Q2, Q, X, Y = data
    S, N = X.shape[0], X.shape[1]
    mean, inv_std, out_scale = net.fit_norm(X)  # computed on the device by the library
    if not use_fields:
        mean[:4], inv_std[:4] = 0.0, 0.0
        net.set_norm(mean, inv_std, out_scale)
    net.set_params(init_params(net.nparams, seed))
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(S, generator=g)
        lr_ep = lr * (0.5 ** (ep // max(1, epochs // 3)))
        tot, nb = 0.0, 0
        for i in range(0, S - batch + 1, batch):
            idx = perm[i:i + batch].to(X.device)
            tot += net.train_step(X[idx].contiguous(), Q[idx].contiguous(), Q2[idx].contiguous(), Y[idx].contiguous(),
                                  lr_ep, lap=lap)
            nb += 1
        losses.append(tot / max(nb, 1))
    return net, {"loss_per_epoch": losses, "mean": mean.tolist(), "inv_std": inv_std.tolist(),
                 "out_scale": out_scale.tolist(), "pairs": S, "nodes": N}


def validation_iterations(net, nx: int, ny: int, seed: int = 999, steps: int = 40, state=None):
    """Mean FGMRES iterations per step (worse species) over steps 4 .. steps + 3 of a seeded run whose
    steps are ch_step_learned with `net` (seed 999: neither a training seed nor the timed seed 1000)."""
    state = state or make_state(nx, ny)
    b0, b1 = seed_bases(seed)
    state.init_seeded(b0, b1, 0.01, seed=int(seed))
    for _ in range(3):  # ch_step_learned starts from the previous state for three steps
        state.step_learned(net)
    its = [max(state.step_learned(net)["iters"]) for _ in range(steps)]
    return float(np.mean(its))


def constant_theta(nparams: int, theta_phi: float, theta_mu: float):
    """Parameters of a network whose theta is constant per field: zero weights, output bias
    (theta_phi, theta_phi, theta_mu, theta_mu) for (phi_p, phi_nfa, mu_p, mu_nfa); with out_scale 1
    its prediction is s + d + theta_c D_c."""
    th = np.zeros(nparams, np.float32)
    th[-8:-4] = [theta_phi, theta_phi, theta_mu, theta_mu]
    return th


def calibrate_theta(net, nx: int, ny: int, seed: int = 999, steps: int = 40, state=None, start=(1.0, 1.0),
                    step: float = 0.1, lo: float = 0.0, hi: float = 1.5, max_moves: int = 20):
    """Fit the two constants (theta_phi, theta_mu) of constant_theta by the FGMRES iterations of a
    validation run (validation_iterations): coordinate search from `start` with steps of `step`,
    then `step` / 2, moving to the best of the four neighbours while it lowers the count.  Leaves
    the best constants in `net` and returns ((theta_phi, theta_mu), iterations, evaluations)."""
    state = state or make_state(nx, ny)
    seen = {}

    def cost(t):
        key = (round(t[0], 4), round(t[1], 4))
        if key not in seen:
            net.set_params(constant_theta(net.nparams, *key))
            seen[key] = validation_iterations(net, nx, ny, seed, steps, state)
        return seen[key]

    best = (float(start[0]), float(start[1]))
    f = cost(best)
    for h in (step, step / 2):
        for _ in range(max_moves):
            cand = [(min(hi, max(lo, best[0] + dx)), min(hi, max(lo, best[1] + dy)))
                    for dx, dy in ((h, 0), (-h, 0), (0, h), (0, -h))]
            fc, tc = min((cost(t), t) for t in cand)
            if fc >= f:
                break
            best, f = tc, fc
    net.set_params(constant_theta(net.nparams, *best))
    return best, f, len(seen)


def train_residual(data, net, system, epochs: int = 8, batch: int = 8, lr: float = 2e-3, seed: int = 0,
                   use_fields: bool = True, precond=None, val_frac: float = 0.1, select: str = "iterations",
                   val_seed: int = 999, val_steps: int = 40):
    """Fit `net` against the residual of the time step (ch_ws_train_residual) on fp64 `data` =
    (Q2, Q, X, Y) from generate_pairs(..., dtype=torch.float64); Y only sets the normalisation.
    With `precond` (a ch.Precond of `system`) the residual is measured in its norm.  The loss is
    the mean ln(|r|^2 / |r_linear extrapolation|^2): below 0 beats linear extrapolation.

    The last `val_frac` of the pairs (the last seeds' trajectories: generate_pairs orders them by
    seed) are held out; their loss (lr = 0: no update) is reported for exactly theta = 1 -- the
    quadratic extrapolation -- and after every epoch.  With select = "iterations" (default) the
    per-field constants (theta_phi, theta_mu) are first fitted by the FGMRES iterations of a
    validation run (calibrate_theta, seed val_seed), the network starts from them (output bias),
    and the kept parameters are those with the fewest validation iterations among theta = 1, the
    fitted constants and the network after every epoch; select = "loss" keeps the lowest held-out
    loss among theta = 1 and the epochs.  Either way theta = 1 is a candidate, so training can only
    improve on it as the selection measures it."""
    Q2, Q, X, Y = data
    S, N = X.shape[0], X.shape[1]
    nval = int(round(S * val_frac)) if val_frac > 0 else 0
    St = S - nval
    mean, inv_std, out_scale = net.fit_norm(X[:St])  # computed on the device by the library
    if not use_fields:
        mean[:4], inv_std[:4] = 0.0, 0.0
        net.set_norm(mean, inv_std, out_scale)

    def held_out_loss():
        tot, nb = 0.0, 0
        for i in range(St, S, batch):
            sl = slice(i, min(i + batch, S))
            tot += net.train_residual(system, X[sl].contiguous(), Q[sl].contiguous(), Q2[sl].contiguous(), 0.0,
                                      precond=precond)
            nb += 1
        return tot / nb if nb else float("nan")

    nx, ny = net.W - 1, net.H - 1
    vstate = make_state(nx, ny) if select == "iterations" else None

    def score(loss):
        return validation_iterations(net, nx, ny, val_seed, val_steps, vstate) if vstate else loss

    quad = constant_theta(net.nparams, 1.0, 1.0)  # zero weights, output bias 1: theta = out_scale = 1
    best, quad_loss, scores, const = None, None, [], None
    if nval:
        net.set_params(quad)
        quad_loss = held_out_loss()
        scores.append(score(quad_loss))
        best = (scores[-1], quad, "quadratic")
    theta0 = init_params(net.nparams, seed)
    if vstate is not None and nval:
        (tp, tm), f, nev = calibrate_theta(net, nx, ny, val_seed, val_steps, vstate)
        const = {"theta_phi": tp, "theta_mu": tm, "iterations": f, "evaluations": nev}
        if f < best[0]:
            best = (f, constant_theta(net.nparams, tp, tm), "constant theta")
        theta0[-8:-4] = [tp, tp, tm, tm]  # the network starts from the fitted constants
    net.set_params(theta0)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses, val = [], []
    for ep in range(epochs):
        perm = torch.randperm(St, generator=g)
        lr_ep = lr * (0.5 ** (ep // max(1, epochs // 3)))
        tot, nb = 0.0, 0
        for i in range(0, St - batch + 1, batch):
            idx = perm[i:i + batch].to(X.device)
            tot += net.train_residual(system, X[idx].contiguous(), Q[idx].contiguous(), Q2[idx].contiguous(), lr_ep,
                                      precond=precond)
            nb += 1
        losses.append(tot / max(nb, 1))
        if nval:
            val.append(held_out_loss())
            scores.append(score(val[-1]))
            if scores[-1] < best[0]:
                best = (scores[-1], net.get_params()[0].copy(), f"epoch {ep + 1}")
    if best is not None:
        net.set_params(best[1])
    return net, {"loss_per_epoch": losses, "held_out_loss_per_epoch": val,
                 "held_out_loss_quadratic": quad_loss, "selection": select,
                 "selection_scores_quadratic_then_epochs": scores, "constant_theta": const,
                 "mean": mean.tolist(),
                 "inv_std": inv_std.tolist(), "out_scale": out_scale.tolist(), "pairs": S, "held_out_pairs": nval,
                 "nodes": N, "selected": best[2] if best else f"epoch {epochs}"}


def zero_net(nx: int, ny: int):
    """A network whose output is zero: its prediction is the linear extrapolation 2 s_k - s_{k-1}."""
    net = ch.WarmStartNet(ny + 1, nx + 1, max_batch=1)
    net.set_params(np.zeros(net.nparams, np.float32))
    return net


def quadratic_net(nx: int, ny: int):
    """A network whose theta is 1 everywhere (zero weights, output bias 1, out_scale 1): its
    prediction is the quadratic extrapolation 3 s_k - 3 s_{k-1} + s_{k-2}."""
    net = ch.WarmStartNet(ny + 1, nx + 1, max_batch=1)
    theta = np.zeros(net.nparams, np.float32)
    theta[-8:-4] = 1.0
    net.set_params(theta)
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    return net


def run_steps(nx: int, ny: int, seed: int, steps: int, net=None, extrapolate: bool = False,
              precision: int = 0, warm_up: int = 0):
    """Advance a seeded run; return per-step stats.  With `net`, every step is ch_step_learned
    (the network's prediction where it beats the previous state, from the fourth step on); with
    `extrapolate`, the same with the zero network, i.e. the guess 2 s_k - s_{k-1}."""
    state = make_state(nx, ny, precision)
    b0, b1 = seed_bases(seed)
    state.init_seeded(b0, b1, 0.01, seed=int(seed))
    for _ in range(warm_up):
        state.step()
    if extrapolate and net is None:
        net = zero_net(nx, ny)
    return [state.step_learned(net) if net is not None else state.step() for _ in range(steps)]
