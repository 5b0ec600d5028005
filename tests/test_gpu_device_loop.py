"""FGMRES with its convergence loop on the device (GPU).

With CUDA graphs on (the default), a plain ch_step is one graph launch: the right-hand sides, the
initial residual, a while node whose body switches between the Arnoldi steps and the end of a
restart cycle (the flags of every run and species decide the next case on the device), the masses
and the statistics.  With graphs off the host drives the same kernels in the same order, reading
the flags after every Arnoldi step.  The two must give bitwise the same steps, statistics and
launch accounting, on one mesh and on a batch, in both precisions, with and without restarts, and
the device loop must return the same statuses when a solve fails.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _solver(lib, batch, **kw):
    if batch:
        runs = [lib.Params(nx=nx, ny=ny) for nx, ny in ((24, 16), (40, 40), (16, 48))]
        p = lib.Params(**kw)
        system = lib.System(lib.Mesh(p, runs=runs), p)
        state = lib.State(system, lib.Precond(system))
        state.init_seeded_batch([0.33, 0.25, 0.40], [0.31, 0.40, 0.22], 0.01, seed=4)
    else:
        p = lib.Params(nx=48, ny=40, **kw)
        system = lib.System(lib.Mesh(p), p)
        state = lib.State(system, lib.Precond(system))
        state.init_seeded(0.33, 0.31, 0.01, seed=3)
    return system, state


def _no_ms(stats):
    return {k: v for k, v in stats.items() if k != "ms"}


def _steps(lib, nsteps, batch, **kw):
    system, state = _solver(lib, batch, **kw)
    lib.profile_read(reset=True)
    out = []
    for _ in range(nsteps):
        st = state.step(check=False)
        runs = [_no_ms(state.run_stats(r)) for r in range(3)] if batch else []
        out.append((st, runs, {k: v.cpu().numpy() for k, v in state.get().items()}))
    prof = lib.profile_read(reset=True)
    return out, prof


@pytest.mark.parametrize("batch", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("restart", [30, 4])
def test_device_loop_equals_host_loop(lib, batch, precision, restart):
    dev, pdev = _steps(lib, 3, batch, graphs=1, precision=precision, restart=restart)
    host, phost = _steps(lib, 3, batch, graphs=0, precision=precision, restart=restart)
    _compare(dev, pdev, host, phost, restart)


@pytest.mark.parametrize("batch", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_device_loop_equals_host_loop_minres(lib, batch, precision):
    """krylov = 1: MINRES's loop (start, iterations, true-residual checks, retargeting) on the device."""
    dev, pdev = _steps(lib, 3, batch, graphs=1, precision=precision, krylov=1)
    host, phost = _steps(lib, 3, batch, graphs=0, precision=precision, krylov=1)
    _compare(dev, pdev, host, phost, None)


def _compare(dev, pdev, host, phost, restart):
    for (sa, ra, ga), (sb, rb, gb) in zip(dev, host):
        assert sa["status"] == sb["status"] == 0
        for key in ("iters", "restarts", "relres", "mass"):
            assert sa[key] == sb[key], key
        assert ra == rb
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])
    if restart == 4:
        assert max(s["restarts"] for s, _, _ in dev) >= 2  # the loop really restarted
    # launch accounting: the same kernels, launches, bytes and FMAs (the host loop's flag
    # reductions and the device loop's control kernel both count as "flags")
    for name in set(pdev) | set(phost):
        if name.startswith("flags"):
            continue
        a, b = pdev.get(name), phost.get(name)
        assert a is not None and b is not None, name
        assert a["launches"] == b["launches"], name
        assert a["bytes"] == pytest.approx(b["bytes"], rel=1e-12), name
        assert a["fmas"] == pytest.approx(b["fmas"], rel=1e-12), name


def test_device_loop_guess_step_equals_host_loop(lib):
    def run(graphs):
        system, state = _solver(lib, False, graphs=graphs)
        state.step()
        g = state.get()
        guess = torch.stack([g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"]], 1).contiguous() * 1.001
        outs = []
        for _ in range(2):
            st = state.step_guess(guess)
            outs.append((st, {k: v.cpu().numpy() for k, v in state.get().items()}))
        return outs

    for (sa, ga), (sb, gb) in zip(run(1), run(0)):
        assert _no_ms(sa) == _no_ms(sb)
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("krylov", [0, 1])
@pytest.mark.parametrize("graphs", [1, 0])
def test_device_loop_statuses(lib, graphs, krylov):
    """Iteration cap and a non-finite state give the same statuses as the host loop, and the state
    stays usable (the next step after a fresh initialisation converges)."""
    p = lib.Params(nx=32, ny=32, max_iter=3, restart=2 if krylov == 0 else 8, graphs=graphs, krylov=krylov)
    system = lib.System(lib.Mesh(p), p)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.33, 0.01, seed=0)
    st = state.step(check=False)
    assert st["status"] == lib.ERR_NOT_CONVERGED
    if krylov == 0:
        assert st["iters"] == [3, 3] and st["restarts"] == 2
    assert all(np.isfinite(v.cpu().numpy()).all() for v in state.get().values())
    n = system.n
    bad = torch.full((n,), 0.33, dtype=torch.float64, device="cuda")
    bad[5] = float("nan")
    state.set(bad, bad.clone())
    st = state.step(check=False)
    assert st["status"] == lib.ERR_NONFINITE
    p2 = lib.Params(nx=32, ny=32, graphs=graphs, krylov=krylov)
    system2 = lib.System(lib.Mesh(p2), p2)
    state2 = lib.State(system2, lib.Precond(system2))
    state2.init_seeded(0.33, 0.33, 0.01, seed=0)
    st = state2.step(check=False)
    assert st["status"] == 0 and max(st["relres"]) <= 1e-8
