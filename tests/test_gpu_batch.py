"""Batched runs (the disjoint union of run meshes) against the oracle, run by run.

Each run r of a batch has its own box, sizes, bases and noise stream (seed + r); the oracle steps
each run on its own mesh from the GPU's input state of that run.  Tolerances as in
test_gpu_parity: fields 1e-10 relative with the solver at rtol 1e-13 (field error <= cond(A) x
rtol; small meshes reach 1e-10 at rtol 1e-12); at rtol 1e-8 the oracle's residual of
every run's solution is <= 1e-8.
"""
import numpy as np
import pytest
import torch

from oracle import ch_oracle as o
from paper_2204_03575_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def make_batch(lib, geoms, **kw):
    runs = [lib.Params(nx=g[0], ny=g[1], Lx=g[2] if len(g) > 2 else 1.0, Ly=g[3] if len(g) > 3 else 1.0)
            for g in geoms]
    p = lib.Params(**kw)
    mesh = lib.Mesh(p, runs=runs)
    system = lib.System(mesh, p)
    state = lib.State(system, lib.Precond(system))
    return mesh, system, state


def split(mesh, arr):
    off = mesh.run_offsets
    return [arr[off[r]:off[r + 1]] for r in range(mesh.nruns)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_parity_per_run(lib, precision):
    geoms = [(8, 12), (16, 16), (24, 10, 10.0, 2.5), (12, 20), (32, 32)]
    bases = [(0.33, 0.33), (0.25, 0.40), (0.40, 0.22), (0.30, 0.35), (0.21, 0.44)]
    mesh, system, state = make_batch(lib, geoms, rtol=1e-14, precision=precision)
    assert mesh.nruns == len(geoms)
    state.init_seeded_batch([b[0] for b in bases], [b[1] for b in bases], 0.01, seed=100)
    solvers = [o.Solver(o.Params(nx=g[0], ny=g[1], Lx=g[2] if len(g) > 2 else 1.0,
                                 Ly=g[3] if len(g) > 3 else 1.0)) for g in geoms]
    g0 = {k: v.cpu().numpy() for k, v in state.get().items()}
    prev = []
    for r, s in enumerate(solvers):
        pp, pn = inputs.initial_state(s.N, bases[r][0], bases[r][1], 0.01, seed=100 + r)
        np.testing.assert_array_equal(split(mesh, g0["phi_p"])[r], pp)   # seeded per run, bitwise
        np.testing.assert_array_equal(split(mesh, g0["phi_nfa"])[r], pn)
        prev.append(o.initial(s.N, pp, pn))
    for step in range(3):
        state.step()
        g = {k: split(mesh, v.cpu().numpy()) for k, v in state.get().items()}
        for r, s in enumerate(solvers):
            ref = s.step(prev[r])
            for gk in ("phi_p", "phi_nfa", "mu_p", "mu_nfa"):
                assert rel(g[gk][r], getattr(ref, gk)) < 1e-10, (step, r, gk)
            st = state.run_stats(r)
            assert st["status"] == 0 and max(st["relres"]) <= 1e-14
            assert abs(st["mass"][0] - o.mass(s.M, g["phi_p"][r])) <= 1e-12 * abs(st["mass"][0])
            prev[r] = o.State(g["phi_p"][r], g["phi_nfa"][r], g["mu_p"][r], g["mu_nfa"][r])


def test_batch_of_one_equals_plain_mesh(lib):
    """A batch holding one run is the plain mesh: identical mesh, matrices and steps."""
    p = lib.Params(nx=40, ny=28)
    plain = lib.State(*(lambda s: (s, lib.Precond(s)))(lib.System(lib.Mesh(p), p)))
    mesh, system, batch = make_batch(lib, [(40, 28)])
    for st in (plain, batch):
        st.init_seeded(0.33, 0.30, 0.01, seed=3)
    for _ in range(2):
        a, b = plain.step(), batch.step()
        assert a["iters"] == b["iters"]
    ga, gb = plain.get(), batch.get()
    for k in ga:
        assert torch.equal(ga[k], gb[k])


def test_batch_runs_converge_independently(lib):
    """Runs whose systems differ in difficulty keep separate iteration counts and residuals."""
    mesh, system, state = make_batch(lib, [(8, 8), (64, 64), (16, 48)])
    state.init_seeded_batch([0.33, 0.30, 0.25], [0.33, 0.30, 0.40], 0.01, seed=7)
    state.step()
    its = [state.run_stats(r)["iters"] for r in range(3)]
    for r in range(3):
        assert max(state.run_stats(r)["relres"]) <= 1e-8
    assert len({tuple(i) for i in its}) > 1


def test_batch_64_runs_full_size_residuals(lib):
    """The batched workload: 64 runs, sizes drawn from {64,96,128,192,256}^2, bases in
    [0.20, 0.45), FP32 V-cycles in FP64 FGMRES.  Every run's step has oracle residual <= 1e-8."""
    spec = inputs.batch_runs(64, seed=0)
    geoms = [(nx, ny) for nx, ny, _, _ in spec]
    mesh, system, state = make_batch(lib, geoms, precision=1)
    state.init_seeded_batch([s[2] for s in spec], [s[3] for s in spec], 0.01, seed=0)
    g0 = {k: split(mesh, v.cpu().numpy()) for k, v in state.get().items()}
    state.step()
    g1 = {k: split(mesh, v.cpu().numpy()) for k, v in state.get().items()}
    cache = {}
    for r, (nx, ny) in enumerate(geoms):
        if (nx, ny) not in cache:
            cache[(nx, ny)] = o.Solver(o.Params(nx=nx, ny=ny), factor=False)
        s = cache[(nx, ny)]
        prev = o.State(g0["phi_p"][r], g0["phi_nfa"][r], g0["mu_p"][r], g0["mu_nfa"][r])
        new = o.State(g1["phi_p"][r], g1["phi_nfa"][r], g1["mu_p"][r], g1["mu_nfa"][r])
        rr = s.relres(prev, new)
        assert max(rr) <= 1e-8, (r, nx, ny, rr)
        assert max(state.run_stats(r)["relres"]) <= 1e-8


def test_batch_patterned_substrate_per_run(lib):
    """With pattern = 1 each run's substrate sixths follow its own Lx: the batch's boundary loads
    equal the oracle's on each run's mesh (unaligned and aligned runs)."""
    geoms = [(8, 12), (24, 10, 10.0, 2.5), (13, 7, 3.0, 1.0)]
    kw = dict(pattern=1, h_p=0.3, h_nfa=-0.2)
    runs = [lib.Params(nx=g[0], ny=g[1], Lx=g[2] if len(g) > 2 else 1.0, Ly=g[3] if len(g) > 3 else 1.0)
            for g in geoms]
    p = lib.Params(**kw)
    mesh = lib.Mesh(p, runs=runs)
    system = lib.System(mesh, p)
    rng = np.random.default_rng(5)
    pp, pn = 0.2 + 0.3 * rng.random(system.n), 0.2 + 0.3 * rng.random(system.n)
    out = system.loads(torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda())
    gp, gn = [split(mesh, t.cpu().numpy()) for t in out[2:]]
    for r, g in enumerate(geoms):
        op = o.Params(nx=g[0], ny=g[1], Lx=g[2] if len(g) > 2 else 1.0, Ly=g[3] if len(g) > 3 else 1.0, **kw)
        egp, egn = o.boundary_load(o.mesh(op), split(mesh, pp)[r], split(mesh, pn)[r], op)
        assert rel(gp[r], egp) < 1e-13 and rel(gn[r], egn) < 1e-13, r


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_run_spanning_reduction_groups(lib, precision):
    """A run whose blocks start mid-grid and span several reduction groups.

    Blocks own at least 256 nodes, and the run-wide sums of a run with more than 16 blocks go
    through groups of 16 consecutive blocks of that run (group rows, per-group tickets).  Here
    the 96 x 96 run (9409 nodes, 37 blocks) starts at block 1, after a one-block run, and a
    one-block run follows it; every run must still match its own oracle step."""
    geoms = [(8, 8), (96, 96), (10, 6)]
    bases = [(0.33, 0.33), (0.28, 0.38), (0.40, 0.25)]
    mesh, system, state = make_batch(lib, geoms, rtol=1e-14, max_iter=2000, precision=precision)
    off = mesh.run_offsets
    assert off[2] - off[1] == 97 * 97 and off[1] - off[0] <= 256
    state.init_seeded_batch([b[0] for b in bases], [b[1] for b in bases], 0.01, seed=300)
    solvers = [o.Solver(o.Params(nx=g[0], ny=g[1])) for g in geoms]
    g0 = {k: split(mesh, v.cpu().numpy()) for k, v in state.get().items()}
    prev = [o.initial(s.N, g0["phi_p"][r], g0["phi_nfa"][r]) for r, s in enumerate(solvers)]
    for step in range(2):
        state.step()
        g = {k: split(mesh, v.cpu().numpy()) for k, v in state.get().items()}
        for r, s in enumerate(solvers):
            ref = s.step(prev[r])
            for gk in ("phi_p", "phi_nfa", "mu_p", "mu_nfa"):
                err = rel(g[gk][r], getattr(ref, gk))
                assert err < 1e-10, (step, r, gk, err)
            st = state.run_stats(r)
            assert st["status"] == 0 and max(st["relres"]) <= 1e-14
            assert abs(st["mass"][0] - o.mass(s.M, g["phi_p"][r])) <= 1e-12 * abs(st["mass"][0])
            prev[r] = o.State(g["phi_p"][r], g["phi_nfa"][r], g["mu_p"][r], g["mu_nfa"][r])
