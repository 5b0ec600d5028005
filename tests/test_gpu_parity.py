"""Parity of the CUDA library (through the C ABI) with the CPU FP64 oracle.

Tolerances: integer/index data bit-exact; assembled values, loads and operator products
to 1e-13 relative (only the summation order differs); time-step fields to 1e-10
relative with the solver run at rtol 1e-12 (the error of a converged solve is bounded
by cond(A) x rtol); at the default rtol 1e-8 the true relative residual of the GPU's
solution, recomputed by the oracle from its own A and b, must be <= 1e-8.
"""
import math

import numpy as np
import pytest
import torch

from oracle import ch_oracle as o
from paper_2204_03575_gb300 import inputs

pytestmark = pytest.mark.gpu

POT = {"poly": 0, "poly_partial": 1, "none": 2, "fh": 3}


def make(ch, **kw):
    """Matching (C params, oracle params)."""
    okw = {k: v for k, v in kw.items() if k in o.Params.__dataclass_fields__}
    op = o.Params(**okw)
    ckw = {k: v for k, v in kw.items() if k != "potential"}
    ckw["potential"] = POT[kw.get("potential", "poly")]
    cp = ch.Params(**ckw)
    return cp, op


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = [dict(nx=32, ny=32), dict(nx=37, ny=23, Lx=10.0, Ly=2.5),
         dict(dim=3, nx=16, ny=16, nz=4, Lz=0.25), dict(dim=3, nx=5, ny=3, nz=4, Lx=10.0, Ly=2.5, Lz=10.0)]


# ---------------------------------------------------------------- mesh and assembly
@pytest.mark.parametrize("kw", CASES)
def test_mesh_parity(lib, kw):
    cp, op = make(lib, **kw)
    mesh = lib.Mesh(cp)
    om = o.mesh(op)
    coords, elems, bot, top = [t.cpu().numpy() for t in mesh.copy()]
    np.testing.assert_allclose(coords, om.coords, rtol=0, atol=1e-15 * np.abs(om.coords).max())
    np.testing.assert_array_equal(elems, om.elems)
    for g, r in ((bot, om.bottom), (top, om.top)):
        assert sorted(map(tuple, np.sort(g, 1))) == sorted(map(tuple, np.sort(r, 1)))


@pytest.mark.parametrize("kw", CASES)
def test_assembly_parity(lib, kw):
    cp, op = make(lib, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    M, K = o.assemble(o.mesh(op))
    rowptr, col, vm, vk, vh = [t.cpu().numpy() for t in system.csr()]
    np.testing.assert_array_equal(rowptr, M.indptr)
    np.testing.assert_array_equal(col, M.indices)
    assert rel(vm, M.data) < 1e-14 and rel(vk, K.data) < 1e-13
    a, c = o.coefficients(op)
    assert rel(vh, a * K.data + math.sqrt(c) * M.data) < 1e-13


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("potential", ["poly", "poly_partial", "none"])
def test_loads_parity(lib, kw, potential):
    cp, op = make(lib, potential=potential, h_p=0.3, h_nfa=-0.2, g_nfa=0.02, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    om = o.mesh(op)
    rng = np.random.default_rng(11)
    pp, pn = 0.2 + 0.3 * rng.random(system.n), 0.2 + 0.3 * rng.random(system.n)
    Fp, Fn, gp, gn = [t.cpu().numpy() for t in system.loads(cuda(pp), cuda(pn))]
    eFp, eFn = o.load_vector(om, pp, pn, potential)
    egp, egn = o.boundary_load(om, pp, pn, op)
    if potential == "none":
        assert np.all(Fp == 0) and np.all(Fn == 0)
    else:
        assert rel(Fp, eFp) < 1e-13 and rel(Fn, eFn) < 1e-13
    assert rel(gp, egp) < 1e-13 and rel(gn, egn) < 1e-13


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("chi", [{}, dict(chi_pn=2.5, chi_ps=-0.4, chi_ns=0.7, N_p=7.0, N_nfa=3.0, N_s=2.0)])
def test_flory_huggins_loads_parity(lib, kw, chi):
    """potential = 3 (Section 2's logarithmic f, reading R14): the device's element rule (its own
    3-point Gauss-Legendre table collapsed onto the simplex) against the oracle's rule, on states
    that reach the guard (values at and below 0 at some nodes, so quadrature points fall below
    fh_delta).  Logarithms are correctly rounded to within an ulp on both sides: 1e-12."""
    cp, op = make(lib, potential="fh", **chi, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    om = o.mesh(op)
    rng = np.random.default_rng(13)
    pp, pn = 0.05 + 0.5 * rng.random(system.n), 0.05 + 0.4 * rng.random(system.n)
    pp[::17] = -0.02
    pn[5::23] = 0.0
    pp[3::29] = 1e-12
    Fp, Fn, gp, gn = [t.cpu().numpy() for t in system.loads(cuda(pp), cuda(pn))]
    eFp, eFn = o.load_vector_fh(om, pp, pn, op)
    assert np.isfinite(Fp).all() and np.isfinite(Fn).all()
    assert rel(Fp, eFp) < 1e-12 and rel(Fn, eFn) < 1e-12
    egp, egn = o.boundary_load(om, pp, pn, op)
    assert rel(gp, egp) < 1e-13 and rel(gn, egn) < 1e-13


@pytest.mark.parametrize("kw", [dict(nx=32, ny=32), dict(dim=3, nx=16, ny=16, nz=4, Lz=0.25)])
def test_flory_huggins_step_parity(lib, kw):
    """Three steps with the Flory-Huggins load: fields 1e-10 against the oracle's direct solve."""
    _, out = run_pair(lib, 3, rtol=1e-13, max_iter=1000, potential="fh", **kw)
    for st, g, _, ref in out:
        assert st["status"] == 0
        for k in ("phi_p", "phi_nfa", "mu_p", "mu_nfa"):
            assert rel(g[k], getattr(ref, k)) < 1e-10, k


@pytest.mark.parametrize("kw", CASES + [dict(nx=36, ny=12, Lx=10.0, Ly=2.5),
                                 dict(dim=3, nx=12, ny=3, nz=5, Lx=10.0, Ly=2.5, Lz=10.0)])
def test_patterned_substrate_loads_parity(lib, kw):
    """Section 4's substrate patterning (p_p, p_nfa alternating on the sixths of [0, Lx]): facets
    cut by a breakpoint (nx not a multiple of 6) and aligned meshes, h != 0 so that the
    field-dependent part of the substrate load is exercised."""
    cp, op = make(lib, pattern=1, h_p=0.3, h_nfa=-0.2, g_nfa=0.02, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    om = o.mesh(op)
    rng = np.random.default_rng(12)
    pp, pn = 0.2 + 0.3 * rng.random(system.n), 0.2 + 0.3 * rng.random(system.n)
    _, _, gp, gn = [t.cpu().numpy() for t in system.loads(cuda(pp), cuda(pn))]
    egp, egn = o.boundary_load(om, pp, pn, op)
    assert rel(gp, egp) < 1e-13 and rel(gn, egn) < 1e-13
    flat = o.boundary_load(om, pp, pn, o.Params(**{**op.__dict__, "pattern": 0}))
    assert rel(gp, flat[0]) > 1e-3  # the pattern changes the load


@pytest.mark.parametrize("kw", CASES[:3])
def test_rhs_and_operator_parity(lib, kw):
    cp, op = make(lib, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    s = o.Solver(op)
    pp, pn = inputs.initial_state(s.N, 0.33, 0.31, 0.01, seed=4)
    b = system.rhs(cuda(pp), cuda(pn)).cpu().numpy()
    bp, bn = s.rhs_pair(o.initial(s.N, pp, pn))
    N = s.N
    assert rel(b[:, 0], bp[:N]) < 1e-13 and rel(b[:, 2], bp[N:]) < 1e-13
    assert rel(b[:, 1], bn[:N]) < 1e-13 and rel(b[:, 3], bn[N:]) < 1e-13
    rng = np.random.default_rng(5)
    x = rng.standard_normal((N, 4))
    y = system.apply_A(cuda(x)).cpu().numpy()
    yp = s.A @ np.concatenate([x[:, 0], x[:, 2]])
    yn = s.A @ np.concatenate([x[:, 1], x[:, 3]])
    assert rel(y[:, 0], yp[:N]) < 1e-13 and rel(y[:, 2], yp[N:]) < 1e-13
    assert rel(y[:, 1], yn[:N]) < 1e-13 and rel(y[:, 3], yn[N:]) < 1e-13


# ---------------------------------------------------------------- preconditioner
@pytest.mark.parametrize("kw", [dict(nx=64, ny=64), dict(nx=128, ny=96), dict(dim=3, nx=16, ny=16, nz=8, Lz=0.5)])
@pytest.mark.parametrize("precision", [0, 1])
def test_vcycle_converges(lib, kw, precision):
    """Repeated V-cycles are a convergent iteration for M and H (error shrinks geometrically).
    coarse_max 256 keeps several levels on every mesh here (the single dense level has its own
    test)."""
    cp, op = make(lib, precision=precision, coarse_max=256, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    pc = lib.Precond(system)
    M, K = o.assemble(o.mesh(op))
    a, c = o.coefficients(op)
    H = (a * K + math.sqrt(c) * M).tocsc()
    rng = np.random.default_rng(2)
    b = rng.standard_normal((system.n, 2))
    import scipy.sparse.linalg as spla
    for which, A in ((0, M.tocsc()), (1, H)):
        exact = np.stack([spla.spsolve(A, b[:, r]) for r in range(2)], 1)
        errs = []
        for k in (1, 2, 4):
            x = pc.vcycle(which, cuda(b), k).cpu().numpy()
            errs.append(np.linalg.norm(x - exact) / np.linalg.norm(exact))
        assert errs[0] < 0.5, (which, errs)
        # a convergent stationary iteration: 3 more cycles cut the error at least 10x
        # (down to the FP32 floor when the cycles run in single precision)
        floor = 1e-6 if precision == 1 else 0.0
        assert errs[1] < max(0.5 * errs[0], floor) and errs[2] < max(0.1 * errs[0], floor), (which, errs)


@pytest.mark.parametrize("kw", [dict(nx=32, ny=32), dict(nx=40, ny=24, Lx=10.0, Ly=2.5),
                                dict(dim=3, nx=8, ny=8, nz=4, Lz=0.5)])
def test_precond_is_algorithm1_in_the_exact_limit(lib, kw):
    """With many V-cycles per inner solve, Prec(v) -> (M^-1 v1, H^-1 M H^-1 v2) (Algorithm 1)."""
    cp, op = make(lib, vcycles_M=40, vcycles_H=40, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    pc = lib.Precond(system)
    M, K = o.assemble(o.mesh(op))
    rng = np.random.default_rng(3)
    v = rng.standard_normal((system.n, 4))
    w = pc.apply(cuda(v)).cpu().numpy()
    w1, w2 = o.algorithm1_exact(M, K, op, v[:, 0:2], v[:, 2:4])
    assert rel(w[:, 0:2], w1) < 1e-9
    assert rel(w[:, 2:4], w2) < 1e-9


@pytest.mark.parametrize("kw", [dict(nx=30, ny=30, coarse_max=1024), dict(nx=70, ny=48, coarse_max=4096)])
def test_dense_coarsest_inverse_above_one_block(lib, kw):
    """A coarsest level above 256 rows is inverted by the grid-wide Gauss-Jordan.  With the whole
    mesh at or below coarse_max the hierarchy is that one dense level, so one V-cycle per inner
    solve already is Algorithm 1 with exact solves."""
    cp, op = make(lib, vcycles_M=1, vcycles_H=1, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    pc = lib.Precond(system)
    assert pc.levels(0) == [(system.n, pc.levels(0)[0][1])] and len(pc.levels(1)) == 1
    M, K = o.assemble(o.mesh(op))
    rng = np.random.default_rng(4)
    v = rng.standard_normal((system.n, 4))
    w = pc.apply(cuda(v)).cpu().numpy()
    w1, w2 = o.algorithm1_exact(M, K, op, v[:, 0:2], v[:, 2:4])
    assert rel(w[:, 0:2], w1) < 1e-11
    assert rel(w[:, 2:4], w2) < 1e-10


def test_hierarchy_levels_coarsen(lib):
    cp, _ = make(lib, nx=128, ny=128)
    pc = lib.Precond(lib.System(lib.Mesh(cp), cp))
    for which in (0, 1):
        lv = pc.levels(which)
        assert lv[0][0] == 129 * 129 and lv[-1][0] <= 512  # coarse_max 0: 512 rows in FP64
        assert all(lv[i + 1][0] < lv[i][0] for i in range(len(lv) - 1))


# ---------------------------------------------------------------- time steps
def run_pair(lib, nsteps, base=(0.33, 0.33), seed=0, **kw):
    """GPU steps, each paired with the oracle's step from the same input (the GPU's previous
    state): out[k] = (stats, gpu fields after step k, input state of step k, oracle step)."""
    cp, op = make(lib, **kw)
    system = lib.System(lib.Mesh(cp), cp)
    pc = lib.Precond(system)
    state = lib.State(system, pc)
    s = o.Solver(op)
    pp, pn = inputs.initial_state(s.N, base[0], base[1], 0.01, seed=seed)
    state.set(cuda(pp), cuda(pn))
    prev = o.initial(s.N, pp, pn)
    out = []
    for _ in range(nsteps):
        stats = state.step()
        g = {k: v.cpu().numpy() for k, v in state.get().items()}
        out.append((stats, g, prev, s.step(prev)))
        prev = o.State(g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"])
    return s, out


FIELDS = (("phi_p", "phi_p"), ("phi_nfa", "phi_nfa"), ("mu_p", "mu_p"), ("mu_nfa", "mu_nfa"))


@pytest.mark.parametrize("precision", [0, 1])
def test_step_parity_2d_config1(lib, precision):
    """32x32 unit square, 0.33 +/- 0.01, 10 steps: every step's fields match the oracle's step
    from the same input."""
    s, out = run_pair(lib, 10, nx=32, ny=32, rtol=1e-12, precision=precision)
    for k, (stats, g, _, nxt) in enumerate(out):
        assert stats["status"] == 0
        for gk, ok in FIELDS:
            assert rel(g[gk], getattr(nxt, ok)) < 1e-10, (k, gk)
        np.testing.assert_array_equal(g["phi_s"], 1.0 - g["phi_p"] - g["phi_nfa"])
        assert math.isclose(stats["mass"][0], o.mass(s.M, g["phi_p"]), rel_tol=1e-12)
        assert math.isclose(stats["mass"][1], o.mass(s.M, g["phi_nfa"]), rel_tol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", [dict(nx=32, ny=32), dict(nx=48, ny=40, restart=5)])
def test_selective_reorthogonalisation_step_parity(lib, precision, kw):
    """gs_reorth = 1 (one Gram-Schmidt projection, the second only where the vector lost more than
    half its squared norm): every step's fields still match the oracle's step at the FP64 parity
    tolerance, with and without restarts; the second pass is taken on some Arnoldi steps, never
    more than there are; gs_reorth = 0 takes it on every one."""
    s, out = run_pair(lib, 6, rtol=1e-12, precision=precision, gs_reorth=1, **kw)
    for k, (stats, g, _, nxt) in enumerate(out):
        assert stats["status"] == 0
        for gk, ok in FIELDS:
            assert rel(g[gk], getattr(nxt, ok)) < 1e-10, (k, gk)
        assert all(0 <= r <= i for r, i in zip(stats["reorth"], stats["iters"]))
    assert sum(sum(st["reorth"]) for st, _, _, _ in out) < sum(sum(st["iters"]) for st, _, _, _ in out)
    _, out0 = run_pair(lib, 2, rtol=1e-12, precision=precision, **kw)
    assert all(st["reorth"] == st["iters"] for st, _, _, _ in out0)


def test_selective_reorthogonalisation_host_loop_matches_graphs(lib):
    """The device-side loop and the host-driven loop run the same selective passes: bitwise the same
    steps."""
    a = run_pair(lib, 2, nx=48, ny=40, gs_reorth=1, graphs=1)[1]
    b = run_pair(lib, 2, nx=48, ny=40, gs_reorth=1, graphs=0)[1]
    for (sa, ga, _, _), (sb, gb, _, _) in zip(a, b):
        assert sa["iters"] == sb["iters"] and sa["reorth"] == sb["reorth"]
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])


def test_trajectory_parity_2d_config1(lib):
    """The whole 10-step GPU trajectory against the oracle's own trajectory (errors compound
    through the explicit nonlinearity; 1e-9 relative)."""
    s, out = run_pair(lib, 10, nx=32, ny=32, rtol=1e-12)
    pp, pn = inputs.initial_state(s.N, 0.33, 0.33, 0.01, seed=0)
    traj = s.run(o.initial(s.N, pp, pn), 10)
    for k, (_, g, _, _) in enumerate(out):
        for gk, ok in FIELDS:
            assert rel(g[gk], getattr(traj[k + 1], ok)) < 1e-9, (k, gk)


@pytest.mark.parametrize("precision", [0, 1])
def test_step_parity_3d_subsize(lib, precision):
    """16x16x4 Kuhn mesh on [0,1]^2 x [0,0.25], 0.30 +/- 0.01: 3 steps.  The 3D saddle system is
    worse conditioned than config 1 (mu errors reach ~1.2e-10 at rtol 1e-12), so parity mode
    solves to 1e-13."""
    _, out = run_pair(lib, 3, base=(0.30, 0.30), dim=3, nx=16, ny=16, nz=4, Lz=0.25, rtol=1e-13,
                      precision=precision)
    for k, (stats, g, _, nxt) in enumerate(out):
        for gk, ok in FIELDS:
            assert rel(g[gk], getattr(nxt, ok)) < 1e-10, (k, gk)


def test_patterned_substrate_step_parity(lib):
    """Two steps on Section 4's 10 x 2.5 box (37 x 23 cells: breakpoints inside facets) with the
    patterned substrate against the oracle's steps from the same inputs."""
    _, out = run_pair(lib, 2, nx=37, ny=23, Lx=10.0, Ly=2.5, pattern=1, rtol=1e-13, max_iter=1000)
    for k, (stats, g, _, nxt) in enumerate(out):
        assert stats["status"] == 0
        for gk, ok in FIELDS:
            assert rel(g[gk], getattr(nxt, ok)) < 1e-10, (k, gk)


@pytest.mark.parametrize("kw", [dict(nx=48, ny=40), dict(nx=37, ny=23, Lx=10.0, Ly=2.5, tau=1e-5, eps=1e-2),
                                dict(nx=64, ny=64, bc_mode=0, evap_sign=-1)])
def test_step_default_tolerance_residual(lib, kw):
    """At rtol 1e-8 the oracle's own residual ||b - A x|| / ||b|| of each GPU step (b from the
    GPU's input state) is <= 1e-8 for both species."""
    s, out = run_pair(lib, 3, **kw)
    for stats, g, prev, _ in out:
        new = o.State(g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"])
        rr = s.relres(prev, new)
        assert max(rr) <= 1e-8, rr
        assert max(stats["relres"]) <= 1e-8


def test_seeded_initial_state_is_bitwise(lib):
    cp, _ = make(lib, nx=40, ny=30)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.30, 0.01, seed=12345)
    g = state.get()
    pp, pn = inputs.initial_state(system.n, 0.33, 0.30, 0.01, seed=12345)
    np.testing.assert_array_equal(g["phi_p"].cpu().numpy(), pp)
    np.testing.assert_array_equal(g["phi_nfa"].cpu().numpy(), pn)
    assert torch.all(g["mu_p"] == 0)


# ---------------------------------------------------------------- degenerate cases and errors
def test_constant_state_fixed_point(lib):
    cp, _ = make(lib, nx=20, ny=20, bc_mode=0, rtol=1e-12)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    n = system.n
    state.set(torch.full((n,), 0.35, dtype=torch.float64, device="cuda"),
              torch.full((n,), 0.25, dtype=torch.float64, device="cuda"))
    state.step()
    g = state.get()
    fp = 7 * 0.35 * 0.25 ** 2 - 0.2 * 0.4
    assert torch.allclose(g["phi_p"], torch.tensor(0.35, dtype=torch.float64), rtol=1e-11)
    assert torch.allclose(g["mu_p"], torch.tensor(fp, dtype=torch.float64), rtol=1e-9)


@pytest.mark.parametrize("kw", [dict(nx=1, ny=1), dict(nx=2, ny=1), dict(dim=3, nx=1, ny=1, nz=1),
                                dict(nx=300, ny=2)])
def test_tiny_and_thin_meshes(lib, kw):
    _, out = run_pair(lib, 2, rtol=1e-12, **kw)
    for stats, g, _, nxt in out:
        for gk, ok in FIELDS:
            assert rel(g[gk], getattr(nxt, ok)) < 1e-10, gk


def test_nonfinite_state_reported(lib):
    cp, _ = make(lib, nx=16, ny=16)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    pp, pn = inputs.initial_state(system.n, 0.33, 0.33, seed=1)
    pp[17] = np.nan
    state.set(cuda(pp), cuda(pn))
    with pytest.raises(lib.ChError) as e:
        state.step()
    assert e.value.status == lib.ERR_NONFINITE


def test_iteration_cap_reported_with_best_iterate(lib):
    cp, _ = make(lib, nx=32, ny=32, max_iter=2)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    pp, pn = inputs.initial_state(system.n, 0.33, 0.33, seed=1)
    state.set(cuda(pp), cuda(pn))
    stats = state.step(check=False)
    assert stats["status"] == lib.ERR_NOT_CONVERGED
    assert all(np.isfinite(v.cpu().numpy()).all() for v in state.get().values())


def test_step_before_set_is_a_state_error(lib):
    cp, _ = make(lib, nx=8, ny=8)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    with pytest.raises(lib.ChError) as e:
        state.step()
    assert e.value.status == lib.ERR_STATE


def test_graph_replay_matches_direct_launches(lib):
    """Arnoldi steps replayed from captured CUDA graphs give bitwise the same steps as direct launches."""
    a = run_pair(lib, 2, nx=48, ny=40, graphs=1)[1]
    b = run_pair(lib, 2, nx=48, ny=40, graphs=0)[1]
    for (sa, ga, _, _), (sb, gb, _, _) in zip(a, b):
        assert sa["iters"] == sb["iters"]
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("precision", [0, 1])
def test_programmatic_dependent_launch_matches_plain_launches(lib, precision):
    """pdl = 1 (V-cycle kernels scheduled while their predecessor drains, waiting on the device
    for its results) and pdl = 0 (plain stream-ordered launches) give bitwise the same steps."""
    a = run_pair(lib, 2, nx=48, ny=40, precision=precision, pdl=1)[1]
    b = run_pair(lib, 2, nx=48, ny=40, precision=precision, pdl=0)[1]
    for (sa, ga, _, _), (sb, gb, _, _) in zip(a, b):
        assert sa["iters"] == sb["iters"]
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("precision", [0, 1])
def test_parallel_m_branch_matches_serial_algorithm1(lib, precision):
    """Algorithm 1's M solve runs as a parallel branch of the H solves, except under per-launch
    event timing, which keeps one stream: both give bitwise the same steps."""
    a = run_pair(lib, 2, nx=48, ny=40, precision=precision)[1]
    lib.profile_enable(True)
    try:
        b = run_pair(lib, 2, nx=48, ny=40, precision=precision)[1]
    finally:
        lib.profile_enable(False)
        lib.profile_read(reset=True)
    for (sa, ga, _, _), (sb, gb, _, _) in zip(a, b):
        assert sa["iters"] == sb["iters"]
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])


def test_minres_step_parity(lib):
    """krylov = 1 (preconditioned MINRES, the paper's Krylov method, with Algorithm 1's fixed
    FP64 V-cycles): per-step fields match the oracle's direct solve like FGMRES's (rtol 1e-12)."""
    out = run_pair(lib, 4, nx=32, ny=32, rtol=1e-12, krylov=1)[1]
    for st, g, _, ref in out:
        assert st["status"] == 0 and max(st["relres"]) <= 1e-12
        for k in ("phi_p", "phi_nfa", "mu_p", "mu_nfa"):
            assert rel(g[k], getattr(ref, k)) < 1e-10, k


@pytest.mark.parametrize("precision", [0, 1])
def test_minres_default_tolerance_and_batch(lib, precision):
    """MINRES at the default rtol reaches the true 1e-8 residual on a 128 x 96 mesh and on a
    batch of runs of different sizes (per-run scalars), in FP64 and with FP32 V-cycles."""
    cp, _ = make(lib, nx=128, ny=96, krylov=1, precision=precision)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.31, 0.01, seed=2)
    for _ in range(3):
        st = state.step()
        assert st["status"] == 0 and max(st["relres"]) <= 1e-8
    pb = lib.Params(precision=precision, krylov=1)
    mesh = lib.Mesh(pb, runs=[lib.Params(nx=nx, ny=ny) for nx, ny in ((24, 16), (40, 40), (16, 48))])
    bsys = lib.System(mesh, pb)
    bstate = lib.State(bsys, lib.Precond(bsys))
    bstate.init_seeded_batch([0.33, 0.25, 0.40], [0.31, 0.40, 0.22], 0.01, seed=4)
    for _ in range(2):
        bstate.step()
        for r in range(3):
            rs = bstate.run_stats(r)
            assert rs["status"] == 0 and max(rs["relres"]) <= 1e-8


def test_bitwise_reproducible(lib):
    a = run_pair(lib, 2, nx=64, ny=64)[1]
    b = run_pair(lib, 2, nx=64, ny=64)[1]
    for (_, ga, _, _), (_, gb, _, _) in zip(a, b):
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k])


# ---------------------------------------------------------------- full size (512 x 512)
def test_full_size_512_residual_and_first_step(lib):
    """The bench mesh (512 x 512): step 1 at rtol 1e-12 matches the oracle's direct solve to
    1e-10; steps at the default rtol 1e-8 have oracle residual <= 1e-8."""
    N = 513 * 513
    pp, pn = inputs.initial_state(N, 0.33, 0.33, 0.01, seed=0)
    cp, op = make(lib, nx=512, ny=512, rtol=1e-12)
    system = lib.System(lib.Mesh(cp), cp)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.33, 0.01, seed=0)
    state.step()
    g = {k: v.cpu().numpy() for k, v in state.get().items()}
    s = o.Solver(op)
    ost = o.initial(N, pp, pn)
    ref = s.step(ost)
    for gk, ok in FIELDS:
        assert rel(g[gk], getattr(ref, ok)) < 1e-10, gk
    del state, system
    cp8, _ = make(lib, nx=512, ny=512)
    system = lib.System(lib.Mesh(cp8), cp8)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.33, 0.01, seed=0)
    prev = ost
    for _ in range(3):
        stats = state.step()
        g = {k: v.cpu().numpy() for k, v in state.get().items()}
        new = o.State(g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"])
        assert max(s.relres(prev, new)) <= 1e-8, stats
        prev = new
