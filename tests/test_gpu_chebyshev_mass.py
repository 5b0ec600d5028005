"""M~ by the Chebyshev semi-iteration on the device (precond_M = 1; Section 3 names it as the
alternative to AMG for the mass matrix) against the oracle (GPU).

ch_mass_solve applies Algorithm 1's step 1 alone.  With precond_M = 1 it runs cheb_M_steps steps of
the semi-iteration on D^-1 M from a zero guess over Wathen's eigenvalue bounds ([1/2, 2] for
triangles, [1/2, 5/2] for tetrahedra); `oracle.ch_oracle.chebyshev_semi_iteration`, pinned on the
CPU to its definition through T_k, runs the same iteration on the oracle's own M.  Tolerances as for
the V-cycles: FP64 1e-12 (summation order), FP32 2e-6 (FP32 rounding of inputs, M and the vectors;
the polynomial is bounded by 1 on the interval, so the amplification is small).  Steps with the
semi-iteration converge to the oracle's step like steps with AMG (the preconditioner changes only
the iteration counts), in FGMRES and in MINRES (a fixed number of steps is a fixed symmetric
positive definite operator).
"""
import numpy as np
import pytest
import torch

from oracle import ch_oracle as o
from paper_2204_03575_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6}
MESHES = [dict(nx=48, ny=40), dict(nx=37, ny=23, Lx=10.0, Ly=2.5), dict(dim=3, nx=12, ny=10, nz=6, Lz=0.5)]


def _oparams(kw):
    return o.Params(**{k: v for k, v in kw.items() if k in o.Params.__dataclass_fields__})


@pytest.mark.parametrize("steps", [1, 3, 5, 9])
@pytest.mark.parametrize("kw", MESHES)
@pytest.mark.parametrize("precision", [0, 1])
def test_semi_iteration_equals_the_oracle(lib, kw, precision, steps):
    p = lib.Params(precision=precision, precond_M=1, cheb_M_steps=steps, **kw)
    system = lib.System(lib.Mesh(p), p)
    pc = lib.Precond(system)
    M, _ = o.assemble(o.mesh(_oparams(kw)))
    rng = np.random.default_rng(steps)
    b = rng.standard_normal((system.n, 2))
    x = pc.mass_solve(torch.from_numpy(b).cuda()).cpu().numpy()
    want = o.chebyshev_semi_iteration(M, b, steps, dim=kw.get("dim", 2))
    err = np.abs(x - want).max() / np.abs(want).max()
    assert err <= TOL[precision], err


@pytest.mark.parametrize("precision", [0, 1])
def test_mass_solve_amg_mode_is_the_m_vcycles(lib, precision):
    """precond_M = 0: ch_mass_solve is the vcycles_M V-cycles of M's hierarchy (ch_vcycle)."""
    p = lib.Params(nx=64, ny=48, precision=precision, vcycles_M=2)
    system = lib.System(lib.Mesh(p), p)
    pc = lib.Precond(system)
    b = torch.randn(system.n, 2, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    np.testing.assert_array_equal(pc.mass_solve(b).cpu().numpy(), pc.vcycle(0, b, 2).cpu().numpy())


@pytest.mark.parametrize("krylov", [0, 1])
@pytest.mark.parametrize("kw", [dict(nx=32, ny=32), dict(dim=3, nx=16, ny=16, nz=4, Lz=0.25)])
def test_steps_with_the_semi_iteration_match_the_oracle(lib, kw, krylov):
    p = lib.Params(precond_M=1, rtol=1e-13, max_iter=1000, krylov=krylov, **kw)
    system = lib.System(lib.Mesh(p), p)
    state = lib.State(system, lib.Precond(system))
    s = o.Solver(_oparams(kw))
    pp, pn = inputs.initial_state(s.N, 0.33, 0.31, 0.01, seed=6)
    state.set(torch.from_numpy(pp).cuda(), torch.from_numpy(pn).cuda())
    prev = o.initial(s.N, pp, pn)
    for _ in range(2):
        st = state.step()
        assert st["status"] == 0
        g = {k: v.cpu().numpy() for k, v in state.get().items()}
        ref = s.step(prev)
        for k in ("phi_p", "phi_nfa", "mu_p", "mu_nfa"):
            r = getattr(ref, k)
            assert np.abs(g[k] - r).max() <= 1e-10 * np.abs(r).max(), k
        prev = o.State(g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"])


@pytest.mark.parametrize("precision", [0, 1])
def test_semi_iteration_at_the_default_tolerance(lib, precision):
    """128 x 96 at rtol 1e-8 in both precisions: every step reaches the true 1e-8 residual."""
    p = lib.Params(nx=128, ny=96, precond_M=1, precision=precision)
    system = lib.System(lib.Mesh(p), p)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.31, 0.01, seed=2)
    for _ in range(3):
        st = state.step()
        assert st["status"] == 0 and max(st["relres"]) <= 1e-8
