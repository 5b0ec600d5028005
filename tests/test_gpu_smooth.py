"""ch_smooth, the V-cycle's finest-level Chebyshev smoother on its own, against the oracle (GPU).

The oracle's `chebyshev_smooth` (written from the semi-iteration's definition and pinned on the
CPU) runs on the device's exported fine matrix and interval (coarse_max 256, so that the finest
level is smoothed, not solved); the device result must agree element
by element at the V-cycle parity tolerances (FP64 1e-12, FP32 2e-6 relative), for one and several
passes, both hierarchies, 2D and 3D.  The call captured in a CUDA graph and replayed gives bitwise
the result of the direct call, and bad arguments are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import ch_oracle as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6}
MESHES = [dict(nx=96, ny=96), dict(nx=70, ny=41, Lx=10.0, Ly=2.5), dict(dim=3, nx=16, ny=12, nz=10, Lz=0.5)]


def _setup(lib, kw, precision, coarse_max=256):
    p = lib.Params(precision=precision, coarse_max=coarse_max, **kw)
    system = lib.System(lib.Mesh(p), p)
    return system, lib.Precond(system)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", MESHES)
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("degree,passes", [(1, 1), (5, 1), (3, 3)])
def test_smooth_equals_the_oracle_smoother(lib, kw, which, precision, degree, passes):
    system, pc = _setup(lib, kw, precision)
    e = pc.level(which, 0)
    rowptr, col, val = [t.cpu().numpy() for t in e["A"]]
    A = sp.csr_matrix((val, col, rowptr), shape=(system.n, system.n))
    rng = np.random.default_rng(31 + degree + which)
    b = rng.standard_normal((system.n, 2))
    x0 = rng.standard_normal((system.n, 2))
    x = torch.from_numpy(x0.copy()).cuda()
    pc.smooth(which, torch.from_numpy(b).cuda(), x, degree, passes)
    got = x.cpu().numpy()
    for k in range(2):
        want = x0[:, k].copy()
        for _ in range(passes):
            want = o.chebyshev_smooth(A, b[:, k], want, degree, e["bounds"])
        err = np.abs(got[:, k] - want).max() / np.abs(want).max()
        assert err <= TOL[precision], (k, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_smooth_captured_in_a_graph_equals_the_direct_call(lib, precision):
    system, pc = _setup(lib, dict(nx=64, ny=48), precision)
    g = torch.Generator(device="cuda").manual_seed(4)
    b = torch.randn(system.n, 2, dtype=torch.float64, device="cuda", generator=g)
    x0 = torch.randn(system.n, 2, dtype=torch.float64, device="cuda", generator=g)
    direct = x0.clone()
    pc.smooth(1, b, direct, 5, 4)
    xg = x0.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            pc.smooth(1, b, xg, 5, 4, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    xg.copy_(x0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(xg, direct)


def test_smooth_rejects_bad_arguments(lib):
    system, pc = _setup(lib, dict(nx=16, ny=16), 0)
    b = torch.zeros(system.n, 2, dtype=torch.float64, device="cuda")
    x = torch.zeros(system.n, 2, dtype=torch.float64, device="cuda")
    for which, degree, passes in ((2, 3, 1), (1, 0, 1), (1, 17, 1), (0, 3, 0)):
        with pytest.raises(lib.ChError) as e:
            pc.smooth(which, b, x, degree, passes)
        assert e.value.status == lib.ERR_ARG
    with pytest.raises(lib.ChError) as e:
        pc.smooth(1, b, b, 3, 1)
    assert e.value.status == lib.ERR_ARG
    system, pc = _setup(lib, dict(nx=8, ny=8), 0, coarse_max=4096)  # one level: solved directly
    assert len(pc.levels(1)) == 1
    b = torch.zeros(system.n, 2, dtype=torch.float64, device="cuda")
    x = torch.zeros(system.n, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.ChError) as e:
        pc.smooth(1, b, x, 3, 1)
    assert e.value.status == lib.ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_smooth_on_a_batch_equals_the_oracle_smoother(lib, precision):
    """A batch of runs of different sizes: the finest level is the per-run lattice form (each row
    looks up its run's strides); the smoother of the disjoint union against the oracle's."""
    p = lib.Params(precision=precision, coarse_max=256)
    mesh = lib.Mesh(p, runs=[lib.Params(nx=40, ny=24), lib.Params(nx=17, ny=33), lib.Params(nx=64, ny=48)])
    system = lib.System(mesh, p)
    pc = lib.Precond(system)
    e = pc.level(1, 0)
    rowptr, col, val = [t.cpu().numpy() for t in e["A"]]
    A = sp.csr_matrix((val, col, rowptr), shape=(system.n, system.n))
    rng = np.random.default_rng(8)
    b = rng.standard_normal((system.n, 2))
    x0 = rng.standard_normal((system.n, 2))
    x = torch.from_numpy(x0.copy()).cuda()
    pc.smooth(1, torch.from_numpy(b).cuda(), x, 4, 2)
    got = x.cpu().numpy()
    for k in range(2):
        want = x0[:, k].copy()
        for _ in range(2):
            want = o.chebyshev_smooth(A, b[:, k], want, 4, e["bounds"])
        err = np.abs(got[:, k] - want).max() / np.abs(want).max()
        assert err <= TOL[precision], (k, err)
