"""The morphology-to-grid projection of Section 5 on the device, bit-exact against the oracle (GPU).

The parity of the object faces an upward ray from a grid point crosses (the paper's method)
telescopes to the value of the image pixel holding the point; ch_morphology_project reads that
pixel, locating it by an exact integer quotient except at ties, and `oracle.morphology_oracle`
computes the same plain definition in numpy (pinned on the CPU to a brute-force crossing count).  Classes are compared bit for bit, mobilities exactly, on random
morphologies (grids finer and coarser than the image, boxes of both orientations), a disk, the
explicit threshold, a morphology from the solver itself, and the smallest sizes.
"""
import numpy as np
import pytest
import torch

from oracle import morphology_oracle as mo

pytestmark = pytest.mark.gpu


def _run(lib, pp, pn, nx, ny, Lx, Ly, gx, gy, threshold=None):
    got = lib.morphology_project(torch.from_numpy(pp).cuda(), None if pn is None else torch.from_numpy(pn).cuda(),
                                 nx, ny, Lx, Ly, gx, gy, threshold=threshold)
    polymer, mu_e, mu_h = [t.cpu().numpy() for t in got]
    ref = mo.project(pp, pn, nx, ny, Lx, Ly, gx, gy, threshold)
    np.testing.assert_array_equal(polymer.astype(bool), ref[0])
    np.testing.assert_array_equal(mu_e, ref[1])
    np.testing.assert_array_equal(mu_h, ref[2])
    return polymer.astype(bool)


@pytest.mark.parametrize("nx,ny,Lx,Ly,gx,gy", [(12, 7, 10.0, 2.5, 31, 17), (64, 32, 10.0, 2.5, 97, 45),
                                                (40, 40, 1.0, 1.0, 13, 11), (33, 80, 2.0, 5.0, 200, 301),
                                                (255, 255, 1.0, 1.0, 1000, 1000),
                                                # grids that are multiples of the image: every
                                                # point's pixel coordinate is an exact tie
                                                (16, 8, 1.0, 1.0, 16, 8), (20, 10, 3.0, 0.7, 60, 30),
                                                (7, 9, 2.5, 10.0, 21, 27)])
def test_projection_equals_the_oracle(lib, nx, ny, Lx, Ly, gx, gy):
    rng = np.random.default_rng(nx * 1000 + gx)
    N = (nx + 1) * (ny + 1)
    pp, pn = rng.random(N), rng.random(N)
    polymer = _run(lib, pp, pn, nx, ny, Lx, Ly, gx, gy)
    assert 0 < polymer.sum() < polymer.size


def test_disk_and_threshold(lib):
    nx, ny, Lx, Ly = 80, 40, 4.0, 2.0
    x = np.tile(np.arange(nx + 1) * (Lx / nx), ny + 1)
    y = np.repeat(np.arange(ny + 1) * (Ly / ny), nx + 1)
    pp = np.where(np.hypot(x - 2.0, y - 1.0) < 0.8, 0.9, 0.1)
    _run(lib, pp, 1.0 - pp, nx, ny, Lx, Ly, 97, 51)
    _run(lib, pp, None, nx, ny, Lx, Ly, 97, 51, threshold=0.5)
    rng = np.random.default_rng(4)
    q = rng.random((nx + 1) * (ny + 1))
    _run(lib, q, None, nx, ny, Lx, Ly, 61, 77, threshold=0.3)


def test_smallest_sizes_and_uniform_images(lib):
    _run(lib, np.array([0.6, 0.1, 0.2, 0.7]), np.array([0.2, 0.5, 0.5, 0.1]), 1, 1, 1.0, 1.0, 1, 1)
    _run(lib, np.array([0.6, 0.1, 0.2, 0.7]), np.array([0.2, 0.5, 0.5, 0.1]), 1, 1, 1.0, 1.0, 5, 3)
    N = 11 * 6
    _run(lib, np.ones(N), np.zeros(N), 10, 5, 3.0, 1.0, 17, 9)      # all polymer
    _run(lib, np.zeros(N), np.ones(N), 10, 5, 3.0, 1.0, 17, 9)      # none


def test_tall_image_agrees(lib):
    """A tall, narrow image (24001 pixel rows) on a coarse grid, and a grid of one column and
    600,000 rows (more row blocks than a grid's second dimension could hold)."""
    nx, ny = 2, 24000
    rng = np.random.default_rng(9)
    N = (nx + 1) * (ny + 1)
    pp, pn = rng.random(N), rng.random(N)
    _run(lib, pp, pn, nx, ny, 1.0, 100.0, 5, 301)
    _run(lib, pp, pn, nx, ny, 1.0, 100.0, 1, 600000)


def test_projection_of_a_solver_morphology(lib):
    """The projection of a state the solver produced (64 x 48 box, 20 steps)."""
    p = lib.Params(nx=64, ny=48, Lx=4.0, Ly=3.0)
    system = lib.System(lib.Mesh(p), p)
    state = lib.State(system, lib.Precond(system))
    state.init_seeded(0.33, 0.33, 0.01, seed=5)
    for _ in range(20):
        state.step()
    g = state.get()
    _run(lib, g["phi_p"].cpu().numpy(), g["phi_nfa"].cpu().numpy(), 64, 48, 4.0, 3.0, 150, 101)


def test_projection_rejects_bad_arguments(lib):
    pp = torch.zeros(4, dtype=torch.float64, device="cuda")
    good = dict(nx=1, ny=1, Lx=1.0, Ly=1.0, gx=2, gy=2)
    for bad in (dict(gx=0), dict(gy=-1), dict(Lx=-1.0), dict(Ly=0.0)):
        kw = {**good, **bad}
        with pytest.raises(lib.ChError) as e:
            lib.morphology_project(pp, pp, kw["nx"], kw["ny"], kw["Lx"], kw["Ly"], max(kw["gx"], 0),
                                   max(kw["gy"], 0))
        assert e.value.status == lib.ERR_ARG
