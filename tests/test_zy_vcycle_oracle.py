"""The device V-cycle against the oracle's V-cycle on the device's own hierarchy (GPU).

ch_precond_level exports every level as the V-cycle uses it: the FP64 set-up matrices A_l and P_l,
the Chebyshev interval of D^-1 A_l and the smoothing degree; the coarsest level is solved exactly.
`oracle.ch_oracle.vcycle`, written from the definition of a V-cycle and pinned on the CPU, runs the
same cycle in numpy, so ch_vcycle (one V-cycle from a zero guess, two right-hand sides) must agree
element by element up to summation order.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import ch_oracle as o

pytestmark = pytest.mark.gpu


def _csr(arrs, ncols):
    rowptr, col, val = [t.cpu().numpy() for t in arrs]
    return sp.csr_matrix((val, col, rowptr), shape=(len(rowptr) - 1, ncols))


def _oracle_levels(pc, which):
    nl = len(pc.levels(which))
    exported = [pc.level(which, l) for l in range(nl)]
    levels = []
    for l, e in enumerate(exported):
        A = _csr(e["A"], e["rows"])
        if l + 1 < nl:
            P = _csr(e["P"], exported[l + 1]["rows"])
            levels.append(dict(A=A, P=P, bounds=e["bounds"], degree=e["degree"]))
        else:
            assert e["P"] is None and e["degree"] == 0
            levels.append(dict(A=A))
    return levels


@pytest.mark.parametrize("kw", [dict(nx=96, ny=96), dict(nx=70, ny=41, Lx=10.0, Ly=2.5),
                                dict(dim=3, nx=16, ny=12, nz=10, Lz=0.5)])
@pytest.mark.parametrize("which", [0, 1])
def test_vcycle_equals_the_oracle_vcycle(lib, kw, which):
    p = lib.Params(precision=0, **kw)
    system = lib.System(lib.Mesh(p), p)
    pc = lib.Precond(system)
    levels = _oracle_levels(pc, which)
    n = system.n
    assert levels[0]["A"].shape == (n, n) and len(levels) >= 2
    # the exported fine matrix is the system's M (which = 0) or H (which = 1)
    rowptr, col, vm, _, vh = [t.cpu().numpy() for t in system.csr()]
    ref = sp.csr_matrix((vm if which == 0 else vh, col, rowptr), shape=(n, n))
    assert abs(levels[0]["A"] - ref).max() == 0
    rng = np.random.default_rng(17 + which)
    b = rng.standard_normal((n, 2))
    x = pc.vcycle(which, torch.from_numpy(b).cuda(), 1).cpu().numpy()
    for k in range(2):
        want = o.vcycle(levels, b[:, k])
        assert np.abs(x[:, k] - want).max() <= 1e-9 * np.abs(want).max(), (which, k)
