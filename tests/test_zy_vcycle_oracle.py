"""The device V-cycle against the oracle's V-cycle (GPU).

ch_precond_level exports every level as the V-cycle uses it: the FP64 set-up matrices A_l and P_l,
the Chebyshev interval of D^-1 A_l and the smoothing degree; the coarsest level is solved exactly.
The oracle takes from the device only what a valid hierarchy may choose freely -- the fine matrix
(checked equal to the system's M or H), the prolongators P_l, the Chebyshev intervals and degrees --
and forms every coarse operator itself as the Galerkin product A_{l+1} = P_l^T A_l P_l
(`oracle.ch_oracle.galerkin_levels`).  The device's own coarse operators must equal those products
to 1e-13 of their largest entry (measured at most 1.8e-16),
and `oracle.ch_oracle.vcycle`, written from the definition of a V-cycle and pinned on the CPU, run on
the oracle's hierarchy must agree with ch_vcycle element by element:
  * FP64 V-cycles (precision 0) up to summation order: 1e-12 relative (measured on a GB300:
    at most 2.7e-16);
  * FP32 V-cycles (precision 1) up to FP32 rounding of the inputs, the operators and every
    intermediate vector: 2e-6 relative (unit roundoff 6e-8, amplified by the Chebyshev polynomials
    and the coarse corrections; measured at most 2.3e-7);
  * one cycle from a zero guess, and two cycles, the second continuing from the first's iterate.
The coarsest level is capped at 256 rows so that every mesh here has several levels in both
precisions (FP32 hierarchies otherwise stop at 2048 rows).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import ch_oracle as o

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6}
MESHES = [dict(nx=96, ny=96), dict(nx=70, ny=41, Lx=10.0, Ly=2.5), dict(dim=3, nx=16, ny=12, nz=10, Lz=0.5)]


def _csr(arrs, ncols):
    rowptr, col, val = [t.cpu().numpy() for t in arrs]
    return sp.csr_matrix((val, col, rowptr), shape=(len(rowptr) - 1, ncols))


def _exported(pc, which):
    nl = len(pc.levels(which))
    exported = [pc.level(which, l) for l in range(nl)]
    out = []
    for l, e in enumerate(exported):
        d = dict(A=_csr(e["A"], e["rows"]), bounds=e["bounds"], degree=e["degree"])
        if l + 1 < nl:
            d["P"] = _csr(e["P"], exported[l + 1]["rows"])
        else:
            assert e["P"] is None and e["degree"] == 0
        out.append(d)
    return out


def _oracle_levels(exported):
    """The oracle's hierarchy: the device's fine matrix and P_l, Galerkin products formed here."""
    fine = exported[0]["A"]
    Ps = [e["P"] for e in exported[:-1]]
    return o.galerkin_levels(fine, Ps, [e["bounds"] for e in exported[:-1]],
                             [e["degree"] for e in exported[:-1]])


def _setup(lib, kw, which, precision):
    p = lib.Params(precision=precision, coarse_max=256, **kw)
    system = lib.System(lib.Mesh(p), p)
    pc = lib.Precond(system)
    exported = _exported(pc, which)
    n = system.n
    assert exported[0]["A"].shape == (n, n) and len(exported) >= 2
    # the exported fine matrix is the system's M (which = 0) or H (which = 1)
    rowptr, col, vm, _, vh = [t.cpu().numpy() for t in system.csr()]
    ref = sp.csr_matrix((vm if which == 0 else vh, col, rowptr), shape=(n, n))
    assert abs(exported[0]["A"] - ref).max() == 0
    return pc, exported, _oracle_levels(exported), n


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", MESHES)
@pytest.mark.parametrize("which", [0, 1])
def test_coarse_operators_are_the_galerkin_products(lib, kw, which, precision):
    """A_{l+1} on the device = P_l^T A_l P_l formed by the oracle from A_0 and the P_l alone."""
    _, exported, levels, _ = _setup(lib, kw, which, precision)
    for l in range(1, len(levels)):
        dev, orc = exported[l]["A"], levels[l]["A"]
        assert dev.shape == orc.shape, l
        scale = abs(orc).max()
        err = abs(dev - orc).max() / scale
        print(f"galerkin which={which} precision={precision} {kw} level {l}: max |dA| / max |A| = {err:.2e}")
        assert err <= 1e-13, (l, err)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", MESHES)
@pytest.mark.parametrize("which", [0, 1])
def test_vcycle_equals_the_oracle_vcycle(lib, kw, which, precision):
    pc, _, levels, n = _setup(lib, kw, which, precision)
    rng = np.random.default_rng(17 + which)
    b = rng.standard_normal((n, 2))
    bd = torch.from_numpy(b).cuda()
    x1 = pc.vcycle(which, bd, 1).cpu().numpy()
    x2 = pc.vcycle(which, bd, 2).cpu().numpy()
    for k in range(2):
        want1 = o.vcycle(levels, b[:, k])
        want2 = o.vcycle(levels, b[:, k], x0=want1.copy())
        for got, want, cyc in ((x1[:, k], want1, 1), (x2[:, k], want2, 2)):
            err = np.abs(got - want).max() / np.abs(want).max()
            print(f"vcycle which={which} precision={precision} {kw} rhs {k} cycles {cyc}: rel err {err:.2e}")
            assert err <= TOL[precision], (which, k, cyc, err)
