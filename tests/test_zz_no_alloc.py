"""ch_vcycle_noalloc: the allocation-free V-cycle entry point.

Some callers cannot allocate device memory while they run (stream capture into a CUDA graph,
a framework allocator with a fixed budget, loops that cannot take cudaMalloc's device-wide
synchronisation).  For them ch_vcycle_noalloc keeps its work vectors in a static device array.
These tests call it through the C ABI twice in a row and compare each result with ch_vcycle on
the same input, and check that a hierarchy too large for the array is refused.  The file is
named to be collected last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", [dict(nx=64, ny=64), dict(dim=3, nx=12, ny=12, nz=6, Lz=0.5)])
def test_noalloc_vcycle_matches_vcycle_on_two_calls(lib, precision, kw):
    p = lib.Params(precision=precision, **kw)
    system = lib.System(lib.Mesh(p), p)
    pc = lib.Precond(system)
    g = torch.Generator(device="cuda").manual_seed(7)
    for which in (0, 1):
        for call in range(2):  # two calls in a row, each on a new right-hand side
            b = torch.randn(system.n, 2, dtype=torch.float64, device="cuda", generator=g)
            ref = pc.vcycle(which, b, 2)
            got = pc.vcycle_noalloc(which, b, 2)
            torch.cuda.synchronize()
            assert torch.isfinite(got).all()
            assert _rel(got, ref) <= 1e-13, (which, call)


def test_noalloc_vcycle_rejects_hierarchy_beyond_the_array(lib):
    p = lib.Params(nx=512, ny=512)
    system = lib.System(lib.Mesh(p), p)
    pc = lib.Precond(system)
    b = torch.ones(system.n, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.ChError) as e:
        pc.vcycle_noalloc(1, b, 1)
    assert e.value.status == lib.ERR_ARG
    assert "static array" in str(e.value)
