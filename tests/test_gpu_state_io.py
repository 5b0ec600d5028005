"""Checkpoint / resume through the C ABI: a state saved after some steps and loaded into a fresh
state (same mesh) steps bitwise like the original; files for another mesh, foreign files,
truncated files and saving an unset state are refused."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def _solver(lib, nx, ny, **kw):
    p = lib.Params(nx=nx, ny=ny, **kw)
    system = lib.System(lib.Mesh(p), p)
    return lib.State(system, lib.Precond(system)), system


@pytest.mark.parametrize("precision", [0, 1])
def test_saved_state_resumes_bitwise(lib, tmp_path, precision):
    a, _ = _solver(lib, 40, 28, precision=precision)
    a.init_seeded(0.33, 0.30, 0.01, seed=11)
    for _ in range(3):
        a.step()
    path = tmp_path / "state.chs"
    a.save(path)
    b, _ = _solver(lib, 40, 28, precision=precision)
    b.load(path)
    assert torch.equal(a.state4(), b.state4())
    for _ in range(2):
        sa, sb = a.step(), b.step()
        assert sa["iters"] == sb["iters"]
    assert torch.equal(a.state4(), b.state4())


def test_load_refuses_other_meshes_and_bad_files(lib, tmp_path):
    a, _ = _solver(lib, 16, 16)
    with pytest.raises(lib.ChError):
        a.save(tmp_path / "unset.chs")  # nothing set yet
    a.init_seeded(0.33, 0.30, 0.01, seed=1)
    path = tmp_path / "a.chs"
    a.save(path)
    other, _ = _solver(lib, 16, 17)
    with pytest.raises(lib.ChError):
        other.load(path)
    junk = tmp_path / "junk.chs"
    junk.write_bytes(b"not a state file at all" * 10)
    with pytest.raises(lib.ChError):
        a.load(junk)
    cut = tmp_path / "cut.chs"
    cut.write_bytes(path.read_bytes()[:100])
    with pytest.raises(lib.ChError):
        a.load(cut)
    with pytest.raises(lib.ChError):
        a.load(tmp_path / "missing.chs")
    # the refused loads left the state as it was
    b, _ = _solver(lib, 16, 16)
    b.load(path)
    assert torch.equal(a.state4(), b.state4())
