"""The device-memory hook (ms_set_allocator): a batch created under PyTorch's
caching allocator takes its memory from it, gives it back when destroyed,
and steps bit for bit like a batch on the library's own pool; a hook that
fails makes the creation fail with MS_ERR_OOM."""
import numpy as np
import pytest

import scenegen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _run(b, sc, s):
    a = torch.from_numpy(np.ascontiguousarray(sc.actions(0, 3))).cuda()
    b.step(a, 3, stream=s)
    torch.cuda.synchronize()
    return b.state().cpu()


def test_batch_memory_from_torch_allocator():
    from paper_2410_00425_b300 import Batch, use_torch_allocator
    sc = scenegen.make_scene("arm", n_envs=32)
    s = torch.cuda.Stream()
    ref = Batch(sc)
    want = _run(ref, sc, s)
    ref.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    use_torch_allocator(True)
    try:
        b = Batch(sc)
        held = torch.cuda.memory_allocated() - before
        assert held >= b.memory_bytes() > 0
        got = _run(b, sc, s)
        b.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        use_torch_allocator(False)
    assert torch.equal(want, got)


def test_failing_hook_makes_creation_fail():
    from paper_2410_00425_b300 import Batch, _ffi
    sc = scenegen.make_scene("small", n_envs=4)
    _ffi.ms_set_allocator(lambda n, d, st: 0, lambda p, d, st: None)
    try:
        with pytest.raises(_ffi.MSError):
            Batch(sc)
    finally:
        _ffi.ms_set_allocator(None, None)
    Batch(sc).close()                               # the library's pool again


def test_hook_needs_both_functions():
    import ctypes as C
    from paper_2410_00425_b300 import _ffi
    f = _ffi.ALLOC_FN(lambda n, d, st, u: None)
    assert _ffi.load().ms_set_allocator(C.cast(f, C.c_void_p), None, None) != 0
