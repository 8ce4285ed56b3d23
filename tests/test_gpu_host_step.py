"""ms_step_host: host actions in, host state or task records out, through one
C-ABI call -- the same results, bit for bit, as ms_step with device buffers
followed by ms_copy_state (or ms_step_ex's records)."""
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


@pytest.mark.parametrize("name", ["arm", "small"])
def test_host_step_equals_device_step(name):
    from paper_2410_00425_b300 import Batch
    sc = scenegen.make_scene(name, n_envs=24)
    s = torch.cuda.Stream()
    a = sc.actions(0, 6)
    ref = Batch(sc)
    dev = Batch(sc)
    h_state = torch.empty((ref.NB, 13), dtype=torch.float32).pin_memory()
    for k in range(3):
        ak = None if a is None else a[2 * k:2 * k + 2]
        ref.step(None if ak is None else torch.from_numpy(np.ascontiguousarray(ak)).cuda(), 2, stream=s)
        dev.step_host(None if ak is None else torch.from_numpy(np.ascontiguousarray(ak)).pin_memory(), 2, h_state,
                      stream=s)
        s.synchronize()
        assert torch.equal(ref.state().cpu(), h_state)
    ref.close()
    dev.close()


def test_host_step_records_equal_device_records():
    from paper_2410_00425_b300 import Batch
    sc = scenegen.make_scene("pick", n_envs=16)
    s = torch.cuda.Stream()
    a = np.ascontiguousarray(sc.actions(0, 3))
    ref = Batch(sc)
    ref.set_task(sc.task, stream=s)
    dev = Batch(sc)
    dev.set_task(sc.task, stream=s)
    rec = torch.full((3, ref.E, ref.record_len()), float("nan"), dtype=torch.float32, device="cuda")
    ref.step(torch.from_numpy(a).cuda(), 3, stream=s, out=rec)
    h_rec = torch.empty((3, dev.E, dev.record_len()), dtype=torch.float32).pin_memory()
    dev.step_host(torch.from_numpy(a).pin_memory(), 3, h_rec, records=True, stream=s)
    s.synchronize()
    assert torch.equal(rec.cpu(), h_rec)
    ref.close()
    dev.close()


def test_host_step_rejects_bad_arguments():
    from paper_2410_00425_b300 import Batch, _ffi
    sc = scenegen.make_scene("small", n_envs=4)
    b = Batch(sc)
    out = np.empty((b.NB, 13), np.float32)
    with pytest.raises(_ffi.MSError):
        _ffi.ms_step_host(b.h, None, 1, None, 0, None)          # no output buffer
    with pytest.raises(_ffi.MSError):
        _ffi.ms_step_host(b.h, None, 1, out, 2, None)           # unknown out_kind
    with pytest.raises(_ffi.MSError):
        _ffi.ms_step_host(b.h, None, 1, out, 1, None)           # records without a task
    b.close()
