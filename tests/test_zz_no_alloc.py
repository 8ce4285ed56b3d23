"""ms_step_noalloc against ms_step, through the C ABI.

ms_step_noalloc serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or an allocation's implicit
synchronisation is unacceptable in their loop): the caller owns every input
and output array and the kernel's workspace is a fixed array inside the
library.  Here the test plays that caller -- it owns the arrays (allocated
through torch) -- and checks that two calls in a row give the same states
as two ms_step calls on a batch built from the same descriptors, within the
tolerance the other GPU tests use (the two paths run the same stages, so
they are expected to agree bit for bit).  The file is collected last so a
run that stops at the first failure has run every other test already.
"""
import ctypes as C

import numpy as np
import pytest

import scenegen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X, TOL_V = 1e-5, 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _dev(arr):
    """Copy a numpy array (any dtype) to a caller-owned device buffer."""
    raw = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    return torch.from_numpy(raw.copy()).cuda()


def test_noalloc_matches_ms_step_on_two_calls():
    from paper_2410_00425_b300 import Batch, _ffi

    sc = scenegen.make_scene("arm", n_envs=48)
    s = torch.cuda.Stream()
    n = 3
    acts = torch.from_numpy(sc.actions(0, 2 * n)).cuda()

    # the existing entry point
    ref = Batch(sc)
    init = ref.state().cpu()                       # normalised quaternions, as created
    torch.cuda.synchronize()
    ref.step(acts[:n].contiguous(), n, stream=s)
    torch.cuda.synchronize()
    ref1 = ref.state().cpu()
    ref.step(acts[n:].contiguous(), n, stream=s)
    torch.cuda.synchronize()
    ref2 = ref.state().cpu()
    ref.close()

    # the same envs through caller-owned device arrays
    NB = int(sc.body_off[-1])
    nb_per = np.diff(sc.body_off)
    nj_per = np.diff(sc.joint_off)
    bodies = _dev(sc.bodies)
    joints = _dev(sc.joints)
    body_off = torch.from_numpy(sc.body_off.astype(np.int32)).cuda()
    joint_off = torch.from_numpy(sc.joint_off.astype(np.int32)).cuda()

    def f4(cols):
        out = torch.zeros((NB, 4), dtype=torch.float32)
        out[:, :len(cols)] = init[:, cols]
        return out.cuda()
    x, q, v, w = f4([0, 1, 2]), f4([3, 4, 5, 6]), f4([7, 8, 9]), f4([10, 11, 12])
    targets = torch.from_numpy(sc.joints["target0"].astype(np.float32)).cuda()
    status = torch.zeros(sc.n_envs, dtype=torch.int32, device="cuda")
    nb = _ffi.ms_noalloc_batch(sc.n_envs, int(nb_per.max()), int(nj_per.max()),
                               body_off.data_ptr(), joint_off.data_ptr(), bodies.data_ptr(),
                               joints.data_ptr(), x.data_ptr(), q.data_ptr(), v.data_ptr(), w.data_ptr(),
                               targets.data_ptr(), status.data_ptr())
    torch.cuda.synchronize()

    def state():
        return torch.cat([x[:, :3], q, v[:, :3], w[:, :3]], dim=1).cpu()

    def close(a, b):
        a = a.numpy().astype(np.float64)
        b = b.numpy().astype(np.float64)
        dx = np.abs(a[:, 0:3] - b[:, 0:3]).max()
        dq = np.abs(a[:, 3:7] - b[:, 3:7]).max()
        dv = np.abs(a[:, 7:13] - b[:, 7:13]).max()
        assert dx <= TOL_X and dq <= TOL_X and dv <= TOL_V, (dx, dq, dv)

    for k, expect in enumerate([ref1, ref2]):
        a = acts[k * n:(k + 1) * n].contiguous()
        a.record_stream(s)
        s.wait_stream(torch.cuda.current_stream())
        _ffi.ms_step_noalloc(nb, sc.params, a, n, s)
        s.synchronize()
        got = state()
        close(got, expect)
        assert int(status.abs().sum().item()) == 0
    assert torch.equal(state(), ref2)              # same stages: bit for bit


def test_noalloc_rejects_bad_arguments():
    from paper_2410_00425_b300 import _ffi
    sc = scenegen.make_scene("small", n_envs=4)
    nb = _ffi.ms_noalloc_batch(4, 65, 0, None, None, None, None, None, None, None, None, None, None)
    with pytest.raises(_ffi.MSError) as ei:
        _ffi.ms_step_noalloc(nb, sc.params, None, 1, None)
    assert ei.value.code == 1 and "max_bodies_per_env" in str(ei.value)
