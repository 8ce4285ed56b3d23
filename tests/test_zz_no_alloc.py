"""ms_step_noalloc against ms_step, through the C ABI.

ms_step_noalloc serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or an allocation's implicit
synchronisation is unacceptable in their loop): the caller owns every input
and output array and the kernel's workspace is a fixed array inside the
library.  Here the test plays that caller -- it owns the arrays (allocated
through torch) -- and checks that two calls in a row give the same states
as two ms_step calls on a batch built from the same descriptors, within the
tolerance the other GPU tests use (the two paths run the same stages, so
they are expected to agree bit for bit), and that envs whose descriptors
break a rule are skipped and marked.  The file is collected last so a
run that stops at the first failure has run every other test already.
"""
import ctypes as C
import dataclasses

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


def _caller_arrays(sc, init):
    """The caller's device arrays of a scene: CSR offsets, descriptors,
    float4 state from a [NB, 13] state, targets, status."""
    NB = int(sc.body_off[-1])

    def f4(cols):
        out = torch.zeros((NB, 4), dtype=torch.float32)
        out[:, :len(cols)] = init[:, cols]
        return out.cuda()
    arr = dict(bodies=_dev(sc.bodies), joints=_dev(sc.joints),
               body_off=torch.from_numpy(sc.body_off.astype(np.int32)).cuda(),
               joint_off=torch.from_numpy(sc.joint_off.astype(np.int32)).cuda(),
               x=f4([0, 1, 2]), q=f4([3, 4, 5, 6]), v=f4([7, 8, 9]), w=f4([10, 11, 12]),
               targets=torch.from_numpy(sc.joints["target0"].astype(np.float32)).cuda(),
               status=torch.zeros(sc.n_envs, dtype=torch.int32, device="cuda"))
    return arr


def _noalloc_batch(sc, arr, max_nb, max_nj):
    from paper_2410_00425_b300 import _ffi
    return _ffi.ms_noalloc_batch(sc.n_envs, max_nb, max_nj, arr["body_off"].data_ptr(), arr["joint_off"].data_ptr(),
                                 arr["bodies"].data_ptr(), arr["joints"].data_ptr() if len(sc.joints) else None,
                                 arr["x"].data_ptr(), arr["q"].data_ptr(), arr["v"].data_ptr(), arr["w"].data_ptr(),
                                 arr["targets"].data_ptr() if len(sc.joints) else None, arr["status"].data_ptr())


def _state(arr):
    return torch.cat([arr["x"][:, :3], arr["q"], arr["v"][:, :3], arr["w"][:, :3]], dim=1).cpu()


def _close(a, b):
    a = a.numpy().astype(np.float64)
    b = b.numpy().astype(np.float64)
    dx = np.abs(a[:, 0:3] - b[:, 0:3]).max()
    dq = np.abs(a[:, 3:7] - b[:, 3:7]).max()
    dv = np.abs(a[:, 7:13] - b[:, 7:13]).max()
    assert dx <= TOL_X and dq <= TOL_X and dv <= TOL_V, (dx, dq, dv)


# arm: capsules and boxes, up to 12 bodies; small: spheres; hand and clutter:
# more than 16 bodies per env, so 32-lane groups
@pytest.mark.parametrize("name,n_envs", [("arm", 48), ("small", 32), ("hand", 16), ("clutter", 24)])
def test_noalloc_matches_ms_step_on_two_calls(name, n_envs):
    from paper_2410_00425_b300 import Batch, _ffi

    sc = scenegen.make_scene(name, n_envs=n_envs)
    s = torch.cuda.Stream()
    n = 3
    a_np = sc.actions(0, 2 * n)
    acts = None if a_np is None else torch.from_numpy(a_np).cuda()

    # the existing entry point
    ref = Batch(sc)
    init = ref.state().cpu()                       # normalised quaternions, as created
    torch.cuda.synchronize()
    refs = []
    for k in range(2):
        ref.step(None if acts is None else acts[k * n:(k + 1) * n].contiguous(), n, stream=s)
        torch.cuda.synchronize()
        refs.append(ref.state().cpu())
    ref.close()

    # the same envs through caller-owned device arrays
    arr = _caller_arrays(sc, init)
    nb = _noalloc_batch(sc, arr, int(np.diff(sc.body_off).max()), int(np.diff(sc.joint_off).max()))
    torch.cuda.synchronize()
    for k, expect in enumerate(refs):
        a = None if acts is None else acts[k * n:(k + 1) * n].contiguous()
        if a is not None:
            a.record_stream(s)
        s.wait_stream(torch.cuda.current_stream())
        _ffi.ms_step_noalloc(nb, sc.params, a, n, s)
        s.synchronize()
        got = _state(arr)
        _close(got, expect)
        assert int(arr["status"].abs().sum().item()) == 0
    assert torch.equal(_state(arr), refs[1])        # same stages: bit for bit


def test_noalloc_skips_invalid_envs_and_keeps_the_bit():
    """Envs that break a descriptor rule, or exceed the declared body count,
    get MS_ENV_INVALID and are left untouched byte for byte, on this call
    and the next (the bit stays set); the other envs step as ms_step
    steps them."""
    from paper_2410_00425_b300 import Batch, _ffi

    sc = scenegen.make_scene("arm", n_envs=8)
    s = torch.cuda.Stream()
    n = 2
    acts = torch.from_numpy(sc.actions(0, 2 * n)).cuda()
    ref = Batch(sc)
    init = ref.state().cpu()
    torch.cuda.synchronize()
    for k in range(2):
        ref.step(acts[k * n:(k + 1) * n].contiguous(), n, stream=s)
    torch.cuda.synchronize()
    expect = ref.state().cpu()
    ref.close()

    bo, jo = sc.body_off, sc.joint_off
    bad = sc.bodies.copy()
    badj = sc.joints.copy()
    bad["type"][bo[0] + 2] = scenegen.HULL            # env 0: a hull, which this path has no library for
    badj["child"][jo[1] + 3] = 12                     # env 1: a joint naming a body past the env's 12
    bad["restitution"][bo[2] + 5] = 2.0               # env 2: restitution outside [0, 1]
    bad["p"][bo[6] + 3, 0] = 0.0                      # env 6: a capsule of radius 0
    bad["mass"][bo[4] + 3] = -1.0                     # env 4: a negative mass
    bsc = dataclasses.replace(sc, bodies=bad, joints=badj)
    arr = _caller_arrays(bsc, init)
    body_off = sc.body_off.astype(np.int32).copy()
    body_off[4] += 1                                  # env 3: 13 bodies (> 12 declared)
    arr["body_off"] = torch.from_numpy(body_off).cuda()
    nb = _noalloc_batch(bsc, arr, 12, int(np.diff(sc.joint_off).max()))
    before = _state(arr)
    t_before = arr["targets"].cpu()
    invalid = [0, 1, 2, 3, 4, 6]
    valid = [5, 7]
    for k in range(2):
        a = acts[k * n:(k + 1) * n].contiguous()
        a.record_stream(s)
        s.wait_stream(torch.cuda.current_stream())
        _ffi.ms_step_noalloc(nb, sc.params, a, n, s)
        s.synchronize()
        st = arr["status"].cpu().numpy()
        assert all(st[e] & 16 for e in invalid), st
        assert all(st[e] == 0 for e in valid), st
    got = _state(arr)
    t_got = arr["targets"].cpu()
    for e in invalid:
        lo, hi = int(body_off[e]), int(body_off[e + 1])
        assert torch.equal(got[lo:hi], before[lo:hi]), e
        assert torch.equal(t_got[jo[e]:jo[e + 1]], t_before[jo[e]:jo[e + 1]]), e
    for e in valid:
        assert torch.equal(got[bo[e]:bo[e + 1]], expect[bo[e]:bo[e + 1]]), e


def test_noalloc_rejects_bad_arguments():
    from paper_2410_00425_b300 import _ffi
    sc = scenegen.make_scene("small", n_envs=4)
    nb = _ffi.ms_noalloc_batch(4, 65, 0, None, None, None, None, None, None, None, None, None, None)
    with pytest.raises(_ffi.MSError) as ei:
        _ffi.ms_step_noalloc(nb, sc.params, None, 1, None)
    assert ei.value.code == 1 and "max_bodies_per_env" in str(ei.value)
