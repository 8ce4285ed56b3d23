"""Contact forces (touch-sensor readout) on the CUDA path against the
oracle: a settled two-box stack and a box sliding down a ramp (closed forms
pinned on the oracle side), one step of the arm and hand workloads from
states the oracle reached, and the plain and batched paths bit-identical."""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import BOX, PLANE, body, pack
from scenegen import validation as V
from _parity import oracle_run, tie_free

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
G = 9.81


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _forces_after_one_step(sc, st64, plain=False):
    """GPU and oracle contact forces after one step from the same float32
    state."""
    from paper_2410_00425_b300 import Batch
    st = st64.astype(np.float32)
    o = oracle.Oracle(sc)
    o.set_state(st.astype(np.float64))
    o.step(1)
    b = Batch(sc)
    b.enable_contact_forces()
    s = torch.cuda.Stream()
    b.set_state(torch.from_numpy(st).cuda(), stream=s)
    b.step(None, 1, stream=s, plain=plain)
    f = b.contact_forces(stream=s)
    torch.cuda.synchronize()
    out = f.cpu().numpy().astype(np.float64)
    b.close()
    return out, o.contact_forces(), o


def test_stack_and_sliding_box_forces_match_the_oracle():
    m1, m2, h1, h2 = 0.2, 0.05, 0.03, 0.02
    stack = pack("stack2", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)),
                             body(BOX, (h1, h1, h1), m1, (0, 0, h1)),
                             body(BOX, (h2, h2, h2), m2, (0.005, -0.004, 2 * h1 + h2))]], [[]],
                 scenegen.default_params(pos_iters=64), 0, 0)
    g, r, _ = _forces_after_one_step(stack, oracle_run(stack, 100).state())
    np.testing.assert_allclose(g, r, rtol=0, atol=1e-3 * (m1 + m2) * G)
    np.testing.assert_allclose(g[1, :3], [0, 0, m1 * G], atol=1e-3 * m1 * G)
    th, mu, m = math.atan(0.6), 0.5, 0.1
    ramp = V.incline([th], mu=mu, mass=m)
    g, r, _ = _forces_after_one_step(ramp, oracle_run(ramp, 60).state())
    fn = m * G * math.cos(th)
    n = np.array([math.sin(th), 0.0, math.cos(th)])
    s_dir = np.array([math.cos(th), 0.0, -math.sin(th)])
    np.testing.assert_allclose(g, r, rtol=0, atol=1e-3 * fn)
    np.testing.assert_allclose(g[1, :3], fn * (n - mu * s_dir), atol=1e-3 * fn)


@pytest.mark.parametrize("name,settle", [("arm", 30), ("hand", 20)])
def test_workload_forces_match_the_oracle(name, settle):
    sc = scenegen.make_scene(name, n_envs=32)
    if sc.n_act:
        sc.action_fn = None
    g, r, o = _forces_after_one_step(sc, oracle_run(sc, settle).state())
    clean = tie_free(o, sc)
    off = sc.body_off
    scale = np.maximum(np.abs(r[:, :3]).max(1, keepdims=True), 1e-2)
    bad = []
    for e in np.nonzero(clean)[0]:
        sl = slice(off[e], off[e + 1])
        if not (np.abs(g[sl] - r[sl]) <= 2e-3 * scale[sl] + 1e-4).all():
            bad.append(int(e))
    assert clean.sum() >= 16
    assert not bad, (bad, np.abs(g - r).max(0))
    assert np.abs(r[:, 3]).max() > 0.1                       # contacts carried force


def test_plain_and_batched_forces_bit_identical():
    from paper_2410_00425_b300 import Batch
    sc = scenegen.make_scene("clutter", n_envs=24)
    outs = []
    for plain in (False, True):
        b = Batch(sc)
        b.enable_contact_forces()
        s = torch.cuda.Stream()
        for _ in range(20):
            b.step(None, 1, stream=s, plain=plain)
        f = b.contact_forces(stream=s)
        torch.cuda.synchronize()
        outs.append(f.cpu().numpy())
        b.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.abs(outs[0][:, 3]).max() > 0


def test_forces_off_is_an_error():
    from paper_2410_00425_b300 import Batch, MSError
    sc = scenegen.make_scene("small", n_envs=4)
    b = Batch(sc)
    with pytest.raises(MSError):
        b.contact_forces()
    b.enable_contact_forces()
    b.step(None, 1)
    f = b.contact_forces()
    torch.cuda.synchronize()
    b.enable_contact_forces(False)
    with pytest.raises(MSError):
        b.contact_forces()
    b.close()
