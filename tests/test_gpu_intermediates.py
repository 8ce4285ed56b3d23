"""Intermediate results of the step compared directly with the oracle's, on
the same float32 state on both sides: the greedy constraint colouring
(integers, exact) and every contact manifold -- its pair, point count, and
each point's witness points, normal and separation.

The state is the initial one, or one the oracle reached after some steps
(objects landed and in contact), rounded to float32 and given to both
sides.  Envs with a tie-adjacent decision in the compared step are counted
and left out; a wrong colour or a manifold point off by more than the
position bar anywhere else fails."""
import numpy as np
import pytest

import oracle
import scenegen

from _parity import TOL_X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


CASES = [("small", 64, 0), ("small", 64, 80), ("arm", 64, 0), ("arm", 64, 60), ("clutter", 128, 0),
         ("clutter", 128, 60), ("hand", 48, 0), ("hand", 48, 30), ("mixed", 60, 0), ("mixed", 60, 40),
         ("hulls", 64, 40), ("hulls", 64, 80)]


def _start_state(sc, pre):
    o = oracle.Oracle(sc)
    if pre:
        o.step(pre, actions=sc.actions(0, pre), threads=8)
    return o.state().astype(np.float32)


@pytest.mark.parametrize("name,n,pre", CASES)
def test_colours_and_manifolds_equal_the_oracle(name, n, pre):
    from paper_2410_00425_b300 import Batch
    sc = scenegen.make_scene(name, n_envs=n)
    st = _start_state(sc, pre)
    a = sc.actions(pre, 1)
    # the oracle: one step from the float32 state
    o = oracle.Oracle(sc)
    o.set_state(st.astype(np.float64))
    o.step(1, actions=a, threads=8)
    # the CUDA path: the same state, the same step
    b = Batch(sc, record_contacts=True)
    s = torch.cuda.Stream()
    b.set_state(torch.from_numpy(st).contiguous(), stream=s)
    b.step(None if a is None else torch.from_numpy(a).cuda(), 1, stream=s)
    torch.cuda.synchronize()
    compared = tied = n_man = n_pts = 0
    worst = 0.0
    for e in range(sc.n_envs):
        if o.ties(e):
            tied += 1
            continue
        compared += 1
        gp, gn, gx = b.contacts(e)
        op, on, ox = o.manifolds(e)
        assert np.array_equal(gp, op), (e, gp.tolist(), op.tolist())
        assert np.array_equal(gn, on), (e, gn.tolist(), on.tolist())
        for m in range(len(op)):
            k = on[m]
            d = np.abs(gx[m, :k].astype(np.float64) - ox[m, :k])
            worst = max(worst, d.max())
            assert d.max() <= TOL_X, (e, m, d.max(0))
            n_pts += k
        n_man += len(op)
        gc, oc = b.colors(e), o.colors(e)
        assert np.array_equal(gc, oc), (e, gc.tolist(), oc.tolist())
    print(f"{name} from step {pre}: {compared} envs compared ({tied} tie-adjacent), {n_man} manifolds, "
          f"{n_pts} points, worst point difference {worst:.2e}")
    assert compared >= 0.6 * sc.n_envs
    assert n_man > 0
