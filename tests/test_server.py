"""Step server through its C ABI (include/ms_server.h): merged launches give
each session exactly the result of stepping it alone, admission respects the
HBM budget, and the latency record is consistent."""
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


def _alone(scene, steps):
    from paper_2410_00425_b300 import Batch
    b = Batch(scene)
    s = torch.cuda.Stream()
    for k in range(steps):
        a = scene.actions(k, 1)
        b.step(None if a is None else torch.from_numpy(a).cuda(), 1, stream=s)
    torch.cuda.synchronize()
    st = b.state().cpu().numpy()
    b.close()
    return st


@pytest.mark.parametrize("merge,inflight", [(True, 1), (True, 4), (False, 1), (False, 3)])
def test_sessions_of_mixed_types_match_stepping_alone(merge, inflight):
    from paper_2410_00425_b300.server import Server
    warm = scenegen.make_scene("arm", n_envs=6)         # a session with the solver variants on
    warm.params = dict(warm.params, linear_damping=0.5, angular_damping=0.3, bounce_threshold=0.5, warm_start=1)
    warm.bodies = warm.bodies.copy()
    warm.bodies["restitution"] = 0.4
    scenes = [scenegen.make_scene("arm", n_envs=8), scenegen.make_scene("clutter", n_envs=16),
              scenegen.make_scene("hand", n_envs=4), scenegen.make_scene("small", n_envs=3), warm]
    srv = Server(8 << 30, merge=merge, max_inflight=inflight)
    sids = [srv.open(sc) for sc in scenes]
    assert all(s is not None for s in sids)
    steps = 4
    tickets = []
    for k in range(steps):
        for sc, sid in zip(scenes, sids):
            a = sc.actions(k, 1)
            tickets.append(srv.submit(sid, None if a is None else a[0]))
    srv.drain()
    res = [srv.poll(t) for t in tickets]
    assert all(r is not None and r["status"] == 0 for r in res)
    assert all(r["latency"] >= 0 and r["t_done"] >= r["t_arrive"] for r in res)
    st = srv.stats()
    assert st["requests_done"] == len(tickets)
    if merge:
        assert st["launches"] <= len(tickets)
        assert st["launches"] >= steps          # one request per session per launch
        assert st["graph_captures"] >= 1
    else:
        assert st["launches"] == len(tickets)
    assert 0 <= st["p50"] <= st["p99"]
    for sc, sid in zip(scenes, sids):
        got = srv.state(sid, int(sc.body_off[-1]))
        np.testing.assert_array_equal(got, _alone(sc, steps))
    srv.close()


def test_admission_against_budget():
    from paper_2410_00425_b300.server import Server
    sc = scenegen.make_scene("clutter", n_envs=64)
    one = scenegen.make_scene("clutter", n_envs=2)
    from paper_2410_00425_b300 import _ffi
    need = _ffi.ms_estimate_bytes(sc.body_off, sc.joint_off, sc.params)
    srv = Server(int(need * 1.5))
    a = srv.open(sc)
    b = srv.open(sc)                             # would exceed the budget
    assert a is not None and b is None
    assert srv.stats()["sessions_rejected"] == 1
    srv.close_session(a)
    c = srv.open(sc)                             # memory came back
    assert c is not None
    assert srv.open(one) is not None
    srv.close()


def test_session_close_waits_for_pending_and_frees_budget():
    from paper_2410_00425_b300.server import Server
    sc = scenegen.make_scene("arm", n_envs=16)
    srv = Server(4 << 30)
    sid = srv.open(sc)
    used = srv.stats()["hbm_used"]
    assert used > 0
    for k in range(5):
        srv.submit(sid, sc.actions(k, 1)[0])
    srv.close_session(sid)
    assert srv.stats()["hbm_used"] == 0
    assert srv.stats()["requests_done"] == 5
    srv.close()
