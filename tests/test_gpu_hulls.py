"""Convex hulls on the CUDA path against the oracle: contact pair sets and
one step from states the oracle settled to, rollouts of non-chaotic envs,
the box-as-hull equivalence, rendering of hull meshes, and the bit-identity
of the plain and batched paths and of launch shapes.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import BOX, HULL, PLANE, SPHERE, body, pack
from scenegen import hulls as H
from _parity import env_errors, gpu_run, non_chaotic, oracle_run, pair_sets_match, tie_free, within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _one_step_from(sc, st64):
    """One step on both sides from the same float32 state."""
    from paper_2410_00425_b300 import Batch
    st = st64.astype(np.float32)
    o = oracle.Oracle(sc)
    o.set_state(st.astype(np.float64))
    o.step(1)
    b = Batch(sc, record_contacts=True)
    s = torch.cuda.Stream()
    b.set_state(torch.from_numpy(st).cuda(), stream=s)
    b.step(None, 1, stream=s)
    torch.cuda.synchronize()
    g = b.state().cpu().numpy().astype(np.float64)
    code, status = b.sync()
    return b, o, g, status


@pytest.mark.parametrize("settle", [40, 80])
def test_one_step_from_settled_states(settle):
    sc = scenegen.make_scene("hulls", n_envs=64)
    st = oracle_run(sc, settle).state()
    b, o, g, status = _one_step_from(sc, st)
    assert sum(len(o.manifolds(e)[0]) for e in range(sc.n_envs)) > 100      # hulls in contact
    bad = pair_sets_match(b, o, sc)
    clean = tie_free(o, sc)
    assert not [e for e in bad if clean[e]], bad
    err = env_errors(sc, g, o.state())
    # resting hull contacts sit on clipping and face-choice thresholds often
    assert clean.mean() >= 0.3
    ok = within(err)
    assert ok[clean].all(), (np.nonzero(clean & ~ok)[0].tolist(), err[clean].max(0))
    assert not status.any()


def test_rollout_non_chaotic():
    sc = scenegen.make_scene("hulls", n_envs=128)
    calm, ost = non_chaotic(sc, 100)
    o = oracle_run(sc, 100)
    _, st, _ = gpu_run(sc, 100)
    clean = calm & tie_free(o, sc)
    print(f"hulls: {clean.sum()} of 128 envs non-chaotic and tie-free")
    assert clean.sum() >= 3
    err = env_errors(sc, st, ost)
    ok = within(err, 10.0)
    assert ok[clean].all(), (np.nonzero(clean & ~ok)[0].tolist(), err[clean].max(0))


def test_plain_path_and_launch_shapes_bit_identical():
    sc = scenegen.make_scene("hulls", n_envs=40)
    _, a, _ = gpu_run(sc, 30)
    _, b, _ = gpu_run(sc, 30, plain=True)
    assert np.array_equal(a, b)
    for tuning in [(4, 2, 0), (32, 1, 1)]:
        _, c, _ = gpu_run(sc, 30, tuning=tuning)
        assert np.array_equal(a, c), tuning


def test_spheres_on_a_hull_follow_the_oracle():
    """Sphere - hull contacts: spheres dropped onto a static random hull and
    onto a box-shaped one.  A rollout to 60 steps (just after landing:
    a sphere rolling down a hull gathers orientation phase as in the
    primitive scenes), and one step from the state the oracle reaches at
    120 steps."""
    g = np.random.default_rng(5)
    assets = [H.hull_asset(H.random_points(g, 12, np.array([0.06, 0.05, 0.04]))), H.box_asset(0.05, 0.05, 0.02)]
    envs = []
    for k in range(8):
        hk = k % 2
        envs.append([body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)),
                     body(HULL, (hk, 0, 0), 0.0, (0, 0, 0.08)),
                     body(SPHERE, (0.01, 0, 0), 0.02, (0.01 * (k - 4) * 0.5, 0.004 * k, 0.2))])
    sc = pack("sphere_hull", envs, [[] for _ in envs], scenegen.default_params(), 0, 0)
    sc.hulls = H.library(assets)
    calm, ost = non_chaotic(sc, 60)
    o = oracle_run(sc, 60)
    b, st, _ = gpu_run(sc, 60, record=True)
    assert sum(len(o.manifolds(e)[0]) for e in range(8)) >= 4             # on the hulls
    clean = calm & tie_free(o, sc)
    assert clean.sum() >= 4
    err = env_errors(sc, st, ost)
    assert within(err, 10.0)[clean].all(), err[clean].max(0)
    b2, o2, g2, _ = _one_step_from(sc, oracle_run(sc, 120).state())
    clean2 = tie_free(o2, sc)
    assert not [e for e in pair_sets_match(b2, o2, sc) if clean2[e]]
    assert within(env_errors(sc, g2, o2.state()))[clean2].all()


def test_capsules_on_a_hull_follow_the_oracle():
    """Capsule - hull contacts: capsules at several tilts dropped onto a
    static random hull and onto a box-shaped one.  A rollout to 40 steps
    (through the first contacts), and one step from the states the oracle
    reaches at 17 and 26 steps, when most capsules touch their hull."""
    from scenegen import CAPSULE
    g = np.random.default_rng(6)
    assets = [H.hull_asset(H.random_points(g, 12, np.array([0.06, 0.05, 0.04]))), H.box_asset(0.05, 0.05, 0.02)]
    envs = []
    for k in range(16):
        q = scenegen.axis_angle_quat((1.0, 0.3 * (k % 3), 0.0), 0.25 * k)
        envs.append([body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)),
                     body(HULL, (k % 2, 0, 0), 0.0, (0, 0, 0.08)),
                     body(CAPSULE, (0.01, 0.02, 0), 0.03, (0.006 * (k - 8), 0.003 * (k % 5), 0.2), quat=q)])
    sc = pack("capsule_hull", envs, [[] for _ in envs], scenegen.default_params(), 0, 0)
    sc.hulls = H.library(assets)
    calm, ost = non_chaotic(sc, 40)
    o = oracle_run(sc, 40)
    _, st, _ = gpu_run(sc, 40)
    assert sum(len(o.manifolds(e)[0]) for e in range(16)) >= 8             # on the hulls
    clean = calm & tie_free(o, sc)
    assert clean.sum() >= 4
    err = env_errors(sc, st, ost)
    assert within(err, 10.0)[clean].all(), (np.nonzero(clean & ~within(err, 10.0))[0].tolist(), err[clean].max(0))
    for settle in (17, 26):
        b2, o2, g2, status = _one_step_from(sc, oracle_run(sc, settle).state())
        clean2 = tie_free(o2, sc)
        assert clean2.sum() >= 8
        on_hull = [e for e in range(16) if any(tuple(p) in ((2, 1), (1, 2)) for p in o2.manifolds(e)[0])]
        assert len(on_hull) >= 6
        assert not [e for e in pair_sets_match(b2, o2, sc) if clean2[e]]
        assert within(env_errors(sc, g2, o2.state()))[clean2].all()
        assert not status.any()


def test_box_hull_on_a_plane_moves_like_the_box():
    hx, hy, hz = 0.03, 0.02, 0.025
    q = scenegen.axis_angle_quat(np.array([0.3, 1.0, 0.2]) / np.linalg.norm([0.3, 1.0, 0.2]), 0.4)
    lib = H.library([H.box_asset(hx, hy, hz)])
    sb = pack("b", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.6),
                     body(BOX, (hx, hy, hz), 0.2, (0, 0, 0.08), quat=q, mu=0.6)]], [[]], scenegen.default_params(), 0, 0)
    sh = pack("h", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.6),
                     body(HULL, (0, 0, 0), 0.2, (0, 0, 0.08), quat=q, mu=0.6)]], [[]], scenegen.default_params(), 0, 0)
    sb.hulls = lib
    sh.hulls = lib
    _, a, _ = gpu_run(sb, 150)
    _, b, _ = gpu_run(sh, 150)
    err = env_errors(sb, a, b)
    assert within(err, 10.0).all(), err


def test_hull_scene_renders_like_the_oracle():
    sc = scenegen.make_scene("hulls", n_envs=8)
    st = oracle_run(sc, 40).state().astype(np.float32)
    from paper_2410_00425_b300 import Batch
    o = oracle.Oracle(sc)
    o.set_state(st.astype(np.float64))
    b = Batch(sc)
    b.set_state(torch.from_numpy(st).cuda())
    cam = scenegen.default_camera("hulls", width=96, height=64)
    col = scenegen.body_colors(sc)
    b.set_camera(cam, col)
    rgba, depth, seg = b.render()
    torch.cuda.synchronize()
    rrgb, rdepth, rseg, ties = o.render(cam, col.astype(np.float64))
    ok = ties == 0
    gseg = seg.cpu().numpy().astype(np.int64)
    assert (ok & (gseg != rseg)).sum() == 0
    assert (rseg[ok] > 5).sum() > 100                                       # hulls in view
    cov = ok & (rseg > 0)
    np.testing.assert_allclose(depth.cpu().numpy()[cov], rdepth[cov], rtol=1e-5)
    d = np.abs(rgba.cpu().numpy()[..., :3].astype(int) - rrgb.astype(int))
    assert d[ok].max() <= 1


def test_bad_hull_library_is_rejected():
    from paper_2410_00425_b300 import Batch, MSError
    sc = pack("bad", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)), body(HULL, (1, 0, 0), 0.1, (0, 0, 0.1))]], [[]],
              scenegen.default_params(), 0, 0)
    sc.hulls = H.library([H.box_asset(0.02, 0.02, 0.02)])
    with pytest.raises(MSError):
        Batch(sc)                                   # index 1 of a 1-hull library
    v, t = H.box_asset(0.02, 0.02, 0.02)
    sc.bodies["p"][1, 0] = 0
    sc.hulls = H.library([(v, t[:-1])])             # a triangle missing: not closed
    with pytest.raises(MSError):
        Batch(sc)
