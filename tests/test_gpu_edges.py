"""Edge cases of the batched step, through the C ABI, against the oracle:
zero steps, a one-env batch, a ragged batch of 1 to 64 bodies per env (the
largest env spilling contact rows to its global slot under every
placement), an env of static bodies only, coincident sphere centres, and an
env frozen by a non-finite state."""
import numpy as np
import pytest

import scenegen
from scenegen import BOX, PLANE, SPHERE, body, pack

from _parity import env_errors, gpu_run, oracle_run, pair_sets_match, tie_free, within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _ragged(sizes, seed=11):
    """One env per entry: size 1 is a lone sphere in free fall; otherwise a
    plane and size - 1 boxes (h = 0.02 m) on a grid 8 cm apart (no box-box
    pair), 1 mm above the plane, yawed by up to 0.2 rad, with small random
    velocities: 4 contact points per box, 252 in the 64-body env."""
    g = np.random.default_rng(seed)
    envs = []
    for n in sizes:
        if n == 1:
            envs.append([body(SPHERE, (0.03, 0, 0), 0.1, (0, 0, 0.5), linvel=tuple(g.normal(0, 0.2, 3)))])
            continue
        bl = [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), group=1)]
        side = int(np.ceil(np.sqrt(n - 1)))
        for k in range(n - 1):
            x, y = (k % side) * 0.08, (k // side) * 0.08
            yaw = g.uniform(-0.2, 0.2)
            q = (0.0, 0.0, np.sin(yaw / 2), np.cos(yaw / 2))
            bl.append(body(BOX, (0.02, 0.02, 0.02), 0.1, (x, y, 0.021), quat=q,
                           linvel=tuple(g.normal(0, 0.05, 3)), group=2))
        envs.append(bl)
    params = scenegen.default_params(contact_capacity=256, pair_capacity=128)
    return pack("ragged", envs, [[] for _ in envs], params, 0, seed)


def test_zero_steps_change_nothing():
    from paper_2410_00425_b300 import Batch
    sc = scenegen.make_scene("arm", n_envs=8)
    b = Batch(sc)
    s = torch.cuda.Stream()
    before = b.state().cpu()
    b.step(None, 0, stream=s)
    b.step(None, 0, stream=s, plain=True)
    torch.cuda.synchronize()
    assert torch.equal(before, b.state().cpu())
    b.close()


@pytest.mark.parametrize("name", ["small", "arm", "clutter", "hand"])
def test_one_env_batch_follows_oracle(name):
    sc = scenegen.make_scene(name, n_envs=1)
    _, st, status = gpu_run(sc, 1, record=True)
    o = oracle_run(sc, 1)
    if tie_free(o, sc)[0]:
        assert within(env_errors(sc, st, o.state()))[0]
    assert status[0] == o.status(0)


SIZES = [1, 2, 3, 8, 17, 33, 64]


def test_ragged_batch_follows_oracle():
    sc = _ragged(SIZES)
    b, st, status = gpu_run(sc, 1, record=True)
    o = oracle_run(sc, 1)
    assert not pair_sets_match(b, o, sc)
    err = env_errors(sc, st, o.state())
    clean = tie_free(o, sc)
    assert clean.sum() >= len(SIZES) - 2
    assert within(err)[clean].all(), err[clean].max(0)
    for e in range(sc.n_envs):
        assert status[e] == o.status(e)
    # ten steps: the boxes settle onto the plane
    _, st10, _ = gpu_run(sc, 10)
    o10 = oracle_run(sc, 10)
    clean10 = tie_free(o10, sc)
    assert within(env_errors(sc, st10, o10.state()), 10.0)[clean10].all()


@pytest.mark.parametrize("tuning", [(32, 1, 1), (16, 2, 0), (8, 4, 2), (32, 2, 2), (16, 4, 2), (8, 2, 0)])
def test_ragged_batch_identical_under_every_placement(tuning):
    sc = _ragged(SIZES * 4)
    _, ref, sref = gpu_run(sc, 3)
    _, st, s2 = gpu_run(sc, 3, tuning=tuning)
    assert np.array_equal(ref, st)
    assert np.array_equal(sref, s2)


def test_env_of_static_bodies_only_stays_put():
    envs = [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)), body(BOX, (0.1, 0.1, 0.1), 0.0, (0, 0, 0.1))],
            [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)), body(SPHERE, (0.02, 0, 0), 0.1, (0, 0, 0.3))]]
    sc = pack("static", envs, [[], []], scenegen.default_params(), 0, 0)
    _, st, status = gpu_run(sc, 5)
    o = oracle_run(sc, 5)
    assert np.array_equal(st[0:2], sc_state(sc)[0:2])
    assert within(env_errors(sc, st, o.state())).all()
    assert not status.any()


def sc_state(sc):
    import oracle
    return oracle.Oracle(sc).state()


def test_coincident_sphere_centres_follow_oracle():
    """Two spheres with the same centre: the normal is +z by the stated rule;
    both sides push them apart along it."""
    envs = [[body(SPHERE, (0.02, 0, 0), 0.1, (0, 0, 0.5)), body(SPHERE, (0.03, 0, 0), 0.2, (0, 0, 0.5))]]
    params = scenegen.default_params(gravity=(0.0, 0.0, 0.0))
    sc = pack("coincident", envs, [[]], params, 0, 0)
    b, st, _ = gpu_run(sc, 1, record=True)
    o = oracle_run(sc, 1)
    gp, gn, gx = b.contacts(0)
    op, on, ox = o.manifolds(0)
    assert np.array_equal(gp, op) and np.array_equal(gn, on)
    assert np.abs(gx[0, :on[0]].astype(np.float64) - ox[0, :on[0]]).max() <= 1e-5
    assert within(env_errors(sc, st, o.state())).all()
    # the position sweeps push them apart along +z; the rigid relax sweep
    # leaves no separating velocity
    assert st[0, 2] > 0.5 > st[1, 2]


def test_non_finite_state_freezes_only_its_env():
    from paper_2410_00425_b300 import Batch
    sc = scenegen.make_scene("small", n_envs=6)
    s = torch.cuda.Stream()
    a = Batch(sc)
    b = Batch(sc)
    st = b.state().cpu().numpy().copy()
    st[sc.body_off[2] + 1, 7] = np.nan                 # a dynamic body of env 2
    b.set_state(torch.from_numpy(st).contiguous(), stream=s)
    a.step(None, 4, stream=s)
    b.step(None, 4, stream=s)
    torch.cuda.synchronize()
    sa, sb = a.state().cpu().numpy(), b.state().cpu().numpy()
    _, status = b.sync()
    bo = sc.body_off
    assert status[2] & 8
    assert np.isnan(sb[bo[2]:bo[3]]).any()
    for e in (0, 1, 3, 4, 5):
        assert status[e] == 0
        assert np.array_equal(sa[bo[e]:bo[e + 1]], sb[bo[e]:bo[e + 1]])
    a.close()
    b.close()
