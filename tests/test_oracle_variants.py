"""Pins of the oracle's optional solver variants: velocity damping,
restitution and warm starting across steps (all off by default).

Damping is checked against the closed form of its recurrence, restitution
against the velocity it must leave after an impact, warm starting against
the equilibrium impulse of a resting box and against the rest it brings,
at one position iteration, to a box on the plane and a hanging chain.  The default parameters must leave every result unchanged.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import validation as V

G = 9.81


def test_variants_off_change_nothing():
    sc = scenegen.make_scene("arm", n_envs=4)
    a = oracle.Oracle(sc)
    a.step(5)
    sc2 = scenegen.make_scene("arm", n_envs=4)
    sc2.params = dict(sc2.params, linear_damping=0.0, angular_damping=0.0, warm_start=0, bounce_threshold=3.0)
    b = oracle.Oracle(sc2)
    b.step(5)
    assert np.array_equal(a.state(), b.state())


@pytest.mark.parametrize("cl,cw", [(0.5, 0.0), (2.0, 3.0)])
def test_damping_follows_its_recurrence(cl, cw):
    """Free flight: v_N = a^N v0 + h g (1 - a^N) / (1 - a), w_N = b^N w0 with
    a = 1/(1 + h c_lin), b = 1/(1 + h c_ang), N substeps; positions follow
    the symplectic sum of the same velocities."""
    sc = V.freefall(n_envs=4, linear_damping=cl, angular_damping=cw)
    o = oracle.Oracle(sc)
    st0 = o.state().copy()
    steps = 25
    o.step(steps)
    st = o.state()
    p = sc.params
    h = p["dt"] / p["substeps"]
    N = steps * p["substeps"]
    a, b = 1.0 / (1.0 + h * cl), 1.0 / (1.0 + h * cw)
    g = np.array(p["gravity"])
    geo = N if a == 1.0 else (1 - a ** N) / (1 - a)
    v_expect = a ** N * st0[:, 7:10] + h * g * geo
    np.testing.assert_allclose(st[:, 7:10], v_expect, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st[:, 10:13], b ** N * st0[:, 10:13], rtol=1e-12, atol=1e-12)
    # x_N = x0 + h sum_{k=1..N} v_k
    vk = np.array([a ** k * st0[:, 7:10] + h * g * ((k if a == 1.0 else (1 - a ** k) / (1 - a)))
                   for k in range(1, N + 1)])
    np.testing.assert_allclose(st[:, 0:3], st0[:, 0:3] + h * vk.sum(0), rtol=1e-11, atol=1e-12)


def _impact_step(e, z0=0.5, **pk):
    sc = V.bouncing_ball(e=e, z0=z0, **pk)
    o = oracle.Oracle(sc)
    for k in range(400):
        vz_before = o.state()[1, 9]
        o.step(1)
        if o.manifolds(0)[1].size:           # the step that made contact
            return vz_before, o, k
    raise AssertionError("no impact")


@pytest.mark.parametrize("e", [0.0, 0.3, 0.8])
def test_restitution_reverses_the_approach_speed(e):
    """Frictionless sphere on the plane: after the impact step the normal
    velocity is -e times the step-start approach speed (the pass solves the
    single normal row exactly), and the ball leaves the plane when e > 0."""
    vz0, o, k = _impact_step(e)
    assert vz0 < -1.0                         # above the bounce threshold
    vz = o.state()[1, 9]
    e32 = float(np.float32(e))                # the scene stores restitution in float32
    if e > 0:
        assert abs(vz - (-e32 * vz0)) < 1e-12 * abs(vz0), (vz, -e32 * vz0)
        # it rises: a later step has no contact
        o.step(3)
        assert o.state()[1, 9] > 0 or o.state()[1, 2] > 0.021
    else:
        assert abs(vz) < 0.05


def test_restitution_below_threshold_does_not_bounce():
    """A slow approach (below bounce_threshold) comes to rest."""
    vz0, o, k = _impact_step(0.8, z0=0.05, bounce_threshold=1.0)
    assert -1.0 < vz0 < 0
    assert abs(o.state()[1, 9]) < 0.05


def test_warm_start_carries_the_equilibrium_impulse():
    """A box at rest on the plane, warm started across steps: the normal
    impulses of a substep sum to m g h (static equilibrium), to 1e-9."""
    sc = V.stack(n_boxes=1, pos_iters=4, warm_start=1)
    o = oracle.Oracle(sc)
    o.step(300)
    rows = o.rows(0)
    p = sc.params
    h = p["dt"] / p["substeps"]
    m = float(sc.bodies["mass"][1])
    normal = rows[:, 2] == 0
    assert abs(rows[normal, 14].sum() - m * G * h) < 1e-9 * m * G * h
    assert normal.sum() == 4


def test_warm_start_brings_a_resting_box_to_rest():
    """A box on the plane solved with one position iteration per substep:
    warm started across steps its contact impulses converge over the steps
    and it rests exactly; restarted cold every step it keeps jittering."""
    res = {}
    for warm in (0, 1):
        sc = V.stack(n_boxes=1, pos_iters=1, warm_start=warm)
        o = oracle.Oracle(sc)
        x0 = o.state()[1, 0:3].copy()
        o.step(200)
        st = o.state()
        res[warm] = (np.abs(st[1, 7:13]).max(), np.abs(st[1, 0:3] - x0).max())
    assert res[1][0] < 1e-12 and res[1][1] < 1e-6, res
    assert res[0][0] > 1e-3, res


def _chain(warm, pos_iters):
    qy = scenegen.axis_angle_quat((0, 0, 1), math.pi / 2)
    r, l = 0.02, 0.1
    bl = [scenegen.body(scenegen.CAPSULE, (r, l, 0), 1.0, (0, 0, 1.0 - l), group=1),
          scenegen.body(scenegen.CAPSULE, (r, l, 0), 0.5, (0, 0, 1.0 - 3 * l), group=2)]
    jl = [scenegen.joint(scenegen.REVOLUTE, -1, 0, (0, 0, 1.0, *qy), (0, 0, l, *qy), -3, 3, 0, 0, 0),
          scenegen.joint(scenegen.REVOLUTE, 0, 1, (0, 0, -l, *qy), (0, 0, l, *qy), -3, 3, 0, 0, 0)]
    return scenegen.pack("chain", [bl], [jl], scenegen.default_params(pos_iters=pos_iters, warm_start=warm), 2, 0)


def test_warm_start_brings_a_hanging_chain_to_rest():
    """Two links hanging from the world on revolute joints, one position
    iteration: the coupled joint rows converge across steps only when their
    impulses are carried."""
    res = {}
    for warm in (0, 1):
        o = oracle.Oracle(_chain(warm, 1))
        o.step(200, actions=np.zeros((200, 1, 2)))
        res[warm] = np.abs(o.state()[:, 7:13]).max()
    assert res[1] < 1e-12, res
    assert res[0] > 1e-5, res


def test_set_state_clears_the_warm_memory():
    """After a set state the next step starts cold: its impulses equal those
    of a fresh world set to the same state, and differ from the warm ones."""
    sc = V.stack(n_boxes=1, pos_iters=2, warm_start=1)
    o = oracle.Oracle(sc)
    o.step(50)
    lam_warm = o.rows(0)[:, 14].copy()
    st = o.state()
    o.set_state(st)                           # clears the warm-start memory
    o.step(1)
    lam_after_reset = o.rows(0)[:, 14].copy()
    o2 = oracle.Oracle(sc)
    o2.set_state(st)
    o2.step(1)
    np.testing.assert_array_equal(lam_after_reset, o2.rows(0)[:, 14])
    assert not np.array_equal(lam_warm, lam_after_reset)
