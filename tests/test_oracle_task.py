"""Pins of the oracle's pick task (the paper's sim2real appendix: Controller /
Action Space, Observation Space, Reward).

Every expected value here is a closed form or a special case fixed by the
paper's definitions: the reward of an ideal grasp is 1 + 1 + 2 + (1 + 3) = 8
and each indicator moves it by its printed coefficient; distances of
atanh(1/2)/z halve a distance term exactly; joint coordinates of bodies
posed by a known rotation or offset equal that rotation or offset; the
controller moves a target by exactly clip(a)(h - l)/2 per step.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import validation as V

R, GR, CLOSE, TOUCH = 0, 1, 2, 3
TCP, CUBE, Q = slice(4, 7), slice(7, 10), slice(10, 13)
TGT = slice(13, 16)
# the probe's float32 inputs: finger x, the cube's side, finger offsets
X0 = float(np.float32(0.4))
C32 = 2.0 * float(np.float32(0.02))


def _probe(n_envs=1):
    sc = V.grasp_probe(n_envs=n_envs)
    o = oracle.Oracle(sc)
    o.set_task(sc.task)
    return sc, o


def _pose(o, edits):
    """edits: {body: (pos, quat)} applied to every env's state."""
    st = o.state()
    nb = 5
    for e in range(o.E):
        for i, (pos, quat) in edits.items():
            if pos is not None:
                st[nb * e + i, 0:3] = pos
            if quat is not None:
                st[nb * e + i, 3:7] = quat
    o.set_state(st)


def _grasp(o, dq=0.01):
    """Reset the controller at the current pose, then move the gripper
    target dq away from the gripper joint: grasped when dq > grasp_tol."""
    o.task_reset()
    t = o.targets()
    t[1::3] += dq
    o.set_targets(t)


def test_initial_record_of_the_probe():
    sc, o = _probe()
    rec, ties = o.observe()
    r = rec[0]
    np.testing.assert_allclose(r[Q], [0.0, -0.02, 0.02], atol=1e-9)
    np.testing.assert_allclose(r[TGT], r[Q], atol=0)              # the reset sets target = q
    np.testing.assert_allclose(r[TCP], [0.4, 0.0, 0.5], atol=1e-9)
    np.testing.assert_allclose(r[CUBE], [0.4, 0.0, 0.5], atol=1e-9)
    assert r[GR] == 0 and r[CLOSE] == 1 and r[TOUCH] == 0 and ties[0] == 0
    # not grasped: r_dist(0) + r_orient(horizontal) + 2 r_dist(|g| - c = 0) = 1 + 1 + 2
    assert abs(r[R] - 4.0) < 1e-6


def test_reward_of_the_ideal_grasp_is_eight():
    """tcp on the cube, fingers level and one cube side apart, grasped, joints
    at their reset values, no table contact: every term at its maximum."""
    sc, o = _probe()
    _grasp(o)
    r = o.observe()[0][0]
    assert r[GR] == 1 and r[CLOSE] == 1 and r[TOUCH] == 0
    assert abs(r[R] - 8.0) < 1e-6


@pytest.mark.parametrize("sign,expect", [(+1, 7.0), (-1, 9.0)])
def test_orientation_term_of_vertical_fingers(sign, expect):
    """Fingers stacked along z, one cube side apart, tcp on the cube: the
    orientation term 1 - up . g/|g| is 0 (g up) or 2 (g down, as printed)."""
    sc, o = _probe()
    c = 0.04
    _pose(o, {2: ([0.4, 0.0, 0.5 - sign * c / 2], None), 3: ([0.4, 0.0, 0.5 + sign * c / 2], None)})
    _grasp(o)
    r = o.observe()[0][0]
    assert r[GR] == 1 and r[CLOSE] == 1
    assert abs(r[R] - expect) < 1e-6


def test_touching_the_table_costs_two():
    """The whole probe lowered until the fingers' bottoms are 0.5 mm above
    the table (within the 1 mm touch distance): 8 - 2."""
    sc, o = _probe()
    z = 0.03 + 0.0005
    _pose(o, {1: ([0.4, 0.0, z], None), 2: ([0.4, -0.02, z], None), 3: ([0.4, 0.02, z], None)})
    _grasp(o)
    r = o.observe()[0][0]
    assert r[TOUCH] == 1
    assert abs(r[R] - 6.0) < 1e-6


def test_table_distance_uses_the_rotated_extent():
    """A finger turned 90 deg about x presents its 0.01 half-extent to the
    table: at z = 0.0125 it clears the 1 mm touch distance upright-rotated,
    while upright (half-height 0.03) it is below the table."""
    sc, o = _probe()
    qx = scenegen.axis_angle_quat((1, 0, 0), math.pi / 2)
    _pose(o, {2: ([0.4, -0.02, 0.0125], qx), 3: ([0.4, 0.02, 0.0125], qx)})
    assert o.observe()[0][0][TOUCH] == 0
    _pose(o, {2: ([0.4, -0.02, 0.0125], [0, 0, 0, 1]), 3: ([0.4, 0.02, 0.0125], [0, 0, 0, 1])})
    assert o.observe()[0][0][TOUCH] == 1
    # the rotated finger at the touch distance less 0.5 mm touches
    _pose(o, {2: ([0.4, -0.02, 0.0105], qx), 3: ([0.4, 0.02, 0.0105], qx)})
    assert o.observe()[0][0][TOUCH] == 1


def test_distance_term_halves_at_atanh_half():
    """tcp moved off the cube by atanh(1/2)/15 (beyond c/2, so tcp_close is
    off): r_dist = 1/2, and the reward is 1/2 + 1 + 0 + 4."""
    sc, o = _probe()
    d = math.atanh(0.5) / 15.0
    _pose(o, {1: ([X0 + d, 0.0, 0.5], None)})
    _grasp(o)
    r = o.observe()[0][0]
    assert r[CLOSE] == 0 and r[GR] == 1
    assert abs(r[R] - 5.5) < 1e-9


def test_finger_gap_term_halves_at_atanh_half():
    """Fingers spread so that |g| - c = atanh(1/2)/40, tcp still on the cube:
    the gap term is 2 x 1/2, the reward 1 + 1 + 1 + 4."""
    sc, o = _probe()
    s = 0.5 * C32 + 0.5 * math.atanh(0.5) / 40.0
    _pose(o, {1: ([X0, 0.0, 0.5], None), 2: ([X0, -s, 0.5], None), 3: ([X0, s, 0.5], None)})
    _grasp(o)
    r = o.observe()[0][0]
    assert r[CLOSE] == 1
    assert abs(r[R] - 7.0) < 1e-9


def test_joint_term_halves_at_atanh_half():
    """The link turned about its hinge by theta = atanh(1/2) pi/4 after the
    reset: |q - q_reset| = theta and the grasp term is 1 + 3/2."""
    sc, o = _probe()
    _grasp(o)
    th = math.atanh(0.5) * math.pi / 4.0
    _pose(o, {4: (None, scenegen.axis_angle_quat((0, 1, 0), th))})
    r = o.observe()[0][0]
    assert abs(r[10] - th) < 1e-12
    assert abs(r[R] - 6.5) < 1e-9


@pytest.mark.parametrize("theta", [-3.0, -1.0, 0.3, 2.9])
def test_revolute_coordinate_is_the_hinge_angle(theta):
    sc, o = _probe()
    _pose(o, {4: (None, scenegen.axis_angle_quat((0, 1, 0), theta))})
    assert abs(o.observe()[0][0][10] - theta) < 1e-6     # float32 quaternion input


@pytest.mark.parametrize("s", [-0.04, 0.0, 0.013])
def test_prismatic_coordinate_is_the_offset_along_the_axis(s):
    sc, o = _probe()
    _pose(o, {2: ([0.4, s, 0.5], None)})
    assert abs(o.observe()[0][0][11] - s) < 1e-7


@pytest.mark.parametrize("dq,expect", [(0.005 + 1e-4, 1), (0.005 - 1e-4, 0), (-(0.005 + 1e-4), 1)])
def test_grasped_when_the_gripper_misses_its_target(dq, expect):
    sc, o = _probe()
    _grasp(o, dq)
    assert o.observe()[0][0][GR] == expect


def test_controller_clips_unnormalises_and_accumulates():
    """q_bar <- q_bar + clip(a, -1, 1) (h - l) / 2 per step; NaN: no change."""
    sc, o = _probe()
    t0 = o.observe()[0][0][TGT].copy()
    acts = np.array([[5.0, -0.5, np.nan],
                     [5.0, np.nan, 0.25],
                     [5.0, -7.0, 1.0]])[:, None, :]
    out, _ = o.step_task(3, actions=acts)
    lo = np.asarray(sc.task["delta_lo"], np.float64)
    hi = np.asarray(sc.task["delta_hi"], np.float64)
    half = (hi - lo) / 2                       # of the float32 bounds
    expect = [t0 + half * np.array([1.0, -0.5, 0.0]),
              t0 + half * np.array([2.0, -0.5, 0.25]),
              t0 + half * np.array([3.0, -1.5, 1.25])]
    for k in range(3):
        np.testing.assert_allclose(out[k, 0, TGT], expect[k], rtol=0, atol=1e-15)


def test_absolute_targets_without_a_task():
    """Without a task an action is an absolute target (unchanged behaviour)."""
    sc = V.grasp_probe()
    o = oracle.Oracle(sc)
    o.step(1, actions=np.array([[[0.3, np.nan, 0.01]]]))
    t = o.targets()
    assert t[0] == 0.3 and t[1] == 0.0 and t[2] == 0.01


def test_task_reset_touches_only_masked_envs():
    sc, o = _probe(n_envs=2)
    acts = np.tile(np.array([[1.0, 1.0, 1.0]]), (1, 2, 1))
    o.step_task(1, actions=acts)
    before = o.observe()[0]
    o.task_reset(np.array([1, 0], np.uint8))
    after = o.observe()[0]
    np.testing.assert_array_equal(after[1], before[1])            # env 1 untouched
    np.testing.assert_array_equal(after[0][TGT], after[0][Q])     # env 0: target = q
    assert not np.array_equal(before[0][TGT], after[0][TGT])


def test_records_of_a_rollout_agree_with_observe():
    """step_task's record of the last step equals observe() afterwards, and
    the tie masks flag decisions within 1e-5 of their thresholds only."""
    sc = scenegen.make_scene("pick", n_envs=8)
    o = oracle.Oracle(sc)
    o.set_task(sc.task)
    out, ties = o.step_task(30)
    rec, t = o.observe()
    np.testing.assert_array_equal(out[-1], rec)
    assert np.isfinite(out).all()
    assert out[:, :, GR].any() and not out[:, :, GR].all()       # both branches visited


def test_set_task_rejects_bad_indices():
    sc = V.grasp_probe()
    o = oracle.Oracle(sc)
    with pytest.raises(ValueError):
        o.set_task(dict(sc.task, cube=0))                          # the plane is not a box
    with pytest.raises(ValueError):
        o.set_task(dict(sc.task, table=1))                         # the cube is not a plane
    with pytest.raises(ValueError):
        o.set_task(dict(sc.task, finger_a=7))
