"""Small scenes with closed-form or invariant outcomes (free fall, incline,
momentum exchange, resting stack, PD pendulum, joint limit, LCP).

Like the rest of :mod:`scenegen` these only describe inputs; the expected
values are derived in the tests from mechanics, not from either implementation.
"""
from __future__ import annotations

import math

import numpy as np

from . import (BOX, CAPSULE, PLANE, PRISMATIC, REVOLUTE, SPHERE, axis_angle_quat, body,
               joint, pack, rng, shoemake_quat)
from . import default_params as _workload_params


def default_params(**kw):
    """The workloads' parameters with rigid rows (contact_hertz = joint_hertz
    = 0) unless asked otherwise: the closed forms these scenes pin are those
    of rigid constraints; the soft rows have pins of their own."""
    return _workload_params(**dict(dict(contact_hertz=0.0, joint_hertz=0.0), **kw))


def freefall(n_envs=16, seed=0, **pk):
    """One dynamic body per env, random pose and velocity, nothing to hit."""
    envs_b, envs_j = [], []
    for e in range(n_envs):
        g = rng(seed, e, 0)
        pos = g.uniform(-1, 1, 3)
        v = g.uniform(-2, 2, 3)
        w = g.uniform(-3, 3, 3)
        if e % 2 == 0:
            b = body(SPHERE, (0.05, 0, 0), 1.0, pos, linvel=v, angvel=w)
        else:
            b = body(BOX, (0.03, 0.02, 0.05), 0.7, pos, shoemake_quat(g), linvel=v, angvel=w)
        envs_b.append([b]); envs_j.append([])
    return pack("freefall", envs_b, envs_j, default_params(**pk), 0, seed)


def incline(thetas, mu=0.5, h=0.02, mass=0.1, **pk):
    """A box resting (d = 0) on a static ramp tilted by theta about +y; one env
    per angle.  Down-slope is the ramp's +x direction."""
    envs_b, envs_j = [], []
    for th in thetas:
        q = axis_angle_quat((0, 1, 0), th)
        ramp_h = (1.0, 0.3, 0.05)
        n = np.array([math.sin(th), 0.0, math.cos(th)])
        s = np.array([math.cos(th), 0.0, -math.sin(th)])
        c = n * (ramp_h[2] + h) - s * 0.7
        envs_b.append([body(BOX, ramp_h, 0.0, (0, 0, 0), q, mu=mu, group=1),
                       body(BOX, (h, h, h), mass, c, q, mu=mu, group=2)])
        envs_j.append([])
    return pack("incline", envs_b, envs_j, default_params(**pk), 0, 0)


def momentum(n_envs=8, seed=0, spheres_only=False, **pk):
    """g = 0, mu = 0: 4 to 6 bodies thrown at each other in a small region."""
    p = default_params(gravity=(0.0, 0.0, 0.0), **pk)
    envs_b, envs_j = [], []
    for e in range(n_envs):
        g = rng(seed, e, 0)
        n = 4 + int(g.integers(0, 3))
        bl = []
        placed = []
        for i in range(n):
            kind = SPHERE if (spheres_only or i % 2 == 0) else BOX
            r = 0.03 + 0.02 * g.random()
            rb = r if kind == SPHERE else r * math.sqrt(3)
            for _ in range(200):
                c = g.uniform(-0.15, 0.15, 3)
                if all(np.linalg.norm(c - pc) > rb + pr + 1e-3 for pc, pr in placed):
                    break
            placed.append((c, rb))
            v = -c * (2.0 + 2.0 * g.random()) + g.uniform(-0.3, 0.3, 3)
            m = 0.2 + g.random()
            if kind == SPHERE:
                bl.append(body(SPHERE, (r, 0, 0), m, c, linvel=v, mu=0.0, group=1))
            else:
                bl.append(body(BOX, (r, r * 0.8, r * 1.2), m, c, shoemake_quat(g), linvel=v,
                               angvel=g.uniform(-2, 2, 3), mu=0.0, group=1))
        envs_b.append(bl); envs_j.append([])
    return pack("momentum", envs_b, envs_j, p, 0, seed)


def stack(n_boxes=3, h=0.02, mass=0.1, mu=0.5, **pk):
    """Boxes on the plane, initially touching (d = 0)."""
    bl = [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=mu, group=1)]
    for k in range(n_boxes):
        bl.append(body(BOX, (h, h, h), mass, (0, 0, h + 2 * h * k), mu=mu, group=2))
    return pack("stack", [bl], [[]], default_params(**pk), 0, 0)


def pendulum(kp=2.0, kd=0.0, amp=0.05, r=0.02, l=0.1, m=1.0, pivot_z=1.0, **pk):
    """A capsule hanging from a world revolute joint about +y, released at
    `amp` rad with the drive target at 0."""
    qy = axis_angle_quat((0, 0, 1), math.pi / 2)        # frame +x -> world +y
    q0 = axis_angle_quat((0, 1, 0), amp)
    R = _rot(q0)
    c = np.array([0, 0, pivot_z]) + R @ np.array([0, 0, -l])
    b = body(CAPSULE, (r, l, 0), m, c, q0, group=1)
    j = joint(REVOLUTE, -1, 0, (0, 0, pivot_z, *qy), (0, 0, l, *qy), -3.0, 3.0, kp, kd, 0.0)
    return pack("pendulum", [[b]], [[j]], default_params(**pk), 1, 0)


def slider(kp=50.0, kd=2.0, m=0.5, s0=0.0, target=0.1, **pk):
    """A box on a world prismatic joint along +x, frame at its centre, g = 0:
    the drive row is the only row with a non-zero error (isolated row)."""
    p = default_params(gravity=(0.0, 0.0, 0.0), **pk)
    b = body(BOX, (0.02, 0.02, 0.02), m, (s0, 0, 0.5), group=1)
    j = joint(PRISMATIC, -1, 0, (0, 0, 0.5, 0, 0, 0, 1), (0, 0, 0, 0, 0, 0, 1),
              -10.0, 10.0, kp, kd, target)
    return pack("slider", [[b]], [[j]], p, 1, 0)


def limit(upper=1.0, target=2.0, kp=10.0, kd=1.0, **pk):
    """A capsule on a world revolute joint driven past its upper limit, g = 0."""
    p = default_params(gravity=(0.0, 0.0, 0.0), **pk)
    qy = axis_angle_quat((0, 0, 1), math.pi / 2)
    b = body(CAPSULE, (0.02, 0.1, 0), 1.0, (0, 0, 0.9), group=1)
    j = joint(REVOLUTE, -1, 0, (0, 0, 1.0, *qy), (0, 0, 0.1, *qy), -upper, upper, kp, kd, target)
    return pack("limit", [[b]], [[j]], p, 1, 0)


def resting_box(tilt=(0.0, 0.0), mu=0.0, h=(0.03, 0.02, 0.025), mass=0.3, seed=0, **pk):
    """A box on the plane, slightly tilted so 1-4 corners are within the margin."""
    q = axis_angle_quat((1, 0, 0), tilt[0])
    q2 = axis_angle_quat((0, 1, 0), tilt[1])
    q = _qmul(q2, q)
    R = _rot(q)
    corners = np.array([[sx * h[0], sy * h[1], sz * h[2]] for sx in (-1, 1) for sy in (-1, 1)
                        for sz in (-1, 1)])
    zmin = (corners @ R.T)[:, 2].min()
    c = np.array([0, 0, -zmin - 0.001])       # 1 mm penetration of the lowest corner
    bl = [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=mu, group=1),
          body(BOX, h, mass, c, q, linvel=(0.0, 0.0, -0.2), angvel=(0.3, -0.2, 0.1), mu=mu, group=2)]
    return pack("resting_box", [bl], [[]], default_params(**pk), 0, seed)


def bouncing_ball(e=0.5, z0=0.5, vz0=0.0, r=0.02, m=0.05, n_envs=1, **pk):
    """A sphere above the plane, frictionless, both with restitution e."""
    envs_b = []
    for k in range(n_envs):
        envs_b.append([body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.0, group=1, restitution=e),
                       body(SPHERE, (r, 0, 0), m, (0.1 * k, 0, z0), linvel=(0.0, 0.0, vz0), mu=0.0, group=2,
                            restitution=e)])
    return pack("bouncing_ball", envs_b, [[] for _ in range(n_envs)], default_params(**pk), 0, 0)


def _rot(q):
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _qmul(a, b):
    av, aw = np.asarray(a[:3]), a[3]
    bv, bw = np.asarray(b[:3]), b[3]
    v = aw * bv + bw * av + np.cross(av, bv)
    return np.array([v[0], v[1], v[2], aw * bw - av @ bv])


def grasp_probe(n_envs=1, **pk):
    """Probe of the pick task's observations and reward (no stepping needed):
    table plane (0); cube of side 0.04 (1) at (0.4, 0, 0.5); two box fingers
    (2, 3; half-extents 0.01, 0.01, 0.03) on prismatic joints along world +y
    through (0.4, 0, 0.5), at y = -0.02 and +0.02 (their joint coordinates);
    a capsule link (4) on a revolute joint about world +y at (0, 0, 1), angle
    0.  Joints: 0 revolute, 1 finger a (the gripper joint), 2 finger b."""
    qy = axis_angle_quat((0, 0, 1), math.pi / 2)      # frame +x -> world +y
    fh = (0.01, 0.01, 0.03)
    envs_b, envs_j = [], []
    for _ in range(n_envs):
        envs_b.append([body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), group=1),
                       body(BOX, (0.02, 0.02, 0.02), 0.05, (0.4, 0.0, 0.5), group=2),
                       body(BOX, fh, 0.05, (0.4, -0.02, 0.5), group=4, mask=1),
                       body(BOX, fh, 0.05, (0.4, 0.02, 0.5), group=4, mask=1),
                       body(CAPSULE, (0.02, 0.1, 0), 1.0, (0.0, 0.0, 1.0), group=8, mask=0)])
        envs_j.append([joint(REVOLUTE, -1, 4, (0, 0, 1.0, *qy), (0, 0, 0, *qy), -3.0, 3.0, 0, 0, 0),
                       joint(PRISMATIC, -1, 2, (0.4, 0, 0.5, *qy), (0, 0, 0, *qy), -0.05, 0.05, 0, 0, 0),
                       joint(PRISMATIC, -1, 3, (0.4, 0, 0.5, *qy), (0, 0, 0, *qy), -0.05, 0.05, 0, 0, 0)])
    sc = pack("grasp_probe", envs_b, envs_j, default_params(**pk), 3, 0)
    lo = np.array([-0.05, -0.005, -0.005], np.float32)
    sc.task = dict(grip_joint=1, finger_a=2, finger_b=3, cube=1, table=0,
                   grasp_tol=float(np.float32(0.005)), touch_tol=float(np.float32(0.001)),
                   delta_lo=lo, delta_hi=-lo)
    return sc
