"""Seeded synthetic scenes for the batched rigid-body step.

This module only *describes* inputs: body and joint descriptors, per-env
offsets, solver parameters and per-step drive targets.  It contains none of
the step's arithmetic (no inertia, no contact, no solver), so both the FP64
oracle and the CUDA path consume it without sharing any of the method.

Every random draw comes from numpy's Philox-4x32-10 bit generator keyed by
(seed, env, stream), so an env's contents do not depend on how many envs are
generated beside it (per-env seeding for replay, paper Sec. "Demonstration
Datasets").  The four scene families stand in for the paper's table-top
PickCube, PickClutterYCB and dextrous rotation workloads (Appendix
"Environments and Robots List"); no dataset asset is read.

Conventions: z-up world, quaternions stored (x, y, z, w), capsule axis and
plane normal along local +z, joint axis along the joint frame's +x.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional

import numpy as np

SPHERE, CAPSULE, BOX, PLANE, HULL = 0, 1, 2, 3, 4
REVOLUTE, PRISMATIC = 0, 1

BODY_DTYPE = np.dtype([
    ("type", "<i4"), ("p", "<f4", (3,)), ("mass", "<f4"),
    ("pos", "<f4", (3,)), ("quat", "<f4", (4,)),
    ("linvel", "<f4", (3,)), ("angvel", "<f4", (3,)),
    ("mu", "<f4"), ("restitution", "<f4"),
    ("group", "<u2"), ("mask", "<u2"),
])
JOINT_DTYPE = np.dtype([
    ("type", "<i4"), ("parent", "<i4"), ("child", "<i4"),
    ("parent_frame", "<f4", (7,)), ("child_frame", "<f4", (7,)),
    ("lower", "<f4"), ("upper", "<f4"), ("kp", "<f4"), ("kd", "<f4"),
    ("target0", "<f4"),
])
assert BODY_DTYPE.itemsize == 84 and JOINT_DTYPE.itemsize == 88

ALL_GROUPS = 0xFFFF


def default_params(**kw) -> Dict:
    p = dict(dt=0.01, substeps=4, pos_iters=8, vel_iters=1,
             gravity=(0.0, 0.0, -9.81), margin=0.01, max_depen_vel=1.0,
             contact_capacity=64, pair_capacity=128,
             linear_damping=0.0, angular_damping=0.0, bounce_threshold=1.0, warm_start=0,
             contact_hertz=30.0, contact_damping_ratio=10.0, joint_hertz=60.0, joint_damping_ratio=2.0)
    p.update(kw)
    return p


@dataclasses.dataclass
class Scene:
    """A batch of envs: flat descriptor tables plus CSR offsets per env."""
    name: str
    bodies: np.ndarray          # BODY_DTYPE [n_bodies_total]
    body_off: np.ndarray        # int32 [E+1]
    joints: np.ndarray          # JOINT_DTYPE [n_joints_total]
    joint_off: np.ndarray       # int32 [E+1]
    params: Dict
    n_act: int                  # A: action slots per env per step (0 = none)
    seed: int
    action_fn: Optional[Callable[[int, int], np.ndarray]] = None
    task: Optional[Dict] = None  # pick task (pick_task); actions are then normalised deltas
    hulls: Optional[Dict] = None  # hull library (scenegen.hulls.library) of HULL bodies

    @property
    def n_envs(self) -> int:
        return len(self.body_off) - 1

    def actions(self, step0: int, n_steps: int) -> Optional[np.ndarray]:
        """Drive targets float32 [n_steps][E][A] for steps step0..step0+n-1.

        NaN means "keep the previous target" for that joint slot."""
        if self.n_act == 0 or self.action_fn is None:
            return None
        return self.action_fn(step0, n_steps)

    def subset(self, envs) -> "Scene":
        """The same envs, re-packed as a smaller batch (envs keep contents)."""
        envs = list(envs)
        bl, jl, bo, jo = [], [], [0], [0]
        for e in envs:
            b = self.bodies[self.body_off[e]:self.body_off[e + 1]]
            j = self.joints[self.joint_off[e]:self.joint_off[e + 1]]
            bl.append(b); jl.append(j)
            bo.append(bo[-1] + len(b)); jo.append(jo[-1] + len(j))
        parent = self
        idx = np.asarray(envs)

        def fn(step0, n):
            a = parent.actions(step0, n)
            return None if a is None else np.ascontiguousarray(a[:, idx, :])
        return Scene(self.name, np.concatenate(bl) if bl else np.zeros(0, BODY_DTYPE),
                     np.asarray(bo, np.int32),
                     np.concatenate(jl) if jl else np.zeros(0, JOINT_DTYPE),
                     np.asarray(jo, np.int32), dict(self.params), self.n_act,
                     self.seed, fn if self.action_fn else None, self.task, self.hulls)


def rng(seed: int, env: int, stream: int) -> np.random.Generator:
    """Philox-4x32-10 keyed by (seed, env, stream)."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, ((env & 0xFFFFFFFF) << 16) | (stream & 0xFFFF)],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def step_rng(seed: int, step: int, kind: int) -> np.random.Generator:
    """Philox-4x32-10 keyed by (seed, step, kind) for per-step batch draws."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, (1 << 63) | ((step & 0xFFFFFFFF) << 8) | (kind & 0xFF)],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def shoemake_quat(g: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake 1992), returned (x, y, z, w)."""
    u1, u2, u3 = g.random(3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    return np.array([a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                     b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)])


def axis_angle_quat(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    s = math.sin(angle / 2)
    return np.array([axis[0] * s, axis[1] * s, axis[2] * s, math.cos(angle / 2)])


def body(type_, p, mass, pos, quat=(0, 0, 0, 1), linvel=(0, 0, 0), angvel=(0, 0, 0),
         mu=0.5, group=1, mask=ALL_GROUPS, restitution=0.0) -> np.ndarray:
    b = np.zeros((), BODY_DTYPE)
    b["type"] = type_
    b["p"] = p
    b["mass"] = mass
    b["pos"] = pos
    b["quat"] = quat
    b["linvel"] = linvel
    b["angvel"] = angvel
    b["mu"] = mu
    b["restitution"] = restitution
    b["group"] = group
    b["mask"] = mask
    return b


def joint(type_, parent, child, parent_frame, child_frame, lower, upper, kp, kd,
          target0=0.0) -> np.ndarray:
    j = np.zeros((), JOINT_DTYPE)
    j["type"] = type_
    j["parent"] = parent
    j["child"] = child
    j["parent_frame"] = parent_frame
    j["child_frame"] = child_frame
    j["lower"] = lower
    j["upper"] = upper
    j["kp"] = kp
    j["kd"] = kd
    j["target0"] = target0
    return j


def pack(name, per_env_bodies: List[List], per_env_joints: List[List], params, n_act, seed,
         action_fn=None) -> Scene:
    bo, jo = [0], [0]
    for b, j in zip(per_env_bodies, per_env_joints):
        bo.append(bo[-1] + len(b)); jo.append(jo[-1] + len(j))
    bodies = np.array([b for env in per_env_bodies for b in env], dtype=BODY_DTYPE) \
        if bo[-1] else np.zeros(0, BODY_DTYPE)
    joints = np.array([j for env in per_env_joints for j in env], dtype=JOINT_DTYPE) \
        if jo[-1] else np.zeros(0, JOINT_DTYPE)
    return Scene(name, bodies, np.asarray(bo, np.int32), joints, np.asarray(jo, np.int32),
                 params, n_act, seed, action_fn)


def _place(g, radii, lo, hi, placed, extra_ok=None, tries=64, gap=1e-3):
    """Rejection-sample a centre whose bounding sphere is `gap` clear of the
    already placed ones; after `tries` failures stack it above them."""
    r = radii
    for _ in range(tries):
        c = lo + (hi - lo) * g.random(3)
        if extra_ok is not None and not extra_ok(c, r):
            continue
        if all(np.linalg.norm(c - pc) >= r + pr + gap for pc, pr in placed):
            return c
    c = lo + (hi - lo) * g.random(3)
    if extra_ok is not None:
        c[0] = min(max(c[0], lo[0]), hi[0]); c[1] = min(max(c[1], lo[1]), hi[1])
    top = max([pc[2] + pr for pc, pr in placed] + [c[2] - r])
    c[2] = top + r + gap
    return c


# ----------------------------------------------------------------------------
# Config "small": plane + 1 box + 3 spheres per env.
# ----------------------------------------------------------------------------
def make_small(n_envs=64, seed=1) -> Scene:
    params = default_params(contact_capacity=32, pair_capacity=16)
    envs_b, envs_j = [], []
    for e in range(n_envs):
        g = rng(seed, e, 0)
        bl = [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.5, group=1)]
        placed = []
        lo, hi = np.array([-0.1, -0.1, 0.05]), np.array([0.1, 0.1, 0.25])
        # box first: bounding sphere radius h*sqrt(3)
        rb = 0.02 * math.sqrt(3.0)
        q = shoemake_quat(g)
        c = _place(g, rb, lo, hi, placed, tries=64)
        placed.append((c, rb))
        bl.append(body(BOX, (0.02, 0.02, 0.02), 0.1, c, q, mu=0.5, group=2))
        for _ in range(3):
            c = _place(g, 0.02, lo, hi, placed, tries=64)
            placed.append((c, 0.02))
            bl.append(body(SPHERE, (0.02, 0, 0), 0.05, c, mu=0.5, group=2))
        envs_b.append(bl); envs_j.append([])
    return pack("small", envs_b, envs_j, params, 0, seed)


# ----------------------------------------------------------------------------
# Config "arm": 7-DoF capsule arm + 2 prismatic box fingers + cube on a plane.
# ----------------------------------------------------------------------------
G_PLANE, G_ARM, G_CUBE = 1, 2, 4


def make_arm(n_envs=4096, seed=2) -> Scene:
    # typical use is 4-12 contact points and < 20 candidate pairs per env
    params = default_params(contact_capacity=32, pair_capacity=48)
    envs_b, envs_j = [], []
    n_act = 9
    qz = axis_angle_quat((0, 1, 0), -math.pi / 2)   # frame +x -> world +z
    qy = axis_angle_quat((0, 0, 1), math.pi / 2)    # frame +x -> world +y
    qny = axis_angle_quat((0, 0, 1), -math.pi / 2)  # frame +x -> world -y
    for e in range(n_envs):
        g = rng(seed, e, 0)
        bl = [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.5, group=G_PLANE)]
        r = 0.04
        base_l = 0.05
        # static base capsule standing on the plane
        zc = r + base_l
        bl.append(body(CAPSULE, (r, base_l, 0), 0.0, (0, 0, zc), group=G_ARM,
                       mask=G_PLANE | G_CUBE))
        top = zc + base_l
        prev_l = base_l
        jl = []
        for k in range(7):
            seg = 0.1 + 0.2 * g.random()
            l = seg / 2
            m = 0.5 + 2.5 * g.random()
            zc = top + l
            bl.append(body(CAPSULE, (r, l, 0), m, (0, 0, zc), group=G_ARM,
                           mask=G_PLANE | G_CUBE))
            qa = qz if k % 2 == 0 else qy
            jl.append(joint(REVOLUTE, k + 1, k + 2,
                            (0, 0, prev_l, *qa), (0, 0, -l, *qa),
                            -2.8, 2.8, 1000.0, 100.0, 0.0))
            top = zc + l
            prev_l = l
        link7 = 8
        # two box fingers on prismatic joints along +y / -y above the last link
        fh = (0.01, 0.01, 0.03)
        anchor_z = prev_l + r + fh[2]
        for sgn, qf in ((1.0, qy), (-1.0, qny)):
            s0 = 0.02
            bl.append(body(BOX, fh, 0.05, (0, sgn * s0, top + r + fh[2]), group=G_ARM,
                           mask=G_PLANE | G_CUBE))
            jl.append(joint(PRISMATIC, link7, len(bl) - 1,
                            (0, 0, anchor_z, *qf), (0, 0, 0, *qf),
                            0.0, 0.04, 1000.0, 100.0, s0))
            # child frame at the finger centre; parent frame on the link axis,
            # so the joint coordinate starts at s0 (the finger's offset).
        cx = 0.4 + 0.2 * (g.random() - 0.5)
        cy = 0.2 * (g.random() - 0.5)
        yaw = 2 * math.pi * g.random()
        bl.append(body(BOX, (0.02, 0.02, 0.02), 0.05, (cx, cy, 0.02),
                       axis_angle_quat((0, 0, 1), yaw), group=G_CUBE))
        envs_b.append(bl); envs_j.append(jl)

    def actions(step0, n):
        # one Philox stream per (step, kind); env e takes row e, so an env's
        # targets do not depend on the batch size.
        out = np.empty((n, n_envs, n_act), np.float32)
        for k in range(n):
            step = step0 + k
            gv = step_rng(seed, step, 0)
            gf = step_rng(seed, step, 1)
            out[k, :, :7] = gv.standard_normal((n_envs, 7)) * 0.3
            out[k, :, 7:] = gf.random((n_envs, 2)) * 0.04
        return out
    return pack("arm", envs_b, envs_j, params, n_act, seed, actions)


# ----------------------------------------------------------------------------
# Config "clutter": 1-32 random boxes/spheres/capsules dropped into a bin.
# ----------------------------------------------------------------------------
def make_clutter(n_envs=16384, seed=3) -> Scene:
    params = default_params(contact_capacity=384, pair_capacity=704)
    envs_b, envs_j = [], []
    for e in range(n_envs):
        g = rng(seed, e, 0)
        bl = [
            body(BOX, (0.15, 0.15, 0.01), 0.0, (0, 0, -0.01), mu=0.5, group=1),
            body(BOX, (0.01, 0.17, 0.1), 0.0, (0.16, 0, 0.1), mu=0.5, group=1),
            body(BOX, (0.01, 0.17, 0.1), 0.0, (-0.16, 0, 0.1), mu=0.5, group=1),
            body(BOX, (0.15, 0.01, 0.1), 0.0, (0, 0.16, 0.1), mu=0.5, group=1),
            body(BOX, (0.15, 0.01, 0.1), 0.0, (0, -0.16, 0.1), mu=0.5, group=1),
        ]
        n = int(g.integers(1, 33))
        placed = []
        lo, hi = np.array([-0.12, -0.12, 0.02]), np.array([0.12, 0.12, 0.6])

        def inside_bin(c, rr):
            return abs(c[0]) + rr <= 0.149 and abs(c[1]) + rr <= 0.149 and c[2] - rr >= 0.001
        for _ in range(n):
            u = g.random()
            kind = BOX if u < 0.4 else (SPHERE if u < 0.7 else CAPSULE)
            s = math.exp(math.log(0.01) + (math.log(0.1) - math.log(0.01)) * g.random())
            dens = 500 + 1500 * g.random()
            mu = 0.3 + 0.7 * g.random()
            if kind == SPHERE:
                p = (s / 2, 0, 0); vol = 4 / 3 * math.pi * (s / 2) ** 3; rb = s / 2
            elif kind == BOX:
                hs = [math.exp(math.log(0.01) + (math.log(0.1) - math.log(0.01)) * g.random()) / 2
                      for _ in range(2)]
                hx, hy, hz = s / 2, hs[0], hs[1]
                p = (hx, hy, hz); vol = 8 * hx * hy * hz; rb = math.sqrt(hx * hx + hy * hy + hz * hz)
            else:
                rc, lc = s / 4, s / 2
                p = (rc, lc, 0)
                vol = math.pi * rc * rc * 2 * lc + 4 / 3 * math.pi * rc ** 3; rb = lc + rc
            q = shoemake_quat(g)
            c = _place(g, rb, lo, hi, placed, extra_ok=inside_bin)
            placed.append((c, rb))
            bl.append(body(kind, p, dens * vol, c, q, mu=mu, group=2))
        envs_b.append(bl); envs_j.append([])
    return pack("clutter", envs_b, envs_j, params, 0, seed)


# ----------------------------------------------------------------------------
# Config "hand": static palm, 4 fingers x (static base + 4 driven capsule links),
# cube resting on the palm.
# ----------------------------------------------------------------------------
def make_hand(n_envs=4096, seed=4, kp=10.0, kd=0.3) -> Scene:
    dt = 1.0 / 120.0
    params = default_params(dt=dt, substeps=8, pos_iters=16, vel_iters=1,
                            contact_capacity=64, pair_capacity=256)
    envs_b, envs_j = [], []
    n_act = 16
    r, l, m = 0.01, 0.02, 0.03
    periods = np.zeros((n_envs, n_act)); phases = np.zeros((n_envs, n_act))
    for e in range(n_envs):
        g = rng(seed, e, 0)
        bl = [body(BOX, (0.05, 0.05, 0.01), 0.0, (0, 0, 0), mu=0.8, group=1),
              body(BOX, (0.035, 0.035, 0.035), 0.1, (0, 0, 0.045), mu=0.8, group=2)]
        jl = []
        for f in range(4):
            th = f * math.pi / 2
            rad = np.array([math.cos(th), math.sin(th), 0.0])
            q_abd = axis_angle_quat((0, 0, 1), th)                 # +x -> radial
            q_curl = axis_angle_quat((0, 0, 1), th + math.pi / 2)  # +x -> tangent
            gf = 1 << (2 + f)
            mask = ALL_GROUPS & ~gf
            xy = rad * 0.048
            # 2 mm above the palm so that no capsule-cube gap equals the margin
            zc = 0.012 + r + l
            bl.append(body(CAPSULE, (r, l, 0), 0.0, (xy[0], xy[1], zc), mu=0.8, group=gf, mask=mask))
            parent = len(bl) - 1
            for k in range(4):
                zc = zc + 2 * l
                bl.append(body(CAPSULE, (r, l, 0), m, (xy[0], xy[1], zc), mu=0.8, group=gf, mask=mask))
                qa = q_abd if k == 0 else q_curl
                jl.append(joint(REVOLUTE, parent, len(bl) - 1, (0, 0, l, *qa), (0, 0, -l, *qa),
                                -1.6, 1.6, kp, kd, 0.0))
                parent = len(bl) - 1
        periods[e] = 1.0 + 2.0 * g.random(n_act)
        phases[e] = 2 * math.pi * g.random(n_act)
        envs_b.append(bl); envs_j.append(jl)

    def actions(step0, n):
        t = (step0 + np.arange(n, dtype=np.float64)) * dt
        a = 0.3 * np.sin(2 * math.pi * t[:, None, None] / periods[None] + phases[None])
        return a.astype(np.float32)
    return pack("hand", envs_b, envs_j, params, n_act, seed, actions)


# ----------------------------------------------------------------------------
# Config "pick": the arm envs driven by the pick task of the paper's sim2real
# appendix -- a target delta joint-position controller with normalised
# actions, proprioception, an is-grasped flag and the dense reward.
# ----------------------------------------------------------------------------
def pick_task(n_act=9) -> Dict:
    """Task descriptor of the arm envs (env-local indices: plane 0, fingers
    9 and 10, cube 11; joints 0-6 revolute, 7-8 the prismatic fingers).
    Delta bounds: +-0.05 rad per step for the revolute joints (the paper's
    Koch values), +-0.005 m for the fingers; grasp_tol 0.005 m on finger
    joint 7 (the paper's 0.02 is in radians for a revolute gripper); a
    finger within 1 mm of the table touches it.  float32 values, as the GPU
    path stores them."""
    lo = np.array([-0.05] * 7 + [-0.005] * 2, np.float32)
    return dict(grip_joint=7, finger_a=9, finger_b=10, cube=11, table=0,
                grasp_tol=float(np.float32(0.005)), touch_tol=float(np.float32(0.001)),
                delta_lo=lo[:n_act], delta_hi=-lo[:n_act])


def make_pick(n_envs=4096, seed=6, nan_frac=0.02, scale=0.7) -> Scene:
    sc = make_arm(n_envs=n_envs, seed=seed)
    A = sc.n_act

    def actions(step0, n):
        # normalised deltas ~ N(0, scale) (some beyond +-1: clipped by the
        # controller), nan_frac of the slots NaN (no change)
        out = np.empty((n, n_envs, A), np.float32)
        for k in range(n):
            g = step_rng(seed, step0 + k, 2)
            out[k] = g.standard_normal((n_envs, A)) * scale
            out[k][g.random((n_envs, A)) < nan_frac] = np.nan
        return out
    sc.name = "pick"
    sc.action_fn = actions
    sc.task = pick_task(A)
    return sc


# ----------------------------------------------------------------------------
# Cameras and body colours for the batched renderer (one camera per env, in
# the env's own frame; the paper's 128 x 128 RGB observation).
# ----------------------------------------------------------------------------
def default_camera(name: str, width=128, height=128) -> Dict:
    """A pinhole per env looking at the scene's working area."""
    if name in ("arm", "pick"):
        eye, target = (1.2, -0.9, 0.9), (0.25, 0.0, 0.25)
    elif name == "hand":
        eye, target = (0.25, -0.2, 0.25), (0.0, 0.0, 0.05)
    elif name == "hulls":
        eye, target = (0.25, -0.2, 0.6), (0.0, 0.0, 0.02)
    else:
        eye, target = (0.45, -0.35, 0.45), (0.0, 0.0, 0.05)
    return dict(eye=eye, target=target, fov_y=math.radians(60.0), near=0.01, width=width, height=height)


PALETTE = np.array([[0.85, 0.33, 0.10], [0.00, 0.45, 0.74], [0.93, 0.69, 0.13], [0.49, 0.18, 0.56],
                    [0.47, 0.67, 0.19], [0.30, 0.75, 0.93], [0.64, 0.08, 0.18], [0.75, 0.75, 0.75]], np.float32)


def body_colors(scene: "Scene") -> np.ndarray:
    """float32 [n_bodies][3]: planes grey, other bodies by env-local index."""
    out = np.empty((len(scene.bodies), 3), np.float32)
    for e in range(scene.n_envs):
        for i in range(scene.body_off[e], scene.body_off[e + 1]):
            k = i - scene.body_off[e]
            out[i] = (0.6, 0.6, 0.6) if scene.bodies["type"][i] == PLANE else PALETTE[k % len(PALETTE)]
    return out


# ----------------------------------------------------------------------------
# Config "mixed": heterogeneous articulations with per-env DOF in one batch --
# arm envs (9 joints), hand envs (16 joints) and clutter envs (no joint)
# interleaved (env e is of type e mod 3), under one set of solver parameters.
# ----------------------------------------------------------------------------
def make_mixed(n_envs=4096, seed=7) -> Scene:
    counts = [(n_envs + 2 - k) // 3 for k in range(3)]
    parts = [make_arm(counts[0], seed), make_hand(counts[1], seed + 1), make_clutter(counts[2], seed + 2)]
    common = default_params(contact_capacity=384, pair_capacity=704)
    for p in parts:
        p.params = dict(common)
    sc = concat(parts, name="mixed")
    offs = np.cumsum([0] + counts)
    out = sc.subset([int(offs[e % 3] + e // 3) for e in range(n_envs)])
    out.name = "mixed"
    return out


# ----------------------------------------------------------------------------
# Config "hulls": convex pieces of decomposed meshes dropped into a bin --
# random convex hulls (6-12 points in an ellipsoid), boxes as in clutter.
# ----------------------------------------------------------------------------
def make_hulls(n_envs=4096, seed=8, pool=128) -> Scene:
    """A pool of `pool` hull assets (asset k drawn from its own stream, so the
    pool does not depend on the batch); each env drops 1-12 of them, chosen
    and posed from the env's own stream, into the clutter bin."""
    from . import hulls as H
    params = default_params(contact_capacity=256, pair_capacity=256)
    assets = []
    for k in range(pool):
        ga = rng(seed, 1_000_000 + k, 1)
        semi = ga.uniform(0.015, 0.04, 3)
        assets.append(H.hull_asset(H.random_points(ga, int(ga.integers(6, 13)), semi)))
    radius = [H.bound_radius(v) for v, _ in assets]
    vol = [H.volume(v, t) for v, t in assets]
    envs_b, envs_j = [], []
    for e in range(n_envs):
        g = rng(seed, e, 0)
        bl = [
            body(BOX, (0.15, 0.15, 0.01), 0.0, (0, 0, -0.01), mu=0.5, group=1),
            body(BOX, (0.01, 0.17, 0.1), 0.0, (0.16, 0, 0.1), mu=0.5, group=1),
            body(BOX, (0.01, 0.17, 0.1), 0.0, (-0.16, 0, 0.1), mu=0.5, group=1),
            body(BOX, (0.17, 0.01, 0.1), 0.0, (0, 0.16, 0.1), mu=0.5, group=1),
            body(BOX, (0.17, 0.01, 0.1), 0.0, (0, -0.16, 0.1), mu=0.5, group=1),
        ]
        placed = []
        for _ in range(int(g.integers(1, 13))):
            k = int(g.integers(0, pool))
            c = _place(g, radius[k], np.array([-0.12, -0.12, 0.03]), np.array([0.12, 0.12, 0.5]), placed)
            placed.append((c, radius[k]))
            bl.append(body(HULL, (k, 0, 0), g.uniform(500.0, 2000.0) * vol[k], c, quat=shoemake_quat(g),
                           mu=float(g.uniform(0.3, 1.0)), group=2))
        envs_b.append(bl); envs_j.append([])
    sc = pack("hulls", envs_b, envs_j, params, 0, seed)
    sc.hulls = H.library(assets)
    return sc


CONFIGS = {
    "small": make_small,
    "arm": make_arm,
    "clutter": make_clutter,
    "hand": make_hand,
    "pick": make_pick,
    "mixed": make_mixed,
    "hulls": make_hulls,
}

CONFIG_SIZES = {"small": 64, "arm": 4096, "clutter": 16384, "hand": 4096, "pick": 4096, "mixed": 4096, "hulls": 4096}


def make_scene(name: str, n_envs: Optional[int] = None, seed: Optional[int] = None, **kw) -> Scene:
    fn = CONFIGS[name]
    args = {}
    if n_envs is not None:
        args["n_envs"] = n_envs
    if seed is not None:
        args["seed"] = seed
    args.update(kw)
    return fn(**args)


def concat(scenes: List[Scene], name="mixed") -> Scene:
    """Concatenate batches with equal solver parameters (heterogeneous batch)."""
    p0 = scenes[0].params
    for s in scenes[1:]:
        assert s.params == p0, "envs of one batch share solver parameters"
    bo, jo = [0], [0]
    for s in scenes:
        for e in range(s.n_envs):
            bo.append(bo[-1] + int(s.body_off[e + 1] - s.body_off[e]))
            jo.append(jo[-1] + int(s.joint_off[e + 1] - s.joint_off[e]))
    A = max(s.n_act for s in scenes)

    def fn(step0, n):
        outs = []
        for s in scenes:
            a = s.actions(step0, n)
            full = np.full((n, s.n_envs, A), np.nan, np.float32)
            if a is not None:
                full[:, :, :a.shape[2]] = a
            outs.append(full)
        return np.concatenate(outs, axis=1)
    return Scene(name, np.concatenate([s.bodies for s in scenes]), np.asarray(bo, np.int32),
                 np.concatenate([s.joints for s in scenes]), np.asarray(jo, np.int32),
                 dict(p0), A, scenes[0].seed, fn if A else None)
