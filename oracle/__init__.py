"""FP64 CPU oracle of the batched rigid-body step -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package's smoke check and the benchmark's CPU-baseline
leg import this module.  It loads ``liboracle.so`` (plain C, built from
``oracle.c`` with gcc, no fast-math) through ctypes; nothing here is shared
with the CUDA path.  ``build()`` compiles it in place.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "oracle.c")

# counter slots (oracle.h)
COUNTERS = ["steps", "pairs_tested", "pairs_candidate",
            "np_ss", "np_sc", "np_sb", "np_sp", "np_cc", "np_cb", "np_cp", "np_bb", "np_bp",
            "contact_points", "constraints", "rows_prep", "row_solve_2dyn", "row_solve_1dyn",
            "warm_apply", "body_integrate", "body_inertia", "colors", "np_sh", "np_xh", "np_hp",
            "sat_face_vert", "sat_edge_pair", "np_ch"]

ST_PAIR_OVERFLOW, ST_CONTACT_OVERFLOW, ST_COLOR_OVERFLOW = 1, 2, 4


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        cmd = ["gcc", "-O2", "-march=native", "-std=gnu11", "-fPIC", "-shared",
               "-o", LIB, SRC, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lp = C.POINTER(C.c_longlong)
        L.oracle_create.restype = P
        L.oracle_create.argtypes = [C.c_int, lp, dp, lp, dp, dp]
        L.oracle_create_hulls.restype = P
        L.oracle_create_hulls.argtypes = [C.c_int, lp, dp, lp, dp, dp, C.c_int, ip, dp, ip, ip]
        L.oracle_hull_inertia.argtypes = [dp, C.c_int, ip, C.c_int, C.c_double, dp]
        L.oracle_destroy.argtypes = [P]
        L.oracle_set_round32.argtypes = [P, C.c_int]
        L.oracle_step.argtypes = [P, dp, C.c_int, C.c_int, C.c_int]
        L.oracle_get_state.argtypes = [P, dp]
        L.oracle_contact_forces.argtypes = [P, dp]
        L.oracle_set_state.argtypes = [P, dp]
        L.oracle_get_targets.argtypes = [P, dp]
        L.oracle_set_targets.argtypes = [P, dp]
        L.oracle_env_status.restype = C.c_uint
        L.oracle_env_status.argtypes = [P, C.c_int]
        L.oracle_env_ties.restype = C.c_longlong
        L.oracle_env_ties.argtypes = [P, C.c_int]
        L.oracle_counters.argtypes = [P, lp]
        L.oracle_get_manifolds.argtypes = [P, C.c_int, C.c_int, ip, ip, dp]
        L.oracle_get_margin_ties.argtypes = [P, C.c_int, C.c_int, ip]
        L.oracle_get_colors.argtypes = [P, C.c_int, C.c_int, ip]
        L.oracle_get_rows.argtypes = [P, C.c_int, C.c_int, dp]
        L.oracle_collide.argtypes = [dp, dp, C.c_double, dp]
        L.oracle_color.argtypes = [C.c_int, ip, ip, ip, ip]
        L.oracle_candidates.argtypes = [dp, dp, C.c_double, dp]
        L.oracle_reduce4.argtypes = [C.c_int, dp, ip]
        L.oracle_tangents.argtypes = [dp, dp, dp]
        L.oracle_inertia.argtypes = [dp, dp]
        up = C.POINTER(C.c_ubyte)
        L.oracle_set_task.argtypes = [P, ip, dp, C.c_int, dp, dp]
        L.oracle_task_reset.argtypes = [P, up]
        L.oracle_step_task.argtypes = [P, dp, C.c_int, C.c_int, C.c_int, dp, up]
        L.oracle_task_observe.argtypes = [P, dp, up]
        L.oracle_render.argtypes = [P, dp, dp, up, dp, ip, up, C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_longlong))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_ubyte))


def body_rows(bodies) -> np.ndarray:
    """Scene body descriptors -> [n][22] float64 rows (exact conversion)."""
    n = len(bodies)
    out = np.zeros((n, 22), np.float64)
    out[:, 0] = bodies["type"]
    out[:, 1:4] = bodies["p"]
    out[:, 4] = bodies["mass"]
    out[:, 5:8] = bodies["pos"]
    out[:, 8:12] = bodies["quat"]
    out[:, 12:15] = bodies["linvel"]
    out[:, 15:18] = bodies["angvel"]
    out[:, 18] = bodies["mu"]
    out[:, 19] = bodies["restitution"]
    out[:, 20] = bodies["group"]
    out[:, 21] = bodies["mask"]
    return out


def joint_rows(joints) -> np.ndarray:
    n = len(joints)
    out = np.zeros((n, 22), np.float64)
    out[:, 0] = joints["type"]
    out[:, 1] = joints["parent"]
    out[:, 2] = joints["child"]
    out[:, 3:10] = joints["parent_frame"]
    out[:, 10:17] = joints["child_frame"]
    out[:, 17] = joints["lower"]
    out[:, 18] = joints["upper"]
    out[:, 19] = joints["kp"]
    out[:, 20] = joints["kd"]
    out[:, 21] = joints["target0"]
    return out


def param_row(p) -> np.ndarray:
    g = p["gravity"]
    return np.array([p["dt"], p["substeps"], p["pos_iters"], p["vel_iters"], g[0], g[1], g[2],
                     p["margin"], p["max_depen_vel"], p["contact_capacity"], p["pair_capacity"],
                     p.get("linear_damping", 0.0), p.get("angular_damping", 0.0),
                     p.get("bounce_threshold", 1.0), p.get("warm_start", 0),
                     p.get("contact_hertz", 0.0), p.get("contact_damping_ratio", 0.0),
                     p.get("joint_hertz", 0.0), p.get("joint_damping_ratio", 0.0)],
                    np.float64)


class Oracle:
    """One oracle world over a scene (every env of it)."""

    def __init__(self, scene, state_override=None):
        L = lib()
        self.scene = scene
        self.E = scene.n_envs
        self.nb = int(scene.body_off[-1])
        self.nj = int(scene.joint_off[-1])
        self._bo = np.ascontiguousarray(scene.body_off, np.int64)
        self._jo = np.ascontiguousarray(scene.joint_off, np.int64)
        self._b = np.ascontiguousarray(body_rows(scene.bodies))
        if state_override is not None:
            self._b[:, 5:8] = state_override[:, 0:3]
        self._j = np.ascontiguousarray(joint_rows(scene.joints)) if self.nj else np.zeros((1, 22))
        self._p = param_row(scene.params)
        hl = getattr(scene, "hulls", None)
        if hl is None:
            self.h = L.oracle_create(self.E, _lp(self._bo), _dp(self._b), _lp(self._jo), _dp(self._j),
                                     _dp(self._p))
        else:
            self._hv = np.ascontiguousarray(hl["verts"], np.float64).reshape(-1)
            self._hvo = np.ascontiguousarray(hl["vert_off"], np.int32)
            self._ht = np.ascontiguousarray(hl["tris"], np.int32).reshape(-1)
            self._hto = np.ascontiguousarray(hl["tri_off"], np.int32)
            self.h = L.oracle_create_hulls(self.E, _lp(self._bo), _dp(self._b), _lp(self._jo), _dp(self._j),
                                           _dp(self._p), len(self._hvo) - 1, _ip(self._hvo), _dp(self._hv),
                                           _ip(self._hto), _ip(self._ht))
            if not self.h:
                raise ValueError("malformed hull in the library")
        self.A = scene.n_act
        self.steps_done = 0

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_destroy(self.h)
            self.h = None

    def step(self, n_steps=1, actions=None, threads=1):
        """Advance n_steps; actions default to the scene's own for these steps."""
        if actions is None and self.A:
            actions = self.scene.actions(self.steps_done, n_steps)
        if actions is not None:
            a = np.ascontiguousarray(actions, np.float64)
            assert a.shape == (n_steps, self.E, self.A), a.shape
            lib().oracle_step(self.h, _dp(a), self.A, n_steps, threads)
        else:
            lib().oracle_step(self.h, None, 0, n_steps, threads)
        self.steps_done += n_steps

    # ------------------------------------------------------------ pick task
    def set_task(self, task):
        """task: dict with grip_joint, finger_a, finger_b, cube, table,
        grasp_tol, touch_tol, delta_lo[A], delta_hi[A] (scenegen.pick_task)."""
        idx = np.array([task["grip_joint"], task["finger_a"], task["finger_b"], task["cube"], task["table"]],
                       np.int32)
        tol = np.array([task["grasp_tol"], task["touch_tol"]], np.float64)
        lo = np.ascontiguousarray(task["delta_lo"], np.float64)
        hi = np.ascontiguousarray(task["delta_hi"], np.float64)
        assert len(lo) == len(hi) == self.A
        if lib().oracle_set_task(self.h, _ip(idx), _dp(tol), self.A, _dp(lo), _dp(hi)) != 0:
            raise ValueError("task indices out of range or of the wrong body type")
        self.D = 10 + 2 * self.A

    def task_reset(self, mask=None):
        m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
        lib().oracle_task_reset(self.h, None if m is None else _up(m))

    def step_task(self, n_steps=1, actions=None, threads=1):
        """Advance n_steps with the task's controller; returns the records
        [n_steps][E][D] and the tie masks [n_steps][E]."""
        if actions is None:
            actions = self.scene.actions(self.steps_done, n_steps)
        a = np.ascontiguousarray(actions, np.float64)
        assert a.shape == (n_steps, self.E, self.A), a.shape
        out = np.zeros((n_steps, self.E, self.D), np.float64)
        ties = np.zeros((n_steps, self.E), np.uint8)
        if lib().oracle_step_task(self.h, _dp(a), self.A, n_steps, threads, _dp(out), _up(ties)) != 0:
            raise RuntimeError("no task set")
        self.steps_done += n_steps
        return out, ties

    def observe(self):
        """The task record of every env at the current state: [E][D], ties [E]."""
        out = np.zeros((self.E, self.D), np.float64)
        ties = np.zeros(self.E, np.uint8)
        if lib().oracle_task_observe(self.h, _dp(out), _up(ties)) != 0:
            raise RuntimeError("no task set")
        return out, ties

    def render(self, camera, body_rgb, threads=8):
        """camera: dict eye, target, fov_y, near, width, height; body_rgb
        [n_bodies][3].  Returns rgb uint8 [E,H,W,3], depth [E,H,W], seg int32
        [E,H,W], ties uint8 [E,H,W]."""
        W, H = int(camera["width"]), int(camera["height"])
        cam = np.array([*camera["eye"], *camera["target"], camera["fov_y"], camera["near"], W, H], np.float64)
        col = np.ascontiguousarray(body_rgb, np.float64)
        assert col.shape == (self.nb, 3)
        rgb = np.zeros((self.E, H, W, 3), np.uint8)
        depth = np.zeros((self.E, H, W), np.float64)
        seg = np.zeros((self.E, H, W), np.int32)
        ties = np.zeros((self.E, H, W), np.uint8)
        if lib().oracle_render(self.h, _dp(cam), _dp(col), _up(rgb), _dp(depth), _ip(seg), _up(ties), threads) != 0:
            raise ValueError("degenerate camera")
        return rgb, depth, seg, ties

    def state(self) -> np.ndarray:
        out = np.zeros((self.nb, 13), np.float64)
        lib().oracle_get_state(self.h, _dp(out))
        return out

    def contact_forces(self) -> np.ndarray:
        """Per body (F[3], f_n) of the last step: contact impulses over the
        last substep / h (oracle_contact_forces)."""
        out = np.zeros((self.nb, 4), np.float64)
        lib().oracle_contact_forces(self.h, _dp(out))
        return out

    def set_round32(self, on: bool):
        """Test probe: store state, rows, impulses and contact data as float32."""
        lib().oracle_set_round32(self.h, 1 if on else 0)

    def set_state(self, st):
        st = np.ascontiguousarray(st, np.float64)
        lib().oracle_set_state(self.h, _dp(st))

    def targets(self) -> np.ndarray:
        out = np.zeros(max(self.nj, 1), np.float64)
        lib().oracle_get_targets(self.h, _dp(out))
        return out[:self.nj]

    def set_targets(self, t):
        t = np.ascontiguousarray(t, np.float64)
        assert t.shape == (self.nj,)
        lib().oracle_set_targets(self.h, _dp(t))

    def status(self, env) -> int:
        return int(lib().oracle_env_status(self.h, env))

    def ties(self, env) -> int:
        return int(lib().oracle_env_ties(self.h, env))

    def counters(self) -> dict:
        out = np.zeros(len(COUNTERS), np.int64)
        lib().oracle_counters(self.h, _lp(out))
        return dict(zip(COUNTERS, out.tolist()))

    def manifolds(self, env, cap=1024):
        pairs = np.zeros((cap, 2), np.int32)
        npts = np.zeros(cap, np.int32)
        pts = np.zeros((cap, 4, 10), np.float64)
        n = lib().oracle_get_manifolds(self.h, env, cap, _ip(pairs), _ip(npts), _dp(pts))
        n = min(n, cap)
        return pairs[:n], npts[:n], pts[:n]

    def margin_ties(self, env, cap=1024):
        pairs = np.zeros((cap, 2), np.int32)
        n = lib().oracle_get_margin_ties(self.h, env, cap, _ip(pairs))
        return pairs[:min(n, cap)]

    def colors(self, env, cap=4096):
        out = np.zeros(cap, np.int32)
        n = lib().oracle_get_colors(self.h, env, cap, _ip(out))
        return out[:min(n, cap)]

    def rows(self, env, cap=8192):
        out = np.zeros((cap, 16), np.float64)
        n = lib().oracle_get_rows(self.h, env, cap, _dp(out))
        return out[:min(n, cap)]


def collide(body_a, body_b, margin=0.01):
    """Narrowphase of one ordered pair (descriptor records or 22-rows)."""
    a = np.ascontiguousarray(body_a if np.ndim(body_a) == 1 and len(body_a) == 22
                             else body_rows(np.atleast_1d(body_a))[0], np.float64)
    b = np.ascontiguousarray(body_b if np.ndim(body_b) == 1 and len(body_b) == 22
                             else body_rows(np.atleast_1d(body_b))[0], np.float64)
    out = np.zeros((8, 10), np.float64)
    n = lib().oracle_collide(_dp(a), _dp(b), margin, _dp(out))
    return out[:n]


def candidates(body_a, body_b, margin=0.01):
    """Candidate points of one ordered pair (22-rows) before the margin
    filter and the reduction to 4: [n][10] = cA, cB, n, d."""
    a = np.ascontiguousarray(body_a, np.float64)
    b = np.ascontiguousarray(body_b, np.float64)
    out = np.zeros((16, 10), np.float64)
    n = lib().oracle_candidates(_dp(a), _dp(b), margin, _dp(out))
    return out[:n]


def reduce4(pts):
    """Indices p1..p4 the manifold reduction keeps of [n][10] candidates."""
    p = np.ascontiguousarray(pts, np.float64)
    sel = np.zeros(4, np.int32)
    if lib().oracle_reduce4(len(p), _dp(p), _ip(sel)) != 4:
        raise ValueError("5 to 16 candidates")
    return sel


def tangents(n):
    """Contact tangent basis (t1, t2) of a unit normal."""
    nn = np.ascontiguousarray(n, np.float64)
    t1, t2 = np.zeros(3), np.zeros(3)
    lib().oracle_tangents(_dp(nn), _dp(t1), _dp(t2))
    return t1, t2


def color(a, b, dyn):
    a = np.ascontiguousarray(a, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    dyn = np.ascontiguousarray(dyn, np.int32)
    out = np.zeros(max(len(a), 1), np.int32)
    nc = lib().oracle_color(len(a), _ip(a), _ip(b), _ip(dyn), _ip(out))
    return nc, out[:len(a)]


def hull_inertia(verts, tris, mass):
    v = np.ascontiguousarray(verts, np.float64).reshape(-1)
    t = np.ascontiguousarray(tris, np.int32).reshape(-1)
    out = np.zeros(3, np.float64)
    if lib().oracle_hull_inertia(_dp(v), len(v) // 3, _ip(t), len(t) // 3, mass, _dp(out)) != 0:
        raise ValueError("malformed hull")
    return out


def inertia(body_row):
    r = np.ascontiguousarray(body_row, np.float64)
    out = np.zeros(3, np.float64)
    lib().oracle_inertia(_dp(r), _dp(out))
    return out
