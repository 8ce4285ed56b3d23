"""ctypes binding of libmsim.so (include/ms.h): argument marshalling only.

Every function keeps the C name.  Device buffers are passed as torch CUDA
tensors (their data_ptr) and streams as torch.cuda.Stream (their raw
handle); nothing here computes any part of the step.  Loading fails loudly
when the library is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsim.so")

MS_OK = 0
STATUS_NAMES = {0: "MS_OK", 1: "MS_ERR_INVALID_ARG", 2: "MS_ERR_OOM", 3: "MS_ERR_CUDA",
                4: "MS_ERR_CONTACT_OVERFLOW", 5: "MS_ERR_COLOR_OVERFLOW", 6: "MS_ERR_NAN",
                7: "MS_ERR_TIMEOUT", 8: "MS_ERR_NOT_ADMITTED", 9: "MS_ERR_BUSY",
                10: "MS_ERR_PAIR_OVERFLOW", 11: "MS_ERR_NOT_FOUND"}
ENV_PAIR_OVERFLOW, ENV_CONTACT_OVERFLOW, ENV_COLOR_OVERFLOW, ENV_NAN = 1, 2, 4, 8


class MSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class ms_sim_params(C.Structure):
    _fields_ = [("dt", C.c_float), ("substeps", C.c_int32), ("pos_iters", C.c_int32),
                ("vel_iters", C.c_int32), ("gravity", C.c_float * 3), ("margin", C.c_float),
                ("max_depen_vel", C.c_float), ("contact_capacity", C.c_int32),
                ("pair_capacity", C.c_int32), ("linear_damping", C.c_float), ("angular_damping", C.c_float),
                ("bounce_threshold", C.c_float), ("warm_start", C.c_int32),
                ("contact_hertz", C.c_float), ("contact_damping_ratio", C.c_float),
                ("joint_hertz", C.c_float), ("joint_damping_ratio", C.c_float)]


class ms_scene_desc(C.Structure):
    _fields_ = [("n_bodies", C.c_int32), ("n_joints", C.c_int32),
                ("bodies", C.c_void_p), ("joints", C.c_void_p)]


class ms_state_view(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("n_bodies", C.c_int32), ("n_joints", C.c_int32),
                ("max_act", C.c_int32), ("x", C.c_void_p), ("q", C.c_void_p), ("v", C.c_void_p),
                ("w", C.c_void_p), ("body_off", C.c_void_p), ("joint_off", C.c_void_p),
                ("targets", C.c_void_p), ("status", C.c_void_p)]


class ms_noalloc_batch(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("max_bodies_per_env", C.c_int32), ("max_joints_per_env", C.c_int32),
                ("body_off", C.c_void_p), ("joint_off", C.c_void_p), ("bodies", C.c_void_p),
                ("joints", C.c_void_p), ("x", C.c_void_p), ("q", C.c_void_p), ("v", C.c_void_p),
                ("w", C.c_void_p), ("targets", C.c_void_p), ("status", C.c_void_p)]


class ms_task_desc(C.Structure):
    _fields_ = [("grip_joint", C.c_int32), ("finger_a", C.c_int32), ("finger_b", C.c_int32),
                ("cube", C.c_int32), ("table", C.c_int32), ("grasp_tol", C.c_float), ("touch_tol", C.c_float),
                ("n_joints", C.c_int32), ("delta_lo", C.c_void_p), ("delta_hi", C.c_void_p)]


MS_STEP_PLAIN = 1


class ms_hull_lib(C.Structure):
    _fields_ = [("n_hulls", C.c_int32), ("vert_off", C.c_void_p), ("verts", C.c_void_p), ("tri_off", C.c_void_p),
                ("tris", C.c_void_p)]


class ms_camera_desc(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("fov_y", C.c_float), ("near", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("body_rgb", C.c_void_p)]


class ms_tuning(C.Structure):
    _fields_ = [("lanes_per_env", C.c_int32), ("warps_per_cta", C.c_int32),
                ("rows_in_smem", C.c_int32), ("ctas_per_sm", C.c_int32)]


_lib = None

# (name, restype, argtypes)
_SIGS = [
    ("ms_create_batch", C.c_int, [C.c_void_p, C.c_int, C.POINTER(ms_sim_params), C.POINTER(C.c_void_p)]),
    ("ms_create_batch_flat", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.POINTER(ms_sim_params), C.POINTER(C.c_void_p)]),
    ("ms_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("ms_step_plain", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("ms_get_state", C.c_int, [C.c_void_p, C.POINTER(ms_state_view)]),
    ("ms_copy_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("ms_set_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("ms_sync", C.c_int, [C.c_void_p, C.c_void_p]),
    ("ms_destroy", C.c_int, [C.c_void_p]),
    ("ms_last_error", C.c_char_p, []),
    ("ms_set_record_contacts", C.c_int, [C.c_void_p, C.c_int]),
    ("ms_enable_contact_forces", C.c_int, [C.c_void_p, C.c_int]),
    ("ms_contact_forces", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ms_get_colors", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_int)]),
    ("ms_get_contacts", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(C.c_int)]),
    ("ms_set_tuning", C.c_int, [C.c_void_p, C.POINTER(ms_tuning)]),
    ("ms_get_tuning", C.c_int, [C.c_void_p, C.POINTER(ms_tuning)]),
    ("ms_autotune", C.c_int, [C.c_void_p, C.c_int, C.c_char_p, C.POINTER(ms_tuning), C.c_void_p]),
    ("ms_memory_bytes", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("ms_estimate_bytes", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(ms_sim_params),
                                    C.POINTER(C.c_size_t)]),
    ("ms_abi_sizes", None, [C.c_void_p]),
    ("ms_step_noalloc", C.c_int, [C.c_void_p, C.POINTER(ms_sim_params), C.c_void_p, C.c_int, C.c_void_p]),
    ("ms_set_task", C.c_int, [C.c_void_p, C.POINTER(ms_task_desc), C.c_void_p]),
    ("ms_task_reset", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ms_task_record_len", C.c_int, [C.c_void_p]),
    ("ms_task_observe", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ms_step_ex", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    ("ms_step_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    ("ms_set_allocator", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ms_set_camera", C.c_int, [C.c_void_p, C.POINTER(ms_camera_desc)]),
    ("ms_create_batch_hulls", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                        C.POINTER(ms_sim_params), C.POINTER(ms_hull_lib), C.POINTER(C.c_void_p)]),
    ("ms_render", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ms_measure_fp32_peak", C.c_int, [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                       C.POINTER(C.c_double)]),
]

EXPORTS = [s[0] for s in _SIGS]


def load(path: str = LIB_PATH):
    """Load libmsim.so; raises if it is missing (build it with
    ``python -m paper_2410_00425_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libmsim.so not built at {path}; run python -m paper_2410_00425_b300.build")
        lib = C.CDLL(path)
        for name, res, args in _SIGS:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        sizes = (C.c_int32 * 5)()
        lib.ms_abi_sizes(sizes)
        expect = [84, 88, C.sizeof(ms_sim_params), C.sizeof(ms_state_view), C.sizeof(ms_tuning)]
        if list(sizes) != expect:
            raise ImportError(f"ABI layout mismatch: library {list(sizes)} vs binding {expect}")
        _lib = lib
    return _lib


def check(code: int):
    if code != MS_OK:
        raise MSError(code, load().ms_last_error().decode())
    return code


def _ptr(t):
    """Raw pointer of a torch tensor / numpy array / None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def make_params(p: dict) -> ms_sim_params:
    sp = ms_sim_params()
    sp.dt = p["dt"]; sp.substeps = p["substeps"]; sp.pos_iters = p["pos_iters"]
    sp.vel_iters = p["vel_iters"]
    for i in range(3):
        sp.gravity[i] = p["gravity"][i]
    sp.margin = p["margin"]; sp.max_depen_vel = p["max_depen_vel"]
    sp.contact_capacity = p["contact_capacity"]; sp.pair_capacity = p["pair_capacity"]
    sp.linear_damping = p.get("linear_damping", 0.0); sp.angular_damping = p.get("angular_damping", 0.0)
    sp.bounce_threshold = p.get("bounce_threshold", 1.0); sp.warm_start = int(p.get("warm_start", 0))
    sp.contact_hertz = p.get("contact_hertz", 0.0); sp.contact_damping_ratio = p.get("contact_damping_ratio", 0.0)
    sp.joint_hertz = p.get("joint_hertz", 0.0); sp.joint_damping_ratio = p.get("joint_damping_ratio", 0.0)
    return sp


# ---- thin wrappers with the C names -------------------------------------
def ms_create_batch_flat(bodies: np.ndarray, body_off: np.ndarray, joints: np.ndarray,
                         joint_off: np.ndarray, params: dict, hulls=None) -> int:
    """hulls: a hull library dict (verts, vert_off, tris, tri_off) or None."""
    L = load()
    if hulls is not None:
        hv = np.ascontiguousarray(hulls["verts"], np.float32)
        hvo = np.ascontiguousarray(hulls["vert_off"], np.int32)
        ht = np.ascontiguousarray(hulls["tris"], np.int32)
        hto = np.ascontiguousarray(hulls["tri_off"], np.int32)
        lib = ms_hull_lib(len(hvo) - 1, hvo.ctypes.data, hv.ctypes.data, hto.ctypes.data, ht.ctypes.data)
        bodies = np.ascontiguousarray(bodies)
        joints = np.ascontiguousarray(joints)
        bo = np.ascontiguousarray(body_off, np.int32)
        jo = np.ascontiguousarray(joint_off, np.int32)
        out = C.c_void_p()
        sp = make_params(params)
        check(L.ms_create_batch_hulls(bodies.ctypes.data, bo.ctypes.data, joints.ctypes.data if len(joints) else None,
                                      jo.ctypes.data, len(bo) - 1, C.byref(sp), C.byref(lib), C.byref(out)))
        return out.value
    bodies = np.ascontiguousarray(bodies)
    joints = np.ascontiguousarray(joints)
    bo = np.ascontiguousarray(body_off, np.int32)
    jo = np.ascontiguousarray(joint_off, np.int32)
    out = C.c_void_p()
    sp = make_params(params)
    check(L.ms_create_batch_flat(bodies.ctypes.data, bo.ctypes.data,
                                 joints.ctypes.data if len(joints) else None, jo.ctypes.data,
                                 len(bo) - 1, C.byref(sp), C.byref(out)))
    return out.value


def ms_create_batch(descs, n_envs: int, params: dict) -> int:
    """descs: ctypes array of ms_scene_desc."""
    L = load()
    out = C.c_void_p()
    sp = make_params(params)
    check(L.ms_create_batch(C.cast(descs, C.c_void_p), n_envs, C.byref(sp), C.byref(out)))
    return out.value


def ms_step(b, actions=None, n_steps=1, stream=None):
    return check(load().ms_step(b, _ptr(actions), n_steps, _stream(stream)))


def ms_step_plain(b, actions=None, n_steps=1, stream=None):
    return check(load().ms_step_plain(b, _ptr(actions), n_steps, _stream(stream)))


def ms_step_ex(b, actions=None, n_steps=1, out=None, flags=0, stream=None):
    return check(load().ms_step_ex(b, _ptr(actions), n_steps, _ptr(out), flags, _stream(stream)))


def ms_step_host(b, actions=None, n_steps=1, out=None, out_kind=0, stream=None):
    """actions, out: host buffers (pinned tensors or arrays)."""
    return check(load().ms_step_host(b, _ptr(actions), n_steps, _ptr(out), out_kind, _stream(stream)))


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p)
_hook = None                                   # the installed callbacks, kept alive


def ms_set_allocator(alloc=None, free=None):
    """alloc(bytes, device, stream) -> int pointer (0 on failure), free(ptr,
    device, stream): Python callables, or None and None for the library's pool."""
    global _hook
    if alloc is None and free is None:
        check(load().ms_set_allocator(None, None, None))
        _hook = None
        return
    a = ALLOC_FN(lambda n, d, st, u: alloc(n, d, st) or None)
    f = FREE_FN(lambda p, d, st, u: free(p, d, st))
    check(load().ms_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None))
    _hook = (a, f)


def ms_set_task(b, task, stream=None):
    """task: dict (grip_joint, finger_a, finger_b, cube, table, grasp_tol,
    touch_tol, delta_lo[A], delta_hi[A]) or None to remove it."""
    L = load()
    if task is None:
        return check(L.ms_set_task(b, None, _stream(stream)))
    lo = np.ascontiguousarray(task["delta_lo"], np.float32)
    hi = np.ascontiguousarray(task["delta_hi"], np.float32)
    t = ms_task_desc(int(task["grip_joint"]), int(task["finger_a"]), int(task["finger_b"]), int(task["cube"]),
                     int(task["table"]), float(task["grasp_tol"]), float(task["touch_tol"]), len(lo),
                     lo.ctypes.data, hi.ctypes.data)
    return check(L.ms_set_task(b, C.byref(t), _stream(stream)))


def ms_task_reset(b, env_mask=None, stream=None):
    m = None if env_mask is None else np.ascontiguousarray(env_mask, np.uint8)
    return check(load().ms_task_reset(b, None if m is None else m.ctypes.data, _stream(stream)))


def ms_task_record_len(b) -> int:
    return int(load().ms_task_record_len(b))


def ms_task_observe(b, out, stream=None):
    return check(load().ms_task_observe(b, _ptr(out), _stream(stream)))


def ms_set_camera(b, camera, body_rgb):
    """camera: dict eye, target, fov_y, near, width, height; body_rgb
    float [n_bodies][3] (host)."""
    col = np.ascontiguousarray(body_rgb, np.float32)
    c = ms_camera_desc()
    for i in range(3):
        c.eye[i] = camera["eye"][i]
        c.target[i] = camera["target"][i]
    c.fov_y = camera["fov_y"]; c.near = camera["near"]
    c.width = int(camera["width"]); c.height = int(camera["height"])
    c.body_rgb = col.ctypes.data
    return check(load().ms_set_camera(b, C.byref(c)))


def ms_render(b, rgba=None, depth=None, seg=None, stream=None):
    return check(load().ms_render(b, _ptr(rgba), _ptr(depth), _ptr(seg), _stream(stream)))


def ms_get_state(b) -> ms_state_view:
    v = ms_state_view()
    check(load().ms_get_state(b, C.byref(v)))
    return v


def ms_copy_state(b, dst, dst_kind, stream=None):
    return check(load().ms_copy_state(b, _ptr(dst), dst_kind, _stream(stream)))


def ms_set_state(b, src, src_kind, env_mask=None, stream=None):
    m = None if env_mask is None else np.ascontiguousarray(env_mask, np.uint8)
    return check(load().ms_set_state(b, _ptr(src), src_kind, None if m is None else m.ctypes.data,
                                     _stream(stream)))


def ms_sync(b):
    """Returns (status code, per-env status bits) without raising."""
    v = ms_get_state(b)
    st = np.zeros(v.n_envs, np.uint32)
    code = load().ms_sync(b, st.ctypes.data)
    return code, st


def ms_destroy(b):
    return check(load().ms_destroy(b))


def ms_last_error() -> str:
    return load().ms_last_error().decode()


def ms_set_record_contacts(b, record=True):
    return check(load().ms_set_record_contacts(b, int(record)))


def ms_enable_contact_forces(b, on=True):
    return check(load().ms_enable_contact_forces(b, int(on)))


def ms_contact_forces(b, out, stream=None):
    return check(load().ms_contact_forces(b, _ptr(out), _stream(stream)))


def ms_get_contacts(b, env, cap=1024):
    pairs = np.zeros((cap, 2), np.int32)
    npts = np.zeros(cap, np.int32)
    pts = np.zeros((cap, 4, 10), np.float32)
    n = C.c_int()
    check(load().ms_get_contacts(b, env, cap, pairs.ctypes.data, npts.ctypes.data, pts.ctypes.data,
                                 C.byref(n)))
    m = min(n.value, cap)
    return pairs[:m], npts[:m], pts[:m]


def ms_set_tuning(b, lanes_per_env, warps_per_cta, rows_in_smem):
    t = ms_tuning(lanes_per_env, warps_per_cta, rows_in_smem, 0)
    return check(load().ms_set_tuning(b, C.byref(t)))


def ms_get_tuning(b) -> dict:
    t = ms_tuning()
    check(load().ms_get_tuning(b, C.byref(t)))
    return dict(lanes_per_env=t.lanes_per_env, warps_per_cta=t.warps_per_cta,
                rows_in_smem=t.rows_in_smem, ctas_per_sm=t.ctas_per_sm)


def ms_autotune(b, n_steps=1, cache_path=None, stream=None) -> dict:
    t = ms_tuning()
    check(load().ms_autotune(b, n_steps, cache_path.encode() if cache_path else None, C.byref(t),
                             _stream(stream)))
    return dict(lanes_per_env=t.lanes_per_env, warps_per_cta=t.warps_per_cta,
                rows_in_smem=t.rows_in_smem, ctas_per_sm=t.ctas_per_sm)


def ms_step_noalloc(nb: ms_noalloc_batch, params: dict, actions=None, n_steps=1, stream=None):
    sp = make_params(params)
    return check(load().ms_step_noalloc(C.byref(nb), C.byref(sp), _ptr(actions), n_steps, _stream(stream)))


def ms_memory_bytes(b) -> int:
    n = C.c_size_t()
    check(load().ms_memory_bytes(b, C.byref(n)))
    return n.value


def ms_estimate_bytes(body_off, joint_off, params: dict) -> int:
    bo = np.ascontiguousarray(body_off, np.int32)
    jo = np.ascontiguousarray(joint_off, np.int32)
    n = C.c_size_t()
    sp = make_params(params)
    check(load().ms_estimate_bytes(bo.ctypes.data, jo.ctypes.data, len(bo) - 1, C.byref(sp), C.byref(n)))
    return n.value


def ms_measure_fp32_peak(seconds: float = 0.5):
    """Measured FP32 FMA rate of the current device: (flop/s, SMs, timed s)."""
    L = load()
    f, n, t = C.c_double(), C.c_int(), C.c_double()
    check(L.ms_measure_fp32_peak(seconds, C.byref(f), C.byref(n), C.byref(t)))
    return f.value, n.value, t.value


def ms_get_colors(b, env: int, cap: int = 4096) -> np.ndarray:
    """Colours of env `env`'s constraints at its last step (recording on)."""
    out = np.zeros(cap, np.int32)
    n = C.c_int()
    check(load().ms_get_colors(b, env, cap, out.ctypes.data, C.byref(n)))
    return out[:min(n.value, cap)]
