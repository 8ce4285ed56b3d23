"""ctypes binding of the step server (include/ms_server.h): marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _ffi


class ms_server_options(C.Structure):
    _fields_ = [("merge", C.c_int32), ("max_requests", C.c_int32), ("coalesce_us", C.c_double),
                ("max_inflight", C.c_int32)]


class ms_request_result(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("session", C.c_uint64), ("done", C.c_int32), ("status", C.c_int32),
                ("t_arrive", C.c_double), ("t_done", C.c_double), ("latency", C.c_double),
                ("launch_envs", C.c_int32)]


class ms_server_stats(C.Structure):
    _fields_ = [("sessions_open", C.c_uint64), ("sessions_admitted", C.c_uint64),
                ("sessions_rejected", C.c_uint64), ("requests_done", C.c_uint64), ("launches", C.c_uint64),
                ("env_steps", C.c_uint64), ("hbm_used", C.c_size_t), ("hbm_budget", C.c_size_t),
                ("p50", C.c_double), ("p99", C.c_double), ("mean", C.c_double), ("busy_s", C.c_double),
                ("graph_captures", C.c_uint64), ("launch_p50", C.c_double), ("launch_p99", C.c_double),
                ("launch_max", C.c_double), ("queue_p50", C.c_double), ("queue_p99", C.c_double),
                ("stage_p99", C.c_double), ("stage_max", C.c_double)]


_SIGS = [
    ("ms_server_create", C.c_int, [C.c_size_t, C.POINTER(ms_server_options), C.POINTER(C.c_void_p)]),
    ("ms_server_open", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.POINTER(_ffi.ms_sim_params), C.POINTER(C.c_uint64)]),
    ("ms_server_close", C.c_int, [C.c_void_p, C.c_uint64]),
    ("ms_server_submit", C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_uint64)]),
    ("ms_server_poll", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(ms_request_result)]),
    ("ms_server_drain", C.c_int, [C.c_void_p]),
    ("ms_server_copy_state", C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p]),
    ("ms_server_stats_get", C.c_int, [C.c_void_p, C.POINTER(ms_server_stats)]),
    ("ms_server_reset_stats", C.c_int, [C.c_void_p]),
    ("ms_server_destroy", C.c_int, [C.c_void_p]),
    ("ms_server_now", C.c_double, []),
]
EXPORTS = [s[0] for s in _SIGS]
_bound = False


def lib():
    global _bound
    L = _ffi.load()
    if not _bound:
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return L


class Server:
    """One ms_server: sessions of resident envs, step requests, latency stats."""

    def __init__(self, hbm_budget_bytes: int, merge: bool = True, max_requests: int = 0, coalesce_us: float = 0.0,
                 max_inflight: int = 0):
        L = lib()
        o = ms_server_options(int(merge), int(max_requests), float(coalesce_us), int(max_inflight))
        h = C.c_void_p()
        _ffi.check(L.ms_server_create(int(hbm_budget_bytes), C.byref(o), C.byref(h)))
        self.h = h.value
        self.n_act = {}

    def close(self):
        if getattr(self, "h", None):
            lib().ms_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open(self, scene):
        """Open a session with the scene's envs; returns the session id, or
        None when the server does not admit it (HBM budget)."""
        L = lib()
        bodies = np.ascontiguousarray(scene.bodies)
        joints = np.ascontiguousarray(scene.joints)
        bo = np.ascontiguousarray(scene.body_off, np.int32)
        jo = np.ascontiguousarray(scene.joint_off, np.int32)
        sp = _ffi.make_params(scene.params)
        sid = C.c_uint64()
        code = L.ms_server_open(self.h, bodies.ctypes.data, bo.ctypes.data,
                                joints.ctypes.data if len(joints) else None, jo.ctypes.data,
                                scene.n_envs, C.byref(sp), C.byref(sid))
        if code == 8:          # MS_ERR_NOT_ADMITTED
            return None
        _ffi.check(code)
        self.n_act[sid.value] = int(np.diff(jo).max()) if scene.n_envs else 0
        return sid.value

    def close_session(self, sid):
        _ffi.check(lib().ms_server_close(self.h, sid))
        self.n_act.pop(sid, None)

    def submit(self, sid, actions=None) -> int:
        t = C.c_uint64()
        a = None if actions is None else np.ascontiguousarray(actions, np.float32)
        _ffi.check(lib().ms_server_submit(self.h, sid, None if a is None else a.ctypes.data, C.byref(t)))
        return t.value

    def poll(self, ticket):
        r = ms_request_result()
        code = lib().ms_server_poll(self.h, ticket, C.byref(r))
        if code == 9:          # MS_ERR_BUSY
            return None
        _ffi.check(code)
        return dict(ticket=r.ticket, session=r.session, status=r.status, t_arrive=r.t_arrive,
                    t_done=r.t_done, latency=r.latency, launch_envs=r.launch_envs)

    def drain(self):
        _ffi.check(lib().ms_server_drain(self.h))

    def state(self, sid, n_bodies):
        out = np.zeros((n_bodies, 13), np.float32)
        _ffi.check(lib().ms_server_copy_state(self.h, sid, out.ctypes.data))
        return out

    def stats(self) -> dict:
        st = ms_server_stats()
        _ffi.check(lib().ms_server_stats_get(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ms_server_stats._fields_}

    def reset_stats(self):
        _ffi.check(lib().ms_server_reset_stats(self.h))

    @staticmethod
    def now() -> float:
        return lib().ms_server_now()
