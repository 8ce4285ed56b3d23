"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point include/ms.h declares, agrees on struct layouts, and rejects bad
arguments synchronously (validation happens before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import scenegen
from paper_2410_00425_b300 import _ffi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _ffi.load()


def declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ms_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2410_00425_b300 import server
    names = declared("ms.h")
    snames = declared("ms_server.h")
    assert "ms_step" in names and "ms_create_batch" in names and "ms_server_submit" in snames
    raw = C.CDLL(_ffi.LIB_PATH)
    for n in names + snames:
        assert hasattr(raw, n), n
    assert set(names) <= set(_ffi.EXPORTS)
    assert set(snames) <= set(server.EXPORTS)
    server.lib()                                  # binds every server signature


def test_debug_library_exports_the_same_entry_points():
    """The bounds-checked twin (-DMS_DEBUG_BOUNDS) builds and exports the
    same C ABI (it is loaded only by its own GPU test)."""
    path = build.build(debug=True)
    raw = C.CDLL(path)
    for n in declared("ms.h") + declared("ms_server.h"):
        assert hasattr(raw, n), n
    assert raw.ms_step(None, None, 1, None) == 1


def test_struct_layouts_match(lib):
    sizes = (C.c_int32 * 5)()
    lib.ms_abi_sizes(sizes)
    assert sizes[0] == scenegen.BODY_DTYPE.itemsize == 84
    assert sizes[1] == scenegen.JOINT_DTYPE.itemsize == 88
    assert sizes[2] == C.sizeof(_ffi.ms_sim_params)


def _create(sc):
    return _ffi.ms_create_batch_flat(sc.bodies, sc.body_off, sc.joints, sc.joint_off, sc.params)


def _bad(sc, fragment):
    with pytest.raises(_ffi.MSError) as ei:
        _create(sc)
    assert ei.value.code == 1, str(ei.value)
    assert fragment in str(ei.value)


def test_invalid_descriptors_rejected(lib):
    base = scenegen.make_scene("arm", n_envs=2)

    sc = scenegen.make_scene("arm", n_envs=2); sc.bodies["type"][3] = 9
    _bad(sc, "bad type")
    sc = scenegen.make_scene("arm", n_envs=2); sc.bodies["mass"][4] = -1
    _bad(sc, "negative mass")
    sc = scenegen.make_scene("arm", n_envs=2); sc.bodies["p"][2, 0] = 0.0
    _bad(sc, "shape size")
    sc = scenegen.make_scene("arm", n_envs=2); sc.bodies["pos"][5, 1] = np.nan
    _bad(sc, "non-finite")
    sc = scenegen.make_scene("arm", n_envs=2); sc.bodies["quat"][5] = 0
    _bad(sc, "zero quaternion")
    sc = scenegen.make_scene("arm", n_envs=2); sc.joints["child"][3] = 40
    _bad(sc, "parent/child")
    sc = scenegen.make_scene("arm", n_envs=2); sc.joints["parent"][1] = sc.joints["child"][1]
    _bad(sc, "parent/child")
    sc = scenegen.make_scene("arm", n_envs=2); sc.joints["lower"][0] = 3.0
    _bad(sc, "lower > upper")
    sc = scenegen.make_scene("arm", n_envs=2); sc.joints["kp"][0] = -1.0
    _bad(sc, "negative gain")
    for key, val, frag in [("dt", 0.0, "dt"), ("substeps", 0, "substeps"), ("pos_iters", -1, "iteration"),
                           ("contact_capacity", 0, "contact_capacity"), ("pair_capacity", 0, "pair_capacity"),
                           ("max_depen_vel", 0.0, "max_depen_vel"), ("margin", -1.0, "margin")]:
        sc = scenegen.make_scene("arm", n_envs=2)
        sc.params[key] = val
        _bad(sc, frag)
    # too many bodies in one env
    bl = [scenegen.body(scenegen.SPHERE, (0.01, 0, 0), 1.0, (i, 0, 0)) for i in range(65)]
    sc = scenegen.pack("big", [bl], [[]], scenegen.default_params(), 0, 0)
    _bad(sc, "n_bodies")
    assert base.n_envs == 2


def test_null_arguments(lib):
    assert lib.ms_step(None, None, 1, None) == 1
    assert lib.ms_step_plain(None, None, 1, None) == 1
    assert lib.ms_sync(None, None) == 1
    assert lib.ms_destroy(None) == 0
    assert lib.ms_copy_state(None, None, 0, None) == 1
    assert lib.ms_set_state(None, None, 0, None, None) == 1
    assert lib.ms_get_state(None, None) == 1
    assert lib.ms_get_contacts(None, 0, 0, None, None, None, None) == 1
    assert lib.ms_enable_contact_forces(None, 1) == 1
    assert lib.ms_contact_forces(None, None, None) == 1
    assert lib.ms_set_tuning(None, None) == 1
    assert lib.ms_autotune(None, 1, None, None, None) == 1
    assert len(_ffi.ms_last_error()) > 0


def test_estimate_bytes_scales_with_envs(lib):
    sc = scenegen.make_scene("arm", n_envs=8)
    a = _ffi.ms_estimate_bytes(sc.body_off, sc.joint_off, sc.params)
    sc2 = scenegen.make_scene("arm", n_envs=16)
    b = _ffi.ms_estimate_bytes(sc2.body_off, sc2.joint_off, sc2.params)
    assert 1.9 * a < b < 2.1 * a


def test_server_rejects_bad_options(lib):
    from paper_2410_00425_b300 import server
    L = server.lib()
    h = C.c_void_p()
    o = server.ms_server_options(1, 0, 0.0, 65)
    assert L.ms_server_create(1 << 30, C.byref(o), C.byref(h)) == 1
    assert "max_inflight" in _ffi.ms_last_error()
    assert L.ms_server_create(1 << 30, None, None) == 1
