"""B300-native batched rigid-body step (sm_103a CUDA behind the C ABI of
include/ms.h).

    import torch, scenegen
    from paper_2410_00425_b300 import Batch
    b = Batch(scenegen.make_scene("arm"))
    b.step(actions_cuda_tensor, n_steps=10, stream=torch.cuda.Stream())

``Batch`` only marshals arguments to the library; every stage of the step
runs in the CUDA kernels of ``libmsim.so``.  There is no CPU fallback:
constructing a batch without the built library or without a CUDA device
raises.
"""
from __future__ import annotations

from . import _ffi
from ._ffi import MSError, load  # noqa: F401


class Batch:
    """Owns one ms_batch (all envs of a scene resident on the current GPU)."""

    def __init__(self, scene, record_contacts: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.scene = scene
        self.E = scene.n_envs
        self.NB = int(scene.body_off[-1])
        self.NJ = int(scene.joint_off[-1])
        self.A = int((scene.joint_off[1:] - scene.joint_off[:-1]).max()) if self.E else 0
        self.h = _ffi.ms_create_batch_flat(scene.bodies, scene.body_off, scene.joints,
                                           scene.joint_off, scene.params, getattr(scene, "hulls", None))
        if record_contacts:
            _ffi.ms_set_record_contacts(self.h, True)

    def close(self):
        if getattr(self, "h", None):
            _ffi.ms_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, actions=None, n_steps: int = 1, stream=None, plain: bool = False, out=None):
        """actions: CUDA float32 tensor [n_steps, E, A] (NaN keeps a target;
        normalised deltas once a task is set).  out: CUDA float32 tensor
        [n_steps, E, record_len] receiving the task records, or None."""
        import torch
        for t, shape in ((actions, (n_steps, self.E, self.A)), (out, (n_steps, self.E, self.record_len()))):
            if t is None:
                continue
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
            assert tuple(t.shape) == shape, (tuple(t.shape), shape)
            if isinstance(stream, torch.cuda.Stream):
                # the step uses the tensor on `stream`: keep its memory from
                # being reused by the caching allocator until then
                t.record_stream(stream)
        if out is None:
            fn = _ffi.ms_step_plain if plain else _ffi.ms_step
            fn(self.h, actions, n_steps, stream)
        else:
            _ffi.ms_step_ex(self.h, actions, n_steps, out, _ffi.MS_STEP_PLAIN if plain else 0, stream)

    # ------------------------------------------------------------- camera
    def set_camera(self, camera, body_rgb):
        """camera: dict eye, target, fov_y, near, width, height (see
        scenegen.default_camera); body_rgb: [n_bodies][3] in [0, 1]."""
        _ffi.ms_set_camera(self.h, camera, body_rgb)
        self.camera = dict(camera)

    def render(self, stream=None, rgba=True, depth=True, seg=True):
        """Images of every env at the current state: rgba uint8 [E, H, W, 4],
        depth float32 [E, H, W], seg int16-stored uint16 [E, H, W] (body + 1)."""
        import torch
        H, W = int(self.camera["height"]), int(self.camera["width"])
        out_rgba = torch.empty((self.E, H, W, 4), dtype=torch.uint8, device="cuda") if rgba else None
        out_depth = torch.empty((self.E, H, W), dtype=torch.float32, device="cuda") if depth else None
        out_seg = torch.empty((self.E, H, W), dtype=torch.int16, device="cuda") if seg else None
        _ffi.ms_render(self.h, out_rgba, out_depth, out_seg, stream)
        return out_rgba, out_depth, out_seg

    # ---------------------------------------------------------- pick task
    def set_task(self, task, stream=None):
        """Set (dict, see scenegen.pick_task) or remove (None) the pick task;
        setting it resets every env's controller."""
        _ffi.ms_set_task(self.h, task, stream)

    def task_reset(self, env_mask=None, stream=None):
        _ffi.ms_task_reset(self.h, env_mask, stream)

    def record_len(self) -> int:
        return _ffi.ms_task_record_len(self.h)

    def observe(self, stream=None):
        """Task records of every env at the current state, [E, record_len]."""
        import torch
        out = torch.empty((self.E, self.record_len()), dtype=torch.float32, device="cuda")
        _ffi.ms_task_observe(self.h, out, stream)
        return out

    def state(self, stream=None):
        """Device copy of the state, float32 [n_bodies, 13]."""
        import torch
        out = torch.empty((self.NB, 13), dtype=torch.float32, device="cuda")
        _ffi.ms_copy_state(self.h, out, 1, stream)
        return out

    def step_host(self, actions, n_steps, out, records=False, stream=None):
        """Host actions in, host state (or, records=True, task records) out,
        through one C-ABI call (ms_step_host)."""
        _ffi.ms_step_host(self.h, actions, n_steps, out, 1 if records else 0, stream)
        return out

    def state_to_host(self, out, stream=None):
        """Copy the state into a (pinned) host tensor [n_bodies, 13]."""
        _ffi.ms_copy_state(self.h, out, 0, stream)
        return out

    def set_state(self, src, env_mask=None, stream=None):
        kind = 1 if getattr(src, "is_cuda", False) else 0
        _ffi.ms_set_state(self.h, src, kind, env_mask, stream)

    def sync(self):
        return _ffi.ms_sync(self.h)

    def contacts(self, env: int, cap: int = 1024):
        return _ffi.ms_get_contacts(self.h, env, cap)

    def colors(self, env: int, cap: int = 4096):
        """Colour of each constraint (joints, then manifolds) of the env's
        last step; needs record_contacts."""
        return _ffi.ms_get_colors(self.h, env, cap)

    def enable_contact_forces(self, on=True):
        """Make every later step write each body's contact force (touch
        sensors, ms_enable_contact_forces)."""
        _ffi.ms_enable_contact_forces(self.h, on)

    def contact_forces(self, stream=None):
        """Per body (F[3], f_n) of the last step, device float32 [n_bodies, 4]."""
        import torch
        out = torch.empty((self.NB, 4), dtype=torch.float32, device="cuda")
        _ffi.ms_contact_forces(self.h, out, stream)
        return out

    def set_tuning(self, lanes_per_env=32, warps_per_cta=4, rows_in_smem=1):
        _ffi.ms_set_tuning(self.h, lanes_per_env, warps_per_cta, rows_in_smem)

    def tuning(self):
        return _ffi.ms_get_tuning(self.h)

    def autotune(self, n_steps=1, cache_path=None, stream=None):
        return _ffi.ms_autotune(self.h, n_steps, cache_path, stream)

    def memory_bytes(self):
        return _ffi.ms_memory_bytes(self.h)


def use_torch_allocator(on=True):
    """Route the device memory of batches created from now on through
    PyTorch's caching allocator (on=False: back to the library's pool).
    Batches keep the allocator they were created with."""
    import torch
    from . import _ffi
    if not on:
        _ffi.ms_set_allocator(None, None)
        return
    _ffi.ms_set_allocator(lambda n, d, st: torch.cuda.caching_allocator_alloc(n, d, st),
                          lambda p, d, st: torch.cuda.caching_allocator_delete(p))

