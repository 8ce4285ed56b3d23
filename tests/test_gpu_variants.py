"""The optional solver variants on the CUDA path against the oracle:
velocity damping, restitution and warm starting across steps.

Warm starting carries state between steps that cannot be transferred to the
oracle, so every comparison is a rollout from the same initial state, held
to the rollout bars (10x the one-step bars) on non-chaotic, tie-free envs.
The variants must not break the bit-identity of the plain and batched paths,
of launch shapes, and of a restored checkpoint with a fresh batch.
"""
import numpy as np
import pytest

import scenegen
from scenegen import validation as V
from _parity import env_errors, gpu_run, non_chaotic, oracle_run, tie_free, within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = dict(linear_damping=0.5, angular_damping=0.3, bounce_threshold=0.5, warm_start=1)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _with(sc, restitution=None, **pk):
    sc.params = dict(sc.params, **pk)
    if restitution is not None:
        sc.bodies = sc.bodies.copy()
        sc.bodies["restitution"] = restitution
    return sc


@pytest.mark.parametrize("name,n,steps,need", [("small", 128, 100, 8), ("clutter", 64, 40, 1),
                                               ("arm", 128, 200, 30)])
def test_rollout_with_variants_follows_oracle(name, n, steps, need):
    """The arm case is the warm-started arm: with soft joint rows it no
    longer gains speed, so its rollouts are compared with the oracle."""
    sc = _with(scenegen.make_scene(name, n_envs=n), restitution=0.4, **VARIANTS)
    calm, ost = non_chaotic(sc, steps)
    o = oracle_run(sc, steps)
    _, st, _ = gpu_run(sc, steps)
    err = env_errors(sc, st, ost)
    clean = calm & tie_free(o, sc)
    print(f"{name}: {clean.sum()} of {n} envs non-chaotic and tie-free")
    assert clean.sum() >= need
    ok = within(err, 10.0)
    bad = np.nonzero(clean & ~ok)[0]
    assert ok[clean].all(), f"envs {bad.tolist()} errors {err[bad].tolist()}"


@pytest.mark.parametrize("e", [0.3, 0.8])
def test_bouncing_ball_follows_oracle(e):
    sc = V.bouncing_ball(e=e, z0=0.5, n_envs=4)
    for steps in (34, 120):                   # just after the first impact; after settling
        o = oracle_run(sc, steps)
        _, st, _ = gpu_run(sc, steps)
        err = env_errors(sc, st, o.state())
        assert within(err, 10.0).all(), (steps, err.max(0))
        if steps == 34:
            assert st[1, 9] > 0.5 * e * 3.0    # on its way up after the bounce


def test_warm_start_hanging_chain_matches_oracle():
    """Joint impulses carried across steps, one position iteration: a double
    pendulum swinging about world x.  The hinge axis and every frame are
    exact in both precisions, so the motion stays exactly planar; about a
    rounded axis the out-of-plane mode of these rigid joint rows grows from
    rounding noise (in the FP64 oracle as well), which no rollout survives."""
    ident = (0.0, 0.0, 0.0, 1.0)
    r, l = 0.02, 0.1
    bl = [scenegen.body(scenegen.CAPSULE, (r, l, 0), 1.0, (0, 0, 1.0 - l), group=1),
          scenegen.body(scenegen.CAPSULE, (r, l, 0), 0.5, (0, 0, 1.0 - 3 * l), angvel=(1.0, 0.0, 0.0), group=2)]
    jl = [scenegen.joint(scenegen.REVOLUTE, -1, 0, (0, 0, 1.0, *ident), (0, 0, l, *ident), -3, 3, 0, 0, 0),
          scenegen.joint(scenegen.REVOLUTE, 0, 1, (0, 0, -l, *ident), (0, 0, l, *ident), -3, 3, 0, 0, 0)]
    sc = scenegen.pack("chain", [bl], [jl], scenegen.default_params(pos_iters=1, warm_start=1), 0, 0)
    for steps in (100, 200):
        o = oracle_run(sc, steps)
        # default launch shape, and 8 lanes per env: three idle lane groups
        # share the env's warp and must follow its warp-wide operations
        for tuning in (None, (8, 1, 0)):
            _, st, _ = gpu_run(sc, steps, tuning=tuning)
            err = env_errors(sc, st, o.state())
            assert within(err, 10.0).all(), (steps, tuning, err)
            assert np.abs(st[:, [0, 7, 11, 12]]).max() == 0.0       # planar


def test_warm_start_resting_box_matches_oracle():
    """One position iteration, warm started: the GPU rests like the oracle."""
    sc = V.stack(n_boxes=1, pos_iters=1, warm_start=1)
    o = oracle_run(sc, 200)
    _, st, _ = gpu_run(sc, 200)
    err = env_errors(sc, st, o.state())
    assert within(err, 10.0).all(), err
    assert np.abs(st[1, 7:13]).max() < 1e-4


@pytest.mark.parametrize("name", ["arm", "clutter"])
def test_plain_path_bit_identical_with_variants(name):
    sc = _with(scenegen.make_scene(name, n_envs=48), restitution=0.4, **VARIANTS)
    _, a, sa = gpu_run(sc, 4)
    _, b, sb = gpu_run(sc, 4, plain=True)
    assert np.array_equal(a, b), np.abs(a - b).max()
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("tuning", [(16, 2, 0), (8, 1, 0), (4, 4, 0), (32, 1, 1)])
def test_tuning_does_not_change_results_with_warm_start(tuning):
    sc = _with(scenegen.make_scene("clutter", n_envs=64), restitution=0.4, **VARIANTS)
    _, ref, _ = gpu_run(sc, 3)
    _, st, _ = gpu_run(sc, 3, tuning=tuning)
    assert np.array_equal(ref, st)


def test_set_state_clears_warm_memory():
    """A restored checkpoint steps like a fresh batch created at that state."""
    from paper_2410_00425_b300 import Batch
    sc = _with(scenegen.make_scene("arm", n_envs=16), **VARIANTS)
    s = torch.cuda.Stream()
    acts = torch.from_numpy(sc.actions(0, 10)).cuda()
    b = Batch(sc)
    b.step(acts[:5].contiguous(), 5, stream=s)
    torch.cuda.synchronize()
    ck = b.state().cpu().contiguous()
    b.step(acts[5:8].contiguous(), 3, stream=s)
    b.set_state(ck, stream=s)                 # back to the checkpoint: memory cleared
    b.step(acts[8:10].contiguous(), 2, stream=s)
    torch.cuda.synchronize()
    got = b.state().cpu()
    # a fresh batch at the checkpoint (its targets as after step 7: set them by one call)
    f = Batch(sc)
    f.set_state(ck, stream=s)
    f.step(acts[5:8].contiguous(), 3, stream=s)     # targets now equal b's at restore
    f.set_state(ck, stream=s)
    f.step(acts[8:10].contiguous(), 2, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(got, f.state().cpu())
    b.close(); f.close()
