"""Shared helpers of the GPU parity tests: run a scene through the CUDA path
and through the oracle, and compare them with the step's tolerances."""
from __future__ import annotations

import numpy as np

import oracle
import scenegen

# tolerances after one step (positions m, velocities m/s, quaternion
# components); rollouts of non-chaotic envs use 10x these.  Angular
# velocity is held to the velocity bar at the body's material points:
# |dw| * r_bound <= TOL_V, r_bound the body's bounding radius.
TOL_X, TOL_V, TOL_Q = 1e-5, 1e-4, 1e-5
TIE_EPS = 1e-5
# relative velocity noise per step of the non-chaotic probe: four float32
# ulps.  A velocity component takes ~40 row impulses per step (4 substeps x
# 10 sweeps), each rounded once in float32; as a random walk that is ~6 ulps.
VEL_NOISE = 4 * 2.0**-24


def bound_radius(bodies):
    p = bodies["p"].astype(np.float64)
    t = bodies["type"]
    r = np.where(t == scenegen.SPHERE, p[:, 0],
                 np.where(t == scenegen.CAPSULE, p[:, 0] + p[:, 1],
                          np.where(t == scenegen.BOX, np.linalg.norm(p, axis=1), 0.0)))
    return r


def gpu_run(scene, n_steps, plain=False, tuning=None, stream=True, record=False, calls=1, records=None):
    """Steps the scene through the CUDA path (its pick task set, if it has
    one).  records: a list that receives the task records of every step,
    float64 [n_steps, E, D]."""
    import torch
    from paper_2410_00425_b300 import Batch
    b = Batch(scene, record_contacts=record)
    if tuning is not None:
        b.set_tuning(*tuning)
    s = torch.cuda.Stream() if stream else None
    if scene.task is not None:
        b.set_task(scene.task, stream=s)
    done = 0
    per = n_steps // calls
    outs = []
    for c in range(calls):
        n = per if c < calls - 1 else n_steps - done
        a = scene.actions(done, n)
        at = None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
        out = None
        if records is not None:
            out = torch.full((n, b.E, b.record_len()), float("nan"), dtype=torch.float32, device="cuda")
            outs.append(out)
        if s is not None:
            s.wait_stream(torch.cuda.current_stream())
        b.step(at, n, stream=s, plain=plain, out=out)
        done += n
    if s is not None:
        torch.cuda.current_stream().wait_stream(s)
    st = b.state(stream=None)
    torch.cuda.synchronize()
    code, status = b.sync()
    if records is not None:
        records.append(torch.cat(outs).cpu().numpy().astype(np.float64))
    return b, st.cpu().numpy().astype(np.float64), status


def oracle_run(scene, n_steps, threads=8, perturb=0.0, records=None):
    """The oracle over the scene (its pick task set, if it has one).
    records: a list that receives (records [n_steps, E, D], tie masks)."""
    o = oracle.Oracle(scene)
    if scene.task is not None:
        o.set_task(scene.task)
    if perturb:
        st = o.state()
        dyn = scene.bodies["mass"] > 0
        st[dyn, 0] += perturb
        o.set_state(st)
    if records is not None:
        records.append(o.step_task(n_steps, threads=threads))
    elif scene.task is not None:
        o.step_task(n_steps, threads=threads)
    else:
        o.step(n_steps, threads=threads)
    return o


def env_errors(scene, a, b):
    """Per-env max errors between two [NB,13] states: position (m), linear
    velocity (m/s), angular velocity as material-point speed |dw| r_bound
    (m/s), quaternion (sign-insensitive)."""
    bo = scene.body_off
    E = scene.n_envs
    rb = bound_radius(scene.bodies)
    out = np.zeros((E, 4))
    for e in range(E):
        s = slice(bo[e], bo[e + 1])
        A, B = a[s], b[s]
        out[e, 0] = np.abs(A[:, 0:3] - B[:, 0:3]).max()
        out[e, 1] = np.abs(A[:, 7:10] - B[:, 7:10]).max()
        out[e, 2] = (np.abs(A[:, 10:13] - B[:, 10:13]).max(1) * rb[s]).max()
        dq = np.minimum(np.abs(A[:, 3:7] - B[:, 3:7]).max(1), np.abs(A[:, 3:7] + B[:, 3:7]).max(1))
        out[e, 3] = dq.max()
    return out


def within(err, scale=1.0):
    return ((err[:, 0] <= TOL_X * scale) & (err[:, 1] <= TOL_V * scale) &
            (err[:, 2] <= TOL_V * scale) & (err[:, 3] <= TOL_Q * scale))


def pair_sets_match(batch, o, scene):
    """Compare kept contact pairs of the last step; pairs the oracle marks as
    margin ties are excluded.  Returns the list of mismatching envs."""
    bad = []
    for e in range(scene.n_envs):
        gp, gn, _ = batch.contacts(e)
        op, on, _ = o.manifolds(e)
        ties = {tuple(t) for t in o.margin_ties(e).tolist()}
        ties |= {(t[1], t[0]) for t in ties}
        G = {tuple(p) for p in gp.tolist()} - ties
        O = {tuple(p) for p in op.tolist()} - ties
        if G != O:
            bad.append(e)
    return bad


def non_chaotic(scene, n_steps, threads=8, seed=11, seeds=None, margin=1.0):
    """Envs whose rollout is insensitive to perturbations of the size the
    float32 path introduces.  Both must hold after n_steps:
      * two FP64 runs from positions 1e-9 m apart stay within 1e-6 m;
      * an FP64 run whose state is rounded to float32 after every step, and
        whose velocities then take VEL_NOISE of relative noise (random sign,
        seeded), stays within the one-step bars (1e-5 m, 1e-4 m/s, 1e-4 m/s,
        1e-5) of the plain FP64 run.  Float32 state storage, amplified
        through the d/h and C/h position-correction biases, and the float32
        solve arithmetic are the perturbations actually present in the
        comparison; a body spinning for many radians accumulates the latter
        as orientation phase.
    seeds (several noise draws, all must pass) and margin (a fraction of
    the one-step bars) make the selection stricter for scenes whose envs
    sit near the edge: stiff drives pressed against a limit, fast fingers.
    Returns (mask, state of the plain FP64 run)."""
    base = oracle_run(scene, n_steps, threads).state()
    pert = oracle_run(scene, n_steps, threads, perturb=1e-9).state()
    calm = env_errors(scene, base, pert)[:, 0] < 1e-6
    for sd in (seeds if seeds is not None else (seed,)):
        o = oracle.Oracle(scene)
        if scene.task is not None:
            o.set_task(scene.task)
        rng = np.random.default_rng(sd)
        for k in range(n_steps):
            if scene.task is not None:
                o.step_task(1, threads=threads)
            else:
                o.step(1, threads=threads)
            st = o.state().astype(np.float32).astype(np.float64)
            st[:, 7:13] *= 1.0 + rng.choice([-1.0, 1.0], size=st[:, 7:13].shape) * VEL_NOISE
            o.set_state(st)
        err = env_errors(scene, base, o.state())
        calm &= within(err, margin)
    return calm, base


def tie_free(o, scene):
    return np.array([o.ties(e) == 0 for e in range(scene.n_envs)])
