"""Shared helpers of the GPU parity tests: run a scene through the CUDA path
and through the oracle, and compare them with the step's tolerances."""
from __future__ import annotations

import numpy as np

import oracle
import scenegen

# tolerances after one step (positions m, velocities m/s, angular
# velocities rad/s, quaternion components); rollouts of non-chaotic envs use
# 10x these.  Angular velocity is also held to the velocity bar at the
# body's material points: |dw| * r_bound <= TOL_V, r_bound the body's
# bounding radius.
TOL_X, TOL_V, TOL_W, TOL_Q = 1e-5, 1e-4, 1e-4, 1e-5
TIE_EPS = 1e-5


def bound_radius(bodies, hulls=None):
    """Radius of each body's bounding sphere about its origin (0 for planes;
    a hull's from its vertices in the scene's hull library)."""
    p = bodies["p"].astype(np.float64)
    t = bodies["type"]
    r = np.where(t == scenegen.SPHERE, p[:, 0],
                 np.where(t == scenegen.CAPSULE, p[:, 0] + p[:, 1],
                          np.where(t == scenegen.BOX, np.linalg.norm(p, axis=1), 0.0)))
    if hulls is not None:
        v, vo = np.asarray(hulls["verts"], np.float64), np.asarray(hulls["vert_off"])
        for i in np.nonzero(t == scenegen.HULL)[0]:
            h = int(p[i, 0])
            r[i] = np.linalg.norm(v[vo[h]:vo[h + 1]], axis=1).max()
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
    (m/s), quaternion (sign-insensitive), angular velocity (rad/s)."""
    bo = scene.body_off
    E = scene.n_envs
    rb = bound_radius(scene.bodies, getattr(scene, "hulls", None))
    out = np.zeros((E, 5))
    for e in range(E):
        s = slice(bo[e], bo[e + 1])
        A, B = a[s], b[s]
        out[e, 0] = np.abs(A[:, 0:3] - B[:, 0:3]).max()
        out[e, 1] = np.abs(A[:, 7:10] - B[:, 7:10]).max()
        out[e, 2] = (np.abs(A[:, 10:13] - B[:, 10:13]).max(1) * rb[s]).max()
        dq = np.minimum(np.abs(A[:, 3:7] - B[:, 3:7]).max(1), np.abs(A[:, 3:7] + B[:, 3:7]).max(1))
        out[e, 3] = dq.max()
        out[e, 4] = np.abs(A[:, 10:13] - B[:, 10:13]).max()
    return out


def within(err, scale=1.0):
    return ((err[:, 0] <= TOL_X * scale) & (err[:, 1] <= TOL_V * scale) &
            (err[:, 2] <= TOL_V * scale) & (err[:, 3] <= TOL_Q * scale) & (err[:, 4] <= TOL_W * scale))


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


def non_chaotic(scene, n_steps, threads=8):
    """Envs whose rollout is insensitive to perturbations of the size the
    float32 path introduces.  At every step of the rollout:
      * two FP64 runs from positions 1e-9 m apart stay within 1e-6 m;
      * an FP64 run that stores every velocity and pose as float32 after each
        update (impulse, gravity, integration) -- the storage precision of
        the float32 path, at the places it rounds -- stays within the
        one-step bars of the plain FP64 run (an impact can amplify the
        rounding for a few steps and recover; such an env is sensitive).
    Returns (mask, state of the plain FP64 run)."""
    runs = [oracle.Oracle(scene) for _ in range(3)]
    base, pert, r32 = runs
    st = pert.state()
    st[scene.bodies["mass"] > 0, 0] += 1e-9
    pert.set_state(st)
    r32.set_round32(True)
    for o in runs:
        if scene.task is not None:
            o.set_task(scene.task)
    calm = np.ones(scene.n_envs, bool)
    for k in range(n_steps):
        a = scene.actions(k, 1)
        for o in runs:
            if scene.task is not None:
                o.step_task(1, actions=a, threads=threads)
            else:
                o.step(1, actions=a, threads=threads)
        ref = base.state()
        calm &= env_errors(scene, ref, pert.state())[:, 0] < 1e-6
        calm &= within(env_errors(scene, ref, r32.state()))
    return calm, base.state()


def tie_free(o, scene):
    return np.array([o.ties(e) == 0 for e in range(scene.n_envs)])
