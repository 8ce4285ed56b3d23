"""Pins of the FP64 oracle against mechanics it must reproduce.

Each test fixes part of the oracle with something other than the oracle:
closed forms (free fall, implicit-Euler drive, pendulum period, incline
acceleration), conservation laws (momentum), brute force (LCP active-set
enumeration, sampled-direction box overlap, exact clip rectangles) and
physical steady states (resting stack, joint limit).  A plausible mistake
in a stage (a sign, a dropped term, a swapped operand) breaks one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import validation as V

G = 9.81


def rot(q):
    return V._rot(q)


# ---------------------------------------------------------------- free fall
def test_freefall_discrete_closed_form():
    """Symplectic Euler with N substeps of h: v_N = v0 + N h g and
    x_N = x0 + N h v0 + h^2 g N(N+1)/2 (x uses the updated velocity)."""
    sc = V.freefall(n_envs=8)
    o = oracle.Oracle(sc)
    steps = 37
    o.step(steps)
    st = o.state()
    p = sc.params
    h = p["dt"] / p["substeps"]
    N = steps * p["substeps"]
    g = np.array(p["gravity"])
    x0 = sc.bodies["pos"].astype(np.float64)
    v0 = sc.bodies["linvel"].astype(np.float64)
    vN = v0 + N * h * g
    xN = x0 + N * h * v0 + h * h * g * N * (N + 1) / 2
    np.testing.assert_allclose(st[:, 7:10], vN, rtol=0, atol=1e-12)
    np.testing.assert_allclose(st[:, 0:3], xN, rtol=0, atol=1e-12)
    # continuous x0 + v0 t + g t^2/2 within h g t / 2
    t = steps * p["dt"]
    xc = x0 + v0 * t + 0.5 * g * t * t
    assert np.all(np.abs(st[:, 0:3] - xc) <= 0.5 * h * G * t + 1e-12)


def test_freefall_rotation_preserves_unit_quaternion_and_axis():
    """Torque-free spin about a fixed world axis: |q| = 1 and, for a sphere
    (isotropic inertia), omega stays constant."""
    sc = V.freefall(n_envs=4)
    o = oracle.Oracle(sc)
    o.step(50)
    st = o.state()
    np.testing.assert_allclose(np.linalg.norm(st[:, 3:7], axis=1), 1.0, atol=1e-14)
    w0 = sc.bodies["angvel"].astype(np.float64)
    np.testing.assert_allclose(st[0::2, 10:13], w0[0::2], atol=0)


# ------------------------------------------------------------------ incline
@pytest.mark.parametrize("dtan", [0.1, -0.1])
def test_incline_slides_iff_tan_exceeds_mu(dtan):
    mu = 0.5
    th = math.atan(mu + dtan)
    # The stuck case runs 32 position iterations: every step restarts the
    # solver cold, and 8 Gauss-Seidel sweeps leave a ~3 % residual slip in
    # the first substep (0.4 mm creep per 500 steps, shrinking ~10x per
    # doubling of iterations) -- a convergence effect, not the friction law.
    sc = V.incline([th], mu=mu, pos_iters=8 if dtan > 0 else 32)
    o = oracle.Oracle(sc)
    s_dir = np.array([math.cos(th), 0.0, -math.sin(th)])
    x0 = sc.bodies["pos"][1].astype(np.float64)
    traj = []
    for k in range(500 if dtan < 0 else 151):
        o.step(1)
        traj.append(o.state()[1, 0:3] @ s_dir)
    traj = np.array(traj)
    if dtan > 0:
        # mean acceleration along the slope over steps 50..150
        dt = sc.params["dt"]
        s50, s100, s150 = traj[49], traj[99], traj[149]
        acc = (s150 - 2 * s100 + s50) / (50 * dt) ** 2
        expect = G * (math.sin(th) - mu * math.cos(th))
        assert abs(acc - expect) <= 0.01 * expect, (acc, expect)
    else:
        assert np.max(np.abs(traj - x0 @ s_dir)) < 1e-4
        st = o.state()
        assert np.linalg.norm(st[1, 0:3] - x0) < 1e-4


# ----------------------------------------------------------- contact forces
def test_contact_forces_of_a_resting_stack_balance_gravity():
    """Two boxes stacked on the plane, settled: the contact force on each box
    is -m g (it does not accelerate), the top box's normal force is m2 g and
    the bottom box's is (m1 + m2) g from the plane plus m2 g from the top
    box; the plane reads the reaction -(m1 + m2) g."""
    from scenegen import BOX, PLANE, body, pack
    m1, m2, h1, h2 = 0.2, 0.05, 0.03, 0.02
    sc = pack("stack2", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)),
                          body(BOX, (h1, h1, h1), m1, (0, 0, h1)),
                          body(BOX, (h2, h2, h2), m2, (0.005, -0.004, 2 * h1 + h2))]], [[]],
              V.default_params(pos_iters=64), 0, 0)
    o = oracle.Oracle(sc)
    o.step(200)
    f = o.contact_forces()
    np.testing.assert_allclose(f[1, :3], [0, 0, m1 * G], atol=1e-9 * m1 * G + 1e-12)
    np.testing.assert_allclose(f[2, :3], [0, 0, m2 * G], atol=1e-9)
    np.testing.assert_allclose(f[0, :3], [0, 0, -(m1 + m2) * G], atol=1e-9)
    np.testing.assert_allclose(f[:, 3], [(m1 + m2) * G, (m1 + 2 * m2) * G, m2 * G], rtol=1e-7)


def test_contact_force_of_a_sliding_box_is_normal_plus_kinetic_friction():
    """A box sliding down a ramp with tan theta > mu: the contact force on it
    is m g cos theta (n - mu s), s the down-slope direction (the pyramid row
    along the slope sits at its bound)."""
    mu, th, m = 0.5, math.atan(0.6), 0.1
    sc = V.incline([th], mu=mu, mass=m)
    o = oracle.Oracle(sc)
    o.step(100)
    f = o.contact_forces()
    n = np.array([math.sin(th), 0.0, math.cos(th)])
    s_dir = np.array([math.cos(th), 0.0, -math.sin(th)])
    fn = m * G * math.cos(th)
    np.testing.assert_allclose(f[1, :3], fn * (n - mu * s_dir), rtol=0, atol=1e-6 * fn)
    np.testing.assert_allclose(f[1, 3], fn, rtol=1e-6)
    np.testing.assert_allclose(f[0, :3], -f[1, :3], atol=1e-12)


# ----------------------------------------------------------------- momentum
def _momenta(sc, st):
    m = sc.bodies["mass"].astype(np.float64)
    P = (m[:, None] * st[:, 7:10])
    return P


@pytest.mark.parametrize("spheres_only", [False, True])
def test_momentum_conserved_without_gravity_and_friction(spheres_only):
    """Linear momentum: any settings.  Angular momentum (spheres only): the
    contact normal is fixed for the whole step, so the pair of normal
    impulses only stays on the line of centres when the rows are applied
    at the poses the narrowphase saw -- one substep and no relax sweep."""
    kw = dict(substeps=1, vel_iters=0) if spheres_only else {}
    sc = V.momentum(n_envs=8, spheres_only=spheres_only, **kw)
    o = oracle.Oracle(sc)
    st0 = o.state()
    m = sc.bodies["mass"].astype(np.float64)
    bo = sc.body_off
    P0 = [(m[bo[e]:bo[e + 1], None] * st0[bo[e]:bo[e + 1], 7:10]).sum(0) for e in range(sc.n_envs)]

    def L_of(st, e):
        # sphere: I = 2/5 m r^2, isotropic
        sl = slice(bo[e], bo[e + 1])
        r = sc.bodies["p"][sl, 0].astype(np.float64)
        I = 0.4 * m[sl] * r * r
        return (np.cross(st[sl, 0:3], m[sl, None] * st[sl, 7:10]) + I[:, None] * st[sl, 10:13]).sum(0)
    L0 = [L_of(st0, e) for e in range(sc.n_envs)]
    contacts = 0
    for _ in range(60):
        o.step(1)
        contacts += o.counters()["contact_points"]
    st = o.state()
    assert contacts > 0, "scene must actually collide"
    for e in range(sc.n_envs):
        P = (m[bo[e]:bo[e + 1], None] * st[bo[e]:bo[e + 1], 7:10]).sum(0)
        scale = np.abs(m[bo[e]:bo[e + 1], None] * st0[bo[e]:bo[e + 1], 7:10]).sum()
        assert np.max(np.abs(P - P0[e])) <= 1e-12 * scale
        if spheres_only:
            Ls = np.abs(np.cross(st0[bo[e]:bo[e + 1], 0:3], m[bo[e]:bo[e + 1], None] *
                                 st0[bo[e]:bo[e + 1], 7:10])).sum()
            assert np.max(np.abs(L_of(st, e) - L0[e])) <= 1e-12 * Ls


def test_momentum_scene_changes_velocities():
    """Guard for the conservation test: collisions do redistribute momentum."""
    sc = V.momentum(n_envs=4)
    o = oracle.Oracle(sc)
    v0 = o.state()[:, 7:10].copy()
    o.step(60)
    assert np.max(np.abs(o.state()[:, 7:10] - v0)) > 0.1


# -------------------------------------------------------------------- stack
def test_resting_stack_stays_put():
    """Three touching boxes on the plane stay within 1e-4 m over 1000 steps.

    Run with 256 position iterations: each step restarts the solver cold,
    and with 8 sweeps the unconverged friction pyramid leaves a small yaw
    twist each step (0.8 mm drift per 200 steps); the drift falls ~50x per
    4x iterations, so it is convergence, not the contact model."""
    sc = V.stack(pos_iters=256)
    o = oracle.Oracle(sc)
    x0 = o.state()[:, 0:3].copy()
    q0 = o.state()[:, 3:7].copy()
    worst = 0.0
    for _ in range(10):
        o.step(100)
        st = o.state()
        worst = max(worst, np.max(np.abs(st[:, 0:3] - x0)))
        qd = np.minimum(np.abs(st[:, 3:7] - q0).max(1), np.abs(st[:, 3:7] + q0).max(1))
        assert np.max(qd) < 1e-4
    assert worst < 1e-4, worst


# ------------------------------------------------------------------ rolling
@pytest.mark.parametrize("kind", ["sphere", "capsule"])
def test_rolling_without_slip_keeps_its_speed(kind):
    """A sphere, and a capsule rolling on its side about its own axis, on a
    horizontal plane with v = w x (0, 0, r): Coulomb friction does no work
    on a rolling contact and nothing in the model resists rolling, so v and
    w stay exactly what they were and the centre stays at height r.  (With
    the contact anchors turned with the body inside a step, a rolling body
    sank by r (1 - cos theta) and was pushed back each step: it sped up.)"""
    from scenegen import CAPSULE, PLANE, SPHERE, body, pack
    r = 0.01
    if kind == "sphere":
        b = body(SPHERE, (r, 0, 0), 0.05, (0.0, 0.0, r))
        w = np.array([0.0, 20.0, 0.0])
    else:
        b = body(CAPSULE, (r, 0.02, 0), 0.05, (0.0, 0.0, r), quat=scenegen.axis_angle_quat((1, 0, 0), math.pi / 2))
        w = np.array([0.0, -20.0, 0.0])                  # along the capsule axis (world y)
    sc = pack("roll", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.8), b]], [[]], V.default_params(), 0, 0)
    o = oracle.Oracle(sc)
    st = o.state()
    v = np.cross(w, [0.0, 0.0, r])
    st[1, 7:10] = v
    st[1, 10:13] = w
    o.set_state(st)
    o.step(300)
    st = o.state()
    np.testing.assert_allclose(st[1, 7:10], v, atol=1e-9)
    np.testing.assert_allclose(st[1, 10:13], w, atol=1e-7)
    assert abs(st[1, 2] - r) < 1e-9
    assert abs(st[1, 0] - v[0] * 3.0) < 1e-6                 # 300 steps of 10 ms


# ---------------------------------------------------------------- pendulum
def _pend_phi(st):
    q = st[0, 3:7]
    return 2 * math.atan2(q[1], q[3])


def _capsule_Iy(r, l, m):
    b = np.zeros(22); b[0] = scenegen.CAPSULE; b[1] = r; b[2] = l; b[4] = m
    return oracle.inertia(b)[1]


def _period(sc, steps, dt):
    o = oracle.Oracle(sc)
    phis = []
    for _ in range(steps):
        o.step(1, actions=np.zeros((1, 1, 1)))
        phis.append(_pend_phi(o.state()))
    phis = np.array(phis)
    t = (np.arange(steps) + 1) * dt
    # zero crossings by linear interpolation
    zc = [t[i] - phis[i] * (t[i + 1] - t[i]) / (phis[i + 1] - phis[i])
          for i in range(steps - 1) if phis[i] == 0 or phis[i] * phis[i + 1] < 0]
    zc = np.array(zc)
    return 2 * np.mean(np.diff(zc)), phis


def test_pd_pendulum_small_angle_period():
    r, l, m, kp = 0.02, 0.1, 1.0, 2.0
    sc = V.pendulum(kp=kp, kd=0.0, r=r, l=l, m=m)
    I = _capsule_Iy(r, l, m) + m * l * l
    T = 2 * math.pi * math.sqrt(I / (kp + m * G * l))
    Tm, _ = _period(sc, 300, sc.params["dt"])
    assert abs(Tm - T) <= 0.01 * T, (Tm, T)


def test_pd_pendulum_damped_period():
    r, l, m, kp = 0.02, 0.1, 1.0, 2.0
    I = _capsule_Iy(r, l, m) + m * l * l
    w0 = math.sqrt((kp + m * G * l) / I)
    kd = 0.2 * I * w0
    sc = V.pendulum(kp=kp, kd=kd, r=r, l=l, m=m)
    Td = 2 * math.pi / math.sqrt(w0 * w0 - (kd / (2 * I)) ** 2)
    Tm, phis = _period(sc, 200, sc.params["dt"])
    assert abs(Tm - Td) <= 0.01 * Td, (Tm, Td)
    assert abs(phis[-1]) < 0.05 * 0.2   # it does decay


# -------------------------------------------------------- drive closed form
def test_isolated_drive_row_equals_implicit_euler():
    """A prismatic slider whose drive row is decoupled from every other row:
    each substep must give (m + h kd + h^2 kp) v' = m v - h kp C exactly,
    after any number of iterations (the row converges in one)."""
    kp, kd, m, target = 50.0, 2.0, 0.5, 0.1
    for iters in (1, 200):
        sc = V.slider(kp=kp, kd=kd, m=m, target=target, substeps=1, pos_iters=iters, vel_iters=0)
        o = oracle.Oracle(sc)
        h = sc.params["dt"]
        x, v = 0.0, 0.0
        for _ in range(20):
            o.step(1, actions=np.full((1, 1, 1), np.nan))
            C = x - float(np.float32(target))  # descriptor stores float32
            v = (m * v - h * kp * C) / (m + h * kd + h * h * kp)
            x = x + h * v
            st = o.state()
            assert abs(st[0, 7] - v) <= 1e-12 * max(1.0, abs(v))
            assert abs(st[0, 0] - x) <= 1e-12
        assert np.all(np.abs(st[0, 8:13]) < 1e-14)


# ------------------------------------------------------------------- limits
def test_joint_limit_holds_steady_state():
    upper = 1.0
    sc = V.limit(upper=upper, target=2.0)
    o = oracle.Oracle(sc)
    phis = []
    for _ in range(400):
        o.step(1, actions=np.full((1, 1, 1), np.nan))
        phis.append(_pend_phi(o.state()))
    phis = np.array(phis)
    assert phis[-1] <= upper + 1e-3
    assert phis[-1] > upper - 0.05       # pushed against the limit
    assert np.max(phis[200:]) <= upper + 1e-3


# -------------------------------------------------------- single-row solve
def test_single_row_one_iteration_is_exact():
    """A sphere touching the plane (d = 0), mu = 0, one substep, one
    iteration: the normal row cancels the approach velocity exactly."""
    sc = scenegen.pack("row", [[scenegen.body(scenegen.PLANE, (0, 0, 0), 0, (0, 0, 0), mu=0.0),
                                scenegen.body(scenegen.SPHERE, (0.05, 0, 0), 1.0, (0.1, 0.2, 0.05),
                                              linvel=(0.3, -0.1, -1.0), mu=0.0)]], [[]],
                       V.default_params(substeps=1, pos_iters=1, vel_iters=0), 0, 0)
    o = oracle.Oracle(sc)
    o.step(1)
    st = o.state()
    assert st[1, 9] == 0.0
    assert st[1, 7] == np.float32(0.3) and st[1, 8] == np.float32(-0.1)
    assert abs(st[1, 2] - np.float32(0.05)) == 0.0


# --------------------------------------------------------------------- LCP
@pytest.mark.parametrize("tilt", [(0.0, 0.0), (0.02, 0.0), (0.015, -0.01), (0.3, 0.2)])
def test_frictionless_contacts_converge_to_lcp_solution(tilt):
    sc = V.resting_box(tilt=tilt, mu=0.0, substeps=1, pos_iters=2000, vel_iters=0)
    o = oracle.Oracle(sc)
    st0 = o.state()
    o.step(1)
    rows = o.rows(0)
    normals = rows[rows[:, 2] == 0]
    n = len(normals)
    assert 1 <= n <= 4
    # Build the LCP w = A lam + q, lam >= 0, w >= 0, lam.w = 0 from the
    # rows' Jacobians and the box's own mass properties.
    m = float(sc.bodies["mass"][1])
    Ib = oracle.inertia(oracle.body_rows(sc.bodies[1:2])[0])
    R = rot(st0[1, 3:7])
    Iinv = R @ np.diag(1.0 / Ib) @ R.T
    J = np.hstack([normals[:, 3:6], normals[:, 6:9]])       # body A = box
    Minv = np.zeros((6, 6)); Minv[:3, :3] = np.eye(3) / m; Minv[3:, 3:] = Iinv
    A = J @ Minv @ J.T
    h = sc.params["dt"]
    v_pre = np.concatenate([st0[1, 7:10] + h * np.array(sc.params["gravity"]), st0[1, 10:13]])
    q = J @ v_pre + normals[:, 13]
    best = None
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            lam = np.zeros(n)
            if S:
                S = list(S)
                try:
                    lam[S] = np.linalg.solve(A[np.ix_(S, S)], -q[S])
                except np.linalg.LinAlgError:
                    continue
            w = A @ lam + q
            if np.all(lam >= -1e-12) and np.all(w >= -1e-10):
                best = lam
                break
        if best is not None:
            break
    assert best is not None
    # the oracle's converged impulses give the same velocity change
    np.testing.assert_allclose(Minv @ J.T @ normals[:, 14], Minv @ J.T @ best, atol=1e-9)
    w = A @ normals[:, 14] + q
    assert np.all(w >= -1e-9) and np.all(normals[:, 14] >= 0)


# ------------------------------------------------------------- narrowphase
def _b(type_, p, pos, quat=(0, 0, 0, 1), mass=1.0):
    """A float64 descriptor row (no float32 rounding of the literals)."""
    r = np.zeros(22)
    r[0] = type_; r[1:4] = p; r[4] = mass; r[5:8] = pos; r[8:12] = quat
    r[18] = 0.5; r[20] = 1; r[21] = 0xFFFF
    return r


def test_sphere_sphere_distance_and_normal():
    A = _b(scenegen.SPHERE, (0.05, 0, 0), (0.1, 0.02, 0.0))
    B = _b(scenegen.SPHERE, (0.04, 0, 0), (0.0, 0.0, 0.0))
    pts = oracle.collide(A, B, 0.1)
    cA, cB = np.array(A[5:8]), np.array(B[5:8])
    dist = np.linalg.norm(cA - cB)
    assert len(pts) == 1
    assert abs(pts[0, 9] - (dist - 0.09)) < 1e-15
    np.testing.assert_allclose(pts[0, 6:9], (cA - cB) / dist, atol=1e-15)
    np.testing.assert_allclose(pts[0, 0:3], cA - 0.05 * (cA - cB) / dist, atol=1e-15)


def test_plane_contacts_closed_form():
    q = V.axis_angle_quat((1, 1, 0), 0.7)
    P = _b(scenegen.PLANE, (0, 0, 0), (0, 0, 0.1), q, mass=0)
    N = rot(q)[:, 2]
    S = _b(scenegen.SPHERE, (0.05, 0, 0), (0.2, -0.1, 0.15))
    pts = oracle.collide(S, P, 0.5)
    assert abs(pts[0, 9] - ((np.array(S[5:8]) - np.array([0, 0, 0.1])) @ N - 0.05)) < 1e-15
    C = _b(scenegen.CAPSULE, (0.02, 0.05, 0), (0.0, 0.3, 0.2), V.axis_angle_quat((0, 1, 0), 0.4))
    pts = oracle.collide(C, P, 1.0)
    Rc = rot(C[8:12])
    ends = [np.array(C[5:8]) - 0.05 * Rc[:, 2], np.array(C[5:8]) + 0.05 * Rc[:, 2]]
    expect = [(e - np.array([0, 0, 0.1])) @ N - 0.02 for e in ends]
    np.testing.assert_allclose(pts[:, 9], expect, atol=1e-15)
    B = _b(scenegen.BOX, (0.03, 0.02, 0.01), (0.0, 0.0, 0.13), V.axis_angle_quat((1, 0, 0), 0.3))
    pts = oracle.collide(B, P, 0.2)
    Rb = rot(B[8:12])
    corners = [np.array(B[5:8]) + Rb @ np.array([sx * 0.03, sy * 0.02, sz * 0.01])
               for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)]
    dists = sorted((c - np.array([0, 0, 0.1])) @ N for c in corners)
    kept = sorted(pts[:, 9])
    # reduction keeps the deepest corner
    assert abs(kept[0] - dists[0]) < 1e-15
    assert len(pts) == 4


def test_capsule_capsule_crossed_segments():
    """Perpendicular segments, one above the other: distance is the offset."""
    A = _b(scenegen.CAPSULE, (0.01, 0.1, 0), (0.02, 0.03, 0.05), V.axis_angle_quat((0, 1, 0), math.pi / 2))
    B = _b(scenegen.CAPSULE, (0.02, 0.1, 0), (0.0, 0.0, 0.0), V.axis_angle_quat((1, 0, 0), math.pi / 2))
    pts = oracle.collide(A, B, 0.1)
    assert len(pts) == 1
    assert abs(pts[0, 9] - (0.05 - 0.03)) < 1e-12
    np.testing.assert_allclose(pts[0, 6:9], [0, 0, 1], atol=1e-12)


def test_capsule_capsule_parallel_gives_two_points():
    A = _b(scenegen.CAPSULE, (0.01, 0.05, 0), (0.03, 0.0, 0.025), V.axis_angle_quat((0, 1, 0), math.pi / 2))
    B = _b(scenegen.CAPSULE, (0.015, 0.05, 0), (0.0, 0.0, 0.0), V.axis_angle_quat((0, 1, 0), math.pi / 2))
    pts = oracle.collide(A, B, 0.1)
    assert len(pts) == 2
    np.testing.assert_allclose(pts[:, 9], 0.025 - 0.025, atol=1e-12)
    np.testing.assert_allclose(sorted(pts[:, 0]), [-0.02, 0.05], atol=1e-12)


def test_sphere_box_outside_and_inside():
    Bx = _b(scenegen.BOX, (0.05, 0.04, 0.03), (0, 0, 0), V.axis_angle_quat((0, 0, 1), 0.3))
    R = rot(Bx[8:12])
    local = np.array([0.08, 0.06, 0.0])    # beyond a vertical edge
    S = _b(scenegen.SPHERE, (0.01, 0, 0), R @ local)
    pts = oracle.collide(S, Bx, 0.1)
    assert abs(pts[0, 9] - (np.hypot(0.03, 0.02) - 0.01)) < 1e-12
    local = np.array([0.01, 0.035, 0.0])   # inside, nearest face +y at 0.005
    S = _b(scenegen.SPHERE, (0.01, 0, 0), R @ local)
    pts = oracle.collide(S, Bx, 0.1)
    assert abs(pts[0, 9] - (-0.005 - 0.01)) < 1e-12
    np.testing.assert_allclose(pts[0, 6:9], R[:, 1], atol=1e-12)


def test_box_face_rest_gives_overlap_rectangle_corners():
    """Axis-aligned box resting on a larger one, offset in x and y: the four
    points are the exact corners of the overlap rectangle."""
    top = _b(scenegen.BOX, (0.03, 0.02, 0.01), (0.05, -0.01, 0.02 + 0.01 - 0.0005))
    bot = _b(scenegen.BOX, (0.06, 0.05, 0.02), (0.0, 0.0, 0.0))
    pts = oracle.collide(top, bot, 0.01)
    assert len(pts) == 4
    xs = sorted({round(x, 12) for x in pts[:, 3]})
    ys = sorted({round(y, 12) for y in pts[:, 4]})
    assert xs == [0.02, 0.06] and ys == [-0.03, 0.01]
    np.testing.assert_allclose(pts[:, 9], -0.0005, atol=1e-12)
    np.testing.assert_allclose(pts[:, 6:9], np.tile([0, 0, 1], (4, 1)), atol=1e-15)
    np.testing.assert_allclose(pts[:, 5], 0.02, atol=1e-15)


def _sat_sep_sampled(A, B, n_dir=20000, seed=0):
    g = np.random.default_rng(seed)
    L = g.standard_normal((n_dir, 3))
    L /= np.linalg.norm(L, axis=1, keepdims=True)
    RA, RB = rot(A[8:12]), rot(B[8:12])
    hA, hB = np.array(A[1:4]), np.array(B[1:4])
    d = np.array(A[5:8]) - np.array(B[5:8])
    ra = np.abs(L @ RA) @ hA
    rb = np.abs(L @ RB) @ hB
    return np.max(np.abs(L @ d) - ra - rb)


@pytest.mark.parametrize("seed", range(6))
def test_box_box_depth_matches_sampled_directions(seed):
    g = scenegen.rng(99, seed, 0)
    hA = g.uniform(0.01, 0.03, 3)
    hB = g.uniform(0.01, 0.03, 3)
    qA, qB = scenegen.shoemake_quat(g), scenegen.shoemake_quat(g)
    dirv = g.standard_normal(3); dirv /= np.linalg.norm(dirv)
    A = _b(scenegen.BOX, hA, dirv * 0.6 * (np.linalg.norm(hA) + np.linalg.norm(hB)) * 0.8, qA)
    B = _b(scenegen.BOX, hB, (0, 0, 0), qB)
    pts = oracle.collide(A, B, 0.0)
    sampled = _sat_sep_sampled(A, B)
    assert len(pts) > 0, "the case must overlap"
    depth = pts[:, 9].min()
    # SAT's separation is the exact maximum over all directions: no sampled
    # direction exceeds it (and the deepest point is at least that deep),
    # and the best of 20k samples comes within the sampling resolution
    assert sampled <= depth + 1e-12
    assert depth - sampled < 1e-3


# ---------------------------------------------------------------- colouring
def test_colouring_valid_greedy_and_bounded():
    g = np.random.default_rng(5)
    nb = 30
    dyn = (g.random(nb) > 0.2).astype(np.int32)
    a = g.integers(-1, nb, 200).astype(np.int32)
    b = g.integers(-1, nb, 200).astype(np.int32)
    b[a == b] = -1                       # constraints join distinct bodies
    nc, col = oracle.color(a, b, dyn)
    assert nc == col.max() + 1
    # validity: two constraints of one colour share no dynamic body
    for c in range(nc):
        seen = set()
        for i in np.nonzero(col == c)[0]:
            for x in (a[i], b[i]):
                if x >= 0 and dyn[x]:
                    assert x not in seen
                    seen.add(x)
    # bound: colours <= max dynamic degree + 1
    deg = np.zeros(nb, int)
    for x in np.concatenate([a, b]):
        if x >= 0 and dyn[x]:
            deg[x] += 1
    assert nc <= deg.max() + 1
    # greedy: each constraint takes the smallest colour free on both bodies
    for i in range(len(a)):
        taken = set()
        for j in range(i):
            share = any(x >= 0 and dyn[x] and x in (a[j], b[j]) for x in (a[i], b[i]))
            if share:
                taken.add(col[j])
        assert col[i] == min(set(range(65)) - taken)


def test_colouring_overflow_reported():
    a = np.zeros(70, np.int32)
    b = np.full(70, -1, np.int32)
    nc, col = oracle.color(a, b, np.ones(1, np.int32))
    assert nc == -1 and col[64] == -1 and col[63] == 63


# ------------------------------------------------------------------ inertia
@pytest.mark.parametrize("kind,p", [(scenegen.SPHERE, (0.03, 0, 0)), (scenegen.BOX, (0.03, 0.02, 0.01)),
                                    (scenegen.CAPSULE, (0.02, 0.05, 0))])
def test_inertia_matches_voxel_quadrature(kind, p):
    """Uniform solid: compare with a midpoint-rule volume integral."""
    m = 1.7
    ext = {scenegen.SPHERE: (p[0],) * 3, scenegen.BOX: p,
           scenegen.CAPSULE: (p[0], p[0], p[0] + p[1])}[kind]
    n = 160
    axes = [np.linspace(-e, e, n, endpoint=False) + e / n for e in ext]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    if kind == scenegen.SPHERE:
        inside = X ** 2 + Y ** 2 + Z ** 2 <= p[0] ** 2
    elif kind == scenegen.BOX:
        inside = np.ones_like(X, bool)
    else:
        zc = np.clip(Z, -p[1], p[1])
        inside = X ** 2 + Y ** 2 + (Z - zc) ** 2 <= p[0] ** 2
    rho = m / inside.sum()
    I = np.array([((Y ** 2 + Z ** 2) * inside).sum(), ((X ** 2 + Z ** 2) * inside).sum(),
                  ((X ** 2 + Y ** 2) * inside).sum()]) * rho
    row = np.zeros(22); row[0] = kind; row[1:4] = p; row[4] = m
    np.testing.assert_allclose(oracle.inertia(row), I, rtol=3e-3)


# -------------------------------------------------------------- determinism
def test_oracle_deterministic_and_thread_independent():
    sc = scenegen.make_scene("clutter", n_envs=12)
    a = oracle.Oracle(sc); a.step(10, threads=1)
    b = oracle.Oracle(sc); b.step(10, threads=5)
    assert np.array_equal(a.state(), b.state())


def test_env_independent_of_batch_composition():
    sc = scenegen.make_scene("arm", n_envs=6)
    full = oracle.Oracle(sc); full.step(5)
    sub = oracle.Oracle(sc.subset([4, 1])); sub.step(5)
    bo = sc.body_off
    st = full.state()
    ss = sub.state()
    n4 = bo[5] - bo[4]
    assert np.array_equal(ss[:n4], st[bo[4]:bo[5]])
    assert np.array_equal(ss[n4:], st[bo[1]:bo[2]])


def test_static_bodies_never_move():
    sc = scenegen.make_scene("clutter", n_envs=4)
    o = oracle.Oracle(sc); o.step(20)
    st = o.state()
    static = sc.bodies["mass"] == 0
    np.testing.assert_array_equal(st[static, 0:3], sc.bodies["pos"][static].astype(np.float64))
    assert np.all(st[static, 7:13] == 0)


# ------------------------------------------------------------------ soft rows
def _soft(hz, zeta, h):
    om = 2 * math.pi * hz
    return om, 1.0 + 2 * zeta * om * h + (h * om) ** 2


@pytest.mark.parametrize("vel_iters", [0, 1])
@pytest.mark.parametrize("delta,v0", [(0.004, 0.0), (-0.002, 0.3)])
def test_isolated_soft_joint_row_is_implicit_euler(vel_iters, delta, v0):
    """A soft joint equality row is a spring-damper of frequency omega and
    damping ratio zeta on the row's effective mass, integrated implicitly:
    a body on a world prismatic joint (axis x, no drive, g = 0), off the axis
    by delta along y with speed v0 along y.  One substep of position
    iterations gives (1 + 2 zeta omega h + h^2 omega^2) v' = v0 - h omega^2
    delta, the position then moves by h v'; a relax sweep (rigid, zero
    bias) then removes v' along the row."""
    hz, zeta = 60.0, 2.0
    sc = V.slider(kp=0.0, kd=0.0, substeps=1, pos_iters=4, vel_iters=vel_iters, joint_hertz=hz,
                  joint_damping_ratio=zeta)
    sc.bodies["pos"][0, 1] = delta
    sc.bodies["linvel"][0, 1] = v0
    d = oracle.body_rows(sc.bodies)
    delta, v0 = d[0, 6], d[0, 13]                       # as stored (float32)
    o = oracle.Oracle(sc)
    o.step(1)
    st = o.state()
    h = sc.params["dt"]
    om, den = _soft(hz, zeta, h)
    v1 = (v0 - h * om * om * delta) / den
    assert abs(st[0, 1] - (delta + h * v1)) < 1e-12
    assert abs(st[0, 8] - (0.0 if vel_iters else v1)) < 1e-12


def test_soft_joint_rows_off_are_rigid():
    """joint_hertz = 0: the equality row removes the whole error in one
    substep (bias C / h) -- the rigid row."""
    sc = V.slider(kp=0.0, kd=0.0, substeps=1, pos_iters=4, vel_iters=0)
    sc.bodies["pos"][0, 1] = 0.004
    o = oracle.Oracle(sc)
    o.step(1)
    assert abs(o.state()[0, 1]) < 1e-12


def _box_stack(n, **pk):
    from scenegen import BOX, PLANE, body, pack
    h, m = 0.02, 0.1
    bl = [body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.5, group=1)]
    bl += [body(BOX, (h, h, h), m, (0, 0, h + 2 * h * k), mu=0.5, group=2) for k in range(n)]
    return pack("stack", [bl], [[]], scenegen.default_params(**pk), 0, 0), h


def test_soft_contact_rest_sinks_by_g_over_omega_squared():
    """A box resting on the plane under soft contacts (30 Hz): each point is a
    spring of stiffness m_eff omega^2 and the four points share the weight,
    so the box settles g / omega^2 into the plane and stays there."""
    sc, h = _box_stack(1, warm_start=1)
    om = 2 * math.pi * sc.params["contact_hertz"]
    o = oracle.Oracle(sc)
    o.step(400)
    st = o.state()
    assert abs(st[1, 2] - (h - 9.81 / om ** 2)) < 1e-9
    assert np.abs(st[1, 7:13]).max() < 1e-9


def test_stack_at_workload_settings_settles_at_its_spring_equilibrium_and_stays():
    """Three touching boxes (0.02 m, 0.1 kg) on the plane at the small
    workload's settings (dt 0.01, 4 substeps, 8 + 1 sweeps, soft contacts,
    warm start): the contacts are springs of m_eff omega^2 with m_eff = m
    (box - plane) and m / 2 (box - box), carrying 3, 2 and 1 weights, so the
    boxes sink by 3, 3 + 4 and 3 + 4 + 2 times g / omega^2.  Each box stays
    within 1e-4 m of that rest pose over 1000 steps."""
    sc, h = _box_stack(3, warm_start=1)
    p = sc.params
    assert (p["dt"], p["substeps"], p["pos_iters"], p["vel_iters"]) == (0.01, 4, 8, 1)
    om = 2 * math.pi * p["contact_hertz"]
    s = 9.81 / om ** 2
    rest = sc.bodies["pos"].astype(np.float64)[1:].copy()
    rest[:, 2] -= np.array([3, 7, 9]) * s
    o = oracle.Oracle(sc)
    o.step(200)                                      # settling
    worst = 0.0
    for _ in range(10):
        o.step(100)
        st = o.state()
        worst = max(worst, np.abs(st[1:, 0:3] - rest).max())
    assert worst < 1e-4, worst
    # the settled state is the spring equilibrium itself, far tighter than the bar
    assert np.abs(o.state()[1:, 2] - rest[:, 2]).max() < 1e-6


@pytest.mark.parametrize("warm", [0, 1])
def test_arm_workload_stays_bounded(warm):
    """The arm workload's light fingers (0.05 kg on 0.5-3 kg links) do not
    gain speed with soft joint rows, cold or warm started: every body stays
    below 10 m/s over 200 steps of random targets (rigid joint rows reach
    100+ m/s in most envs)."""
    sc = scenegen.make_scene("arm", n_envs=32)
    sc.params = dict(sc.params, warm_start=warm)
    o = oracle.Oracle(sc)
    top = 0.0
    for k in range(4):
        o.step(50, actions=sc.actions(50 * k, 50), threads=8)
        top = max(top, np.linalg.norm(o.state()[:, 7:10], axis=1).max())
    assert top < 10.0, top


@pytest.mark.parametrize("u", [1.0, 0.3])
def test_speculative_soft_contact_closed_form(u):
    """A sphere a gap d above the plane, approaching at speed u, g = 0, one
    substep of one position sweep: the soft normal row keeps the speculative
    bias d / h, so it acts only if u > d / h and then leaves the normal
    speed -u + ms (u - d / h), ms = a2 / (1 + a2) the contact mass scale."""
    from scenegen import PLANE, SPHERE, body, pack
    h, d, r, hz, zeta = 0.0025, 0.001, 0.02, 30.0, 10.0
    sc = pack("spec", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)),
                        body(SPHERE, (r, 0, 0), 0.1, (0, 0, r + d), linvel=(0, 0, -u))]], [[]],
              scenegen.default_params(dt=h, substeps=1, pos_iters=1, vel_iters=0, gravity=(0.0, 0.0, 0.0),
                                      contact_hertz=hz, contact_damping_ratio=zeta), 0, 0)
    rows = oracle.body_rows(sc.bodies)
    d, u = rows[1, 7] - rows[1, 1], -rows[1, 14]                # as stored (float32)
    o = oracle.Oracle(sc)
    o.step(1)
    om = 2 * math.pi * hz
    a2 = h * om * (2 * zeta + h * om)
    ms = a2 / (1 + a2)
    vz = -u + ms * (u - d / h) if u > d / h else -u
    assert abs(o.state()[1, 9] - vz) < 1e-12
