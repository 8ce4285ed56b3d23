"""Pins of the oracle's convex hulls: mass properties, the hull contact
routines and rendering.

A hull made of a box's corners must behave exactly like the box primitive
(mass properties, contact with a plane, rendering); sphere-hull gaps follow
from the geometry; the hull-hull penetration depth is the best separation
over sampled directions; inertia of an octahedron and of random hulls meets
its closed form / a grid quadrature.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import validation as V
from scenegen import BOX, HULL, PLANE, SPHERE, body, pack
from scenegen import hulls as H


def _scene(bodies, assets, **pk):
    """A probe scene with rigid rows, like the other pin scenes."""
    sc = pack("hull_probe", [bodies], [[]], V.default_params(**pk), 0, 0)
    sc.hulls = H.library(assets)
    return sc


def test_box_hull_inertia_is_the_box_formula():
    v, t = H.box_asset(0.03, 0.02, 0.05)
    m = 2.0
    I = oracle.hull_inertia(v, t, m)
    hx, hy, hz = (float(np.float32(x)) for x in (0.03, 0.02, 0.05))
    np.testing.assert_allclose(I, [m / 3 * (hy * hy + hz * hz), m / 3 * (hx * hx + hz * hz), m / 3 * (hx * hx + hy * hy)],
                               rtol=1e-12)


def test_octahedron_inertia():
    """|x| + |y| + |z| <= a: E[x^2] = a^2 / 10, so I = m a^2 / 5 about every axis."""
    a = 0.5
    v = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, a], [0, 0, -a]], np.float64)
    vv, tt = H.hull_asset(v)
    I = oracle.hull_inertia(vv, tt, 3.0)
    np.testing.assert_allclose(I, 3.0 * a * a / 5, rtol=1e-6)


def test_random_hull_inertia_matches_quadrature():
    g = np.random.default_rng(3)
    v, t = H.hull_asset(H.random_points(g, 12, np.array([0.03, 0.02, 0.04])))
    I = oracle.hull_inertia(v, t, 1.0)
    vv = v.astype(np.float64)
    a, b, c = vv[t[:, 0]], vv[t[:, 1]], vv[t[:, 2]]
    n = np.cross(b - a, c - a); d = (n * a).sum(1)
    lo, hi = vv.min(0), vv.max(0)
    N = 90
    axes = [lo[k] + (hi[k] - lo[k]) * (np.arange(N) + 0.5) / N for k in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    inside = ((P @ n.T) <= d).all(1)
    Q = P[inside]
    rho = 1.0 / inside.sum()
    Iq = rho * np.array([(Q[:, 1] ** 2 + Q[:, 2] ** 2).sum(), (Q[:, 0] ** 2 + Q[:, 2] ** 2).sum(),
                         (Q[:, 0] ** 2 + Q[:, 1] ** 2).sum()])
    np.testing.assert_allclose(I, Iq, rtol=2e-2)


def test_box_hull_on_a_plane_moves_like_the_box():
    """Dropped tilted onto a plane, a hull of a box's corners and the box
    primitive produce the same contacts and the same trajectory."""
    hx, hy, hz = 0.03, 0.02, 0.025
    q = scenegen.axis_angle_quat(np.array([0.3, 1.0, 0.2]) / np.linalg.norm([0.3, 1.0, 0.2]), 0.4)
    plane = body(PLANE, (0, 0, 0), 0.0, (0, 0, 0), mu=0.6)
    box = body(BOX, (hx, hy, hz), 0.2, (0, 0, 0.08), quat=q, mu=0.6)
    hull = body(HULL, (0, 0, 0), 0.2, (0, 0, 0.08), quat=q, mu=0.6)
    sb = _scene([plane, box], [H.box_asset(hx, hy, hz)])
    sh = _scene([plane, hull], [H.box_asset(hx, hy, hz)])
    ob, oh = oracle.Oracle(sb), oracle.Oracle(sh)
    for _ in range(6):
        ob.step(25); oh.step(25)
        np.testing.assert_allclose(oh.state(), ob.state(), rtol=0, atol=1e-9)
    assert oh.state()[1, 2] < 0.03                      # it has landed


def test_box_resting_on_a_box_hull_rests_like_on_a_box():
    hx = 0.05
    lower_box = body(BOX, (hx, hx, hx), 0.0, (0, 0, hx))
    lower_hull = body(HULL, (0, 0, 0), 0.0, (0, 0, hx))
    top = body(BOX, (0.02, 0.03, 0.015), 0.1, (0.01, -0.005, 2 * hx + 0.015 + 0.002))
    plane = body(PLANE, (0, 0, 0), 0.0, (0, 0, 0))
    a = oracle.Oracle(_scene([plane, lower_box, top], [H.box_asset(hx, hx, hx)], pos_iters=16))
    b = oracle.Oracle(_scene([plane, lower_hull, top], [H.box_asset(hx, hx, hx)], pos_iters=16))
    a.step(200); b.step(200)
    np.testing.assert_allclose(b.state()[2, 0:3], a.state()[2, 0:3], atol=1e-5)
    assert np.abs(b.state()[2, 7:13]).max() < 1e-3


def _manifold(bodies, assets):
    sc = _scene(bodies, assets, gravity=(0.0, 0.0, 0.0))
    o = oracle.Oracle(sc)
    o.step(1)
    return o.manifolds(0)


def test_sphere_above_a_hull_face_and_near_a_vertex():
    hv, ht = H.box_asset(0.05, 0.05, 0.05)
    r = 0.01
    # above the +z face, 4 mm gap
    pairs, npts, pts = _manifold([body(SPHERE, (r, 0, 0), 0.1, (0.01, 0.02, 0.05 + r + 0.004)),
                                  body(HULL, (0, 0, 0), 0.0, (0, 0, 0))], [(hv, ht)])
    assert npts[0] == 1
    assert abs(pts[0, 0, 9] - 0.004) < 1e-7
    np.testing.assert_allclose(pts[0, 0, 6:9], [0, 0, 1], atol=1e-7)
    # off the corner (0.05, 0.05, 0.05) along (1, 1, 1): gap = 0.006
    u = np.ones(3) / math.sqrt(3)
    c = 0.05 + u * (r + 0.006)
    pairs, npts, pts = _manifold([body(SPHERE, (r, 0, 0), 0.1, tuple(c)),
                                  body(HULL, (0, 0, 0), 0.0, (0, 0, 0))], [(hv, ht)])
    assert abs(pts[0, 0, 9] - 0.006) < 1e-6
    np.testing.assert_allclose(pts[0, 0, 6:9], u, atol=1e-5)


def test_sphere_centre_inside_a_hull_is_pushed_out_of_the_nearest_face():
    hv, ht = H.box_asset(0.05, 0.04, 0.03)
    r = 0.01
    pairs, npts, pts = _manifold([body(SPHERE, (r, 0, 0), 0.1, (0.0, 0.035, 0.0)),
                                  body(HULL, (0, 0, 0), 0.0, (0, 0, 0))], [(hv, ht)])
    np.testing.assert_allclose(pts[0, 0, 6:9], [0, 1, 0], atol=1e-7)   # +y face is nearest (5 mm)
    assert abs(pts[0, 0, 9] - (-0.005 - r)) < 1e-7


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_hull_hull_depth_is_the_best_separating_direction(seed):
    g = np.random.default_rng(seed)
    a = H.hull_asset(H.random_points(g, 10, np.array([0.04, 0.03, 0.035])))
    b = H.hull_asset(H.random_points(g, 9, np.array([0.03, 0.04, 0.03])))
    qa, qb = scenegen.shoemake_quat(g), scenegen.shoemake_quat(g)
    xa, xb = np.array([0.0, 0.0, 0.0]), np.array([0.01, 0.015, 0.02])
    bodies = [body(HULL, (0, 0, 0), 0.1, tuple(xa), quat=qa), body(HULL, (1, 0, 0), 0.1, tuple(xb), quat=qb)]
    pairs, npts, pts = _manifold(bodies, [a, b])
    assert len(npts) == 1 and npts[0] >= 1
    dmin = pts[0, :npts[0], 9].min()
    # separation along u: min_B u.x - max_A u.x, best over many directions
    from scenegen.validation import _rot
    VA = a[0].astype(np.float64) @ np.array(_rot(qa)).T + xa
    VB = b[0].astype(np.float64) @ np.array(_rot(qb)).T + xb
    U = g.standard_normal((200000, 3)); U /= np.linalg.norm(U, axis=1)[:, None]
    sep = (VB @ U.T).min(0) - (VA @ U.T).max(0)
    best = sep.max()
    assert best <= dmin + 1e-9 + 1e-4       # no direction separates more than SAT found (1e-4: face preference)
    assert dmin - best < 2e-3, (dmin, best)


def test_box_hull_renders_like_the_box():
    hx, hy, hz = 0.06, 0.04, 0.05
    q = scenegen.axis_angle_quat((0.0, 0.6, 0.8), 0.7)
    cam = dict(eye=(0.4, -0.3, 0.3), target=(0, 0, 0), fov_y=math.radians(50), near=0.01, width=64, height=48)
    plane = body(PLANE, (0, 0, 0), 0.0, (0, 0, -0.1))
    ob = oracle.Oracle(_scene([plane, body(BOX, (hx, hy, hz), 0.0, (0, 0, 0), quat=q)], [H.box_asset(hx, hy, hz)]))
    oh = oracle.Oracle(_scene([plane, body(HULL, (0, 0, 0), 0.0, (0, 0, 0), quat=q)], [H.box_asset(hx, hy, hz)]))
    col = np.array([[0.5, 0.5, 0.5], [0.9, 0.3, 0.1]])
    rb, db, sb, tb = ob.render(cam, col)
    rh, dh, sh, th = oh.render(cam, col)
    np.testing.assert_array_equal(sb, sh)
    np.testing.assert_array_equal(rb, rh)
    np.testing.assert_allclose(dh, db, rtol=1e-12)
    assert (sh == 2).sum() > 100


def test_capsule_over_a_hull_face_gets_two_points():
    """A capsule along x lying 3 mm above the top face of a box-shaped hull,
    over one of the face's two triangles: its two ends, at the gap."""
    from scenegen import CAPSULE
    hv, ht = H.box_asset(0.05, 0.05, 0.05)
    r, l = 0.01, 0.02
    q = scenegen.axis_angle_quat((0, 1, 0), math.pi / 2)              # capsule axis along x
    pairs, npts, pts = _manifold([body(CAPSULE, (r, l, 0), 0.1, (0.0, -0.03, 0.05 + r + 0.003), quat=q),
                                  body(HULL, (0, 0, 0), 0.0, (0, 0, 0))], [(hv, ht)])
    assert npts[0] == 2
    np.testing.assert_allclose(pts[0, :2, 9], 0.003, atol=1e-7)
    np.testing.assert_allclose(sorted(pts[0, :2, 3]), [-l, l], atol=1e-7)   # cB x = the segment's ends
    np.testing.assert_allclose(pts[0, :2, 6:9], [[0, 0, 1], [0, 0, 1]], atol=1e-7)


def test_capsule_beside_a_hull_corner_takes_the_closest_points():
    """A vertical capsule whose lower end sits outside the corner (0.05,
    0.05, 0.05): no face region holds it, so the exact closest points give
    the gap |end - corner| - r."""
    from scenegen import CAPSULE
    hv, ht = H.box_asset(0.05, 0.05, 0.05)
    r, l = 0.01, 0.02
    end = np.array([0.06, 0.06, 0.055])
    pairs, npts, pts = _manifold([body(CAPSULE, (r, l, 0), 0.1, tuple(end + [0, 0, l])),
                                  body(HULL, (0, 0, 0), 0.0, (0, 0, 0))], [(hv, ht)])
    gap = np.linalg.norm(end - 0.05)
    assert npts[0] == 1
    assert abs(pts[0, 0, 9] - (gap - r)) < 1e-7
    np.testing.assert_allclose(pts[0, 0, 6:9], (end - 0.05) / gap, atol=1e-6)
    np.testing.assert_allclose(pts[0, 0, 3:6], [0.05, 0.05, 0.05], atol=1e-7)


def test_capsule_across_a_hull_edge_takes_the_edge_axis():
    """A capsule in the xz plane crossing over the top +x edge (along y) of a
    box-shaped hull, skew to it, 4 mm out along the edge's outward bisector:
    the segment x edge axis separates most; the gap is 4 mm."""
    from scenegen import CAPSULE
    hv, ht = H.box_asset(0.05, 0.05, 0.05)
    r, l = 0.01, 0.02
    bis = np.array([1.0, 0.0, 1.0]) / math.sqrt(2)
    c = np.array([0.05, 0.0, 0.05]) + bis * (r + 0.004)
    q = scenegen.axis_angle_quat((0, 1, 0), -math.pi / 4)             # capsule axis (1, 0, -1)/sqrt(2)
    pairs, npts, pts = _manifold([body(CAPSULE, (r, l, 0), 0.1, tuple(c), quat=q),
                                  body(HULL, (0, 0, 0), 0.0, (0, 0, 0))], [(hv, ht)])
    assert npts[0] == 1
    assert abs(pts[0, 0, 9] - 0.004) < 1e-6
    np.testing.assert_allclose(pts[0, 0, 6:9], bis, atol=1e-6)


def test_capsule_dropped_on_a_hull_lands_and_keeps_its_energy():
    """A capsule dropped onto a static hull bounces off it onto the plane:
    it stays above both, its energy never grows after the first contact,
    and once it rolls on the plane (no rolling resistance in the model) its
    speed is constant and its centre stays at height r."""
    from scenegen import CAPSULE
    g = np.random.default_rng(9)
    assets = [H.hull_asset(H.random_points(g, 12, np.array([0.06, 0.05, 0.03])))]
    r, l, m = 0.01, 0.02, 0.05
    sc = pack("cap_hull", [[body(PLANE, (0, 0, 0), 0.0, (0, 0, 0)), body(HULL, (0, 0, 0), 0.0, (0, 0, 0.03)),
                            body(CAPSULE, (r, l, 0), m, (0.005, 0.0, 0.15),
                                 quat=scenegen.axis_angle_quat((1, 0, 0), 1.2))]], [[]],
              V.default_params(), 0, 0)
    sc.hulls = H.library(assets)
    o = oracle.Oracle(sc)
    # principal moments of the capsule about its axis (z) and across it
    vc, vs = math.pi * r * r * 2 * l, 4.0 / 3.0 * math.pi * r ** 3
    mc, ms_ = m * vc / (vc + vs), m * vs / (vc + vs)
    Iz = mc * r * r / 2 + ms_ * 2 * r * r / 5
    Ix = (mc * (3 * r * r + 4 * l * l) / 12 + ms_ * (2 * r * r / 5 + l * l + 3 * l * r / 4))

    def energy(st):
        x, q, v, w = st[2, 0:3], st[2, 3:7], st[2, 7:10], st[2, 10:13]
        R = _qmat(q)
        wl = R.T @ w
        return 0.5 * m * v @ v + 0.5 * (Ix * (wl[0] ** 2 + wl[1] ** 2) + Iz * wl[2] ** 2) + m * 9.81 * x[2]

    es, zs = [], []
    for k in range(40):
        o.step(10)
        st = o.state()
        assert np.isfinite(st).all()
        es.append(energy(st))
        zs.append(st[2, 2])
    assert min(zs) > r - 1e-3                                         # never through the plane
    e = np.array(es[2:])                                              # after the first contact
    assert (np.diff(e) <= 1e-6 * e[0]).all(), np.diff(e).max()
    st = o.state()
    assert abs(st[2, 2] - r) < 1e-4 and abs(st[2, 9]) < 1e-6          # rolling on the plane
    np.testing.assert_allclose(es[-1], es[-10], rtol=1e-6)


def _qmat(q):
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
