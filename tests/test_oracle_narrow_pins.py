"""Pins of the oracle's narrowphase routines that the workloads call and the
older pins leave open: sphere - capsule, capsule - box (face, clipped face,
edge, and the exact fallback), box - box edge - edge, box - box face clipping
at a general orientation against an exact rational polygon intersection,
the manifold reduction's four selection rules, the tangent basis rule, and
the principal frame of the hull assets.

Every expected value is a closed form of the configuration or is computed
here by a different construction than the oracle's (exact rationals,
brute-force geometry); each configuration is also moved by a random rigid
motion, which the contacts must follow (points and normals rotate,
separations do not change).  Contact geometry: n points from B toward A,
d = n . (cA - cB), A the lower shape rank (sphere < capsule < box < plane)."""
from fractions import Fraction as Fr
import itertools
import math

import numpy as np
import pytest

import oracle
import scenegen

SPHERE, CAPSULE, BOX = scenegen.SPHERE, scenegen.CAPSULE, scenegen.BOX


# ----------------------------------------------------------------- helpers
def qmul(a, b):
    ax, ay, az, aw = a
    bx, by, bz, bw = b
    return np.array([aw * bx + bw * ax + ay * bz - az * by, aw * by + bw * ay + az * bx - ax * bz,
                     aw * bz + bw * az + ax * by - ay * bx, aw * bw - ax * bx - ay * by - az * bz])


def quat_axis_angle(axis, ang):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    return np.array([*(a * math.sin(ang / 2)), math.cos(ang / 2)])


def rotm(q):
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def quat_of(R):
    """A unit quaternion of a rotation matrix (largest-component branch)."""
    R = np.asarray(R, np.float64)
    t = np.trace(R)
    if t > 0:
        s = math.sqrt(t + 1.0) * 2
        q = [(R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s, 0.25 * s]
    else:
        i = int(np.argmax(np.diag(R)))
        j, k = (i + 1) % 3, (i + 2) % 3
        s = math.sqrt(1.0 + R[i, i] - R[j, j] - R[k, k]) * 2
        q = [0.0] * 4
        q[i] = 0.25 * s
        q[j] = (R[j, i] + R[i, j]) / s
        q[k] = (R[k, i] + R[i, k]) / s
        q[3] = (R[k, j] - R[j, k]) / s
    q = np.array(q)
    return q / np.linalg.norm(q)


def body(type_, p, pos, quat=(0, 0, 0, 1), mass=1.0):
    r = np.zeros(22)
    r[0] = type_; r[1:4] = p; r[4] = mass; r[5:8] = pos; r[8:12] = quat
    r[18] = 0.5; r[20] = 1; r[21] = 0xFFFF
    return r


class Motion:
    """A seeded rigid motion x -> R x + t applied to whole configurations."""

    def __init__(self, seed):
        g = np.random.default_rng(seed)
        self.q = np.array([0, 0, 0, 1.0]) if seed == 0 else quat_of(rotm(scenegen.shoemake_quat(g)))
        self.R = rotm(self.q)
        self.t = np.zeros(3) if seed == 0 else g.uniform(-0.5, 0.5, 3)

    def body(self, type_, p, pos, quat=(0, 0, 0, 1)):
        return body(type_, p, self.R @ np.asarray(pos, np.float64) + self.t, qmul(self.q, quat))

    def point(self, x):
        return self.R @ np.asarray(x, np.float64) + self.t

    def vec(self, v):
        return self.R @ np.asarray(v, np.float64)


def check_point(pt, cA, cB, n, d, M, tol=1e-12):
    np.testing.assert_allclose(pt[0:3], M.point(cA), atol=tol)
    np.testing.assert_allclose(pt[3:6], M.point(cB), atol=tol)
    np.testing.assert_allclose(pt[6:9], M.vec(n), atol=tol)
    assert abs(pt[9] - d) < tol, (pt[9], d)
    # d is the separation of the witness points along n
    assert abs(pt[6:9] @ (pt[0:3] - pt[3:6]) - pt[9]) < tol


SEEDS = [0, 1, 2, 3]


# ---------------------------------------------------------- sphere - capsule
@pytest.mark.parametrize("seed", SEEDS)
def test_sphere_capsule_beside_the_segment(seed):
    """Sphere centre beside the segment's interior: the closest point is its
    perpendicular foot on the axis, d = distance - r_s - r_c."""
    M = Motion(seed)
    r_s, r_c, l = 0.02, 0.015, 0.06
    C = M.body(CAPSULE, (r_c, l, 0), (0, 0, 0))                # axis along z
    c = np.array([0.03, 0.04, 0.025])                          # foot (0, 0, 0.025)
    S = M.body(SPHERE, (r_s, 0, 0), c)
    pts = oracle.collide(S, C, 1.0)
    assert len(pts) == 1
    dist = math.hypot(0.03, 0.04)                               # 0.05
    n = np.array([0.6, 0.8, 0.0])
    check_point(pts[0], c - r_s * n, np.array([0, 0, 0.025]) + r_c * n, n, dist - r_s - r_c, M)


@pytest.mark.parametrize("seed", SEEDS)
def test_sphere_capsule_beyond_an_end_clamps_to_the_end(seed):
    """Sphere centre past the +z end: the clamped closest point is the end
    point, n along the centre - end direction."""
    M = Motion(seed)
    r_s, r_c, l = 0.02, 0.015, 0.06
    C = M.body(CAPSULE, (r_c, l, 0), (0, 0, 0))
    end = np.array([0, 0, l])
    c = end + np.array([0.012, 0.0, 0.035])                     # |offset| = 0.037
    S = M.body(SPHERE, (r_s, 0, 0), c)
    pts = oracle.collide(S, C, 1.0)
    dist = math.hypot(0.012, 0.035)
    n = (c - end) / dist
    check_point(pts[0], c - r_s * n, end + r_c * n, n, dist - r_s - r_c, M)
    # and below the -z end, the other clamp
    c2 = -end + np.array([0.0, -0.02, -0.021])
    S2 = M.body(SPHERE, (r_s, 0, 0), c2)
    pts = oracle.collide(S2, C, 1.0)
    dist = math.hypot(0.02, 0.021)
    n = (c2 + end) / dist
    check_point(pts[0], c2 - r_s * n, -end + r_c * n, n, dist - r_s - r_c, M)


# ------------------------------------------------------------- capsule - box
H = np.array([0.05, 0.04, 0.03])           # box half-extents


def capsule_along(u, centre, M, r, half):
    """A capsule (radius r, half-length half) whose axis (local +z) is u."""
    u = np.asarray(u, np.float64) / np.linalg.norm(u)
    z = np.array([0, 0, 1.0])
    ax = np.cross(z, u)
    s = np.linalg.norm(ax)
    q = np.array([0, 0, 0, 1.0]) if s < 1e-15 else quat_axis_angle(ax, math.atan2(s, z @ u))
    return M.body(CAPSULE, (r, half, 0), centre, q)


@pytest.mark.parametrize("seed", SEEDS)
def test_capsule_lying_over_a_box_face_gives_its_two_ends(seed):
    """A capsule lying flat over the +z face, inside the face's slab: two
    points under the segment ends, at the gap."""
    M = Motion(seed)
    r, half, gap = 0.01, 0.02, 0.004
    Bx = M.body(BOX, H, (0, 0, 0))
    centre = np.array([0.01, -0.005, H[2] + r + gap])
    u = np.array([1.0, 0.5, 0.0]) / math.sqrt(1.25)
    C = capsule_along(u, centre, M, r, half)
    pts = oracle.collide(C, Bx, 0.05)
    assert len(pts) == 2
    z = np.array([0, 0, 1.0])
    # the oracle orients the segment by the capsule's local +z: ends -half, +half
    for pt, s in zip(pts, (-half, half)):
        e = centre + s * u
        check_point(pt, e - r * z, np.array([e[0], e[1], H[2]]), z, gap, M)


@pytest.mark.parametrize("seed", SEEDS)
def test_capsule_over_a_face_is_clipped_to_the_face(seed):
    """A tilted capsule over the +z face whose upper end lies past the face's
    +x side: the face case clips the segment at x = hx; both points sit at
    the face plane under the segment, d = the axis height - hz - r."""
    M = Motion(seed)
    r = 0.01
    s0 = np.array([-0.02, 0.01, 0.035 + r])
    s1 = np.array([0.09, 0.01, 0.045 + r])
    Bx = M.body(BOX, H, (0, 0, 0))
    C = capsule_along(s1 - s0, 0.5 * (s0 + s1), M, r, 0.5 * np.linalg.norm(s1 - s0))
    pts = oracle.collide(C, Bx, 0.05)
    assert len(pts) == 2
    z = np.array([0, 0, 1.0])
    t_clip = (H[0] - s0[0]) / (s1[0] - s0[0])
    for pt, t in zip(pts, (0.0, t_clip)):
        q = s0 + t * (s1 - s0)
        check_point(pt, q - r * z, np.array([q[0], q[1], H[2]]), z, q[2] - H[2] - r, M)


@pytest.mark.parametrize("seed", SEEDS)
def test_capsule_crossing_over_a_box_edge_gives_the_edge_point(seed):
    """The segment crosses over the box edge (x = hx, z = hz) at right angles
    to it, diagonally above: the edge axis (1, 0, 1)/sqrt 2 beats both faces
    and the point is the segment - edge closest pair, d = sqrt2 a - r."""
    M = Motion(seed)
    r, a, half = 0.006, 0.01, 0.03
    Bx = M.body(BOX, H, (0, 0, 0))
    centre = np.array([H[0] + a, 0.004, H[2] + a])
    u = np.array([1.0, 0.0, -1.0]) / math.sqrt(2)
    C = capsule_along(u, centre, M, r, half)
    pts = oracle.collide(C, Bx, 0.05)
    assert len(pts) == 1
    n = np.array([1.0, 0.0, 1.0]) / math.sqrt(2)
    check_point(pts[0], centre - r * n, np.array([H[0], 0.004, H[2]]), n, math.sqrt(2) * a - r, M)


@pytest.mark.parametrize("seed", SEEDS)
def test_capsule_parallel_to_an_edge_falls_back_to_exact_closest_points(seed):
    """A capsule parallel to the box edge (x = hx, z = hz), diagonally off
    it: no SAT axis of the routine is the diagonal, the best face's slab
    misses the segment, and the exact segment - box closest points give
    d = sqrt2 a - r along the diagonal."""
    M = Motion(seed)
    r, a, half = 0.004, 0.01, 0.02
    Bx = M.body(BOX, H, (0, 0, 0))
    centre = np.array([H[0] + a, 0.0, H[2] + a])
    C = capsule_along((0, 1, 0), centre, M, r, half)
    pts = oracle.collide(C, Bx, 0.05)
    assert len(pts) == 1
    n = np.array([1.0, 0.0, 1.0]) / math.sqrt(2)
    # the witness lies on the edge; along it any point is as close: compare
    # the geometry that is unique (d, n, and that cB is on the edge)
    np.testing.assert_allclose(pts[0, 6:9], M.vec(n), atol=1e-12)
    assert abs(pts[0, 9] - (math.sqrt(2) * a - r)) < 1e-12
    cB_local = M.R.T @ (pts[0, 3:6] - M.t)
    np.testing.assert_allclose(cB_local[[0, 2]], [H[0], H[2]], atol=1e-12)
    assert abs(cB_local[1]) <= half + 1e-12


# -------------------------------------------------------- box - box, edges
@pytest.mark.parametrize("seed", SEEDS)
def test_box_box_crossed_edges_give_one_edge_edge_point(seed):
    """Two cubes turned 45 degrees about x and y: A's lowest edge (along x)
    crosses over B's highest edge (along y) at a gap g.  The edge axis
    A_x x B_y = z wins; one point at the crossing, d = g."""
    M = Motion(seed)
    h, g = 0.05, 0.003
    c = h * math.sqrt(2)
    qa = quat_axis_angle((1, 0, 0), math.pi / 4)
    qb = quat_axis_angle((0, 1, 0), math.pi / 4)
    xa = np.array([0.004, -0.006, 2 * c + g])
    B = M.body(BOX, (h, h, h), (0, 0, 0), qb)
    A = M.body(BOX, (h, h, h), xa, qa)
    pts = oracle.collide(A, B, 0.05)
    assert len(pts) == 1
    z = np.array([0, 0, 1.0])
    # A's edge runs along x through (*, -0.006, c + g), B's along y through
    # (0, *, c): the closest points are where they cross, above each other
    check_point(pts[0], np.array([0.0, -0.006, c + g]), np.array([0.0, -0.006, c]), z, g, M)


# ------------------------------------------- box - box, face clipping (exact)
def frac_rot(c, s, axis):
    """Exact rotation matrix (Fractions) by the angle with cosine c, sine s."""
    assert c * c + s * s == 1
    o, z = Fr(1), Fr(0)
    if axis == 0:
        return [[o, z, z], [z, c, -s], [z, s, c]]
    if axis == 1:
        return [[c, z, s], [z, o, z], [-s, z, c]]
    return [[c, -s, z], [s, c, z], [z, z, o]]


def fmat(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(3)) for j in range(3)] for i in range(3)]


def fvec(A, v):
    return [sum(A[i][k] * v[k] for k in range(3)) for i in range(3)]


def ftr(A):
    return [[A[j][i] for j in range(3)] for i in range(3)]


def polygon_intersection(quad, hu, hv):
    """Vertices of quad (convex, 2D, Fractions) intersected with the
    rectangle [-hu, hu] x [-hv, hv], computed as a point set: quad vertices
    inside the rectangle, rectangle corners inside the quad, and crossings of
    a quad edge with a rectangle edge.  Exact."""
    rect = [(hu, hv), (-hu, hv), (-hu, -hv), (hu, -hv)]

    def inside_rect(p):
        return -hu <= p[0] <= hu and -hv <= p[1] <= hv

    def cross2(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    sgn = 1 if cross2(quad[0], quad[1], quad[2]) > 0 else -1

    def inside_quad(p):
        return all(sgn * cross2(quad[i], quad[(i + 1) % 4], p) >= 0 for i in range(4))

    out = set(p for p in quad if inside_rect(p))
    out |= set(p for p in rect if inside_quad(p))
    for i in range(4):
        a, b = quad[i], quad[(i + 1) % 4]
        for j in range(4):
            c, d = rect[j], rect[(j + 1) % 4]
            den = (b[0] - a[0]) * (d[1] - c[1]) - (b[1] - a[1]) * (d[0] - c[0])
            if den == 0:
                continue
            t = ((c[0] - a[0]) * (d[1] - c[1]) - (c[1] - a[1]) * (d[0] - c[0])) / den
            s = ((c[0] - a[0]) * (b[1] - a[1]) - (c[1] - a[1]) * (b[0] - a[0])) / den
            if 0 <= t <= 1 and 0 <= s <= 1:
                out.add((a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])))
    return out


CLIP_CASES = [
    # reference box, incident box (half-extents), incident centre in the
    # reference frame, in-plane turn (cos, sin), tilt about x (cos, sin);
    # each tilted so that the reference face's separation beats the
    # incident face's by more than the 1e-4 m face preference
    dict(hr=(Fr(1, 10), Fr(1, 50), Fr(1, 50)), hi=(Fr(3, 100), Fr(3, 100), Fr(1, 100)),
         c=(Fr(-85, 1000), Fr(3, 1000), Fr(1, 50) + Fr(1, 100) - Fr(1, 1000)),
         turn=(Fr(15, 17), Fr(8, 17)), tilt=(Fr(399, 401), Fr(40, 401))),
    dict(hr=(Fr(6, 100), Fr(5, 100), Fr(2, 100)), hi=(Fr(4, 100), Fr(2, 100), Fr(1, 100)),
         c=(Fr(-3, 100), Fr(4, 100), Fr(2, 100) + Fr(1, 100) + Fr(1, 2000)),
         turn=(Fr(3, 5), Fr(4, 5)), tilt=(Fr(399, 401), Fr(-40, 401))),
    dict(hr=(Fr(4, 100), Fr(4, 100), Fr(1, 100)), hi=(Fr(4, 100), Fr(4, 100), Fr(1, 100)),
         c=(Fr(1, 100), Fr(-1, 200), Fr(1, 100) + Fr(1, 100) - Fr(3, 1000)),
         turn=(Fr(12, 13), Fr(5, 13)), tilt=(Fr(1599, 1601), Fr(80, 1601))),
]


@pytest.mark.parametrize("case", range(len(CLIP_CASES)))
@pytest.mark.parametrize("ref_is_b", [True, False])
def test_box_box_face_clipping_equals_exact_polygon_intersection(case, ref_is_b):
    """The reference box lies at a general orientation (an exact rational
    rotation); the incident box rests on its top face, turned and tilted.
    The clip output must be the exact intersection of the incident face's
    projection with the reference face, each vertex at the incident face's
    exact height: checked against exact rational arithmetic (a point-set
    construction, not a Sutherland-Hodgman pass).  ref_is_b: the reference
    box is the second body of the pair (n from it toward the first); else
    the first, the incident box lying under it upside down."""
    cs = CLIP_CASES[case]
    RR = fmat(frac_rot(Fr(3, 5), Fr(4, 5), 2), frac_rot(Fr(5, 13), Fr(12, 13), 0))   # reference rotation
    Rrel = fmat(frac_rot(*cs["turn"], 2), frac_rot(*cs["tilt"], 0))
    if not ref_is_b:
        # flip the configuration upside down in the reference frame: the
        # reference box's -z face is then the contact face
        flip = frac_rot(Fr(-1), Fr(0), 0)
        Rrel = fmat(flip, Rrel)
    RI = fmat(RR, Rrel)
    xr = [Fr(1, 10), Fr(-1, 20), Fr(3, 100)]
    cl = list(cs["c"])
    if not ref_is_b:
        cl = [cl[0], -cl[1], -cl[2]]
    xi = [xr[k] + fvec(RR, cl)[k] for k in range(3)]
    hr, hi = cs["hr"], cs["hi"]
    f = lambda m: np.array([[float(x) for x in row] for row in m])
    qR, qI = quat_of(f(RR)), quat_of(f(RI))
    Bref = body(BOX, [float(x) for x in hr], [float(x) for x in xr], qR)
    Binc = body(BOX, [float(x) for x in hi], [float(x) for x in xi], qI)
    pair = (Binc, Bref) if ref_is_b else (Bref, Binc)
    cand = oracle.candidates(*pair, 0.01)

    # exact: the incident face is the incident box's face turned most toward
    # the reference face; its corners in the reference frame
    up = 1 if ref_is_b else -1
    nloc = [Fr(0), Fr(0), Fr(up)]                         # reference face normal, reference frame
    Rl = fmat(ftr(RR), RI)                                # incident axes in the reference frame
    best = None
    for ax, sg in itertools.product(range(3), (1, -1)):
        dd = sg * sum(Rl[k][ax] * nloc[k] for k in range(3))
        if best is None or dd < best[0]:
            best = (dd, ax, sg)
    _, ax, sg = best
    o1, o2 = (ax + 1) % 3, (ax + 2) % 3
    corners = []
    for s1, s2 in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        loc = [Fr(0)] * 3
        loc[ax] = sg * hi[ax]; loc[o1] = s1 * hi[o1]; loc[o2] = s2 * hi[o2]
        corners.append([cl[k] + fvec(Rl, loc)[k] for k in range(3)])
    quad = [(p[0], p[1]) for p in corners]
    poly = polygon_intersection(quad, hr[0], hr[1])
    # the incident face plane z = a u + b v + c through three corners
    p0, p1, p2 = corners[0], corners[1], corners[2]
    m = [[p0[0], p0[1], Fr(1)], [p1[0], p1[1], Fr(1)], [p2[0], p2[1], Fr(1)]]
    det = lambda M: (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                     + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))
    D = det(m)
    rhs = [p0[2], p1[2], p2[2]]
    sol = []
    for col in range(3):
        mm = [row[:] for row in m]
        for r_ in range(3):
            mm[r_][col] = rhs[r_]
        sol.append(det(mm) / D)
    height = lambda u, v: sol[0] * u + sol[1] * v + sol[2]

    assert len(cand) == len(poly), (len(cand), len(poly))
    RRf = f(RR)
    nref_w = RRf @ np.array([0, 0, float(up)])
    exact = [(float(u), float(v), float(height(u, v))) for u, v in poly]
    seen = set()
    for c_ in cand:
        x_inc = c_[0:3] if ref_is_b else c_[3:6]           # the point on the incident face
        x_ref = c_[3:6] if ref_is_b else c_[0:3]           # its projection on the reference face
        loc = RRf.T @ (x_inc - np.array([float(v) for v in xr]))
        k = min(range(len(exact)), key=lambda i: abs(exact[i][0] - loc[0]) + abs(exact[i][1] - loc[1]))
        assert k not in seen
        seen.add(k)
        np.testing.assert_allclose(loc, exact[k], atol=1e-12)
        dist = up * exact[k][2] - float(hr[2])
        assert abs(c_[9] - dist) < 1e-12
        lref = RRf.T @ (x_ref - np.array([float(v) for v in xr]))
        np.testing.assert_allclose(lref, [exact[k][0], exact[k][1], up * float(hr[2])], atol=1e-12)
        # n from B toward A
        np.testing.assert_allclose(c_[6:9], nref_w if ref_is_b else -nref_w, atol=1e-12)


def test_clip_cases_actually_clip():
    """The fixtures exercise clipping: each case's exact intersection has a
    vertex that is not a corner of the incident face, and one case has more
    than four."""
    counts = []
    for cs in CLIP_CASES:
        Rrel = fmat(frac_rot(*cs["turn"], 2), frac_rot(*cs["tilt"], 0))
        hi = cs["hi"]
        quad = []
        for s1, s2 in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
            p = fvec(Rrel, [s1 * hi[0], s2 * hi[1], -hi[2]])
            quad.append((cs["c"][0] + p[0], cs["c"][1] + p[1]))
        poly = polygon_intersection(quad, cs["hr"][0], cs["hr"][1])
        assert poly - set(quad)
        counts.append(len(poly))
    assert max(counts) > 4


# ------------------------------------------------------- manifold reduction
def shoelace(p, q, r):
    return 0.5 * abs((q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0]))


def reduce_brute(P2, d):
    """The reduction rules, evaluated in the points' own 2D plane
    coordinates: p1 = deepest, p2 = farthest from p1, p3 = largest triangle
    (p1, p2, p), p4 = largest summed area of (p1, p2, p), (p2, p3, p),
    (p3, p1, p); the first index wins ties."""
    n = len(P2)
    i1 = int(np.argmin(d))
    rest = [k for k in range(n) if k != i1]
    i2 = max(rest, key=lambda k: (np.sum((P2[k] - P2[i1]) ** 2), -k))
    rest = [k for k in rest if k != i2]
    i3 = max(rest, key=lambda k: (shoelace(P2[i1], P2[i2], P2[k]), -k))
    rest = [k for k in rest if k != i3]
    i4 = max(rest, key=lambda k: (shoelace(P2[i1], P2[i2], P2[k]) + shoelace(P2[i2], P2[i3], P2[k]) +
                                  shoelace(P2[i3], P2[i1], P2[k]), -k))
    return [i1, i2, i3, i4]


REDUCE_SETS = [
    # (2D points, depths): every selection wins by a clear gap (no near
    # ties), and each set also separates every wrong variant of the rules
    # (see test_reduction_fixtures_discriminate)
    ([(0.09, 0.41), (-0.9, 0.36), (-0.26, 0.18), (0.34, 0.34), (0.05, 0.11), (-0.6, -0.01)],
     [-0.0032, -0.0011, -0.0008, 0.0006, -0.0016, -0.0039]),
    ([(0.16, 0.3), (0.85, 0.17), (-0.12, -0.4), (0.45, 0.28), (-0.86, -0.4), (-0.67, -0.01), (-0.24, -0.68)],
     [-0.0008, 0.0, -0.002, 0.001, -0.0034, -0.0037, 0.0002]),
    ([(0.65, 0.47), (-0.64, 0.47), (-0.47, 0.02), (-0.96, 0.83), (-0.31, 0.39), (-0.76, -0.61), (0.52, 0.4)],
     [-0.0004, -0.0016, -0.0002, 0.0014, 0.0009, 0.0007, -0.0013]),
]


@pytest.mark.parametrize("k", range(len(REDUCE_SETS)))
@pytest.mark.parametrize("seed", [0, 5, 6])
def test_manifold_reduction_selects_the_stated_points(k, seed):
    pts2, d = REDUCE_SETS[k]
    P2 = np.array(pts2, np.float64) * 0.05
    g = np.random.default_rng(seed)
    R = np.eye(3) if seed == 0 else rotm(scenegen.shoemake_quat(g))
    o = g.uniform(-0.3, 0.3, 3)
    cand = np.zeros((len(P2), 10))
    for i, (u, v) in enumerate(P2):
        x = o + R @ np.array([u, v, 0.0])
        cand[i, 3:6] = x
        cand[i, 0:3] = x + R @ np.array([0, 0, d[i]])
        cand[i, 6:9] = R[:, 2]
        cand[i, 9] = d[i]
    assert list(oracle.reduce4(cand)) == reduce_brute(P2, np.array(d))


def test_reduction_fixtures_discriminate():
    """Each wrong variant of a rule picks a different set on every fixture:
    p2 nearest instead of farthest, p3 by distance from p1 instead of area,
    p4 by the single triangle (p1, p2, p) or by distance from p3."""
    def variant(P2, d, which):
        n = len(P2)
        i1 = int(np.argmin(d))
        rest = [k for k in range(n) if k != i1]
        key2 = (lambda k: -np.sum((P2[k] - P2[i1]) ** 2)) if which == "p2" else (lambda k: np.sum((P2[k] - P2[i1]) ** 2))
        i2 = max(rest, key=key2)
        rest = [k for k in rest if k != i2]
        key3 = (lambda k: np.sum((P2[k] - P2[i1]) ** 2)) if which == "p3" else (lambda k: shoelace(P2[i1], P2[i2], P2[k]))
        i3 = max(rest, key=key3)
        rest = [k for k in rest if k != i3]
        if which == "p4a":
            key4 = lambda k: shoelace(P2[i1], P2[i2], P2[k])
        elif which == "p4b":
            key4 = lambda k: np.sum((P2[k] - P2[i3]) ** 2)
        else:
            key4 = lambda k: (shoelace(P2[i1], P2[i2], P2[k]) + shoelace(P2[i2], P2[i3], P2[k]) +
                              shoelace(P2[i3], P2[i1], P2[k]))
        return [i1, i2, i3, max(rest, key=key4)]
    for which in ("p2", "p3", "p4a", "p4b"):
        assert all(variant(np.array(p) * 0.05, np.array(d), which) != reduce_brute(np.array(p) * 0.05, np.array(d))
                   for p, d in REDUCE_SETS), which


# ------------------------------------------------------------- tangent basis
@pytest.mark.parametrize("n,axis", [
    ((0, 0, 1), 0),                                  # all of x, y tiny: the first, x
    ((0.05, 0.0, 1), 0),                             # |n_x| within 0.1 of min |n_y| = 0: still x
    ((0.0, 0.05, 1), 0),
    ((0.2, 0.0, 1), 1),                              # x beyond 0.1 of the min: y
    ((-math.sin(0.45), 0.0, math.cos(0.45)), 1),     # an incline normal in the xz-plane: t1 along y x n
    ((0.3, 0.5, 0.2), 2),                            # the smallest component z
    ((0.7, 0.05, 0.14), 1),                          # z within 0.1 of y, but y comes first
    ((0.0, 1.0, 0.0), 0),
])
def test_tangent_basis_rule(n, axis):
    """t1 = normalize(n x e_k), k = the first axis whose |n_k| is within 0.1
    of the smallest |n_i|; t2 = n x t1; an orthonormal right-handed frame."""
    n = np.asarray(n, np.float64)
    n = n / np.linalg.norm(n)
    t1, t2 = oracle.tangents(n)
    e = np.eye(3)[axis]
    expect = np.cross(n, e)
    expect /= np.linalg.norm(expect)
    np.testing.assert_allclose(t1, expect, atol=1e-15)
    np.testing.assert_allclose(t2, np.cross(n, expect), atol=1e-15)
    np.testing.assert_allclose([t1 @ n, t2 @ n, t1 @ t2, t1 @ t1, t2 @ t2], [0, 0, 0, 1, 1], atol=1e-15)
    assert np.linalg.det(np.stack([t1, t2, n])) > 0


# ----------------------------------------------------- hull principal frame
# a degree-2 exact cubature on a tetrahedron (4 points, barycentric
# (a, b, b, b) permutations, equal weights): integrates x_i x_j exactly
_TET_A = (5 + 3 * math.sqrt(5)) / 20
_TET_B = (5 - math.sqrt(5)) / 20


def solid_moments_cubature(v, t):
    """Volume, first and second moments of a closed outward mesh by exact
    degree-2 cubature over the tetrahedra (interior point, triangle) --
    signed volumes, so any interior point works."""
    o = v.mean(0)
    vol, m1, m2 = 0.0, np.zeros(3), np.zeros((3, 3))
    for tri in t:
        P = [o, v[tri[0]], v[tri[1]], v[tri[2]]]
        V6 = np.dot(P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))
        w = V6 / 6.0
        vol += w
        for i in range(4):
            bary = np.full(4, _TET_B)
            bary[i] = _TET_A
            x = sum(bary[k] * P[k] for k in range(4))
            m1 += w / 4 * x
            m2 += w / 4 * np.outer(x, x)
    return vol, m1, m2


@pytest.mark.parametrize("seed", range(6))
def test_hull_assets_are_in_their_principal_frame(seed):
    """scenegen's hull assets (shared input of both sides) are delivered in
    the solid's principal frame: centroid at the origin, off-diagonal
    second moments zero -- to float32 rounding of the stored vertices."""
    from scenegen import hulls
    g = np.random.default_rng(seed)
    pts = hulls.random_points(g, int(g.integers(6, 13)), g.uniform(0.01, 0.05, 3))
    v32, t = hulls.hull_asset(pts)
    v = v32.astype(np.float64)
    vol, m1, m2 = solid_moments_cubature(v, t)
    assert vol > 0
    size = np.abs(v).max()
    assert np.linalg.norm(m1 / vol) < 1e-6 * size
    C = m2 / vol
    off = max(abs(C[0, 1]), abs(C[0, 2]), abs(C[1, 2]))
    assert off < 1e-6 * np.trace(C), (off, np.diag(C))
    # and the frame is right-handed: the hull's own orientation is kept
    # (outward triangles stay outward, positive volume)
    assert vol > 0


def test_cubature_is_exact_on_a_box():
    """The cubature itself: a box's second moments (h^2/3 per axis)."""
    from scenegen import hulls
    v, t = hulls.box_asset(0.03, 0.02, 0.01)
    h = np.abs(v.astype(np.float64)).max(0)               # the stored (float32) half-extents
    vol, m1, m2 = solid_moments_cubature(v.astype(np.float64), t)
    assert abs(vol - 8 * h.prod()) < 1e-18
    np.testing.assert_allclose(m1, 0.0, atol=1e-20)
    np.testing.assert_allclose(m2 / vol, np.diag(h ** 2 / 3), atol=1e-16)
