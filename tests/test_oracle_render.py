"""Pins of the oracle's camera renderer (the paper's batched RGB / depth /
segmentation rendering, restated as a triangle rasteriser).

Each expected value is computed here from the geometry alone, independently
of the rasteriser: the pixel centres inside a projected box face or sphere
outline, the view depth of a ray hitting a plane, which of two boxes is in
front, and the Lambert factor of a face turned to the light.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import BOX, PLANE, SPHERE, body, pack
from scenegen import validation

W = H = 64
FOV = math.radians(60.0)
F = 0.5 * H / math.tan(0.5 * FOV)


def _scene(bodies):
    return pack("render_probe", [bodies], [[]], scenegen.default_params(), 0, 0)


def _render(bodies, eye, target, colors=None, near=0.01, size=None):
    sc = _scene(bodies)
    o = oracle.Oracle(sc)
    w, h = size or (W, H)
    cam = dict(eye=eye, target=target, fov_y=FOV, near=near, width=w, height=h)
    col = np.full((len(bodies), 3), 0.5) if colors is None else np.asarray(colors, np.float64)
    rgb, depth, seg, ties = o.render(cam, col, threads=1)
    return rgb[0], depth[0], seg[0], ties[0]


def _basis(eye, target):
    eye, target = np.asarray(eye, float), np.asarray(target, float)
    fw = (target - eye) / np.linalg.norm(target - eye)
    rt = np.cross(fw, [0, 0, 1.0]); rt /= np.linalg.norm(rt)
    up = np.cross(rt, fw)
    return eye, rt, up, fw


def _project(p, eye, target):
    e, rt, up, fw = _basis(eye, target)
    d = np.asarray(p, float) - e
    x, y, z = d @ rt, d @ up, d @ fw
    return 0.5 * W + F * x / z, 0.5 * H - F * y / z, z


def _centres(w=W, h=H):
    j, i = np.mgrid[0:h, 0:w]
    return i + 0.5, j + 0.5


# a wide image as well: the focal length follows the height, columns the width
@pytest.mark.parametrize("size", [(64, 64), (96, 40)])
def test_face_on_box_covers_its_projected_square_at_constant_depth(size):
    w, hh = size
    f = 0.5 * hh / math.tan(0.5 * FOV)
    h = 0.125                                # binary-exact sizes: float32 inputs are exact
    rgb, depth, seg, ties = _render([body(BOX, (h, h, h), 0.0, (0, 0, 0))], (0, -1.0, 0), (0, 0, 0), size=size)
    half = f * h / (1.0 - h)                 # the -y face at view depth 0.875
    x, y = _centres(w, hh)
    inside = (np.abs(x - 0.5 * w) <= half) & (np.abs(y - 0.5 * hh) <= half)
    ok = ties == 0
    np.testing.assert_array_equal(seg[ok] == 1, inside[ok])
    assert inside.sum() >= 100 and (ok & inside).sum() > 0.8 * inside.sum()
    np.testing.assert_allclose(depth[inside & ok], 1.0 - h, rtol=1e-12)
    assert (depth[~inside & ok] == 0).all()


@pytest.mark.parametrize("size", [(64, 64), (96, 40)])
def test_ground_depth_is_the_ray_plane_distance(size):
    """The camera stands inside the plane's 4 m square, so its triangles cross
    the near plane and are clipped; every pixel looking down hits z = 0 at the
    analytic view depth."""
    w, hh = size
    f = 0.5 * hh / math.tan(0.5 * FOV)
    eye, target = (0.3, -0.2, 0.5), (0.6, 0.4, 0.0)
    rgb, depth, seg, ties = _render([body(PLANE, (0, 0, 0), 0.0, (0, 0, 0))], eye, target, size=size)
    e, rt, up, fw = _basis(eye, target)
    x, y = _centres(w, hh)
    dirs = ((x - 0.5 * w) / f)[..., None] * rt + (-(y - 0.5 * hh) / f)[..., None] * up + fw
    t = -e[2] / dirs[..., 2]                 # view depth of the hit (dirs has unit view z)
    hit = e + t[..., None] * dirs
    on = (dirs[..., 2] < 0) & (np.abs(hit[..., 0]) < 2) & (np.abs(hit[..., 1]) < 2) & (ties == 0)
    assert on.sum() > 0.5 * w * hh
    assert (seg[on] == 1).all()
    np.testing.assert_allclose(depth[on], t[on], rtol=1e-9)


def test_sphere_outline_is_the_projected_equator_polygon():
    """A sphere seen along its pole axis from 1 m: the silhouette of the UV
    mesh is its equator ring, a regular 12-gon of circumradius r."""
    r = 0.25
    q = scenegen.axis_angle_quat((0, 1, 0), math.pi / 2)      # body z -> world x
    rgb, depth, seg, ties = _render([body(SPHERE, (r, 0, 0), 0.0, (0, 0, 0), quat=q)], (-1.0, 0, 0), (0, 0, 0))
    R = np.array(validation._rot(q))
    ring = [R @ np.array([r * math.cos(2 * math.pi * j / 12), r * math.sin(2 * math.pi * j / 12), 0.0])
            for j in range(12)]
    poly = np.array([_project(p, (-1.0, 0, 0), (0, 0, 0))[:2] for p in ring])
    x, y = _centres()
    inside = np.ones((H, W), bool)
    c = poly.mean(0)
    for k in range(12):
        a, b = poly[k], poly[(k + 1) % 12]
        side = (b[0] - a[0]) * (y - a[1]) - (b[1] - a[1]) * (x - a[0])
        ref = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        inside &= side * np.sign(ref) >= 0
    ok = ties == 0
    np.testing.assert_array_equal(seg[ok] == 1, inside[ok])
    # the pole faces the camera: depth at the centre pixel pair is ~ 1 - r
    assert abs(depth[H // 2, W // 2] - (1.0 - r)) < 0.02


def test_nearer_box_occludes_the_farther():
    near = body(BOX, (0.0625, 0.0625, 0.0625), 0.0, (0, -0.25, 0))
    far = body(BOX, (0.125, 0.125, 0.125), 0.0, (0.03125, 0.25, 0.0))
    rgb, depth, seg, ties = _render([far, near], (0, -1.0, 0), (0, 0, 0))
    ok = ties == 0
    # the near box (index 1) covers the image centre; the far one (index 0) its rim
    assert seg[H // 2, W // 2] == 2
    half_near = F * 0.0625 / 0.6875
    x, y = _centres()
    front = (np.abs(x - 0.5 * W) <= half_near) & (np.abs(y - 0.5 * H) <= half_near)
    np.testing.assert_array_equal(seg[front & ok], 2)
    np.testing.assert_allclose(depth[front & ok], 0.6875, rtol=1e-12)
    assert ((seg == 1) & ~front).sum() > 50
    np.testing.assert_allclose(depth[(seg == 1) & ok], 1.125, rtol=1e-12)


def test_face_turned_to_the_light_is_fully_lit():
    L = np.array([0.3, 0.2, 1.0]); L /= np.linalg.norm(L)
    # quaternion turning body +z onto L
    ax = np.cross([0, 0, 1.0], L); ang = math.acos(L[2])
    q = scenegen.axis_angle_quat(ax / np.linalg.norm(ax), ang)
    base = (0.8, 0.4, 0.2)
    rgb, depth, seg, ties = _render([body(BOX, (0.1, 0.1, 0.1), 0.0, (0, 0, 0), quat=q)], tuple(1.0 * L), (0, 0, 0),
                                    colors=[base])
    ok = (ties == 0) & (seg == 1)
    assert ok.sum() > 100
    expect = [int(math.floor(255 * c + 0.5)) for c in base]
    # float32 quaternion input: the face normal is L to ~1e-7; the byte is exact
    assert (rgb[ok] == expect).all(axis=1).mean() > 0.99


def test_back_facing_plane_is_not_drawn():
    rgb, depth, seg, ties = _render([body(PLANE, (0, 0, 0), 0.0, (0, 0, 0))], (0.2, -0.1, -0.5), (0, 0.3, 0.0))
    assert (seg == 0).all()


def test_degenerate_camera_is_rejected():
    sc = _scene([body(BOX, (0.1, 0.1, 0.1), 0.0, (0, 0, 0))])
    o = oracle.Oracle(sc)
    with pytest.raises(ValueError):
        o.render(dict(eye=(0, 0, 1), target=(0, 0, 0), fov_y=FOV, near=0.01, width=8, height=8), np.ones((1, 3)))
