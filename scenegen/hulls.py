"""Convex hull assets: stand-ins for the convex pieces of decomposed meshes.

An asset is a set of vertices and outward, counter-clockwise triangles.  Like
the output of a mesh-preparation tool, every asset is delivered in its own
principal frame: the centroid of the solid at the origin and its principal
axes of inertia along x, y, z, so that a body's frame is its principal frame.
(Both the oracle and the CUDA path compute the mass properties they use from
the asset themselves.)

A scene's hull library concatenates its assets:
    verts    float32 [NV][3]     vert_off int32 [H + 1]
    tris     int32   [NT][3]     tri_off  int32 [H + 1]   (indices local to the hull)
A hull body has type HULL and p = (hull index, 0, 0).
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

MAX_HULL_VERTS = 16


def _solid_moments(v: np.ndarray, t: np.ndarray):
    """Volume, centroid and second-moment matrix of a closed triangle mesh
    (divergence theorem over tetrahedra from the origin)."""
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    vol6 = np.einsum("ij,ij->i", a, np.cross(b, c))
    vol = vol6.sum() / 6.0
    cen = ((a + b + c) * vol6[:, None]).sum(0) / 24.0 / vol
    s = a + b + c
    w = vol6 / 120.0
    C = (np.einsum("k,ki,kj->ij", w, a, a) + np.einsum("k,ki,kj->ij", w, b, b) +
         np.einsum("k,ki,kj->ij", w, c, c) + np.einsum("k,ki,kj->ij", w, s, s))
    return vol, cen, C


def hull_asset(points: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Convex hull of the points (qhull), outward triangles, re-expressed in
    the solid's principal frame.  Returns (verts float32, tris int32)."""
    from scipy.spatial import ConvexHull
    pts = np.asarray(points, np.float64)
    h = ConvexHull(pts)
    used = np.unique(h.simplices)
    remap = -np.ones(len(pts), np.int64)
    remap[used] = np.arange(len(used))
    v = pts[used]
    t = remap[h.simplices]
    # outward orientation: the normal points away from the interior
    inner = v.mean(0)
    for k in range(len(t)):
        a, b, c = v[t[k]]
        if np.dot(np.cross(b - a, c - a), a - inner) < 0:
            t[k] = t[k][[0, 2, 1]]
    vol, cen, _ = _solid_moments(v, t)
    v = v - cen
    _, _, C = _solid_moments(v, t)
    _, axes = np.linalg.eigh(C)
    if np.linalg.det(axes) < 0:
        axes[:, 2] = -axes[:, 2]
    v = v @ axes                      # coordinates along the principal axes
    return v.astype(np.float32), t.astype(np.int32)


def box_asset(hx: float, hy: float, hz: float) -> Tuple[np.ndarray, np.ndarray]:
    """A box as a hull: its 8 corners, 12 outward triangles (already in its
    principal frame)."""
    v = np.array([[sx * hx, sy * hy, sz * hz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], np.float32)
    faces = [(1, 3, 7, 5), (2, 0, 4, 6), (3, 2, 6, 7), (0, 1, 5, 4), (4, 5, 7, 6), (2, 3, 1, 0)]
    t = []
    for a, b, c, d in faces:
        t += [(a, b, c), (a, c, d)]
    return v, np.array(t, np.int32)


def volume(verts: np.ndarray, tris: np.ndarray) -> float:
    return float(_solid_moments(np.asarray(verts, np.float64), np.asarray(tris))[0])


def library(assets: List[Tuple[np.ndarray, np.ndarray]]) -> Dict:
    vo, to = [0], [0]
    for v, t in assets:
        assert len(v) <= MAX_HULL_VERTS, len(v)
        vo.append(vo[-1] + len(v)); to.append(to[-1] + len(t))
    return dict(verts=np.concatenate([a[0] for a in assets]).astype(np.float32) if assets else np.zeros((0, 3), np.float32),
                vert_off=np.asarray(vo, np.int32),
                tris=np.concatenate([a[1] for a in assets]).astype(np.int32) if assets else np.zeros((0, 3), np.int32),
                tri_off=np.asarray(to, np.int32))


def random_points(g: np.random.Generator, n: int, semi: np.ndarray) -> np.ndarray:
    """n points inside an ellipsoid with the given semi-axes (rejection)."""
    out = []
    while len(out) < n:
        p = g.uniform(-1, 1, 3)
        if p @ p <= 1.0:
            out.append(p * semi)
    return np.array(out)


def bound_radius(verts: np.ndarray) -> float:
    return float(np.sqrt((np.asarray(verts, np.float64) ** 2).sum(1).max()))
