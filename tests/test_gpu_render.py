"""The CUDA rasteriser against the oracle's renderer, on the same float32
body poses (the scene's, or states the oracle stepped to).

Bars.  Segmentation is compared exactly on pixels the oracle does not flag
(a coverage decision within 1e-3 pixel of an edge, or two depths within
1e-5): float32 screen coordinates are good to ~1e-5 pixel at 128 x 128.
Depth: relative 1e-5 (a float32 perspective division chain of ~10 roundings).
RGB: the shade is a float32 product against the oracle's FP64 one, so a byte
may round the other way: |diff| <= 1.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import BOX, body, pack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00425_b300 import build
    build.build()


def _both(sc, cam, steps=0):
    """Render the scene (after `steps` oracle steps, the state handed to the
    GPU batch rounded to float32) on both sides."""
    from paper_2410_00425_b300 import Batch
    o = oracle.Oracle(sc)
    if steps:
        o.step(steps, threads=8)
    st = o.state().astype(np.float32)
    o.set_state(st.astype(np.float64))
    b = Batch(sc)
    b.set_state(torch.from_numpy(st).cuda())
    col = scenegen.body_colors(sc)
    b.set_camera(cam, col)
    rgba, depth, seg = b.render()
    torch.cuda.synchronize()
    g = (rgba.cpu().numpy(), depth.cpu().numpy().astype(np.float64), seg.cpu().numpy().astype(np.int64))
    r = o.render(cam, col.astype(np.float64))
    b.close()
    return g, r


def _check(g, r, min_cov=0.05):
    (grgba, gdepth, gseg), (rrgb, rdepth, rseg, ties) = g, r
    ok = ties == 0
    assert ok.mean() > 0.98
    bad = ok & (gseg != rseg)
    assert not bad.any(), (np.argwhere(bad)[:5].tolist(), bad.sum())
    cov = ok & (rseg > 0)
    assert cov.mean() > min_cov
    np.testing.assert_allclose(gdepth[cov], rdepth[cov], rtol=1e-5)
    assert (gdepth[ok & (rseg == 0)] == 0).all()
    d = np.abs(grgba[..., :3].astype(int) - rrgb.astype(int))
    assert d[ok].max() <= 1, d[ok].max()
    assert (grgba[..., 3][cov] == 255).all()


@pytest.mark.parametrize("steps", [0, 30])
def test_pick_scene_matches_oracle(steps):
    sc = scenegen.make_scene("pick", n_envs=16)
    cam = scenegen.default_camera("pick")
    g, r = _both(sc, cam, steps)
    _check(g, r)


def test_clutter_scene_matches_oracle():
    sc = scenegen.make_scene("clutter", n_envs=12)
    cam = scenegen.default_camera("clutter", width=96, height=64)
    g, r = _both(sc, cam, steps=20)
    _check(g, r)


def test_hand_scene_matches_oracle():
    sc = scenegen.make_scene("hand", n_envs=8)
    cam = scenegen.default_camera("hand", width=64, height=64)
    g, r = _both(sc, cam, steps=5)
    _check(g, r)


def test_face_on_box_exact_square_wide_image():
    """The oracle pin's geometry on the GPU: 96 x 40 image, box of half-size
    0.125 at 1 m: the covered pixels are exactly the centres inside the
    projected square, at depth 0.875."""
    sc = pack("render_probe", [[body(BOX, (0.125, 0.125, 0.125), 0.0, (0, 0, 0))]], [[]],
              scenegen.default_params(), 0, 0)
    from paper_2410_00425_b300 import Batch
    b = Batch(sc)
    cam = dict(eye=(0, -1.0, 0), target=(0, 0, 0), fov_y=math.radians(60), near=0.01, width=96, height=40)
    b.set_camera(cam, np.array([[1.0, 0.5, 0.25]], np.float32))
    rgba, depth, seg = b.render()
    seg = seg.cpu().numpy()[0]
    depth = depth.cpu().numpy()[0]
    F = 20.0 / math.tan(math.radians(30))
    half = F * 0.125 / 0.875
    j, i = np.mgrid[0:40, 0:96]
    x, y = i + 0.5, j + 0.5
    inside = (np.abs(x - 48) <= half) & (np.abs(y - 20) <= half)
    far = (np.abs(np.abs(x - 48) - half) > 1e-3) & (np.abs(np.abs(y - 20) - half) > 1e-3)
    np.testing.assert_array_equal((seg == 1)[far], inside[far])
    np.testing.assert_allclose(depth[inside & far], 0.875, rtol=1e-6)


def test_render_is_deterministic_and_outputs_optional():
    sc = scenegen.make_scene("pick", n_envs=8)
    from paper_2410_00425_b300 import Batch, _ffi
    b = Batch(sc)
    b.set_camera(scenegen.default_camera("pick"), scenegen.body_colors(sc))
    s = torch.cuda.Stream()
    a = b.render(stream=s)
    c = b.render()
    torch.cuda.synchronize()
    for u, v in zip(a, c):
        assert torch.equal(u, v)
    seg = torch.zeros((8, 128, 128), dtype=torch.int16, device="cuda")
    _ffi.ms_render(b.h, None, None, seg, None)
    torch.cuda.synchronize()
    assert torch.equal(seg, a[2])


def test_camera_errors():
    from paper_2410_00425_b300 import Batch, MSError, _ffi
    sc = scenegen.make_scene("small", n_envs=2)
    b = Batch(sc)
    with pytest.raises(MSError):
        _ffi.ms_render(b.h, None, None, None, None)               # no camera yet
    col = scenegen.body_colors(sc)
    cam = scenegen.default_camera("small")
    with pytest.raises(MSError):
        b.set_camera(dict(cam, eye=(0, 0, 1), target=(0, 0, 0)), col)   # vertical view
    with pytest.raises(MSError):
        b.set_camera(dict(cam, width=256, height=128), col)             # z-buffer too large
    with pytest.raises(MSError):
        b.set_camera(cam, col * 2.0)                                      # colours outside [0, 1]
    b.set_camera(cam, col)
    rgba, depth, seg = b.render()
    torch.cuda.synchronize()
    assert (seg.cpu().numpy() > 0).any()
