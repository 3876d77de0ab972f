"""Oracle pins of the cutting and near-clip planes of §5.5.

An affine box with a constant scalar: every pixel's opacity is
1 - exp(-sigma A L) with L the length of the ray's slab through the box
(closed form) clipped to the kept half-space of the cutting plane, or to
t >= t_near for the near plane, including the eye inside the box (an exit
without an entry: the segment starts on the near plane).  A plane that keeps
the whole volume leaves the image unchanged; one that cuts all of it away
leaves it empty; on the twisted bar a plane through the middle keeps the
pixels whose rays never cross it.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes
from tests.test_oracle_bspline import _affine_block
from tests.test_oracle_intersect import _slab

COL = np.array([0.25, 0.5, 0.625, 0.75])       # exact in float32
SIGMA = 1.5


def _box_scene(rng, eye_offset, fovy=40.0, **params):
    blk, A, b = _affine_block(rng)
    blk.scalar_cp = np.full(blk.geom_cp.shape[:3], 0.3)
    tf = scenes.TransferFunction(np.array([0, 1], np.float32), np.array([COL, COL], np.float32), SIGMA,
                                 lo=0.0, hi=1.0)
    centre = b + A @ np.full(3, 0.5)
    diag = 2 * np.linalg.norm(A @ np.ones(3))
    cam = scenes.Camera(False, tuple(centre + np.asarray(eye_offset)), tuple(centre), (0, 0, 1), fovy_deg=fovy)
    sc = scenes.Scene("box", [blk], scenes.SCALAR_CP, tf, cam, 24, 24,
                      scenes.RenderParams(ds=diag / 50, early_alpha=2.0, **params))
    return sc, A, b


def _check(sc, A, b, t_lo_fn):
    img = oracle.render(sc)
    hit = 0
    for y in range(sc.height):
        for x in range(sc.width):
            o, d = oracle.ray(sc.camera, sc.width, sc.height, x, y)
            s = _slab(A, b, o, d)
            L = 0.0
            if s is not None:
                t0, t1 = t_lo_fn(o, d, max(s[0], 0.0), s[1])
                L = max(0.0, t1 - t0)
            hit += L > 0
            assert img[y, x, 3] == pytest.approx(1 - np.exp(-SIGMA * COL[3] * L), abs=1e-11), (x, y)
    return hit


def test_cutting_plane_closed_form():
    rng = np.random.default_rng(60)
    sc, A, b = _box_scene(rng, (1.6, 0.6, 1.1), fovy=55.0)
    full = _check(sc, A, b, lambda o, d, t0, t1: (t0, t1))
    centre = b + A @ np.full(3, 0.5)
    n = np.array([0.3, -0.8, 0.52])
    n /= np.linalg.norm(n)
    w = -n @ (centre + 0.1 * A @ np.ones(3))
    sc.params.cut_planes = ((n[0], n[1], n[2], w),)

    def clip(o, d, t0, t1):
        fo, fd = n @ o + w, n @ d
        tc = -fo / fd
        return (t0, min(t1, tc)) if fd > 0 else (max(t0, tc), t1)

    assert 0.2 * full < _check(sc, A, b, clip) < full


def test_two_cutting_planes_closed_form():
    rng = np.random.default_rng(61)
    sc, A, b = _box_scene(rng, (1.4, -1.1, 0.9), fovy=55.0)
    full = _check(sc, A, b, lambda o, d, t0, t1: (t0, t1))
    centre = b + A @ np.full(3, 0.5)
    planes = []
    for n in (np.array([1.0, 0.2, 0.0]), np.array([-0.1, 0.3, -1.0])):
        n = n / np.linalg.norm(n)
        planes.append((n, -n @ centre))
    sc.params.cut_planes = tuple((n[0], n[1], n[2], w) for n, w in planes)

    def clip(o, d, t0, t1):
        for n, w in planes:
            fo, fd = n @ o + w, n @ d
            tc = -fo / fd
            t0, t1 = (t0, min(t1, tc)) if fd > 0 else (max(t0, tc), t1)
        return t0, t1

    assert 0.1 * full < _check(sc, A, b, clip) < full


def test_near_plane_with_the_eye_inside_the_box():
    """Rays start inside the box: only exits are found; the near plane
    supplies the entries."""
    rng = np.random.default_rng(62)
    sc, A, b = _box_scene(rng, (0.05, 0.02, -0.03), fovy=60.0, near_clip=0.15)
    f = np.asarray(sc.camera.target) - np.asarray(sc.camera.eye)
    f /= np.linalg.norm(f)

    def clip(o, d, t0, t1):
        return max(t0, 0.15 / (d @ f)), t1

    assert _check(sc, A, b, clip) == sc.width * sc.height


def test_near_plane_cutting_the_front_of_the_box():
    rng = np.random.default_rng(63)
    sc, A, b = _box_scene(rng, (1.6, 0.6, 1.1), fovy=55.0)
    dist = np.linalg.norm(np.asarray(sc.camera.eye) - np.asarray(sc.camera.target))
    sc.params.near_clip = dist - 0.2
    f = np.asarray(sc.camera.target) - np.asarray(sc.camera.eye)
    f /= np.linalg.norm(f)

    def clip(o, d, t0, t1):
        return max(t0, sc.params.near_clip / (d @ f)), t1

    assert _check(sc, A, b, clip) > 100


def test_planes_that_keep_all_or_nothing_on_the_twisted_bar():
    sc = scenes.config(1, width=64, height=36)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    ref = oracle.render(sc, vol)
    assert ref[..., 3].max() > 0.2
    keep = dataclasses.replace(sc, params=dataclasses.replace(sc.params, cut_planes=((0.0, 0.0, 1.0, -100.0),)))
    np.testing.assert_array_equal(oracle.render(keep, vol), ref)
    cut = dataclasses.replace(sc, params=dataclasses.replace(sc.params, cut_planes=((0.0, 0.0, 1.0, 100.0),)))
    assert np.abs(oracle.render(cut, vol)).max() == 0.0
    # a plane across the bar's axis: pixels whose segments stay on the kept side are unchanged
    half = dataclasses.replace(sc, params=dataclasses.replace(sc.params, cut_planes=((0.0, 0.0, 1.0, -4.0),)))
    img = oracle.render(half, vol)
    changed = np.abs(img - ref).max(-1) > 0
    assert 0.05 < changed[ref[..., 3] > 0].mean() < 0.95
    for y, x in np.argwhere(changed)[:20]:
        pairs, _ = vol.pixel_pairs(sc.camera, 64, 36, x, y)
        o, d = oracle.ray(sc.camera, 64, 36, x, y)
        zs = [(o + t * d)[2] for pr in pairs for t in (pr.t_in, pr.t_out)]
        assert max(zs) > 4.0                    # only segments reaching z > 4 change
