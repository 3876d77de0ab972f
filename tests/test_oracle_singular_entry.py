"""Oracle pins of the singular-entry rule of §5.4 (Eq. 22) on a block whose
Jacobian vanishes on a boundary face.

The untwisted, unjittered degenerate cube has the closed form
phi(u, v, w) = (u, v, 1 - (1 - w)^3) (its three upper control-point layers
coincide), so det J = 3 (1 - w)^2 is zero on the whole top face.  A ray
entering through the top face has a singular Jacobian at its entry point:
the entry moves delta = 1e-4 diag along the ray and its parameter point
solves phi(p) = g_in + delta d, which here is known in closed form.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes


def _flat_cube(scalar=None, direction=(0.0, 0.0, 1.0), width=32, height=32):
    return scenes.degenerate_cube(twist=0.0, jitter=0.0, scalar=scalar, direction=direction, width=width,
                                  height=height)


def test_closed_form_map():
    sc = _flat_cube()
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    p = np.random.default_rng(3).uniform(0, 1, (50, 3))
    phi, J, _ = vol.eval(0, p)
    np.testing.assert_allclose(phi, np.stack([p[:, 0], p[:, 1], 1 - (1 - p[:, 2]) ** 3], 1), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(J), 3 * (1 - p[:, 2]) ** 2, atol=1e-13)


def test_top_face_entry_moves_by_delta():
    sc = _flat_cube()
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    diag = vol.diag
    assert abs(diag - math.sqrt(3)) < 1e-12
    delta = 1e-4 * diag
    checked = 0
    for x, y in ((16, 16), (12, 19), (20, 13)):
        o, d = oracle.ray(sc.camera, sc.width, sc.height, x, y)
        assert abs(d[2] + 1) < 1e-12                                     # straight down
        if not (0 < o[0] < 1 and 0 < o[1] < 1):
            continue
        pairs, um = vol.pixel_pairs(sc.camera, sc.width, sc.height, x, y)
        assert um == 0 and len(pairs) == 1
        pr = pairs[0]
        t_top = o[2] - 1.0                                              # the ray meets z = 1 at t_top
        assert abs(pr.t_in - (t_top + delta)) < 1e-12
        np.testing.assert_allclose(pr.p_in, [o[0], o[1], 1 - delta ** (1 / 3)], atol=1e-10)
        np.testing.assert_allclose(pr.p_out, [o[0], o[1], 0.0], atol=1e-12)
        assert abs(pr.t_out - o[2]) < 1e-12
        checked += 1
    assert checked == 3


def test_constant_density_drops_exactly_delta():
    """Constant scalar: alpha = 1 - exp(-sigma A (L - delta)) with L = 1, the
    closed form of the emission-absorption integral over the shortened pair."""
    sc = _flat_cube(scalar=0.5)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    img = oracle.render(sc, vol, n_threads=1)
    A0, C0 = float(sc.tf.rgba[0, 3]), sc.tf.rgba[0, :3].astype(float)
    L = 1.0 - 1e-4 * vol.diag
    expect = 1 - math.exp(-sc.tf.sigma * A0 * L)
    x, y = 16, 16
    assert abs(img[y, x, 3] - expect) < 1e-12
    np.testing.assert_allclose(img[y, x, :3], C0 * expect, atol=1e-12)


def test_regular_entries_are_untouched():
    """Rays entering through the side faces of the block (det J > 0 there)
    keep the plain pairs of Alg. 2; only top-face entries move."""
    sc = _flat_cube(direction=(1.0, 0.2, -0.3))
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    img, st = oracle.render(sc, vol, stats=True)
    assert st[..., 0].sum() > 100
    assert st[..., 5].sum() == 0


def test_twisted_degenerate_cube_renders():
    """Twisted and jittered: every top-face entry is moved, no Newton
    solve fails, no pixel is NaN."""
    sc = scenes.degenerate_cube(width=48, height=48)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    img, st = oracle.render(sc, vol, stats=True)
    assert np.isfinite(img).all()
    assert st[..., 5].sum() > 200 and st[..., 2].sum() == 0
    assert img[..., 3].max() > 0.3


def test_walk_into_the_block_finds_the_boundary():
    """§5.4's walk along the ray: from a point above the flat degenerate cube
    (outside the block) toward a point inside, the first point inside is where
    the ray crosses the top face z = 1 (closed form), with its parameter
    point on the face w = 1."""
    sc = _flat_cube()
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    o = np.array([0.3, 0.6, 3.0])
    d = np.array([0.2, -0.1, -1.0])
    d /= np.linalg.norm(d)
    t_top = (3.0 - 1.0) / -d[2]
    t0, t1 = t_top - 0.3, t_top + 0.5
    got = vol.walk_into_block(0, o, d, t0, t1, [0.5, 0.5, 1.0], [0.5, 0.5, 0.5])
    assert got is not None
    t, p = got
    assert abs(t - t_top) < 1e-12
    g = o + t * d
    np.testing.assert_allclose(p[:2], g[:2], atol=1e-9)
    assert abs(p[2] - 1.0) < 1e-4                   # w = 1 - (1 - z)^(1/3) is steep at the face
    assert vol.walk_into_block(0, o, d, t0, t_top - 0.1, [0.5, 0.5, 1.0], [0.5, 0.5, 0.9]) is None
