"""Oracle pins of the von Mises scalar of §6.2 (Eq. 24).

The strain tensor is the symmetric part of the Jacobian of u o phi^-1 (the
displacement as a function of the world point); rho is its von Mises value.
Pins that do not restate the oracle's arithmetic:

* homogeneous strain on a curved map: a displacement whose control points
  are M times the geometry's (plus a constant) is u = M phi + t exactly, so
  u o phi^-1 (g) = M g + t whatever the map; the strain is sym(M) at every
  point and rho takes the textbook values of uniaxial strain (|e|),
  equibiaxial strain (|e|), pure shear (sqrt(3)/2 |gamma|), hydrostatic
  strain and an infinitesimal rotation (both 0);
* a rigid rotation Q of geometry and displacement together leaves rho
  unchanged (the strain turns to Q sigma Q^T);
* the Jacobian of u o phi^-1 by central differences in world space, through
  the oracle's Newton inverse of phi, reproduces rho on a nonlinear field.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes


def _with_disp(sc, disp_of_block):
    blocks = [dataclasses.replace(b, disp_cp=disp_of_block(b)) for b in sc.blocks]
    return dataclasses.replace(sc, blocks=blocks, scalar_mode=scenes.SCALAR_VONMISES)


def _homogeneous(M, t=(0.1, -0.2, 0.3)):
    M = np.asarray(M, float)
    return lambda b: b.geom_cp @ M.T + np.asarray(t)


def _points(seed, n=40):
    return np.random.default_rng(seed).uniform(0.02, 0.98, (n, 3))


CASES = [
    # (name, M, textbook von Mises value)
    ("uniaxial", np.diag([2e-3, 0.0, 0.0]), 2e-3),
    ("uniaxial_compression", np.diag([0.0, 0.0, -5e-3]), 5e-3),
    ("equibiaxial", np.diag([1e-3, 1e-3, 0.0]), 1e-3),
    ("pure_shear", np.array([[0.0, 4e-3, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), math.sqrt(3) / 2 * 4e-3),
    ("hydrostatic", 3e-3 * np.eye(3), 0.0),
    ("rotation", np.array([[0.0, -2e-3, 0.0], [2e-3, 0.0, 0.0], [0.0, 0.0, 0.0]]), 0.0),
]


@pytest.mark.parametrize("name,M,want", CASES, ids=[c[0] for c in CASES])
def test_homogeneous_strain_on_curved_map(name, M, want):
    # the twisted cube and the bent beam: curved maps with jitter
    for sc, blocks in ((scenes.config(0), [0]), (scenes.config(2, width=64, height=36), [0, 5, 15])):
        sv = _with_disp(sc, _homogeneous(M))
        vol = oracle.OracleVolume(sv.blocks, sv.scalar_mode)
        for b in blocks:
            _, _, rho = vol.eval(b, _points(b + 7))
            np.testing.assert_allclose(rho, want, atol=1e-12 + 1e-9 * want)


def test_uniaxial_strain_along_any_axis():
    # a uniaxial strain e along a random unit axis a: M = e a a^T
    rng = np.random.default_rng(11)
    sc = scenes.config(0)
    for _ in range(4):
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        e = rng.uniform(-1e-2, 1e-2)
        sv = _with_disp(sc, _homogeneous(e * np.outer(a, a)))
        vol = oracle.OracleVolume(sv.blocks, sv.scalar_mode)
        _, _, rho = vol.eval(0, _points(3))
        np.testing.assert_allclose(rho, abs(e), rtol=1e-9)


def _smooth_disp(seed):
    rng = np.random.default_rng(seed)
    k = rng.normal(size=(3, 3))
    ph = rng.uniform(0, 2 * math.pi, 3)
    amp = rng.uniform(5e-3, 2e-2, 3)
    return lambda b: np.stack([amp[r] * np.sin(b.geom_cp @ k[r] + ph[r]) for r in range(3)], -1)


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_rigid_rotation_invariance():
    sc = scenes.config(0)
    sv = _with_disp(sc, _smooth_disp(5))
    Q = _rot(8)
    blocks_r = [dataclasses.replace(b, geom_cp=b.geom_cp @ Q.T, disp_cp=b.disp_cp @ Q.T) for b in sv.blocks]
    v0 = oracle.OracleVolume(sv.blocks, sv.scalar_mode)
    v1 = oracle.OracleVolume(blocks_r, sv.scalar_mode)
    p = _points(9)
    _, _, r0 = v0.eval(0, p)
    _, _, r1 = v1.eval(0, p)
    assert r0.max() > 1e-3
    np.testing.assert_allclose(r1, r0, rtol=1e-10, atol=1e-14)


def test_world_space_jacobian_by_differences():
    """sigma = sym(d(u o phi^-1)/dg), the derivative taken by central
    differences in g through the oracle's inverse; rho from sigma with the
    standard von Mises expression written in principal-stress form (the
    eigenvalues of the deviator: sqrt(3/2 |dev sigma|^2))."""
    sc = scenes.config(0)
    sv = _with_disp(sc, _smooth_disp(21))
    vol = oracle.OracleVolume(sv.blocks, sv.scalar_mode)
    # u itself through a second volume whose "geometry" is the displacement
    ublocks = [dataclasses.replace(b, geom_cp=b.disp_cp, disp_cp=None) for b in sv.blocks]
    uvol = oracle.OracleVolume(ublocks, scenes.SCALAR_DETJ)
    h = 1e-5
    for p in _points(4, n=12):
        g, _, rho = vol.eval(0, p)
        A = np.zeros((3, 3))
        for c in range(3):
            vals = []
            for s in (1, -1):
                gg = g[0].copy()
                gg[c] += s * h
                q, _ = vol.invert(0, gg, p)
                u, _, _ = uvol.eval(0, q)
                vals.append(u[0])
            A[:, c] = (vals[0] - vals[1]) / (2 * h)
        sig = 0.5 * (A + A.T)
        dev = sig - np.trace(sig) / 3 * np.eye(3)
        want = math.sqrt(1.5 * np.sum(dev * dev))
        assert abs(rho[0] - want) <= 1e-7 * max(1.0, want) + 1e-9, (p, rho[0], want)


def test_needs_displacement():
    sc = scenes.config(0)
    with pytest.raises(ValueError):
        oracle.OracleVolume(sc.blocks, scenes.SCALAR_VONMISES)
