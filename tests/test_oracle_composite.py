"""Pins of the oracle's compositing (Alg. 1 with supersampling, §3.2.1):
constant density closes to 1 - exp(-sigma L) for any sampling, pairs
compose, early termination, and convergence to the continuous volume
render integral (Eq. 2) computed with scipy quadrature."""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from paper_1404_3363_gb300 import scenes


def _tf(r, rgba, sigma):
    return scenes.TransferFunction(np.asarray(r, np.float32), np.asarray(rgba, np.float32), sigma)


@pytest.mark.parametrize("K", [1, 4, 7])
def test_constant_density_closed_form(K):
    rng = np.random.default_rng(30)
    col = np.array([0.25, 0.5, 0.75, 0.375])
    tf = _tf([0, 1], [col, col], 3.0)
    for _ in range(10):
        s = np.concatenate([[0], np.cumsum(rng.uniform(0.001, 0.2, rng.integers(1, 40)))])
        rho = rng.uniform(0, 1, len(s))
        out = oracle.composite(tf, s, rho, K=K, early=2.0)
        a = 1 - np.exp(-3.0 * col[3] * s[-1])
        assert out[3] == pytest.approx(a, abs=1e-14)
        np.testing.assert_allclose(out[:3], col[:3] * a, atol=1e-14)


def test_two_segments_compose():
    col1 = np.array([1.0, 0.0, 0.0, 0.5])
    col2 = np.array([0.0, 1.0, 0.0, 0.25])
    # rho 0 -> col1, rho 1 -> col2, a step TF (repeated knot)
    tf = _tf([0, 0.5, 0.5, 1], [col1, col1, col2, col2], 2.0)
    s = np.array([0, 0.3, 0.6, 0.6, 1.0, 1.4])
    rho = np.array([0.1, 0.1, 0.1, 0.9, 0.9, 0.9])
    out = oracle.composite(tf, s, rho, K=4, early=2.0)
    a1 = 1 - np.exp(-2 * 0.5 * 0.6)
    a2 = 1 - np.exp(-2 * 0.25 * 0.8)
    assert out[0] == pytest.approx(a1, abs=1e-14)
    assert out[1] == pytest.approx((1 - a1) * a2, abs=1e-14)
    assert out[3] == pytest.approx(a1 + (1 - a1) * a2, abs=1e-14)


def test_early_termination():
    col = np.array([0.5, 0.5, 0.5, 1.0])
    tf = _tf([0, 1], [col, col], 50.0)
    s = np.linspace(0, 2, 41)
    out = oracle.composite(tf, s, np.zeros_like(s), K=4, early=1 - 1e-4)
    full = oracle.composite(tf, s, np.zeros_like(s), K=4, early=2.0)
    assert out[3] >= 1 - 1e-4 and out[3] < full[3]
    assert abs(out[3] - full[3]) <= 1e-4


def test_converges_to_volume_render_integral():
    """Linear rho along the ray and a one-segment linear TF: the composite
    converges to the emission-absorption integral (Eq. 2) at second order."""
    sigma = 2.0
    # TF values are stored as float32: use the rounded values on both sides
    c0 = np.array([0.2, 0.9, 0.4, 0.1], np.float32).astype(np.float64)
    c1 = np.array([0.8, 0.1, 0.6, 0.9], np.float32).astype(np.float64)
    tf = _tf([0, 1], [c0, c1], sigma)
    L = 1.7
    r0, r1 = 0.15, 0.85

    def rgba(s):
        r = r0 + (r1 - r0) * s / L
        return c0 + r * (c1 - c0)

    def tau(s):   # optical depth from 0 to s
        return quad(lambda u: sigma * rgba(u)[3], 0, s, epsabs=1e-14)[0]

    ref_a = 1 - np.exp(-tau(L))
    ref_c = [quad(lambda s: sigma * rgba(s)[3] * rgba(s)[k] * np.exp(-tau(s)), 0, L, epsabs=1e-13)[0]
             for k in range(3)]
    errs = []
    for n in (8, 16, 32, 64):
        s = np.linspace(0, L, n + 1)
        rho = r0 + (r1 - r0) * s / L
        out = oracle.composite(tf, s, rho, K=1, early=2.0)
        assert out[3] == pytest.approx(ref_a, abs=1e-13)   # exact: A linear in s
        errs.append(np.abs(out[:3] - ref_c).max())
    errs = np.array(errs)
    assert errs[-1] < 5e-4
    slopes = np.log2(errs[:-1] / errs[1:])
    assert np.all(np.abs(slopes - 2) < 0.3), slopes


def test_affine_box_image_constant_density():
    """Whole image of an affine box with a constant scalar: every pixel is
    1 - exp(-sigma A L) with L the closed-form slab length."""
    from tests.test_oracle_bspline import _affine_block
    from tests.test_oracle_intersect import _slab
    rng = np.random.default_rng(31)
    blk, A, b = _affine_block(rng)
    blk.scalar_cp = np.full(blk.geom_cp.shape[:3], 0.3)
    col = np.array([0.25, 0.5, 0.625, 0.75])   # exact in float32
    tf = scenes.TransferFunction(np.array([0, 1], np.float32), np.array([col, col], np.float32), 1.5,
                                 lo=0.0, hi=1.0)
    centre = b + A @ np.full(3, 0.5)
    diag = 2 * np.linalg.norm(A @ np.ones(3))
    cam = scenes.Camera(False, tuple(centre + np.array([3.0, 1.0, 2.0])), tuple(centre), (0, 0, 1),
                        fovy_deg=40.0)
    sc = scenes.Scene("box", [blk], scenes.SCALAR_CP, tf, cam, 24, 24,
                      scenes.RenderParams(ds=diag / 50, early_alpha=2.0))
    img = oracle.render(sc)
    for y in range(24):
        for x in range(24):
            o, d = oracle.ray(cam, 24, 24, x, y)
            ref = _slab(A, b, o, d)
            L = 0.0 if ref is None else ref[1] - ref[0]
            a = 1 - np.exp(-1.5 * col[3] * L)
            assert img[y, x, 3] == pytest.approx(a, abs=1e-12)
