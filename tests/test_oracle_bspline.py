"""Pins of the oracle's spline evaluation (Eq. 1) against independent facts:
scipy's B-spline basis, the Bernstein closed form of a single element,
partition of unity, linear precision at Greville points, finite differences
of the value, and the closed forms of det J and Eq. 23 on affine maps."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle
from paper_1404_3363_gb300 import scenes


def _block_from(knots, degree, cp, scal=None):
    return scenes.Block(tuple(degree), [np.asarray(k, float) for k in knots], cp, scal)


def _random_knots(rng, n, p):
    inner = np.sort(rng.uniform(0, 1, n - p - 1))
    if n - p - 1 >= 2 and p >= 2:
        inner[1] = inner[0]          # a double knot (still C^{p-2})
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


@pytest.mark.parametrize("p,n", [(1, 4), (2, 7), (3, 9), (3, 4)])
def test_basis_matches_scipy(p, n):
    rng = np.random.default_rng(1)
    kn = _random_knots(rng, n, p)
    cp = rng.normal(size=(p + 1, p + 1, n, 3))
    blk = _block_from([kn, scenes.open_uniform_knots(p + 1, p), scenes.open_uniform_knots(p + 1, p)],
                      (p, p, p), cp)
    vol = oracle.OracleVolume([blk], scenes.SCALAR_DETJ)
    xr = rng.uniform(0, 1, 200)
    x = np.concatenate([xr, kn[p:n + 1]])
    x = x[x < 1.0]
    N, dN = vol.basis(0, 0, x, n)
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1
        bs = BSpline(kn, c, p)
        np.testing.assert_allclose(N[:, i], bs(x), atol=1e-14)
        # derivatives away from knots (one-sided at knots for p = 1)
        m = len(xr)
        np.testing.assert_allclose(dN[:m, i], bs.derivative()(x[:m]), rtol=1e-11, atol=1e-11)


def test_partition_of_unity_and_endpoint():
    rng = np.random.default_rng(2)
    kn = _random_knots(rng, 8, 3)
    cp = rng.normal(size=(4, 4, 8, 3))
    blk = _block_from([kn, scenes.open_uniform_knots(4, 3), scenes.open_uniform_knots(4, 3)], (3, 3, 3), cp)
    vol = oracle.OracleVolume([blk], scenes.SCALAR_DETJ)
    x = np.concatenate([rng.uniform(0, 1, 100), [0.0, 1.0]])
    N, dN = vol.basis(0, 0, x, 8)
    np.testing.assert_allclose(N.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dN.sum(1), 0.0, atol=1e-10)
    assert (N >= -1e-15).all()
    # clamped ends interpolate the end control points
    assert N[-2, 0] == pytest.approx(1.0) and N[-1, -1] == pytest.approx(1.0)


def test_single_element_is_bernstein():
    from math import comb
    rng = np.random.default_rng(3)
    kn = np.array([0, 0, 0, 0, 1, 1, 1, 1.0])
    cp = rng.normal(size=(4, 4, 4, 3))
    scal = rng.normal(size=(4, 4, 4))
    blk = _block_from([kn, kn, kn], (3, 3, 3), cp, scal)
    vol = oracle.OracleVolume([blk], scenes.SCALAR_CP)
    P = rng.uniform(0, 1, (50, 3))
    phi, J, rho = vol.eval(0, P)

    def B(i, x):
        return comb(3, i) * x ** i * (1 - x) ** (3 - i)
    for q, (u, v, w) in enumerate(P):
        ref = np.zeros(3)
        rs = 0.0
        for k in range(4):
            for j in range(4):
                for i in range(4):
                    wt = B(i, u) * B(j, v) * B(k, w)
                    ref += wt * cp[k, j, i]
                    rs += wt * scal[k, j, i]
        np.testing.assert_allclose(phi[q], ref, atol=1e-13)
        assert rho[q] == pytest.approx(rs, abs=1e-13)


def _affine_block(rng, p=(2, 3, 2), n=(5, 6, 4)):
    A = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    b = rng.normal(size=3)
    kn = [scenes.open_uniform_knots(n[d], p[d]) for d in range(3)]
    gu, gv, gw = (scenes.greville(kn[d], p[d]) for d in range(3))
    W_, V_, U_ = np.meshgrid(gw, gv, gu, indexing="ij")
    P = np.stack([U_, V_, W_], -1)
    cp = P @ A.T + b
    return _block_from(kn, p, cp), A, b


def test_linear_precision_affine_map():
    rng = np.random.default_rng(4)
    blk, A, b = _affine_block(rng)
    for mode, ref in [(scenes.SCALAR_DETJ, np.linalg.det(A)),
                      (scenes.SCALAR_QUALITY, np.linalg.det(A) / np.linalg.norm(A))]:
        vol = oracle.OracleVolume([blk], mode)
        P = rng.uniform(0, 1, (100, 3))
        phi, J, rho = vol.eval(0, P)
        np.testing.assert_allclose(phi, P @ A.T + b, atol=1e-12)
        np.testing.assert_allclose(J, np.broadcast_to(A, J.shape), atol=1e-11)
        np.testing.assert_allclose(rho, ref, rtol=1e-11)


def test_partials_match_finite_differences():
    sc = scenes.config(1, width=8, height=8)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(5)
    P = rng.uniform(0.05, 0.95, (40, 3))
    phi, J, _ = vol.eval(0, P)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fp, _, _ = vol.eval(0, P + e)
        fm, _, _ = vol.eval(0, P - e)
        np.testing.assert_allclose(J[:, :, c], (fp - fm) / (2 * h), rtol=1e-6, atol=1e-6)


def test_twisted_bar_is_valid_parametrisation():
    """det J > 0 over the bar (assumption 4 of §5), quality in (0, 1/sqrt(3)*...]."""
    sc = scenes.config(1, width=8, height=8)
    vol = oracle.OracleVolume(sc.blocks, scenes.SCALAR_DETJ)
    g = (np.arange(9) + 0.5) / 9
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    _, _, dj = vol.eval(0, P)
    assert (dj > 0).all()
    for i in (0, 2):
        s = scenes.config(i, width=8, height=8)
        v = oracle.OracleVolume(s.blocks, scenes.SCALAR_DETJ)
        for b in range(len(s.blocks)):
            _, _, dj = v.eval(b, P)
            assert (dj > 0).all()
