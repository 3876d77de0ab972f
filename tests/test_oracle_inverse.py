"""Pins of the oracle's preimage computation: the paper's printed Table 1
(§5.3) for the RK tableaux and the ODE right-hand side, closed-form inverses
of affine maps for the RF Newton (§5.1), agreement of the two independent
FP64 routes (per-sample Newton vs RKF45 on the pulled-back ODE of §5.2), and
the invariants that the exit lies on a face and det J > 0 along the ray."""
import os

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes
from tests.test_oracle_bspline import _affine_block

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_convergence.txt")
METHODS = {"RK1": 1, "RK2": 2, "RK3": 3, "RK4": 4, "RK4_38": 5, "RKF": 6}
ORDERS = {"RK1": 1, "RK2": 2, "RK3": 3, "RK4": 4, "RK4_38": 4, "RKF": 5}


def _golden():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rows[k] = np.array([float(x) for x in v])
    return rows


def test_table1_explicit_rk_matches_printed_values():
    g = _golden()
    ds = g["ds"]
    for name, m in METHODS.items():
        ours = np.array([oracle.table1(m, h, c=1.0) for h in ds])
        printed = g[name]
        # magnitudes as printed (two digits) within 30 %
        np.testing.assert_allclose(ours, printed, rtol=0.3, err_msg=name)
        # observed orders between successive halvings: close to the printed
        # table's own (pre-asymptotic) slopes and to the method's order
        slopes = np.log2(ours[:-1] / ours[1:])
        printed_slopes = np.log2(printed[:-1] / printed[1:])
        assert np.all(np.abs(slopes - printed_slopes) < 0.25), (name, slopes, printed_slopes)
        assert np.all(np.abs(slopes - ORDERS[name]) < 0.5), (name, slopes)


def test_table1_root_finding_reaches_tolerance():
    g = _golden()
    for tol, key in [(1e-3, "RF_1e-3"), (1e-14, "RF_1e-14")]:
        ours = np.array([oracle.table1(7, h, rf_tol=tol) for h in g["ds"]])
        assert np.all(ours <= max(tol, 1e-15))
        if tol == 1e-3:
            np.testing.assert_allclose(ours, g[key], rtol=0.1)
        else:
            assert np.all(ours < 1e-15)


def test_table1_plants_are_caught():
    """Dropping or mis-scaling the perpendicular term c V_perp (Eq. 10) moves
    the third-order row off the printed values, so the pin sees it."""
    g = _golden()
    for c in (0.0, 0.5, 5.0):
        bad = np.array([oracle.table1(3, h, c=c) for h in g["ds"]])
        assert not np.allclose(bad, g["RK3"], rtol=0.3), c


def test_rf_inverts_affine_map_exactly():
    rng = np.random.default_rng(20)
    blk, A, b = _affine_block(rng)
    vol = oracle.OracleVolume([blk], scenes.SCALAR_DETJ)
    for _ in range(50):
        p = rng.uniform(0, 1, 3)
        q, it = vol.invert(0, A @ p + b, rng.uniform(0, 1, 3))
        assert it >= 0
        np.testing.assert_allclose(q, p, atol=1e-12)


def test_rf_and_rkf45_routes_agree():
    sc = scenes.config(0, width=40, height=40)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    a = oracle.render(sc, vol, method=0)
    b = oracle.render(sc, vol, method=1)
    assert np.abs(a).max() > 0.1
    assert np.abs(a - b).max() < 1e-9
    sc1 = scenes.config(1, width=96, height=54)
    vol1 = oracle.OracleVolume(sc1.blocks, sc1.scalar_mode)
    a = oracle.render(sc1, vol1, method=0, window=(40, 56, 0, 54))
    b = oracle.render(sc1, vol1, method=1, window=(40, 56, 0, 54))
    assert np.abs(a).max() > 0.1
    assert np.abs(a - b).max() < 1e-9


@pytest.mark.parametrize("cfg", [0, 1])
def test_trace_invariants(cfg):
    """Every sample maps onto the ray (pixel accuracy, Def. 1), depth is
    monotone, det J > 0, and the last sample is the exit point on a face."""
    sc = scenes.config(cfg, width=48, height=48)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(21)
    n = 0
    for _ in range(200):
        x, y = rng.integers(0, 48, 2)
        pairs, um = vol.pixel_pairs(sc.camera, 48, 48, x, y)
        o, d = oracle.ray(sc.camera, 48, 48, x, y)
        for pr in pairs:
            rows = oracle.trace_pair(vol, sc, o, d, pr)
            s, P = rows[:, 0], rows[:, 1:4]
            phi, J, _ = vol.eval(pr.block, P)
            g = o + (pr.t_in + s)[:, None] * d
            assert np.abs(phi - g).max() < 1e-10
            assert np.all(np.diff((phi - o) @ d) > 0)
            assert np.all(np.linalg.det(J) > 0)
            assert s[-1] == pytest.approx(pr.t_out - pr.t_in, abs=1e-12)
            np.testing.assert_allclose(P[-1], pr.p_out, atol=1e-9)
            n += 1
        if n > 25:
            break
    assert n > 10
