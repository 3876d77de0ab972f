"""Oracle pins of the fixed-step explicit RK family of §5.2-5.3 in the render
path (one step of the tableau per sample interval, stage points clamped to
the parameter box as in §5.4).

* Affine geometry: the pulled-back field is constant along the exact
  parameter-space ray (J is constant and V = d on it), so every consistent
  method reproduces the root-finding render exactly.
* Curved block (the twisted bar): halving ds divides the parameter error
  against the root-finding trace by 2^q for a method of order q (Euler 1,
  midpoint 2, Kutta 3, RK4 and its 3/8 rule 4, Fehlberg's fifth-order
  weights 5); a dropped stage, a wrong weight or a wrong node breaks the
  order.  The tableaux themselves are pinned to the printed Table 1 values
  in test_oracle_inverse.py.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes
from tests.test_oracle_bspline import _affine_block

FIXED = [oracle.FIXED_EULER, oracle.FIXED_MIDPOINT, oracle.FIXED_KUTTA3, oracle.FIXED_RK4, oracle.FIXED_RK4_38,
         oracle.FIXED_FEHLBERG5]


def test_fixed_step_methods_are_exact_on_affine_geometry():
    rng = np.random.default_rng(40)
    blk, A, b = _affine_block(rng)
    blk.scalar_cp = rng.uniform(0, 1, blk.geom_cp.shape[:3])
    centre = b + A @ np.full(3, 0.5)
    cam = scenes.Camera(False, tuple(centre + np.array([3.0, 1.0, 2.0])), tuple(centre), (0, 0, 1), fovy_deg=40.0)
    tf = scenes.TransferFunction(np.array([0, 0.5, 1], np.float32),
                                 np.array([[0.2, 0.4, 0.6, 0.5], [0.9, 0.1, 0.3, 0.8], [0.3, 0.7, 0.2, 0.4]],
                                          np.float32), 3.0)
    sc = scenes.Scene("affine", [blk], scenes.SCALAR_CP, tf, cam, 20, 20, scenes.RenderParams())
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    ref = oracle.render(sc, vol, method=oracle.METHOD_RF)
    assert ref[..., 3].max() > 0.3
    for m in FIXED:
        img = oracle.render(sc, vol, method=m)
        assert np.abs(img - ref).max() < 1e-12, m


@pytest.fixture(scope="module")
def bar_pair():
    sc = scenes.config(1, width=64, height=36)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    pairs, _ = vol.pixel_pairs(sc.camera, 64, 36, 30, 18)
    o, d = oracle.ray(sc.camera, 64, 36, 30, 18)
    return sc, vol, o, d, pairs[0]


def _param_error(bar_pair, method, ds):
    sc, vol, o, d, pr = bar_pair
    s2 = dataclasses.replace(sc, params=dataclasses.replace(sc.params, ds=ds, early_alpha=2.0))
    got = oracle.trace_pair(vol, s2, o, d, pr, method=method)
    ref = oracle.trace_pair(vol, s2, o, d, pr, method=oracle.METHOD_RF)
    assert got.shape == ref.shape
    np.testing.assert_array_equal(got[:, 0], ref[:, 0])          # the same sample points
    return np.abs(got[:, 1:4] - ref[:, 1:4]).max()


@pytest.mark.parametrize("method", FIXED)
def test_fixed_step_order_on_the_twisted_bar(bar_pair, method):
    L = bar_pair[4].t_out - bar_pair[4].t_in
    q = oracle.FIXED_ORDER[method]
    errs = np.array([_param_error(bar_pair, method, L / k) for k in (4, 8, 16)])
    slopes = np.log2(errs[:-1] / errs[1:])
    assert errs[0] > 1e-9                      # measurably inexact at the coarse step
    assert abs(slopes[0] - q) < 0.5, slopes
    if q < 5:                                  # the finest fifth-order error nears the reference's own tolerance
        assert abs(slopes[1] - q) < 0.5, slopes
