"""Implicit Euler of §5.2 on the GPU (rk_method 7: one step per sample
interval, Newton on G(z) = z - ds W(p + z) with the exact Jacobian from the
spline Hessian), against the oracle taking the same steps in FP64 (max
|dRGBA| <= 1e-3), through the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_RGBA = 1e-3
IRK1 = 7


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


def _render(ivv, sc, flags=0):
    vol = ivv.volume_for(sc)
    img = vol.render(sc.camera, sc.params, sc.width, sc.height, flags=flags)
    torch.cuda.synchronize()
    return vol, img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("cfg,size,c", [(0, (48, 48), 1.0), (1, (120, 72), 1.0), (1, (120, 72), 100.0),
                                        (2, (96, 60), 1.0), (4, (128, 72), 100.0)])
def test_implicit_euler_matches_oracle(ivv, cfg, size, c):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = scenes.PRECISION_FP32
    sc.params.rk_method = IRK1
    sc.params.c = c
    vol, img = _render(ivv, sc)
    ref = oracle.render(sc, oracle.OracleVolume(sc.blocks, sc.scalar_mode), method=oracle.IMPLICIT_EULER)
    assert ref[..., 3].max() > 0.1
    err = np.abs(img - ref).max()
    assert err <= TOL_RGBA, (cfg, c, err)


def test_implicit_euler_mixed_precision(ivv):
    sc = scenes.config(2, width=96, height=60)
    sc.params.precision = scenes.PRECISION_MIXED
    sc.params.rk_method = IRK1
    sc.params.c = 100.0
    vol, img = _render(ivv, sc)
    ref = oracle.render(sc, oracle.OracleVolume(sc.blocks, sc.scalar_mode), method=oracle.IMPLICIT_EULER)
    assert np.abs(img - ref).max() <= TOL_RGBA


def test_implicit_euler_exact_on_affine_geometry(ivv):
    from tests.test_oracle_bspline import _affine_block
    rng = np.random.default_rng(42)
    blk, A, b = _affine_block(rng)
    blk.scalar_cp = rng.uniform(0, 1, blk.geom_cp.shape[:3])
    centre = b + A @ np.full(3, 0.5)
    cam = scenes.Camera(False, tuple(centre + np.array([3.0, 1.0, 2.0])), tuple(centre), (0, 0, 1),
                        fovy_deg=40.0)
    tf = scenes.TransferFunction(np.array([0, 0.5, 1], np.float32),
                                 np.array([[0.2, 0.4, 0.6, 0.5], [0.9, 0.1, 0.3, 0.8], [0.3, 0.7, 0.2, 0.4]],
                                          np.float32), 3.0)
    sc = scenes.Scene("affine", [blk], scenes.SCALAR_CP, tf, cam, 40, 40,
                      scenes.RenderParams(rk_method=IRK1, c=100.0))
    vol, img = _render(ivv, sc)
    ref = oracle.render(sc, method=oracle.METHOD_RF)
    assert ref[..., 3].max() > 0.3
    assert np.abs(img - ref).max() <= TOL_RGBA


@pytest.mark.parametrize("c", [1.0, 100.0])
def test_implicit_euler_counters_show_quadratic_newton(ivv, c):
    """One evaluation per Newton iteration plus the last sample of each
    pair; with the exact Jacobian Newton needs about three iterations per
    step and never reaches the iteration cap."""
    sc = scenes.config(1, width=96, height=54)
    sc.params.rk_method = IRK1
    sc.params.c = c
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    vol.render(sc.camera, sc.params, sc.width, sc.height, flags=ivv.FLAG_STATS)
    s = vol.stats()
    assert s["rk_steps"] > 0 and s["rk_rejects"] == 0
    assert s["samples"] == s["rk_steps"] + s["pairs"]
    iters = s["rhs_evals"] - s["pairs"]
    assert iters >= s["rk_steps"]
    assert iters / s["rk_steps"] <= 4.0, iters / s["rk_steps"]
    assert s["step_cap"] == 0


def test_implicit_euler_stays_on_the_ray_at_large_c(ivv):
    """Delta P (Eq. 5): the stiff pull-back (c = 100) keeps implicit Euler's
    samples closer to the view ray than explicit Euler's at c = 1."""
    sc = scenes.config(1, width=96, height=54)
    dp = {}
    for method, c in ((1, 1.0), (IRK1, 100.0)):
        sc.params.rk_method = method
        sc.params.c = c
        vol = ivv.volume_for(sc)
        vol.reset_stats()
        vol.render(sc.camera, sc.params, sc.width, sc.height, flags=ivv.FLAG_STATS)
        dp[method] = vol.stats()["max_delta_p"]
    assert dp[IRK1] < dp[1], dp
