"""The fixed-step RK family of §5.2-5.3 on the GPU (rk_method 1-6: Euler,
midpoint, Kutta-3, RK4, RK4 3/8, Fehlberg's fifth-order weights), one step
per sample interval, against the oracle taking the same steps in FP64
(max |dRGBA| <= 1e-3), through the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_RGBA = 1e-3
METHODS = [1, 2, 3, 4, 5, 6]
STAGES = {1: 1, 2: 2, 3: 3, 4: 4, 5: 4, 6: 6}


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


def _render(ivv, sc, prec=0, flags=0):
    vol = ivv.volume_for(sc)
    img = vol.render(sc.camera, sc.params, sc.width, sc.height, flags=flags)
    torch.cuda.synchronize()
    return vol, img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("cfg,size", [(0, (48, 48)), (1, (120, 72)), (2, (96, 60))])
@pytest.mark.parametrize("method", METHODS)
def test_fixed_step_matches_oracle(ivv, cfg, size, method):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = scenes.PRECISION_FP32
    sc.params.rk_method = method
    vol, img = _render(ivv, sc)
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    ref = oracle.render(sc, ov, method=10 + method)
    assert ref[..., 3].max() > 0.1
    err = np.abs(img - ref).max()
    assert err <= TOL_RGBA, (cfg, method, err)


def test_fixed_step_mixed_precision(ivv):
    sc = scenes.config(2, width=96, height=60)
    sc.params.precision = scenes.PRECISION_MIXED
    sc.params.rk_method = 4
    vol, img = _render(ivv, sc)
    ref = oracle.render(sc, oracle.OracleVolume(sc.blocks, sc.scalar_mode), method=14)
    assert np.abs(img - ref).max() <= TOL_RGBA


def test_fixed_step_exact_on_affine_geometry(ivv):
    """Constant pulled-back field along the exact ray: even Euler matches
    the root-finding oracle."""
    from tests.test_oracle_bspline import _affine_block
    rng = np.random.default_rng(41)
    blk, A, b = _affine_block(rng)
    blk.scalar_cp = rng.uniform(0, 1, blk.geom_cp.shape[:3])
    centre = b + A @ np.full(3, 0.5)
    cam = scenes.Camera(False, tuple(centre + np.array([3.0, 1.0, 2.0])), tuple(centre), (0, 0, 1),
                        fovy_deg=40.0)
    tf = scenes.TransferFunction(np.array([0, 0.5, 1], np.float32),
                                 np.array([[0.2, 0.4, 0.6, 0.5], [0.9, 0.1, 0.3, 0.8], [0.3, 0.7, 0.2, 0.4]],
                                          np.float32), 3.0)
    sc = scenes.Scene("affine", [blk], scenes.SCALAR_CP, tf, cam, 40, 40, scenes.RenderParams(rk_method=1))
    vol, img = _render(ivv, sc)
    ref = oracle.render(sc, method=oracle.METHOD_RF)
    assert ref[..., 3].max() > 0.3
    assert np.abs(img - ref).max() <= TOL_RGBA


@pytest.mark.parametrize("method", METHODS)
def test_fixed_step_counters(ivv, method):
    """s right-hand sides per step plus one per pair start, no rejections."""
    sc = scenes.config(1, width=96, height=54)
    sc.params.rk_method = method
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    vol.render(sc.camera, sc.params, sc.width, sc.height, flags=ivv.FLAG_STATS)
    s = vol.stats()
    assert s["rk_rejects"] == 0 and s["rk_steps"] > 0
    assert s["rhs_evals"] == s["samples"] + (STAGES[method] - 1) * s["rk_steps"]
    assert s["samples"] == s["rk_steps"] + s["pairs"]


def test_fixed_step_argument_errors(ivv):
    sc = scenes.config(0, width=16, height=16)
    vol = ivv.volume_for(sc)
    for bad, msg in [(dict(rk_method=8), "rk_method"), (dict(rk_method=4, method=1, precision=scenes.PRECISION_FP32), "ODE method"),
                     (dict(rk_method=4, precision=scenes.PRECISION_FP64), "FP32 or MIXED")]:
        prm = dataclasses.replace(sc.params, **bad)
        with pytest.raises(ivv.IvvError, match=msg):
            vol.render(sc.camera, prm, 16, 16)


def test_fixed_step_pixel_accuracy_follows_the_order(ivv):
    """Delta P (Eq. 5) of the samples: Euler's drift off the ray exceeds
    RK4's by orders of magnitude on the twisted bar."""
    sc = scenes.config(1, width=96, height=54)
    dp = {}
    for method in (1, 4):
        sc.params.rk_method = method
        vol = ivv.volume_for(sc)
        vol.reset_stats()
        vol.render(sc.camera, sc.params, sc.width, sc.height, flags=ivv.FLAG_STATS)
        dp[method] = vol.stats()["max_delta_p"]
    assert dp[1] > 0 and dp[4] >= 0
    assert dp[1] > 20 * dp[4], dp
