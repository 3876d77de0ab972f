"""The von Mises scalar of §6.2 (Eq. 24) on the GPU through the C ABI.

* Homogeneous strain on a curved map: displacement control points M times
  the geometry's make u o phi^-1 affine, so every sample's strain is sym(M)
  and rho is the textbook value (uniaxial |e|, pure shear sqrt(3)/2 |gamma|,
  a rigid rotation 0) wherever the device evaluates it.
* The loaded beam (the bent beam with a cantilever displacement spline)
  rendered by every integrator path that evaluates the scalar -- the split
  FP32 / mixed shading pass, the fused FP64 integrator, the fixed-step family,
  per-sample root finding -- against the oracle's image (max |dRGBA| <= 1e-3).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_RGBA = 1e-3


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


def _homogeneous(sc, M, t=(0.05, -0.02, 0.01)):
    M = np.asarray(M, float)
    blocks = [dataclasses.replace(b, disp_cp=b.geom_cp @ M.T + np.asarray(t)) for b in sc.blocks]
    return dataclasses.replace(sc, blocks=blocks, scalar_mode=scenes.SCALAR_VONMISES)


@pytest.mark.parametrize("M,want", [
    (np.diag([2e-3, 0.0, 0.0]), 2e-3),
    (np.array([[0.0, 4e-3, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), math.sqrt(3) / 2 * 4e-3),
    (np.array([[0.0, -2e-3, 0.0], [2e-3, 0.0, 0.0], [0.0, 0.0, 0.0]]), 0.0),
], ids=["uniaxial", "pure_shear", "rotation"])
def test_homogeneous_strain_on_device(ivv, M, want):
    sc = _homogeneous(scenes.config(1, width=8, height=8), M)       # the twisted bar: a curved map
    vol = ivv.volume_for(sc)
    p = torch.tensor(np.random.default_rng(5).uniform(0, 1, (4096, 3)), dtype=torch.float32, device="cuda")
    _, _, rho = vol.eval_points(0, p)
    torch.cuda.synchronize()
    rho = rho.cpu().numpy().astype(np.float64)
    # FP32 partials of phi and u: relative error of a few 1e-6 of |J_u|
    assert np.abs(rho - want).max() <= 2e-4 * 4e-3, np.abs(rho - want).max()
    vol.close()


def _loaded_beam(w=256, h=144):
    return scenes.bent_beam(width=w, height=h, displacement=True)


@pytest.fixture(scope="module")
def beam_ref():
    sc = _loaded_beam()
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    return ov, oracle.render(sc, ov)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_loaded_beam_matches_oracle(ivv, beam_ref, prec):
    _, ref = beam_ref
    sc = _loaded_beam()
    sc.params.precision = prec
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    img = vol.render(sc.camera, sc.params, sc.width, sc.height, flags=ivv.FLAG_STATS)
    torch.cuda.synchronize()
    st = vol.stats()
    img = img.cpu().numpy().astype(np.float64)
    assert ref[..., 3].max() > 0.3
    # the split integration counts its shading pass's scalar evaluations;
    # the fused FP64 integrator evaluates the scalar with each sample
    assert (st["rho_evals"] if prec != 2 else st["samples"]) > 10000
    err = np.abs(img - ref).max()
    assert err <= TOL_RGBA, err
    vol.close()


def test_loaded_beam_root_finding(ivv, beam_ref):
    """Per-sample root finding (§5.1): the scalar at each Newton solution."""
    _, ref = beam_ref
    sc = _loaded_beam()
    sc.params.method = 1
    sc.params.use_mlp_guess = 2
    sc.params.rf_tol = 1e-3
    vol = ivv.volume_for(sc)
    img = vol.render(sc.camera, sc.params, sc.width, sc.height)
    torch.cuda.synchronize()
    err = np.abs(img.cpu().numpy().astype(np.float64) - ref).max()
    assert err <= TOL_RGBA, err
    vol.close()


def test_loaded_beam_fixed_step(ivv):
    """The fixed-step family's scalar at the step ends (midpoint, one step
    per sample interval) against the oracle's same method."""
    sc = _loaded_beam(160, 90)
    sc.params.rk_method = 2
    vol = ivv.volume_for(sc)
    img = vol.render(sc.camera, sc.params, sc.width, sc.height)
    torch.cuda.synchronize()
    ref = oracle.render(sc, oracle.OracleVolume(sc.blocks, sc.scalar_mode), method=oracle.FIXED_MIDPOINT)
    err = np.abs(img.cpu().numpy().astype(np.float64) - ref).max()
    assert ref[..., 3].max() > 0.3
    assert err <= TOL_RGBA, err
    vol.close()


def test_batch_rejects_von_mises(ivv):
    sc = _loaded_beam(32, 32)
    vol = ivv.volume_for(sc)
    with pytest.raises(ivv.IvvError) as e:
        ivv.Batch([(vol, sc.camera, 32, 32, None)])
    assert e.value.status == 7
    vol.close()
