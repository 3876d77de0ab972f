"""§5.4, singular Jacobian at the entry point (Eq. 22), on the GPU through
the C ABI: the degenerate-face cube (three coincident upper control-point
layers, det J = 0 on its whole top face) rendered from above, so that most
rays enter where the Jacobian is singular.  Images against the oracle, which
applies the same rule in FP64 (max |dRGBA| <= 1e-3); the counters show the
moved entries and, in mixed precision, the FP64 3x3 solves of the Newton
iterations that start next to the singular face."""
import dataclasses

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


def _render(ivv, sc, flags=0):
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    img = vol.render(sc.camera, sc.params, sc.width, sc.height, flags=flags)
    torch.cuda.synchronize()
    return vol, img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("ortho", [True, False])
def test_degenerate_cube_matches_oracle(ivv, prec, ortho):
    sc = scenes.degenerate_cube(width=160, height=160, ortho=ortho)
    sc.params.precision = prec
    vol, img = _render(ivv, sc, flags=ivv.FLAG_STATS)
    st = vol.stats()
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    ref, rs = oracle.render(sc, ov, stats=True)
    assert np.isfinite(img).all()
    assert ref[..., 3].max() > 0.3
    assert rs[..., 5].sum() > 1000                                     # the oracle moved that many entries
    assert abs(st["entry_shrinks"] - rs[..., 5].sum()) <= 0.01 * rs[..., 5].sum(), (st["entry_shrinks"], rs[..., 5].sum())
    if prec == 1:
        assert st["fp64_solves"] > 0
    err = np.abs(img - ref).max()
    assert err <= TOL_RGBA, err


@pytest.mark.parametrize("rk_method,c", [(2, 1.0), (4, 1.0), (7, 100.0)])
def test_degenerate_cube_other_integrators(ivv, rk_method, c):
    """The moved entries serve every integrator (the rule acts on the pairs)."""
    sc = scenes.degenerate_cube(width=128, height=128)
    sc.params = dataclasses.replace(sc.params, rk_method=rk_method, c=c, precision=1)
    vol, img = _render(ivv, sc)
    method = {2: oracle.FIXED_MIDPOINT, 4: oracle.FIXED_RK4, 7: oracle.IMPLICIT_EULER}[rk_method]
    ref = oracle.render(sc, oracle.OracleVolume(sc.blocks, sc.scalar_mode), method=method)
    assert np.isfinite(img).all()
    assert np.abs(img - ref).max() <= TOL_RGBA


def test_degenerate_cube_rf_method(ivv):
    sc = scenes.degenerate_cube(width=128, height=128)
    sc.params = dataclasses.replace(sc.params, method=1, rf_tol=1e-3)
    vol, img = _render(ivv, sc)
    ref = oracle.render(sc, oracle.OracleVolume(sc.blocks, sc.scalar_mode))
    assert np.isfinite(img).all()
    assert np.abs(img - ref).max() <= TOL_RGBA


def test_moved_entries_match_the_oracle_pairs(ivv):
    """Pair counts, blocks and entry depths t_in (moved by delta) per pixel."""
    sc = scenes.degenerate_cube(width=128, height=128)
    sc.params.precision = 1
    vol = ivv.volume_for(sc)
    cg, pg, bg = vol.render_pairs(sc.camera, sc.params, sc.width, sc.height, max_pairs=4)
    cg, pg = cg.cpu().numpy(), pg.cpu().numpy().astype(np.float64)
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    co, po, bo = ov.window_pairs(sc.camera, sc.width, sc.height, cap=4)
    same = cg == co
    assert same.mean() > 0.999
    m = same & (co > 0)
    assert m.sum() > 3000
    assert np.abs(pg[0][m][:, 3] - po[0][m][:, 3]).max() <= 2e-4
    assert np.abs(pg[0][m][:, 7] - po[0][m][:, 7]).max() <= 2e-4


def test_regular_volumes_take_no_fixup(ivv):
    """Volumes without a face where det J comes close to zero skip the check
    (no launch, no counts)."""
    sc = scenes.config(1, width=96, height=54)
    vol, img = _render(ivv, sc, flags=ivv.FLAG_STATS)
    assert vol.stats()["entry_shrinks"] == 0
