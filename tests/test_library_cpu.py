"""CPU checks of the C-ABI library: it builds, loads and exports every
function include/ivv.h declares; its host preparation (knot insertion,
degree elevation, face extraction, validation) reproduces the oracle's
Cox-de Boor evaluation; invalid descriptions are rejected with statuses."""
import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import build as libbuild
from paper_1404_3363_gb300 import ivv, scenes
from tests.test_oracle_bspline import _affine_block


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ivv.load()


def test_exports_every_declared_function(lib):
    names = ivv.header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("cfg", [0, 1, 2, 4])
def test_bezier_extraction_matches_oracle(lib, cfg):
    sc = scenes.config(cfg, width=8, height=8)
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(40 + cfg)
    P = rng.uniform(0, 1, (300, 3))
    P[:27] = np.stack(np.meshgrid(*[[0.0, 0.5, 1.0]] * 3, indexing="ij"), -1).reshape(-1, 3)
    for b in range(0, len(sc.blocks), max(1, len(sc.blocks) // 4)):
        f1, J1, r1 = ivv.host_eval(sc.blocks, sc.scalar_mode, b, P)
        f2, J2, r2 = ov.eval(b, P)
        np.testing.assert_allclose(f1, f2, atol=1e-12)
        np.testing.assert_allclose(J1, J2, atol=1e-10 * np.abs(J2).max())
        np.testing.assert_allclose(r1, r2, atol=1e-12 * max(1.0, np.abs(r2).max()))


def test_degree_elevation_and_mixed_degrees(lib):
    """Blocks of degrees (1,2,3) are raised to cubic without changing phi."""
    rng = np.random.default_rng(41)
    kn = [scenes.open_uniform_knots(n, p) for n, p in ((4, 1), (5, 2), (7, 3))]
    inner = np.sort(rng.uniform(0.1, 0.9, 3))
    kn[2] = np.concatenate([np.zeros(4), inner, np.ones(4)])
    cp = rng.normal(size=(7, 5, 4, 3)) * 0.01 + scenes._grid(np.linspace(0, 1, 4), np.linspace(0, 1, 5),
                                                           np.linspace(0, 1, 7))
    blk = scenes.Block((1, 2, 3), kn, cp, rng.uniform(0, 1, (7, 5, 4)))
    ov = oracle.OracleVolume([blk], scenes.SCALAR_CP)
    P = rng.uniform(0, 1, (200, 3))
    f1, J1, r1 = ivv.host_eval([blk], scenes.SCALAR_CP, 0, P)
    f2, J2, r2 = ov.eval(0, P)
    np.testing.assert_allclose(f1, f2, atol=1e-13)
    np.testing.assert_allclose(J1, J2, atol=1e-11)
    np.testing.assert_allclose(r1, r2, atol=1e-13)


def test_affine_block_jacobian(lib):
    rng = np.random.default_rng(42)
    blk, A, b = _affine_block(rng)
    P = rng.uniform(0, 1, (50, 3))
    f, J, r = ivv.host_eval([blk], scenes.SCALAR_QUALITY, 0, P)
    np.testing.assert_allclose(f, P @ A.T + b, atol=1e-12)
    np.testing.assert_allclose(r, np.linalg.det(A) / np.linalg.norm(A), rtol=1e-12)


def test_invalid_descriptions_are_rejected(lib):
    sc = scenes.config(0)
    good = sc.blocks[0]

    def status_of(blocks, mode=scenes.SCALAR_CP):
        with pytest.raises(ivv.IvvError) as e:
            ivv.host_eval(blocks, mode, 0, np.zeros((1, 3)))
        return e.value.status

    bad = scenes.Block(good.degree, [good.knots[0][::-1].copy(), good.knots[1], good.knots[2]], good.geom_cp,
                       good.scalar_cp)
    assert status_of([bad]) == 1                                    # knots not non-decreasing
    bad = scenes.Block(good.degree, good.knots, good.geom_cp, None)
    assert status_of([bad]) == 1                                    # CP mode without scalars
    bad = scenes.Block((4, 3, 3), [np.r_[np.zeros(5), np.ones(5)], good.knots[1], good.knots[2]],
                       np.zeros((4, 4, 5, 3)), np.zeros((4, 4, 5)))
    assert status_of([bad]) == 7                                    # degree 4 unsupported
    flipped = good.geom_cp.copy()
    flipped[..., 0] = -flipped[..., 0]                              # mirror: det J < 0
    bad = scenes.Block(good.degree, good.knots, flipped, good.scalar_cp)
    assert status_of([bad]) == 6
    nan = good.geom_cp.copy()
    nan[0, 0, 0, 0] = np.nan
    assert status_of([scenes.Block(good.degree, good.knots, nan, good.scalar_cp)]) == 1
    assert status_of([good], mode=7) == 1
