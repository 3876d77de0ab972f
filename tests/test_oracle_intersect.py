"""Pins of the oracle's stage 1-2 (§4.1 intersections, §4.2 Alg. 2):
closed-form ray/parallelepiped intersections for affine blocks, brute force
against a dense triangulation of the faces evaluated with scipy, and
hand-built hit lists for the blockwise pairing."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle
from paper_1404_3363_gb300 import scenes
from tests.test_oracle_bspline import _affine_block


def _slab(A, b, o, d):
    """t-interval where A^-1 (o + t d - b) lies in [0,1]^3."""
    Ai = np.linalg.inv(A)
    q0 = Ai @ (o - b)
    q1 = Ai @ d
    lo, hi = -np.inf, np.inf
    for k in range(3):
        if abs(q1[k]) < 1e-300:
            if not (0 <= q0[k] <= 1):
                return None
            continue
        a, c = (0 - q0[k]) / q1[k], (1 - q0[k]) / q1[k]
        lo, hi = max(lo, min(a, c)), min(hi, max(a, c))
    return (lo, hi) if hi > lo else None


def test_affine_block_closed_form():
    rng = np.random.default_rng(10)
    blk, A, b = _affine_block(rng)
    vol = oracle.OracleVolume([blk], scenes.SCALAR_DETJ)
    centre = b + A @ np.full(3, 0.5)
    n_hit = 0
    for _ in range(60):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = centre - 6 * d + 0.6 * rng.normal(size=3)
        ref = _slab(A, b, o, d)
        hits = vol.hits(o, d)
        pairs, um = oracle.pair_hits(hits)
        if ref is None:
            assert len(pairs) == 0
            continue
        n_hit += 1
        assert um == 0 and len(pairs) == 1
        pr = pairs[0]
        assert pr.t_in == pytest.approx(ref[0], abs=1e-10)
        assert pr.t_out == pytest.approx(ref[1], abs=1e-10)
        Ai = np.linalg.inv(A)
        np.testing.assert_allclose(pr.p_in, Ai @ (o + ref[0] * d - b), atol=1e-10)
        np.testing.assert_allclose(pr.p_out, Ai @ (o + ref[1] * d - b), atol=1e-10)
    assert n_hit > 20


def _face_grid(blk, face, n):
    """Dense grid of points of one face, evaluated with scipy (independent)."""
    nd = face // 2
    ad, bd = (nd + 1) % 3, (nd + 2) % 3
    g = np.linspace(0, 1, n)
    p = np.zeros((n, n, 3))
    p[..., nd] = face % 2
    p[..., ad] = g[:, None]
    p[..., bd] = g[None, :]
    mats = []
    for dd in range(3):
        x = p[..., dd].ravel()
        nb = len(blk.knots[dd]) - blk.degree[dd] - 1
        Bm = BSpline.design_matrix(np.clip(x, 0, 1 - 1e-15), blk.knots[dd], blk.degree[dd]).toarray()
        mats.append(Bm.reshape(n, n, nb))
    cp = blk.geom_cp   # [w][v][u][3]
    return np.einsum("abi,abj,abk,kjir->abr", mats[0], mats[1], mats[2], cp)


def _ray_tri_ts(o, d, P):
    """Moller-Trumbore intersections of a ray with the grid's triangles."""
    a, b, c = P[:-1, :-1].reshape(-1, 3), P[1:, :-1].reshape(-1, 3), P[:-1, 1:].reshape(-1, 3)
    e, f, g = P[1:, 1:].reshape(-1, 3), c, b
    ts = []
    for p0, p1, p2 in ((a, b, c), (e, f, g)):
        e1, e2 = p1 - p0, p2 - p0
        h = np.cross(d, e2)
        det = np.einsum("ij,ij->i", e1, h)
        ok = np.abs(det) > 1e-14
        inv = np.where(ok, 1 / np.where(ok, det, 1), 0)
        s = o - p0
        u = inv * np.einsum("ij,ij->i", s, h)
        q = np.cross(s, e1)
        v = inv * (q @ d)
        t = inv * np.einsum("ij,ij->i", e2, q)
        m = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
        ts.extend(t[m].tolist())
    return sorted(ts)


def test_twisted_cube_hits_match_dense_triangulation():
    sc = scenes.config(0)
    blk = sc.blocks[0]
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    grids = [_face_grid(blk, f, 301) for f in range(6)]
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(40):
        x, y = rng.integers(16, 48, 2)
        o, d = oracle.ray(sc.camera, 64, 64, x, y)
        hits = vol.hits(o, d)
        ref = sorted(t for G in grids for t in _ray_tri_ts(o, d, G))
        # merge triangle duplicates on shared edges
        merged = []
        for t in ref:
            if not merged or t - merged[-1] > 1e-6:
                merged.append(t)
        got = [h.t for h in hits]
        if len(merged) != len(got):
            # a grazing ray can split differently on the triangulation; such
            # rays must have a pair of hits closer than the triangulation error
            gaps = np.diff(sorted(got + merged)) if got + merged else []
            assert min(gaps, default=0) < 1e-3
            continue
        np.testing.assert_allclose(got, merged, atol=2e-4)
        checked += 1
    assert checked >= 30


def test_hits_are_inside_outside_transitions():
    """Midpoints of every pair invert to the interior; points just beyond the
    ends of a pair do not invert inside the block (Eq. 7 with clamping)."""
    sc = scenes.config(0)
    vol = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(12)
    for _ in range(30):
        x, y = rng.integers(0, 64, 2)
        o, d = oracle.ray(sc.camera, 64, 64, x, y)
        pairs, um = vol.pixel_pairs(sc.camera, 64, 64, x, y)
        assert um == 0
        for pr in pairs:
            assert pr.t_out > pr.t_in
            g = o + 0.5 * (pr.t_in + pr.t_out) * d
            p, it = vol.invert(pr.block, g, np.full(3, 0.5))
            assert it >= 0 and ((p > 0) & (p < 1)).all()
            for t in (pr.t_in - 1e-3, pr.t_out + 1e-3):
                p, it = vol.invert(pr.block, o + t * d, np.full(3, 0.5))
                phi, _, _ = vol.eval(pr.block, p)
                assert np.linalg.norm(phi[0] - (o + t * d)) > 1e-5
            # the entry and exit parameters lie on a face of [0,1]^3
            for q in (pr.p_in, pr.p_out):
                q = np.array(q)
                assert np.min(np.minimum(np.abs(q), np.abs(q - 1))) < 1e-12


def _h(t, block, front):
    return oracle.Hit(t, (0.0, 0.0, 0.0), block, 0, front)


def test_alg2_blockwise_pairing():
    # two blocks sharing a face: exit of block 0 and entry of block 1 coincide
    hits = [_h(1.0, 0, 1), _h(2.0, 0, 0), _h(2.0, 1, 1), _h(3.0, 1, 0)]
    pairs, um = oracle.pair_hits(hits[::-1])
    assert um == 0
    assert [(p.block, p.t_in, p.t_out) for p in pairs] == [(0, 1.0, 2.0), (1, 2.0, 3.0)]
    # coincident records listed in the "wrong" order still pair by block
    hits = [_h(1.0, 0, 1), _h(2.0, 1, 1), _h(2.0, 0, 0), _h(3.0, 1, 0)]
    pairs, um = oracle.pair_hits(hits)
    assert [(p.block, p.t_in, p.t_out) for p in pairs] == [(0, 1.0, 2.0), (1, 2.0, 3.0)]
    # non-convex block: two chords of one block, exits taken nearest first
    hits = [_h(5.0, 0, 0), _h(1.0, 0, 1), _h(4.0, 0, 1), _h(2.0, 0, 0)]
    pairs, um = oracle.pair_hits(hits)
    assert [(p.t_in, p.t_out) for p in pairs] == [(1.0, 2.0), (4.0, 5.0)]
    # an exit without an entry (eye inside the block) is dropped and counted
    pairs, um = oracle.pair_hits([_h(2.0, 0, 0), _h(3.0, 1, 1), _h(4.0, 1, 0)])
    assert [(p.block, p.t_in) for p in pairs] == [(1, 3.0)] and um == 1
    # an unmatched entry is counted too
    pairs, um = oracle.pair_hits([_h(1.0, 0, 1), _h(2.0, 0, 0), _h(3.0, 0, 1)])
    assert len(pairs) == 1 and um == 1
