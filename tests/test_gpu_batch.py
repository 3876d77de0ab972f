"""Batched rendering (ivv_batch_*) on the GPU, through the C ABI.

A batch renders every request with one launch per stage over all requests,
from the merged volume pool, replayed from a CUDA graph.  Checked here:
images against the FP64 oracle (max |dRGBA| <= 1e-3) on small requests of
all three volumes with per-request cameras and transfer functions; agreement
with the single-frame path; invariance under the K2 tile shape; the step
batch and K5 occupancy variants against the oracle; graph replay, camera
updates, the autotuner, counters, argument errors; and the full 64-request
workload (about 31 M pixels) on pixels sampled against the oracle one by one.
"""
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


@pytest.fixture(scope="module")
def pool(ivv):
    """The three volumes of the batched workload and oracle copies."""
    vols, reqs = scenes.batch_requests()
    gpu = [ivv.volume_for(v) for v in vols]
    orc = [oracle.OracleVolume(v.blocks, v.scalar_mode) for v in vols]
    return vols, reqs, gpu, orc


def _small(reqs, sizes, n):
    """The first n requests with small ragged image sizes (several tiles of
    every shape, partial edge tiles)."""
    out = []
    for i, q in enumerate(reqs[:n]):
        w, h = sizes[i % len(sizes)]
        out.append(dataclasses.replace(q, width=w, height=h))
    return out


SIZES = [(40, 24), (33, 17), (48, 40), (25, 31), (56, 9), (17, 46)]


def _scene(vols, q):
    return dataclasses.replace(vols[q.volume], camera=q.camera, tf=q.tf, width=q.width, height=q.height,
                               params=scenes.RenderParams())


def _batch(ivv, gpu, reqs, params=None):
    items = [(gpu[q.volume], q.camera, q.width, q.height, q.tf) for q in reqs]
    return ivv.Batch(items, params)


def _np(t):
    return t.cpu().numpy().astype(np.float64)


def test_batch_matches_oracle(ivv, pool):
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 12)
    assert {q.volume for q in small} == {0, 1, 2}
    b = _batch(ivv, gpu, small)
    outs = b.render()
    torch.cuda.synchronize()
    lit = 0
    for q, out in zip(small, outs):
        ref = oracle.render(_scene(vols, q), orc[q.volume])
        err = np.abs(_np(out) - ref).max()
        assert err <= TOL_RGBA, (q.volume, q.width, q.height, err)
        lit += int((ref[..., 3] > 0.05).sum())
    assert lit > 500, "the requests see their volumes"


def test_batch_equals_single_frame_path(ivv, pool):
    """Same cameras, transfer functions and parameters through ivv_render.
    The batch integrator composites inside the ODE kernel, the single-frame
    FP32 path in a separate shading pass over the stored sample points: the
    same steps and samples, with the scalar and the compositing rounded in a
    different order, so the images agree to rounding amplified by the
    transfer function's slope (both match the oracle to 1e-3 elsewhere)."""
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 9)
    b = _batch(ivv, gpu, small)
    outs = [o.clone() for o in b.render()]
    worst = 0.0
    for q, out in zip(small, outs):
        v = gpu[q.volume]
        v.set_transfer_function(q.tf)
        one = v.render(q.camera, scenes.RenderParams(), q.width, q.height)
        worst = max(worst, (one - out).abs().max().item())
    for k, v in enumerate(gpu):
        v.set_transfer_function(vols[k].tf)
    assert worst <= 2e-4, worst


def test_tile_shapes_give_identical_images(ivv, pool):
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 8)
    b = _batch(ivv, gpu, small)
    base = [o.clone() for o in b.render()]
    t = b.tuning
    assert (t["tile_w"], t["tile_h"], t["step_samples"]) == (8, 4, 8)
    for tw, th in [(4, 8), (16, 2), (8, 4)]:
        b.tuning = dict(t, tile_w=tw, tile_h=th)
        outs = b.render()
        torch.cuda.synchronize()
        for x, y in zip(base, outs):
            assert torch.equal(x, y), (tw, th)


@pytest.mark.parametrize("step,ctas", [(4, 1), (16, 2), (8, 3)])
def test_step_batch_and_occupancy_variants_match_oracle(ivv, pool, step, ctas):
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 6)
    b = _batch(ivv, gpu, small)
    b.tuning = dict(b.tuning, step_samples=step, k5_ctas_per_sm=ctas)
    outs = b.render()
    torch.cuda.synchronize()
    for q, out in zip(small, outs):
        ref = oracle.render(_scene(vols, q), orc[q.volume])
        assert np.abs(_np(out) - ref).max() <= TOL_RGBA, (step, ctas, q.volume)


def test_graph_replay_eager_and_camera_update(ivv, pool):
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 6)
    b = _batch(ivv, gpu, small)
    eager = [o.clone() for o in b.render(flags=ivv.FLAG_TIMING)]
    assert not b.info()["graph_ready"]
    g1 = [o.clone() for o in b.render()]
    assert b.info()["graph_ready"]
    for o in b.outputs:
        o.fill_(-1.0)
    g2 = b.render()
    torch.cuda.synchronize()
    for x, y, z in zip(eager, g1, g2):
        assert torch.equal(x, y) and torch.equal(y, z)
    st = b.stage_times()
    assert all(v >= 0 for v in st.values()) and st["integrate"] > 0
    # a new camera for request 2 reaches the captured graph through the request table
    q = small[2]
    other = [r for r in reqs[12:] if r.volume == q.volume][0].camera
    keep = [o.clone() for o in g2]
    b.set_camera(2, other)
    outs = b.render()
    torch.cuda.synchronize()
    ref = oracle.render(dataclasses.replace(_scene(vols, q), camera=other), orc[q.volume])
    assert np.abs(_np(outs[2]) - ref).max() <= TOL_RGBA
    assert not torch.equal(outs[2], keep[2])
    for k in (0, 1, 3):
        assert torch.equal(outs[k], keep[k])


def test_camera_change_beyond_the_sample_buffer(ivv, pool):
    """The split integration's sample buffer is sized by the first render;
    zooming every camera in afterwards multiplies the samples, and the pixels
    that no longer fit are rendered by the fused integrator: the images still
    match the oracle, and the zoomed-out cameras render as before."""
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 4)
    b = _batch(ivv, gpu, small)
    first = [o.clone() for o in b.render()]
    torch.cuda.synchronize()
    zoomed = []
    for i, q in enumerate(small):
        c = q.camera
        eye = tuple(np.asarray(c.target) + (np.asarray(c.eye) - np.asarray(c.target)) / 3.0)
        cam = dataclasses.replace(c, eye=eye, ortho_height=c.ortho_height / 3.0)
        zoomed.append(cam)
        b.set_camera(i, cam)
    outs = b.render()
    torch.cuda.synchronize()
    for i, q in enumerate(small):
        ref = oracle.render(dataclasses.replace(_scene(vols, q), camera=zoomed[i]), orc[q.volume])
        assert np.abs(_np(outs[i]) - ref).max() <= TOL_RGBA, i
    for i, q in enumerate(small):
        b.set_camera(i, q.camera)
    again = b.render()
    torch.cuda.synchronize()
    for x, y in zip(first, again):
        assert torch.equal(x, y)


def test_autotune_picks_a_valid_shape(ivv, pool):
    vols, reqs, gpu, orc = pool
    small = _small(reqs, [(128, 96), (96, 128)], 6)
    b = _batch(ivv, gpu, small)
    best, ms = b.autotune(reps=1)
    assert (best["tile_w"], best["tile_h"]) in [(8, 4), (4, 8), (16, 2)]
    assert best["step_samples"] in (4, 8, 16) and 1 <= best["k5_ctas_per_sm"] <= 4
    assert ms > 0 and b.tuning == best and b.info()["graph_ready"]
    outs = b.render()
    torch.cuda.synchronize()
    q = small[0]
    ref = oracle.render(_scene(vols, q), orc[q.volume])
    assert np.abs(_np(outs[0]) - ref).max() <= TOL_RGBA


def test_batch_counters_add_up(ivv, pool):
    """The batch's rays, pairs and fragments are the sums over its requests
    rendered one by one; nothing overflows."""
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 9)
    b = _batch(ivv, gpu, small)
    b.reset_stats()
    b.render(flags=ivv.FLAG_STATS)
    s = b.stats()
    tot = {"rays": 0, "pairs": 0, "fragments": 0}
    for q in small:
        v = gpu[q.volume]
        v.set_transfer_function(q.tf)
        v.reset_stats()
        v.render(q.camera, scenes.RenderParams(), q.width, q.height, flags=ivv.FLAG_STATS)
        one = v.stats()
        for k in tot:
            tot[k] += one[k]
    for k, v in enumerate(gpu):
        v.set_transfer_function(vols[k].tf)
    for k in tot:
        assert s[k] == tot[k], (k, s[k], tot[k])
    assert s["abuf_overflow"] == 0 and s["pair_overflow"] == 0 and s["step_cap"] == 0
    assert s["rhs_evals"] >= 3 * (s["rk_steps"] + s["rk_rejects"]) + s["pairs"]


def test_batch_argument_errors(ivv, pool):
    vols, reqs, gpu, orc = pool
    q = reqs[0]
    item = (gpu[q.volume], q.camera, 32, 32, q.tf)
    with pytest.raises(ivv.IvvError, match="ODE"):
        ivv.Batch([item], scenes.RenderParams(method=1))
    with pytest.raises(ivv.IvvError, match="FP32 or MIXED"):
        ivv.Batch([item], scenes.RenderParams(precision=scenes.PRECISION_FP64))
    for rk in (1, 7):
        with pytest.raises(ivv.IvvError, match="BS3"):
            ivv.Batch([item], scenes.RenderParams(rk_method=rk))
    big = scenes.TransferFunction(np.linspace(0, 1, 65).astype(np.float32),
                                  np.full((65, 4), 0.5, np.float32), 4.0)
    with pytest.raises(ivv.IvvError, match="tf_n"):
        ivv.Batch([(gpu[q.volume], q.camera, 32, 32, big)])
    bad = torch.empty(32 * 32 * 4 + 1, dtype=torch.float32, device="cuda")[1:].view(32, 32, 4)
    with pytest.raises(ivv.IvvError, match="aligned"):
        ivv.Batch([item], outputs=[bad])
    b = ivv.Batch([item])
    with pytest.raises(ivv.IvvError):
        b.tuning = dict(b.tuning, tile_w=16, tile_h=8)
    with pytest.raises(ivv.IvvError):
        b.tuning = dict(b.tuning, step_samples=5)
    with pytest.raises(ivv.IvvError):
        b.set_camera(1, q.camera)
    # a quadratic volume cannot share a batch with the cubic ones
    quad = ivv.Volume([_quadratic_block()], scenes.SCALAR_CP)
    quad.set_transfer_function(q.tf)
    with pytest.raises(ivv.IvvError, match="common degree"):
        ivv.Batch([item, (quad, q.camera, 32, 32, None)])


def _quadratic_block():
    """One triquadratic Bezier block: a sheared, bulged unit cube (det J > 0)
    with a seeded scalar."""
    g = np.linspace(0.0, 1.0, 3)
    W, V, U = np.meshgrid(g, g, g, indexing="ij")
    cp = np.stack([U + 0.2 * V, V + 0.1 * np.sin(np.pi * U), W + 0.15 * U * V], axis=-1)
    kn = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    rho = np.random.default_rng(53).uniform(0, 1, (3, 3, 3))
    return scenes.Block((2, 2, 2), (kn, kn, kn), cp, rho)


def test_quadratic_batch_matches_oracle(ivv, pool):
    vols, reqs, gpu, orc = pool
    blk = _quadratic_block()
    sc = dataclasses.replace(vols[0], blocks=[blk], scalar_mode=scenes.SCALAR_CP, params=scenes.RenderParams())
    vol = ivv.volume_for(sc)
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(54)
    items, scs = [], []
    for k, (w, h) in enumerate([(40, 28), (23, 37)]):
        cam = scenes._ortho_camera_for(sc.blocks, rng)
        tf = scenes._random_tf(rng, 8, 4.0)
        items.append((vol, cam, w, h, tf))
        scs.append(dataclasses.replace(sc, camera=cam, tf=tf, width=w, height=h))
    b = ivv.Batch(items)
    outs = b.render()
    torch.cuda.synchronize()
    for s2, out in zip(scs, outs):
        ref = oracle.render(s2, ov)
        assert ref[..., 3].max() > 0.05
        assert np.abs(_np(out) - ref).max() <= TOL_RGBA


def test_mixed_precision_batch_matches_oracle(ivv, pool):
    vols, reqs, gpu, orc = pool
    small = _small(reqs, SIZES, 6)
    b = _batch(ivv, gpu, small, scenes.RenderParams(precision=scenes.PRECISION_MIXED))
    outs = b.render()
    torch.cuda.synchronize()
    for q, out in zip(small, outs):
        ref = oracle.render(_scene(vols, q), orc[q.volume])
        assert np.abs(_np(out) - ref).max() <= TOL_RGBA


def test_full_batched_workload_sampled(ivv, pool):
    """The 64-request workload at its own sizes (256^2 .. 1024^2): pixels
    sampled per request against the oracle, one by one; uneven pair counts."""
    vols, reqs, gpu, orc = pool
    b = _batch(ivv, gpu, reqs)
    info = b.info()
    assert info["n_requests"] == 64 and info["n_pixels"] == sum(q.width * q.height for q in reqs)
    b.render(flags=ivv.FLAG_STATS)
    s = b.stats()
    assert s["abuf_overflow"] == 0 and s["pair_overflow"] == 0
    assert s["pairs"] > s["rays"]                       # several pairs on some rays
    outs = b.render()
    torch.cuda.synchronize()
    rng = np.random.default_rng(52)
    worst = 0.0
    for q, out in zip(reqs, outs):
        img = out.cpu().numpy()
        cov = np.argwhere(img[..., 3] > 0)
        picks = [cov[rng.integers(len(cov))]] if len(cov) else []
        picks.append(np.array([rng.integers(q.height), rng.integers(q.width)]))
        sc = _scene(vols, q)
        for y, x in picks:
            ref = oracle.render(sc, orc[q.volume], window=(x, x + 1, y, y + 1), n_threads=1)[0, 0]
            worst = max(worst, np.abs(img[y, x].astype(np.float64) - ref).max())
    assert worst <= TOL_RGBA, worst


def test_full_batched_workload_rows(ivv, pool):
    """The 64-request workload at its own sizes: every 16th row of every
    request (from row 5) and its middle covered row, every pixel of them,
    against the oracle (silhouettes and grazing rays included, where random
    pixels rarely land)."""
    vols, reqs, gpu, orc = pool
    b = _batch(ivv, gpu, reqs)
    outs = b.render()
    torch.cuda.synchronize()
    worst, rows = 0.0, 0
    for i, (q, out) in enumerate(zip(reqs, outs)):
        img = out.cpu().numpy()
        cov = np.flatnonzero(img[..., 3].max(axis=1) > 0)
        ys = set(range(5, q.height, 16))
        if len(cov):
            ys.add(int(cov[len(cov) // 2]))
        for y in sorted(ys):
            ref = oracle.render(_scene(vols, q), orc[q.volume], window=(0, q.width, y, y + 1))[0]
            err = float(np.abs(img[y].astype(np.float64) - ref).max())
            assert err <= TOL_RGBA, (i, q.volume, q.width, y, err)
            worst = max(worst, err)
            rows += ref[:, 3].max() > 0
    assert rows > 600
