"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: images max |dRGBA| <= 1e-3; entry/exit parameters <= 1e-5
(pixels away from silhouettes; see the per-test notes); spline evaluation at
FP32 rounding of the control-point magnitudes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_RGBA = 1e-3
TOL_PARAM = 1e-5


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


def _gpu_image(ivv, sc, flags=0, window=None, width=None, height=None):
    vol = ivv.volume_for(sc)
    img = vol.render(sc.camera, sc.params, width or sc.width, height or sc.height, flags=flags, window=window)
    torch.cuda.synchronize()
    return vol, img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("cfg", [1, 2])
def test_eval_points_match_oracle(ivv, cfg):
    sc = scenes.config(cfg, width=8, height=8)
    vol = ivv.volume_for(sc)
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(50)
    P = rng.uniform(0, 1, (4096, 3)).astype(np.float32)
    for b in (0, len(sc.blocks) - 1):
        phi, J, rho = vol.eval_points(b, torch.from_numpy(P).cuda())
        f2, J2, r2 = ov.eval(b, P.astype(np.float64))
        scale = np.abs(f2).max()
        np.testing.assert_allclose(phi.cpu().numpy(), f2, atol=4e-6 * scale)
        np.testing.assert_allclose(J.cpu().numpy(), J2, atol=3e-6 * np.abs(J2).max())
        np.testing.assert_allclose(rho.cpu().numpy(), r2, atol=2e-5 * max(1.0, np.abs(r2).max()))


@pytest.mark.parametrize("cfg,size,prec", [(0, (64, 64), 0), (1, (200, 120), 0), (1, (200, 120), 1),
                                           (2, (160, 96), 1), (4, (160, 90), 1)])
def test_entry_exit_pairs_match_oracle(ivv, cfg, size, prec):
    """Stages 1-2 on the GPU: per pixel the oracle's pair count and block, and
    entry/exit parameters within 1e-5 (FP32: hits within 0.2 of grazing get
    2e-4; MIXED refines those in FP64 and is held to 1e-5 everywhere)."""
    from tests.test_library_cpu import compare_pairs
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = prec
    vol = ivv.volume_for(sc)
    cnt, pairs, blk = vol.render_pairs(sc.camera, sc.params, sc.width, sc.height, max_pairs=16)
    torch.cuda.synchronize()
    cnt, pairs, blk = cnt.cpu().numpy(), pairs.cpu().numpy().astype(np.float64), blk.cpu().numpy()
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    checked, worst = compare_pairs(ov, sc, cnt, pairs, blk, TOL_PARAM, graze_cos=0.2 if prec == 0 else -1.0)
    assert checked > 0.02 * sc.width * sc.height


@pytest.mark.parametrize("cfg,size,prec", [(0, (64, 64), 2), (0, (64, 64), 0), (1, (200, 120), 0),
                                           (1, (200, 120), 1), (2, (160, 96), 1), (4, (160, 90), 1)])
def test_image_matches_oracle(ivv, cfg, size, prec):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = prec
    vol, img = _gpu_image(ivv, sc)
    ref = oracle.render(sc)
    err = np.abs(img - ref).max()
    assert ref[..., 3].max() > 0.2, "workload renders something"
    assert err <= TOL_RGBA, err
    st = vol.stats()
    assert st["abuf_overflow"] == 0 and st["pair_overflow"] == 0 and st["step_cap"] == 0


@pytest.mark.parametrize("cfg,prec", [(1, 0), (1, 1), (2, 0), (2, 1)])
def test_full_frame_1080p_every_pixel(ivv, cfg, prec):
    """1920x1080 frames of the twisted bar and the bent beam in the
    benchmark's launch: every pixel against the oracle (element by element,
    background included)."""
    sc = scenes.config(cfg)
    sc.params.precision = prec
    vol, img = _gpu_image(ivv, sc)
    assert (img[..., 3] > 0).sum() > 10_000
    ref = oracle.render(sc)
    err = np.abs(img - ref)
    assert err.max() <= TOL_RGBA, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_full_frame_cube_1024_silhouette_sliver(ivv):
    """The twisted cube at 1024x1024 from a camera whose view grazes the edge
    where the top face bends over a side face (a sliver of the block a pixel
    wide): every pixel against the oracle."""
    import dataclasses
    vols, reqs = scenes.batch_requests()
    q = reqs[37]
    sc = dataclasses.replace(vols[q.volume], camera=q.camera, tf=q.tf, width=q.width, height=q.height,
                             params=scenes.RenderParams())
    for prec in (0, 1):
        sc.params.precision = prec
        vol, img = _gpu_image(ivv, sc)
        ref = oracle.render(sc)
        err = np.abs(img - ref)
        assert err.max() <= TOL_RGBA, (prec, err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("cfg,prec", [(1, 0), (1, 1)])
def test_full_frame_entry_exit_points(ivv, cfg, prec):
    """Entry/exit parameters of every pixel of the 1080p bar against the
    oracle's FP64 intersections: 1e-5 everywhere with the FP64 polish of the
    hits within |cos| < 0.35 of grazing (MIXED); plain FP32 within its
    rounding bound 4e-6 / |cos| (|cos| of the ray and the face normal; about
    1e-5 at |cos| = 0.4)."""
    sc = scenes.config(cfg)
    sc.params.precision = prec
    W, H = sc.width, sc.height
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    co, po, bo = ov.window_pairs(sc.camera, W, H)
    vol = ivv.volume_for(sc)
    cap = int(co.max())
    cg, pg, bg = vol.render_pairs(sc.camera, sc.params, W, H, max_pairs=cap)
    cg, pg, bg = cg.cpu().numpy(), pg.cpu().numpy().astype(np.float64), bg.cpu().numpy()
    diff = np.flatnonzero(cg != co)
    for q in diff:                       # only chords too short to contribute may differ
        short = [k for k in range(max(cg[q], co[q])) if
                 (k < co[q] and po[k, q, 7] - po[k, q, 3] < 1e-4 * ov.diag) or
                 (k < cg[q] and pg[k, q, 7] - pg[k, q, 3] < 1e-4 * ov.diag)]
        assert abs(int(cg[q]) - int(co[q])) <= len(short), (q, cg[q], co[q])
    same = cg == co
    eye = np.asarray(sc.camera.eye, float)
    checked = 0
    for k in range(cap):
        m = same & (co > k)
        assert (bg[k][m] == bo[k][m]).all()
        for a in (0, 4):
            got, ref = pg[k][m][:, a:a + 3], po[k][m][:, a:a + 3]
            e = np.abs(got - ref).max(axis=1)
            assert np.abs(pg[k][m][:, a + 3] - po[k][m][:, a + 3]).max() <= 2e-4
            if prec == 1:
                assert e.max() <= TOL_PARAM, e.max()
            else:
                cosg = np.ones(len(e))
                for blk in np.unique(bo[k][m]):
                    q = bo[k][m] == blk
                    phi, J, _ = ov.eval(int(blk), ref[q])
                    face = np.argmin(np.minimum(np.abs(ref[q]), np.abs(ref[q] - 1)), axis=1)
                    nrm = np.linalg.inv(J)[np.arange(int(q.sum())), face]
                    d = phi - eye
                    cosg[q] = np.abs((nrm * d).sum(1)) / (np.linalg.norm(nrm, axis=1) * np.linalg.norm(d, axis=1))
                bound = 4e-6 / np.maximum(cosg, 0.02)
                assert (e <= bound).all(), (e / bound).max()
                if (cosg >= 0.4).any():
                    assert e[cosg >= 0.4].max() <= TOL_PARAM, e[cosg >= 0.4].max()
            checked += len(e)
    assert checked > 200_000


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_4k_backstep_every_8th_row(ivv, prec):
    """3840x2160 backward-facing step (the frame whose sample list is sized
    from the exact scanned total, read back once): every pixel of every 8th
    row against the oracle -- the rows the benchmark checks, which cross the
    shear layer where the integration tolerance decides the error -- and the
    split path's counters."""
    sc = scenes.config(4)
    sc.params.precision = prec
    vol, img = _gpu_image(ivv, sc)
    vol.reset_stats()
    vol.render(sc.camera, sc.params, sc.width, sc.height, flags=ivv.FLAG_STATS)
    st = vol.stats()
    assert st["rho_evals"] == st["samples"] > 10_000_000          # the split integration ran
    assert st["abuf_overflow"] == 0 and st["pair_overflow"] == 0 and st["step_cap"] == 0
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    worst = 0.0
    for y in range(4, sc.height, 8):
        ref = oracle.render(sc, ov, window=(0, sc.width, y, y + 1))[0]
        worst = max(worst, np.abs(img[y] - ref).max())
    assert worst <= TOL_RGBA, worst


def test_window_equals_crop_and_is_deterministic(ivv):
    sc = scenes.config(1, width=200, height=120)
    vol = ivv.volume_for(sc)
    full = vol.render(sc.camera, sc.params, 200, 120).clone()
    again = vol.render(sc.camera, sc.params, 200, 120).clone()
    assert torch.equal(full, again)
    win = vol.render(sc.camera, sc.params, 37, 29, window=(81, 45, 200, 120))
    torch.cuda.synchronize()
    assert torch.equal(win, full[45:74, 81:118])


def test_ragged_and_tiny_images(ivv):
    for (w, h) in [(1, 1), (17, 13), (33, 1), (5, 71)]:
        sc = scenes.config(0, width=w, height=h)
        sc.params.precision = 0
        _, img = _gpu_image(ivv, sc)
        ref = oracle.render(sc)
        assert np.abs(img - ref).max() <= TOL_RGBA, (w, h)


def test_empty_view_is_zero(ivv):
    sc = scenes.config(1, width=96, height=64)
    cam = sc.camera
    # look away from the bar
    t = np.array(cam.target)
    e = np.array(cam.eye)
    sc.camera = scenes.Camera(False, tuple(e), tuple(2 * e - t), cam.up, fovy_deg=30.0)
    vol, img = _gpu_image(ivv, sc)
    assert np.abs(img).max() == 0.0
    assert vol.stats()["rays"] == 0


def test_constant_density_closed_form(ivv):
    """Affine box, constant scalar: alpha = 1 - exp(-sigma A L) per pixel."""
    from tests.test_oracle_bspline import _affine_block
    from tests.test_oracle_intersect import _slab
    rng = np.random.default_rng(52)
    blk, A, b = _affine_block(rng)
    blk.scalar_cp = np.full(blk.geom_cp.shape[:3], 0.3)
    col = np.array([0.25, 0.5, 0.625, 0.75])
    tf = scenes.TransferFunction(np.array([0, 1], np.float32), np.array([col, col], np.float32), 1.5,
                                 lo=0.0, hi=1.0)
    centre = b + A @ np.full(3, 0.5)
    cam = scenes.Camera(False, tuple(centre + np.array([3.0, 1.0, 2.0])), tuple(centre), (0, 0, 1), fovy_deg=40.0)
    sc = scenes.Scene("box", [blk], scenes.SCALAR_CP, tf, cam, 48, 40,
                      scenes.RenderParams(ds=0.05, early_alpha=2.0))
    _, img = _gpu_image(ivv, sc)
    for y in range(40):
        for x in range(48):
            o, d = oracle.ray(cam, 48, 40, x, y)
            ref = _slab(A, b, o, d)
            L = 0.0 if ref is None else ref[1] - ref[0]
            a = 1 - math.exp(-1.5 * col[3] * L)
            assert abs(img[y, x, 3] - a) <= 1e-4, (x, y, img[y, x, 3], a)


def test_stats_and_timing(ivv):
    sc = scenes.config(1, width=200, height=120)
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    vol.render(sc.camera, sc.params, 200, 120, flags=ivv.FLAG_STATS | ivv.FLAG_TIMING)
    st = vol.stats()
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    ref, rs = oracle.render(sc, ov, stats=True)
    assert abs(st["rays"] - (rs[..., 0] > 0).sum()) <= 3
    assert abs(st["samples"] - rs[..., 3].sum()) <= 0.01 * rs[..., 3].sum()
    # every accepted or rejected step costs three right-hand sides; pair starts
    # and dense-output samples add one each
    assert st["rhs_evals"] >= 3 * (st["rk_steps"] + st["rk_rejects"]) + st["pairs"]
    assert st["rk_steps"] > 0
    assert 0 < st["max_delta_p"] <= 1.0          # pixel accuracy, Eq. 5
    t = vol.stage_times()
    assert set(t) == {"project", "intersect", "pair", "integrate"} and all(v >= 0 for v in t.values())


def test_render_to_host_async_pipeline(ivv):
    """Frames queued with render_to_host_async (each copy overlapping the next
    render, two device images used in turn, grown when the window grows)
    equal the blocking render_to_host frame by frame once wait_host returns."""
    import dataclasses
    sc = scenes.config(1, width=96, height=64)
    vol = ivv.volume_for(sc)
    cams = [sc.camera, dataclasses.replace(sc.camera, eye=tuple(1.1 * e for e in sc.camera.eye))]
    sizes = [(96, 64), (96, 64), (128, 80), (96, 64), (128, 80), (128, 80)]
    refs = []
    for i, (w, h) in enumerate(sizes):
        ref = np.zeros((h, w, 4), np.float32)
        vol.render_to_host(cams[i % 2], sc.params, w, h, ref)
        refs.append(ref)
    outs = []
    for i, (w, h) in enumerate(sizes):
        out = torch.full((h, w, 4), float("nan"), dtype=torch.float32).pin_memory()
        vol.render_to_host_async(cams[i % 2], sc.params, w, h, out)
        outs.append(out)
    vol.wait_host()
    for i, (ref, out) in enumerate(zip(refs, outs)):
        got = out.numpy()
        assert not np.isnan(got).any(), i
        assert np.abs(got - ref).max() <= 1e-5, i
    assert max(r[..., 3].max() for r in refs) > 0.05


def test_render_to_host_and_errors(ivv):
    sc = scenes.config(0, width=40, height=30)
    sc.params.precision = 0
    vol = ivv.volume_for(sc)
    host = np.zeros((30, 40, 4), np.float32)
    vol.render_to_host(sc.camera, sc.params, 40, 30, host)
    dev = vol.render(sc.camera, sc.params, 40, 30)
    assert np.array_equal(host, dev.cpu().numpy())
    with pytest.raises(ivv.IvvError) as e:
        vol.render(sc.camera, sc.params, 0, 30)
    assert e.value.status == 1
    with pytest.raises(ivv.IvvError) as e:
        vol.render(sc.camera, sc.params, 40, 30, window=(10, 10, 40, 30))   # window outside the image
    assert e.value.status == 1
    bad = scenes.Camera(False, sc.camera.eye, sc.camera.eye, sc.camera.up)
    with pytest.raises(ivv.IvvError):
        vol.render(bad, sc.params, 40, 30)
    # windows beyond 2^27 pixels are refused before any allocation
    import ctypes as C
    L = ivv.load()
    cam = ivv.camera_struct(sc.camera)
    prm = ivv.params_struct(sc.params, 0, None)
    need = C.c_size_t()
    assert L.ivv_workspace_size(vol.h, 20000, 20000, 0, C.byref(need)) == 1
    assert L.ivv_render(vol.h, C.byref(cam), C.byref(prm), 20000, 20000, C.c_void_p(dev.data_ptr()), None, 0,
                        None) == 1
    assert "2^27" in L.ivv_last_error().decode()
