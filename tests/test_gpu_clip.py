"""Cutting and near-clip planes (§5.5) on the GPU against the oracle
(max |dRGBA| <= 1e-3), through the C ABI: an affine box (closed forms in the
oracle pins), the eye inside the box, the twisted bar and cube in FP32,
mixed and FP64, with the RF method and a fixed-step integrator, and the
clipped entry/exit points on their plane."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1404_3363_gb300 import scenes
from tests.test_oracle_clip import _box_scene

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


def _gpu(ivv, sc):
    vol = ivv.volume_for(sc)
    img = vol.render(sc.camera, sc.params, sc.width, sc.height)
    torch.cuda.synchronize()
    return vol, img.cpu().numpy().astype(np.float64)


def _plane_through(point, n):
    n = np.asarray(n, float)
    n = n / np.linalg.norm(n)
    return (n[0], n[1], n[2], -float(n @ np.asarray(point)))


def test_cutting_planes_on_an_affine_box(ivv):
    rng = np.random.default_rng(60)
    sc, A, b = _box_scene(rng, (1.6, 0.6, 1.1), fovy=55.0)
    centre = b + A @ np.full(3, 0.5)
    for planes in [(_plane_through(centre + 0.1 * A @ np.ones(3), (0.3, -0.8, 0.52)),),
                   (_plane_through(centre, (1.0, 0.2, 0.0)), _plane_through(centre, (-0.1, 0.3, -1.0)))]:
        sc.params.cut_planes = planes
        _, img = _gpu(ivv, sc)
        ref = oracle.render(sc)
        assert ref[..., 3].max() > 0.1
        assert np.abs(img - ref).max() <= TOL_RGBA


def test_near_plane_with_the_eye_inside_the_box(ivv):
    rng = np.random.default_rng(62)
    sc, A, b = _box_scene(rng, (0.05, 0.02, -0.03), fovy=60.0, near_clip=0.15)
    _, img = _gpu(ivv, sc)
    ref = oracle.render(sc)
    assert (ref[..., 3] > 0).all()
    assert np.abs(img - ref).max() <= TOL_RGBA
    # without the near plane the rays that start inside the box see nothing
    sc.params.near_clip = 0.0
    _, img0 = _gpu(ivv, sc)
    assert np.abs(img0).max() == 0.0


@pytest.mark.parametrize("cfg,size,prec,method,rk", [(1, (120, 72), 0, 0, 0), (1, (120, 72), 1, 0, 0),
                                                     (1, (120, 72), 0, 1, 0), (1, (120, 72), 0, 0, 4),
                                                     (0, (48, 48), 2, 0, 0), (2, (96, 60), 1, 0, 0)])
def test_cutting_plane_and_near_plane_on_curved_volumes(ivv, cfg, size, prec, method, rk):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    lo, hi = sc.cp_bbox()
    centre = 0.5 * (lo + hi)
    eye = np.asarray(sc.camera.eye)
    dist = np.linalg.norm(np.asarray(sc.camera.target) - eye)
    sc.params = dataclasses.replace(sc.params, precision=prec, method=method, rk_method=rk,
                                    rf_tol=1e-3 if method == 1 else sc.params.rf_tol,
                                    cut_planes=(_plane_through(centre + 0.07 * (hi - lo), (0.2, 0.5, 1.0)),),
                                    near_clip=dist - 0.1 * np.linalg.norm(hi - lo))
    _, img = _gpu(ivv, sc)
    ref = oracle.render(sc)
    full = oracle.render(dataclasses.replace(sc, params=dataclasses.replace(sc.params, cut_planes=(),
                                                                            near_clip=0.0)))
    assert np.abs(ref - full).max() > 0.05, "the planes change the image"
    assert ref[..., 3].max() > 0.05
    err = np.abs(img - ref).max()
    assert err <= TOL_RGBA, (cfg, prec, method, rk, err)


def test_clipped_ends_lie_on_the_plane(ivv):
    sc = scenes.config(1, width=120, height=72)
    lo, hi = sc.cp_bbox()
    pl = _plane_through(0.5 * (lo + hi), (0.0, 0.3, 1.0))
    sc.params.cut_planes = (pl,)
    vol = ivv.volume_for(sc)
    cnt, pairs, blk = vol.render_pairs(sc.camera, sc.params, sc.width, sc.height, max_pairs=16)
    torch.cuda.synchronize()
    cnt, pairs = cnt.cpu().numpy(), pairs.cpu().numpy().astype(np.float64)
    n = np.asarray(pl[:3])
    on_plane, pts = 0, []
    for pix in np.nonzero(cnt)[0]:
        x, y = pix % sc.width, pix // sc.width
        o, d = oracle.ray(sc.camera, sc.width, sc.height, x, y)
        for q in range(cnt[pix]):
            for base in (0, 4):
                t = pairs[q, pix, base + 3]
                g = o + t * d
                assert n @ g + pl[3] <= 1e-4                       # on the kept side
                if abs(n @ g + pl[3]) < 1e-4:
                    on_plane += 1
                    pts.append((pairs[q, pix, base:base + 3], g))
    assert on_plane > 20
    P = torch.tensor(np.array([p for p, _ in pts]), dtype=torch.float32, device="cuda")
    phi, _, _ = vol.eval_points(0, P)
    G = np.array([g for _, g in pts])
    assert np.abs(phi.cpu().numpy() - G).max() < 2e-4 * np.linalg.norm(hi - lo)


def test_batch_rejects_clipping(ivv):
    vols, reqs = scenes.batch_requests()
    q = reqs[0]
    v = ivv.volume_for(vols[q.volume])
    with pytest.raises(ivv.IvvError, match="cutting or near-clip"):
        ivv.Batch([(v, q.camera, 32, 32, q.tf)], scenes.RenderParams(near_clip=1.0))


def test_clip_argument_errors(ivv):
    sc = scenes.config(1, width=16, height=16)
    vol = ivv.volume_for(sc)
    for bad in [dict(near_clip=-1.0), dict(cut_planes=((0.0, 0.0, 0.0, 1.0),)),
                dict(cut_planes=((float("nan"), 0.0, 1.0, 0.0),))]:
        with pytest.raises(ivv.IvvError):
            vol.render(sc.camera, dataclasses.replace(sc.params, **bad), 16, 16)


@pytest.mark.parametrize("cfg,method", [(1, 0), (2, 0), (2, 1)])
def test_sample_lists_counted_by_k4_or_after_the_fix_ups(ivv, cfg, method):
    """Without planes K4 counts each pixel's samples into the sample lists;
    with a plane the counts run after the fix-up solves.  A near plane just
    in front of the eye moves no pair end, so both routes see the same pairs
    and must give the same image, value for value (split ODE integration and
    per-sample root finding)."""
    sc = scenes.config(cfg, width=200, height=120)
    sc.params.method = method
    if method == 1:
        sc.params.use_mlp_guess = 2
        sc.params.rf_tol = 1e-3
    vol = ivv.volume_for(sc)
    a = vol.render(sc.camera, sc.params, sc.width, sc.height).clone()
    near = dataclasses.replace(sc.params, near_clip=1e-4)
    b = vol.render(sc.camera, near, sc.width, sc.height)
    torch.cuda.synchronize()
    assert a[..., 3].max().item() > 0.1
    assert torch.equal(a, b), (a - b).abs().max().item()
    vol.close()
