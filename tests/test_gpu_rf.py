"""Root-finding ray integration (§5.1) on the GPU, batched over all samples,
and what the learned initial guess gains over the plain guesses.

Images from every initial guess must match the oracle within 1e-3; the
learned guess must need markedly fewer Newton iterations than Newton from the
block's parameter centre (the plain fallback) on the same samples."""
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


def _render(ivv, vol, sc, method, guess, flags=0):
    sc.params.method = method
    sc.params.use_mlp_guess = guess
    img = vol.render(sc.camera, sc.params, sc.width, sc.height, flags=flags)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("cfg,size", [(0, (64, 64)), (1, (200, 120)), (2, (160, 96)), (4, (160, 90))])
def test_rf_images_match_oracle(ivv, cfg, size):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = scenes.PRECISION_FP32
    sc.params.rf_tol = 1e-3          # 1e-3 of a pixel half width: image parity, not only pixel accuracy
    vol = ivv.volume_for(sc)
    ref = oracle.render(sc)
    for guess in (ivv.GUESS_CHORD, ivv.GUESS_CENTER):
        img = _render(ivv, vol, sc, ivv.METHOD_RF, guess)
        err = np.abs(img - ref).max()
        assert err <= TOL_RGBA, (guess, err)


def test_learned_guess_renders_the_same_image(ivv):
    sc = scenes.config(0, width=64, height=64)
    sc.params.precision = scenes.PRECISION_FP32
    sc.params.rf_tol = 1e-3
    vol = ivv.volume_for(sc)
    vol.train_guess(samples_per_block=1 << 16, epochs=16, batch=2048, lr=3e-3, seed=3)
    ref = oracle.render(sc)
    vol.reset_stats()
    img = _render(ivv, vol, sc, ivv.METHOD_RF, ivv.GUESS_MLP, flags=ivv.FLAG_STATS)
    assert np.abs(img - ref).max() <= TOL_RGBA
    assert vol.stats()["rf_unconverged"] == 0


@pytest.mark.parametrize("cfg", [0, 2])
def test_learned_guess_gains_over_plain_newton(ivv, cfg):
    """Locating interior world points (Eq. 6 per point): Newton from the
    learned guess against plain Newton from the block's parameter centre.
    Both must reach the same preimages; the learned guess must need clearly
    fewer iterations and less time."""
    sc = scenes.config(cfg, width=8, height=8)
    vol = ivv.volume_for(sc)
    losses = vol.train_guess(samples_per_block=1 << 17, epochs=24, batch=2048, lr=3e-3, seed=4)
    assert max(losses) < 2e-3, losses
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(80 + cfg)
    nb = len(sc.blocks)
    n_per = 65536 // nb
    P = rng.uniform(0.02, 0.98, (nb * n_per, 3))
    blk = np.repeat(np.arange(nb), n_per).astype(np.int32)
    G = np.concatenate([ov.eval(b, P[b * n_per:(b + 1) * n_per])[0] for b in range(nb)])
    g4 = torch.zeros((len(P), 4), dtype=torch.float32, device="cuda")
    g4[:, :3] = torch.from_numpy(G.astype(np.float32)).cuda()
    bt = torch.from_numpy(blk).cuda()
    tol = 1e-5 * ov.diag
    res = {}
    for guess in (ivv.GUESS_CENTER, ivv.GUESS_MLP):
        vol.invert_points(g4, bt, guess, tol)          # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p, its = vol.invert_points(g4, bt, guess, tol)
        e1.record()
        torch.cuda.synchronize()
        its = its.cpu().numpy()
        p = p.cpu().numpy()[:, :3]
        ok = its >= 0
        assert ok.mean() > 0.995, (guess, ok.mean())
        assert np.abs(p[ok] - P[ok]).max() < 2e-4, guess
        res[guess] = (its[ok].mean(), e0.elapsed_time(e1))
    print("workload", cfg, "Newton iterations / ms  centre:", res[ivv.GUESS_CENTER], " learned:", res[ivv.GUESS_MLP])
    assert res[ivv.GUESS_MLP][0] < 0.75 * res[ivv.GUESS_CENTER][0], res


@pytest.mark.parametrize("cfg,prec,guess", [(1, 0, 2), (2, 0, 2), (2, 1, 1)],
                         ids=["bar-chord-fp32", "beam-chord-fp32", "beam-learned-mixed"])
def test_full_frame_1080p_every_pixel(ivv, cfg, prec, guess):
    """The benchmark's root-finding frames at 1920x1080 (rf_tol 1e-3 of the
    pixel half width): the chord guess in FP32, and on the beam the learned
    guess (trained as the benchmark trains it) with mixed precision; every
    pixel against the oracle."""
    sc = scenes.config(cfg)
    sc.params.precision = prec
    sc.params.rf_tol = 1e-3
    vol = ivv.volume_for(sc)
    if guess == 1:
        vol.train_guess(samples_per_block=1 << 20, epochs=8, batch=4096, lr=3e-3, seed=1)
    vol.reset_stats()
    img = _render(ivv, vol, sc, 1, guess, flags=ivv.FLAG_STATS)
    st = vol.stats()
    assert (img[..., 3] > 0).sum() > 10_000
    assert st["rf_unconverged"] <= 1e-4 * st["samples"], (st["rf_unconverged"], st["samples"])
    ref = oracle.render(sc)
    err = np.abs(img - ref)
    assert err.max() <= TOL_RGBA, (err.max(), np.unravel_index(err.argmax(), err.shape))
    vol.close()
