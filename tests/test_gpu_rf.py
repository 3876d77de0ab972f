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


def test_learned_guess_gains_over_plain_newton(ivv):
    sc = scenes.config(1, width=200, height=120)
    sc.params.precision = scenes.PRECISION_FP32
    sc.params.rf_tol = 1e-3
    vol = ivv.volume_for(sc)
    losses = vol.train_guess(samples_per_block=1 << 17, epochs=24, batch=2048, lr=3e-3, seed=3)
    assert losses[0] < 1e-4
    ref = oracle.render(sc)
    iters = {}
    for guess in (ivv.GUESS_CENTER, ivv.GUESS_MLP, ivv.GUESS_CHORD):
        vol.reset_stats()
        img = _render(ivv, vol, sc, ivv.METHOD_RF, guess, flags=ivv.FLAG_STATS)
        st = vol.stats()
        assert np.abs(img - ref).max() <= TOL_RGBA, guess
        assert st["rf_unconverged"] <= 0.001 * st["samples"], (guess, st["rf_unconverged"])
        iters[guess] = st["rf_newton_iters"] / max(1, st["samples"])
    # fewer Newton iterations per sample than from the block centre
    assert iters[ivv.GUESS_MLP] < 0.6 * iters[ivv.GUESS_CENTER], iters
