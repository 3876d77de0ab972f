"""The learned initial guess on the render path, through the C ABI.

Stage 2's fix-up solves that have no chord context -- entries on the near
plane (§5.5) and entries moved off a singular face (§5.4) -- start Newton
from the block's trained network when use_mlp_guess = IVV_GUESS_MLP.  The
images must equal the oracle's (which starts those solves from the plain
guesses: the preimage is unique) within 1e-3, and the counters show what the
learned guess gains: Newton iterations of the fix-up solves against the plain
starts (the exit point of the block for a near-plane entry, Eq. 22's x_0 with
its fallbacks for a singular entry).  Measured: on near-plane entries of the
twisted bar no gain (about three iterations either way); on the singular
entries of the degenerate-face cube half the iterations."""
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


def _render(ivv, vol, sc, guess):
    prm = dataclasses.replace(sc.params, use_mlp_guess=guess)
    vol.reset_stats()
    img = vol.render(sc.camera, prm, sc.width, sc.height, flags=ivv.FLAG_STATS)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), vol.stats()


@pytest.mark.parametrize("prec", [0, 1])
def test_near_plane_entries_from_the_learned_guess(ivv, prec):
    """The twisted bar seen along its axis with the near plane through its
    middle: every covered ray enters on the plane, and the plain start (the
    block's exit point) lies half the bar's length further on."""
    sc = scenes.config(1, width=240, height=136)
    sc.camera = scenes.Camera(False, (0.62, 0.55, -5.0), (0.5, 0.5, 4.0), (0.0, 1.0, 0.0), fovy_deg=20.0)
    sc.params = dataclasses.replace(sc.params, near_clip=9.0, precision=prec)
    vol = ivv.volume_for(sc)
    losses = vol.train_guess(samples_per_block=1 << 17, epochs=16, batch=2048, lr=3e-3, seed=5)
    assert max(losses) < 5e-3, losses
    ref = oracle.render(sc)
    assert ref[..., 3].max() > 0.1
    plain, sp = _render(ivv, vol, sc, ivv.GUESS_CENTER)
    learned, sl = _render(ivv, vol, sc, ivv.GUESS_MLP)
    assert np.abs(plain - ref).max() <= TOL_RGBA
    assert np.abs(learned - ref).max() <= TOL_RGBA
    assert sl["unmatched"] == sp["unmatched"]
    print("near-plane entries: fix-up Newton iterations plain %d, learned %d" % (sp["entry_newton"], sl["entry_newton"]))
    assert sp["entry_newton"] > 1000
    # Newton from the exit point already converges in about three
    # iterations here (the bar's map is nearly linear along its axis): the
    # learned start may not cost more
    assert sl["entry_newton"] <= 1.1 * sp["entry_newton"], (sp["entry_newton"], sl["entry_newton"])


def test_singular_entries_from_the_learned_guess(ivv):
    """Degenerate-face cube: Eq. 22's x_0 lies next to the singular face,
    where Newton on the cubic collapse overshoots; the learned guess lands on
    the far side of the root, from which Newton converges monotonically."""
    sc = scenes.degenerate_cube(width=160, height=160)
    sc.params.precision = 1
    vol = ivv.volume_for(sc)
    vol.train_guess(samples_per_block=1 << 17, epochs=16, batch=2048, lr=3e-3, seed=6)
    ref = oracle.render(sc)
    plain, sp = _render(ivv, vol, sc, ivv.GUESS_CENTER)
    learned, sl = _render(ivv, vol, sc, ivv.GUESS_MLP)
    assert np.abs(plain - ref).max() <= TOL_RGBA
    assert np.abs(learned - ref).max() <= TOL_RGBA
    assert sl["entry_shrinks"] == sp["entry_shrinks"] > 1000
    print("singular entries: fix-up Newton iterations plain %d, learned %d" % (sp["entry_newton"], sl["entry_newton"]))
    assert sl["entry_newton"] < 0.8 * sp["entry_newton"], (sp["entry_newton"], sl["entry_newton"])


def test_learned_guess_needs_a_trained_network(ivv):
    sc = scenes.config(0, width=16, height=16)
    sc.params.use_mlp_guess = 1
    vol = ivv.volume_for(sc)
    with pytest.raises(ivv.IvvError) as e:
        vol.render(sc.camera, sc.params, 16, 16)
    assert e.value.status == 1
