"""Failure statuses of the render (the overflow and cap paths), through the
C ABI: capacities shrunk with ivv_set_limits make fragments, candidates and
pairs overflow and iterations hit their caps; every case must return its
status from ivv_check_frame, never fault, and leave the pixels that the
shrunk capacity does not touch exactly as the default render has them."""
import dataclasses

import numpy as np
import pytest

from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ABUF_OVERFLOW, NONCONVERGED = 4, 5


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


def _render(vol, sc):
    img = vol.render(sc.camera, sc.params, sc.width, sc.height)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def test_default_limits_report_ok(ivv):
    sc = scenes.config(2, width=160, height=96)
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    _render(vol, sc)
    assert vol.check_frame() == (0, "")
    assert vol.limits() == {"max_frags": 32, "max_pairs": 16, "items_per_pixel": 16, "max_rk_steps": 200000,
                            "max_newton": 16}


def test_pair_overflow_keeps_single_pair_pixels(ivv):
    """The bent beam has rays through several blocks: with one pair slot the
    pixels of one pair render as before and the frame reports the drops."""
    sc = scenes.config(2, width=160, height=96)
    vol = ivv.volume_for(sc)
    ref = _render(vol, sc)
    cnt, _, _ = vol.render_pairs(sc.camera, sc.params, sc.width, sc.height)
    cnt = cnt.cpu().numpy().reshape(sc.height, sc.width)
    assert (cnt > 1).sum() > 100 and (cnt == 1).sum() > 100
    vol.reset_stats()
    vol.set_limits(max_pairs=1)
    img = _render(vol, sc)
    st, msg = vol.check_frame()
    assert st == ABUF_OVERFLOW and "pair" in msg, (st, msg)
    assert vol.stats()["pair_overflow"] > 0
    assert np.isfinite(img).all()
    np.testing.assert_array_equal(img[cnt <= 1], ref[cnt <= 1])
    assert np.abs(img[cnt > 1] - ref[cnt > 1]).max() > 1e-3      # the dropped pairs are missing
    vol.set_limits()
    np.testing.assert_array_equal(_render(vol, sc), ref)
    assert vol.check_frame()[0] == 0                              # nothing new since the last check


@pytest.mark.parametrize("field", ["max_frags", "items_per_pixel"])
def test_fragment_and_candidate_overflow(ivv, field):
    """One fragment slot, or one stage-1 candidate per pixel of the window
    (the twisted cube zoomed to fill the window: every ray meets at least
    two face patches)."""
    sc = scenes.config(0, width=64, height=64)
    sc.camera = dataclasses.replace(sc.camera, ortho_height=0.35 * sc.camera.ortho_height)
    vol = ivv.volume_for(sc)
    ref = _render(vol, sc)
    vol.reset_stats()
    vol.set_limits(**{field: 1})
    img = _render(vol, sc)
    st, msg = vol.check_frame()
    assert st == ABUF_OVERFLOW, (st, msg)
    assert vol.stats()["abuf_overflow"] > 0
    assert np.isfinite(img).all() and img.min() >= 0 and img[..., 3].max() <= 1.0
    assert (ref[..., 3] > 0).mean() > 0.9
    bg = ref[..., 3] == 0
    assert (img[bg] == 0).all()                                   # background untouched
    vol.set_limits()
    np.testing.assert_array_equal(_render(vol, sc), ref)


def test_rk_step_cap(ivv):
    sc = scenes.config(1, width=120, height=72)
    vol = ivv.volume_for(sc)
    ref = _render(vol, sc)
    vol.reset_stats()
    vol.set_limits(max_rk_steps=1)
    img = _render(vol, sc)
    st, msg = vol.check_frame()
    assert st == NONCONVERGED and "step cap" in msg, (st, msg)
    assert vol.stats()["step_cap"] > 0
    assert np.isfinite(img).all() and img[..., 3].max() <= 1.0
    bg = ref[..., 3] == 0
    assert (img[bg] == 0).all()
    vol.set_limits()
    np.testing.assert_array_equal(_render(vol, sc), ref)


def test_rf_newton_cap(ivv):
    sc = scenes.config(1, width=120, height=72)
    sc.params = dataclasses.replace(sc.params, method=1, use_mlp_guess=0)
    vol = ivv.volume_for(sc)
    vol.reset_stats()
    _render(vol, sc)
    assert vol.check_frame()[0] == 0
    sc.params = dataclasses.replace(sc.params, rf_tol=1e-4)
    vol.set_limits(max_newton=1)
    img = _render(vol, sc)
    st, msg = vol.check_frame()
    assert st == NONCONVERGED and "RF" in msg, (st, msg)
    assert np.isfinite(img).all()


def test_limits_are_validated(ivv):
    sc = scenes.config(0, width=16, height=16)
    vol = ivv.volume_for(sc)
    for bad in ({"max_frags": 0}, {"max_frags": 33}, {"max_pairs": 17}, {"items_per_pixel": 0},
                {"max_rk_steps": 0}, {"max_newton": 65}):
        with pytest.raises(ivv.IvvError) as e:
            vol.set_limits(**bad)
        assert e.value.status == 1
    assert vol.limits()["max_frags"] == 32
