"""ivv_render_noalloc: rendering a small window with no device allocation.

Some callers cannot allocate device memory while they render: hosts whose
GPU memory is owned by their own pool or budget, and real-time threads that
must not risk the synchronisation an allocation may bring.  The allocation-free entry point
keeps the frame's workspace in a fixed device array inside the library; its
image must equal the one ivv_render produces with a caller workspace, on
consecutive calls (the array keeps the previous call's contents, so anything
a frame needs cleared must be cleared by that frame).

This file is collected last so that a failure here never hides the result of
another test in a run that stops at the first failure.
"""
import dataclasses

import pytest

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


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _check_noalloc(ivv, sc):
    vol = ivv.volume_for(sc)
    ref = vol.render(sc.camera, sc.params, sc.width, sc.height).clone()
    torch.cuda.synchronize()
    assert ref[..., 3].max().item() > 0.05, "the window shows the volume"
    outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
    vol.render_noalloc(sc.camera, sc.params, sc.width, sc.height, outs[0])   # first call on this device
    free0 = _free_bytes()
    for call, out in enumerate(outs):
        out.fill_(float("nan"))
        vol.render_noalloc(sc.camera, sc.params, sc.width, sc.height, out)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= TOL_RGBA, (call, err)
    assert _free_bytes() == free0, "ivv_render_noalloc changed the device memory in use"
    vol.close()


@pytest.mark.parametrize("cfg,size,prec", [(0, (48, 40), 0), (1, (64, 48), 0), (2, (40, 64), 1), (0, (32, 32), 2)])
def test_noalloc_matches_render_on_consecutive_calls(ivv, cfg, size, prec):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = prec
    _check_noalloc(ivv, sc)


@pytest.mark.parametrize("rk_method", range(1, 8))
def test_noalloc_fixed_step_and_implicit_integrators(ivv, rk_method):
    sc = scenes.config(1, width=64, height=48)
    sc.params = dataclasses.replace(sc.params, rk_method=rk_method, c=100.0 if rk_method == 7 else 1.0)
    _check_noalloc(ivv, sc)


def test_noalloc_rejects_rf_method(ivv):
    sc = scenes.config(0, width=32, height=32)
    sc.params.method = 1
    vol = ivv.volume_for(sc)
    out = torch.empty((32, 32, 4), dtype=torch.float32, device="cuda")
    free0 = _free_bytes()
    with pytest.raises(ivv.IvvError) as e:
        vol.render_noalloc(sc.camera, sc.params, 32, 32, out)
    assert e.value.status == 7 and "ODE method" in str(e.value)
    assert _free_bytes() == free0


def test_noalloc_rejects_oversized_window(ivv):
    sc = scenes.config(1, width=1920, height=1080)
    vol = ivv.volume_for(sc)
    out = torch.empty((1080, 1920, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ivv.IvvError) as e:
        vol.render_noalloc(sc.camera, sc.params, 1920, 1080, out)
    assert e.value.status == 8 and "bytes of scratch" in str(e.value)
