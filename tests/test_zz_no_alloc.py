"""ivv_render_noalloc: rendering a small window with no device allocation.

Some callers cannot allocate device memory while they render: a CUDA graph
being recorded (allocation cannot be captured), hosts whose GPU memory is
owned by their own pool or budget, and real-time threads that must not risk
the synchronisation an allocation may bring.  The allocation-free entry point
keeps the frame's workspace in a fixed device array inside the library; its
image must equal the one ivv_render produces with a caller workspace, on
consecutive calls (the array keeps the previous call's contents, so anything
a frame needs cleared must be cleared by that frame).

This file is collected last so that a failure here never hides the result of
another test in a run that stops at the first failure.
"""
import numpy as np
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


@pytest.mark.parametrize("cfg,size,prec", [(0, (48, 40), 0), (1, (64, 48), 0), (2, (40, 64), 1)])
def test_noalloc_matches_render_on_consecutive_calls(ivv, cfg, size, prec):
    sc = scenes.config(cfg, width=size[0], height=size[1])
    sc.params.precision = prec
    vol = ivv.volume_for(sc)
    ref = vol.render(sc.camera, sc.params, sc.width, sc.height).clone()
    torch.cuda.synchronize()
    assert ref[..., 3].max().item() > 0.05, "the window shows the volume"
    for call in range(2):
        out = torch.full_like(ref, float("nan"))
        vol.render_noalloc(sc.camera, sc.params, sc.width, sc.height, out)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= TOL_RGBA, (call, err)


def test_noalloc_rejects_oversized_window(ivv):
    sc = scenes.config(1, width=1920, height=1080)
    vol = ivv.volume_for(sc)
    out = torch.empty((1080, 1920, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ivv.IvvError) as e:
        vol.render_noalloc(sc.camera, sc.params, 1920, 1080, out)
    assert e.value.status == 8 and "bytes of scratch" in str(e.value)
