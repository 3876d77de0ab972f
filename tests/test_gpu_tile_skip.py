"""Tiles without candidate patches (stages 1-2 of a single frame).

The cull (K2a) finishes the 8 x 4 warp tiles whose rays meet no patch box:
it writes their pair counts and zero pixels and leaves a 16 x 16 tile flag
unset, and the pairing kernel (K4) skips every unflagged 16 x 16 tile and
clears the flags it finds set.  The flags live in the caller's workspace
between frames, so these tests render through a workspace that holds the
previous frame's flags, or arbitrary bytes, and require the image of a fresh
workspace (to rounding: fragments of equal depth may reach the pairing in
either order), with every pixel written.
"""
import dataclasses

import pytest

from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _same(x, y):
    return not torch.isnan(x).any() and (x - y).abs().max().item() <= TOL


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


def _moved(cam, dx):
    eye = tuple(e + d for e, d in zip(cam.eye, dx))
    target = tuple(t + d for t, d in zip(cam.target, dx))
    return dataclasses.replace(cam, eye=eye, target=target)


def _render(vol, sc, cam):
    out = torch.full((sc.height, sc.width, 4), float("nan"), dtype=torch.float32, device="cuda")
    vol.render(cam, sc.params, sc.width, sc.height, out=out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("cfg,prec", [(1, 0), (2, 1), (4, 0)])
def test_stale_tile_flags_change_nothing(ivv, cfg, prec):
    sc = scenes.config(cfg, width=200, height=136)
    sc.params.precision = prec
    cam_b = _moved(sc.camera, (0.21, -0.13, 0.0))
    fresh = _render(ivv.volume_for(sc), sc, cam_b)
    assert not torch.isnan(fresh).any()
    assert fresh[..., 3].max().item() > 0.05, "the moved camera still sees the volume"
    assert (fresh[..., 3] == 0).any(), "and some empty tiles"
    vol = ivv.volume_for(sc)
    a = _render(vol, sc, sc.camera)                 # leaves camera A's tiles in the workspace
    assert not torch.isnan(a).any()
    b = _render(vol, sc, cam_b)
    assert _same(b, fresh)
    again = _render(vol, sc, cam_b)                 # flags cleared by the previous frame's K4
    assert _same(again, fresh)


@pytest.mark.parametrize("fill", [0, 255, 1])
def test_workspace_bytes_do_not_matter(ivv, fill):
    sc = scenes.config(1, width=160, height=120)
    fresh = _render(ivv.volume_for(sc), sc, sc.camera)
    vol = ivv.volume_for(sc)
    vol.workspace(sc.width, sc.height, sc.params.precision)
    vol._ws.fill_(fill)                             # flags all clear, all set, or set to 0x01010101
    out = _render(vol, sc, sc.camera)
    assert _same(out, fresh)
