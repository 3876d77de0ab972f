"""The learned initial guess on the GPU: the training kernel's gradient
against the FP64 reference network, the tensor-core inference against an
FP64 forward pass that rounds where the kernel rounds (FP16 weights and
activations), and a short training run on the twisted bar."""
import numpy as np
import pytest

from oracle import mlp
from paper_1404_3363_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ivv():
    from paper_1404_3363_gb300 import build, ivv as mod
    assert torch.cuda.is_available(), "a CUDA device is required"
    build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def bar(ivv):
    sc = scenes.config(1, width=64, height=64)
    return sc, ivv.volume_for(sc)


def _f4(a):
    out = np.zeros((a.shape[0], 4), np.float32)
    out[:, :3] = a
    return torch.from_numpy(out).cuda()


def test_training_gradient_matches_fp64_reference(ivv, bar):
    sc, vol = bar
    rng = np.random.default_rng(70)
    theta = (mlp.init(3) + 0.05 * rng.normal(size=mlp.N_PARAMS)).astype(np.float32)
    vol.set_guess_weights(0, theta)
    n = 1000                                    # not a multiple of the 128-sample CTA
    x = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    p = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    loss, grad = vol.guess_loss_grad(0, _f4(x), _f4(p))
    L, g = mlp.loss_grad(theta.astype(np.float64), x.astype(np.float64), p.astype(np.float64))
    assert loss == pytest.approx(L, rel=1e-5)
    scale = np.abs(g).max()
    np.testing.assert_allclose(grad, g, atol=1e-5 * scale, rtol=1e-4)


def test_tensor_core_inference(ivv, bar):
    sc, vol = bar
    rng = np.random.default_rng(71)
    theta = (mlp.init(4) + 0.05 * rng.normal(size=mlp.N_PARAMS)).astype(np.float32)
    vol.set_guess_weights(0, theta)
    w, c, inv_h = vol.get_guess_weights(0)
    np.testing.assert_array_equal(w, theta)
    n = 1001
    g = (c + rng.uniform(-1, 1, (n, 3)) / inv_h).astype(np.float32)
    out = vol.guess_points(_f4(g), torch.zeros(n, dtype=torch.int32, device="cuda")).cpu().numpy()[:, :3]
    # FP64 forward with the kernel's rounding points: FP16 weights, FP16
    # inputs of layers 2 and 3, FP32 (here FP64) accumulation
    x = ((g.astype(np.float64) - c.astype(np.float64)) * np.float64(np.float32(inv_h)))
    h16 = mlp.unpack(theta.astype(np.float16).astype(np.float64))
    r16 = lambda a: a.astype(np.float16).astype(np.float64)
    h1 = r16(np.maximum(x @ h16["W1"].T + h16["b1"], 0))
    h2 = r16(np.maximum(h1 @ h16["W2"].T + h16["b2"], 0))
    ref16 = h2 @ h16["W3"].T + h16["b3"]
    np.testing.assert_allclose(out, ref16, atol=2e-3 * max(1.0, np.abs(ref16).max()))
    ref64, _ = mlp.forward(theta.astype(np.float64), x)
    assert np.abs(out - ref64).max() < 0.05 * max(1.0, np.abs(ref64).max())


def test_training_learns_the_inverse_map(ivv, bar):
    sc, vol = bar
    losses = vol.train_guess(samples_per_block=1 << 17, epochs=24, batch=2048, lr=3e-3, seed=5)
    assert losses[0] < 1e-3, losses          # RMS parameter error below 0.02
    # fresh points: parameter error of the guess
    import oracle
    ov = oracle.OracleVolume(sc.blocks, sc.scalar_mode)
    rng = np.random.default_rng(72)
    P = rng.uniform(0.02, 0.98, (4096, 3))
    G, _, _ = ov.eval(0, P)
    out = vol.guess_points(_f4(G.astype(np.float32)), torch.zeros(4096, dtype=torch.int32, device="cuda"))
    err = np.abs(out.cpu().numpy()[:, :3] - P)
    assert err.mean() < 0.02 and np.percentile(err.max(1), 99) < 0.1, (err.mean(), err.max())
