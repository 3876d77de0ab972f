"""FP64 reference of the initial-guess network (test infrastructure only).

A 3-64-64-3 perceptron with ReLU hidden layers maps a point g of a block,
normalised to the block's control-point box (g_hat = (g - centre) / half_size),
to a parameter-space guess p_hat.  Loss per batch: mean over points of
||p_hat - p||^2.  Forward and backward are written out with matrix products
(numpy) so the device training kernels' gradients can be checked against them;
the backward pass is pinned to central finite differences of the loss.

Parameter layout (one flat vector, as the library stores it per block):
W1 [64][3], b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3].
"""
import numpy as np

H = 64
SHAPES = [("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (3, H)), ("b3", (3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in SHAPES])


def forward(theta, x):
    """p_hat [n][3] for normalised inputs x [n][3]; also the activations."""
    w = unpack(theta)
    z1 = x @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"].T + w["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(theta, x, p):
    y, _ = forward(theta, x)
    return float(np.mean(np.sum((y - p) ** 2, axis=1)))


def loss_grad(theta, x, p):
    """(loss, flat gradient) of the mean squared error over the batch."""
    w = unpack(theta)
    y, (x, z1, h1, z2, h2) = forward(theta, x)
    n = x.shape[0]
    dy = 2.0 * (y - p) / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = (dy @ w["W3"]) * (z2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ w["W2"]) * (z1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return float(np.mean(np.sum((y - p) ** 2, axis=1))), pack(g)


def init(seed, scale=1.0):
    """He-style initialisation (as the library's default, seeded the same way
    only in distribution; tests pass explicit weights to both sides)."""
    rng = np.random.default_rng(seed)
    parts = {"W1": rng.normal(0, np.sqrt(2 / 3), (H, 3)) * scale, "b1": np.zeros(H),
             "W2": rng.normal(0, np.sqrt(2 / H), (H, H)) * scale, "b2": np.zeros(H),
             "W3": rng.normal(0, np.sqrt(1 / H), (3, H)) * scale, "b3": np.full(3, 0.5)}
    return pack(parts)
