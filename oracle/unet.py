"""Plain FP64 oracle of the learned preconditioner network (test infrastructure).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A 3-level 2D U-Net mapping 7 input channels (the three components of a
residual vector, scaled, the normalised log opacity, and the state at which
the Jacobian is taken: the reduced flux F / (cE) in two channels and the
normalised log energy; input_planes) to 3 output channels.
All convolutions are 3x3, stride 1, zero padding 1, weights laid out
W[ky, kx, ci, co] with bias b[co]; ReLU after every convolution but the last;
2x2 average pooling down; nearest-neighbour 2x upsampling followed by channel
concatenation [upsampled, skip]. Arrays are NHWC (batch, y, x, channel).

The paper has no learned preconditioner; this network and its training are
the library's own design. The oracle gives the forward pass and the exact
backward pass of the loss
    L = (1/B) sum_b ||y_b - t_b||^2 / (H W 3)
(the mean squared error per output element)
by plain loops over layers (numpy einsum for each 3x3 tap). Pinned by central
finite differences (tests/test_oracle_unet.py).
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

# (name, cin, cout, relu) in execution order; "pool"/"up" markers separate levels
C1, C2, C3 = 16, 32, 32
CIN = 7
LAYERS: List[Tuple[str, int, int, bool]] = [
    ("e1a", CIN, C1, True), ("e1b", C1, C1, True),
    ("e2a", C1, C2, True), ("e2b", C2, C2, True),
    ("e3a", C2, C3, True), ("e3b", C3, C3, True),
    ("d2a", C3 + C2, C2, True), ("d2b", C2, C1, True),
    ("d1a", C1 + C1, C1, True), ("d1b", C1, 3, False),
]


def param_shapes() -> List[Tuple[str, tuple]]:
    out = []
    for name, ci, co, _ in LAYERS:
        out.append((name + ".w", (3, 3, ci, co)))
        out.append((name + ".b", (co,)))
    return out


def num_params() -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(theta: np.ndarray) -> Dict[str, np.ndarray]:
    """Flat parameter vector (layer order, W then b, C order) -> dict."""
    out, k = {}, 0
    for name, shp in param_shapes():
        m = int(np.prod(shp))
        out[name] = theta[k:k + m].reshape(shp)
        k += m
    return out


def flatten(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([p[name].ravel() for name, _ in param_shapes()])


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 cin))), zero biases; the last layer is
    scaled by 1e-3 so that the network starts as a near-zero correction."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co, relu in LAYERS:
        std = np.sqrt(2.0 / (9 * ci)) * (1.0 if relu else 1e-3)
        p[name + ".w"] = rng.standard_normal((3, 3, ci, co)) * std
        p[name + ".b"] = np.zeros(co)
    return flatten(p)


def input_planes(E, Fx, Fy, sigma_f, dx, c):
    """The four input channels that do not depend on the Krylov vector, from the
    linearisation state: (log10(sigma_f dx) - 0.5) / 2.5, F_x / (cE) and F_y / (cE)
    with E floored at 1e-30 and clipped to [-1, 1], and (log10 E + 3) / 3."""
    E = np.maximum(np.asarray(E, dtype=np.float64), 1e-30)
    logsig = (np.log10(np.maximum(np.asarray(sigma_f, dtype=np.float64) * dx, 1e-30)) - 0.5) / 2.5
    fx = np.clip(np.asarray(Fx, dtype=np.float64) / (c * E), -1.0, 1.0)
    fy = np.clip(np.asarray(Fy, dtype=np.float64) / (c * E), -1.0, 1.0)
    return np.stack([logsig, fx, fy, (np.log10(E) + 3.0) / 3.0], axis=-1)


# ------------------------------------------------------------------ layers
def conv3x3(x, w, b):
    """y[n,i,j,co] = b[co] + sum_{dy,dx,ci} x[n,i+dy-1,j+dx-1,ci] w[dy,dx,ci,co] (zero padding)."""
    n, H, W, ci = x.shape
    xp = np.zeros((n, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.broadcast_to(b, (n, H, W, w.shape[3])).copy()
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nijc,cd->nijd", xp[:, dy:dy + H, dx:dx + W, :], w[dy, dx])
    return y


def conv3x3_backward(x, w, gy):
    """Gradients (gx, gw, gb) of conv3x3 for upstream gradient gy."""
    n, H, W, ci = x.shape
    xp = np.zeros((n, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[dy, dx] = np.einsum("nijc,nijd->cd", xp[:, dy:dy + H, dx:dx + W, :], gy)
            gxp[:, dy:dy + H, dx:dx + W, :] += np.einsum("nijd,cd->nijc", gy, w[dy, dx])
    gb = gy.sum(axis=(0, 1, 2))
    return gxp[:, 1:-1, 1:-1, :], gw, gb


def pool2(x):
    n, H, W, c = x.shape
    return x.reshape(n, H // 2, 2, W // 2, 2, c).mean(axis=(2, 4))


def pool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(gy):
    n, H, W, c = gy.shape
    return gy.reshape(n, H // 2, 2, W // 2, 2, c).sum(axis=(2, 4))


# ------------------------------------------------------------------ network
def forward(theta: np.ndarray, x: np.ndarray, keep: bool = False):
    """U-Net forward pass on NHWC x (H, W divisible by 4)."""
    p = unflatten(theta)
    cache = {}

    def layer(name, inp):
        y = conv3x3(inp, p[name + ".w"], p[name + ".b"])
        relu = dict((l[0], l[3]) for l in LAYERS)[name]
        out = np.maximum(y, 0.0) if relu else y
        cache[name] = (inp, out)
        return out

    s1 = layer("e1b", layer("e1a", x))
    s2 = layer("e2b", layer("e2a", pool2(s1)))
    h3 = layer("e3b", layer("e3a", pool2(s2)))
    d2 = layer("d2b", layer("d2a", np.concatenate([up2(h3), s2], axis=3)))
    y = layer("d1b", layer("d1a", np.concatenate([up2(d2), s1], axis=3)))
    return (y, cache) if keep else y


def loss(theta, x, t):
    y = forward(theta, x)
    per = float(np.prod(t.shape[1:]))
    return float((((y - t) ** 2).sum(axis=(1, 2, 3)) / per).mean())


def grad(theta: np.ndarray, x: np.ndarray, t: np.ndarray):
    """(loss, dL/dtheta) by the chain rule through every layer."""
    p = unflatten(theta)
    y, cache = forward(theta, x, keep=True)
    B = x.shape[0]
    per = float(np.prod(t.shape[1:]))
    L = float((((y - t) ** 2).sum(axis=(1, 2, 3)) / per).mean())
    gy = 2.0 * (y - t) / per / B
    g = {}
    relu = dict((l[0], l[3]) for l in LAYERS)

    def back(name, gout):
        inp, out = cache[name]
        gpre = gout * (out > 0) if relu[name] else gout
        gx, gw, gb = conv3x3_backward(inp, p[name + ".w"], gpre)
        g[name + ".w"] = gw
        g[name + ".b"] = gb
        return gx

    gcat1 = back("d1a", back("d1b", gy))
    g_up_d2, g_s1 = gcat1[..., :C1], gcat1[..., C1:]
    gcat2 = back("d2a", back("d2b", up2_backward(g_up_d2)))
    g_up_h3, g_s2 = gcat2[..., :C3], gcat2[..., C3:]
    g_s2 = g_s2 + pool2_backward(back("e3a", back("e3b", up2_backward(g_up_h3))))
    g_s1 = g_s1 + pool2_backward(back("e2a", back("e2b", g_s2)))
    back("e1a", back("e1b", g_s1))
    return L, flatten(g)
