"""Plain FP64 oracle of how flexible GMRES applies the learned preconditioner
(test infrastructure).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned component: these forms are the library's own design
(m1_set_learned_form). With M the point-block Jacobi inverse, J the Jacobian,
N the network as a map from a scaled residual vector to a correction (the
opacity and state planes fixed at the Newton iterate), n the number of
unknowns and s(x) = ||x||_2 / sqrt(n) the RMS of a vector (1 for a zero vector):
    additive:   z = M v + s (N(v / s) - N(0)),               s = s(v)
    two-stage:  z1 = M v,  r1 = v - J z1,
                z = z1 + M r1 + s1 (N(r1 / s1) - N(0)),      s1 = s(r1)
Both are exact, z = J^-1 v, when N is the linear map (J^-1 - M), the part of the
inverse point-block Jacobi misses, which is what the training pairs target
(m1_nn_make_pair: input J e, target e - M J e). Pinned by that property, by
their reduction to Richardson sweeps with M when N is zero, and by their
positive homogeneity (tests/test_oracle_learned.py).
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import unet


def rms(x: np.ndarray) -> float:
    """||x||_2 / sqrt(n), or 1 for a zero vector."""
    s = float(np.linalg.norm(x)) / np.sqrt(x.size)
    return s if s > 0.0 else 1.0


def additive(v: np.ndarray, Minv: Callable, net: Callable) -> np.ndarray:
    """z = M v + s (N(v / s) - N(0)), s the RMS of v."""
    s = rms(v)
    return Minv(v) + s * (net(v / s) - net(np.zeros_like(v)))


def two_stage(v: np.ndarray, A: Callable, Minv: Callable, net: Callable) -> np.ndarray:
    """z1 = M v, r1 = v - J z1, z = z1 + M r1 + s1 (N(r1 / s1) - N(0)), s1 the RMS of r1."""
    z1 = Minv(v)
    r1 = v - A(z1)
    s1 = rms(r1)
    return z1 + Minv(r1) + s1 * (net(r1 / s1) - net(np.zeros_like(v)))


def unet_map(theta: np.ndarray, planes: np.ndarray, H: int, W: int) -> Callable:
    """The network as a map of component-major vectors (E, Fx, Fy; H W each) to
    component-major corrections: the vector's three channels beside the four
    fixed planes (input_planes, H W x 4), NHWC, one image."""
    N = H * W

    def apply(x: np.ndarray) -> np.ndarray:
        ch = x.reshape(3, N).T  # (N, 3)
        inp = np.concatenate([ch, planes.reshape(N, 4)], axis=1).reshape(1, H, W, unet.CIN)
        y = unet.forward(theta, inp).reshape(N, 3)
        return y.T.reshape(-1)

    return apply
