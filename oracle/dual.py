"""Forward-mode dual numbers over numpy arrays (oracle test infrastructure).

A Dual carries a value array ``v`` and a directional-derivative array ``d``.
Evaluating the oracle's residual on Dual(U, v) gives (R(U), J(U) v) exactly,
up to rounding. Non-smooth points follow fixed tie-breaks:
  * max/min keep the FIRST argument on equality;
  * sqrt at 0 has derivative 0;
  * a clamp that is active has derivative 0.
Plain numpy arrays and floats mix freely with Duals (they are constants).
"""
from __future__ import annotations

import numpy as np


class Dual:
    __slots__ = ("v", "d")
    __array_priority__ = 1000.0

    def __init__(self, v, d=None):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.zeros_like(self.v) if d is None else np.asarray(d, dtype=np.float64)

    # arithmetic -----------------------------------------------------------
    def __add__(self, o):
        o = lift(o)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = lift(o)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        o = lift(o)
        return Dual(o.v - self.v, o.d - self.d)

    def __mul__(self, o):
        o = lift(o)
        return Dual(self.v * o.v, self.d * o.v + self.v * o.d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = lift(o)
        q = self.v / o.v
        return Dual(q, (self.d - q * o.d) / o.v)

    def __rtruediv__(self, o):
        return lift(o) / self

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __getitem__(self, idx):
        return Dual(self.v[idx], self.d[idx])

    @property
    def shape(self):
        return self.v.shape


def lift(x) -> Dual:
    return x if isinstance(x, Dual) else Dual(x, np.zeros_like(np.asarray(x, dtype=np.float64)))


def value(x):
    return x.v if isinstance(x, Dual) else np.asarray(x, dtype=np.float64)


def deriv(x):
    return x.d if isinstance(x, Dual) else np.zeros_like(np.asarray(x, dtype=np.float64))


def is_dual(*xs) -> bool:
    return any(isinstance(x, Dual) for x in xs)


def where(cond, a, b):
    """Elementwise select (value and derivative together)."""
    if is_dual(a, b):
        a, b = lift(a), lift(b)
        return Dual(np.where(cond, a.v, b.v), np.where(cond, a.d, b.d))
    return np.where(cond, a, b)


def sqrt(x):
    """Square root; derivative 0 where the value is 0."""
    if isinstance(x, Dual):
        s = np.sqrt(x.v)
        with np.errstate(divide="ignore", invalid="ignore"):
            d = np.where(s > 0.0, x.d / (2.0 * np.where(s > 0.0, s, 1.0)), 0.0)
        return Dual(s, d)
    return np.sqrt(x)


def max_first(a, b):
    """max(a, b) keeping ``a`` unless b > a strictly."""
    return where(value(b) > value(a), b, a)


def min_first(a, b):
    """min(a, b) keeping ``a`` unless b < a strictly."""
    return where(value(b) < value(a), b, a)


def concat(parts, axis):
    if is_dual(*parts):
        parts = [lift(p) for p in parts]
        return Dual(np.concatenate([p.v for p in parts], axis=axis),
                    np.concatenate([p.d for p in parts], axis=axis))
    return np.concatenate(parts, axis=axis)


def take(x, idx, axis):
    """np.take keeping the axis (idx is a list)."""
    if isinstance(x, Dual):
        return Dual(np.take(x.v, idx, axis=axis), np.take(x.d, idx, axis=axis))
    return np.take(x, idx, axis=axis)


def slice_axis(x, sl, axis):
    index = [slice(None)] * value(x).ndim
    index[axis] = sl
    return x[tuple(index)]
