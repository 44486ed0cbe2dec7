"""Aggregation multigrid preconditioner: plain FP64 oracle (test infrastructure).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's best CPU preconditioner is algebraic multigrid (Sect. 3.3.2, Sect. 4); this is its
structured-grid analogue for the 2D radiation-only Newton system J(U) delta = -R:

- the Jacobian as a 5-point stencil of n_u x n_u blocks per cell, in the order
  (C, W, E, S, N) = (self, -x, +x, -y, +y) neighbour, read off J by probing J v with
  vectors that are 1 on one unknown of every cell of one colour class (cells of a class are
  far enough apart that their stencils do not overlap); a coupling through a
  non-periodic boundary ghost lands in C, one through a periodic wrap in the wrapped
  neighbour's block;
- 2 x 2 cell aggregates per level (ceil at odd sizes), piecewise-constant prolongation P
  (a coarse value copied to the cells of its aggregate) and restriction P^T (sum over the
  aggregate), the Galerkin operator A_c = P^T A P, which is again a 5-point block stencil:
  a fine coupling to a cell of the same aggregate adds to C, one to another aggregate
  adds to the block of its own direction;
- coarsening until both sides are at most COARSEST cells;
- a V(1,1) cycle with damped point-block Jacobi smoothing (omega = OMEGA, the block
  inverses of the C blocks), the finest level's operator applied as J v itself, and
  COARSE_SWEEPS damped block-Jacobi sweeps from zero on the coarsest level.

Pinned in tests/test_oracle_mg.py: the assembled stencil reproduces J v; the Galerkin
stencil reproduces P^T A P on vectors; the cycle is linear in r; with no smoothing and an
exact coarsest solve the two-level cycle equals P A_c^-1 P^T r.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

OMEGA = 0.7
COARSEST = 16
COARSE_SWEEPS = 10
# stencil positions and their (dx, dy) offsets
STENCIL = ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1))


def colouring(n: int, periodic: bool) -> int:
    """Period m of the colour classes along one axis: cells with equal index mod m are
    at least 3 apart (also across a periodic wrap), so their 5-point stencils are disjoint."""
    if not periodic:
        return 3
    for m in range(3, n + 1):
        r = n % m
        if r == 0 or (r >= 3 and m - r >= 3):
            return m
    return n


def _neighbour(ix, iy, s, nx, ny, px, py):
    """Index of neighbour s of cells (ix, iy), or -1 outside a non-periodic boundary."""
    dx, dy = STENCIL[s]
    jx, jy = ix + dx, iy + dy
    if px:
        jx = jx % nx
    if py:
        jy = jy % ny
    ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
    return np.where(ok, jy * nx + jx, -1)


def assemble_blocks(jv, nu: int, nx: int, ny: int, px: bool, py: bool) -> np.ndarray:
    """A[s, r, c, i]: d R_r(cell i) / d U_c(neighbour s of i), from probes of jv(v)."""
    N = nx * ny
    A = np.zeros((5, nu, nu, N))
    mx, my = colouring(nx, px), colouring(ny, py)
    ix, iy = np.arange(N) % nx, np.arange(N) // nx
    colour = (ix % mx) + mx * (iy % my)
    nbs = [_neighbour(ix, iy, s, nx, ny, px, py) for s in range(5)]
    for col in range(mx * my):
        probed = colour == col
        for c in range(nu):
            v = np.zeros(nu * N)
            v[c * N + np.nonzero(probed)[0]] = 1.0
            y = jv(v)
            for s in range(5):
                j = nbs[s]
                hit = (j >= 0) & probed[np.maximum(j, 0)]
                for r in range(nu):
                    A[s, r, c, hit] = y[r * N + np.nonzero(hit)[0]]
    return A


def apply_stencil(A: np.ndarray, x: np.ndarray, nx: int, ny: int, px: bool, py: bool) -> np.ndarray:
    """y = A x for a 5-point block stencil (x, y component-major: [c * N + cell])."""
    nu, N = A.shape[1], nx * ny
    X = x.reshape(nu, N)
    Y = np.zeros((nu, N))
    ix, iy = np.arange(N) % nx, np.arange(N) // nx
    for s in range(5):
        j = _neighbour(ix, iy, s, nx, ny, px, py)
        ok = j >= 0
        xs = np.where(ok[None, :], X[:, np.maximum(j, 0)], 0.0)
        Y += np.einsum("rci,ci->ri", A[s], xs)
    return Y.ravel()


def aggregate(nx: int, ny: int) -> Tuple[np.ndarray, int, int]:
    """Aggregate index of every cell (2 x 2 blocks) and the coarse sizes."""
    nxc, nyc = (nx + 1) // 2, (ny + 1) // 2
    N = nx * ny
    ix, iy = np.arange(N) % nx, np.arange(N) // nx
    return (iy // 2) * nxc + ix // 2, nxc, nyc


def galerkin(A: np.ndarray, nx: int, ny: int, px: bool, py: bool) -> Tuple[np.ndarray, int, int]:
    """A_c = P^T A P as a coarse 5-point block stencil."""
    nu, N = A.shape[1], nx * ny
    agg, nxc, nyc = aggregate(nx, ny)
    Ac = np.zeros((5, nu, nu, nxc * nyc))
    ix, iy = np.arange(N) % nx, np.arange(N) // nx
    for s in range(5):
        j = _neighbour(ix, iy, s, nx, ny, px, py)
        ok = j >= 0
        same = ok & (agg[np.maximum(j, 0)] == agg)
        other = ok & ~same
        for r in range(nu):
            for c in range(nu):
                np.add.at(Ac[0, r, c], agg[same], A[s, r, c, same])
                np.add.at(Ac[s, r, c], agg[other], A[s, r, c, other])
    return Ac, nxc, nyc


def prolong(zc: np.ndarray, nu: int, nx: int, ny: int) -> np.ndarray:
    agg, _, _ = aggregate(nx, ny)
    return zc.reshape(nu, -1)[:, agg].ravel()


def restrict(r: np.ndarray, nu: int, nx: int, ny: int) -> np.ndarray:
    agg, nxc, nyc = aggregate(nx, ny)
    out = np.zeros((nu, nxc * nyc))
    R = r.reshape(nu, -1)
    for c in range(nu):
        np.add.at(out[c], agg, R[c])
    return out.ravel()


def block_inverses(A: np.ndarray) -> np.ndarray:
    """Dinv[i] = (C block of cell i)^-1."""
    C = np.moveaxis(A[0], -1, 0)  # (N, nu, nu)
    return np.linalg.inv(C)


def apply_blocks(Dinv: np.ndarray, r: np.ndarray) -> np.ndarray:
    nu, N = Dinv.shape[1], Dinv.shape[0]
    return np.einsum("irc,ci->ri", Dinv, r.reshape(nu, N)).ravel()


class Hierarchy:
    """Levels 1.. of the aggregation hierarchy; level 0 applies J v through `jv`."""

    def __init__(self, jv, nu: int, nx: int, ny: int, px: bool, py: bool, coarsest: int = COARSEST):
        self.jv, self.nu, self.px, self.py = jv, nu, px, py
        A = assemble_blocks(jv, nu, nx, ny, px, py)
        self.sizes: List[Tuple[int, int]] = [(nx, ny)]
        self.ops: List[np.ndarray] = [A]
        self.dinv: List[np.ndarray] = [block_inverses(A)]
        while nx > coarsest or ny > coarsest:
            A, nx, ny = galerkin(A, nx, ny, px, py)
            self.sizes.append((nx, ny))
            self.ops.append(A)
            self.dinv.append(block_inverses(A))

    def apply_op(self, lvl: int, x: np.ndarray) -> np.ndarray:
        if lvl == 0:
            return self.jv(x)
        nx, ny = self.sizes[lvl]
        return apply_stencil(self.ops[lvl], x, nx, ny, self.px, self.py)

    def cycle(self, r: np.ndarray, lvl: int = 0, omega: float = OMEGA, nu1: int = 1, nu2: int = 1,
              sweeps: int = COARSE_SWEEPS) -> np.ndarray:
        """One V(nu1, nu2) cycle from zero: z ~ A_lvl^-1 r."""
        D = self.dinv[lvl]
        if lvl == len(self.ops) - 1:
            z = np.zeros_like(r)
            for _ in range(sweeps):
                z = z + omega * apply_blocks(D, r - self.apply_op(lvl, z))
            return z
        nx, ny = self.sizes[lvl]
        z = np.zeros_like(r)
        for _ in range(nu1):
            z = z + omega * apply_blocks(D, r - self.apply_op(lvl, z))
        rc = restrict(r - self.apply_op(lvl, z), self.nu, nx, ny)
        z = z + prolong(self.cycle(rc, lvl + 1, omega, nu1, nu2, sweeps), self.nu, nx, ny)
        for _ in range(nu2):
            z = z + omega * apply_blocks(D, r - self.apply_op(lvl, z))
        return z
