"""Plain FP64 CPU oracle of the implicit solve (test infrastructure only).

Newton-Raphson on the backward-Euler residual (Sect. 3.3.1) with restarted,
right-preconditioned GMRES (preconditioning as in Sect. 3.3.2: solve
A K^-1 y = b, then x = K^-1 y) and a point-block Jacobi K (the block form
of the Jacobi preconditioner of Sect. 3.3.2: K keeps each cell's own
n_u x n_u block of A).

GMRES follows the textbook algorithm (Saad 2003, Alg. 6.9 with restarts):
modified Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix,
least-squares update at the end of each cycle. The paper uses BiCGStab;
GMRES(30) is the Krylov method this library implements.

Tiny grids also get the dense Jacobian assembled column by column from J e_k
and a partial-pivot LU solve (numpy.linalg.solve), the linear-system pin.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from .m1 import Scheme


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    converged: bool
    resid: float  # true ||b - A x|| at exit
    history: List[float] = field(default_factory=list)


def gmres(A: Callable, b: np.ndarray, Minv: Callable, rtol: float = 1e-10, restart: int = 30,
          maxiter: int = 3000, x0: Optional[np.ndarray] = None) -> GmresResult:
    """Right-preconditioned restarted GMRES(restart) for A x = b.

    Stops when the Arnoldi residual estimate drops to rtol * ||b|| and the
    true residual confirms it (else it restarts from the current x).
    """
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return GmresResult(np.zeros(n), 0, True, 0.0, hist)
    target = rtol * bnorm
    total = 0
    while True:
        r = b - A(x)
        beta = np.linalg.norm(r)
        hist.append(beta)
        if beta <= target or total >= maxiter:
            return GmresResult(x, total, beta <= target, beta, hist)
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for j in range(m):
            w = A(Minv(V[j]))
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # apply previous rotations to column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den if den > 0 else 1.0
            sn[j] = H[j + 1, j] / den if den > 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k_used = j + 1
            total += 1
            if abs(g[j + 1]) <= target or H[j, j] == 0.0 or total >= maxiter:
                break
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):  # back substitution on the rotated H
            y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:]) / H[i, i]
        x = x + Minv(V[:k_used].T @ y)


def bicgstab(A: Callable, b: np.ndarray, Minv: Callable, rtol: float = 1e-10, maxiter: int = 3000
             ) -> GmresResult:
    """Right-preconditioned BiCGStab (the paper's Krylov solver, Sect. 3.3.1) for A x = b.

    van der Vorst's recurrence on A M^-1 y = b, x = M^-1 y, from x = 0 with the shadow
    residual equal to b; one iteration is two products with A and two with M^-1. Stops when
    ||r|| (the recurred residual, checked after each half step) is at most rtol ||b||.
    The returned count is the number of full or half iterations taken.
    """
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    hist = [bnorm]
    if bnorm == 0.0:
        return GmresResult(x, 0, True, 0.0, hist)
    target = rtol * bnorm
    r = b.copy()
    rhat = b.copy()
    rho = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    it = 0
    while it < maxiter:
        rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = Minv(p)
        v = A(phat)
        alpha = rho_new / (rhat @ v)
        s = r - alpha * v
        it += 1
        if np.linalg.norm(s) <= target:
            x = x + alpha * phat
            hist.append(np.linalg.norm(s))
            return GmresResult(x, it, True, np.linalg.norm(s), hist)
        shat = Minv(s)
        t = A(shat)
        omega = (t @ s) / (t @ t)
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho = rho_new
        hist.append(np.linalg.norm(r))
        if hist[-1] <= target:
            return GmresResult(x, it, True, hist[-1], hist)
    return GmresResult(x, it, False, hist[-1], hist)


def block_jacobi(blocks: np.ndarray, N: int, nu: int) -> Callable:
    """K^-1 r with K the point-block diagonal of the Jacobian."""
    inv = np.linalg.inv(blocks)  # (N, nu, nu)

    def apply(r):
        rr = r.reshape(nu, N).T  # (N, nu)
        z = np.einsum("nij,nj->ni", inv, rr)
        return z.T.reshape(-1)

    return apply


@dataclass
class NewtonResult:
    u: np.ndarray
    converged: bool
    newton_iters: int
    gmres_iters: int
    res0: float
    res: float
    history: List[float] = field(default_factory=list)
    fallback: Optional[np.ndarray] = None  # grid-shaped mask of the flagged cells (realizability=True)
    fallback_rounds: int = 0               # times the flagged set grew


def admissible_theta(scheme: Scheme, u: np.ndarray, delta: np.ndarray, flagged: np.ndarray) -> np.ndarray:
    """Per-cell step factors for the fallback cells: theta_i = 1 when U_i + delta_i is
    admissible (E > 0, |F| <= cE), else 0.9 times the first of 1/2, 1/4, ... (at most
    40 halvings) that is; 1 in every unflagged cell. The admissible set is convex, so
    the admissible part of the segment from an admissible U_i is an interval."""
    N, d, c = scheme.N, scheme.d, scheme.c
    E, dE = u[:N], delta[:N]
    F, dF = u[N:(1 + d) * N].reshape(d, N), delta[N:(1 + d) * N].reshape(d, N)
    m = np.asarray(flagged).ravel()
    th = np.ones(N)
    for _ in range(40):
        Et = E + th * dE
        Ft = F + th * dF
        ok = (Et > 0.0) & (np.sqrt((Ft * Ft).sum(0)) <= c * Et)
        bad = m & ~ok
        if not bad.any():
            break
        th = np.where(bad, 0.5 * th, th)
    return np.where(m & (th < 1.0), 0.9 * th, th)


def newton_solve(scheme: Scheme, rtol: float = 1e-8, newton_max: int = 30,
                 gmres_rtol: float = 1e-4, restart: int = 30, gmres_max: int = 3000,
                 precond: str = "bj", line_search: bool = True, dense: bool = False,
                 realizability: bool = False, check_every: int = 5) -> NewtonResult:
    """Backward-Euler step by Newton-Raphson (Sect. 3.3.1) from U^n.

    Converged when ||R(U^k)||_2 <= rtol ||R(U^n)||_2 (2-norm over all unknowns).
    Each Newton step solves J delta = -R to gmres_rtol (``dense``: exactly, by
    LU of the assembled Jacobian; tiny grids only); the step is damped by
    halving theta (up to 6 times) until ||R|| decreases by the Armijo factor
    (1 - 1e-4 theta); the last trial is taken if none does.

    ``realizability``: the library's a posteriori admissibility fallback (Sect.
    3.1.3 leaves f > 1 possible with the AP + WB scheme and names the centred
    source as a remedy; the fallback scheme is described with Scheme). Checks
    run when the iterate has converged and after every ``check_every`` Newton
    steps without convergence (0: only at convergence). A check flags the cells
    with E <= 0 or |F| > cE that are not flagged yet; when there are none and
    Newton has not converged, it flags instead the unflagged cells whose largest
    residual component is at least a tenth of the largest one (Newton stalls on
    the AP + WB system where the fallback one converges). Flagging resets newly
    flagged inadmissible cells of the iterate to U^n (admissible), rebuilds the scheme
    with the grown set and re-takes ||R(U^n)|| as the reference. In flagged
    cells every Newton update is scaled per cell so that they stay admissible
    (admissible_theta), before the line search. Newton steps of all rounds count
    against newton_max. Converged: the last scheme's residual meets rtol at a
    check that flags nothing.
    """
    p = scheme.p
    mask = None
    if realizability:
        mask = np.zeros(scheme.shape, dtype=bool) if scheme.fallback is None else scheme.fallback.copy()
    un = scheme.pack(scheme.Un)
    u = un.copy()
    R = scheme.residual(u)
    r0 = np.linalg.norm(R)
    hist = [r0]
    rn = r0
    its = 0
    git = 0
    rounds = 0
    since = 0
    N, nu = scheme.N, scheme.nu
    while True:
        due = rn <= rtol * r0 or (check_every > 0 and since >= check_every)
        if realizability and due:
            since = 0
            new = scheme.inadmissible(u) & ~mask
            reset = new.any()
            if not reset and rn > rtol * r0:
                Rc = np.abs(R.reshape(nu, N)).max(axis=0).reshape(scheme.shape)
                new = (Rc >= 0.1 * Rc.max()) & ~mask
            if new.any():
                mask |= new
                rounds += 1
                if reset:
                    u = np.where(np.tile(new.ravel(), nu), un, u)
                scheme = Scheme(p, mask)
                r0 = np.linalg.norm(scheme.residual(un))
                R = scheme.residual(u)
                rn = np.linalg.norm(R)
                hist.append(rn)
                continue
        if rn <= rtol * r0 or its >= newton_max:
            break
        if dense:
            delta = dense_solve(scheme, u, -R)
        else:
            if precond == "bj":
                Minv = block_jacobi(scheme.diag_blocks(u), N, nu)
            else:
                Minv = lambda r: r  # noqa: E731
            res = gmres(lambda v: scheme.jv(u, v), -R, Minv, rtol=gmres_rtol, restart=restart,
                        maxiter=gmres_max)
            git += res.iters
            delta = res.x
        if realizability and mask.any():
            delta = delta * np.tile(admissible_theta(scheme, u, delta, mask), nu)
        theta = 1.0
        for _ in range(7):
            ut = u + theta * delta
            Rt = scheme.residual(ut)
            rt = np.linalg.norm(Rt)
            if not line_search or rt <= (1.0 - 1e-4 * theta) * rn:
                break
            theta *= 0.5
        u, R, rn = ut, Rt, rt
        its += 1
        since += 1
        hist.append(rn)
    out = NewtonResult(u, bool(rn <= rtol * r0), its, git, r0, rn, hist)
    if realizability:
        out.fallback = mask
        out.fallback_rounds = rounds
    return out


def block_tridiagonal_part(J: np.ndarray, nu: int, N: int) -> np.ndarray:
    """The couplings of a 1D dense Jacobian (unknowns [k N + i]) between cells i and j
    with |i - j| <= 1, no periodic wrap: the matrix the line preconditioner solves."""
    i = np.arange(nu * N) % N
    return np.where(np.abs(i[:, None] - i[None, :]) <= 1, J, 0.0)


def dense_jacobian(scheme: Scheme, u: np.ndarray) -> np.ndarray:
    """J assembled column by column as J e_k (tiny grids only)."""
    n = u.size
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        J[:, k] = scheme.jv(u, e)
    return J


def dense_solve(scheme: Scheme, u: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = J(u)^-1 b by partial-pivot LU (LAPACK gesv via numpy)."""
    return np.linalg.solve(dense_jacobian(scheme, u), b)
