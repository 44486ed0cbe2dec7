"""Plain FP64 CPU oracle of the grey M1 discretisation (Bloch et al. 2021).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this
module: only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm use it. It shares no code with the CUDA library.

What it computes, in the paper's order and notation (one face array per axis,
numpy vectorised over cells, written for reading rather than speed):

* M1 closure, Sect. 2.2: f = F/(cE), chi = (3+4f^2)/(5+2 sqrt(4-3f^2)),
  D = (1-chi)/2 I + (3chi-1)/2 n(x)n, P = D E.
* M1 eigenvalues, Eq. (eigenvalues), Sect. 3.1.1.
* HLL fluxes F*, P*, Sect. 3.1.1, with lambda+ = max(0, lambda_max),
  lambda- = min(0, lambda_min).
* Asymptotic-preserving correction alpha, Eq. (asymptoticCorrection), Sect. 3.1.3.
* Well-balanced flux source, Eqs. (wb_smart) and (boundaryCondition), Sect. 3.1.2;
  the centred alternative Eq. (wb_naive).
* Energy exchange with the gas, Eqs. (momentModel) and (internalEnergyEqua).
* The backward-Euler residual of the scheme of Sect. 3.1.1 and its exact
  directional derivative (forward-mode dual numbers, oracle.dual).
* The semi-implicit step (Sect. 3.1: sources implicit, fluxes explicit), whose
  WB source is the tridiagonal operator of Appendix B.

Readings where the paper is silent (listed with the design notes):
* lambda at a face: Davis estimate over both neighbour states,
  lambda+ = max(floor, lmax_L, lmax_R), lambda- = min(-floor, lmin_L, lmin_R);
  lambda in F*, P* at the new time level (flag implicit_eigs = True, the
  reading of Sect. 3.3.1) or frozen at time n (implicit_eigs = False);
  alpha (with its lambdas) always at time n.
* f is clamped to 1 (Sect. 6 remedy) with E_safe = max(E, 1e-300) in f only.
* Multi-D: unsplit sum over axes; normal/tangential split of f for the
  eigenvalues; the WB source of F_b acts along its own axis b.
* Eq. (boundaryCondition) replaces the WB face term at every non-periodic
  boundary face by -c (P_bb,in - P_bb,ghost)/dx with the ghost's P.
* In the semi-implicit step that boundary term uses the pressures at time n.
* Ghosts: outflow = copy, periodic = wrap, reflect = copy with the normal
  flux negated, Dirichlet = given (E, F) where the face mask is 1.
"""
from __future__ import annotations

from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dual as du
from .dual import Dual, concat, max_first, min_first, sqrt, take, value, where

TINY_E = 1e-300
TINY_DEN = 1e-300


class Closure:
    """M1 closure quantities of a set of cells (Sect. 2.2)."""

    def __init__(self, E, F, c):
        d = len(F)
        Es = where(value(E) > TINY_E, E, TINY_E)
        cE = c * Es
        F2 = F[0] * F[0]
        for b in range(1, d):
            F2 = F2 + F[b] * F[b]
        # |F| > c E: keep the direction n = F/|F| and clamp |f| to 1.
        clamped = value(F2) > value(cE) * value(cE)
        with np.errstate(divide="ignore", invalid="ignore"):
            nF = sqrt(where(clamped, F2, 1.0))
            den = where(clamped, nF, cE)
            self.fvec = [F[b] / den for b in range(d)]
        f2 = self.fvec[0] * self.fvec[0]
        for b in range(1, d):
            f2 = f2 + self.fvec[b] * self.fvec[b]
        self.f2 = where(clamped, 1.0, f2)
        self.f = sqrt(self.f2)
        self.xi = sqrt(4.0 - 3.0 * self.f2)
        self.chi = (3.0 + 4.0 * self.f2) / (5.0 + 2.0 * self.xi)
        # (3 chi - 1)/2 n(x)n = g f(x)f with g = (3 chi - 1)/(2 f^2). Since
        # 3 chi - 1 = 2 (2 - xi) and f^2 = (4 - xi^2)/3, g = 3/(2 + xi): the same
        # tensor, written without the 0/0 at f = 0.
        g = 3.0 / (2.0 + self.xi)
        iso = (1.0 - self.chi) / 2.0
        self.D = [[None] * d for _ in range(d)]
        for a in range(d):
            for b in range(d):
                t = g * self.fvec[a] * self.fvec[b]
                self.D[a][b] = iso + t if a == b else t
        self.E = E

    def pressure(self, a, b):
        """P_ab = D_ab E."""
        return self.D[a][b] * self.E


def eigenvalues(cl: Closure, a: int, c: float):
    """lambda_max, lambda_min along axis a, Eq. (eigenvalues) (Berthon et al. 2007),
    with f_x the normal component and f_y^2 the sum of the tangential squares."""
    d = len(cl.fvec)
    fx = cl.fvec[a]
    fy2 = 0.0
    for b in range(d):
        if b != a:
            fy2 = fy2 + cl.fvec[b] * cl.fvec[b]
    xi = cl.xi
    X = (xi - 1.0) * (xi + 2.0) * (2.0 * (xi - 1.0) * (xi + 2.0) + 3.0 * fy2)
    root = sqrt(where(value(X) > 0.0, X, 0.0))
    half = np.sqrt(2.0) * root / (np.sqrt(3.0) * xi * (xi + 2.0))
    return c * (fx / xi + half), c * (fx / xi - half)


class Scheme:
    """The discretisation of one Problem (seeded_inputs.Problem).

    ``fallback`` (grid-shaped, nonzero = flagged) selects, cell by cell, the
    admissible fallback that Sect. 3.1.3 names for states where the AP + WB
    scheme gives f > 1: a flagged cell takes the centred flux source of
    Eq. (wb_naive), and every face of a flagged cell takes alpha = 1 and the
    wave speeds -c, +c (HLL with the largest speeds the M1 system allows). With
    every cell flagged this is the HLL scheme with fixed speeds and the centred
    source, whose backward-Euler update keeps |F| <= cE when sigma_f >= sigma_a
    (the paper's single sigma). Needs wave speeds frozen at time n or fixed."""

    def __init__(self, prob, fallback=None):
        self.p = prob
        self.d = prob.dim
        self.c = prob.c
        self.dt = prob.dt
        self.dx = prob.dx
        self.shape = prob.shape
        self.N = prob.ncell
        self.nu = prob.n_u
        self.fallback = None
        if fallback is not None and np.any(fallback):
            if prob.implicit_eigs and not prob.fixed_eigs:
                raise ValueError("the fallback needs wave speeds frozen at time n or fixed")
            self.fallback = np.asarray(fallback).reshape(self.shape) != 0
        self.Un = self.unpack(prob.state_vector())
        self.lam_n = [self._speeds_at(self.Un, a) for a in range(self.d)]
        self.alpha = [self._alpha_axis(a) for a in range(self.d)]
        if self.fallback is not None:
            for a in range(self.d):
                m = self._fallback_faces(a)
                lp, lm = self.lam_n[a]
                self.lam_n[a] = (np.where(m, self.c, lp), np.where(m, -self.c, lm))
                self.alpha[a] = np.where(m, 1.0, self.alpha[a])

    def _fallback_faces(self, a: int):
        """Faces along axis a with a flagged cell on either side (a boundary face
        follows its one cell; a periodic face both of its cells)."""
        flag = self.pad_sigma(self.fallback.astype(float), a)
        fL, fR = self.LR(flag, a)
        return (fL > 0) | (fR > 0)

    # ------------------------------------------------------------------ layout
    def ax(self, a: int) -> int:
        """numpy axis of grid axis a (x is the last numpy axis)."""
        return self.d - 1 - a

    def unpack(self, vec) -> list:
        """Flat [E, F_0.., (T)] vector (or Dual) -> list of grid-shaped components."""
        N = self.N
        if isinstance(vec, Dual):
            return [Dual(vec.v[k * N:(k + 1) * N].reshape(self.shape),
                         vec.d[k * N:(k + 1) * N].reshape(self.shape)) for k in range(self.nu)]
        vec = np.asarray(vec, dtype=np.float64)
        return [vec[k * N:(k + 1) * N].reshape(self.shape) for k in range(self.nu)]

    def pack(self, comps) -> np.ndarray:
        return np.concatenate([np.asarray(value(c)).ravel() for c in comps])

    def pack_deriv(self, comps) -> np.ndarray:
        return np.concatenate([np.asarray(du.deriv(c)).ravel() for c in comps])

    # ------------------------------------------------------------------ ghosts
    def _ghost(self, comps, a: int, side: int):
        ax, n = self.ax(a), self.p.n[a]
        kind = self.p.bc[a][side]
        if kind == "periodic":
            src = n - 1 if side == 0 else 0
            return [take(c, [src], ax) for c in comps]
        edge = 0 if side == 0 else n - 1
        g = [take(c, [edge], ax) for c in comps]
        if kind == "reflect":
            g[1 + a] = -g[1 + a]
        elif kind == "dirichlet":
            Eg, Fg, mask = self.p.boundary[(a, side)]
            m = np.expand_dims(np.asarray(mask) != 0, ax)
            g[0] = where(m, np.expand_dims(Eg, ax), g[0])
            for b in range(self.d):
                g[1 + b] = where(m, np.expand_dims(Fg[b], ax), g[1 + b])
        elif kind != "outflow":
            raise ValueError(f"unknown boundary kind {kind}")
        return g

    def pad(self, comps, a: int) -> list:
        """Each component with one ghost layer on both sides along axis a."""
        lo, hi = self._ghost(comps, a, 0), self._ghost(comps, a, 1)
        return [concat([lo[k], comps[k], hi[k]], self.ax(a)) for k in range(len(comps))]

    def pad_sigma(self, s, a: int):
        ax, n = self.ax(a), self.p.n[a]
        if self.p.bc[a][0] == "periodic":
            lo, hi = take(s, [n - 1], ax), take(s, [0], ax)
        else:
            lo, hi = take(s, [0], ax), take(s, [n - 1], ax)
        return concat([lo, s, hi], ax)

    def LR(self, x, a: int):
        """Left/right cell values of every face along axis a of a padded array."""
        ax = self.ax(a)
        return du.slice_axis(x, slice(0, -1), ax), du.slice_axis(x, slice(1, None), ax)

    def diff(self, faces, a: int):
        """faces[i+1/2] - faces[i-1/2] for every cell along axis a."""
        lo, hi = self.LR(faces, a)
        return hi - lo

    # ------------------------------------------------------------ face physics
    def speeds(self, lmaxL, lminL, lmaxR, lminR):
        """lambda+ and lambda- of a face (Sect. 3.1.1), Davis estimate over L and R."""
        if self.p.fixed_eigs:
            one = np.ones(value(lmaxL).shape)
            return self.c * one, -self.c * one
        floor = self.p.lambda_floor
        lp = max_first(max_first(floor, lmaxL), lmaxR)
        lm = min_first(min_first(-floor, lminL), lminR)
        return lp, lm

    def hll(self, a, Pd, cl, lp, lm):
        """HLL interface fluxes along axis a (Sect. 3.1.1): F* and the c^2 P* row
        vector (P*_b for each flux component b)."""
        d, c = self.d, self.c
        den = lp - lm
        ok = value(den) >= TINY_DEN
        inv = where(ok, 1.0 / where(ok, den, 1.0), 0.0)
        EL, ER = self.LR(Pd[0], a)
        FaL, FaR = self.LR(Pd[1 + a], a)
        Fstar = (lp * FaL - lm * FaR) * inv + lp * lm * inv * (ER - EL)
        Pstar = []
        for b in range(d):
            PL, PR = self.LR(cl.pressure(a, b), a)
            FbL, FbR = self.LR(Pd[1 + b], a)
            Pstar.append((c * c * (lp * PL - lm * PR) + lp * lm * (FbR - FbL)) * inv)
        return Fstar, Pstar

    def _speeds_at(self, U, a: int):
        """(lambda+, lambda-) of every face along axis a for the state U."""
        Pd = self.pad(U[:1 + self.d], a)
        cl = Closure(Pd[0], Pd[1:1 + self.d], self.c)
        lmax, lmin = eigenvalues(cl, a, self.c)
        lmaxL, lmaxR = self.LR(lmax, a)
        lminL, lminR = self.LR(lmin, a)
        return self.speeds(lmaxL, lminL, lmaxR, lminR)

    def _alpha_axis(self, a: int):
        """alpha_{i+1/2} of every face along axis a from the time-n state,
        Eq. (asymptoticCorrection); 1 everywhere when the correction is off."""
        p = self.p
        faces_shape = list(self.shape)
        faces_shape[self.ax(a)] += 1
        if not p.ap_correction:
            return np.ones(faces_shape)
        Pd = self.pad(self.Un, a)
        cl = Closure(Pd[0], Pd[1:1 + self.d], self.c)
        lp, lm = self.lam_n[a]
        fL, fR = self.LR(cl.f, a)
        fbar = 0.5 * (fL + fR)
        sL, sR = self.LR(self.pad_sigma(p.sigma_f, a), a)
        sig = 0.5 * (sL + sR)
        den = lp - lm
        ok = den >= TINY_DEN
        term = np.where(ok, lp * lm / (self.c * np.where(ok, den, 1.0)), 0.0)
        return 1.0 / (1.0 - 3.0 * sig * self.dx[a] * (1.0 - fbar * fbar) * term)

    # ------------------------------------------------------------ hyperbolic
    def flux_divergence(self, U, new_level: bool = True):
        """sum_a (alpha F*_{+} - alpha F*_{-})/dx_a and sum_a (P*_{b,+} - P*_{b,-})/dx_a.

        The wave speeds are those of U when ``new_level`` and the problem's
        ``implicit_eigs`` flag are set (eigenvalues at the new time level),
        else the time-n speeds."""
        d = self.d
        divE = 0.0
        divF = [0.0] * d
        for a in range(d):
            Pd = self.pad(U[:1 + d], a)
            cl = Closure(Pd[0], Pd[1:1 + d], self.c)
            if new_level and self.p.implicit_eigs:
                lmax, lmin = eigenvalues(cl, a, self.c)
                lmaxL, lmaxR = self.LR(lmax, a)
                lminL, lminR = self.LR(lmin, a)
                lp, lm = self.speeds(lmaxL, lminL, lmaxR, lminR)
            else:
                lp, lm = self.lam_n[a]
            Fstar, Pstar = self.hll(a, Pd, cl, lp, lm)
            divE = divE + self.diff(self.alpha[a] * Fstar, a) / self.dx[a]
            for b in range(d):
                divF[b] = divF[b] + self.diff(Pstar[b], a) / self.dx[a]
        return divE, divF

    # ------------------------------------------------------------ sources
    def wb_faces(self, U, b: int):
        """Face values Phi = sigma_{i+1/2} F_{b,i+1/2} along axis b, Eq. (wb_smart),
        with Eq. (boundaryCondition) on non-periodic boundary faces."""
        d, p = self.d, self.p
        Pd = self.pad(U[:1 + d], b)
        FL, FR = self.LR(Pd[1 + b], b)
        sL, sR = self.LR(self.pad_sigma(p.sigma_f, b), b)
        Phi = (0.5 * (sL + sR)) * (0.5 * (FL + FR))
        if p.wb_boundary and any(k != "periodic" for k in p.bc[b]):
            cl = Closure(Pd[0], Pd[1:1 + d], self.c)
            Pbb = cl.pressure(b, b)
            PL, PR = self.LR(Pbb, b)
            bnd = -self.c * (PR - PL) / self.dx[b]
            ax, n = self.ax(b), p.n[b]
            parts = []
            parts.append(du.slice_axis(bnd if p.bc[b][0] != "periodic" else Phi, slice(0, 1), ax))
            parts.append(du.slice_axis(Phi, slice(1, n), ax))
            parts.append(du.slice_axis(bnd if p.bc[b][1] != "periodic" else Phi, slice(n, n + 1), ax))
            Phi = concat(parts, ax)
        return Phi

    def flux_source(self, U, b: int):
        """{sigma F_b}_i: Eq. (wb_smart) (well-balanced) or Eq. (wb_naive); flagged
        fallback cells take Eq. (wb_naive)."""
        naive = self.p.sigma_f * U[1 + b]
        if self.p.well_balanced:
            Phi = self.wb_faces(U, b)
            lo, hi = self.LR(Phi, b)
            wb = 0.5 * (hi + lo)
            return wb if self.fallback is None else where(self.fallback, naive, wb)
        return naive

    def emission(self, U):
        """a_r T^4 (gas coupled) or the frozen emission field B."""
        if self.p.gas:
            T = U[1 + self.d]
            return self.p.a_r * T * T * T * T
        return self.p.B

    # ------------------------------------------------------------ residual
    def residual_comps(self, U):
        """Backward-Euler residual of Sect. 3.1.1 (components, grid-shaped)."""
        p, d, dt, c = self.p, self.d, self.dt, self.c
        Un = self.Un
        divE, divF = self.flux_divergence(U)
        exch = c * p.sigma_a * dt * (self.emission(U) - U[0])
        RE = U[0] - Un[0] + dt * divE - exch
        if p.S is not None:
            RE = RE - dt * p.S
        R = [RE]
        for b in range(d):
            R.append(U[1 + b] - Un[1 + b] + dt * divF[b] + c * dt * self.flux_source(U, b))
        if p.gas:
            R.append(p.rho_cv * (U[1 + d] - Un[1 + d]) + exch)
        return R

    def residual(self, u: np.ndarray) -> np.ndarray:
        return self.pack(self.residual_comps(self.unpack(u)))

    def jv(self, u: np.ndarray, v: np.ndarray) -> np.ndarray:
        """J(u) v: the dual part of the residual at Dual(u, v)."""
        return self.pack_deriv(self.residual_comps(self.unpack(Dual(u, v))))

    def diag_blocks(self, u: np.ndarray) -> np.ndarray:
        """Point blocks J_ii = dR_i/dU_i, shape (N, n_u, n_u), [cell, row, col].

        Cells are coloured so that no two cells of one colour are axis
        neighbours (wrap included); seeding component k of every cell of one
        colour then gives column k of each seeded cell's own block.
        """
        d, N, nu = self.d, self.N, self.nu
        mods = []
        for a in range(d):
            n = self.p.n[a]
            m = 2
            if "periodic" in self.p.bc[a]:
                while n > 1 and (n - 1) % m == 0 and m < n:
                    m += 1
            mods.append(m)
        coords = np.indices(self.shape)  # numpy-axis order
        blocks = np.zeros((N, nu, nu))
        for color in np.ndindex(*mods):
            sel = np.ones(self.shape, dtype=bool)
            for a in range(d):
                sel &= (coords[self.ax(a)] % mods[a]) == color[a]
            idx = np.flatnonzero(sel.ravel())
            if idx.size == 0:
                continue
            for k in range(nu):
                v = np.zeros(nu * N)
                v[k * N + idx] = 1.0
                jv = self.jv(u, v).reshape(nu, N)
                blocks[idx, :, k] = jv[:, idx].T
        return blocks

    # ------------------------------------------------------------ semi-implicit step
    def explicit_step(self):
        """One semi-implicit step (Sect. 3.1): HLL fluxes and alpha at time n,
        implicit energy exchange, implicit (WB or centred) flux source."""
        p, d, dt, c = self.p, self.d, self.dt, self.c
        Un = self.Un
        divE, divF = self.flux_divergence(Un, new_level=False)
        Es = Un[0] - dt * divE
        if p.S is not None:
            Es = Es + dt * p.S
        k = c * p.sigma_a * dt
        out = [None] * self.nu
        if p.gas:
            T = self._gas_temperature(Es, Un[1 + d], k)
            out[0] = (Es + k * p.a_r * T ** 4) / (1.0 + k)
            out[1 + d] = T
        else:
            out[0] = (Es + k * p.B) / (1.0 + k)
        for b in range(d):
            Fs = Un[1 + b] - dt * divF[b]
            if p.well_balanced:
                out[1 + b] = self._wb_implicit_solve(Fs, b)
            else:
                out[1 + b] = Fs / (1.0 + c * dt * p.sigma_f)
        return out

    def _gas_temperature(self, Es, Tn, k):
        """Root T of rho c_v (T - T^n) + k/(1+k) (a_r T^4 - E*) = 0 per cell
        (backward-Euler exchange of Eqs. momentModel/internalEnergyEqua with
        E eliminated); Newton from the upper bound max(T^n, (E*/a_r)^(1/4))."""
        p = self.p
        w = k / (1.0 + k)
        T = np.maximum(Tn, (np.maximum(Es, 0.0) / p.a_r) ** 0.25)
        for _ in range(200):
            g = p.rho_cv * (T - Tn) + w * (p.a_r * T ** 4 - Es)
            dg = p.rho_cv + 4.0 * w * p.a_r * T ** 3
            step = g / dg
            T = T - step
            if np.all(np.abs(step) <= 1e-15 * np.abs(T)):
                break
        return T

    def _wb_implicit_solve(self, Fs, b: int):
        """Solve (I + c dt W_b) F_b = F*_b, W_b the WB operator along axis b
        (Appendix B form, r = c sigma_{j+1/2} dt / 4), one sparse solve."""
        p, dt, c = self.p, self.dt, self.c
        ax, n = self.ax(b), p.n[b]
        N = self.N
        ids = np.arange(N).reshape(self.shape)
        sig = p.sigma_f
        rows, cols, vals = [ids.ravel()], [ids.ravel()], [np.ones(N)]
        rhs = np.array(Fs, dtype=np.float64).copy()
        # interior (and periodic) faces: face between cell j and its +1 neighbour
        nf = n if p.bc[b][1] == "periodic" else n - 1
        for j in range(nf):
            jp = (j + 1) % n
            iL = np.take(ids, [j], ax).ravel()
            iR = np.take(ids, [jp], ax).ravel()
            r = c * dt * 0.5 * (np.take(sig, [j], ax) + np.take(sig, [jp], ax)).ravel() / 4.0
            for i_row in (iL, iR):
                rows += [i_row, i_row]
                cols += [iL, iR]
                vals += [r, r]
        # boundary faces of non-periodic sides
        Fn = [self.Un[k] for k in range(self.nu)]
        for side in (0, 1):
            kind = p.bc[b][side]
            if kind == "periodic":
                continue
            edge = 0 if side == 0 else n - 1
            ie = np.take(ids, [edge], ax).ravel()
            if p.wb_boundary:
                # Eq. (boundaryCondition) with the pressures at time n
                g = self._ghost(Fn[:1 + self.d], b, side)
                inner = [np.take(x, [edge], ax) for x in Fn[:1 + self.d]]
                clg = Closure(g[0], g[1:], c)
                cli = Closure(inner[0], inner[1:], c)
                Pg, Pi = clg.pressure(b, b), cli.pressure(b, b)
                Phi = -c * (Pi - Pg) / self.dx[b] if side == 0 else -c * (Pg - Pi) / self.dx[b]
                rhs_flat = rhs.reshape(-1)
                rhs_flat[ie] -= 0.5 * c * dt * np.asarray(Phi).ravel()
                rhs = rhs_flat.reshape(self.shape)
            else:
                r = c * dt * np.take(sig, [edge], ax).ravel() / 4.0
                rows.append(ie); cols.append(ie)
                if kind == "outflow":
                    vals.append(2.0 * r)
                elif kind == "reflect":
                    # the ghost's normal flux is -F_b: the face average vanishes
                    vals.append(0.0 * r)
                elif kind == "dirichlet":
                    Eg, Fg, mask = p.boundary[(b, side)]
                    m = (np.asarray(mask) != 0).ravel()
                    vals.append(np.where(m, r, 2.0 * r))
                    rhs_flat = rhs.reshape(-1)
                    rhs_flat[ie] -= np.where(m, r * np.asarray(Fg[b]).ravel(), 0.0)
                    rhs = rhs_flat.reshape(self.shape)
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N))
        x = spla.spsolve(A.tocsc(), rhs.ravel())
        return x.reshape(self.shape)

    # ------------------------------------------------------------ advection by the gas flow
    def advect_internal_energy(self, u_faces):
        """Explicit first-order upwind transport of e = rho c_v T by prescribed face
        velocities (the frozen-hydrodynamics stand-in of the operator split of
        Sect. 3.2, step 1): e* = e - dt sum_a (u e_up)_{+} - (u e_up)_{-} / dx_a,
        e_up the upwind cell value (ghost rules of the state: copy / wrap).
        Returns T* = e* / (rho c_v)."""
        p, d = self.p, self.d
        e = p.rho_cv * self.Un[1 + d]
        div = 0.0
        for a in range(d):
            ep = self.pad_sigma(e, a)  # copy (outflow/reflect/Dirichlet) or wrap (periodic)
            eL, eR = self.LR(ep, a)
            u = np.asarray(u_faces[a])
            flux = np.where(u > 0.0, u * eL, u * eR)
            div = div + self.diff(flux, a) / self.dx[a]
        return (e - self.dt * div) / p.rho_cv

    def velocity_sources(self, u_faces):
        """Explicit velocity-dependent radiation sources over dt (Sect. 2.1 with the first-order
        expansion in u/c; applied explicitly after the implicit step, step 3 of the splitting of
        Sect. 2.3). Cell velocity u = mean of the two face velocities along each axis; with the
        closure pressure P of the current state, B = a_r T^4 (gas) or the frozen emission, and
        sigma the flux opacity:
            S_E = (sigma / c) u.F + (sigma / c) E |u|^2 + (sigma / c) u.(P u)
            S_F = sigma P u + sigma B u + (sigma / c^2) u (u.F)
            E' = E + dt S_E,  F' = F + c dt S_F,  rho c_v T' = rho c_v T - dt S_E (gas).
        Returns the new state as a list of components."""
        p, d, c, dt = self.p, self.d, self.c, self.dt
        U = [np.array(x, dtype=float) for x in self.Un]
        E, F = U[0], U[1:1 + d]
        u = []
        for a in range(d):
            lo, hi = self.LR(np.asarray(u_faces[a], dtype=float), a)  # the two faces of every cell
            u.append(0.5 * (lo + hi))
        cl = Closure(E, F, c)
        Pu = [sum(cl.pressure(a, b) * u[b] for b in range(d)) for a in range(d)]
        uF = sum(u[a] * F[a] for a in range(d))
        uu = sum(u[a] * u[a] for a in range(d))
        uPu = sum(u[a] * Pu[a] for a in range(d))
        sig = np.asarray(p.sigma_f, dtype=float)
        B = p.a_r * U[1 + d] ** 4 if p.gas else np.asarray(p.B, dtype=float)
        SE = (sig / c) * uF + (sig / c) * E * uu + (sig / c) * uPu
        out = [E + dt * SE]
        for a in range(d):
            SF = sig * Pu[a] + sig * B * u[a] + (sig / c ** 2) * u[a] * uF
            out.append(F[a] + c * dt * SF)
        if p.gas:
            out.append(U[1 + d] - dt * SE / np.asarray(p.rho_cv, dtype=float))
        return out

    # ------------------------------------------------------------ diagnostics
    def realizability_violations(self, u) -> int:
        """Number of cells with |F| > c E (admissibility is not guaranteed, Sect. 3.1.3)."""
        U = self.unpack(u)
        F2 = sum(np.asarray(U[1 + b]) ** 2 for b in range(self.d))
        return int(np.count_nonzero(np.sqrt(F2) > self.c * U[0]))

    def inadmissible(self, u) -> np.ndarray:
        """Grid-shaped mask of the cells outside the admissible set: E <= 0 or
        |F| > c E (Sect. 2.2: f = |F| / (cE) must not exceed 1)."""
        U = self.unpack(u)
        F2 = sum(np.asarray(U[1 + b]) ** 2 for b in range(self.d))
        E = np.asarray(U[0])
        return ~(E > 0.0) | (np.sqrt(F2) > self.c * E)
