// m1_device.cuh — device-side discretisation of the grey M1 step.
//
// One template family evaluates, for one cell, the backward-Euler residual of
// the scheme of Bloch et al. (A&A 2021) Sect. 3.1.1:
//   R_E = E - E^n + dt sum_a (alpha F*_{a,+} - alpha F*_{a,-}) / dx_a
//         - c sigma_a dt (emission - E) - dt S
//   R_F = F - F^n + dt sum_a (P*_{a,+} - P*_{a,-}) / dx_a + c dt {sigma F}
//   R_T = rho c_v (T - T^n) + c sigma_a dt (a_r T^4 - E)          (gas coupling)
// with the M1 closure of Sect. 2.2, the eigenvalues of Eq. (eigenvalues), the
// HLL fluxes of Sect. 3.1.1, alpha of Eq. (asymptoticCorrection) (precomputed
// at time n) and the well-balanced source of Eqs. (wb_smart, boundaryCondition).
//
// The scalar type S is either the real type R (double or float) or Dual<R>
// (forward-mode dual numbers), so the same code gives R(U), J(U) v (seed v
// everywhere) and the point blocks J_ii (seed one own-cell component).
// Non-smooth points: max/min keep the first argument on ties in the order
// (floor, left, right); sqrt(0) has derivative 0; an active clamp |f| <= 1 has
// zero derivative in |f|.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "m1_df.cuh"

namespace m1 {

// ---------------------------------------------------------------- dual numbers
template <class R>
struct Dual {
    R v, d;
};

// RealOf: the real type of the arithmetic; MemOf: the type of the arrays in
// memory (double for the double-word arithmetic DF of the FP64 path)
template <class S> struct RealOf { using type = S; };
template <class R> struct RealOf<Dual<R>> { using type = R; };
template <class S> struct MemOf { using type = typename RealOf<S>::type; };
template <> struct MemOf<DF> { using type = double; };
template <> struct MemOf<Dual<DF>> { using type = double; };

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ float val(float x) { return x; }
__device__ __forceinline__ DF val(DF x) { return x; }
template <class R> __device__ __forceinline__ R val(const Dual<R>& x) { return x.v; }

// a value of the arithmetic as the array type M
template <class M> __device__ __forceinline__ M to_mem(double x) { return (M)x; }
template <class M> __device__ __forceinline__ M to_mem(float x) { return (M)x; }
template <class M> __device__ __forceinline__ M to_mem(DF x) { return (M)df_to_double(x); }
__device__ __forceinline__ double dbl(double x) { return x; }
__device__ __forceinline__ double dbl(float x) { return x; }
__device__ __forceinline__ double dbl(DF x) { return df_to_double(x); }
__device__ __forceinline__ float to_f32(double x) { return (float)x; }
__device__ __forceinline__ float to_f32(DF x) { return x.hi; }  // hi = RN(hi + lo)

template <class S> __device__ __forceinline__ S cst(typename RealOf<S>::type x);
template <> __device__ __forceinline__ double cst<double>(double x) { return x; }
template <> __device__ __forceinline__ float cst<float>(float x) { return x; }
template <> __device__ __forceinline__ DF cst<DF>(DF x) { return x; }
template <> __device__ __forceinline__ Dual<double> cst<Dual<double>>(double x) { return {x, 0.0}; }
template <> __device__ __forceinline__ Dual<float> cst<Dual<float>>(float x) { return {x, 0.0f}; }
template <> __device__ __forceinline__ Dual<DF> cst<Dual<DF>>(DF x) { return {x, DF(0.0f, 0.0f)}; }

template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.d + b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.d - b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a) { return {-a.v, -a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
    R q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, R b) { return {a.v + b, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator+(R a, Dual<R> b) { return {a + b.v, b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, R b) { return {a.v - b, a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(R a, Dual<R> b) { return {a - b.v, -b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, R b) { return {a.v * b, a.d * b}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(R a, Dual<R> b) { return {a * b.v, a * b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, R b) { return {a.v / b, a.d / b}; }
template <class R> __device__ __forceinline__ Dual<R> operator/(R a, Dual<R> b) {
    R q = a / b.v;
    return {q, -q * b.d / b.v};
}

// dual double-words against plain doubles (grid scalars and arrays)
__device__ __forceinline__ Dual<DF> operator+(Dual<DF> a, double b) { return a + DF(b); }
__device__ __forceinline__ Dual<DF> operator+(double a, Dual<DF> b) { return DF(a) + b; }
__device__ __forceinline__ Dual<DF> operator-(Dual<DF> a, double b) { return a - DF(b); }
__device__ __forceinline__ Dual<DF> operator-(double a, Dual<DF> b) { return DF(a) - b; }
__device__ __forceinline__ Dual<DF> operator*(Dual<DF> a, double b) { return a * DF(b); }
__device__ __forceinline__ Dual<DF> operator*(double a, Dual<DF> b) { return DF(a) * b; }
__device__ __forceinline__ Dual<DF> operator/(Dual<DF> a, double b) { return a / DF(b); }
__device__ __forceinline__ Dual<DF> operator/(double a, Dual<DF> b) { return DF(a) / b; }

__device__ __forceinline__ double msqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float msqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ DF msqrt(DF x) { return df_sqrt(x); }
template <class R> __device__ __forceinline__ Dual<R> msqrt(Dual<R> x) {
    R s = msqrt(x.v);
    return {s, s > R(0) ? x.d / (R(2) * s) : R(0)};
}

template <class S> __device__ __forceinline__ S sel(bool c, const S& a, const S& b) { return c ? a : b; }
// max/min that keep the first argument unless the second is strictly larger/smaller
template <class S> __device__ __forceinline__ S max_first(const S& a, const S& b) { return val(b) > val(a) ? b : a; }
template <class S> __device__ __forceinline__ S min_first(const S& a, const S& b) { return val(b) < val(a) ? b : a; }

template <class R> struct Tiny;
template <> struct Tiny<double> {
    static __device__ __forceinline__ double e() { return 1e-300; }
    static __device__ __forceinline__ double den() { return 1e-300; }
};
template <> struct Tiny<float> {
    static __device__ __forceinline__ float e() { return 1e-30f; }
    static __device__ __forceinline__ float den() { return 1e-30f; }
};
template <> struct Tiny<DF> {
    static __device__ __forceinline__ DF e() { return DF(1e-30f, 0.0f); }
    static __device__ __forceinline__ DF den() { return DF(1e-30f, 0.0f); }
};

// 1 / x for a positive wave-speed difference: IEEE division in FP64; in FP32 the
// hardware reciprocal (__fdividef, within 2 ulp), ample for the FP32 operator
template <class R> __device__ __forceinline__ R recip_den(R x);
template <> __device__ __forceinline__ double recip_den<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float recip_den<float>(float x) { return __fdividef(1.0f, x); }
template <> __device__ __forceinline__ DF recip_den<DF>(DF x) { return DF(1.0f, 0.0f) / x; }

// ---------------------------------------------------------------- grid data
enum { BC_OUTFLOW = 0, BC_PERIODIC = 1, BC_REFLECT = 2, BC_DIRICHLET = 3 };

// Everything a stencil kernel needs, passed by value. Arrays of type R are
// the precision of the kernel (double for the FP64 path, float for the FP32
// inner path); face arrays hold n_a + 1 faces along axis a.
template <class R>
struct Dev {
    int dim, nx, ny, nz;
    long long N;
    int n[3];
    long long stride[3];
    R dx[3], inv_dx[3];
    R c, a_r, dt, lambda_floor;
    int bc[3][2];
    int gas, wb, ap, fixed_eigs, wb_boundary, implicit_eigs;
    const R* sig_a;
    const R* sig_f;
    const R* B;       // frozen emission (no gas), may be null
    const R* S;       // source, may be null
    const R* rho_cv;  // gas only
    const R* Un;      // time-n state (n_u * N)
    const R* alpha[3];
    const R* lam_p[3];  // time-n lambda+ per face
    const R* lam_m[3];  // time-n lambda- per face
    const R* bE[3][2];
    const R* bF[3][2];  // dim * M
    const unsigned char* bmask[3][2];
    long long bM[3];    // cells per face of axis a
    // admissibility fallback (implicit step): nonzero = the cell takes the
    // centred flux source of Eq. (wb_naive); its faces carry alpha = 1 and
    // speeds -c, +c in the face arrays. Null: no cell is flagged.
    const unsigned char* fb;
    // FP64 residual and J v (Dev<double> only): nonzero = computed in the
    // double-word arithmetic DF (m1_df.cuh) instead of FP64 operations
    int df;
};

__device__ __forceinline__ long long face_index(const int* n, const int* coord, int a, int fa) {
    if (a == 0) return ((long long)coord[2] * n[1] + coord[1]) * (n[0] + 1) + fa;
    if (a == 1) return ((long long)coord[2] * (n[1] + 1) + fa) * n[0] + coord[0];
    return ((long long)fa * n[1] + coord[1]) * n[0] + coord[0];
}

// index of the cell within the boundary face of axis a (x fastest over the other axes)
__device__ __forceinline__ long long bface_cell(const int* n, const int* coord, int a) {
    if (a == 0) return (long long)coord[2] * n[1] + coord[1];
    if (a == 1) return (long long)coord[2] * n[0] + coord[0];
    return (long long)coord[1] * n[0] + coord[0];
}

// ---------------------------------------------------------------- state, closure
template <class S, int DIM>
struct St {
    S E;
    S F[DIM];
    S T;
};

template <class S, int DIM>
struct Cl {
    S f[DIM];   // reduced flux f = F / (c E) (direction kept, |f| clamped to 1)
    S f2;       // |f|^2
    S xi;       // sqrt(4 - 3 f^2)
    S iso;      // (1 - chi) / 2
    S g;        // (3 chi - 1) / (2 f^2) = 3 / (2 + xi)
    S E;
};

// M1 closure, Sect. 2.2: chi = (3 + 4 f^2) / (5 + 2 xi), D = (1-chi)/2 I + g f(x)f.
template <class S, int DIM>
__device__ __forceinline__ Cl<S, DIM> closure(const St<S, DIM>& u, typename RealOf<S>::type c) {
    using R = typename RealOf<S>::type;
    Cl<S, DIM> k;
    S Es = sel(val(u.E) > Tiny<R>::e(), u.E, cst<S>(Tiny<R>::e()));
    S cE = c * Es;
    S F2 = u.F[0] * u.F[0];
#pragma unroll
    for (int b = 1; b < DIM; ++b) F2 = F2 + u.F[b] * u.F[b];
    const bool clamped = val(F2) > val(cE) * val(cE);
    S den = clamped ? msqrt(F2) : cE;
    S inv = R(1) / den;
#pragma unroll
    for (int b = 0; b < DIM; ++b) k.f[b] = u.F[b] * inv;
    S f2 = k.f[0] * k.f[0];
#pragma unroll
    for (int b = 1; b < DIM; ++b) f2 = f2 + k.f[b] * k.f[b];
    k.f2 = clamped ? cst<S>(R(1)) : f2;
    k.xi = msqrt(R(4) - R(3) * k.f2);
    S chi = (R(3) + R(4) * k.f2) / (R(5) + R(2) * k.xi);
    k.iso = (R(1) - chi) * R(0.5);
    k.g = R(3) / (R(2) + k.xi);
    k.E = u.E;
    return k;
}

template <class S, int DIM>
__device__ __forceinline__ S pressure(const Cl<S, DIM>& k, int a, int b) {
    S t = k.g * k.f[a] * k.f[b];
    if (a == b) t = t + k.iso;
    return t * k.E;
}

// M1 eigenvalues along axis a, Eq. (eigenvalues), with f_x the normal and f_y^2
// the tangential part of f; xi - 1 is formed as 3 (1 - f^2) / (xi + 1).
template <class S, int DIM>
__device__ __forceinline__ void eigen(const Cl<S, DIM>& k, int a, typename RealOf<S>::type c, S& lmax, S& lmin) {
    using R = typename RealOf<S>::type;
    S fx = k.f[a];
    S fy2 = cst<S>(R(0));
#pragma unroll
    for (int b = 0; b < DIM; ++b)
        if (b != a) fy2 = fy2 + k.f[b] * k.f[b];
    S xm1 = R(3) * (R(1) - k.f2) / (k.xi + R(1));
    S xp2 = k.xi + R(2);
    S X = xm1 * xp2 * (R(2) * xm1 * xp2 + R(3) * fy2);
    S root = val(X) > R(0) ? msqrt(X) : cst<S>(R(0));
    const R s23 = R(0.81649658092772603273);  // sqrt(2) / sqrt(3)
    S half = s23 * root / (k.xi * xp2);
    S mid = fx / k.xi;
    lmax = c * (mid + half);
    lmin = c * (mid - half);
}

// ---------------------------------------------------------------- loaders
// Loaders read arrays of type R and give values of the arithmetic type A
// (R itself, or the double-word DF for R = double)
template <class R, class A = R>
struct LoadPlain {
    const R* U;
    long long N;
    __device__ __forceinline__ A get(int comp, long long idx, long long) const { return A(U[comp * N + idx]); }
};
template <class R, class A = R>
struct LoadDir {  // U + eps v
    const R* U;
    const R* v;
    long long N;
    __device__ __forceinline__ Dual<A> get(int comp, long long idx, long long) const {
        return {A(U[comp * N + idx]), A(v[comp * N + idx])};
    }
};
template <class R, class A = R>
struct LoadSeed {  // seed component k of the own cell only
    const R* U;
    long long N;
    int k;
    __device__ __forceinline__ Dual<A> get(int comp, long long idx, long long own) const {
        return {A(U[comp * N + idx]), (idx == own && comp == k) ? A(1) : A(0)};
    }
};

template <class S, int DIM, bool GAS, class L>
__device__ __forceinline__ St<S, DIM> load_state(const L& ld, long long idx, long long own) {
    St<S, DIM> u;
    u.E = ld.get(0, idx, own);
#pragma unroll
    for (int b = 0; b < DIM; ++b) u.F[b] = ld.get(1 + b, idx, own);
    if constexpr (GAS) u.T = ld.get(1 + DIM, idx, own);
    return u;
}

// Neighbour of the cell along axis a (side 0 = low, 1 = high), ghost rules of
// the physical boundaries: outflow = copy, periodic = wrap, reflect = copy with
// F_a negated, Dirichlet = the given (E, F) where the face mask is set.
template <class S, int DIM, bool GAS, class R, class L>
__device__ __forceinline__ St<S, DIM> neighbour(const Dev<R>& g, const L& ld, const St<S, DIM>& self,
                                                long long idx, const int* coord, int a, int side,
                                                R& sig_nb, bool& boundary) {
    const int ca = coord[a] + (side ? 1 : -1);
    boundary = false;
    if (ca >= 0 && ca < g.n[a]) {
        long long j = idx + (side ? g.stride[a] : -g.stride[a]);
        sig_nb = g.sig_f[j];
        return load_state<S, DIM, GAS>(ld, j, idx);
    }
    const int kind = g.bc[a][side];
    if (kind == BC_PERIODIC) {
        long long j = idx + (side ? -(long long)(g.n[a] - 1) * g.stride[a] : (long long)(g.n[a] - 1) * g.stride[a]);
        sig_nb = g.sig_f[j];
        return load_state<S, DIM, GAS>(ld, j, idx);
    }
    boundary = true;
    sig_nb = g.sig_f[idx];
    St<S, DIM> u = self;
    if (kind == BC_REFLECT) {
        u.F[a] = cst<S>(R(0)) - u.F[a];
    } else if (kind == BC_DIRICHLET) {
        long long m = bface_cell(g.n, coord, a);
        const unsigned char* mk = g.bmask[a][side];
        if (mk == nullptr || mk[m]) {
            u.E = cst<S>(g.bE[a][side][m]);
#pragma unroll
            for (int b = 0; b < DIM; ++b) u.F[b] = cst<S>(g.bF[a][side][b * g.bM[a] + m]);
        }
    }
    return u;
}

// HLL interface fluxes of Sect. 3.1.1 along axis a between L and R.
template <class S, int DIM>
__device__ __forceinline__ void hll(const St<S, DIM>& uL, const St<S, DIM>& uR, const Cl<S, DIM>& kL,
                                    const Cl<S, DIM>& kR, const S& lp, const S& lm, int a,
                                    typename RealOf<S>::type c, S& Fs, S* Ps) {
    using R = typename RealOf<S>::type;
    S den = lp - lm;
    const bool ok = val(den) >= Tiny<R>::den();
    S inv = ok ? R(1) / den : cst<S>(R(0));
    S pm = lp * lm * inv;
    Fs = (lp * uL.F[a] - lm * uR.F[a]) * inv + pm * (uR.E - uL.E);
    const R c2 = c * c;
#pragma unroll
    for (int b = 0; b < DIM; ++b)
        Ps[b] = c2 * (lp * pressure(kL, a, b) - lm * pressure(kR, a, b)) * inv + pm * (uR.F[b] - uL.F[b]);
}

template <class S>
__device__ __forceinline__ void wave_speeds(const S& lmaxL, const S& lminL, const S& lmaxR, const S& lminR,
                                            typename RealOf<S>::type floor, S& lp, S& lm) {
    using R = typename RealOf<S>::type;
    lp = max_first(max_first(cst<S>(floor), lmaxL), lmaxR);
    lm = min_first(min_first(cst<S>(R(0) - floor), lminL), lminR);
}

// ---------------------------------------------------------------- the cell residual
// Residual components of cell idx (coord = its (x, y, z) indices) for the
// state given by the loader; out[0] = R_E, out[1 + b] = R_F_b, out[1 + DIM] = R_T.
template <class S, int DIM, bool GAS, class R, class L>
__device__ __forceinline__ void cell_residual(const Dev<R>& g, const L& ld, long long idx, const int* coord,
                                              S* out) {
    const St<S, DIM> self = load_state<S, DIM, GAS>(ld, idx, idx);
    const Cl<S, DIM> ks = closure(self, g.c);
    const R sig_self = g.sig_f[idx];
    const R dt = g.dt;
    const bool wbc = g.wb && !(g.fb && g.fb[idx]);  // well-balanced source in this cell
    S RE = self.E - g.Un[idx];
    S RF[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) RF[b] = self.F[b] - g.Un[(1 + b) * g.N + idx];
    S phi[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) phi[b] = cst<S>(R(0));

#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        S lmaxS, lminS;
        if (g.implicit_eigs && !g.fixed_eigs) eigen(ks, a, g.c, lmaxS, lminS);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            R sig_nb;
            bool boundary;
            const St<S, DIM> nb = neighbour<S, DIM, GAS>(g, ld, self, idx, coord, a, side, sig_nb, boundary);
            const Cl<S, DIM> kn = closure(nb, g.c);
            const St<S, DIM>& uL = side ? self : nb;
            const St<S, DIM>& uR = side ? nb : self;
            const Cl<S, DIM>& kL = side ? ks : kn;
            const Cl<S, DIM>& kR = side ? kn : ks;
            const int fa = coord[a] + side;
            const long long fidx = face_index(g.n, coord, a, fa);
            S lp, lm;
            if (g.fixed_eigs) {
                lp = cst<S>(g.c);
                lm = cst<S>(R(0) - g.c);
            } else if (g.implicit_eigs) {
                S lmaxN, lminN;
                eigen(kn, a, g.c, lmaxN, lminN);
                if (side)
                    wave_speeds(lmaxS, lminS, lmaxN, lminN, g.lambda_floor, lp, lm);
                else
                    wave_speeds(lmaxN, lminN, lmaxS, lminS, g.lambda_floor, lp, lm);
            } else {
                lp = cst<S>(g.lam_p[a][fidx]);
                lm = cst<S>(g.lam_m[a][fidx]);
            }
            S Fs, Ps[DIM];
            hll(uL, uR, kL, kR, lp, lm, a, g.c, Fs, Ps);
            const R w = (side ? dt : -dt) * g.inv_dx[a];
            RE = RE + (w * g.alpha[a][fidx]) * Fs;
#pragma unroll
            for (int b = 0; b < DIM; ++b) RF[b] = RF[b] + w * Ps[b];
            if (wbc) {
                if (boundary && g.wb_boundary) {
                    // Eq. (boundaryCondition): sigma F at the face = -c (P_R - P_L) / dx
                    phi[a] = phi[a] - g.c * g.inv_dx[a] * (pressure(kR, a, a) - pressure(kL, a, a));
                } else {
                    phi[a] = phi[a] + (R(0.25) * (sig_self + sig_nb)) * (uL.F[a] + uR.F[a]);
                }
            }
        }
    }
    const R cdt = g.c * dt;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
        S src = wbc ? R(0.5) * phi[b] : sig_self * self.F[b];
        RF[b] = RF[b] + cdt * src;
    }
    S emis;
    if constexpr (GAS) {
        S T2 = self.T * self.T;
        emis = g.a_r * (T2 * T2);
    } else {
        emis = cst<S>(g.B ? g.B[idx] : R(0));
    }
    S exch = (cdt * g.sig_a[idx]) * (emis - self.E);
    RE = RE - exch;
    if (g.S) RE = RE - dt * g.S[idx];
    out[0] = RE;
#pragma unroll
    for (int b = 0; b < DIM; ++b) out[1 + b] = RF[b];
    if constexpr (GAS) out[1 + DIM] = g.rho_cv[idx] * (self.T - g.Un[(1 + DIM) * g.N + idx]) + exch;
}

// lambda+-(U^n) and alpha (Eq. asymptoticCorrection with f_{i+1/2} = (f_i + f_{i+1})/2
// and sigma_{i+1/2} = (sigma_i + sigma_{i+1})/2) of face f of axis a (faces
// indexed like cells with n_a + 1 along a).
// A: the arithmetic (double, or the double-word DF)
template <int DIM, class A = double>
__device__ __forceinline__ void face_time_n(const Dev<double>& g, int a, long long f, double& lp_out,
                                            double& lm_out, double& al_out) {
    int fn[3] = {g.n[0], g.n[1], g.n[2]};
    fn[a] += 1;
    int coord[3];
    {
        long long q = f / fn[0];
        coord[0] = (int)(f - q * fn[0]);
        coord[2] = (int)(q / fn[1]);
        coord[1] = (int)(q - (long long)coord[2] * fn[1]);
    }
    const int fa = coord[a];
    LoadPlain<double, A> ld{g.Un, g.N};
    // the cell on the right of the face unless the face is the high boundary
    int cc[3] = {coord[0], coord[1], coord[2]};
    const bool high = (fa == g.n[a]);
    cc[a] = high ? g.n[a] - 1 : fa;
    const long long idx = ((long long)cc[2] * g.n[1] + cc[1]) * g.n[0] + cc[0];
    St<A, DIM> self = load_state<A, DIM, false>(ld, idx, idx);
    double sig_nb;
    bool bnd;
    St<A, DIM> nb;
    if (high) {
        nb = neighbour<A, DIM, false>(g, ld, self, idx, cc, a, 1, sig_nb, bnd);
    } else if (fa == 0) {
        nb = neighbour<A, DIM, false>(g, ld, self, idx, cc, a, 0, sig_nb, bnd);
    } else {
        const long long j = idx - g.stride[a];
        nb = load_state<A, DIM, false>(ld, j, idx);
        sig_nb = g.sig_f[j];
    }
    const St<A, DIM>& uL = high ? self : nb;
    const St<A, DIM>& uR = high ? nb : self;
    const Cl<A, DIM> kL = closure(uL, g.c), kR = closure(uR, g.c);
    A lp, lm;
    if (g.fixed_eigs) {
        lp = A(g.c);
        lm = A(-g.c);
    } else {
        A xL, nL, xR, nR;
        eigen(kL, a, g.c, xL, nL);
        eigen(kR, a, g.c, xR, nR);
        wave_speeds(xL, nL, xR, nR, g.lambda_floor, lp, lm);
    }
    A al = A(1);
    if (g.ap) {
        const A fbar = A(0.5) * (msqrt(kL.f2) + msqrt(kR.f2));
        const A sig = A(0.5) * (A(g.sig_f[idx]) + A(sig_nb));
        const A den = lp - lm;
        const A term = den >= Tiny<A>::den() ? lp * lm / (A(g.c) * den) : A(0);
        al = A(1) / (A(1) - A(3) * sig * A(g.dx[a]) * (A(1) - fbar * fbar) * term);
    }
    lp_out = dbl(lp);
    lm_out = dbl(lm);
    al_out = dbl(al);
}

// Gauss-Jordan inverse with partial pivoting of one NU x NU block (FP64);
// false (and x = I) when a pivot vanishes.
__device__ __forceinline__ double absval(double x) { return fabs(x); }
__device__ __forceinline__ DF absval(DF x) { return x.hi < 0.0f ? -x : x; }

template <int NU, class T = double>
__device__ __forceinline__ bool invert_block(T (&a)[NU][NU], T (&x)[NU][NU]) {
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
        for (int c = 0; c < NU; ++c) x[r][c] = (r == c) ? T(1) : T(0);
    bool bad = false;
#pragma unroll
    for (int col = 0; col < NU; ++col) {
        int piv = col;
        T best = absval(a[col][col]);
#pragma unroll
        for (int r = col + 1; r < NU; ++r)
            if (absval(a[r][col]) > best) {
                best = absval(a[r][col]);
                piv = r;
            }
        if (!(best > T(0))) bad = true;
#pragma unroll
        for (int r = col + 1; r < NU; ++r) {
            if (r == piv) {
#pragma unroll
                for (int c = 0; c < NU; ++c) {
                    T t = a[col][c];
                    a[col][c] = a[r][c];
                    a[r][c] = t;
                    t = x[col][c];
                    x[col][c] = x[r][c];
                    x[r][c] = t;
                }
            }
        }
        const T inv = bad ? T(0) : T(1) / a[col][col];
#pragma unroll
        for (int c = 0; c < NU; ++c) {
            a[col][c] = a[col][c] * inv;
            x[col][c] = x[col][c] * inv;
        }
#pragma unroll
        for (int r = 0; r < NU; ++r) {
            if (r == col) continue;
            const T m = a[r][col];
#pragma unroll
            for (int c = 0; c < NU; ++c) {
                a[r][c] = a[r][c] - m * a[col][c];
                x[r][c] = x[r][c] - m * x[col][c];
            }
        }
    }
    if (bad) {
#pragma unroll
        for (int r = 0; r < NU; ++r)
#pragma unroll
            for (int c = 0; c < NU; ++c) x[r][c] = (r == c) ? T(1) : T(0);
    }
    return !bad;
}

__device__ __forceinline__ void cell_coord(long long idx, int nx, int ny, int* coord) {
    long long q = idx / nx;
    coord[0] = (int)(idx - q * nx);
    coord[2] = (int)(q / ny);
    coord[1] = (int)(q - (long long)coord[2] * ny);
}

}  // namespace m1
