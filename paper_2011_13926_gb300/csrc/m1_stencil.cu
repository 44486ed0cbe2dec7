// m1_stencil.cu — stencil kernels of the grey M1 step (residual, J v, point
// blocks, time-n face data, block Jacobi, semi-implicit step).
//
// One thread per cell (or face, or grid line). All loads of a field are
// coalesced along x; neighbours along y/z are the same field offset by a row
// or plane, so a warp's loads stay contiguous.
#include <stdio.h>

#include "m1_internal.h"

#include <algorithm>
#include <type_traits>

namespace m1 {

static constexpr int kThreads = 256;

// Range guard of the double-word residual: a cell whose residual is not
// finite or exceeds 2^100 (where FP32's exponent range, and with it the
// double-word arithmetic, runs out) makes its block's partial sum +inf, so
// that the host sees a non-finite norm and recomputes in FP64
__device__ __forceinline__ void df_range_guard(double, double&) {}
__device__ __forceinline__ void df_range_guard(float, double&) {}
__device__ __forceinline__ void df_range_guard(DF o, double& ss) {
    if (!(fabsf(o.hi) <= 0x1p100f)) ss = __longlong_as_double(0x7ff0000000000000LL);
}

int stencil_blocks(long long N) { return (int)((N + kThreads - 1) / kThreads); }

// ------------------------------------------------------------------ time-n faces
template <int DIM, class A>
__global__ void k_faces_time_n(Dev<double> g, int a, double* lam_p, double* lam_m, double* alpha) {
    const long long nfaces = g.N / g.n[a] * (g.n[a] + 1);
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfaces) return;
    double lp, lm, al;
    face_time_n<DIM, A>(g, a, f, lp, lm, al);
    lam_p[f] = lp;
    lam_m[f] = lm;
    alpha[f] = al;
}

void launch_faces_time_n(const Dev<double>& g, double* const lam_p[3], double* const lam_m[3],
                         double* const alpha[3], cudaStream_t s) {
    for (int a = 0; a < g.dim; ++a) {
        const long long nf = g.N / g.n[a] * (g.n[a] + 1);
        const int nb = (int)((nf + kThreads - 1) / kThreads);
#define FACES(D, A) k_faces_time_n<D, A><<<nb, kThreads, 0, s>>>(g, a, lam_p[a], lam_m[a], alpha[a])
        if (g.df) {
            switch (g.dim) {
                case 1: FACES(1, DF); break;
                case 2: FACES(2, DF); break;
                default: FACES(3, DF); break;
            }
        } else {
            switch (g.dim) {
                case 1: FACES(1, double); break;
                case 2: FACES(2, double); break;
                default: FACES(3, double); break;
            }
        }
#undef FACES
    }
}

// ------------------------------------------------------------------ block reduction helpers
// sum over a block of nthreads threads (any shape; tid the linear thread
// index, nthreads a multiple of 32), fixed order; valid in tid 0
__device__ __forceinline__ double block_sum_linear(double v, int tid, int nthreads) {
    __shared__ double red_l[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = tid & 31, w = tid >> 5;
    if (lane == 0) red_l[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (nthreads >> 5) ? red_l[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// sum over a one-dimensional block; valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// ------------------------------------------------------------------ residual
// A: the arithmetic (double, or the double-word DF on FP64 arrays)
template <class A, int DIM, bool GAS>
__global__ void __launch_bounds__(kThreads, std::is_same<A, DF>::value ? 3 : 1)
    k_residual(Dev<double> g, const double* __restrict__ U,
                                                       double* __restrict__ Rout, double* partials) {
    constexpr int NU = 1 + DIM + (GAS ? 1 : 0);
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double ss = 0.0;
    if (idx < g.N) {
        int coord[3];
        cell_coord(idx, g.n[0], g.n[1], coord);
        LoadPlain<double, A> ld{U, g.N};
        A out[NU];
        cell_residual<A, DIM, GAS>(g, ld, idx, coord, out);
#pragma unroll
        for (int k = 0; k < NU; ++k) {
            const double o = dbl(out[k]);
            Rout[k * g.N + idx] = o;
            ss += o * o;
        }
#pragma unroll
        for (int k = 0; k < NU; ++k) df_range_guard(out[k], ss);
    }
    if (partials) {
        const double t = block_sum(ss);
        if (threadIdx.x == 0) partials[blockIdx.x] = t;
    }
}

// ------------------------------------------------------------------ J v
// R: the arrays (double or float); A: the arithmetic (R, or DF on FP64 arrays)
template <class R, class A, int DIM, bool GAS>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 1)
    k_jv(Dev<R> g, const R* __restrict__ U, const R* __restrict__ v, R* __restrict__ Jv) {
    constexpr int NU = 1 + DIM + (GAS ? 1 : 0);
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int coord[3];
    cell_coord(idx, g.n[0], g.n[1], coord);
    LoadDir<R, A> ld{U, v, g.N};
    Dual<A> out[NU];
    cell_residual<Dual<A>, DIM, GAS>(g, ld, idx, coord, out);
#pragma unroll
    for (int k = 0; k < NU; ++k) Jv[k * g.N + idx] = to_mem<R>(out[k].d);
}

// ------------------------------------------------------------------ 2D tiled residual and J v
// 2D residual (MODE kTileResidual, S = R), J v by dual numbers (kTileJvDual,
// S = Dual<R>, the derivative parts) or J v from the pressure Jacobian
// frozen at the Newton iterate (kTileJvLinear, S = R) with the closure of
// every cell computed once per CTA: a 32 x 8 tile plus a one-cell halo (axis
// neighbours only; ghosts by the boundary rules) is staged in shared memory
// as (E, F, P), then each thread forms its four HLL faces and the sources in
// the order of cell_residual. Terms that do not depend on U (U^n, the
// emission B, the source S) enter the residual only: they carry no
// derivative. For frozen (time-n) or fixed wave speeds, where J v is linear
// in v but for dP = (dP/dU) v; kTileJvLinear reads dP/dU (from
// k_pressure_jacobian2d) for the cells of the domain and takes the ghosts by
// dual numbers through the boundary rules. The residual variant also writes
// the block's partial sum of squares.
constexpr int kTX = 32, kTY = 8;
constexpr int kTileResidual = 0, kTileJvDual = 1, kTileJvLinear = 2, kTileJvLinearPre = 3;
// level 0 of the multigrid cycle (radiation only): down = pre-smoothing
// z = omega M^-1 r (written), residual r - J z and its 2 x 2 restriction;
// up = z + P zc, residual, post-smoothing into zout
constexpr int kTileMgDown0 = 4, kTileMgUp0 = 5;

template <class R>
struct TileMg {
    const R* r = nullptr;   // level-0 right-hand side
    const R* z = nullptr;   // up: the pre-smoothed iterate
    const R* zc = nullptr;  // up: the level-1 correction
    int nxc = 0, nyc = 0;   // level-1 sizes
    R* rc = nullptr;        // down: level-1 right-hand side
    R* zout = nullptr;      // down: z; up: the smoothed iterate
    R omega = R(0);
};

// Loader of U + eps (z + P zc) for the ghosts of the multigrid up pass
template <class R>
struct LoadProlong {
    const R* U;
    const R* z;
    const R* zc;
    long long N, Nc;
    int nx, nxc;
    __device__ __forceinline__ Dual<R> get(int comp, long long idx, long long) const {
        const long long I = (long long)((idx / nx) / 2) * nxc + (idx % nx) / 2;
        return {U[comp * N + idx], z[comp * N + idx] + zc[comp * Nc + I]};
    }
};

template <class S>
struct CellT {
    S E, Fx, Fy, Pxx, Pxy, Pyy;
};

// dP/dU of one cell in 2D: row r of (Pxx, Pxy, Pyy), column c of (E, Fx, Fy)
// at pj[(3 r + c) N + idx]; with gas, d(a_r T^4)/dT at pj[9 N + idx]; in the
// precision R of the J v that applies it
template <class R, bool GAS>
__global__ void __launch_bounds__(kThreads) k_pressure_jacobian2d(Dev<R> g, const R* __restrict__ U,
                                                                   R* __restrict__ pj) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long N = g.N;
    const R E = U[idx], Fx = U[N + idx], Fy = U[2 * N + idx];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        St<Dual<R>, 2> u;
        u.E = Dual<R>{E, c == 0 ? R(1) : R(0)};
        u.F[0] = Dual<R>{Fx, c == 1 ? R(1) : R(0)};
        u.F[1] = Dual<R>{Fy, c == 2 ? R(1) : R(0)};
        const Cl<Dual<R>, 2> k = closure(u, g.c);
        pj[(3 * 0 + c) * N + idx] = pressure(k, 0, 0).d;
        pj[(3 * 1 + c) * N + idx] = pressure(k, 0, 1).d;
        pj[(3 * 2 + c) * N + idx] = pressure(k, 1, 1).d;
    }
    if constexpr (GAS) {
        const R T = U[3 * N + idx];
        pj[9 * N + idx] = R(4) * g.a_r * T * T * T;
    }
}

// Loader of U + eps M^-1 v for the fused preconditioned J v: the direction
// at a cell is its point-block inverse (NU x NU, row-major planes) times v
template <class R, int NU>
struct LoadPre {
    const R* U;
    const R* v;
    const R* binv;
    long long N;
    __device__ __forceinline__ Dual<R> get(int comp, long long idx, long long) const {
        R z = R(0);
#pragma unroll
        for (int c = 0; c < NU; ++c) z += binv[(long long)(comp * NU + c) * N + idx] * v[(long long)c * N + idx];
        return {U[comp * N + idx], z};
    }
};

// FP32 instantiations are held to 64 registers (four CTAs per SM): they are
// bound by global-load latency, and occupancy hides it
// double-word instantiations at three CTAs per SM: their dependent FP32 chains
// need the warps
template <class S, bool GAS, int MODE>
__global__ void __launch_bounds__(kTX* kTY, std::is_same<typename RealOf<S>::type, float>::value
                                                ? 4
                                                : (std::is_same<typename RealOf<S>::type, DF>::value ? 3 : 1))
    k_stencil2d_tiled(Dev<typename MemOf<S>::type> g, const typename MemOf<S>::type* __restrict__ U,
                      const typename MemOf<S>::type* __restrict__ v, const typename MemOf<S>::type* __restrict__ pj,
                      const typename MemOf<S>::type* __restrict__ binv, typename MemOf<S>::type* __restrict__ out,
                      double* __restrict__ partials, TileMg<typename MemOf<S>::type> mgp) {
    using R = typename RealOf<S>::type;  // arithmetic
    using M = typename MemOf<S>::type;   // arrays
    constexpr bool RES = MODE == kTileResidual;
    constexpr bool MGD = MODE == kTileMgDown0, MGU = MODE == kTileMgUp0;
    constexpr bool LIN = MODE == kTileJvLinear || MODE == kTileJvLinearPre || MGD || MGU;
    constexpr bool PRE = MODE == kTileJvLinearPre || MGD;
    static_assert(!(MGD || MGU) || !GAS, "the fused multigrid level 0 is radiation only");
    constexpr int NU = GAS ? 4 : 3;
    static_assert((MODE == kTileJvDual) == std::is_same<S, Dual<R>>::value, "dual numbers only for kTileJvDual");
    __shared__ CellT<S> cs[kTY + 2][kTX + 2];
    const int nx = g.n[0], ny = g.n[1];
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const long long N = g.N;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    // this thread's cell and its face data, loaded before the halo so that
    // their latency overlaps the staging
    const int ix = x0 + threadIdx.x, iy = y0 + threadIdx.y;
    const bool valid = ix < nx && iy < ny;
    const long long idx = valid ? (long long)iy * nx + ix : 0;
    const int coord[3] = {ix, iy, 0};
    R sig_self = R(0), sig_nb[2][2], lpf[2][2], lmf[2][2], alf[2][2];
    bool wbc = g.wb;  // well-balanced source in this cell (the fallback takes the centred one)
    if (valid) {
        if (g.fb) wbc = wbc && !g.fb[idx];
        // the cell's faces: x-faces ix -+ 1/2 at fx, fx + 1 (nx + 1 per row); y-faces
        // iy -+ 1/2 at fy, fy + nx
        const long long fx = (long long)iy * (nx + 1) + ix, fy = idx;
        sig_self = g.sig_f[idx];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int ca = coord[a] + (side ? 1 : -1);
                const bool inside = ca >= 0 && ca < g.n[a];
                const bool periodic = g.bc[a][side] == BC_PERIODIC;
                R sn = sig_self;
                if (inside)
                    sn = g.sig_f[idx + (side ? g.stride[a] : -g.stride[a])];
                else if (periodic)
                    sn = g.sig_f[idx + (side ? -(long long)(g.n[a] - 1) : (long long)(g.n[a] - 1)) * g.stride[a]];
                sig_nb[a][side] = sn;
                const long long fidx = a == 0 ? fx + side : fy + (side ? nx : 0);
                if (g.fixed_eigs) {
                    lpf[a][side] = g.c;
                    lmf[a][side] = -g.c;
                } else {
                    lpf[a][side] = g.lam_p[a][fidx];
                    lmf[a][side] = g.lam_m[a][fidx];
                }
                alf[a][side] = g.alpha[a][fidx];
            }
        }
    }
    for (int t = tid; t < (kTX + 2) * (kTY + 2); t += kTX * kTY) {
        const int hx = t % (kTX + 2), hy = t / (kTX + 2);
        int gx = x0 + hx - 1, gy = y0 + hy - 1;
        const bool in_x = gx >= 0 && gx < nx, in_y = gy >= 0 && gy < ny;
        if (!(in_x || in_y)) continue;              // corner: no face needs it
        if (gx > nx || gy > ny) continue;           // beyond the last ghost of a ragged tile
        if ((hx == 0 || hx == kTX + 1) && (hy == 0 || hy == kTY + 1)) continue;  // tile corners
        CellT<S> c;
        bool staged = false;
        if constexpr (LIN) {
            if (in_x && in_y) {
                staged = true;
                const long long k = (long long)gy * nx + gx;
                R z[3];
                if constexpr (MGU) {  // z + P zc
                    const long long Nc = (long long)mgp.nxc * mgp.nyc;
                    const long long I = (long long)(gy / 2) * mgp.nxc + gx / 2;
#pragma unroll
                    for (int r = 0; r < 3; ++r) z[r] = mgp.z[r * N + k] + mgp.zc[r * Nc + I];
                } else if constexpr (PRE) {  // z = M^-1 v at this cell (rows E, Fx, Fy of the block inverse)
                    R vv[NU];
#pragma unroll
                    for (int q = 0; q < NU; ++q) vv[q] = v[q * N + k];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        R acc = R(0);
#pragma unroll
                        for (int q = 0; q < NU; ++q) acc += binv[(long long)(r * NU + q) * N + k] * vv[q];
                        z[r] = acc;
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 3; ++r) z[r] = v[r * N + k];
                }
                c.E = z[0];
                c.Fx = z[1];
                c.Fy = z[2];
                R d[3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    d[r] = pj[(3 * r) * N + k] * z[0] + pj[(3 * r + 1) * N + k] * z[1] + pj[(3 * r + 2) * N + k] * z[2];
                c.Pxx = d[0];
                c.Pxy = d[1];
                c.Pyy = d[2];
            }
        }
        if (!staged) {
            // residual: plain values; dual J v: dual numbers; linear J v: the
            // ghosts by dual numbers through the boundary rules
            using SD = std::conditional_t<RES, R, Dual<R>>;
            using L = std::conditional_t<
                RES, LoadPlain<M, R>,
                std::conditional_t<PRE, LoadPre<R, NU>, std::conditional_t<MGU, LoadProlong<R>, LoadDir<M, R>>>>;
            L ld;
            if constexpr (RES) {
                ld = L{U, N};
            } else if constexpr (PRE) {
                ld = L{U, v, binv, N};
            } else if constexpr (MGU) {
                ld = L{U, mgp.z, mgp.zc, N, (long long)mgp.nxc * mgp.nyc, nx, mgp.nxc};
            } else {
                ld = L{U, v, N};
            }
            St<SD, 2> u;
            if (in_x && in_y) {
                const long long k = (long long)gy * nx + gx;
                u = load_state<SD, 2, false>(ld, k, k);
            } else {
                // ghost of the adjacent boundary cell along the axis that left the domain
                const int a = in_x ? 1 : 0;
                const int side = a == 0 ? (gx < 0 ? 0 : 1) : (gy < 0 ? 0 : 1);
                int cc[3] = {a == 0 ? (gx < 0 ? 0 : nx - 1) : gx, a == 1 ? (gy < 0 ? 0 : ny - 1) : gy, 0};
                const long long k = (long long)cc[1] * nx + cc[0];
                const St<SD, 2> self = load_state<SD, 2, false>(ld, k, k);
                M sn;
                bool bnd;
                u = neighbour<SD, 2, false>(g, ld, self, k, cc, a, side, sn, bnd);
            }
            const Cl<SD, 2> k = closure(u, g.c);
            if constexpr (LIN) {
                c.E = u.E.d;
                c.Fx = u.F[0].d;
                c.Fy = u.F[1].d;
                c.Pxx = pressure(k, 0, 0).d;
                c.Pxy = pressure(k, 0, 1).d;
                c.Pyy = pressure(k, 1, 1).d;
            } else {
                c.E = u.E;
                c.Fx = u.F[0];
                c.Fy = u.F[1];
                c.Pxx = pressure(k, 0, 0);
                c.Pxy = pressure(k, 0, 1);
                c.Pyy = pressure(k, 1, 1);
            }
        }
        cs[hy][hx] = c;
    }
    __syncthreads();
    double ss = 0.0;
    R mg_res[3] = {R(0), R(0), R(0)};
    if (valid) {
        const CellT<S>& me = cs[threadIdx.y + 1][threadIdx.x + 1];
        const R dt = g.dt, c = g.c, c2 = g.c * g.c;
        S RE = me.E, RFx = me.Fx, RFy = me.Fy;
        if constexpr (RES) {
            RE = RE - g.Un[idx];
            RFx = RFx - g.Un[N + idx];
            RFy = RFy - g.Un[2 * N + idx];
        }
        S phi[2] = {cst<S>(R(0)), cst<S>(R(0))};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int hx = threadIdx.x + 1 + (a == 0 ? (side ? 1 : -1) : 0);
                const int hy = threadIdx.y + 1 + (a == 1 ? (side ? 1 : -1) : 0);
                const CellT<S>& nb = cs[hy][hx];
                const CellT<S>& Lc = side ? me : nb;
                const CellT<S>& Rc = side ? nb : me;
                const int ca = coord[a] + (side ? 1 : -1);
                const bool inside = ca >= 0 && ca < g.n[a];
                const bool periodic = g.bc[a][side] == BC_PERIODIC;
                const bool boundary = !inside && !periodic;
                const R lp = lpf[a][side], lm = lmf[a][side];
                const R den = lp - lm;
                const R inv = den >= Tiny<R>::den() ? recip_den<R>(den) : R(0);
                const R pm = lp * lm * inv;
                const S FaL = a == 0 ? Lc.Fx : Lc.Fy, FaR = a == 0 ? Rc.Fx : Rc.Fy;
                const S Fs = (lp * FaL - lm * FaR) * inv + pm * (Rc.E - Lc.E);
                // P*_b = c^2 (lp P_ab,L - lm P_ab,R) inv + pm (F_b,R - F_b,L)
                const S PaxL = a == 0 ? Lc.Pxx : Lc.Pxy, PaxR = a == 0 ? Rc.Pxx : Rc.Pxy;
                const S PayL = a == 0 ? Lc.Pxy : Lc.Pyy, PayR = a == 0 ? Rc.Pxy : Rc.Pyy;
                const S Psx = c2 * (lp * PaxL - lm * PaxR) * inv + pm * (Rc.Fx - Lc.Fx);
                const S Psy = c2 * (lp * PayL - lm * PayR) * inv + pm * (Rc.Fy - Lc.Fy);
                const R w = (side ? dt : -dt) * g.inv_dx[a];
                RE = RE + (w * alf[a][side]) * Fs;
                RFx = RFx + w * Psx;
                RFy = RFy + w * Psy;
                if (wbc) {
                    if (boundary && g.wb_boundary) {
                        const S PR = a == 0 ? Rc.Pxx : Rc.Pyy, PL = a == 0 ? Lc.Pxx : Lc.Pyy;
                        phi[a] = phi[a] - c * g.inv_dx[a] * (PR - PL);
                    } else {
                        phi[a] = phi[a] + (R(0.25) * (sig_self + sig_nb[a][side])) * (FaL + FaR);
                    }
                }
            }
        }
        const R cdt = c * dt;
        if (wbc) {
            RFx = RFx + cdt * (R(0.5) * phi[0]);
            RFy = RFy + cdt * (R(0.5) * phi[1]);
        } else {
            RFx = RFx + cdt * (sig_self * me.Fx);
            RFy = RFy + cdt * (sig_self * me.Fy);
        }
        S emis;
        S T;
        if constexpr (GAS) {
            if constexpr (MODE == kTileJvDual) {
                T = S{U[3 * N + idx], v[3 * N + idx]};
            } else if constexpr (MODE == kTileJvLinear) {
                T = v[3 * N + idx];
            } else if constexpr (PRE) {
                R acc = R(0);
#pragma unroll
                for (int q = 0; q < NU; ++q) acc += binv[(long long)(3 * NU + q) * N + idx] * v[q * N + idx];
                T = acc;
            } else {
                T = U[3 * N + idx];
            }
            if constexpr (LIN) {
                emis = pj[9 * N + idx] * T;
            } else {
                const S T2 = T * T;
                emis = g.a_r * (T2 * T2);
            }
        } else {
            emis = cst<S>(RES && g.B ? g.B[idx] : R(0));
        }
        const S exch = (cdt * g.sig_a[idx]) * (emis - me.E);
        RE = RE - exch;
        if constexpr (MODE == kTileJvDual) {
            out[idx] = to_mem<M>(RE.d);
            out[N + idx] = to_mem<M>(RFx.d);
            out[2 * N + idx] = to_mem<M>(RFy.d);
            if constexpr (GAS) out[3 * N + idx] = to_mem<M>((g.rho_cv[idx] * T + exch).d);
        } else if constexpr (MGD) {
            // z = omega z', residual r - omega J z' (kept for the restriction)
            const R zr[3] = {me.E, me.Fx, me.Fy}, jz[3] = {RE, RFx, RFy};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                mgp.zout[q * N + idx] = mgp.omega * zr[q];
                mg_res[q] = mgp.r[q * N + idx] - mgp.omega * jz[q];
            }
        } else if constexpr (MGU) {
            // zout = zz + omega M^-1 (r - J zz)
            const R zz[3] = {me.E, me.Fx, me.Fy}, jz[3] = {RE, RFx, RFy};
            R res[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) res[q] = mgp.r[q * N + idx] - jz[q];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                R a = R(0);
#pragma unroll
                for (int c2i = 0; c2i < 3; ++c2i) a += binv[(long long)(q * 3 + c2i) * N + idx] * res[c2i];
                mgp.zout[q * N + idx] = zz[q] + mgp.omega * a;
            }
        } else if constexpr (LIN) {
            out[idx] = RE;
            out[N + idx] = RFx;
            out[2 * N + idx] = RFy;
            if constexpr (GAS) out[3 * N + idx] = g.rho_cv[idx] * T + exch;
        } else {
            if (g.S) RE = RE - dt * g.S[idx];
            df_range_guard(RE, ss);
            df_range_guard(RFx, ss);
            df_range_guard(RFy, ss);
            const double oE = dbl(RE), oFx = dbl(RFx), oFy = dbl(RFy);
            out[idx] = oE;
            out[N + idx] = oFx;
            out[2 * N + idx] = oFy;
            ss += oE * oE + oFx * oFx + oFy * oFy;
            if constexpr (GAS) {
                const S RT = g.rho_cv[idx] * (T - g.Un[3 * N + idx]) + exch;
                df_range_guard(RT, ss);
                const double oT = dbl(RT);
                out[3 * N + idx] = oT;
                ss += oT * oT;
            }
        }
    }
    if constexpr (RES) {
        if (partials) {
            const double t = block_sum_linear(ss, tid, kTX * kTY);
            if (tid == 0) partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    }
    if constexpr (MGD) {
        // 2 x 2 aggregates of the tile (origins even): the root thread sums them
        __shared__ R rs[kTY][kTX][3];
#pragma unroll
        for (int q = 0; q < 3; ++q) rs[threadIdx.y][threadIdx.x][q] = mg_res[q];
        __syncthreads();
        const int tx = threadIdx.x, ty = threadIdx.y;
        if ((tx & 1) == 0 && (ty & 1) == 0 && valid) {
            const long long Nc = (long long)mgp.nxc * mgp.nyc;
            const long long I = (long long)(iy / 2) * mgp.nxc + ix / 2;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                mgp.rc[q * Nc + I] = (rs[ty][tx][q] + rs[ty][tx + 1][q]) + (rs[ty + 1][tx][q] + rs[ty + 1][tx + 1][q]);
        }
    }
}

// ------------------------------------------------------------------ point blocks
template <class R, int DIM, bool GAS>
__global__ void __launch_bounds__(kThreads) k_diag(Dev<R> g, const R* __restrict__ U, R* __restrict__ blocks) {
    constexpr int NU = 1 + DIM + (GAS ? 1 : 0);
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int coord[3];
    cell_coord(idx, g.n[0], g.n[1], coord);
    for (int k = 0; k < NU; ++k) {
        LoadSeed<R> ld{U, g.N, k};
        Dual<R> out[NU];
        cell_residual<Dual<R>, DIM, GAS>(g, ld, idx, coord, out);
#pragma unroll
        for (int r = 0; r < NU; ++r) blocks[(long long)(r * NU + k) * g.N + idx] = out[r].d;
    }
}

#define M1_DISPATCH(DIMV, GASV, CALL) \
    do {                              \
        if ((DIMV) == 1) {            \
            if (GASV) {               \
                CALL(1, true);        \
            } else {                  \
                CALL(1, false);       \
            }                         \
        } else if ((DIMV) == 2) {     \
            if (GASV) {               \
                CALL(2, true);        \
            } else {                  \
                CALL(2, false);       \
            }                         \
        } else {                      \
            if (GASV) {               \
                CALL(3, true);        \
            } else {                  \
                CALL(3, false);       \
            }                         \
        }                             \
    } while (0)

static bool tiled2d(const Dev<double>& g) { return g.dim == 2 && !(g.implicit_eigs && !g.fixed_eigs); }

long long residual_partial_count(int dim, const int n[3]) {
    const long long N = (long long)n[0] * n[1] * n[2];
    long long nb = stencil_blocks(N);
    if (dim == 2) nb = std::max(nb, (long long)((n[0] + kTX - 1) / kTX) * ((n[1] + kTY - 1) / kTY));
    return nb;
}

template <class A>
static int residual_f64(const Dev<double>& g, const double* U, double* R, double* partials, long long capacity,
                        cudaStream_t s) {
    if (tiled2d(g)) {
        const dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY), block(kTX, kTY);
        const long long nb = (long long)grid.x * grid.y;
        if (!partials || nb <= capacity) {
            if (g.gas)
                k_stencil2d_tiled<A, true, kTileResidual><<<grid, block, 0, s>>>(g, U, nullptr, nullptr, nullptr, R,
                                                                                partials, {});
            else
                k_stencil2d_tiled<A, false, kTileResidual><<<grid, block, 0, s>>>(g, U, nullptr, nullptr, nullptr, R,
                                                                                 partials, {});
            return (int)nb;
        }
    }
    const int nb = stencil_blocks(g.N);
#define CALL(D, G) k_residual<A, D, G><<<nb, kThreads, 0, s>>>(g, U, R, partials)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
    return nb;
}

int launch_residual_f64(const Dev<double>& g, const double* U, double* R, double* partials, long long capacity,
                        cudaStream_t s) {
    return g.df ? residual_f64<DF>(g, U, R, partials, capacity, s) : residual_f64<double>(g, U, R, partials, capacity, s);
}

// S: Dual<R>, or Dual<DF> on FP64 arrays
template <class S>
static bool jv_tiled(const Dev<typename MemOf<S>::type>& g, const typename MemOf<S>::type* U,
                     const typename MemOf<S>::type* v, typename MemOf<S>::type* Jv, cudaStream_t s) {
    if (g.dim != 2 || (g.implicit_eigs && !g.fixed_eigs)) return false;
    dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY), block(kTX, kTY);
    if (g.gas)
        k_stencil2d_tiled<S, true, kTileJvDual><<<grid, block, 0, s>>>(g, U, v, nullptr, nullptr, Jv, nullptr, {});
    else
        k_stencil2d_tiled<S, false, kTileJvDual><<<grid, block, 0, s>>>(g, U, v, nullptr, nullptr, Jv, nullptr, {});
    return true;
}

bool jv_linear_available(const Dev<double>& g) { return tiled2d(g); }

int pressure_jacobian_size(const Dev<double>& g) { return 9 + (g.gas ? 1 : 0); }

template <class R>
static void pressure_jacobian_launch(const Dev<R>& g, const R* U, R* pj, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
    if (g.gas)
        k_pressure_jacobian2d<R, true><<<nb, kThreads, 0, s>>>(g, U, pj);
    else
        k_pressure_jacobian2d<R, false><<<nb, kThreads, 0, s>>>(g, U, pj);
}
void launch_pressure_jacobian_f64(const Dev<double>& g, const double* U, double* pj, cudaStream_t s) {
    pressure_jacobian_launch<double>(g, U, pj, s);
}
void launch_pressure_jacobian_f32(const Dev<float>& g, const float* U, float* pj, cudaStream_t s) {
    pressure_jacobian_launch<float>(g, U, pj, s);
}

template <class R>
static void jv_linear(const Dev<R>& g, const R* U, const R* pj, const R* binv, const R* v, R* Jv, cudaStream_t s) {
    const dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY), block(kTX, kTY);
    if (binv) {
        if (g.gas)
            k_stencil2d_tiled<R, true, kTileJvLinearPre><<<grid, block, 0, s>>>(g, U, v, pj, binv, Jv, nullptr, {});
        else
            k_stencil2d_tiled<R, false, kTileJvLinearPre><<<grid, block, 0, s>>>(g, U, v, pj, binv, Jv, nullptr, {});
    } else {
        if (g.gas)
            k_stencil2d_tiled<R, true, kTileJvLinear><<<grid, block, 0, s>>>(g, U, v, pj, nullptr, Jv, nullptr, {});
        else
            k_stencil2d_tiled<R, false, kTileJvLinear><<<grid, block, 0, s>>>(g, U, v, pj, nullptr, Jv, nullptr, {});
    }
}
void launch_jv_linear_f64(const Dev<double>& g, const double* U, const double* pj, const double* v, double* Jv,
                          cudaStream_t s) {
    jv_linear<double>(g, U, pj, nullptr, v, Jv, s);
}
void launch_jv_linear_f32(const Dev<float>& g, const float* U, const float* pj, const float* v, float* Jv,
                          cudaStream_t s) {
    jv_linear<float>(g, U, pj, nullptr, v, Jv, s);
}
void launch_jv_linear_pre_f32(const Dev<float>& g, const float* U, const float* pj, const float* binv,
                              const float* v, float* Jv, cudaStream_t s) {
    jv_linear<float>(g, U, pj, binv, v, Jv, s);
}

void launch_mg_down0_f32(const Dev<float>& g, const float* U, const float* pj, const float* binv, const float* r,
                         float omega, float* z, int nxc, int nyc, float* rc, cudaStream_t s) {
    const dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY), block(kTX, kTY);
    TileMg<float> m;
    m.r = r;
    m.nxc = nxc;
    m.nyc = nyc;
    m.rc = rc;
    m.zout = z;
    m.omega = omega;
    k_stencil2d_tiled<float, false, kTileMgDown0><<<grid, block, 0, s>>>(g, U, r, pj, binv, nullptr, nullptr, m);
}

void launch_mg_up0_f32(const Dev<float>& g, const float* U, const float* pj, const float* binv, const float* r,
                       const float* z, const float* zc, int nxc, int nyc, float omega, float* zout, cudaStream_t s) {
    const dim3 grid((g.n[0] + kTX - 1) / kTX, (g.n[1] + kTY - 1) / kTY), block(kTX, kTY);
    TileMg<float> m;
    m.r = r;
    m.z = z;
    m.zc = zc;
    m.nxc = nxc;
    m.nyc = nyc;
    m.zout = zout;
    m.omega = omega;
    k_stencil2d_tiled<float, false, kTileMgUp0><<<grid, block, 0, s>>>(g, U, nullptr, pj, binv, nullptr, nullptr, m);
}

void launch_jv_f64(const Dev<double>& g, const double* U, const double* v, double* Jv, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
    if (g.df) {
        if (jv_tiled<Dual<DF>>(g, U, v, Jv, s)) return;
#define CALL(D, G) k_jv<double, DF, D, G><<<nb, kThreads, 0, s>>>(g, U, v, Jv)
        M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
        return;
    }
    if (jv_tiled<Dual<double>>(g, U, v, Jv, s)) return;
#define CALL(D, G) k_jv<double, double, D, G><<<nb, kThreads, 0, s>>>(g, U, v, Jv)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
}

void launch_jv_f32(const Dev<float>& g, const float* U, const float* v, float* Jv, cudaStream_t s) {
    if (jv_tiled<Dual<float>>(g, U, v, Jv, s)) return;
    const int nb = stencil_blocks(g.N);
#define CALL(D, G) k_jv<float, float, D, G><<<nb, kThreads, 0, s>>>(g, U, v, Jv)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
}

void launch_diag_f64(const Dev<double>& g, const double* U, double* blocks, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
#define CALL(D, G) k_diag<double, D, G><<<nb, kThreads, 0, s>>>(g, U, blocks)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
}

void launch_diag_f32(const Dev<float>& g, const float* U, float* blocks, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
#define CALL(D, G) k_diag<float, D, G><<<nb, kThreads, 0, s>>>(g, U, blocks)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
}

// ------------------------------------------------------------------ block inverse / apply
// Gauss-Jordan with partial pivoting on each cell's NU x NU block (FP64).
template <int NU, class B>
__global__ void k_block_inverse(long long N, const B* __restrict__ blocks, double* __restrict__ binv64,
                                float* __restrict__ binv32, int* singular) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // FP32 blocks (the mixed path's) are inverted in double words, FP64 ones in FP64
    using T = std::conditional_t<std::is_same<B, float>::value, DF, double>;
    T a[NU][NU], x[NU][NU];
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
        for (int c = 0; c < NU; ++c) a[r][c] = T(blocks[(long long)(r * NU + c) * N + i]);
    if (!invert_block<NU, T>(a, x)) atomicAdd(singular, 1);
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
        for (int c = 0; c < NU; ++c) {
            const double xv = dbl(x[r][c]);
            binv64[(long long)(r * NU + c) * N + i] = xv;
            if (binv32) binv32[(long long)(r * NU + c) * N + i] = to_f32(x[r][c]);
        }
}

template <class B>
static void block_inverse(int nu, long long N, const B* blocks, double* binv64, float* binv32, int* singular,
                          cudaStream_t s) {
    const int nb = stencil_blocks(N);
    switch (nu) {
        case 2: k_block_inverse<2, B><<<nb, kThreads, 0, s>>>(N, blocks, binv64, binv32, singular); break;
        case 3: k_block_inverse<3, B><<<nb, kThreads, 0, s>>>(N, blocks, binv64, binv32, singular); break;
        case 4: k_block_inverse<4, B><<<nb, kThreads, 0, s>>>(N, blocks, binv64, binv32, singular); break;
        default: k_block_inverse<5, B><<<nb, kThreads, 0, s>>>(N, blocks, binv64, binv32, singular); break;
    }
}
void launch_block_inverse(int nu, long long N, const double* blocks, double* binv64, float* binv32, int* singular,
                          cudaStream_t s) {
    block_inverse<double>(nu, N, blocks, binv64, binv32, singular, s);
}
void launch_block_inverse_f32(int nu, long long N, const float* blocks, double* binv64, float* binv32,
                              int* singular, cudaStream_t s) {
    block_inverse<float>(nu, N, blocks, binv64, binv32, singular, s);
}

template <class R, int NU>
__global__ void k_bj_apply(long long N, const R* __restrict__ binv, const R* __restrict__ r, R* __restrict__ z) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    R rr[NU];
#pragma unroll
    for (int c = 0; c < NU; ++c) rr[c] = r[(long long)c * N + i];
#pragma unroll
    for (int q = 0; q < NU; ++q) {
        R acc = R(0);
#pragma unroll
        for (int c = 0; c < NU; ++c) acc += binv[(long long)(q * NU + c) * N + i] * rr[c];
        z[(long long)q * N + i] = acc;
    }
}

template <class R>
static void bj_apply(int nu, long long N, const R* binv, const R* r, R* z, cudaStream_t s) {
    const int nb = stencil_blocks(N);
    switch (nu) {
        case 2: k_bj_apply<R, 2><<<nb, kThreads, 0, s>>>(N, binv, r, z); break;
        case 3: k_bj_apply<R, 3><<<nb, kThreads, 0, s>>>(N, binv, r, z); break;
        case 4: k_bj_apply<R, 4><<<nb, kThreads, 0, s>>>(N, binv, r, z); break;
        default: k_bj_apply<R, 5><<<nb, kThreads, 0, s>>>(N, binv, r, z); break;
    }
}
void launch_bj_apply_f64(int nu, long long N, const double* binv, const double* r, double* z, cudaStream_t s) {
    bj_apply<double>(nu, N, binv, r, z, s);
}
void launch_bj_apply_f32(int nu, long long N, const float* binv, const float* r, float* z, cudaStream_t s) {
    bj_apply<float>(nu, N, binv, r, z, s);
}

// ------------------------------------------------------------------ semi-implicit step
// Hyperbolic update at time n (alpha and lambda at n) and the backward-Euler
// energy exchange: writes E^{n+1} (and T^{n+1}) into Unew and F* into Fstar.
template <int DIM, bool GAS>
__global__ void __launch_bounds__(kThreads) k_explicit_hyp(Dev<double> g, double* __restrict__ Unew,
                                                           double* __restrict__ Fstar) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int coord[3];
    cell_coord(idx, g.n[0], g.n[1], coord);
    LoadPlain<double> ld{g.Un, g.N};
    const St<double, DIM> self = load_state<double, DIM, GAS>(ld, idx, idx);
    const Cl<double, DIM> ks = closure(self, g.c);
    double divE = 0.0, divF[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) divF[b] = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            double sig_nb;
            bool boundary;
            const St<double, DIM> nb = neighbour<double, DIM, GAS>(g, ld, self, idx, coord, a, side, sig_nb, boundary);
            const Cl<double, DIM> kn = closure(nb, g.c);
            const long long fidx = face_index(g.n, coord, a, coord[a] + side);
            double Fs, Ps[DIM];
            if (side)
                hll(self, nb, ks, kn, g.lam_p[a][fidx], g.lam_m[a][fidx], a, g.c, Fs, Ps);
            else
                hll(nb, self, kn, ks, g.lam_p[a][fidx], g.lam_m[a][fidx], a, g.c, Fs, Ps);
            const double w = (side ? 1.0 : -1.0) * g.inv_dx[a];
            divE += w * g.alpha[a][fidx] * Fs;
#pragma unroll
            for (int b = 0; b < DIM; ++b) divF[b] += w * Ps[b];
        }
    }
    double Es = self.E - g.dt * divE;
    if (g.S) Es += g.dt * g.S[idx];
    const double k = g.c * g.sig_a[idx] * g.dt;
    if constexpr (GAS) {
        // rho c_v (T - T^n) + k/(1+k) (a_r T^4 - E*) = 0: Newton from the upper bound
        const double w = k / (1.0 + k), rc = g.rho_cv[idx], Tn = self.T;
        double T = fmax(Tn, sqrt(sqrt(fmax(Es, 0.0) / g.a_r)));
        for (int it = 0; it < 100; ++it) {
            const double T3 = T * T * T;
            const double f = rc * (T - Tn) + w * (g.a_r * T3 * T - Es);
            const double df = rc + 4.0 * w * g.a_r * T3;
            const double st = f / df;
            T -= st;
            if (fabs(st) <= 1e-15 * fabs(T)) break;
        }
        const double T2 = T * T;
        Unew[idx] = (Es + k * g.a_r * T2 * T2) / (1.0 + k);
        Unew[(1 + DIM) * g.N + idx] = T;
    } else {
        Unew[idx] = (Es + k * (g.B ? g.B[idx] : 0.0)) / (1.0 + k);
    }
#pragma unroll
    for (int b = 0; b < DIM; ++b) Fstar[b * g.N + idx] = self.F[b] - g.dt * divF[b];
}

void launch_explicit_hyp(const Dev<double>& g, double* Unew, double* Fstar, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
#define CALL(D, G) k_explicit_hyp<D, G><<<nb, kThreads, 0, s>>>(g, Unew, Fstar)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
}

// Explicit first-order upwind transport of the gas internal energy e = rho c_v T
// by prescribed face velocities (frozen-hydrodynamics step of the operator
// split): e* = e - dt sum_a ((u e_up)_{+} - (u e_up)_{-}) / dx_a, ghosts copy
// the boundary cell (wrap when periodic). Writes T* into Tout.
template <int DIM>
__global__ void k_advect(Dev<double> g, const double* __restrict__ u0, const double* __restrict__ u1,
                         const double* __restrict__ u2, double* __restrict__ Tout) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    int coord[3];
    cell_coord(idx, g.n[0], g.n[1], coord);
    const double* Tn = g.Un + (1 + DIM) * g.N;
    const double e = g.rho_cv[idx] * Tn[idx];
    const double* uf[3] = {u0, u1, u2};
    double div = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int ca = coord[a] + (side ? 1 : -1);
            long long j = idx;
            if (ca >= 0 && ca < g.n[a])
                j = idx + (side ? g.stride[a] : -g.stride[a]);
            else if (g.bc[a][side] == BC_PERIODIC)
                j = idx + (side ? -(long long)(g.n[a] - 1) : (long long)(g.n[a] - 1)) * g.stride[a];
            const double en = g.rho_cv[j] * Tn[j];
            const double u = uf[a][face_index(g.n, coord, a, coord[a] + side)];
            const double eL = side ? e : en, eR = side ? en : e;
            const double flux = u > 0.0 ? u * eL : u * eR;
            div += (side ? flux : -flux) * g.inv_dx[a];
        }
    }
    Tout[idx] = (e - g.dt * div) / g.rho_cv[idx];
}

void launch_advect(const Dev<double>& g, const double* const u[3], double* Tout, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
    switch (g.dim) {
        case 1: k_advect<1><<<nb, kThreads, 0, s>>>(g, u[0], u[1], u[2], Tout); break;
        case 2: k_advect<2><<<nb, kThreads, 0, s>>>(g, u[0], u[1], u[2], Tout); break;
        default: k_advect<3><<<nb, kThreads, 0, s>>>(g, u[0], u[1], u[2], Tout); break;
    }
}

// Explicit velocity-dependent radiation sources over dt (Sect. 2.1, first order
// in u/c; step 3 of the splitting of Sect. 2.3): with the cell velocity u the
// mean of its two face velocities, the closure pressure P of the current state,
// B = a_r T^4 (gas) or the frozen emission and sigma the flux opacity,
//   S_E = (sigma/c) u.F + (sigma/c) E |u|^2 + (sigma/c) u.(P u)
//   S_F = sigma P u + sigma B u + (sigma/c^2) u (u.F)
//   E' = E + dt S_E, F' = F + c dt S_F, rho c_v T' = rho c_v T - dt S_E (gas).
template <int DIM, bool GAS>
__global__ void k_velocity_sources(Dev<double> g, const double* __restrict__ u0, const double* __restrict__ u1,
                                   const double* __restrict__ u2, double* __restrict__ Uout) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long N = g.N;
    int coord[3];
    cell_coord(idx, g.n[0], g.n[1], coord);
    const double* uf[3] = {u0, u1, u2};
    double u[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
        u[a] = 0.5 * (uf[a][face_index(g.n, coord, a, coord[a])] + uf[a][face_index(g.n, coord, a, coord[a] + 1)]);
    St<double, DIM> st;
    st.E = g.Un[idx];
#pragma unroll
    for (int b = 0; b < DIM; ++b) st.F[b] = g.Un[(1 + b) * N + idx];
    st.T = GAS ? g.Un[(1 + DIM) * N + idx] : 0.0;
    const Cl<double, DIM> k = closure(st, g.c);
    double Pu[DIM], uF = 0.0, uu = 0.0, uPu = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < DIM; ++b) t += pressure(k, a, b) * u[b];
        Pu[a] = t;
        uF += u[a] * st.F[a];
        uu += u[a] * u[a];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) uPu += u[a] * Pu[a];
    const double c = g.c, dt = g.dt, sig = g.sig_f[idx];
    double B;
    if constexpr (GAS) {
        const double T2 = st.T * st.T;
        B = g.a_r * (T2 * T2);
    } else {
        B = g.B ? g.B[idx] : 0.0;
    }
    const double SE = (sig / c) * uF + (sig / c) * st.E * uu + (sig / c) * uPu;
    Uout[idx] = st.E + dt * SE;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double SF = sig * Pu[a] + sig * B * u[a] + (sig / (c * c)) * u[a] * uF;
        Uout[(1 + a) * N + idx] = st.F[a] + c * dt * SF;
    }
    if constexpr (GAS) Uout[(1 + DIM) * N + idx] = st.T - dt * SE / g.rho_cv[idx];
}

void launch_velocity_sources(const Dev<double>& g, const double* const u[3], double* Uout, cudaStream_t s) {
    const int nb = stencil_blocks(g.N);
#define CALL(D, G) k_velocity_sources<D, G><<<nb, kThreads, 0, s>>>(g, u[0], u[1], u[2], Uout)
    M1_DISPATCH(g.dim, g.gas, CALL);
#undef CALL
}

// One thread per grid line along axis b: solve (I + c dt W_b) F_b = F*_b, the
// Appendix B tridiagonal form with r_{j+1/2} = c sigma_{j+1/2} dt / 4 (interior
// faces), Eq. (boundaryCondition) at time n on non-periodic boundary faces (or
// the plain face average with the ghost), Thomas' algorithm, and
// Sherman-Morrison for the cyclic system of a periodic axis.
template <int DIM>
__global__ void k_wb_lines(Dev<double> g, int b, const double* __restrict__ Fstar, double* __restrict__ Fout,
                           double* __restrict__ cp, double* __restrict__ dp, double* __restrict__ zp) {
    const long long nlines = g.N / g.n[b];
    const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    int ln[3] = {g.n[0], g.n[1], g.n[2]};
    ln[b] = 1;
    int coord[3];
    cell_coord(line, ln[0], ln[1], coord);
    coord[b] = 0;
    const long long base = ((long long)coord[2] * g.n[1] + coord[1]) * g.n[0] + coord[0];
    const long long st = g.stride[b];
    const int n = g.n[b];
    const double q = g.c * g.dt * 0.125;  // r_{j+1/2} = q (sigma_j + sigma_{j+1})
    const double* sig = g.sig_f;
    const double* rhs = Fstar + (long long)b * g.N;
    const bool periodic = g.bc[b][0] == BC_PERIODIC;

    if (!g.wb) {  // centred source, Eq. (wb_naive): diagonal
        for (int j = 0; j < n; ++j) {
            const long long i = base + j * st;
            Fout[i] = rhs[i] / (1.0 + g.c * g.dt * sig[i]);
        }
        return;
    }
    if (periodic && n <= 2) {
        if (n == 1) {
            Fout[base] = rhs[base] / (1.0 + 4.0 * 2.0 * q * sig[base]);
            return;
        }
        const long long i0 = base, i1 = base + st;
        const double r = 2.0 * q * (sig[i0] + sig[i1]);  // two faces, both between cells 0 and 1
        const double d = 1.0 + r, o = r;
        const double det = d * d - o * o;
        Fout[i0] = (d * rhs[i0] - o * rhs[i1]) / det;
        Fout[i1] = (d * rhs[i1] - o * rhs[i0]) / det;
        return;
    }
    // boundary contributions (non-periodic)
    double diag0 = 0.0, diagN = 0.0, rhs0 = 0.0, rhsN = 0.0;
    if (!periodic) {
        LoadPlain<double> ld{g.Un, g.N};
        for (int side = 0; side < 2; ++side) {
            int cc[3] = {coord[0], coord[1], coord[2]};
            cc[b] = side ? n - 1 : 0;
            const long long ie = base + (long long)cc[b] * st;
            double ddiag = 0.0, drhs = 0.0;
            const int kind = g.bc[b][side];
            if (g.wb_boundary) {
                const St<double, DIM> self = load_state<double, DIM, false>(ld, ie, ie);
                double sig_nb;
                bool bnd;
                const St<double, DIM> gh = neighbour<double, DIM, false>(g, ld, self, ie, cc, b, side, sig_nb, bnd);
                const double Pi = pressure(closure(self, g.c), b, b), Pg = pressure(closure(gh, g.c), b, b);
                const double phi = side ? -g.c * (Pg - Pi) * g.inv_dx[b] : -g.c * (Pi - Pg) * g.inv_dx[b];
                drhs = -0.5 * g.c * g.dt * phi;
            } else {
                const double r = 2.0 * q * sig[ie];
                if (kind == BC_OUTFLOW) {
                    ddiag = 2.0 * r;
                } else if (kind == BC_DIRICHLET) {
                    const long long m = bface_cell(g.n, cc, b);
                    const unsigned char* mk = g.bmask[b][side];
                    if (mk == nullptr || mk[m]) {
                        ddiag = r;
                        drhs = -r * g.bF[b][side][(long long)b * g.bM[b] + m];
                    } else {
                        ddiag = 2.0 * r;
                    }
                }  // reflect: the face average vanishes
            }
            if (side) {
                diagN = ddiag;
                rhsN = drhs;
            } else {
                diag0 = ddiag;
                rhs0 = drhs;
            }
        }
    }
    // coefficients of row j: lower a_j = r_{j-1/2}, upper c_j = r_{j+1/2}, diag 1 + a_j + c_j (+ boundary)
    auto rface = [&](int j) -> double {  // r between cell j and j+1 (j+1 wrapped)
        const int jp = (j + 1 == n) ? 0 : j + 1;
        return q * (sig[base + (long long)j * st] + sig[base + (long long)jp * st]);
    };
    const double rwrap = periodic ? rface(n - 1) : 0.0;
    // Sherman-Morrison pieces (periodic): A = T + u v^T with gamma = -b_0
    double gamma = 0.0;
    double prev_c = 0.0, prev_d = 0.0, prev_z = 0.0;
    double rlo = periodic ? rwrap : 0.0;  // r_{-1/2}
    for (int j = 0; j < n; ++j) {
        const long long i = base + (long long)j * st;
        const double rhi = (j < n - 1) ? rface(j) : (periodic ? rwrap : 0.0);
        double bj = 1.0 + rlo + rhi;
        double dj = rhs[i];
        if (!periodic) {
            if (j == 0) {
                bj += diag0;
                dj += rhs0;
            }
            if (j == n - 1) {
                bj += diagN;
                dj += rhsN;
            }
        }
        double aj = (j > 0) ? rlo : 0.0;
        double cj = (j < n - 1) ? rhi : 0.0;
        double uj = 0.0;
        if (periodic) {
            if (j == 0) {
                gamma = -bj;
                bj -= gamma;
                uj = gamma;
            }
            if (j == n - 1) {
                bj -= rwrap * rwrap / gamma;
                uj = rwrap;
            }
        }
        const double m = (j == 0) ? bj : bj - aj * prev_c;
        const double cpj = cj / m;
        const double dpj = (dj - aj * prev_d) / m;
        const double zpj = (uj - aj * prev_z) / m;
        cp[i] = cpj;
        dp[i] = dpj;
        if (periodic) zp[i] = zpj;
        prev_c = cpj;
        prev_d = dpj;
        prev_z = zpj;
        rlo = rhi;
    }
    // back substitution (y in dp, z in zp)
    double ny = dp[base + (long long)(n - 1) * st], nz = periodic ? zp[base + (long long)(n - 1) * st] : 0.0;
    Fout[base + (long long)(n - 1) * st] = ny;
    if (periodic) zp[base + (long long)(n - 1) * st] = nz;
    for (int j = n - 2; j >= 0; --j) {
        const long long i = base + (long long)j * st;
        ny = dp[i] - cp[i] * ny;
        Fout[i] = ny;
        if (periodic) {
            nz = zp[i] - cp[i] * nz;
            zp[i] = nz;
        }
    }
    if (periodic) {
        // x = y - (v.y)/(1 + v.z) z with v = (1, 0, ..., 0, rwrap / gamma)
        const long long i0 = base, iN = base + (long long)(n - 1) * st;
        const double vy = Fout[i0] + rwrap / gamma * Fout[iN];
        const double vz = zp[i0] + rwrap / gamma * zp[iN];
        const double fac = vy / (1.0 + vz);
        for (int j = 0; j < n; ++j) {
            const long long i = base + (long long)j * st;
            Fout[i] -= fac * zp[i];
        }
    }
}

void launch_wb_lines(const Dev<double>& g, int b, const double* Fstar, double* Fout, double* work, cudaStream_t s) {
    const long long nlines = g.N / g.n[b];
    const int nb = (int)((nlines + 127) / 128);
    double* cp = work;
    double* dp = work + g.N;
    double* zp = work + 2 * g.N;
    switch (g.dim) {
        case 1: k_wb_lines<1><<<nb, 128, 0, s>>>(g, b, Fstar, Fout, cp, dp, zp); break;
        case 2: k_wb_lines<2><<<nb, 128, 0, s>>>(g, b, Fstar, Fout, cp, dp, zp); break;
        default: k_wb_lines<3><<<nb, 128, 0, s>>>(g, b, Fstar, Fout, cp, dp, zp); break;
    }
}

}  // namespace m1
