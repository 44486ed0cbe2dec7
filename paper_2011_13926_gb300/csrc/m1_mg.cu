// m1_mg.cu — aggregation multigrid V-cycle for the 2D Newton system (FP32).
//
// The structured-grid analogue of the algebraic multigrid the paper found best
// among its preconditioners (Sect. 3.3.2, Sect. 4):
//   level 0: the Jacobian itself, applied matrix-free by the linear J v, its
//     point-block inverses (the block-Jacobi ones) as smoother; its 5-point
//     stencil of n_u x n_u blocks (C, W, E, S, N = self, -x, +x, -y, +y), only
//     needed to build the coarse levels, is assembled directly from the
//     pressure Jacobian (radiation only, k_mg_assemble2d) or read off J v by
//     coloured probes (a vector that is 1 on one unknown of every cell of one
//     colour class; cells of a class are >= 3 apart, also across a periodic
//     wrap, so each response entry belongs to one probed cell);
//   levels >= 1: 2 x 2 cell aggregates, piecewise-constant prolongation P,
//     restriction P^T (the sum over the aggregate) and the Galerkin stencil
//     P^T A P — again a 5-point block stencil (a fine coupling inside the
//     aggregate adds to C, one leaving it adds to the block of its direction);
//   the cycle: V(1,1) with damped point-block Jacobi (omega = 0.7) from zero,
//     10 damped sweeps from zero on the coarsest level (both sides <= 16 cells,
//     one CTA, the iterate in shared memory).
// Blocks are stored A[((s n_u + r) n_u + c) N + i]; the block inverses of the
// C blocks [(r n_u + c) N + i] like the block-Jacobi ones.
#include "m1_internal.h"

#include <algorithm>

namespace m1 {

constexpr float kMgOmega = 0.7f;
constexpr int kMgCoarsest = 16;
constexpr int kMgCoarseSweeps = 10;
constexpr int kMgThreads = 256;

int mg_colour_period(int n, bool periodic) {
    if (!periodic) return 3;
    for (int m = 3; m <= n; ++m) {
        const int r = n % m;
        if (r == 0 || (r >= 3 && m - r >= 3)) return m;
    }
    return n;
}

// Programmatic dependent launch within the cycle's chain of coarse-level
// kernels: each lets its successor launch as soon as all of its own blocks
// run, and the successor waits for it (a hardware grid dependency) before
// reading anything the chain writes; before the wait a kernel only reads the
// hierarchy (stencils, block inverses), written before the cycle began. A
// kernel launched without the attribute passes both at once.
__device__ __forceinline__ void mg_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void mg_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// neighbour s of cell (ix, iy) on an nx x ny level, -1 beyond a non-periodic side
__device__ __forceinline__ long long mg_nb(int ix, int iy, int s, int nx, int ny, bool px, bool py) {
    int jx = ix + (s == 1 ? -1 : s == 2 ? 1 : 0);
    int jy = iy + (s == 3 ? -1 : s == 4 ? 1 : 0);
    if (px) jx = jx < 0 ? jx + nx : (jx >= nx ? jx - nx : jx);
    if (py) jy = jy < 0 ? jy + ny : (jy >= ny ? jy - ny : jy);
    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) return -1;
    return (long long)jy * nx + jx;
}

// ------------------------------------------------------------------ probing
__global__ void k_mg_probe(int nu, int nx, int ny, int mx, int my, int colour, int comp, float* __restrict__ v) {
    const long long N = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)(i / nx);
        const bool hit = (ix % mx) + mx * (iy % my) == colour;
        for (int c = 0; c < nu; ++c) v[c * N + i] = (hit && c == comp) ? 1.f : 0.f;
    }
}

template <int NU>
__global__ void k_mg_extract(int nx, int ny, bool px, bool py, int mx, int my, int colour, int comp,
                             const float* __restrict__ y, float* __restrict__ A) {
    const long long N = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)(i / nx);
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const long long j = mg_nb(ix, iy, s, nx, ny, px, py);
            if (j < 0) continue;
            const int jx = (int)(j % nx), jy = (int)(j / nx);
            if ((jx % mx) + mx * (jy % my) != colour) continue;
#pragma unroll
            for (int r = 0; r < NU; ++r) A[((long long)(s * NU + r) * NU + comp) * N + i] = y[r * N + i];
        }
    }
}

// ------------------------------------------------------------------ level-0 stencil, direct
// The linear J v of cell i (2D, radiation only, frozen or fixed wave speeds) is
// a linear function of the staged derivative quantities (E, Fx, Fy, Pxx, Pxy,
// Pyy) at five positions: the cell (0) and its faces' neighbours W, E, S, N
// (1..4), with the formulas of the linear tiled J v. mg_lin_self gives the terms
// of the cell's own tuple outside the faces, mg_lin_face one face's flux and
// well-balanced source terms; their sum over the faces is J v of the cell.
struct MgFace {
    float lp, lm, al, sn;  // wave speeds, alpha, the neighbour's flux opacity
    float inv, pm;         // 1 / (lp - lm) (0 when it vanishes) and lp lm inv, once per face
    bool boundary;         // a non-periodic boundary face (the neighbour is a ghost)
};

__device__ __forceinline__ void mg_lin_self(const Dev<float>& g, const float* me, float sig_self, float sig_a,
                                            bool wbc, float* out) {
    const float cdt = g.c * g.dt;
    out[0] = me[0] + (cdt * sig_a) * me[0];  // minus the exchange - c sigma_a dt dE
    out[1] = wbc ? me[1] : me[1] + cdt * (sig_self * me[1]);
    out[2] = wbc ? me[2] : me[2] + cdt * (sig_self * me[2]);
}

// face (a, side) of the cell; me and nb the tuples of the cell and of the
// neighbour across the face (either may be zero); adds to out
__device__ __forceinline__ void mg_lin_face(const Dev<float>& g, const float* me, const float* nb, const MgFace& f,
                                            int a, int side, float sig_self, bool wbc, float* out) {
    const float c = g.c, c2 = g.c * g.c, cdt = g.c * g.dt;
    const float* L = side ? me : nb;
    const float* Rr = side ? nb : me;
    const float FaL = a == 0 ? L[1] : L[2], FaR = a == 0 ? Rr[1] : Rr[2];
    const float Fs = (f.lp * FaL - f.lm * FaR) * f.inv + f.pm * (Rr[0] - L[0]);
    const float PaxL = a == 0 ? L[3] : L[4], PaxR = a == 0 ? Rr[3] : Rr[4];
    const float PayL = a == 0 ? L[4] : L[5], PayR = a == 0 ? Rr[4] : Rr[5];
    const float Psx = c2 * (f.lp * PaxL - f.lm * PaxR) * f.inv + f.pm * (Rr[1] - L[1]);
    const float Psy = c2 * (f.lp * PayL - f.lm * PayR) * f.inv + f.pm * (Rr[2] - L[2]);
    const float w = (side ? g.dt : -g.dt) * g.inv_dx[a];
    out[0] += (w * f.al) * Fs;
    out[1] += w * Psx;
    out[2] += w * Psy;
    if (wbc) {
        float ph;
        if (f.boundary && g.wb_boundary) {
            const float PR = a == 0 ? Rr[3] : Rr[5], PL = a == 0 ? L[3] : L[5];
            ph = -c * g.inv_dx[a] * (PR - PL);
        } else {
            ph = (0.25f * (sig_self + f.sn)) * (FaL + FaR);
        }
        out[1 + a] += cdt * (0.5f * ph);
    }
}

// A0 blocks of every cell: column c of block s is mg_lin_out with a unit
// derivative of unknown c at that position's cell (its pressure derivative the
// column of dP/dU there); a boundary ghost depends on the cell itself (dual
// numbers through the boundary rule), so it enters the C block.
// three CTAs per SM (at most 85 registers): the kernel is latency-bound
__global__ void __launch_bounds__(kMgThreads, 3) k_mg_assemble2d(Dev<float> g, const float* __restrict__ U,
                                                                const float* __restrict__ pj,
                                float* __restrict__ A) {
    const int nx = g.n[0];
    const long long N = g.N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)(i / nx);
        const int coord[3] = {ix, iy, 0};
        const float sig_self = g.sig_f[i], sig_a = g.sig_a[i];
        const bool wbc = g.wb && !(g.fb && g.fb[i]);
        MgFace fc[4];
        long long nbi[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                MgFace& f = fc[2 * a + side];
                const int ca = coord[a] + (side ? 1 : -1);
                const bool inside = ca >= 0 && ca < g.n[a];
                const bool periodic = g.bc[a][side] == BC_PERIODIC;
                f.boundary = !inside && !periodic;
                long long j = -1;
                if (inside)
                    j = i + (side ? g.stride[a] : -g.stride[a]);
                else if (periodic)
                    j = i + (side ? -(long long)(g.n[a] - 1) : (long long)(g.n[a] - 1)) * g.stride[a];
                nbi[2 * a + side] = j;
                f.sn = j >= 0 ? g.sig_f[j] : sig_self;
                const long long fidx = face_index(g.n, coord, a, coord[a] + side);
                if (g.fixed_eigs) {
                    f.lp = g.c;
                    f.lm = -g.c;
                } else {
                    f.lp = g.lam_p[a][fidx];
                    f.lm = g.lam_m[a][fidx];
                }
                f.al = g.alpha[a][fidx];
                const float den = f.lp - f.lm;
                f.inv = den >= Tiny<float>::den() ? 1.f / den : 0.f;
                f.pm = f.lp * f.lm * f.inv;
            }
        }
        const float zero[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const LoadSeed<float> ld{U, N, -1};  // in-domain loads (not taken on a boundary face): no seed
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            // C: the cell's own unknown c (unit derivative, dP the column c of dP/dU),
            // and through the boundary rules the ghosts of its boundary faces
            float t0[6] = {c == 0 ? 1.f : 0.f, c == 1 ? 1.f : 0.f, c == 2 ? 1.f : 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < 3; ++r) t0[3 + r] = pj[(long long)(3 * r + c) * N + i];
            float out[3];
            mg_lin_self(g, t0, sig_self, sig_a, wbc, out);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                float gh[6];
                if (fc[p].boundary) {  // the ghost's derivatives in the cell's unknown c (dual numbers)
                    St<Dual<float>, 2> self;
                    self.E = Dual<float>{U[i], c == 0 ? 1.f : 0.f};
                    self.F[0] = Dual<float>{U[N + i], c == 1 ? 1.f : 0.f};
                    self.F[1] = Dual<float>{U[2 * N + i], c == 2 ? 1.f : 0.f};
                    float sn;
                    bool bnd;
                    const St<Dual<float>, 2> u = neighbour<Dual<float>, 2, false>(g, ld, self, i, coord, p / 2, p % 2,
                                                                                 sn, bnd);
                    const Cl<Dual<float>, 2> k = closure(u, g.c);
                    gh[0] = u.E.d;
                    gh[1] = u.F[0].d;
                    gh[2] = u.F[1].d;
                    gh[3] = pressure(k, 0, 0).d;
                    gh[4] = pressure(k, 0, 1).d;
                    gh[5] = pressure(k, 1, 1).d;
                } else {
#pragma unroll
                    for (int q = 0; q < 6; ++q) gh[q] = 0.f;
                }
                mg_lin_face(g, t0, gh, fc[p], p / 2, p % 2, sig_self, wbc, out);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) A[((long long)(0 * 3 + r) * 3 + c) * N + i] = out[r];
            // W, E, S, N: the neighbour's unknown c enters through the one face they share
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                float o[3] = {0.f, 0.f, 0.f};
                const long long X = nbi[p];
                if (X >= 0) {
                    float tn[6] = {c == 0 ? 1.f : 0.f, c == 1 ? 1.f : 0.f, c == 2 ? 1.f : 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int r = 0; r < 3; ++r) tn[3 + r] = pj[(long long)(3 * r + c) * N + X];
                    mg_lin_face(g, zero, tn, fc[p], p / 2, p % 2, sig_self, wbc, o);
                }
#pragma unroll
                for (int r = 0; r < 3; ++r) A[((long long)((1 + p) * 3 + r) * 3 + c) * N + i] = o[r];
            }
        }
    }
}

// ------------------------------------------------------------------ Galerkin
template <int NU>
__global__ void k_mg_galerkin(int nx, int ny, bool px, bool py, const float* __restrict__ Af, int nxc, int nyc,
                              float* __restrict__ Ac) {
    const long long Nf = (long long)nx * ny, Nc = (long long)nxc * nyc;
    for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < Nc; I += (long long)gridDim.x * blockDim.x) {
        const int Ix = (int)(I % nxc), Iy = (int)(I / nxc);
        float acc[5][NU][NU];
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int r = 0; r < NU; ++r)
#pragma unroll
                for (int c = 0; c < NU; ++c) acc[s][r][c] = 0.f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int ix = 2 * Ix + dx, iy = 2 * Iy + dy;
                if (ix >= nx || iy >= ny) continue;
                const long long i = (long long)iy * nx + ix;
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    const long long j = mg_nb(ix, iy, s, nx, ny, px, py);
                    if (j < 0) continue;
                    const int jx = (int)(j % nx), jy = (int)(j / nx);
                    const bool same = (jx / 2 == Ix) && (jy / 2 == Iy);
#pragma unroll
                    for (int r = 0; r < NU; ++r)
#pragma unroll
                        for (int c = 0; c < NU; ++c) {
                            const float a = Af[((long long)(s * NU + r) * NU + c) * Nf + i];
                            if (same)
                                acc[0][r][c] += a;
                            else
                                acc[s][r][c] += a;
                        }
                }
            }
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int r = 0; r < NU; ++r)
#pragma unroll
                for (int c = 0; c < NU; ++c) Ac[((long long)(s * NU + r) * NU + c) * Nc + I] = acc[s][r][c];
    }
}

// ------------------------------------------------------------------ cycle pieces
// z = omega D^-1 r
template <int NU>
__global__ void k_mg_jacobi0(long long N, const float* __restrict__ Dinv, const float* __restrict__ r,
                             float* __restrict__ z) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float ri[NU];
#pragma unroll
        for (int c = 0; c < NU; ++c) ri[c] = r[c * N + i];
#pragma unroll
        for (int q = 0; q < NU; ++q) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NU; ++c) a += Dinv[(long long)(q * NU + c) * N + i] * ri[c];
            z[q * N + i] = kMgOmega * a;
        }
    }
}

// coarsest level: sweeps of z <- z + omega D^-1 (r - A z) from zero, one CTA
// with one thread per cell (N <= kMgCoarsest^2): each thread keeps its stencil
// row, block inverse and residual in registers, the iterate is double-buffered
// in shared memory
template <int NU>
__global__ void __launch_bounds__(kMgCoarsest* kMgCoarsest) k_mg_coarsest(int nx, int ny, bool px, bool py,
                                                                          const float* __restrict__ A,
                                                                          const float* __restrict__ Dinv,
                                                                          const float* __restrict__ r,
                                                                          float* __restrict__ zout, int sweeps) {
    __shared__ float zs[2][NU][kMgCoarsest * kMgCoarsest];
    const int N = nx * ny;
    const int i = threadIdx.x;
    const bool own = i < N;
    float a[5][NU][NU], d[NU][NU], ri[NU];
    long long nb[5];
    mg_pdl_trigger();
    if (own) {
        const int ix = i % nx, iy = i / nx;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            nb[s] = mg_nb(ix, iy, s, nx, ny, px, py);
#pragma unroll
            for (int q = 0; q < NU; ++q)
#pragma unroll
                for (int c = 0; c < NU; ++c) a[s][q][c] = A[((long long)(s * NU + q) * NU + c) * N + i];
        }
#pragma unroll
        for (int q = 0; q < NU; ++q)
#pragma unroll
            for (int c = 0; c < NU; ++c) d[q][c] = Dinv[(long long)(q * NU + c) * N + i];
#pragma unroll
        for (int c = 0; c < NU; ++c) zs[0][c][i] = 0.f;
    }
    mg_pdl_wait();
    if (own)
#pragma unroll
        for (int q = 0; q < NU; ++q) ri[q] = r[q * N + i];
    __syncthreads();
    int cur = 0;
    for (int k = 0; k < sweeps; ++k) {
        if (own) {
            float res[NU];
#pragma unroll
            for (int q = 0; q < NU; ++q) res[q] = ri[q];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                if (nb[s] < 0) continue;
#pragma unroll
                for (int q = 0; q < NU; ++q)
#pragma unroll
                    for (int c = 0; c < NU; ++c) res[q] -= a[s][q][c] * zs[cur][c][nb[s]];
            }
#pragma unroll
            for (int q = 0; q < NU; ++q) {
                float t = 0.f;
#pragma unroll
                for (int c = 0; c < NU; ++c) t += d[q][c] * res[c];
                zs[cur ^ 1][q][i] = zs[cur][q][i] + kMgOmega * t;
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    if (own)
#pragma unroll
        for (int c = 0; c < NU; ++c) zout[c * N + i] = zs[cur][c][i];
}

// ------------------------------------------------------------------ tiled assembled levels
// A 32 x 8 tile of cells plus its axis halo (a periodic side wraps, a cell
// beyond a non-periodic side holds 0: its couplings are zero) in shared memory.
constexpr int kMgTX = 32, kMgTY = 8;

// halo index (hx, hy) of a tile at (x0, y0) -> cell, or -1
__device__ __forceinline__ long long mg_halo_cell(int x0, int y0, int hx, int hy, int nx, int ny, bool px, bool py) {
    int gx = x0 + hx - 1, gy = y0 + hy - 1;
    if (px) gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
    if (py) gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) return -1;
    return (long long)gy * nx + gx;
}

// down: z = omega D^-1 r (written), rc = P^T (r - A z) — pre-smoothing,
// residual and restriction of one assembled level in one pass
template <int NU>
__global__ void __launch_bounds__(kMgTX* kMgTY, 4) k_mg_down(int nx, int ny, bool px, bool py,
                                                        const float* __restrict__ A, const float* __restrict__ Dinv,
                                                        const float* __restrict__ r, float* __restrict__ z,
                                                        int nxc, int nyc, float* __restrict__ rc) {
    __shared__ float zt[kMgTY + 2][kMgTX + 2][NU];
    __shared__ float rs[kMgTY][kMgTX][NU];
    const long long N = (long long)nx * ny, Nc = (long long)nxc * nyc;
    const int x0 = blockIdx.x * kMgTX, y0 = blockIdx.y * kMgTY;
    const int tid = threadIdx.y * kMgTX + threadIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ix = x0 + tx, iy = y0 + ty;
    const bool valid = ix < nx && iy < ny;
    const long long i = valid ? (long long)iy * nx + ix : 0;
    mg_pdl_trigger();
    // this cell's stencil row (in flight during the wait and the staging), then
    // its right-hand side
    float a[5][NU][NU], ri[NU];
    if (valid) {
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int q = 0; q < NU; ++q)
#pragma unroll
                for (int c = 0; c < NU; ++c) a[s][q][c] = A[((long long)(s * NU + q) * NU + c) * N + i];
    }
    mg_pdl_wait();
    if (valid)
#pragma unroll
        for (int c = 0; c < NU; ++c) ri[c] = r[c * N + i];
    for (int t = tid; t < (kMgTX + 2) * (kMgTY + 2); t += kMgTX * kMgTY) {
        const int hx = t % (kMgTX + 2), hy = t / (kMgTX + 2);
        if ((hx == 0 || hx == kMgTX + 1) && (hy == 0 || hy == kMgTY + 1)) continue;  // corners
        const long long j = mg_halo_cell(x0, y0, hx, hy, nx, ny, px, py);
        float rj[NU];
#pragma unroll
        for (int c = 0; c < NU; ++c) rj[c] = j >= 0 ? r[c * N + j] : 0.f;
#pragma unroll
        for (int q = 0; q < NU; ++q) {
            float a = 0.f;
            if (j >= 0)
#pragma unroll
                for (int c = 0; c < NU; ++c) a += Dinv[(long long)(q * NU + c) * N + j] * rj[c];
            zt[hy][hx][q] = kMgOmega * a;
        }
    }
    __syncthreads();
    float res[NU];
#pragma unroll
    for (int c = 0; c < NU; ++c) res[c] = 0.f;
    if (valid) {
#pragma unroll
        for (int c = 0; c < NU; ++c) {
            z[c * N + i] = zt[ty + 1][tx + 1][c];
            res[c] = ri[c];
        }
        const int hx[5] = {tx + 1, tx, tx + 2, tx + 1, tx + 1}, hy[5] = {ty + 1, ty + 1, ty + 1, ty, ty + 2};
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int q = 0; q < NU; ++q)
#pragma unroll
                for (int c = 0; c < NU; ++c) res[q] -= a[s][q][c] * zt[hy[s]][hx[s]][c];
    }
#pragma unroll
    for (int c = 0; c < NU; ++c) rs[ty][tx][c] = res[c];
    __syncthreads();
    if ((tx & 1) == 0 && (ty & 1) == 0 && valid) {
        const long long I = (long long)(iy / 2) * nxc + ix / 2;
#pragma unroll
        for (int c = 0; c < NU; ++c)
            rc[c * Nc + I] = (rs[ty][tx][c] + rs[ty][tx + 1][c]) + (rs[ty + 1][tx][c] + rs[ty + 1][tx + 1][c]);
    }
}

// up: zz = z + P zc, zout = zz + omega D^-1 (r - A zz) on one assembled level
template <int NU>
__global__ void __launch_bounds__(kMgTX* kMgTY, 3) k_mg_up(int nx, int ny, bool px, bool py,
                                                      const float* __restrict__ A, const float* __restrict__ Dinv,
                                                      const float* __restrict__ r, const float* __restrict__ z,
                                                      const float* __restrict__ zc, int nxc, int nyc,
                                                      float* __restrict__ zout) {
    __shared__ float zt[kMgTY + 2][kMgTX + 2][NU];
    const long long N = (long long)nx * ny, Nc = (long long)nxc * nyc;
    const int x0 = blockIdx.x * kMgTX, y0 = blockIdx.y * kMgTY;
    const int tid = threadIdx.y * kMgTX + threadIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ix = x0 + tx, iy = y0 + ty;
    const bool valid = ix < nx && iy < ny;
    const long long i = valid ? (long long)iy * nx + ix : 0;
    mg_pdl_trigger();
    // this cell's stencil row and block inverse (in flight during the wait and
    // the staging), then its right-hand side
    float a[5][NU][NU], d[NU][NU], ri[NU];
    if (valid) {
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int q = 0; q < NU; ++q)
#pragma unroll
                for (int c = 0; c < NU; ++c) a[s][q][c] = A[((long long)(s * NU + q) * NU + c) * N + i];
#pragma unroll
        for (int q = 0; q < NU; ++q)
#pragma unroll
            for (int c = 0; c < NU; ++c) d[q][c] = Dinv[(long long)(q * NU + c) * N + i];
    }
    mg_pdl_wait();
    if (valid)
#pragma unroll
        for (int q = 0; q < NU; ++q) ri[q] = r[q * N + i];
    for (int t = tid; t < (kMgTX + 2) * (kMgTY + 2); t += kMgTX * kMgTY) {
        const int hx = t % (kMgTX + 2), hy = t / (kMgTX + 2);
        if ((hx == 0 || hx == kMgTX + 1) && (hy == 0 || hy == kMgTY + 1)) continue;  // corners
        const long long j = mg_halo_cell(x0, y0, hx, hy, nx, ny, px, py);
        const long long J = j >= 0 ? (long long)((j / nx) / 2) * nxc + (j % nx) / 2 : 0;
#pragma unroll
        for (int c = 0; c < NU; ++c) zt[hy][hx][c] = j >= 0 ? z[c * N + j] + zc[c * Nc + J] : 0.f;
    }
    __syncthreads();
    if (!valid) return;
    float res[NU];
#pragma unroll
    for (int c = 0; c < NU; ++c) res[c] = ri[c];
    const int hx[5] = {tx + 1, tx, tx + 2, tx + 1, tx + 1}, hy[5] = {ty + 1, ty + 1, ty + 1, ty, ty + 2};
#pragma unroll
    for (int s = 0; s < 5; ++s)
#pragma unroll
        for (int q = 0; q < NU; ++q)
#pragma unroll
            for (int c = 0; c < NU; ++c) res[q] -= a[s][q][c] * zt[hy[s]][hx[s]][c];
#pragma unroll
    for (int q = 0; q < NU; ++q) {
        float t = 0.f;
#pragma unroll
        for (int c = 0; c < NU; ++c) t += d[q][c] * res[c];
        zout[q * N + i] = zt[ty + 1][tx + 1][q] + kMgOmega * t;
    }
}

// level 0: rc = P^T (r - w) with w = J z computed by the linear J v
template <int NU>
__global__ void k_mg_restrict_diff(int nx, int ny, const float* __restrict__ r, const float* __restrict__ w,
                                   int nxc, int nyc, float* __restrict__ rc) {
    const long long N = (long long)nx * ny, Nc = (long long)nxc * nyc;
    for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < Nc; I += (long long)gridDim.x * blockDim.x) {
        const int Ix = (int)(I % nxc), Iy = (int)(I / nxc);
        float acc[NU];
#pragma unroll
        for (int c = 0; c < NU; ++c) acc[c] = 0.f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int ix = 2 * Ix + dx, iy = 2 * Iy + dy;
                if (ix >= nx || iy >= ny) continue;
                const long long i = (long long)iy * nx + ix;
#pragma unroll
                for (int c = 0; c < NU; ++c) acc[c] += r[c * N + i] - w[c * N + i];
            }
#pragma unroll
        for (int c = 0; c < NU; ++c) rc[c * Nc + I] = acc[c];
    }
}

// level 0: z += P zc
template <int NU>
__global__ void k_mg_prolong_add(int nx, int ny, const float* __restrict__ zc, int nxc, int nyc, float* __restrict__ z) {
    const long long N = (long long)nx * ny, Nc = (long long)nxc * nyc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)(i / nx);
        const long long I = (long long)(iy / 2) * nxc + ix / 2;
#pragma unroll
        for (int c = 0; c < NU; ++c) z[c * N + i] += zc[c * Nc + I];
    }
}

// level 0: zout = z + omega D^-1 (r - w)
template <int NU>
__global__ void k_mg_post0(long long N, const float* __restrict__ Dinv, const float* __restrict__ r,
                           const float* __restrict__ w, const float* __restrict__ z, float* __restrict__ zout) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float res[NU];
#pragma unroll
        for (int c = 0; c < NU; ++c) res[c] = r[c * N + i] - w[c * N + i];
#pragma unroll
        for (int q = 0; q < NU; ++q) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NU; ++c) a += Dinv[(long long)(q * NU + c) * N + i] * res[c];
            zout[q * N + i] = z[q * N + i] + kMgOmega * a;
        }
    }
}

// ------------------------------------------------------------------ host side
static int grid_for(long long n) { return (int)std::min<long long>((n + kMgThreads - 1) / kMgThreads, 152LL * 16); }

void mg_plan(MgHierarchy& H, int nu, int nx, int ny, bool px, bool py) {
    H.nu = nu;
    H.px = px;
    H.py = py;
    H.nlev = 0;
    for (;;) {
        H.nx[H.nlev] = nx;
        H.ny[H.nlev] = ny;
        ++H.nlev;
        if ((nx <= kMgCoarsest && ny <= kMgCoarsest) || H.nlev == kMgMaxLevels) break;
        nx = (nx + 1) / 2;
        ny = (ny + 1) / 2;
    }
}

template <int NU>
static void assemble_level0(MgHierarchy& H, const MgJvOp& J, cudaStream_t s) {
    const int nx = H.nx[0], ny = H.ny[0];
    const long long N = (long long)nx * ny;
    const int mx = mg_colour_period(nx, H.px), my = mg_colour_period(ny, H.py);
    cudaMemsetAsync(H.A[0], 0, sizeof(float) * 5 * NU * NU * N, s);
    for (int col = 0; col < mx * my; ++col)
        for (int c = 0; c < NU; ++c) {
            k_mg_probe<<<grid_for(N), kMgThreads, 0, s>>>(NU, nx, ny, mx, my, col, c, H.probe);
            J.apply(J.ctx, H.probe, H.w0, s);
            k_mg_extract<NU><<<grid_for(N), kMgThreads, 0, s>>>(nx, ny, H.px, H.py, mx, my, col, c, H.w0, H.A[0]);
        }
}

template <int NU>
static void build_coarse(MgHierarchy& H, double* inv64_scratch, int* singular, cudaStream_t s) {
    // level 0's smoother: the inverses of A0's C blocks (the point-block Jacobi ones)
    launch_block_inverse_f32(NU, (long long)H.nx[0] * H.ny[0], H.A[0], inv64_scratch, H.Dinv[0], singular, s);
    for (int l = 1; l < H.nlev; ++l) {
        const long long Nc = (long long)H.nx[l] * H.ny[l];
        k_mg_galerkin<NU><<<grid_for(Nc), kMgThreads, 0, s>>>(H.nx[l - 1], H.ny[l - 1], H.px, H.py, H.A[l - 1],
                                                               H.nx[l], H.ny[l], H.A[l]);
        launch_block_inverse_f32(NU, Nc, H.A[l], inv64_scratch, H.Dinv[l], singular, s);
    }
}

int mg_launches_per_build(const MgHierarchy& H, bool direct) {
    const int mx = mg_colour_period(H.nx[0], H.px), my = mg_colour_period(H.ny[0], H.py);
    // direct assembly or probes + extracts (their J v counted by the caller's operator), Galerkin + inverse
    return (direct ? 1 : 2 * mx * my * H.nu) + 1 + 2 * (H.nlev - 1);
}

void mg_build(MgHierarchy& H, const MgJvOp& J, const MgDirect* direct, double* inv64_scratch, int* singular,
              cudaStream_t s) {
    if (H.nu == 3) {
        if (direct) {
            const long long N = (long long)H.nx[0] * H.ny[0];
            k_mg_assemble2d<<<grid_for(N), kMgThreads, 0, s>>>(*direct->g, direct->U, direct->pj, H.A[0]);
        } else {
            assemble_level0<3>(H, J, s);
        }
        build_coarse<3>(H, inv64_scratch, singular, s);
    } else {
        assemble_level0<4>(H, J, s);
        build_coarse<4>(H, inv64_scratch, singular, s);
    }
}

template <int NU>
static void cycle(const MgHierarchy& H, const MgJvOp& J, const float* r0, float* zout, cudaStream_t s) {
    // level 0 pre-smoothing and restriction
    const int nx0 = H.nx[0], ny0 = H.ny[0];
    const long long N0 = (long long)nx0 * ny0;
    const bool fused = J.down0 && J.up0 && H.nlev > 1;  // level 0 in two tiled passes
    if (!fused) k_mg_jacobi0<NU><<<grid_for(N0), kMgThreads, 0, s>>>(N0, H.Dinv[0], r0, H.z[0]);
    if (H.nlev == 1) {
        // the fine grid is already the coarsest: the coarsest level's sweeps with J
        // itself, ping-ponging between z[0] and z2[0], the last one into zout
        float* a = H.z[0];
        float* b = H.z2[0];
        for (int k = 1; k < kMgCoarseSweeps; ++k) {
            J.apply(J.ctx, a, H.w0, s);
            float* dst = k == kMgCoarseSweeps - 1 ? zout : b;
            k_mg_post0<NU><<<grid_for(N0), kMgThreads, 0, s>>>(N0, H.Dinv[0], r0, H.w0, a, dst);
            b = a;
            a = dst;
        }
        if (kMgCoarseSweeps == 1) cudaMemcpyAsync(zout, a, sizeof(float) * NU * N0, cudaMemcpyDeviceToDevice, s);
        return;
    }
    const long long N1 = (long long)H.nx[1] * H.ny[1];
    if (fused) {
        J.down0(J.ctx, r0, kMgOmega, H.z[0], H.nx[1], H.ny[1], H.r[1], s);
    } else {
        J.apply(J.ctx, H.z[0], H.w0, s);
        k_mg_restrict_diff<NU><<<grid_for(N1), kMgThreads, 0, s>>>(nx0, ny0, r0, H.w0, H.nx[1], H.ny[1], H.r[1]);
    }
    // down the assembled levels
    for (int l = 1; l < H.nlev - 1; ++l) {
        const dim3 grid((H.nx[l] + kMgTX - 1) / kMgTX, (H.ny[l] + kMgTY - 1) / kMgTY), block(kMgTX, kMgTY);
        launch_pdl(k_mg_down<NU>, grid, block, s, H.nx[l], H.ny[l], H.px, H.py, (const float*)H.A[l],
                   (const float*)H.Dinv[l], (const float*)H.r[l], H.z[l], H.nx[l + 1], H.ny[l + 1], H.r[l + 1]);
    }
    const int L = H.nlev - 1;
    launch_pdl(k_mg_coarsest<NU>, dim3(1), dim3(kMgCoarsest * kMgCoarsest), s, H.nx[L], H.ny[L], H.px, H.py,
               (const float*)H.A[L], (const float*)H.Dinv[L], (const float*)H.r[L], H.z2[L], kMgCoarseSweeps);
    // up
    for (int l = L - 1; l >= 1; --l) {
        const dim3 grid((H.nx[l] + kMgTX - 1) / kMgTX, (H.ny[l] + kMgTY - 1) / kMgTY), block(kMgTX, kMgTY);
        launch_pdl(k_mg_up<NU>, grid, block, s, H.nx[l], H.ny[l], H.px, H.py, (const float*)H.A[l],
                   (const float*)H.Dinv[l], (const float*)H.r[l], (const float*)H.z[l], (const float*)H.z2[l + 1],
                   H.nx[l + 1], H.ny[l + 1], H.z2[l]);
    }
    // level 0: prolong, J v, post-smoothing
    if (fused) {
        J.up0(J.ctx, r0, H.z[0], H.z2[1], H.nx[1], H.ny[1], kMgOmega, zout, s);
        return;
    }
    k_mg_prolong_add<NU><<<grid_for(N0), kMgThreads, 0, s>>>(nx0, ny0, H.z2[1], H.nx[1], H.ny[1], H.z[0]);
    J.apply(J.ctx, H.z[0], H.w0, s);
    k_mg_post0<NU><<<grid_for(N0), kMgThreads, 0, s>>>(N0, H.Dinv[0], r0, H.w0, H.z[0], zout);
}

int mg_launches_per_cycle(const MgHierarchy& H, bool fused) {
    if (H.nlev == 1) return 1 + 2 * (kMgCoarseSweeps - 1);
    return (fused ? 2 : 6) + (H.nlev - 2) + 1 + (H.nlev - 2);
}

double mg_cycle_bytes(const MgHierarchy& H, bool fused, bool fixed_eigs) {
    // minimum traffic in FP32 words: level 0 reads r, M^-1, dP/dU and the face
    // data (sigma_a, sigma_f, alpha per axis, lambda+- per axis unless fixed)
    // and writes z in the down pass and zout in the up pass; assembled levels
    // read A (5 n_u^2), M^-1 (n_u^2), r and z per pass; restriction and
    // prolongation add n_u words per coarse cell
    const double nu = H.nu, faces = 2.0 + 2.0 + (fixed_eigs ? 0.0 : 4.0);
    auto cells = [&](int l) { return (double)H.nx[l] * H.ny[l]; };
    if (H.nlev == 1) return 4.0 * cells(0) * kMgCoarseSweeps * (3.0 * nu + nu * nu + 9.0 + faces);
    double w = 0.0;
    const double lvl0 = fused ? (nu + nu * nu + 9.0 + faces + nu) + (2.0 * nu + nu * nu + 9.0 + faces + nu)
                              : 2.0 * (3.0 * nu + nu * nu + 9.0 + faces) + 4.0 * nu;
    w += cells(0) * lvl0 + 2.0 * nu * cells(1);
    for (int l = 1; l < H.nlev - 1; ++l)
        w += cells(l) * 2.0 * (5.0 * nu * nu + nu * nu + 3.0 * nu) + 2.0 * nu * cells(l + 1);
    w += cells(H.nlev - 1) * (5.0 * nu * nu + nu * nu + 2.0 * nu);
    return 4.0 * w;
}

void mg_cycle(const MgHierarchy& H, const MgJvOp& J, const float* r0, float* zout, cudaStream_t s) {
    if (H.nu == 3)
        cycle<3>(H, J, r0, zout, s);
    else
        cycle<4>(H, J, r0, zout, s);
}

}  // namespace m1
