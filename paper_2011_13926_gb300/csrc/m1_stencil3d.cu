// m1_stencil3d.cu — J v of the 3D backward-Euler residual (Sect. 3.1.1 scheme),
// tiled in x-y and marching in z (2.5D), for wave speeds frozen at time n or
// fixed.
//
// With the wave speeds frozen, J v is linear in the derivative quantities of
// the cells, dE, dF and dP = (dP/dU) v: the HLL fluxes, the asymptotic
// correction, the well-balanced or centred flux source and the exchange are
// linear combinations of them with coefficients that depend only on the face
// data and the opacities. Each CTA owns a 32 x 8 column of cells over a slab of
// z planes. For every plane it evaluates the closure of each cell of the tile
// and its one-cell x-y halo once, by forward-mode dual numbers along v (ghosts
// through the boundary rules), and keeps (dE, dF, dP) of three consecutive
// planes in a shared-memory ring; each thread then forms the six faces and the
// sources of its cell of the middle plane, in the order of cell_residual.
#include "m1_internal.h"

namespace m1 {
namespace {

constexpr int kTX3 = 32, kTY3 = 8, kKZ3 = 16;  // tile and slab depth
constexpr int kHX3 = kTX3 + 2, kHY3 = kTY3 + 2;

template <class R>
struct CellD3 {
    R dE, dF[3], dP[6];  // P components (xx, xy, xz, yy, yz, zz)
    R sig;               // flux opacity of the cell (ghost: the boundary rule's)
};

__device__ __forceinline__ int pidx(int a, int b) {  // (a, b) -> index of the symmetric 3 x 3 tensor
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

// derivative quantities of the cell at (gx, gy, gz), which may be a ghost along
// one axis; false for positions no face needs (out along two axes, or past the
// last ghost)
template <class R, class A, bool GAS>
__device__ __forceinline__ bool stage_cell(const Dev<R>& g, const R* __restrict__ U, const R* __restrict__ v,
                                           int gx, int gy, int gz, CellD3<A>& c) {
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const bool ix = gx >= 0 && gx < n0, iy = gy >= 0 && gy < n1, iz = gz >= 0 && gz < n2;
    const int out = (!ix) + (!iy) + (!iz);
    if (out > 1 || gx < -1 || gx > n0 || gy < -1 || gy > n1 || gz < -1 || gz > n2) return false;
    LoadDir<R, A> ld{U, v, g.N};
    St<Dual<A>, 3> u;
    if (out == 0) {
        const long long k = ((long long)gz * n1 + gy) * n0 + gx;
        u = load_state<Dual<A>, 3, GAS>(ld, k, k);
        c.sig = g.sig_f[k];
    } else {
        const int a = !ix ? 0 : (!iy ? 1 : 2);
        const int side = a == 0 ? (gx < 0 ? 0 : 1) : (a == 1 ? (gy < 0 ? 0 : 1) : (gz < 0 ? 0 : 1));
        int cc[3] = {gx, gy, gz};
        cc[a] = side ? g.n[a] - 1 : 0;
        const long long k = ((long long)cc[2] * n1 + cc[1]) * n0 + cc[0];
        const St<Dual<A>, 3> self = load_state<Dual<A>, 3, GAS>(ld, k, k);
        R sn;
        bool bnd;
        u = neighbour<Dual<A>, 3, GAS>(g, ld, self, k, cc, a, side, sn, bnd);
        c.sig = sn;
    }
    const Cl<Dual<A>, 3> kl = closure(u, g.c);
    c.dE = u.E.d;
#pragma unroll
    for (int b = 0; b < 3; ++b) c.dF[b] = u.F[b].d;
    c.dP[0] = pressure(kl, 0, 0).d;
    c.dP[1] = pressure(kl, 0, 1).d;
    c.dP[2] = pressure(kl, 0, 2).d;
    c.dP[3] = pressure(kl, 1, 1).d;
    c.dP[4] = pressure(kl, 1, 2).d;
    c.dP[5] = pressure(kl, 2, 2).d;
    return true;
}

// R: the arrays; A: the arithmetic (R, or the double-word DF on FP64 arrays)
// FP32: four CTAs per SM (64 registers), double words three (80)
template <class R, class A, bool GAS>
__global__ void __launch_bounds__(kTX3* kTY3, std::is_same<A, float>::value ? 4 : (std::is_same<A, DF>::value ? 3 : 1))
    k_jv3d_tiled(Dev<R> g, const R* __restrict__ U,
                                                          const R* __restrict__ v, R* __restrict__ Jv) {
    extern __shared__ __align__(16) unsigned char smem3[];
    CellD3<A>(*ring)[kHY3][kHX3] = reinterpret_cast<CellD3<A>(*)[kHY3][kHX3]>(smem3);
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const long long N = g.N;
    const int x0 = blockIdx.x * kTX3, y0 = blockIdx.y * kTY3, z0 = blockIdx.z * kKZ3;
    const int z1 = min(z0 + kKZ3, n2);
    const int tid = threadIdx.y * kTX3 + threadIdx.x;
    const int ix = x0 + threadIdx.x, iy = y0 + threadIdx.y;
    const bool col = ix < n0 && iy < n1;
    auto stage_plane = [&](int gz) {
        CellD3<A>(*pl)[kHX3] = ring[(gz + 3) % 3];
        for (int t = tid; t < kHX3 * kHY3; t += kTX3 * kTY3) {
            const int hx = t % kHX3, hy = t / kHX3;
            CellD3<A> c;
            if (stage_cell<R, A, GAS>(g, U, v, x0 + hx - 1, y0 + hy - 1, gz, c)) pl[hy][hx] = c;
        }
    };
    stage_plane(z0 - 1);
    stage_plane(z0);
    const A dt = g.dt, c = g.c, c2 = g.c * g.c, cdt = g.c * g.dt;
    for (int iz = z0; iz < z1; ++iz) {
        stage_plane(iz + 1);
        __syncthreads();
        if (col) {
            const long long idx = ((long long)iz * n1 + iy) * n0 + ix;
            const int coord[3] = {ix, iy, iz};
            const CellD3<A>& me = ring[(iz + 3) % 3][threadIdx.y + 1][threadIdx.x + 1];
            const A sig_self = me.sig;
            const bool wbc = g.wb && !(g.fb && g.fb[idx]);
            A RE = me.dE, RF[3] = {me.dF[0], me.dF[1], me.dF[2]};
            A phi[3] = {A(0), A(0), A(0)};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int o = side ? 1 : -1;
                    const CellD3<A>& nb = a == 2 ? ring[(iz + o + 3) % 3][threadIdx.y + 1][threadIdx.x + 1]
                                                 : ring[(iz + 3) % 3][threadIdx.y + 1 + (a == 1 ? o : 0)]
                                                       [threadIdx.x + 1 + (a == 0 ? o : 0)];
                    const CellD3<A>& Lc = side ? me : nb;
                    const CellD3<A>& Rc = side ? nb : me;
                    const int ca = coord[a] + o;
                    const bool inside = ca >= 0 && ca < g.n[a];
                    const bool boundary = !inside && g.bc[a][side] != BC_PERIODIC;
                    const long long fidx = face_index(g.n, coord, a, coord[a] + side);
                    A lp, lm;
                    if (g.fixed_eigs) {
                        lp = c;
                        lm = -c;
                    } else {
                        lp = g.lam_p[a][fidx];
                        lm = g.lam_m[a][fidx];
                    }
                    const A den = lp - lm;
                    const A inv = den >= Tiny<A>::den() ? A(1) / den : A(0);
                    const A pm = lp * lm * inv;
                    const A Fs = (lp * Lc.dF[a] - lm * Rc.dF[a]) * inv + pm * (Rc.dE - Lc.dE);
                    const A w = (side ? dt : -dt) * g.inv_dx[a];
                    RE += (w * g.alpha[a][fidx]) * Fs;
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int q = pidx(a, b);
                        const A Ps = c2 * (lp * Lc.dP[q] - lm * Rc.dP[q]) * inv + pm * (Rc.dF[b] - Lc.dF[b]);
                        RF[b] += w * Ps;
                    }
                    if (wbc) {
                        if (boundary && g.wb_boundary) {
                            const int q = pidx(a, a);
                            phi[a] -= c * g.inv_dx[a] * (Rc.dP[q] - Lc.dP[q]);
                        } else {
                            phi[a] += (A(0.25) * (sig_self + nb.sig)) * (Lc.dF[a] + Rc.dF[a]);
                        }
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < 3; ++b) RF[b] += cdt * (wbc ? A(0.5) * phi[b] : sig_self * me.dF[b]);
            A demis = A(0), dT = A(0);
            if constexpr (GAS) {
                const A T = U[4 * N + idx];
                dT = v[4 * N + idx];
                demis = A(4) * g.a_r * T * T * T * dT;
            }
            const A exch = (cdt * g.sig_a[idx]) * (demis - me.dE);
            RE -= exch;
            Jv[idx] = to_mem<R>(RE);
#pragma unroll
            for (int b = 0; b < 3; ++b) Jv[(1 + b) * N + idx] = to_mem<R>(RF[b]);
            if constexpr (GAS) Jv[4 * N + idx] = to_mem<R>(g.rho_cv[idx] * dT + exch);
        }
        __syncthreads();  // the ring slot of plane iz - 1 is staged next
    }
}

template <class R, class A, bool GAS>
void launch3d(const Dev<R>& g, const R* U, const R* v, R* Jv, cudaStream_t s) {
    constexpr int bytes = 3 * kHY3 * kHX3 * (int)sizeof(CellD3<A>);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_jv3d_tiled<R, A, GAS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        attr = true;
    }
    const dim3 grid((g.n[0] + kTX3 - 1) / kTX3, (g.n[1] + kTY3 - 1) / kTY3, (g.n[2] + kKZ3 - 1) / kKZ3);
    k_jv3d_tiled<R, A, GAS><<<grid, dim3(kTX3, kTY3), bytes, s>>>(g, U, v, Jv);
}

template <class R>
bool eligible(const Dev<R>& g) {
    return g.dim == 3 && !(g.implicit_eigs && !g.fixed_eigs);
}

}  // namespace

bool launch_jv3d_tiled_f64(const Dev<double>& g, const double* U, const double* v, double* Jv, cudaStream_t s) {
    if (!eligible(g)) return false;
    if (g.df) {
        if (g.gas)
            launch3d<double, DF, true>(g, U, v, Jv, s);
        else
            launch3d<double, DF, false>(g, U, v, Jv, s);
    } else if (g.gas) {
        launch3d<double, double, true>(g, U, v, Jv, s);
    } else {
        launch3d<double, double, false>(g, U, v, Jv, s);
    }
    return true;
}

bool launch_jv3d_tiled_f32(const Dev<float>& g, const float* U, const float* v, float* Jv, cudaStream_t s) {
    if (!eligible(g)) return false;
    if (g.gas)
        launch3d<float, float, true>(g, U, v, Jv, s);
    else
        launch3d<float, float, false>(g, U, v, Jv, s);
    return true;
}

}  // namespace m1
