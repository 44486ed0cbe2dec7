// m1_mg.cu — aggregation multigrid V-cycle for the 2D Newton system (FP32).
//
// The structured-grid analogue of the algebraic multigrid the paper found best
// among its preconditioners (Sect. 3.3.2, Sect. 4):
//   level 0: the Jacobian itself, applied matrix-free by the linear J v, its
//     point-block inverses (the block-Jacobi ones) as smoother; its 5-point
//     stencil of n_u x n_u blocks (C, W, E, S, N = self, -x, +x, -y, +y) is read
//     off J v by coloured probes (a vector that is 1 on one unknown of every
//     cell of one colour class; cells of a class are >= 3 apart, also across a
//     periodic wrap, so each response entry belongs to one probed cell), only to
//     build the coarse levels;
//   levels >= 1: 2 x 2 cell aggregates, piecewise-constant prolongation P,
//     restriction P^T (the sum over the aggregate) and the Galerkin stencil
//     P^T A P — again a 5-point block stencil (a fine coupling inside the
//     aggregate adds to C, one leaving it adds to the block of its direction);
//   the cycle: V(1,1) with damped point-block Jacobi (omega = 0.7) from zero,
//     10 damped sweeps from zero on the coarsest level (both sides <= 32 cells,
//     one CTA, the iterate in shared memory).
// Blocks are stored A[((s n_u + r) n_u + c) N + i]; the block inverses of the
// C blocks [(r n_u + c) N + i] like the block-Jacobi ones.
#include "m1_internal.h"

#include <algorithm>

namespace m1 {

constexpr float kMgOmega = 0.7f;
constexpr int kMgCoarsest = 32;
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

// (A z)_i on an assembled level, z optionally plus the prolonged coarse zc
template <int NU>
__device__ __forceinline__ void mg_apply_cell(const float* __restrict__ A, const float* __restrict__ z,
                                              const float* __restrict__ zc, int nx, int ny, bool px, bool py,
                                              int nxc, int ix, int iy, long long N, long long Nc, float* out) {
    const long long i = (long long)iy * nx + ix;
#pragma unroll
    for (int r = 0; r < NU; ++r) out[r] = 0.f;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const long long j = mg_nb(ix, iy, s, nx, ny, px, py);
        if (j < 0) continue;
        float zj[NU];
        const long long J = zc ? (long long)((j / nx) / 2) * nxc + (j % nx) / 2 : 0;
#pragma unroll
        for (int c = 0; c < NU; ++c) zj[c] = z[c * N + j] + (zc ? zc[c * Nc + J] : 0.f);
#pragma unroll
        for (int r = 0; r < NU; ++r)
#pragma unroll
            for (int c = 0; c < NU; ++c) out[r] += A[((long long)(s * NU + r) * NU + c) * N + i] * zj[c];
    }
}

// rc = P^T (r - A z) on an assembled level (one thread per coarse cell)
template <int NU>
__global__ void k_mg_resid_restrict(int nx, int ny, bool px, bool py, const float* __restrict__ A,
                                    const float* __restrict__ r, const float* __restrict__ z, int nxc, int nyc,
                                    float* __restrict__ rc) {
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
                float az[NU];
                mg_apply_cell<NU>(A, z, nullptr, nx, ny, px, py, nxc, ix, iy, N, Nc, az);
#pragma unroll
                for (int c = 0; c < NU; ++c) acc[c] += r[c * N + i] - az[c];
            }
#pragma unroll
        for (int c = 0; c < NU; ++c) rc[c * Nc + I] = acc[c];
    }
}

// zout = zz + omega D^-1 (r - A zz), zz = z + P zc, on an assembled level
template <int NU>
__global__ void k_mg_prolong_post(int nx, int ny, bool px, bool py, const float* __restrict__ A,
                                  const float* __restrict__ Dinv, const float* __restrict__ r,
                                  const float* __restrict__ z, const float* __restrict__ zc, int nxc, int nyc,
                                  float* __restrict__ zout) {
    const long long N = (long long)nx * ny, Nc = (long long)nxc * nyc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)(i / nx);
        float az[NU], res[NU];
        mg_apply_cell<NU>(A, z, zc, nx, ny, px, py, nxc, ix, iy, N, Nc, az);
        const long long I = (long long)(iy / 2) * nxc + ix / 2;
#pragma unroll
        for (int c = 0; c < NU; ++c) res[c] = r[c * N + i] - az[c];
#pragma unroll
        for (int q = 0; q < NU; ++q) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NU; ++c) a += Dinv[(long long)(q * NU + c) * N + i] * res[c];
            zout[q * N + i] = z[q * N + i] + zc[q * Nc + I] + kMgOmega * a;
        }
    }
}

// coarsest level: sweeps of z <- z + omega D^-1 (r - A z) from zero, one CTA,
// the iterate double-buffered in shared memory (N <= kMgCoarsest^2)
template <int NU>
__global__ void __launch_bounds__(1024) k_mg_coarsest(int nx, int ny, bool px, bool py, const float* __restrict__ A,
                                                      const float* __restrict__ Dinv, const float* __restrict__ r,
                                                      float* __restrict__ zout, int sweeps) {
    __shared__ float zs[2][NU][kMgCoarsest * kMgCoarsest];
    const int N = nx * ny;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
#pragma unroll
        for (int c = 0; c < NU; ++c) zs[0][c][i] = 0.f;
    __syncthreads();
    int cur = 0;
    for (int k = 0; k < sweeps; ++k) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int ix = i % nx, iy = i / nx;
            float res[NU];
#pragma unroll
            for (int q = 0; q < NU; ++q) res[q] = r[q * N + i];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const long long j = mg_nb(ix, iy, s, nx, ny, px, py);
                if (j < 0) continue;
#pragma unroll
                for (int q = 0; q < NU; ++q)
#pragma unroll
                    for (int c = 0; c < NU; ++c)
                        res[q] -= A[((long long)(s * NU + q) * NU + c) * N + i] * zs[cur][c][j];
            }
#pragma unroll
            for (int q = 0; q < NU; ++q) {
                float a = 0.f;
#pragma unroll
                for (int c = 0; c < NU; ++c) a += Dinv[(long long)(q * NU + c) * N + i] * res[c];
                zs[cur ^ 1][q][i] = zs[cur][q][i] + kMgOmega * a;
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x)
#pragma unroll
        for (int c = 0; c < NU; ++c) zout[c * N + i] = zs[cur][c][i];
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
    for (int l = 1; l < H.nlev; ++l) {
        const long long Nc = (long long)H.nx[l] * H.ny[l];
        k_mg_galerkin<NU><<<grid_for(Nc), kMgThreads, 0, s>>>(H.nx[l - 1], H.ny[l - 1], H.px, H.py, H.A[l - 1],
                                                               H.nx[l], H.ny[l], H.A[l]);
        launch_block_inverse_f32(NU, Nc, H.A[l], inv64_scratch, H.Dinv[l], singular, s);
    }
}

int mg_launches_per_build(const MgHierarchy& H) {
    const int mx = mg_colour_period(H.nx[0], H.px), my = mg_colour_period(H.ny[0], H.py);
    return 1 + 2 * mx * my * H.nu + 2 * (H.nlev - 1);  // memset aside: probes + extracts, Galerkin + inverse
}

void mg_build(MgHierarchy& H, const MgJvOp& J, double* inv64_scratch, int* singular, cudaStream_t s) {
    if (H.nu == 3) {
        assemble_level0<3>(H, J, s);
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
    k_mg_jacobi0<NU><<<grid_for(N0), kMgThreads, 0, s>>>(N0, H.Dinv[0], r0, H.z[0]);
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
    J.apply(J.ctx, H.z[0], H.w0, s);
    const long long N1 = (long long)H.nx[1] * H.ny[1];
    k_mg_restrict_diff<NU><<<grid_for(N1), kMgThreads, 0, s>>>(nx0, ny0, r0, H.w0, H.nx[1], H.ny[1], H.r[1]);
    // down the assembled levels
    for (int l = 1; l < H.nlev - 1; ++l) {
        const long long N = (long long)H.nx[l] * H.ny[l], Nc = (long long)H.nx[l + 1] * H.ny[l + 1];
        k_mg_jacobi0<NU><<<grid_for(N), kMgThreads, 0, s>>>(N, H.Dinv[l], H.r[l], H.z[l]);
        k_mg_resid_restrict<NU><<<grid_for(Nc), kMgThreads, 0, s>>>(H.nx[l], H.ny[l], H.px, H.py, H.A[l], H.r[l],
                                                                     H.z[l], H.nx[l + 1], H.ny[l + 1], H.r[l + 1]);
    }
    const int L = H.nlev - 1;
    k_mg_coarsest<NU><<<1, 1024, 0, s>>>(H.nx[L], H.ny[L], H.px, H.py, H.A[L], H.Dinv[L], H.r[L], H.z2[L],
                                         kMgCoarseSweeps);
    // up
    for (int l = L - 1; l >= 1; --l) {
        const long long N = (long long)H.nx[l] * H.ny[l];
        k_mg_prolong_post<NU><<<grid_for(N), kMgThreads, 0, s>>>(H.nx[l], H.ny[l], H.px, H.py, H.A[l], H.Dinv[l],
                                                                  H.r[l], H.z[l], H.z2[l + 1], H.nx[l + 1],
                                                                  H.ny[l + 1], H.z2[l]);
    }
    // level 0: prolong, J v, post-smoothing
    k_mg_prolong_add<NU><<<grid_for(N0), kMgThreads, 0, s>>>(nx0, ny0, H.z2[1], H.nx[1], H.ny[1], H.z[0]);
    J.apply(J.ctx, H.z[0], H.w0, s);
    k_mg_post0<NU><<<grid_for(N0), kMgThreads, 0, s>>>(N0, H.Dinv[0], r0, H.w0, H.z[0], zout);
}

int mg_launches_per_cycle(const MgHierarchy& H) {
    if (H.nlev == 1) return 1 + 2 * (kMgCoarseSweeps - 1);
    return 6 + 2 * (H.nlev - 2) + 1 + (H.nlev - 2);
}

void mg_cycle(const MgHierarchy& H, const MgJvOp& J, const float* r0, float* zout, cudaStream_t s) {
    if (H.nu == 3)
        cycle<3>(H, J, r0, zout, s);
    else
        cycle<4>(H, J, r0, zout, s);
}

}  // namespace m1
