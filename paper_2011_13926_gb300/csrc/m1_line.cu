// m1_line.cu — block-tridiagonal line preconditioner for 1D grids (FP64).
//
// On a 1D grid the backward-Euler residual of cell i depends on cells i - 1,
// i, i + 1 only (HLL faces, the well-balanced face averages, the boundary
// ghosts through the edge cells), so J is block tridiagonal with n_u x n_u
// blocks L_i = dR_i/dU_{i-1}, D_i = dR_i/dU_i, U_i = dR_i/dU_{i+1}. The
// preconditioner is that block-tridiagonal matrix, solved exactly by block
// Gaussian elimination along the line (the block Thomas algorithm); on a
// non-periodic grid it is J itself, and GMRES converges in one step. On a
// periodic grid the wrap's two corner blocks are left out. The blocks come
// from dual numbers, one seeded unknown of one neighbour at a time; the
// factorisation and the two substitution sweeps run in one thread (a line
// is one sequential recurrence; 1D grids are small).
#include "m1_internal.h"

namespace m1 {

constexpr int kLineThreads = 256;

// seed component k of cell j
struct LoadSeedAt {
    const double* U;
    long long N;
    int k;
    long long j;
    __device__ __forceinline__ Dual<double> get(int comp, long long idx, long long) const {
        return {U[comp * N + idx], (idx == j && comp == k) ? 1.0 : 0.0};
    }
};

// blocks[((o n_u + r) n_u + c) N + i] = dR_r(i) / dU_c(i + o - 1), o = 0, 1, 2
// (left, self, right); a neighbour beyond a non-periodic end gives a zero block
template <bool GAS>
__global__ void __launch_bounds__(kLineThreads) k_line_assemble1d(Dev<double> g, const double* __restrict__ U,
                                                              double* __restrict__ blocks) {
    constexpr int NU = 2 + (GAS ? 1 : 0);
    const long long N = g.N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int coord[3] = {(int)i, 0, 0};
    const bool periodic = g.bc[0][0] == BC_PERIODIC;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        long long j = i + o - 1;
        const bool outside = j < 0 || j >= N;
        if (outside && periodic) j = j < 0 ? j + N : j - N;
#pragma unroll
        for (int c = 0; c < NU; ++c) {
            Dual<double> out[NU];
            if (outside && !periodic) {
#pragma unroll
                for (int r = 0; r < NU; ++r) out[r] = Dual<double>{0.0, 0.0};
            } else {
                LoadSeedAt ld{U, N, c, j};
                cell_residual<Dual<double>, 1, GAS>(g, ld, i, coord, out);
            }
#pragma unroll
            for (int r = 0; r < NU; ++r) blocks[((long long)(o * NU + r) * NU + c) * N + i] = out[r].d;
        }
    }
}

// Gauss-Jordan inverse with partial pivoting of an NU x NU block; false if singular
template <int NU>
__device__ bool line_inverse(const double (&A)[NU][NU], double (&Ai)[NU][NU]) {
    double a[NU][2 * NU];
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
        for (int c = 0; c < NU; ++c) {
            a[r][c] = A[r][c];
            a[r][NU + c] = r == c ? 1.0 : 0.0;
        }
    for (int col = 0; col < NU; ++col) {
        int piv = col;
        for (int r = col + 1; r < NU; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (!(fabs(a[piv][col]) > 0.0)) return false;
        if (piv != col)
            for (int c = 0; c < 2 * NU; ++c) {
                const double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        const double inv = 1.0 / a[col][col];
        for (int c = 0; c < 2 * NU; ++c) a[col][c] *= inv;
        for (int r = 0; r < NU; ++r) {
            if (r == col) continue;
            const double f = a[r][col];
            for (int c = 0; c < 2 * NU; ++c) a[r][c] -= f * a[col][c];
        }
    }
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
        for (int c = 0; c < NU; ++c) Ai[r][c] = a[r][NU + c];
    return true;
}

template <int NU>
__device__ __forceinline__ void line_block(const double* B, int o, long long N, long long i, double (&X)[NU][NU]) {
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
        for (int c = 0; c < NU; ++c) X[r][c] = B[((long long)(o * NU + r) * NU + c) * N + i];
}

// block Thomas factorisation: D'_0 = D_0; M_i = L_i D'_{i-1}^-1, D'_i = D_i - M_i U_{i-1};
// stores M_i and D'_i^-1 as [(r n_u + c) N + i]
template <int NU>
__global__ void k_line_factor(long long N, const double* __restrict__ B, double* __restrict__ Mf,
                              double* __restrict__ Dinv, int* singular) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double Dp[NU][NU], Di[NU][NU], L[NU][NU], Up[NU][NU], M[NU][NU];
    line_block<NU>(B, 1, N, 0, Dp);
    if (!line_inverse<NU>(Dp, Di)) *singular = 1;
    for (int r = 0; r < NU; ++r)
        for (int c = 0; c < NU; ++c) {
            Dinv[(long long)(r * NU + c) * N] = Di[r][c];
            Mf[(long long)(r * NU + c) * N] = 0.0;
        }
    for (long long i = 1; i < N; ++i) {
        line_block<NU>(B, 0, N, i, L);
        line_block<NU>(B, 2, N, i - 1, Up);
        line_block<NU>(B, 1, N, i, Dp);
        for (int r = 0; r < NU; ++r)
            for (int c = 0; c < NU; ++c) {
                double s = 0.0;
                for (int k = 0; k < NU; ++k) s += L[r][k] * Di[k][c];
                M[r][c] = s;
            }
        for (int r = 0; r < NU; ++r)
            for (int c = 0; c < NU; ++c) {
                double s = Dp[r][c];
                for (int k = 0; k < NU; ++k) s -= M[r][k] * Up[k][c];
                Dp[r][c] = s;
            }
        if (!line_inverse<NU>(Dp, Di)) *singular = 1;
        for (int r = 0; r < NU; ++r)
            for (int c = 0; c < NU; ++c) {
                Dinv[(long long)(r * NU + c) * N + i] = Di[r][c];
                Mf[(long long)(r * NU + c) * N + i] = M[r][c];
            }
    }
}

// z = T^-1 r: y_i = r_i - M_i y_{i-1} forward, z_i = D'_i^-1 (y_i - U_i z_{i+1}) backward (y kept in z)
template <int NU>
__global__ void k_line_solve(long long N, const double* __restrict__ B, const double* __restrict__ Mf,
                             const double* __restrict__ Dinv, const double* __restrict__ r, double* __restrict__ z) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double y[NU];
    for (int c = 0; c < NU; ++c) y[c] = r[c * N];
    for (int c = 0; c < NU; ++c) z[c * N] = y[c];
    for (long long i = 1; i < N; ++i) {
        double yi[NU];
        for (int q = 0; q < NU; ++q) {
            double s = r[q * N + i];
            for (int c = 0; c < NU; ++c) s -= Mf[(long long)(q * NU + c) * N + i] * y[c];
            yi[q] = s;
        }
        for (int c = 0; c < NU; ++c) {
            y[c] = yi[c];
            z[c * N + i] = yi[c];
        }
    }
    double x[NU] = {};
    for (long long i = N - 1; i >= 0; --i) {
        double t[NU];
        for (int q = 0; q < NU; ++q) {
            double s = z[q * N + i];
            if (i + 1 < N)
                for (int c = 0; c < NU; ++c) s -= B[((long long)(2 * NU + q) * NU + c) * N + i] * x[c];
            t[q] = s;
        }
        for (int q = 0; q < NU; ++q) {
            double s = 0.0;
            for (int c = 0; c < NU; ++c) s += Dinv[(long long)(q * NU + c) * N + i] * t[c];
            x[q] = s;
        }
        for (int q = 0; q < NU; ++q) z[q * N + i] = x[q];
    }
}

void launch_line_build(const Dev<double>& g, const double* U, double* blocks, double* Mf, double* Dinv,
                       int* singular, cudaStream_t s) {
    const int nb = (int)((g.N + kLineThreads - 1) / kLineThreads);
    if (g.gas) {
        k_line_assemble1d<true><<<nb, kLineThreads, 0, s>>>(g, U, blocks);
        k_line_factor<3><<<1, 32, 0, s>>>(g.N, blocks, Mf, Dinv, singular);
    } else {
        k_line_assemble1d<false><<<nb, kLineThreads, 0, s>>>(g, U, blocks);
        k_line_factor<2><<<1, 32, 0, s>>>(g.N, blocks, Mf, Dinv, singular);
    }
}

void launch_line_solve(int nu, long long N, const double* blocks, const double* Mf, const double* Dinv,
                       const double* r, double* z, cudaStream_t s) {
    if (nu == 3)
        k_line_solve<3><<<1, 32, 0, s>>>(N, blocks, Mf, Dinv, r, z);
    else
        k_line_solve<2><<<1, 32, 0, s>>>(N, blocks, Mf, Dinv, r, z);
}

}  // namespace m1
