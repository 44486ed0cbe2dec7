// m1_fallback.cu — kernels of the admissibility fallback of the implicit step.
//
// Sect. 3.1.3 of Bloch et al. (2021) cannot show that the asymptotic-preserving,
// well-balanced scheme keeps f = |F| / (cE) <= 1, observes f > 1 near free
// streaming, and names two remedies: enforcing f < 1, or the centred source of
// Eq. (wb_naive). The library applies the second one a posteriori, cell by
// cell: a flagged cell takes the centred flux source, and each face of a flagged
// cell takes alpha = 1 and the speeds -c, +c (HLL with the largest speeds of the
// M1 system). With sigma_f >= sigma_a the backward-Euler update of that scheme
// is a convex combination of admissible states, so it stays admissible.
//
// The kernels here: the face fix-up of the time-n face data, the two flagging
// rules (inadmissible cells; cells where Newton stalls, by the size of their
// residual), the largest per-cell residual, and the per-cell step factor that
// keeps flagged cells admissible during the Newton iteration.
#include "m1_internal.h"

namespace m1 {
namespace {

constexpr int kFbThreads = 256;

inline int fb_blocks(long long n) { return (int)std::min<long long>((n + kFbThreads - 1) / kFbThreads, 152LL * 16); }

// Faces of axis a with a flagged cell on either side get lambda+ = c,
// lambda- = -c, alpha = 1. A non-periodic boundary face follows its one cell;
// the two end faces of a periodic axis (the same physical face) follow both.
__global__ void k_fallback_faces(int a, int nx, int ny, int nz, int periodic, double c,
                                 const unsigned char* __restrict__ fb, double* __restrict__ lam_p,
                                 double* __restrict__ lam_m, double* __restrict__ alpha) {
    int fn[3] = {nx, ny, nz};
    const int n[3] = {nx, ny, nz};
    fn[a] += 1;
    const long long nf = (long long)fn[0] * fn[1] * fn[2];
    const long long stride[3] = {1, nx, (long long)nx * ny};
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf;
         f += (long long)gridDim.x * blockDim.x) {
        int coord[3];
        {
            const long long q = f / fn[0];
            coord[0] = (int)(f - q * fn[0]);
            coord[2] = (int)(q / fn[1]);
            coord[1] = (int)(q - (long long)coord[2] * fn[1]);
        }
        const int fa = coord[a];
        int cc[3] = {coord[0], coord[1], coord[2]};
        cc[a] = 0;
        const long long base = ((long long)cc[2] * ny + cc[1]) * nx + cc[0];
        int left = fa - 1, right = fa;
        if (left < 0) left = periodic ? n[a] - 1 : right;
        if (right >= n[a]) right = periodic ? 0 : left;
        const bool flagged = fb[base + (long long)left * stride[a]] || fb[base + (long long)right * stride[a]];
        if (flagged) {
            lam_p[f] = c;
            lam_m[f] = -c;
            alpha[f] = 1.0;
        }
    }
}

// Flag the unflagged cells that meet the rule. rule 0: outside the admissible
// set, E <= 0 or |F| > cE (their iterate is reset to U^n, which is
// admissible); rule 1: the largest residual component of the cell is at least
// `thresh` (admissible cells where Newton stalls: their iterate is kept).
// count += cells flagged.
__global__ void k_fallback_flag(int rule, int nu, int dim, long long N, double c, double thresh,
                                double* __restrict__ U, const double* __restrict__ R, const double* __restrict__ Un,
                                unsigned char* __restrict__ fb, unsigned long long* __restrict__ count) {
    unsigned long long mine = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        if (fb[i]) continue;
        bool flag;
        if (rule == 0) {
            const double E = U[i];
            double F2 = 0.0;
            for (int b = 0; b < dim; ++b) {
                const double F = U[(1 + b) * N + i];
                F2 += F * F;
            }
            flag = !(E > 0.0) || sqrt(F2) > c * E;
        } else {
            double m = 0.0;
            for (int k = 0; k < nu; ++k) m = fmax(m, fabs(R[k * N + i]));
            flag = m >= thresh;
        }
        if (flag) {
            fb[i] = 1;
            if (rule == 0)
                for (int k = 0; k < nu; ++k) U[k * N + i] = Un[k * N + i];
            ++mine;
        }
    }
    // warp sum, one atomic per warp with a flag (the count is an integer: order-free)
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

// out = max over cells and components of |R| (non-negative doubles order like
// their bit patterns, so the maximum is taken on the integers: order-free)
__global__ void k_residual_absmax(int nu, long long N, const double* __restrict__ R,
                                  unsigned long long* __restrict__ out) {
    double m = 0.0;
    const long long n = (long long)nu * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(R[i]));
    unsigned long long b = (unsigned long long)__double_as_longlong(m);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

// In every flagged cell scale the Newton update delta (all components) by
// theta_i: 1 when U_i + delta_i is admissible, else 0.9 times the first of
// 1/2, 1/4, ... (at most 40 halvings) that is. The admissible set is convex,
// so from an admissible U_i the admissible part of the segment is an interval.
__global__ void k_admissible_theta(int nu, int dim, long long N, double c, const double* __restrict__ U,
                                   double* __restrict__ delta, const unsigned char* __restrict__ fb) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        if (!fb[i]) continue;
        const double E = U[i], dE = delta[i];
        double F[3] = {0.0, 0.0, 0.0}, dF[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < dim; ++b) {
            F[b] = U[(1 + b) * N + i];
            dF[b] = delta[(1 + b) * N + i];
        }
        double th = 1.0;
        for (int k = 0; k < 40; ++k) {
            const double Et = E + th * dE;
            double F2 = 0.0;
            for (int b = 0; b < dim; ++b) {
                const double Ft = F[b] + th * dF[b];
                F2 += Ft * Ft;
            }
            if (Et > 0.0 && sqrt(F2) <= c * Et) break;
            th *= 0.5;
        }
        if (th < 1.0) {
            th *= 0.9;
            for (int k = 0; k < nu; ++k) delta[k * N + i] *= th;
        }
    }
}

}  // namespace

void launch_fallback_faces(const Dev<double>& g, const unsigned char* fb, double* const lam_p[3],
                           double* const lam_m[3], double* const alpha[3], cudaStream_t s) {
    for (int a = 0; a < g.dim; ++a) {
        const long long nf = g.N / g.n[a] * (g.n[a] + 1);
        k_fallback_faces<<<fb_blocks(nf), kFbThreads, 0, s>>>(a, g.n[0], g.n[1], g.n[2], g.bc[a][0] == BC_PERIODIC,
                                                             (double)g.c, fb, lam_p[a], lam_m[a], alpha[a]);
    }
}

void launch_fallback_flag(int rule, int nu, int dim, long long N, double c, double thresh, double* U,
                          const double* R, const double* Un, unsigned char* fb, unsigned long long* count,
                          cudaStream_t s) {
    k_fallback_flag<<<fb_blocks(N), kFbThreads, 0, s>>>(rule, nu, dim, N, c, thresh, U, R, Un, fb, count);
}

void launch_residual_absmax(int nu, long long N, const double* R, unsigned long long* out, cudaStream_t s) {
    k_residual_absmax<<<fb_blocks((long long)nu * N), kFbThreads, 0, s>>>(nu, N, R, out);
}

void launch_admissible_theta(int nu, int dim, long long N, double c, const double* U, double* delta,
                             const unsigned char* fb, cudaStream_t s) {
    k_admissible_theta<<<fb_blocks(N), kFbThreads, 0, s>>>(nu, dim, N, c, U, delta, fb);
}

}  // namespace m1
