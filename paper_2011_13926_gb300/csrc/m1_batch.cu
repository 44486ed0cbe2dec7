// m1_batch.cu — many independent implicit M1 steps in one persistent launch.
//
// Each CTA of a persistent kernel takes a problem from a device work queue
// (one atomic counter) and runs that problem's whole backward-Euler step on
// its own: time-n face data, Newton on the FP64 residual, point-block Jacobi
// built in FP32 and inverted in FP64, FP32 GMRES(m) (classical Gram-Schmidt
// with the same reorthogonalisation test as the single-grid path, FP64
// Hessenberg least squares) under FP64 refinement, and the Armijo line search.
// Only CTA-wide barriers are used: no CTA ever waits for another, so there is
// nothing to time out. Problems are grouped by size class; each class has its
// own persistent launch with a CTA size picked by m1_batch_tune, and the
// launches of all classes run concurrently from one captured CUDA graph.
// A class can instead run through single-grid contexts, one problem after
// another on a side stream while the graph runs: one SM per problem is slow
// for large grids (a 256^2 problem takes seconds on one SM and milliseconds on
// all of them). Classes above kGridPathCells cells start on that path, and
// m1_batch_tune times both paths per class.
//
// Scope: 2D radiation-only grids (n_u = 3) with periodic, outflow or reflecting
// boundaries, frozen (time-n) or fixed wave speeds.
#include <math.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/m1.h"
#include "m1_internal.h"

using namespace m1;

namespace {

constexpr int kM = kMaxRestart;  // GMRES(m) basis bound
constexpr int kNU = 3;
constexpr long long kGridPathCells = 128 * 128;  // larger classes start on the single-grid path

struct Prob {
    Dev<double> g64;
    Dev<float> g32;
    long long N, n, ld;
    double dt;
    double *U, *R, *Ut, *Rt, *b, *x, *r, *w64;  // FP64 vectors (n)
    float *U32;                                  // FP32 linearisation point (n)
    float *sigf32, *siga32, *B32, *Un32;         // FP32 copies of the inputs
    float *lp32[2], *lm32[2], *al32[2];          // FP32 face data
    int cls;                                     // size class
};

struct Work {
    float* V;       // (m+1) x ld
    float* w;       // ld
    float* z;       // ld
    float* binv;    // 9 N
    double* xin;    // n: inner solution accumulator
};

struct Opts {
    double newton_rtol, gmres_rtol;
    int newton_max, restart, gmres_max, refine_max, line_search;
};

// ---------------------------------------------------------------- block helpers
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];  // every thread, same order
    return t;
}

// compensated FP32 accumulation (TwoSum) of a thread's partial dot product
struct Comp {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float p) {
        const float s = hi + p;
        const float bb = s - hi;
        lo += (hi - (s - bb)) + (p - bb);
        hi = s;
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------- stencil pieces
__device__ void faces(const Prob& P) {
    for (int a = 0; a < 2; ++a) {
        const long long nf = P.N / P.g64.n[a] * (P.g64.n[a] + 1);
        for (long long f = threadIdx.x; f < nf; f += blockDim.x) {
            double lp, lm, al;
            if (P.g64.df)
                face_time_n<2, DF>(P.g64, a, f, lp, lm, al);
            else
                face_time_n<2, double>(P.g64, a, f, lp, lm, al);
            const_cast<double*>(P.g64.lam_p[a])[f] = lp;
            const_cast<double*>(P.g64.lam_m[a])[f] = lm;
            const_cast<double*>(P.g64.alpha[a])[f] = al;
            P.lp32[a][f] = (float)lp;
            P.lm32[a][f] = (float)lm;
            P.al32[a][f] = (float)al;
        }
    }
    for (long long i = threadIdx.x; i < P.N; i += blockDim.x) {
        P.sigf32[i] = (float)P.g64.sig_f[i];
        P.siga32[i] = (float)P.g64.sig_a[i];
        P.B32[i] = P.g64.B ? (float)P.g64.B[i] : 0.f;
    }
    for (long long i = threadIdx.x; i < P.n; i += blockDim.x) P.Un32[i] = (float)P.g64.Un[i];
    __syncthreads();
}

// R = R(U) (FP64 arrays; the arithmetic A is FP64 or double words); returns ||R||^2
template <class A>
__device__ double residual(const Prob& P, const double* U, double* R, double* red) {
    double ss = 0.0;
    LoadPlain<double, A> ld{U, P.N};
    for (long long i = threadIdx.x; i < P.N; i += blockDim.x) {
        int coord[3];
        cell_coord(i, P.g64.n[0], P.g64.n[1], coord);
        A out[kNU];
        cell_residual<A, 2, false>(P.g64, ld, i, coord, out);
#pragma unroll
        for (int k = 0; k < kNU; ++k) {
            const double o = dbl(out[k]);
            R[k * P.N + i] = o;
            ss += o * o;
        }
    }
    return block_sum(ss, red);
}

// R: the arrays, A: the arithmetic (R, or double words on FP64 arrays)
template <class R, class A = R>
__device__ void jv(const Dev<R>& g, long long N, const R* U, const R* v, R* out) {
    LoadDir<R, A> ld{U, v, N};
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        int coord[3];
        cell_coord(i, g.n[0], g.n[1], coord);
        Dual<A> o[kNU];
        cell_residual<Dual<A>, 2, false>(g, ld, i, coord, o);
#pragma unroll
        for (int k = 0; k < kNU; ++k) out[k * N + i] = to_mem<R>(o[k].d);
    }
    __syncthreads();
}

__device__ void bj_build(const Prob& P, float* binv) {
    for (long long i = threadIdx.x; i < P.N; i += blockDim.x) {
        int coord[3];
        cell_coord(i, P.g32.n[0], P.g32.n[1], coord);
        DF a[kNU][kNU], x[kNU][kNU];  // FP32 blocks, inverted in double words
        for (int k = 0; k < kNU; ++k) {
            LoadSeed<float> ld{P.U32, P.N, k};
            Dual<float> o[kNU];
            cell_residual<Dual<float>, 2, false>(P.g32, ld, i, coord, o);
#pragma unroll
            for (int r = 0; r < kNU; ++r) a[r][k] = DF(o[r].d);
        }
        invert_block<kNU, DF>(a, x);
#pragma unroll
        for (int r = 0; r < kNU; ++r)
#pragma unroll
            for (int c = 0; c < kNU; ++c) binv[(long long)(r * kNU + c) * P.N + i] = to_f32(x[r][c]);
    }
    __syncthreads();
}

__device__ void bj_apply(const Prob& P, const float* binv, const float* in, float* out) {
    for (long long i = threadIdx.x; i < P.N; i += blockDim.x) {
        float rr[kNU];
#pragma unroll
        for (int c = 0; c < kNU; ++c) rr[c] = in[c * P.N + i];
#pragma unroll
        for (int q = 0; q < kNU; ++q) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < kNU; ++c) acc += binv[(long long)(q * kNU + c) * P.N + i] * rr[c];
            out[q * P.N + i] = acc;
        }
    }
    __syncthreads();
}

// FP32 GMRES(m) with restarts on J32 c = rhs (rhs in W.V[0] on entry, unit norm);
// c accumulates (FP64) into W.xin. Returns the Arnoldi steps taken.
__device__ int inner_gmres(const Prob& P, const Work& W, double tol, int maxit, int m, double* red, double* sm) {
    double* H = sm;                       // (m+1) x m, column-major
    double* cs = H + (kM + 1) * kM;
    double* sn = cs + kM;
    double* g = sn + kM;                  // m+1
    double* y = g + kM + 1;               // m
    double* h = y + kM;                   // m+1
    const long long n = P.n, ld = P.ld;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) W.xin[e] = 0.0;
    int total = 0;
    bool first = true;
    for (;;) {
        double beta;
        if (first) {
            beta = 1.0;  // V_0 = rhs / 1
        } else {
            // restart: r = rhs - J xin, the right-hand side is kept in basis row kM
            for (long long e = threadIdx.x; e < n; e += blockDim.x) W.w[e] = (float)W.xin[e];
            __syncthreads();
            jv<float>(P.g32, P.N, P.U32, W.w, W.z);
            double ss = 0.0;
            for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                const float rv = W.V[(long long)kM * ld + e] - W.z[e];  // row kM keeps the right-hand side
                W.V[e] = rv;
                ss += (double)rv * rv;
            }
            beta = sqrt(block_sum(ss, red));
            const float inv = beta > 0.0 ? (float)(1.0 / beta) : 0.f;
            for (long long e = threadIdx.x; e < n; e += blockDim.x) W.V[e] *= inv;
            __syncthreads();
        }
        first = false;
        if (beta <= tol || total >= maxit) return total;
        if (threadIdx.x == 0) {
            for (int i = 0; i <= m; ++i) g[i] = 0.0;
            g[0] = beta;
        }
        __syncthreads();
        int k = 0;
        double est = beta;
        const int maxk = min(m, maxit - total);
        for (int j = 0; j < maxk; ++j) {
            const float* Vj = W.V + (long long)j * ld;
            bj_apply(P, W.binv, Vj, W.z);
            jv<float>(P.g32, P.N, P.U32, W.z, W.w);
            // classical Gram-Schmidt, second pass when ||w - Vh||^2 < ||w||^2 / 2
            double rest = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                double wn2 = 0.0;
                {
                    Comp c;
                    for (long long e = threadIdx.x; e < n; e += blockDim.x) c.add(W.w[e] * W.w[e]);
                    wn2 = block_sum(c.get(), red);
                }
                double hh = 0.0;
                for (int i = 0; i <= j; ++i) {
                    Comp c;
                    const float* Vi = W.V + (long long)i * ld;
                    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                        const float p = Vi[e] * W.w[e];
                        c.add(p);
                        c.lo += fmaf(Vi[e], W.w[e], -p);
                    }
                    const double hi = block_sum(c.get(), red);
                    if (threadIdx.x == 0) h[i] = (pass == 0 ? 0.0 : h[i]) + hi;
                    hh += hi * hi;
                    // subtract at once (modified order within the pass is not needed for CGS)
                    red[64 + i] = hi;  // keep this pass's coefficient
                }
                __syncthreads();
                for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                    float xw = W.w[e];
                    for (int i = 0; i <= j; ++i) xw = fmaf(-(float)red[64 + i], W.V[(long long)i * ld + e], xw);
                    W.w[e] = xw;
                }
                __syncthreads();
                rest = wn2 - hh;
                if (rest > 0.5 * wn2) break;
            }
            double nrm;
            {
                Comp c;
                for (long long e = threadIdx.x; e < n; e += blockDim.x) c.add(W.w[e] * W.w[e]);
                nrm = sqrt(block_sum(c.get(), red));
            }
            if (threadIdx.x == 0) {
                double* col = H + (long long)j * (kM + 1);
                for (int i = 0; i <= j; ++i) col[i] = h[i];
                col[j + 1] = nrm;
                for (int i = 0; i < j; ++i) {
                    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
                    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                    col[i] = t;
                }
                const double aa = col[j], bb = col[j + 1];
                const double den = hypot(aa, bb);
                cs[j] = den > 0.0 ? aa / den : 1.0;
                sn[j] = den > 0.0 ? bb / den : 0.0;
                col[j] = den;
                col[j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                red[63] = fabs(g[j + 1]);
            }
            const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
            float* Vn = W.V + (long long)(j + 1) * ld;
            for (long long e = threadIdx.x; e < n; e += blockDim.x) Vn[e] = W.w[e] * inv;
            __syncthreads();
            est = red[63];
            k = j + 1;
            ++total;
            if (est <= tol || nrm == 0.0) break;
        }
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double t = g[i];
                for (int q = i + 1; q < k; ++q) t -= H[(long long)q * (kM + 1) + i] * y[q];
                const double d = H[(long long)i * (kM + 1) + i];
                y[i] = d != 0.0 ? t / d : 0.0;
            }
        }
        __syncthreads();
        // xin += M^-1 (V y): combination into w (FP32), preconditioner into z
        for (long long e = threadIdx.x; e < n; e += blockDim.x) {
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += y[i] * (double)W.V[(long long)i * ld + e];
            W.w[e] = (float)acc;
        }
        __syncthreads();
        bj_apply(P, W.binv, W.w, W.z);
        for (long long e = threadIdx.x; e < n; e += blockDim.x) W.xin[e] += (double)W.z[e];
        __syncthreads();
        if (est <= tol) return total;
    }
}

// ---------------------------------------------------------------- the persistent kernel
__global__ void __launch_bounds__(512) k_batch_solve(const Prob* __restrict__ probs, const int* __restrict__ order, int count,
                              int* queue, const Work* __restrict__ works, m1_batch_problem_info* info, Opts o) {
    extern __shared__ double smem[];
    double* red = smem;                  // 32 warps + scratch (128 doubles)
    double* sm = smem + 128;             // Hessenberg, rotations, g, y, h
    __shared__ int pid;
    const Work W = works[blockIdx.x];
    for (;;) {
        if (threadIdx.x == 0) pid = atomicAdd(queue, 1);
        __syncthreads();
        const int q = pid;
        __syncthreads();
        if (q >= count) return;
        const int p = order[q];
        const Prob& P = probs[p];
        const long long n = P.n;
        faces(P);
        // Newton from U^n
        for (long long e = threadIdx.x; e < n; e += blockDim.x) P.U[e] = P.g64.Un[e];
        __syncthreads();
        const double r0 = sqrt(residual<double>(P, P.U, P.R, red));
        // double words for this problem's residuals and refinement J v when its grid
        // allows them and the Newton target is 32 times above their rounding floor,
        // measured as ||R_dw(U^n) - R(U^n)||
        bool df = false;
        if (P.g64.df) {
            const double rd = sqrt(residual<DF>(P, P.U, P.Rt, red));
            double ss = 0.0;
            for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                const double d = P.R[e] - P.Rt[e];
                ss += d * d;
            }
            const double floor = sqrt(block_sum(ss, red));
            df = rd == rd && rd <= 1e300 && o.newton_rtol * r0 >= 32.0 * floor;
        }
        double rn = r0;
        int nit = 0, git = 0;
        bool bad = !(r0 == r0);
        while (!bad && rn > o.newton_rtol * r0 && nit < o.newton_max) {
            for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                P.U32[e] = (float)P.U[e];
                P.b[e] = -P.R[e];
                P.x[e] = 0.0;
                P.r[e] = -P.R[e];
            }
            __syncthreads();
            bj_build(P, W.binv);
            // FP32 inner solves refined against the FP64 linear residual r = b - J x
            const double bn = rn;
            double rr = rn;
            for (int sweep = 0; sweep <= o.refine_max && rr > o.gmres_rtol * bn && git < o.gmres_max; ++sweep) {
                const float inv = (float)(1.0 / rr);
                for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                    const float v = (float)(P.r[e]) * inv;
                    W.V[e] = v;
                    W.V[(long long)kM * P.ld + e] = v;  // the right-hand side, kept for restarts
                }
                __syncthreads();
                const double inner_tol = fmax(0.5 * o.gmres_rtol * bn / rr, 1e-6);
                git += inner_gmres(P, W, inner_tol, o.gmres_max - git, o.restart, red, sm);
                for (long long e = threadIdx.x; e < n; e += blockDim.x) P.x[e] += rr * W.xin[e];
                __syncthreads();
                if (df)
                    jv<double, DF>(P.g64, P.N, P.U, P.x, P.w64);
                else
                    jv<double, double>(P.g64, P.N, P.U, P.x, P.w64);
                double ss = 0.0;
                for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                    const double v = P.b[e] - P.w64[e];
                    P.r[e] = v;
                    ss += v * v;
                }
                rr = sqrt(block_sum(ss, red));
            }
            // line search on the FP64 residual
            double theta = 1.0, rt = 0.0;
            for (int ls = 0; ls < 7; ++ls) {
                for (long long e = threadIdx.x; e < n; e += blockDim.x) P.Ut[e] = P.U[e] + theta * P.x[e];
                __syncthreads();
                rt = sqrt(df ? residual<DF>(P, P.Ut, P.Rt, red) : residual<double>(P, P.Ut, P.Rt, red));
                if (!o.line_search || rt <= (1.0 - 1e-4 * theta) * rn) break;
                theta *= 0.5;
            }
            for (long long e = threadIdx.x; e < n; e += blockDim.x) {
                P.U[e] = P.Ut[e];
                P.R[e] = P.Rt[e];
            }
            __syncthreads();
            rn = rt;
            ++nit;
            bad = !(rn == rn);
        }
        if (threadIdx.x == 0) {
            info[p].converged = (!bad && rn <= o.newton_rtol * r0) ? 1 : 0;
            info[p].newton_iters = nit;
            info[p].gmres_iters = git;
            info[p].res0 = r0;
            info[p].res = rn;
        }
        __syncthreads();
    }
}

size_t smem_bytes() { return sizeof(double) * (128 + (kM + 1) * kM + 2 * kM + (kM + 1) + kM + (kM + 1) + 8); }

}  // namespace

// ============================================================================ host side
struct m1_batch {
    cudaStream_t s = nullptr;       // the library's own stream (capturable), synchronised per call
    cudaStream_t user = nullptr;    // the caller's stream (ordered before each call)
    int nprob = 0;
    std::vector<m1_grid_desc> descs;
    std::vector<Prob> hp;               // host copies of the problem descriptors
    Prob* dprobs = nullptr;
    std::vector<void*> allocs;
    std::vector<int> cls;               // size class of each problem
    int ncls = 0;
    std::vector<std::vector<int>> members;
    int* dorder = nullptr;              // problems ordered by class
    std::vector<int> cls_offset;
    int* dqueue = nullptr;              // one counter per class
    std::vector<int> bs;                // CTA size per class (persistent path)
    std::vector<char> on_grid;          // per class: 1 = the single-grid path
    std::vector<m1_ctx*> gctx;          // per problem: its single-grid context (created on first use)
    std::vector<m1_batch_problem_info> ginfo;  // per problem: the single-grid path's result
    cudaStream_t gs = nullptr;          // stream of the single-grid contexts
    std::vector<int> grid;              // persistent CTAs per class
    std::vector<Work*> dworks;          // per class: grid Work slots
    m1_batch_problem_info* dinfo = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    cudaGraphExec_t exec = nullptr;
    Opts graph_opts{};
    bool have_graph = false;
    std::string err;
};

namespace {

m1_status bfail(m1_batch* b, m1_status st, const std::string& m) {
    if (b) b->err = m;
    return st;
}

template <class T>
m1_status balloc(m1_batch* b, T** p, size_t count) {
    if (cudaMalloc((void**)p, sizeof(T) * (count ? count : 1)) != cudaSuccess)
        return bfail(b, M1_ERR_NOMEM, "cudaMalloc failed");
    b->allocs.push_back(*p);
    return M1_OK;
}

#define BCK(expr)                       \
    do {                                \
        m1_status st_ = (expr);         \
        if (st_ != M1_OK) return st_;   \
    } while (0)

m1_status alloc_works(m1_batch* B, int c) {
    long long ldmax = 0, Nmax = 0;
    for (int p : B->members[c]) {
        ldmax = std::max(ldmax, B->hp[p].ld);
        Nmax = std::max(Nmax, B->hp[p].N);
    }
    std::vector<Work> w(B->grid[c]);
    for (auto& x : w) {
        BCK(balloc(B, &x.V, (size_t)(kM + 1) * ldmax));
        BCK(balloc(B, &x.w, ldmax));
        BCK(balloc(B, &x.z, ldmax));
        BCK(balloc(B, &x.binv, (size_t)kNU * kNU * Nmax));
        BCK(balloc(B, &x.xin, ldmax));
    }
    Work* dw;
    BCK(balloc(B, &dw, w.size()));
    if (cudaMemcpy(dw, w.data(), sizeof(Work) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(B, M1_ERR_CUDA, "copy of work slots failed");
    B->dworks[c] = dw;
    return M1_OK;
}

void launch_class(m1_batch* B, int c, const Opts& o, cudaStream_t s) {
    cudaMemsetAsync(B->dqueue + c, 0, sizeof(int), s);
    k_batch_solve<<<B->grid[c], B->bs[c], smem_bytes(), s>>>(B->dprobs, B->dorder + B->cls_offset[c],
                                                             (int)B->members[c].size(), B->dqueue + c,
                                                             B->dworks[c], B->dinfo, o);
}

}  // namespace

extern "C" {

m1_status m1_batch_create(int nprob, const m1_grid_desc* descs, void* stream, m1_batch** out) {
    if (!out || nprob < 1 || !descs) return M1_ERR_ARG;
    *out = nullptr;
    for (int k = 0; k < nprob; ++k) {
        const m1_grid_desc& d = descs[k];
        if (d.dim != 2 || d.gas_coupling || (d.implicit_eigs && !d.fixed_eigs) || d.n[2] != 1 || d.n[0] < 1 ||
            d.n[1] < 1)
            return M1_ERR_ARG;
        for (int a = 0; a < 2; ++a)
            for (int sd = 0; sd < 2; ++sd)
                if (d.bc[a][sd] == M1_BC_DIRICHLET || d.bc[a][sd] < 0 || d.bc[a][sd] > 3) return M1_ERR_ARG;
    }
    m1_batch* B = new (std::nothrow) m1_batch();
    if (!B) return M1_ERR_NOMEM;
    B->user = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking) != cudaSuccess) {
        delete B;
        return M1_ERR_CUDA;
    }
    cudaStreamSynchronize(B->user);
    B->nprob = nprob;
    B->descs.assign(descs, descs + nprob);
    B->hp.resize(nprob);
    auto cleanup = [&](m1_status st) {
        m1_batch_destroy(B);
        return st;
    };
    // size classes: distinct cell counts
    std::map<long long, int> cmap;
    for (int k = 0; k < nprob; ++k) cmap[(long long)descs[k].n[0] * descs[k].n[1]] = 0;
    int c = 0;
    for (auto& kv : cmap) kv.second = c++;
    B->ncls = c;
    B->members.resize(c);
    B->cls.resize(nprob);
    for (int k = 0; k < nprob; ++k) {
        B->cls[k] = cmap[(long long)descs[k].n[0] * descs[k].n[1]];
        B->members[B->cls[k]].push_back(k);
    }
    std::vector<int> order;
    for (int q = 0; q < c; ++q) {
        B->cls_offset.push_back((int)order.size());
        for (int p : B->members[q]) order.push_back(p);
    }
    for (int k = 0; k < nprob; ++k) {
        const m1_grid_desc& d = descs[k];
        Prob& P = B->hp[k];
        const long long N = (long long)d.n[0] * d.n[1];
        P.N = N;
        P.n = 3 * N;
        P.ld = (P.n + 63) / 64 * 64;
        P.cls = B->cls[k];
        Dev<double>& g = P.g64;
        g = Dev<double>{};
        g.dim = 2;
        g.nx = d.n[0];
        g.ny = d.n[1];
        g.nz = 1;
        g.N = N;
        for (int a = 0; a < 3; ++a) {
            g.n[a] = d.n[a];
            const double dx = (d.hi[a] - d.lo[a]) / d.n[a];
            g.dx[a] = dx;
            g.inv_dx[a] = 1.0 / dx;
            g.bM[a] = N / d.n[a];
            for (int sd = 0; sd < 2; ++sd) g.bc[a][sd] = d.bc[a][sd];
        }
        g.stride[0] = 1;
        g.stride[1] = d.n[0];
        g.stride[2] = N;
        g.c = d.c;
        g.a_r = d.a_r;
        g.lambda_floor = d.lambda_floor;
        g.gas = 0;
        g.wb = d.well_balanced;
        g.ap = d.ap_correction;
        g.fixed_eigs = d.fixed_eigs;
        g.wb_boundary = d.wb_boundary;
        g.implicit_eigs = 0;
        g.df = fp64_df_scalars_ok(d.c, d.a_r, false, 2, g.dx) ? 1 : 0;
        double *siga, *sigf, *Bf, *Un;
        if (balloc(B, &siga, N) || balloc(B, &sigf, N) || balloc(B, &Bf, N) || balloc(B, &Un, P.n) ||
            balloc(B, &P.U, P.n) || balloc(B, &P.R, P.n) || balloc(B, &P.Ut, P.n) || balloc(B, &P.Rt, P.n) ||
            balloc(B, &P.b, P.n) || balloc(B, &P.x, P.n) || balloc(B, &P.r, P.n) || balloc(B, &P.w64, P.n) ||
            balloc(B, &P.U32, P.n) || balloc(B, &P.sigf32, N) || balloc(B, &P.siga32, N) || balloc(B, &P.B32, N) ||
            balloc(B, &P.Un32, P.n))
            return cleanup(M1_ERR_NOMEM);
        cudaMemset(Bf, 0, sizeof(double) * N);
        g.sig_a = siga;
        g.sig_f = sigf;
        g.B = Bf;
        g.S = nullptr;
        g.rho_cv = nullptr;
        g.Un = Un;
        for (int a = 0; a < 2; ++a) {
            const long long nf = N / d.n[a] * (d.n[a] + 1);
            double *lp, *lm, *al;
            if (balloc(B, &lp, nf) || balloc(B, &lm, nf) || balloc(B, &al, nf) || balloc(B, &P.lp32[a], nf) ||
                balloc(B, &P.lm32[a], nf) || balloc(B, &P.al32[a], nf))
                return cleanup(M1_ERR_NOMEM);
            g.lam_p[a] = lp;
            g.lam_m[a] = lm;
            g.alpha[a] = al;
        }
        // the FP32 view of the same problem
        Dev<float>& f = P.g32;
        f = Dev<float>{};
        f.dim = 2;
        f.nx = g.nx;
        f.ny = g.ny;
        f.nz = 1;
        f.N = N;
        for (int a = 0; a < 3; ++a) {
            f.n[a] = g.n[a];
            f.dx[a] = (float)g.dx[a];
            f.inv_dx[a] = (float)g.inv_dx[a];
            f.bM[a] = g.bM[a];
            f.stride[a] = g.stride[a];
            for (int sd = 0; sd < 2; ++sd) f.bc[a][sd] = g.bc[a][sd];
        }
        f.c = (float)g.c;
        f.a_r = (float)g.a_r;
        f.lambda_floor = (float)g.lambda_floor;
        f.wb = g.wb;
        f.ap = g.ap;
        f.fixed_eigs = g.fixed_eigs;
        f.wb_boundary = g.wb_boundary;
        f.sig_a = P.siga32;
        f.sig_f = P.sigf32;
        f.B = P.B32;
        f.Un = P.Un32;
        for (int a = 0; a < 2; ++a) {
            f.lam_p[a] = P.lp32[a];
            f.lam_m[a] = P.lm32[a];
            f.alpha[a] = P.al32[a];
        }
    }
    if (balloc(B, &B->dprobs, nprob) || balloc(B, &B->dorder, nprob) || balloc(B, &B->dqueue, c) ||
        balloc(B, &B->dinfo, nprob))
        return cleanup(M1_ERR_NOMEM);
    cudaMemcpy(B->dorder, order.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice);
    // default CTA size per class: 256 up to 16k cells, 512 above; one or two CTAs per SM
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    B->bs.resize(c);
    B->grid.resize(c);
    B->dworks.assign(c, nullptr);
    for (int q = 0; q < c; ++q) {
        const long long N = B->hp[B->members[q][0]].N;
        B->bs[q] = N <= 16384 ? 256 : 512;
        B->on_grid.push_back(N > kGridPathCells ? 1 : 0);
        B->grid[q] = std::max(1, std::min((int)B->members[q].size(), nsm));
        if (alloc_works(B, q) != M1_OK) return cleanup(M1_ERR_NOMEM);
    }
    B->gctx.assign(nprob, nullptr);
    B->ginfo.assign(nprob, m1_batch_problem_info{});
    if (cudaStreamCreateWithFlags(&B->gs, cudaStreamNonBlocking) != cudaSuccess) return cleanup(M1_ERR_CUDA);
    B->side.resize(c);
    B->ev.resize(c + 1);
    for (int q = 0; q < c; ++q) cudaStreamCreateWithFlags(&B->side[q], cudaStreamNonBlocking);
    for (auto& e : B->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (cudaFuncSetAttribute(k_batch_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()) !=
        cudaSuccess)
        return cleanup(M1_ERR_CUDA);
    *out = B;
    return M1_OK;
}

m1_status m1_batch_destroy(m1_batch* B) {
    if (!B) return M1_OK;
    if (B->s) cudaStreamSynchronize(B->s);
    for (m1_ctx* x : B->gctx)
        if (x) m1_destroy(x);
    if (B->gs) cudaStreamDestroy(B->gs);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    for (auto s : B->side) cudaStreamDestroy(s);
    for (auto e : B->ev) cudaEventDestroy(e);
    for (void* p : B->allocs) cudaFree(p);
    if (B->s) cudaStreamDestroy(B->s);
    delete B;
    return M1_OK;
}

m1_status m1_batch_set_problem(m1_batch* B, int k, const double* sigma_a, const double* sigma_f, const double* E,
                               const double* F, const double* Bem, m1_mem mem) {
    if (!B || k < 0 || k >= B->nprob || !sigma_a || !E || !F) return M1_ERR_ARG;
    const Prob& P = B->hp[k];
    const cudaMemcpyKind kind = mem == M1_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t fb = sizeof(double) * P.N;
    if (cudaMemcpyAsync((void*)P.g64.sig_a, sigma_a, fb, kind, B->s) != cudaSuccess ||
        cudaMemcpyAsync((void*)P.g64.sig_f, sigma_f ? sigma_f : sigma_a, fb, kind, B->s) != cudaSuccess ||
        cudaMemcpyAsync((void*)P.g64.Un, E, fb, kind, B->s) != cudaSuccess ||
        cudaMemcpyAsync((void*)(P.g64.Un + P.N), F, 2 * fb, kind, B->s) != cudaSuccess)
        return bfail(B, M1_ERR_CUDA, "copy failed");
    if (Bem && cudaMemcpyAsync((void*)P.g64.B, Bem, fb, kind, B->s) != cudaSuccess)
        return bfail(B, M1_ERR_CUDA, "copy failed");
    return cudaStreamSynchronize(B->s) == cudaSuccess ? M1_OK : bfail(B, M1_ERR_CUDA, "sync failed");
}

static m1_status run(m1_batch* B, const Opts& o, bool use_graph) {
    bool any = false;
    for (int c = 0; c < B->ncls; ++c) any = any || !B->on_grid[c];
    if (!any) return M1_OK;
    if (!use_graph) {
        for (int c = 0; c < B->ncls; ++c)
            if (!B->on_grid[c]) launch_class(B, c, o, B->s);
        return cudaGetLastError() == cudaSuccess ? M1_OK : bfail(B, M1_ERR_CUDA, "launch failed");
    }
    const bool same = B->have_graph && memcmp(&B->graph_opts, &o, sizeof(Opts)) == 0;
    if (!same) {
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e0 = cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal);
        if (e0 != cudaSuccess) return bfail(B, M1_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e0));
        cudaEventRecord(B->ev[B->ncls], B->s);
        for (int c = 0; c < B->ncls; ++c) {
            if (B->on_grid[c]) continue;
            cudaStreamWaitEvent(B->side[c], B->ev[B->ncls], 0);
            launch_class(B, c, o, B->side[c]);
            cudaEventRecord(B->ev[c], B->side[c]);
            cudaStreamWaitEvent(B->s, B->ev[c], 0);
        }
        const cudaError_t e1 = cudaStreamEndCapture(B->s, &graph);  // always ends the capture
        if (e1 != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return bfail(B, M1_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e1));
        }
        const cudaError_t e = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(B, M1_ERR_CUDA, "graph instantiation failed");
        B->graph_opts = o;
        B->have_graph = true;
    }
    return cudaGraphLaunch(B->exec, B->s) == cudaSuccess ? M1_OK : bfail(B, M1_ERR_CUDA, "graph launch failed");
}

// problem k through its single-grid context on B->gs: the batch's time-n data
// (device) in, one implicit step (FP32 inner GMRES under FP64 refinement, the
// caller's multigrid or else point-block Jacobi), the solution into P.U
static m1_status grid_solve(m1_batch* B, int k, const m1_solver_opts* so) {
    Prob& P = B->hp[k];
    if (!B->gctx[k] && m1_init_grid(&B->descs[k], (void*)B->gs, &B->gctx[k]) != M1_OK)
        return bfail(B, M1_ERR_NOMEM, "single-grid context");
    m1_ctx* x = B->gctx[k];
    const Dev<double>& g = P.g64;
    m1_status st = m1_set_opacity(x, g.sig_a, g.sig_f, M1_MEM_DEVICE);
    if (st == M1_OK) st = m1_set_state(x, g.Un, g.Un + P.N, nullptr, nullptr, M1_MEM_DEVICE);
    if (st == M1_OK) st = m1_set_emission(x, g.B, M1_MEM_DEVICE);
    if (st != M1_OK) return bfail(B, st, m1_last_error(x));
    m1_solver_opts o;
    m1_default_opts(&o);
    if (so) o = *so;
    o.advance = 0;
    o.precision = M1_PREC_MIXED;
    if (o.precond != M1_PRECOND_MG) o.precond = M1_PRECOND_BJ;
    o.krylov = M1_KRYLOV_GMRES;
    m1_step_info info{};
    st = m1_implicit_step(x, P.dt, &o, &info);
    m1_batch_problem_info& bi = B->ginfo[k];
    bi.converged = info.converged;
    bi.newton_iters = info.newton_iters;
    bi.gmres_iters = info.gmres_iters;
    bi.res0 = info.res0;
    bi.res = info.res;
    if (st != M1_OK && st != M1_ERR_NOT_CONVERGED) return bfail(B, st, m1_last_error(x));
    if (st == M1_ERR_NOT_CONVERGED) return M1_OK;  // reported through info, as on the persistent path
    return m1_get_solution(x, P.U, M1_MEM_DEVICE) == M1_OK ? M1_OK : bfail(B, M1_ERR_CUDA, m1_last_error(x));
}

static m1_status grid_class(m1_batch* B, int c, const m1_solver_opts* so) {
    for (int k : B->members[c]) {
        const m1_status st = grid_solve(B, k, so);
        if (st != M1_OK) return st;
    }
    return M1_OK;
}

static Opts to_opts(const m1_solver_opts* so) {
    m1_solver_opts d;
    m1_default_opts(&d);
    if (so) d = *so;
    Opts o;
    o.newton_rtol = d.newton_rtol;
    o.gmres_rtol = d.gmres_rtol;
    o.newton_max = d.newton_max;
    o.restart = std::min(std::max(d.restart, 1), kM - 1);  // one basis row keeps the right-hand side
    o.gmres_max = d.gmres_max;
    o.refine_max = d.refine_max;
    o.line_search = d.line_search;
    return o;
}

m1_status m1_batch_implicit_step(m1_batch* B, const double* dts, const m1_solver_opts* so, m1_batch_problem_info* info,
                                 double* elapsed_ms) {
    if (!B || !dts) return M1_ERR_ARG;
    for (int k = 0; k < B->nprob; ++k) {
        if (!(dts[k] > 0.0)) return bfail(B, M1_ERR_ARG, "dt must be positive");
        B->hp[k].dt = dts[k];
        B->hp[k].g64.dt = dts[k];
        B->hp[k].g32.dt = (float)dts[k];
    }
    if (cudaStreamSynchronize(B->user) != cudaSuccess) return bfail(B, M1_ERR_CUDA, "caller stream failed");
    if (cudaMemcpyAsync(B->dprobs, B->hp.data(), sizeof(Prob) * B->nprob, cudaMemcpyHostToDevice, B->s) != cudaSuccess)
        return bfail(B, M1_ERR_CUDA, "copy failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, B->s);
    m1_status st = run(B, to_opts(so), true);
    // the single-grid classes on their own stream, concurrently with the graph
    cudaStreamWaitEvent(B->gs, e0, 0);
    for (int c = 0; c < B->ncls && st == M1_OK; ++c)
        if (B->on_grid[c]) st = grid_class(B, c, so);
    cudaEvent_t eg;
    cudaEventCreateWithFlags(&eg, cudaEventDisableTiming);
    cudaEventRecord(eg, B->gs);
    cudaStreamWaitEvent(B->s, eg, 0);
    cudaEventRecord(e1, B->s);
    if (cudaStreamSynchronize(B->s) != cudaSuccess) st = bfail(B, M1_ERR_CUDA, "batched solve failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(eg);
    if (elapsed_ms) *elapsed_ms = ms;
    if (st != M1_OK) return st;
    if (info) {
        if (cudaMemcpy(info, B->dinfo, sizeof(m1_batch_problem_info) * B->nprob, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return bfail(B, M1_ERR_CUDA, "copy failed");
        for (int k = 0; k < B->nprob; ++k)
            if (B->on_grid[B->cls[k]]) info[k] = B->ginfo[k];
    }
    return M1_OK;
}

m1_status m1_batch_get_solution(const m1_batch* B, int k, double* U, m1_mem mem) {
    if (!B || k < 0 || k >= B->nprob || !U) return M1_ERR_ARG;
    const Prob& P = B->hp[k];
    return cudaMemcpy(U, P.U, sizeof(double) * P.n, mem == M1_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                          : cudaMemcpyDeviceToHost) == cudaSuccess
               ? M1_OK
               : M1_ERR_CUDA;
}

m1_status m1_batch_tune(m1_batch* B, const double* dts, const m1_solver_opts* so, int* chosen) {
    if (!B || !dts) return M1_ERR_ARG;
    const int cand[3] = {128, 256, 512};
    for (int k = 0; k < B->nprob; ++k) {
        B->hp[k].dt = dts[k];
        B->hp[k].g64.dt = dts[k];
        B->hp[k].g32.dt = (float)dts[k];
    }
    if (cudaMemcpy(B->dprobs, B->hp.data(), sizeof(Prob) * B->nprob, cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(B, M1_ERR_CUDA, "copy failed");
    const Opts o = to_opts(so);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c = 0; c < B->ncls; ++c) {
        float best = 1e30f;
        int bbest = B->bs[c];
        bool grid_best = false;
        {  // the single-grid path
            cudaEventRecord(e0, B->gs);
            const m1_status st = grid_class(B, c, so);
            cudaEventRecord(e1, B->gs);
            if (st != M1_OK || cudaStreamSynchronize(B->gs) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st != M1_OK ? st : bfail(B, M1_ERR_CUDA, "tuning run failed");
            }
            cudaEventElapsedTime(&best, e0, e1);
            grid_best = true;
        }
        for (int bs : cand) {
            B->bs[c] = bs;
            cudaEventRecord(e0, B->s);
            launch_class(B, c, o, B->s);
            cudaEventRecord(e1, B->s);
            if (cudaStreamSynchronize(B->s) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return bfail(B, M1_ERR_CUDA, "tuning launch failed");
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bbest = bs;
                grid_best = false;
            } else if (ms > 3.f * best) {
                break;  // far behind the best: the other CTA sizes will not close the gap
            }
        }
        B->bs[c] = bbest;
        B->on_grid[c] = grid_best ? 1 : 0;
        if (chosen) chosen[c] = grid_best ? 0 : bbest;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->have_graph = false;  // re-capture with the chosen sizes
    return M1_OK;
}

m1_status m1_batch_set_class(m1_batch* B, int c, int threads) {
    if (!B || c < 0 || c >= B->ncls) return M1_ERR_ARG;
    if (threads != 0 && threads != 128 && threads != 256 && threads != 512)
        return bfail(B, M1_ERR_ARG, "threads must be 0, 128, 256 or 512");
    B->on_grid[c] = threads == 0 ? 1 : 0;
    if (threads) B->bs[c] = threads;
    B->have_graph = false;
    return M1_OK;
}

int m1_batch_num_classes(const m1_batch* B) { return B ? B->ncls : 0; }

const char* m1_batch_last_error(const m1_batch* B) { return B ? B->err.c_str() : "null batch"; }

}  // extern "C"
