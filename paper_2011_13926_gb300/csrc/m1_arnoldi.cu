// m1_arnoldi.cu — fused Arnoldi step of restarted GMRES (classical
// Gram-Schmidt with selective reorthogonalisation).
//
// One Arnoldi step j on the new vector w = A M^-1 V_j is three launches of one
// kernel, each a single pass over V_0..V_j and w:
//   dots: per-block partial sums of h1 = V^T w and ||w||^2;
//   dots of the residual: every block first sums the partial rows of the
//     first pass (fixed order, so all blocks agree bit for bit) and applies
//     the Daniel-Gragg-Kaufman-Stewart test ||w - V h1||^2 = ||w||^2 -
//     ||h1||^2 > ||w||^2 / 2; when it holds the blocks return at once,
//     otherwise w' = w - V h1 is formed on the fly, element by element, and
//     the partial sums of h2 = V^T w' and ||w'||^2 are written, so the
//     classical second Gram-Schmidt pass costs one read of the basis, not two;
//   update: every block sums the partial rows (both passes when the second
//     ran), forms beta and writes V_{j+1} = (w - V h1 [- V h2]) / beta with the
//     same rounding of w' as the second pass; block 0 applies the Givens
//     rotations to Hessenberg column h1 (+ h2), beta and updates the residual
//     estimate |g_{j+1}|.
// Every pass is one grid-stride sweep in which a thread loads the 16-byte slot
// q of all rows at once into registers (the rows are a compile-time count, so
// the loads are issued back to back and the accumulation chains interleave).
// For FP32 vectors the sums stay in double-float FP32 arithmetic through the
// warp, block and cross-block reductions and reach FP64 once per column:
// GB300 runs FP64 at a small fraction of its FP32 rate, and FP64 reductions
// in every lane cost a fifth of a dots pass. FP64 vectors accumulate in FP64.
// All sums are in a fixed order, so results are reproducible run to run. The
// Hessenberg least-squares problem stays in FP64 on the device.
#include "m1_internal.h"

#include <algorithm>

namespace m1 {

static constexpr int kOrThreads = 128;            // threads per block (one 16-byte slot each per row)
static constexpr int kCols = kMaxRestart + 1;     // partial row: h_0..h_{kCols-1}, then ||w||^2
static constexpr int kHLd = kMaxRestart + 1;
static_assert(kCols + 1 == 32, "the partial-row reduction reads rows of 32 eight-byte columns");
static_assert(kOrThreads == 128, "the partial-row reduction maps 128 threads onto 8 x 16 column pairs");

enum GsMode : int { kDots = 0, kDotsResidual = 1, kUpdate = 2 };

struct TwoF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum_acc(TwoF& acc, float p, float perr) {
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += err + perr;
}

// (a.hi, a.lo) + (b.hi, b.lo): TwoSum of the high parts, low parts added
__device__ __forceinline__ TwoF df_add(TwoF a, TwoF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    return TwoF{s, a.lo + b.lo + err};
}

template <class T> struct Acc;
template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ void add_prod4(const double2& a, const double2& b) {
        v = fma(a.x, b.x, v);
        v = fma(a.y, b.y, v);
    }
    __device__ __forceinline__ double get() const { return v; }
    // sum over the warp (valid in every lane)
    __device__ __forceinline__ double warp_total() const {
        double t = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        return t;
    }
};
template <> struct Acc<float> {
    TwoF t;
    __device__ __forceinline__ void zero() { t.hi = 0.f; t.lo = 0.f; }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        two_sum_acc(t, p, e);
    }
    // four products by an FMA chain (FP32 rounding), then one compensated add
    __device__ __forceinline__ void add_prod4(const float4& a, const float4& b) {
        float p = a.x * b.x;
        p = fmaf(a.y, b.y, p);
        p = fmaf(a.z, b.z, p);
        p = fmaf(a.w, b.w, p);
        two_sum_acc(t, p, 0.f);
    }
    __device__ __forceinline__ double get() const { return (double)t.hi + (double)t.lo; }
    // sum over the warp by double-float additions in FP32 (valid in every lane)
    __device__ __forceinline__ TwoF warp_total() const {
        TwoF a = t;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, a.hi, o);
            const float bl = __shfl_xor_sync(0xffffffffu, a.lo, o);
            a = df_add(a, TwoF{bh, bl});
        }
        return a;
    }
};

// Per-column partial sums: double-float pairs for FP32 vectors (so that no
// lane does FP64 work before the final reduction converts each column once: FP64
// is a narrow pipe on this GPU), FP64 for FP64 vectors. Both are 8 bytes, a
// partial row of 32 columns is 256 bytes, and two columns load as 16 bytes.
template <class T> struct Part;
template <> struct Part<float> {
    using type = TwoF;
    using pair = float4;
    static __device__ __forceinline__ TwoF zero() { return TwoF{0.f, 0.f}; }
    static __device__ __forceinline__ TwoF add(TwoF a, TwoF b) { return df_add(a, b); }
    static __device__ __forceinline__ double to_double(TwoF a) { return (double)a.hi + (double)a.lo; }
    static __device__ __forceinline__ void split(const float4& v, TwoF& c0, TwoF& c1) {
        c0 = TwoF{v.x, v.y};
        c1 = TwoF{v.z, v.w};
    }
};
template <> struct Part<double> {
    using type = double;
    using pair = double2;
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double to_double(double a) { return a; }
    static __device__ __forceinline__ void split(const double2& v, double& c0, double& c1) {
        c0 = v.x;
        c1 = v.y;
    }
};


// Hessenberg column j from h (j+1 entries, shared memory) and beta = ||w - V h||:
// apply the previous rotations (cs, sn staged in shared memory), form rotation
// j, rotate g; one thread, no dependent global loads.
__device__ void givens_column(const ArnoldiDev& K, double* col, const double* scs, const double* ssn, double beta,
                              int j) {
    col[j + 1] = beta;
    for (int i = 0; i < j; ++i) {
        const double t = scs[i] * col[i] + ssn[i] * col[i + 1];
        col[i + 1] = -ssn[i] * col[i] + scs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    const double den = hypot(a, b);
    const double c = den > 0.0 ? a / den : 1.0;
    const double s = den > 0.0 ? b / den : 0.0;
    col[j] = den;
    col[j + 1] = 0.0;
    double* H = K.H + (long long)j * kHLd;
    for (int i = 0; i <= j + 1; ++i) H[i] = col[i];
    K.cs[j] = c;
    K.sn[j] = s;
    const double gj = K.g[j];
    K.g[j + 1] = -s * gj;
    K.g[j] = c * gj;
    K.resid[0] = fabs(s * gj);
    K.resid[1] = beta;
    K.nrm2[1] = beta * beta;
    K.nrm2[2] = beta > 0.0 ? 1.0 / beta : 0.0;  // the update pass scales by it
}

// 16-byte vectors of the basis element type (rows of V start on 256-byte
// boundaries: the basis stride is a multiple of 64 elements)
template <class T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
};

// w -= a v, component-wise FMA
__device__ __forceinline__ void fnma(float4& x, float a, const float4& v) {
    x.x = fmaf(-a, v.x, x.x);
    x.y = fmaf(-a, v.y, x.y);
    x.z = fmaf(-a, v.z, x.z);
    x.w = fmaf(-a, v.w, x.w);
}
__device__ __forceinline__ void fnma(double2& x, double a, const double2& v) {
    x.x = fma(-a, v.x, x.x);
    x.y = fma(-a, v.y, x.y);
}
__device__ __forceinline__ void scale(float4& x, float a) {
    x.x *= a;
    x.y *= a;
    x.z *= a;
    x.w *= a;
}
__device__ __forceinline__ void scale(double2& x, double a) {
    x.x *= a;
    x.y *= a;
}

// Fixed-order sum of the partial rows part[0 .. nb) (kCols + 1 eight-byte
// columns each) into tot[] (FP64), by all kOrThreads threads of the block:
// thread t adds the column pair (2 (t % 16), 2 (t % 16) + 1) of rows t / 16,
// t / 16 + 8, ... with 16-byte loads; only the pairs holding columns 0..j and
// the ||.||^2 column are read. Every block that calls it on the same rows gets
// the same values bit for bit.
template <class T>
__device__ void reduce_rows(const double* part_raw, int nb, int j, typename Part<T>::type (*tot8)[kCols + 1],
                            double* tot) {
    using P = Part<T>;
    using PT = typename P::type;
    const int tid = threadIdx.x;
    const int c2 = tid & 15, r0 = tid >> 4;
    const bool need = 2 * c2 <= j || c2 == 15;
    PT s0 = P::zero(), s1 = P::zero();
    if (need) {
        const PT* base = reinterpret_cast<const PT*>(part_raw);
#pragma unroll 8
        for (int b = r0; b < nb; b += 8) {
            const typename P::pair v =
                __ldcg(reinterpret_cast<const typename P::pair*>(base + (long long)b * (kCols + 1)) + c2);
            PT x0, x1;
            P::split(v, x0, x1);
            s0 = P::add(s0, x0);
            s1 = P::add(s1, x1);
        }
    }
    tot8[r0][2 * c2] = s0;
    tot8[r0][2 * c2 + 1] = s1;
    __syncthreads();
    if (tid <= kCols) {
        PT v = tot8[0][tid];
#pragma unroll
        for (int r = 1; r < 8; ++r) v = P::add(v, tot8[r][tid]);
        tot[tid] = P::to_double(v);
    }
    __syncthreads();
}

// Gram-Schmidt pass of Arnoldi step j (mode: kDots, kDotsResidual, kUpdate).
// The dots passes only write one partial row per block; the next pass reduces
// them itself, in every block (a short parallel prologue instead of one
// block's serial tail): the residual-dots pass decides the
// Daniel-Gragg-Kaufman-Stewart test from the first dots, the update from both,
// and block 0 of the update rotates the Hessenberg column.
// NC >= j + 1 (a multiple of 4, at most 32) is the compile-time number of rows
// a thread loads per 16-byte slot: all of them are issued before any is used,
// so each thread keeps NC loads in flight. Rows above j re-read row j (an L1/L2
// hit), their h is zero and their accumulators are never read, so the loops
// carry no branch and the NC accumulation chains interleave.
template <class T, int NC>
__global__ void __launch_bounds__(kOrThreads) k_gram_schmidt(ArnoldiDev K, T* __restrict__ V,
                                                             const T* __restrict__ w, int j, int mode) {
    using VT = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    using P = Part<T>;
    using PT = typename P::type;
    __shared__ T h1s[kCols + 1], h2s[kCols + 1];
    __shared__ PT red[kOrThreads / 32][kCols + 1];
    __shared__ PT tot8[8][kCols + 1];
    __shared__ double tot1[kCols + 1], tot2[kCols + 1];
    __shared__ double col[kCols + 1], scs[kCols], ssn[kCols];
    const int tid = threadIdx.x;
    const int nb = K.grid_dots[j];
    bool reorth = false;
    double beta2 = 0.0;
    if (mode != kDots) {
        // h1 = V^T w and ||w||^2 from the first dots pass; the second pass when
        // ||w - V h1||^2 = ||w||^2 - ||h1||^2 is not above ||w||^2 / 2
        reduce_rows<T>(K.partials, nb, j, tot8, tot1);
        double hh = 0.0;
        for (int i = 0; i <= j; ++i) hh += tot1[i] * tot1[i];
        const double wn2 = tot1[kCols];
        beta2 = wn2 - hh;
        reorth = !(beta2 > 0.5 * wn2);
        if (mode == kDotsResidual && !reorth) return;  // uniform over the grid
        if (mode == kUpdate && reorth) {
            reduce_rows<T>(K.partials2, nb, j, tot8, tot2);
            double hh2 = 0.0;
            for (int i = 0; i <= j; ++i) hh2 += tot2[i] * tot2[i];
            beta2 = tot2[kCols] - hh2;
        }
        if (tid <= kCols) {
            h1s[tid] = tid <= j ? (T)tot1[tid] : T(0);
            h2s[tid] = (tid <= j && reorth) ? (T)tot2[tid] : T(0);
        }
        __syncthreads();
    }
    const bool dots = mode != kUpdate;
    const double beta = sqrt(fmax(beta2, 0.0));
    const T inv = dots ? T(1) : (beta > 0.0 ? (T)(1.0 / beta) : T(0));
    if (mode == kUpdate && blockIdx.x == 0) {
        // the Hessenberg column h1 (+ h2), beta: rotations, g, the estimate
        if (tid <= j) {
            K.h1[tid] = tot1[tid];
            if (reorth) K.h2[tid] = tot2[tid];
            col[tid] = reorth ? tot1[tid] + tot2[tid] : tot1[tid];
        }
        if (tid < j) {
            scs[tid] = K.cs[tid];
            ssn[tid] = K.sn[tid];
        }
        __syncthreads();
        if (tid == 0) {
            *K.reorth = reorth ? 1 : 0;
            K.resid[2] = reorth ? 1.0 : 0.0;
            givens_column(K, col, scs, ssn, beta, j);
            if (K.resid_host) {
                K.resid_host[0] = K.resid[0];
                K.resid_host[1] = K.resid[1];
                K.resid_host[2] = K.resid[2];
            }
        }
    }
    Acc<T> acc[NC];
    Acc<T> ww;
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i].zero();
    ww.zero();
    const long long n = K.n, ld = K.ld;
    const long long nv = n / W;
    const VT* rows[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) rows[i] = reinterpret_cast<const VT*>(V + (long long)min(i, j) * ld);
    VT* out = reinterpret_cast<VT*>(V + (long long)(j + 1) * ld);
    // U slots per thread per trip (U x NC loads in flight), then single slots
    constexpr int U = NC <= 4 ? 8 : NC <= 8 ? 4 : NC <= 16 ? 2 : 1;
    const long long S = (long long)gridDim.x * kOrThreads;
    auto slot = [&](const VT* v, VT x, long long q) {
        if (mode != kDots) {
#pragma unroll
            for (int i = 0; i < NC; ++i) fnma(x, h1s[i], v[i]);
        }
        if (dots) {
            ww.add_prod4(x, x);
#pragma unroll
            for (int i = 0; i < NC; ++i) acc[i].add_prod4(v[i], x);
        } else {
            if (reorth) {
#pragma unroll
                for (int i = 0; i < NC; ++i) fnma(x, h2s[i], v[i]);
            }
            scale(x, inv);
            out[q] = x;
        }
    };
    long long q = (long long)blockIdx.x * kOrThreads + tid;
    for (; q + (U - 1) * S < nv; q += U * S) {
        VT v[U][NC], x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int i = 0; i < NC; ++i) v[u][i] = __ldg(rows[i] + q + u * S);
            x[u] = __ldg(reinterpret_cast<const VT*>(w) + q + u * S);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) slot(v[u], x[u], q + u * S);
    }
    for (; q < nv; q += S) {
        VT v[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) v[i] = __ldg(rows[i] + q);
        slot(v, __ldg(reinterpret_cast<const VT*>(w) + q), q);
    }
    if (blockIdx.x == 0) {  // the n % W scalar tail
        for (long long e = nv * W + tid; e < n; e += kOrThreads) {
            T x = w[e];
            if (mode != kDots)
                for (int i = 0; i <= j; ++i) x = fma(-h1s[i], V[i * ld + e], x);
            if (dots) {
                ww.add_prod(x, x);
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    if (i <= j) acc[i].add_prod(V[i * ld + e], x);
            } else {
                if (reorth)
                    for (int i = 0; i <= j; ++i) x = fma(-h2s[i], V[i * ld + e], x);
                V[(long long)(j + 1) * ld + e] = x * inv;
            }
        }
    }
    if (!dots) return;
    // this block's partial row: h_0..h_j and ||x||^2
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        if (i <= j) {
            const PT v = acc[i].warp_total();
            if (lane == 0) red[wid][i] = v;
        }
    }
    {
        const PT v = ww.warp_total();
        if (lane == 0) red[wid][kCols] = v;
    }
    __syncthreads();
    PT* part = reinterpret_cast<PT*>(mode == kDots ? K.partials : K.partials2) + (long long)blockIdx.x * (kCols + 1);
    if (tid <= j || tid == kCols) {
        PT v = red[0][tid];
#pragma unroll
        for (int qq = 1; qq < kOrThreads / 32; ++qq) v = P::add(v, red[qq][tid]);
        part[tid] = v;
    }
}

template <class T, int NC>
static int gs_grid_one(int j, long long n, int sms, bool dots) {
    (void)j;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_schmidt<T, NC>, kOrThreads, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const long long nv = n / Vec<T>::W;
    const long long tiles = std::max(1LL, (nv + kOrThreads - 1) / kOrThreads);
    // every block of the next pass reads the dots passes' partial rows: at most
    // three blocks per SM keep that prologue short
    if (dots) occ = std::min(occ, 3);
    return (int)std::min<long long>({(long long)occ * sms, tiles, (long long)kMaxGsBlocks});
}

// the accumulator size of step j: j + 1 rounded up to a multiple of 4
template <class T, int NC = 4>
static int gs_grid_for(int j, long long n, int sms, bool dots) {
    if constexpr (NC < 32) {
        if (j + 1 > NC) return gs_grid_for<T, NC + 4>(j, n, sms, dots);
    }
    return gs_grid_one<T, NC>(j, n, sms, dots);
}

template <class T>
static void gs_grid_table(long long n, int* grid, int* grid_dots) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int j = 0; j < kMaxRestart; ++j) {
        grid[j] = gs_grid_for<T>(j, n, sms, false);
        grid_dots[j] = gs_grid_for<T>(j, n, sms, true);
    }
}

void arnoldi_grid_table(long long n, bool fp32, int* grid, int* grid_dots) {
    if (fp32)
        gs_grid_table<float>(n, grid, grid_dots);
    else
        gs_grid_table<double>(n, grid, grid_dots);
}

template <class T, int NC>
static void gs_launch(const ArnoldiDev& K, T* V, const T* w, int j, cudaStream_t s) {
    const dim3 gdots(K.grid_dots[j]), gupd(K.grid[j]);
    k_gram_schmidt<T, NC><<<gdots, kOrThreads, 0, s>>>(K, V, w, j, kDots);
    k_gram_schmidt<T, NC><<<gdots, kOrThreads, 0, s>>>(K, V, w, j, kDotsResidual);
    k_gram_schmidt<T, NC><<<gupd, kOrThreads, 0, s>>>(K, V, w, j, kUpdate);
}

template <class T, int NC = 4>
static void arnoldi_step(const ArnoldiDev& K, T* V, const T* w, int j, cudaStream_t s) {
    if constexpr (NC < 32) {
        if (j + 1 > NC) return arnoldi_step<T, NC + 4>(K, V, w, j, s);
    }
    gs_launch<T, NC>(K, V, w, j, s);
}

void launch_arnoldi_step_f64(const ArnoldiDev& K, double* V, double* w, int j, cudaStream_t s) {
    arnoldi_step<double>(K, V, w, j, s);
}

void launch_arnoldi_step_f32(const ArnoldiDev& K, float* V, float* w, int j, cudaStream_t s) {
    arnoldi_step<float>(K, V, w, j, s);
}

}  // namespace m1
