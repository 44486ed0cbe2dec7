// m1_arnoldi.cu — fused Arnoldi step of restarted GMRES (classical
// Gram-Schmidt with selective reorthogonalisation).
//
// One Arnoldi step j on the new vector w = A M^-1 V_j is four kernels:
//   dots(pass 1): h = V_{0..j}^T w and ||w||^2 in one pass over w; the last
//     block to finish sums the per-block partials in a fixed order, tests
//     ||w - V h||^2 = ||w||^2 - ||h||^2 against ||w||^2 / 2 (the Daniel-Gragg-
//     Kaufman-Stewart criterion), and when no second pass is needed applies
//     the Givens rotations to Hessenberg column j and updates the residual
//     estimate |g_{j+1}|;
//   update(pass 1): w - V h, written straight into V_{j+1} (normalised) when no
//     second pass is needed, else back into w;
//   dots/update(pass 2): the classical second Gram-Schmidt pass, only when the
//     criterion asked for it (otherwise the blocks return at once).
// FP32 vectors accumulate their dot products in double-float arithmetic
// (error-free TwoProd with FMA and TwoSum), FP64 vectors in FP64; the
// cross-block sums are FP64 in a fixed order, so results are reproducible.
// The Hessenberg least-squares problem stays in FP64 on the device.
#include "m1_internal.h"

namespace m1 {

static constexpr int kArThreads = 256;
static constexpr int kCols = kMaxRestart + 1;
static constexpr int kHLd = kMaxRestart + 1;

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

template <class T> struct Acc;
template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double get() const { return v; }
};
template <> struct Acc<float> {
    TwoF t;
    __device__ __forceinline__ void zero() { t.hi = 0.f; t.lo = 0.f; }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        two_sum_acc(t, p, e);
    }
    __device__ __forceinline__ double get() const { return (double)t.hi + (double)t.lo; }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Hessenberg column j from h (j+1 entries) and beta = ||w - V h||; rotations.
__device__ void givens_column(const ArnoldiDev& K, const double* h, double beta, int j) {
    double* col = K.H + (long long)j * kHLd;
    for (int i = 0; i <= j; ++i) col[i] = h[i];
    col[j + 1] = beta;
    for (int i = 0; i < j; ++i) {
        const double t = K.cs[i] * col[i] + K.sn[i] * col[i + 1];
        col[i + 1] = -K.sn[i] * col[i] + K.cs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    const double den = hypot(a, b);
    const double c = den > 0.0 ? a / den : 1.0;
    const double s = den > 0.0 ? b / den : 0.0;
    K.cs[j] = c;
    K.sn[j] = s;
    col[j] = den;
    col[j + 1] = 0.0;
    K.g[j + 1] = -s * K.g[j];
    K.g[j] = c * K.g[j];
    K.resid[0] = fabs(K.g[j + 1]);
    K.resid[1] = beta;
    K.nrm2[1] = beta * beta;
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
__device__ __forceinline__ float comp(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ double comp(const double2& v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ void setc(float4& v, int k, float x) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void setc(double2& v, int k, double x) {
    if (k == 0) v.x = x; else v.y = x;
}

// JMAX accumulators per thread (the smallest bucket >= j + 1 is launched, so
// early Arnoldi steps keep their registers low and their occupancy high)
template <class T, int JMAX>
__global__ void __launch_bounds__(kArThreads) k_arnoldi_dots(ArnoldiDev K, const T* __restrict__ V,
                                                             const T* __restrict__ w, int j, int pass) {
    if (pass == 2 && *K.reorth == 0) return;
    using VT = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    __shared__ double red[kArThreads / 32][kCols + 1];
    __shared__ bool last;
    Acc<T> acc[JMAX];
    Acc<T> ww;
#pragma unroll
    for (int i = 0; i < JMAX; ++i) acc[i].zero();
    ww.zero();
    const long long n = K.n, ld = K.ld;
    const long long nv = n / W;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; q + stride < nv; q += 2 * stride) {  // two vectors in flight per row
        const VT wa = reinterpret_cast<const VT*>(w)[q];
        const VT wb = reinterpret_cast<const VT*>(w)[q + stride];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            ww.add_prod(comp(wa, k), comp(wa, k));
            ww.add_prod(comp(wb, k), comp(wb, k));
        }
#pragma unroll
        for (int i = 0; i < JMAX; ++i)
            if (i <= j) {
                const VT va = reinterpret_cast<const VT*>(V + i * ld)[q];
                const VT vb = reinterpret_cast<const VT*>(V + i * ld)[q + stride];
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    acc[i].add_prod(comp(va, k), comp(wa, k));
                    acc[i].add_prod(comp(vb, k), comp(wb, k));
                }
            }
    }
    for (; q < nv; q += stride) {
        const VT wv = reinterpret_cast<const VT*>(w)[q];
#pragma unroll
        for (int k = 0; k < W; ++k) ww.add_prod(comp(wv, k), comp(wv, k));
#pragma unroll
        for (int i = 0; i < JMAX; ++i)
            if (i <= j) {
                const VT vv = reinterpret_cast<const VT*>(V + i * ld)[q];
#pragma unroll
                for (int k = 0; k < W; ++k) acc[i].add_prod(comp(vv, k), comp(wv, k));
            }
    }
    if (blockIdx.x == 0) {  // scalar tail
        for (long long e = nv * W + threadIdx.x; e < n; e += blockDim.x) {
            const T we = w[e];
            ww.add_prod(we, we);
#pragma unroll
            for (int i = 0; i < JMAX; ++i)
                if (i <= j) acc[i].add_prod(V[i * ld + e], we);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < JMAX; ++i) {
        if (i <= j) {
            const double t = warp_sum_d(acc[i].get());
            if (lane == 0) red[wid][i] = t;
        }
    }
    {
        const double t = warp_sum_d(ww.get());
        if (lane == 0) red[wid][kCols] = t;
    }
    __syncthreads();
    double* part = K.partials + (long long)blockIdx.x * (kCols + 1);
    for (int i = threadIdx.x; i <= kCols; i += blockDim.x) {
        if (i <= j || i == kCols) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q][i];
            part[i] = t;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(K.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    // the last block: fixed-order sums of the partials
    __shared__ double tot[kCols + 1];
    for (int i = wid; i <= kCols; i += (int)(blockDim.x >> 5)) {
        if (i <= j || i == kCols) {
            double t = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(K.partials + (long long)b * (kCols + 1) + i);
            t = warp_sum_d(t);
            if (lane == 0) tot[i] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *K.counter = 0u;
        double* h = pass == 1 ? K.h1 : K.h2;
        double hh = 0.0;
        for (int i = 0; i <= j; ++i) {
            h[i] = tot[i];
            hh += tot[i] * tot[i];
        }
        const double wn2 = tot[kCols];
        const double rest = wn2 - hh;
        if (pass == 1 && !(rest > 0.5 * wn2)) {
            *K.reorth = 1;  // second pass decides the column
            K.resid[2] = 1.0;
        } else {
            if (pass == 1) K.resid[2] = 0.0;
            if (pass == 1) *K.reorth = 0;
            double hsum[kCols];
            for (int i = 0; i <= j; ++i) hsum[i] = K.h1[i] + (pass == 2 ? K.h2[i] : 0.0);
            givens_column(K, hsum, sqrt(fmax(rest, 0.0)), j);
        }
    }
}

template <class T, int JMAX>
__global__ void __launch_bounds__(kArThreads) k_arnoldi_update(ArnoldiDev K, T* __restrict__ V, T* __restrict__ w,
                                                               int j, int pass) {
    const int reorth = *K.reorth;
    if (pass == 2 && reorth == 0) return;
    using VT = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    __shared__ T hs[kCols];
    const double* h = pass == 1 ? K.h1 : K.h2;
    if (threadIdx.x < kCols) hs[threadIdx.x] = threadIdx.x <= j ? (T)h[threadIdx.x] : T(0);
    __syncthreads();
    const bool final_pass = (pass == 2) || (reorth == 0);
    const double b2 = K.nrm2[1];
    const T inv = final_pass ? (b2 > 0.0 ? (T)(1.0 / sqrt(b2)) : T(0)) : T(1);
    T* out = final_pass ? V + (long long)(j + 1) * K.ld : w;
    const long long n = K.n, ld = K.ld;
    const long long nv = n / W;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; q + stride < nv; q += 2 * stride) {  // two vectors in flight per row
        VT xa = reinterpret_cast<const VT*>(w)[q];
        VT xb = reinterpret_cast<const VT*>(w)[q + stride];
#pragma unroll
        for (int i = 0; i < JMAX; ++i)
            if (i <= j) {
                const VT va = reinterpret_cast<const VT*>(V + i * ld)[q];
                const VT vb = reinterpret_cast<const VT*>(V + i * ld)[q + stride];
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    setc(xa, k, fma(-hs[i], comp(va, k), comp(xa, k)));
                    setc(xb, k, fma(-hs[i], comp(vb, k), comp(xb, k)));
                }
            }
#pragma unroll
        for (int k = 0; k < W; ++k) {
            setc(xa, k, comp(xa, k) * inv);
            setc(xb, k, comp(xb, k) * inv);
        }
        reinterpret_cast<VT*>(out)[q] = xa;
        reinterpret_cast<VT*>(out)[q + stride] = xb;
    }
    for (; q < nv; q += stride) {
        VT x = reinterpret_cast<const VT*>(w)[q];
#pragma unroll
        for (int i = 0; i < JMAX; ++i)
            if (i <= j) {
                const VT vv = reinterpret_cast<const VT*>(V + i * ld)[q];
#pragma unroll
                for (int k = 0; k < W; ++k) setc(x, k, fma(-hs[i], comp(vv, k), comp(x, k)));
            }
#pragma unroll
        for (int k = 0; k < W; ++k) setc(x, k, comp(x, k) * inv);
        reinterpret_cast<VT*>(out)[q] = x;
    }
    if (blockIdx.x == 0) {
        for (long long e = nv * W + threadIdx.x; e < n; e += blockDim.x) {
            T x = w[e];
#pragma unroll
            for (int i = 0; i < JMAX; ++i)
                if (i <= j) x = fma(-hs[i], V[i * ld + e], x);
            out[e] = x * inv;
        }
    }
}

template <class T, int JMAX>
static void arnoldi_pass(const ArnoldiDev& K, T* V, T* w, int j, int pass, cudaStream_t s) {
    k_arnoldi_dots<T, JMAX><<<K.blocks, kArThreads, 0, s>>>(K, V, w, j, pass);
    k_arnoldi_update<T, JMAX><<<K.blocks, kArThreads, 0, s>>>(K, V, w, j, pass);
}

template <class T>
static void arnoldi_step(const ArnoldiDev& K, T* V, T* w, int j, cudaStream_t s) {
    for (int pass = 1; pass <= 2; ++pass) {
        if (j < 4)
            arnoldi_pass<T, 4>(K, V, w, j, pass, s);
        else if (j < 8)
            arnoldi_pass<T, 8>(K, V, w, j, pass, s);
        else if (j < 16)
            arnoldi_pass<T, 16>(K, V, w, j, pass, s);
        else
            arnoldi_pass<T, kCols>(K, V, w, j, pass, s);
    }
}

void launch_arnoldi_step_f64(const ArnoldiDev& K, double* V, double* w, int j, cudaStream_t s) {
    arnoldi_step<double>(K, V, w, j, s);
}

void launch_arnoldi_step_f32(const ArnoldiDev& K, float* V, float* w, int j, cudaStream_t s) {
    arnoldi_step<float>(K, V, w, j, s);
}

}  // namespace m1
