// m1_arnoldi.cu — fused Arnoldi step of restarted GMRES (classical
// Gram-Schmidt with selective reorthogonalisation).
//
// One Arnoldi step j on the new vector w = A M^-1 V_j is four kernels:
//   dots(pass 1): h = V_{0..j}^T w and ||w||^2 (basis vectors in groups of 8
//     over a second grid dimension, w shared through L2); the last
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
// (each 16-byte group of four products by an FMA chain, then an error-free
// TwoSum into a (hi, lo) pair), FP64 vectors in FP64; the
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
    __device__ __forceinline__ void add_prod4(const double2& a, const double2& b) {
        v = fma(a.x, b.x, v);
        v = fma(a.y, b.y, v);
    }
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
    // four products by an FMA chain (FP32 rounding), then one compensated add
    __device__ __forceinline__ void add_prod4(const float4& a, const float4& b) {
        float p = a.x * b.x;
        p = fmaf(a.y, b.y, p);
        p = fmaf(a.z, b.z, p);
        p = fmaf(a.w, b.w, p);
        two_sum_acc(t, p, 0.f);
    }
    __device__ __forceinline__ double get() const { return (double)t.hi + (double)t.lo; }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

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

// Dots: grid (bx, G). Block (x, y) accumulates the dot products of basis
// vectors i in [8y, 8y + 8) with w (and ||w||^2 when y == 0) over its
// element stride; the last block of the whole grid sums the partials.
constexpr int kGroup = 8;

template <class T>
__global__ void __launch_bounds__(kArThreads) k_arnoldi_dots(ArnoldiDev K, const T* __restrict__ V,
                                                             const T* __restrict__ w, int j, int pass) {
    if (pass == 2 && *K.reorth == 0) return;
    using VT = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    __shared__ double red[kArThreads / 32][kGroup + 1];
    __shared__ bool last;
    const int i0 = blockIdx.y * kGroup;
    const int ni = min(kGroup, j + 1 - i0);  // >= 1
    const bool with_norm = blockIdx.y == 0;
    Acc<T> acc[kGroup];
    Acc<T> ww;
#pragma unroll
    for (int i = 0; i < kGroup; ++i) acc[i].zero();
    ww.zero();
    const long long n = K.n, ld = K.ld;
    const long long nv = n / W;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T* Vg = V + (long long)i0 * ld;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; q + stride < nv; q += 2 * stride) {  // two vectors in flight per row
        const VT wa = reinterpret_cast<const VT*>(w)[q];
        const VT wb = reinterpret_cast<const VT*>(w)[q + stride];
        if (with_norm) {
            ww.add_prod4(wa, wa);
            ww.add_prod4(wb, wb);
        }
#pragma unroll
        for (int i = 0; i < kGroup; ++i)
            if (i < ni) {
                const VT va = reinterpret_cast<const VT*>(Vg + i * ld)[q];
                const VT vb = reinterpret_cast<const VT*>(Vg + i * ld)[q + stride];
                acc[i].add_prod4(va, wa);
                acc[i].add_prod4(vb, wb);
            }
    }
    for (; q < nv; q += stride) {
        const VT wv = reinterpret_cast<const VT*>(w)[q];
        if (with_norm) ww.add_prod4(wv, wv);
#pragma unroll
        for (int i = 0; i < kGroup; ++i)
            if (i < ni) {
                const VT vv = reinterpret_cast<const VT*>(Vg + i * ld)[q];
                acc[i].add_prod4(vv, wv);
            }
    }
    if (blockIdx.x == 0) {  // scalar tail
        for (long long e = nv * W + threadIdx.x; e < n; e += blockDim.x) {
            const T we = w[e];
            if (with_norm) ww.add_prod(we, we);
#pragma unroll
            for (int i = 0; i < kGroup; ++i)
                if (i < ni) acc[i].add_prod(Vg[i * ld + e], we);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
        if (i < ni) {
            const double t = warp_sum_d(acc[i].get());
            if (lane == 0) red[wid][i] = t;
        }
    }
    if (with_norm) {
        const double t = warp_sum_d(ww.get());
        if (lane == 0) red[wid][kGroup] = t;
    }
    __syncthreads();
    double* part = K.partials + (long long)blockIdx.x * (kCols + 1);
    for (int i = threadIdx.x; i <= kGroup; i += blockDim.x) {
        if (i < ni || (i == kGroup && with_norm)) {
            double t = 0.0;
            for (int qq = 0; qq < (int)(blockDim.x >> 5); ++qq) t += red[qq][i];
            part[i < kGroup ? i0 + i : kCols] = t;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(K.counter, 1u) == gridDim.x * gridDim.y - 1);
    __syncthreads();
    if (!last) return;
    // the last block: fixed-order sums of the partials over the x blocks
    __shared__ double tot[kCols + 1];
    for (int i = wid; i <= kCols; i += (int)(blockDim.x >> 5)) {
        if (i <= j || i == kCols) {
            double t = 0.0;
#pragma unroll 12
            for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(K.partials + (long long)b * (kCols + 1) + i);
            t = warp_sum_d(t);
            if (lane == 0) tot[i] = t;
        }
    }
    __syncthreads();  // tot[] complete
    // stage the previous rotations and the column (h1 [+ h2]) in shared memory
    __shared__ double col[kCols + 1], scs[kCols], ssn[kCols];
    double* h = pass == 1 ? K.h1 : K.h2;
    if (threadIdx.x <= j) {
        const double hv = tot[threadIdx.x];
        h[threadIdx.x] = hv;
        col[threadIdx.x] = pass == 2 ? K.h1[threadIdx.x] + hv : hv;
    }
    if (threadIdx.x < j) {
        scs[threadIdx.x] = K.cs[threadIdx.x];
        ssn[threadIdx.x] = K.sn[threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *K.counter = 0u;
        double hh = 0.0;
        for (int i = 0; i <= j; ++i) hh += tot[i] * tot[i];
        const double wn2 = tot[kCols];
        const double rest = wn2 - hh;
        if (pass == 1 && !(rest > 0.5 * wn2)) {
            *K.reorth = 1;  // second pass decides the column
            K.resid[2] = 1.0;
        } else {
            if (pass == 1) {
                K.resid[2] = 0.0;
                *K.reorth = 0;
            }
            givens_column(K, col, scs, ssn, sqrt(fmax(rest, 0.0)), j);
        }
    }
}

// Update: out = (w - sum_{i<=j} h_i V_i) * inv; the loop over i has a runtime
// bound (unrolled by 4) so that the loads of the basis are not all hoisted.
template <class T>
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
#pragma unroll 4
        for (int i = 0; i <= j; ++i) {
            const VT va = reinterpret_cast<const VT*>(V + i * ld)[q];
            const VT vb = reinterpret_cast<const VT*>(V + i * ld)[q + stride];
            const T hi = hs[i];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                setc(xa, k, fma(-hi, comp(va, k), comp(xa, k)));
                setc(xb, k, fma(-hi, comp(vb, k), comp(xb, k)));
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
#pragma unroll 4
        for (int i = 0; i <= j; ++i) {
            const VT vv = reinterpret_cast<const VT*>(V + i * ld)[q];
            const T hi = hs[i];
#pragma unroll
            for (int k = 0; k < W; ++k) setc(x, k, fma(-hi, comp(vv, k), comp(x, k)));
        }
#pragma unroll
        for (int k = 0; k < W; ++k) setc(x, k, comp(x, k) * inv);
        reinterpret_cast<VT*>(out)[q] = x;
    }
    if (blockIdx.x == 0) {
        for (long long e = nv * W + threadIdx.x; e < n; e += blockDim.x) {
            T x = w[e];
            for (int i = 0; i <= j; ++i) x = fma(-hs[i], V[i * ld + e], x);
            out[e] = x * inv;
        }
    }
}

template <class T>
static void arnoldi_step(const ArnoldiDev& K, T* V, T* w, int j, cudaStream_t s) {
    const dim3 gd(K.blocks, (j + kGroup) / kGroup);  // ceil((j + 1) / 8) groups of basis vectors
    for (int pass = 1; pass <= 2; ++pass) {
        k_arnoldi_dots<T><<<gd, kArThreads, 0, s>>>(K, V, w, j, pass);
        k_arnoldi_update<T><<<2 * K.blocks, kArThreads, 0, s>>>(K, V, w, j, pass);
    }
}

void launch_arnoldi_step_f64(const ArnoldiDev& K, double* V, double* w, int j, cudaStream_t s) {
    arnoldi_step<double>(K, V, w, j, s);
}

void launch_arnoldi_step_f32(const ArnoldiDev& K, float* V, float* w, int j, cudaStream_t s) {
    arnoldi_step<float>(K, V, w, j, s);
}

}  // namespace m1
