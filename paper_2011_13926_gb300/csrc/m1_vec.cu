// m1_vec.cu — vector kernels around the Krylov solver: norms (warp shuffles +
// block reductions, FP64 accumulation in a fixed order so that results are
// reproducible run to run), linear combinations, precision conversions, the
// least-squares back substitution and the realizability count.
#include "m1_internal.h"

namespace m1 {

static constexpr int kRedThreads = 256;
static constexpr int kRedBlocks = 608;  // 4 x 152 SMs; fixed so sums are deterministic
static constexpr int kMaxCols = kMaxRestart + 1;

int reduce_blocks() { return kRedBlocks; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of partials[b * ncols + c] over b for each column c (one block, fixed order)
__global__ void k_finish_sum(const double* __restrict__ partials, int nparts, int ncols, double* __restrict__ out) {
    __shared__ double red[kRedThreads / 32];
    for (int c = 0; c < ncols; ++c) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) t += partials[(long long)b * ncols + c];
        t = warp_sum(t);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x < 32) {
            double u = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            u = warp_sum(u);
            if (threadIdx.x == 0) out[c] = u;
        }
        __syncthreads();
    }
}

void launch_finish_sum(const double* partials, int nparts, int ncols, double* out, cudaStream_t s) {
    k_finish_sum<<<1, kRedThreads, 0, s>>>(partials, nparts, ncols, out);
}

template <class T>
__global__ void k_norm2(const T* __restrict__ x, long long n, double* __restrict__ partials) {
    __shared__ double red[kRedThreads / 32];
    double t = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        t += v * v;
    }
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        u = warp_sum(u);
        if (threadIdx.x == 0) partials[blockIdx.x] = u;
    }
}

// FP32 vector: squares accumulated per thread in double-float FP32 (TwoSum),
// one FP64 conversion per thread, so the narrow FP64 pipe sees no per-element work
__global__ void k_norm2_f32(const float* __restrict__ x, long long n, double* __restrict__ partials) {
    __shared__ double red[kRedThreads / 32];
    float hi = 0.f, lo = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = x[i];
        const float p = v * v;
        const float pe = fmaf(v, v, -p);
        const float s = hi + p;
        const float bb = s - hi;
        lo += ((hi - (s - bb)) + (p - bb)) + pe;
        hi = s;
    }
    double t = (double)hi + (double)lo;
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        u = warp_sum(u);
        if (threadIdx.x == 0) partials[blockIdx.x] = u;
    }
}

void launch_norm2_f64(const double* x, long long n, double* partials, double* out, cudaStream_t s) {
    k_norm2<double><<<kRedBlocks, kRedThreads, 0, s>>>(x, n, partials);
    launch_finish_sum(partials, kRedBlocks, 1, out, s);
}
void launch_norm2_f32(const float* x, long long n, double* partials, double* out, cudaStream_t s) {
    k_norm2_f32<<<kRedBlocks, kRedThreads, 0, s>>>(x, n, partials);
    launch_finish_sum(partials, kRedBlocks, 1, out, s);
}

template <class T>
__global__ void k_scale_inv_sqrt(const T* __restrict__ x, const double* __restrict__ nrm2, T* __restrict__ y,
                                 long long n) {
    __shared__ T sc;
    if (threadIdx.x == 0) {
        const double nn = nrm2[0];
        sc = (T)(nn > 0.0 ? 1.0 / sqrt(nn) : 0.0);
    }
    __syncthreads();
    const T s = sc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}
void launch_scale_inv_sqrt_f64(const double* x, const double* nrm2, double* y, long long n, cudaStream_t s) {
    k_scale_inv_sqrt<double><<<kRedBlocks, kRedThreads, 0, s>>>(x, nrm2, y, n);
}
void launch_scale_inv_sqrt_f32(const float* x, const double* nrm2, float* y, long long n, cudaStream_t s) {
    k_scale_inv_sqrt<float><<<kRedBlocks, kRedThreads, 0, s>>>(x, nrm2, y, n);
}

__global__ void k_scale_f64_to_f32(const double* __restrict__ x, const double* __restrict__ nrm2,
                                   float* __restrict__ y, long long n) {
    const double nn = nrm2[0];
    const double s = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)(x[i] * s);
}
void launch_scale_f64_to_f32(const double* x, const double* nrm2, float* y, long long n, cudaStream_t s) {
    k_scale_f64_to_f32<<<kRedBlocks, kRedThreads, 0, s>>>(x, nrm2, y, n);
}

// x += sum_{i<k} y_i Z_i; rows of Z start on 256-byte boundaries (ld % 64 == 0),
// x is a separate 256-byte-aligned allocation: two elements per thread step
template <class T>
__global__ void k_lincomb_add(const T* __restrict__ Z, long long ld, int k, const double* __restrict__ y,
                              double* __restrict__ x, long long n) {
    __shared__ double ys[kMaxCols];
    if (threadIdx.x < kMaxCols) ys[threadIdx.x] = threadIdx.x < k ? y[threadIdx.x] : 0.0;
    __syncthreads();
    const long long n2 = n / 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += (long long)gridDim.x * blockDim.x) {
        double2 acc = reinterpret_cast<const double2*>(x)[q];
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const T* zi = Z + i * ld + 2 * q;
            acc.x += ys[i] * (double)zi[0];
            acc.y += ys[i] * (double)zi[1];
        }
        reinterpret_cast<double2*>(x)[q] = acc;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
        double acc = x[n - 1];
        for (int i = 0; i < k; ++i) acc += ys[i] * (double)Z[i * ld + n - 1];
        x[n - 1] = acc;
    }
}
// FP32 basis: the k-term combination in FP32 (FMA chain with the weights
// rounded to FP32; it feeds an inner correction solved to a relative 1e-4),
// then one FP64 add per element
__global__ void k_lincomb_add_f32(const float* __restrict__ Z, long long ld, int k, const double* __restrict__ y,
                                  double* __restrict__ x, long long n) {
    __shared__ float ys[kMaxCols];
    if (threadIdx.x < kMaxCols) ys[threadIdx.x] = threadIdx.x < k ? (float)y[threadIdx.x] : 0.f;
    __syncthreads();
    const long long n4 = n / 4;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const float4 z = __ldg(reinterpret_cast<const float4*>(Z + i * ld) + q);
            const float yi = ys[i];
            a.x = fmaf(yi, z.x, a.x);
            a.y = fmaf(yi, z.y, a.y);
            a.z = fmaf(yi, z.z, a.z);
            a.w = fmaf(yi, z.w, a.w);
        }
        double2* xp = reinterpret_cast<double2*>(x) + 2 * q;
        double2 x0 = xp[0], x1 = xp[1];
        x0.x += (double)a.x;
        x0.y += (double)a.y;
        x1.x += (double)a.z;
        x1.y += (double)a.w;
        xp[0] = x0;
        xp[1] = x1;
    }
    if (blockIdx.x == 0) {
        for (long long e = n4 * 4 + threadIdx.x; e < n; e += blockDim.x) {
            float a = 0.f;
            for (int i = 0; i < k; ++i) a = fmaf(ys[i], Z[i * ld + e], a);
            x[e] += (double)a;
        }
    }
}

void launch_lincomb_add_f64(const double* Z, long long ld, int k, const double* y, double* x, long long n,
                            cudaStream_t s) {
    k_lincomb_add<double><<<kRedBlocks, kRedThreads, 0, s>>>(Z, ld, k, y, x, n);
}
void launch_lincomb_add_f32_to_f64(const float* Z, long long ld, int k, const double* y, double* x, long long n,
                                   cudaStream_t s) {
    k_lincomb_add_f32<<<kRedBlocks, kRedThreads, 0, s>>>(Z, ld, k, y, x, n);
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i];
}
void launch_axpy_f64(double a, const double* x, double* y, long long n, cudaStream_t s) {
    k_axpby<<<kRedBlocks, kRedThreads, 0, s>>>(a, x, 1.0, y, y, n);
}
void launch_axpby_f64(double a, const double* x, double b, const double* y, double* out, long long n,
                      cudaStream_t s) {
    k_axpby<<<kRedBlocks, kRedThreads, 0, s>>>(a, x, b, y, out, n);
}

// out = a x + b y in FP32 (out may alias x or y: each element is read and written by one thread)
__global__ void k_axpby_f32(float a, const float* x, float b, const float* y, float* out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i];
}
void launch_axpby_f32(float a, const float* x, float b, const float* y, float* out, long long n, cudaStream_t s) {
    k_axpby_f32<<<kRedBlocks, kRedThreads, 0, s>>>(a, x, b, y, out, n);
}

template <class A, class B>
__global__ void k_convert(const A* __restrict__ x, B* __restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (B)x[i];
}
void launch_f64_to_f32(const double* x, float* y, long long n, cudaStream_t s) {
    k_convert<double, float><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n);
}
void launch_f32_to_f64(const float* x, double* y, long long n, cudaStream_t s) {
    k_convert<float, double><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n);
}

__global__ void k_backsolve(const double* H, const double* g, int k, double* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int ldh = kMaxRestart + 1;
    for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int q = i + 1; q < k; ++q) t -= H[(long long)q * ldh + i] * y[q];
        const double d = H[(long long)i * ldh + i];
        y[i] = d != 0.0 ? t / d : 0.0;
    }
}
void launch_backsolve(const double* H, const double* g, int k, double* y, cudaStream_t s) {
    k_backsolve<<<1, 32, 0, s>>>(H, g, k, y);
}

__global__ void k_realizability(const double* __restrict__ U, int dim, long long N, double c,
                                unsigned long long* count) {
    unsigned long long local = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double E = U[i];
        double F2 = 0.0;
        for (int b = 0; b < dim; ++b) {
            const double f = U[(1 + b) * N + i];
            F2 += f * f;
        }
        if (sqrt(F2) > c * E || !(E == E)) ++local;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}
void launch_realizability(const double* U, int dim, long long N, double c, unsigned long long* count,
                          cudaStream_t s) {
    k_realizability<<<kRedBlocks, kRedThreads, 0, s>>>(U, dim, N, c, count);
}

}  // namespace m1
