// m1_bicgstab.cu — vector kernels of right-preconditioned BiCGStab, the
// Krylov solver of the paper (Sect. 3.3.1; van der Vorst's method), with every
// recurrence scalar kept on the device.
//
// One iteration on A M^-1 y = b (x = M^-1 y accumulated directly):
//   rho' = (rhat, r);  beta = (rho' / rho) (alpha / omega)   [finish, kRho]
//   p = r + beta (p - omega v)                                [k_bs_p]
//   phat = M^-1 p;  v = A phat                                [caller]
//   alpha = rho' / (rhat, v)                                  [dots + finish, kAlpha]
//   s = r - alpha v                                           [k_bs_s]
//   shat = M^-1 s;  t = A shat                                [caller]
//   omega = (t, s) / (t, t)                                   [dots + finish, kOmega]
//   x += alpha phat + omega shat;  r = s - omega t,
//   with (rhat, r) and ||r||^2 of the new r in the same pass  [k_bs_xr + finish, kRho]
// Dot products of FP32 vectors accumulate in double-float FP32 per thread and
// warp and in FP64 across blocks; FP64 vectors in FP64; all sums are in a
// fixed order. A zero denominator sets the breakdown flag and zero step sizes.
#include "m1_internal.h"

#include <algorithm>

namespace m1 {

constexpr int kBsThreads = 256;
constexpr int kBsBlocks = 2 * 152;
constexpr int kBsMaxDots = 3;

// double-float accumulator for FP32 products, FP64 for FP64
template <class T> struct BsAcc;
template <> struct BsAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        const float s = hi + p;
        const float bb = s - hi;
        lo += ((hi - (s - bb)) + (p - bb)) + e;
        hi = s;
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};
template <> struct BsAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double get() const { return v; }
};

__device__ __forceinline__ double bs_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block partials of up to kBsMaxDots dot products (a_k, b_k) into part[block * kBsMaxDots + k]
template <class T>
__device__ __forceinline__ void bs_block_partials(BsAcc<T>* acc, int nd, double* part) {
    __shared__ double red[kBsThreads / 32][kBsMaxDots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < nd; ++k) {
        const double v = bs_warp_sum(acc[k].get());
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < nd) {
        double v = 0.0;
        for (int q = 0; q < kBsThreads / 32; ++q) v += red[q][threadIdx.x];
        part[(long long)blockIdx.x * kBsMaxDots + threadIdx.x] = v;
    }
}

template <class T>
__global__ void __launch_bounds__(kBsThreads) k_bs_dots(const T* __restrict__ a0, const T* __restrict__ b0,
                                                        const T* __restrict__ a1, const T* __restrict__ b1,
                                                        long long n, int nd, double* __restrict__ part) {
    BsAcc<T> acc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        acc[0].add(a0[i], b0[i]);
        if (nd > 1) acc[1].add(a1[i], b1[i]);
    }
    bs_block_partials<T>(acc, nd, part);
}

// p = r + beta (p - omega v)
template <class T>
__global__ void k_bs_p(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ v,
                       const double* __restrict__ sc, long long n) {
    const T beta = (T)sc[kBsBeta], omega = (T)sc[kBsOmega];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

// s = r - alpha v
template <class T>
__global__ void k_bs_s(T* __restrict__ s, const T* __restrict__ r, const T* __restrict__ v,
                       const double* __restrict__ sc, long long n) {
    const T alpha = (T)sc[kBsAlpha];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = r[i] - alpha * v[i];
}

// x += alpha phat + omega shat (x in FP64); r = s - omega t; partials of (rhat, r) and (r, r)
template <class T>
__global__ void __launch_bounds__(kBsThreads) k_bs_xr(double* __restrict__ x, T* __restrict__ r,
                                                      const T* __restrict__ phat, const T* __restrict__ shat,
                                                      const T* __restrict__ s, const T* __restrict__ t,
                                                      const T* __restrict__ rhat, const double* __restrict__ sc,
                                                      long long n, double* __restrict__ part) {
    const double alpha = sc[kBsAlpha], omega = sc[kBsOmega];
    const T om = (T)omega;
    BsAcc<T> acc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] += alpha * (double)phat[i] + omega * (double)shat[i];
        const T ri = s[i] - om * t[i];
        r[i] = ri;
        acc[0].add(rhat[i], ri);
        acc[1].add(ri, ri);
    }
    bs_block_partials<T>(acc, 2, part);
}

// one block: fixed-order sums of the partials, then the mode's scalar update
__global__ void k_bs_finish(const double* __restrict__ part, int nb, int nd, int mode, double* __restrict__ sc,
                            double* __restrict__ host_slot) {
    __shared__ double red[32][kBsMaxDots];
    __shared__ double tot[kBsMaxDots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < nd; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[(long long)b * kBsMaxDots + k];
        v = bs_warp_sum(v);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < nd) {
        double v = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[q][threadIdx.x];
        tot[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (mode == kBsModeRho) {  // tot = ((rhat, r), (r, r)); first call: rho = alpha = omega = 1
        const double rho_new = tot[0];
        const double rho = sc[kBsRho], alpha = sc[kBsAlpha], omega = sc[kBsOmega];
        const bool ok = rho != 0.0 && omega != 0.0 && rho_new == rho_new;
        sc[kBsBeta] = ok ? (rho_new / rho) * (alpha / omega) : 0.0;
        if (!ok) sc[kBsBreak] = 1.0;
        sc[kBsRho] = rho_new;
        sc[kBsRR] = tot[1];
        if (host_slot) {
            host_slot[0] = tot[1];
            host_slot[1] = sc[kBsBreak];
        }
    } else if (mode == kBsModeAlpha) {  // tot = ((rhat, v))
        const double rv = tot[0];
        const bool ok = rv != 0.0 && rv == rv;
        sc[kBsAlpha] = ok ? sc[kBsRho] / rv : 0.0;
        if (!ok) sc[kBsBreak] = 1.0;
    } else {  // kBsModeOmega: tot = ((t, s), (t, t))
        const bool ok = tot[1] > 0.0;
        sc[kBsOmega] = ok ? tot[0] / tot[1] : 0.0;
        if (!ok) sc[kBsBreak] = 1.0;
    }
}

static int bs_grid(long long n) { return (int)std::min<long long>(kBsBlocks, (n + kBsThreads - 1) / kBsThreads); }

template <class T>
static void bs_dots(const T* a0, const T* b0, const T* a1, const T* b1, long long n, int nd, double* part, int mode,
                    double* sc, double* host_slot, cudaStream_t s) {
    const int nb = bs_grid(n);
    k_bs_dots<T><<<nb, kBsThreads, 0, s>>>(a0, b0, a1 ? a1 : a0, b1 ? b1 : b0, n, nd, part);
    k_bs_finish<<<1, 1024, 0, s>>>(part, nb, nd, mode, sc, host_slot);
}

template <class T>
static void bs_p(T* p, const T* r, const T* v, const double* sc, long long n, cudaStream_t s) {
    k_bs_p<T><<<bs_grid(n), kBsThreads, 0, s>>>(p, r, v, sc, n);
}
template <class T>
static void bs_s(T* sv, const T* r, const T* v, const double* sc, long long n, cudaStream_t s) {
    k_bs_s<T><<<bs_grid(n), kBsThreads, 0, s>>>(sv, r, v, sc, n);
}
template <class T>
static void bs_xr(double* x, T* r, const T* phat, const T* shat, const T* sv, const T* t, const T* rhat, double* sc,
                  long long n, double* part, double* host_slot, cudaStream_t s) {
    const int nb = bs_grid(n);
    k_bs_xr<T><<<nb, kBsThreads, 0, s>>>(x, r, phat, shat, sv, t, rhat, sc, n, part);
    k_bs_finish<<<1, 1024, 0, s>>>(part, nb, 2, kBsModeRho, sc, host_slot);
}

void launch_bs_dots_f64(const double* a0, const double* b0, const double* a1, const double* b1, long long n, int nd,
                        double* part, int mode, double* sc, double* host_slot, cudaStream_t s) {
    bs_dots<double>(a0, b0, a1, b1, n, nd, part, mode, sc, host_slot, s);
}
void launch_bs_dots_f32(const float* a0, const float* b0, const float* a1, const float* b1, long long n, int nd,
                        double* part, int mode, double* sc, double* host_slot, cudaStream_t s) {
    bs_dots<float>(a0, b0, a1, b1, n, nd, part, mode, sc, host_slot, s);
}
void launch_bs_p_f64(double* p, const double* r, const double* v, const double* sc, long long n, cudaStream_t s) {
    bs_p<double>(p, r, v, sc, n, s);
}
void launch_bs_p_f32(float* p, const float* r, const float* v, const double* sc, long long n, cudaStream_t s) {
    bs_p<float>(p, r, v, sc, n, s);
}
void launch_bs_s_f64(double* sv, const double* r, const double* v, const double* sc, long long n, cudaStream_t s) {
    bs_s<double>(sv, r, v, sc, n, s);
}
void launch_bs_s_f32(float* sv, const float* r, const float* v, const double* sc, long long n, cudaStream_t s) {
    bs_s<float>(sv, r, v, sc, n, s);
}
void launch_bs_xr_f64(double* x, double* r, const double* phat, const double* shat, const double* sv,
                      const double* t, const double* rhat, double* sc, long long n, double* part, double* host_slot,
                      cudaStream_t s) {
    bs_xr<double>(x, r, phat, shat, sv, t, rhat, sc, n, part, host_slot, s);
}
void launch_bs_xr_f32(double* x, float* r, const float* phat, const float* shat, const float* sv, const float* t,
                      const float* rhat, double* sc, long long n, double* part, double* host_slot, cudaStream_t s) {
    bs_xr<float>(x, r, phat, shat, sv, t, rhat, sc, n, part, host_slot, s);
}
int bs_partial_rows() { return kBsBlocks * kBsMaxDots; }

}  // namespace m1
