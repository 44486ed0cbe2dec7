// m1_unet.cu — the learned preconditioner network: a 3-level 2D U-Net
// (63,443 parameters), its forward and backward kernels, loss, Adam, and the
// packing between Krylov vectors and network tensors.
//
// Layers (all 3x3 convolutions, stride 1, zero padding, weights W[ky][kx][ci][co]):
//   e1a 4->16, e1b 16->16 | pool | e2a 16->32, e2b 32->32 | pool |
//   e3a 32->32, e3b 32->32 | up, cat(e2b) | d2a 64->32, d2b 32->16 | up, cat(e1b) |
//   d1a 32->16, d1b 16->3 (linear); ReLU after every other convolution.
// Tensors are NHWC. Activations are stored in FP32 for training and in BF16
// for inference; weights are FP32 masters with a BF16 copy (the forward pass
// always uses BF16-rounded weights); every product is accumulated in FP32.
//
// The convolution kernel stages a 16x16-pixel tile plus halo of 16 input
// channels and the matching 9x16x16 weight block in shared memory; each thread
// owns one output pixel and 16 output channels. The backward data pass is the
// same kernel on the flipped, transposed weights; the weight gradient is a
// per-CTA partial sum over pixel tiles reduced in a fixed order.
#include <cuda_bf16.h>
#include <math.h>

#include <string>
#include <vector>

#include "../../include/m1.h"
#include "m1_internal.h"

namespace {

constexpr int kT = 16;       // pixel tile edge
constexpr int kCC = 16;      // channel chunk (input and output)
constexpr int kDwGrid = 304; // CTAs of the weight-gradient kernel

struct LayerSpec {
    const char* name;
    int cin, cout;
    bool relu;
};
constexpr int kLayers = 10;
const LayerSpec kSpec[kLayers] = {
    {"e1a", 4, 16, true},  {"e1b", 16, 16, true}, {"e2a", 16, 32, true}, {"e2b", 32, 32, true},
    {"e3a", 32, 32, true}, {"e3b", 32, 32, true}, {"d2a", 64, 32, true}, {"d2b", 32, 16, true},
    {"d1a", 32, 16, true}, {"d1b", 16, 3, false},
};

template <class T> __device__ __forceinline__ float ld(const T* p, long long i);
template <> __device__ __forceinline__ float ld<float>(const float* p, long long i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
    return __bfloat162float(p[i]);
}
template <class T> __device__ __forceinline__ void st(T* p, long long i, float v);
template <> __device__ __forceinline__ void st<float>(float* p, long long i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16* p, long long i, float v) {
    p[i] = __float2bfloat16(v);
}

// y[b,i,j,co] = bias[co] + sum x[b,i+dy-1,j+dx-1,ci] w[dy][dx][ci][co]; optional
// ReLU; optional multiplicative mask (mask > 0) for backward passes.
// Grid: (ceil(W/16), ceil(H/16), B), 256 threads.
template <class Tin, class Tout>
__global__ void __launch_bounds__(256) k_conv3x3(const Tin* __restrict__ x, int cin, const float* __restrict__ w,
                                                 const float* __restrict__ bias, Tout* __restrict__ y, int cout,
                                                 int H, int W, int relu, const float* __restrict__ mask) {
    __shared__ float xs[kT + 2][kT + 2][kCC + 1];  // +1: conflict-free strided reads
    __shared__ __align__(16) float ws[9][kCC][kCC];
    const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
    const int j0 = blockIdx.x * kT, i0 = blockIdx.y * kT, b = blockIdx.z;
    const int i = i0 + ty, j = j0 + tx;
    const long long img = (long long)b * H * W;
    for (int co0 = 0; co0 < cout; co0 += kCC) {
        const int nco = min(kCC, cout - co0);
        float acc[kCC];
#pragma unroll
        for (int c = 0; c < kCC; ++c) acc[c] = (bias && c < nco) ? bias[co0 + c] : 0.f;
        for (int ci0 = 0; ci0 < cin; ci0 += kCC) {
            const int nci = min(kCC, cin - ci0);
            __syncthreads();
            for (int t = threadIdx.x; t < (kT + 2) * (kT + 2) * kCC; t += blockDim.x) {
                const int c = t % kCC, px = (t / kCC) % (kT + 2), py = t / (kCC * (kT + 2));
                const int gi = i0 + py - 1, gj = j0 + px - 1;
                float v = 0.f;
                if (c < nci && gi >= 0 && gi < H && gj >= 0 && gj < W)
                    v = ld(x, (img + (long long)gi * W + gj) * cin + ci0 + c);
                xs[py][px][c] = v;
            }
            for (int t = threadIdx.x; t < 9 * kCC * kCC; t += blockDim.x) {
                const int co = t % kCC, c = (t / kCC) % kCC, tap = t / (kCC * kCC);
                ws[tap][c][co] = (c < nci && co < nco) ? w[((long long)tap * cin + ci0 + c) * cout + co0 + co] : 0.f;
            }
            __syncthreads();
            for (int c = 0; c < nci; ++c) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const float xv = xs[ty + tap / 3][tx + tap % 3][c];
                    const float4* w4 = reinterpret_cast<const float4*>(&ws[tap][c][0]);
#pragma unroll
                    for (int q = 0; q < kCC / 4; ++q) {
                        const float4 wv = w4[q];
                        acc[4 * q + 0] = fmaf(xv, wv.x, acc[4 * q + 0]);
                        acc[4 * q + 1] = fmaf(xv, wv.y, acc[4 * q + 1]);
                        acc[4 * q + 2] = fmaf(xv, wv.z, acc[4 * q + 2]);
                        acc[4 * q + 3] = fmaf(xv, wv.w, acc[4 * q + 3]);
                    }
                }
            }
        }
        if (i < H && j < W) {
            const long long o = (img + (long long)i * W + j) * cout + co0;
#pragma unroll
            for (int c = 0; c < kCC; ++c) {
                if (c < nco) {
                    float v = acc[c];
                    if (relu) v = fmaxf(v, 0.f);
                    if (mask) v = mask[o + c] > 0.f ? v : 0.f;
                    st(y, o + c, v);
                }
            }
        }
    }
}

// Wt[dy][dx][co][ci] = W[2-dy][2-dx][ci][co]: the backward data pass as a convolution
__global__ void k_flip_weights(const float* __restrict__ w, float* __restrict__ wt, int cin, int cout) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 9 * cin * cout) return;
    const int co = t % cout, ci = (t / cout) % cin, tap = t / (cout * cin);
    wt[((long long)(8 - tap) * cout + co) * cin + ci] = w[t];
}

// g *= (out > 0) in place (gradient of a ReLU output -> pre-activation)
__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ out, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        if (!(out[k] > 0.f)) g[k] = 0.f;
}

// Partial weight/bias gradients: CTA c sums over the pixel tiles c, c + G, ...
// part[c][tap][ci][co] and part[c][9*cin*cout + co] (bias). Channel chunks of 16.
__global__ void __launch_bounds__(256) k_conv3x3_dw(const float* __restrict__ x, int cin,
                                                    const float* __restrict__ g, int cout, int B, int H, int W,
                                                    float* __restrict__ part) {
    __shared__ float xs[kT + 2][kT + 2][kCC];
    __shared__ float gs[kT][kT][kCC];
    const int tilesx = (W + kT - 1) / kT, tilesy = (H + kT - 1) / kT;
    const long long ntiles = (long long)B * tilesx * tilesy;
    const long long nw = 9LL * cin * cout;
    float* myp = part + (long long)blockIdx.x * (nw + cout);
    for (int co0 = 0; co0 < cout; co0 += kCC) {
        const int nco = min(kCC, cout - co0);
        for (int ci0 = 0; ci0 < cin; ci0 += kCC) {
            const int nci = min(kCC, cin - ci0);
            // each thread owns entries e = threadIdx.x + 256 k of the 9 x 16 x 16 chunk
            float acc[9];
            float bacc = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = 0.f;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                const int b = (int)(tile / (tilesx * tilesy));
                const int rem = (int)(tile % (tilesx * tilesy));
                const int i0 = (rem / tilesx) * kT, j0 = (rem % tilesx) * kT;
                const long long img = (long long)b * H * W;
                __syncthreads();
                for (int t = threadIdx.x; t < (kT + 2) * (kT + 2) * kCC; t += blockDim.x) {
                    const int c = t % kCC, px = (t / kCC) % (kT + 2), py = t / (kCC * (kT + 2));
                    const int gi = i0 + py - 1, gj = j0 + px - 1;
                    float v = 0.f;
                    if (c < nci && gi >= 0 && gi < H && gj >= 0 && gj < W)
                        v = x[(img + (long long)gi * W + gj) * cin + ci0 + c];
                    xs[py][px][c] = v;
                }
                for (int t = threadIdx.x; t < kT * kT * kCC; t += blockDim.x) {
                    const int c = t % kCC, px = (t / kCC) % kT, py = t / (kCC * kT);
                    const int gi = i0 + py, gj = j0 + px;
                    float v = 0.f;
                    if (c < nco && gi < H && gj < W) v = g[(img + (long long)gi * W + gj) * cout + co0 + c];
                    gs[py][px][c] = v;
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const int e = threadIdx.x + 256 * k;  // e = (tap, ci, co) in the 9 x 16 x 16 chunk
                    const int co = e % kCC, ci = (e / kCC) % kCC, tap = e / (kCC * kCC);
                    const int dy = tap / 3, dx = tap % 3;
                    float s = 0.f;
                    for (int py = 0; py < kT; ++py)
#pragma unroll 4
                        for (int px = 0; px < kT; ++px) s = fmaf(xs[py + dy][px + dx][ci], gs[py][px][co], s);
                    acc[k] += s;
                }
                if (ci0 == 0 && threadIdx.x < kCC) {
                    float s = 0.f;
                    for (int py = 0; py < kT; ++py)
                        for (int px = 0; px < kT; ++px) s += gs[py][px][threadIdx.x];
                    bacc += s;
                }
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int e = threadIdx.x + 256 * k;
                const int co = e % kCC, ci = (e / kCC) % kCC, tap = e / (kCC * kCC);
                if (ci < nci && co < nco) myp[((long long)tap * cin + ci0 + ci) * cout + co0 + co] = acc[k];
            }
            if (ci0 == 0 && threadIdx.x < nco) myp[nw + co0 + threadIdx.x] = bacc;
        }
    }
}

// out[e] = sum_c part[c][e] over the kDwGrid CTAs, fixed order
__global__ void k_reduce_parts(const float* __restrict__ part, long long stride, long long n, int nparts,
                               float* __restrict__ out) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < nparts; ++c) s += part[(long long)c * stride + e];
        out[e] = s;
    }
}

template <class T>
__global__ void k_pool2(const T* __restrict__ x, T* __restrict__ y, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        long long r = k / C;
        const int j = (int)(r % Wo);
        r /= Wo;
        const int i = (int)(r % Ho);
        const int b = (int)(r / Ho);
        const long long base = (((long long)b * H + 2 * i) * W + 2 * j) * C + c;
        const float s = ld(x, base) + ld(x, base + C) + ld(x, base + (long long)W * C) + ld(x, base + (long long)W * C + C);
        st(y, k, 0.25f * s);
    }
}

__global__ void k_pool2_bwd(const float* __restrict__ gy, float* __restrict__ gx, int B, int H, int W, int C,
                            int accumulate) {
    const long long n = (long long)B * H * W * C;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        long long r = k / C;
        const int j = (int)(r % W);
        r /= W;
        const int i = (int)(r % H);
        const int b = (int)(r / H);
        const float v = 0.25f * gy[(((long long)b * (H / 2) + i / 2) * (W / 2) + j / 2) * C + c];
        gx[k] = accumulate ? gx[k] + v : v;
    }
}

// y[:, :, :, 0:C1] = up2(a), y[:, :, :, C1:C1+C2] = s (skip), at the fine resolution H x W
template <class T>
__global__ void k_up_cat(const T* __restrict__ a, int C1, const T* __restrict__ s, int C2, T* __restrict__ y,
                         int B, int H, int W) {
    const int C = C1 + C2;
    const long long n = (long long)B * H * W * C;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C);
        const long long p = k / C;
        const int j = (int)(p % W);
        const int i = (int)((p / W) % H);
        const int b = (int)(p / ((long long)W * H));
        float v;
        if (c < C1)
            v = ld(a, (((long long)b * (H / 2) + i / 2) * (W / 2) + j / 2) * C1 + c);
        else
            v = ld(s, p * C2 + (c - C1));
        st(y, k, v);
    }
}

// backward of up_cat: ga (coarse, summed over the 2x2 children) and gs (+=)
__global__ void k_up_cat_bwd(const float* __restrict__ gy, float* __restrict__ ga, int C1, float* __restrict__ gs,
                             int C2, int B, int H, int W) {
    const int C = C1 + C2;
    const long long nc = (long long)B * (H / 2) * (W / 2) * C1;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(k % C1);
        long long r = k / C1;
        const int j = (int)(r % (W / 2));
        r /= (W / 2);
        const int i = (int)(r % (H / 2));
        const int b = (int)(r / (H / 2));
        float s = 0.f;
        for (int di = 0; di < 2; ++di)
            for (int dj = 0; dj < 2; ++dj)
                s += gy[(((long long)b * H + 2 * i + di) * W + 2 * j + dj) * C + c];
        ga[k] = s;
    }
    const long long nf = (long long)B * H * W * C2;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += (long long)gridDim.x * blockDim.x) {
        const long long p = k / C2;
        const int c = (int)(k % C2);
        gs[k] += gy[p * C + C1 + c];
    }
}

// per-sample relative squared error and its gradient dy = 2 (y - t) / ||t_b||^2 / B
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, long long per, int B,
                       float* __restrict__ gy, double* __restrict__ loss) {
    __shared__ double red[2][8];
    const int b = blockIdx.x;
    double num = 0.0, den = 0.0;
    for (long long k = threadIdx.x; k < per; k += blockDim.x) {
        const double d = (double)y[b * per + k] - (double)t[b * per + k];
        num += d * d;
        den += (double)t[b * per + k] * t[b * per + k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = num;
        red[1][threadIdx.x >> 5] = den;
    }
    __syncthreads();
    __shared__ double tot[2];
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += red[0][q];
            c += red[1][q];
        }
        tot[0] = a;
        tot[1] = fmax(c, 1e-30);
        loss[b] = a / tot[1] / B;
    }
    __syncthreads();
    const float sc = (float)(2.0 / tot[1] / B);
    for (long long k = threadIdx.x; k < per; k += blockDim.x) gy[b * per + k] = sc * (y[b * per + k] - t[b * per + k]);
}

__global__ void k_adam(float* __restrict__ th, __nv_bfloat16* __restrict__ th16, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float t = th[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        th[k] = t;
        th16[k] = __float2bfloat16(t);
    }
}

__global__ void k_round_bf16(const float* __restrict__ a, float* __restrict__ r, __nv_bfloat16* __restrict__ h,
                             long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat16 q = __float2bfloat16(a[k]);
        h[k] = q;
        r[k] = __bfloat162float(q);
    }
}

// network input from a component-major Krylov vector v (E, Fx, Fy; N = H*W
// each): x = [v / s, logsig] in NHWC, s = scale
template <class T>
__global__ void k_pack_input(const float* __restrict__ v, long long N, const float* __restrict__ logsig, float scale,
                             T* __restrict__ x) {
    const float inv = 1.f / scale;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        st(x, 4 * p + 0, v[p] * inv);
        st(x, 4 * p + 1, v[N + p] * inv);
        st(x, 4 * p + 2, v[2 * N + p] * inv);
        st(x, 4 * p + 3, logsig[p]);
    }
}

// z (component-major) += scale * y (NHWC, 3 channels)
template <class T>
__global__ void k_unpack_add(const T* __restrict__ y, long long N, float scale, float* __restrict__ z) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        z[p] += scale * ld(y, 3 * p + 0);
        z[N + p] += scale * ld(y, 3 * p + 1);
        z[2 * N + p] += scale * ld(y, 3 * p + 2);
    }
}

__global__ void k_widen(const __nv_bfloat16* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = __bfloat162float(a[k]);
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ============================================================================ the network object
struct m1_nn {
    int H = 0, W = 0, B = 0;
    cudaStream_t s = nullptr;
    long long nparams = 0;
    long long woff[kLayers] = {}, boff[kLayers] = {};
    float* theta = nullptr;        // FP32 masters
    float* theta_r = nullptr;      // FP32 copy of the BF16-rounded weights (the forward pass uses these)
    __nv_bfloat16* theta16 = nullptr;
    float* grad = nullptr;
    float *adam_m = nullptr, *adam_v = nullptr;
    float* wflip = nullptr;        // flipped weights of one layer (backward data pass)
    float* dwpart = nullptr;       // per-CTA weight-gradient partials
    long long dwpart_size = 0;
    // activations, FP32 (training) and BF16 (inference); index by layer output + the cat/pool tensors
    std::vector<float*> act;       // FP32 tensors
    std::vector<__nv_bfloat16*> act16;
    std::vector<float*> gact;      // gradients
    double* loss_dev = nullptr;
    double* loss_host = nullptr;
    long long adam_t = 0;
    std::string err;
};

namespace {

// tensor slots (same order for act / act16 / gact)
enum Slot {
    S_IN = 0,  // B x H x W x 4
    S_E1A, S_E1B, S_P1, S_E2A, S_E2B, S_P2, S_E3A, S_E3B, S_C2, S_D2A, S_D2B, S_C1, S_D1A, S_OUT, S_T, S_COUNT
};

long long slot_elems(const m1_nn* nn, int sl) {
    const long long f = (long long)nn->B * nn->H * nn->W, h = f / 4, q = f / 16;
    switch (sl) {
        case S_IN: return f * 4;
        case S_E1A: case S_E1B: return f * 16;
        case S_P1: return h * 16;
        case S_E2A: case S_E2B: return h * 32;
        case S_P2: return q * 32;
        case S_E3A: case S_E3B: return q * 32;
        case S_C2: return h * 64;
        case S_D2A: return h * 32;
        case S_D2B: return h * 16;
        case S_C1: return f * 32;
        case S_D1A: return f * 16;
        case S_OUT: case S_T: return f * 3;
    }
    return 0;
}

m1_status nn_fail(m1_nn* nn, m1_status st, const std::string& m) {
    if (nn) nn->err = m;
    return st;
}

#define NCK(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return nn_fail(nn, e_ == cudaErrorMemoryAllocation ? M1_ERR_NOMEM : M1_ERR_CUDA,    \
                           std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

template <class Tin, class Tout>
void conv(m1_nn* nn, const Tin* x, int cin, const float* w, const float* b, Tout* y, int cout, int H, int W, int relu,
          const float* mask) {
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, nn->B);
    k_conv3x3<Tin, Tout><<<grid, 256, 0, nn->s>>>(x, cin, w, b, y, cout, H, W, relu, mask);
}

// forward pass; T = float (training, keeps every activation) or bf16 (inference)
template <class T>
void forward(m1_nn* nn, T* const* A) {
    const int H = nn->H, W = nn->W, B = nn->B;
    const float* th = nn->theta_r;
    auto L = [&](int l, const T* in, T* out, int H_, int W_) {
        conv<T, T>(nn, in, kSpec[l].cin, th + nn->woff[l], th + nn->boff[l], out, kSpec[l].cout, H_, W_,
                   kSpec[l].relu ? 1 : 0, nullptr);
    };
    L(0, A[S_IN], A[S_E1A], H, W);
    L(1, A[S_E1A], A[S_E1B], H, W);
    k_pool2<T><<<grid_for(slot_elems(nn, S_P1)), 256, 0, nn->s>>>(A[S_E1B], A[S_P1], B, H, W, 16);
    L(2, A[S_P1], A[S_E2A], H / 2, W / 2);
    L(3, A[S_E2A], A[S_E2B], H / 2, W / 2);
    k_pool2<T><<<grid_for(slot_elems(nn, S_P2)), 256, 0, nn->s>>>(A[S_E2B], A[S_P2], B, H / 2, W / 2, 32);
    L(4, A[S_P2], A[S_E3A], H / 4, W / 4);
    L(5, A[S_E3A], A[S_E3B], H / 4, W / 4);
    k_up_cat<T><<<grid_for(slot_elems(nn, S_C2)), 256, 0, nn->s>>>(A[S_E3B], 32, A[S_E2B], 32, A[S_C2], B, H / 2, W / 2);
    L(6, A[S_C2], A[S_D2A], H / 2, W / 2);
    L(7, A[S_D2A], A[S_D2B], H / 2, W / 2);
    k_up_cat<T><<<grid_for(slot_elems(nn, S_C1)), 256, 0, nn->s>>>(A[S_D2B], 16, A[S_E1B], 16, A[S_C1], B, H, W);
    L(8, A[S_C1], A[S_D1A], H, W);
    L(9, A[S_D1A], A[S_OUT], H, W);
}

// backward of conv layer l: gout is dL/d(out) (masked in place to dL/d(pre)),
// weight/bias gradients into nn->grad, dL/d(in) into gin (null: not needed)
void layer_backward(m1_nn* nn, int l, const float* in, const float* out, float* gout, float* gin, int H, int W) {
    const int ci = kSpec[l].cin, co = kSpec[l].cout;
    const long long n_out = (long long)nn->B * H * W * co;
    if (kSpec[l].relu) k_relu_mask<<<grid_for(n_out), 256, 0, nn->s>>>(gout, out, n_out);
    k_conv3x3_dw<<<kDwGrid, 256, 0, nn->s>>>(in, ci, gout, co, nn->B, H, W, nn->dwpart);
    const long long nw = 9LL * ci * co;
    k_reduce_parts<<<grid_for(nw + co), 256, 0, nn->s>>>(nn->dwpart, nw + co, nw + co, kDwGrid, nn->grad + nn->woff[l]);
    // biases follow the weights of the same layer in the flat vector (boff = woff + nw)
    if (gin) {
        k_flip_weights<<<(int)((nw + 255) / 256), 256, 0, nn->s>>>(nn->theta_r + nn->woff[l], nn->wflip, ci, co);
        conv<float, float>(nn, gout, co, nn->wflip, nullptr, gin, ci, H, W, 0, nullptr);
    }
}

void backward(m1_nn* nn) {
    const int H = nn->H, W = nn->W, B = nn->B;
    float* const* A = nn->act.data();
    float* const* G = nn->gact.data();
    layer_backward(nn, 9, A[S_D1A], A[S_OUT], G[S_OUT], G[S_D1A], H, W);
    layer_backward(nn, 8, A[S_C1], A[S_D1A], G[S_D1A], G[S_C1], H, W);
    // split the concatenation: coarse part -> d2b output (upsample adjoint), skip -> e1b output
    cudaMemsetAsync(G[S_E1B], 0, sizeof(float) * slot_elems(nn, S_E1B), nn->s);
    k_up_cat_bwd<<<grid_for(slot_elems(nn, S_C1)), 256, 0, nn->s>>>(G[S_C1], G[S_D2B], 16, G[S_E1B], 16, B, H, W);
    layer_backward(nn, 7, A[S_D2A], A[S_D2B], G[S_D2B], G[S_D2A], H / 2, W / 2);
    layer_backward(nn, 6, A[S_C2], A[S_D2A], G[S_D2A], G[S_C2], H / 2, W / 2);
    cudaMemsetAsync(G[S_E2B], 0, sizeof(float) * slot_elems(nn, S_E2B), nn->s);
    k_up_cat_bwd<<<grid_for(slot_elems(nn, S_C2)), 256, 0, nn->s>>>(G[S_C2], G[S_E3B], 32, G[S_E2B], 32, B, H / 2, W / 2);
    layer_backward(nn, 5, A[S_E3A], A[S_E3B], G[S_E3B], G[S_E3A], H / 4, W / 4);
    layer_backward(nn, 4, A[S_P2], A[S_E3A], G[S_E3A], G[S_P2], H / 4, W / 4);
    k_pool2_bwd<<<grid_for(slot_elems(nn, S_E2B)), 256, 0, nn->s>>>(G[S_P2], G[S_E2B], B, H / 2, W / 2, 32, 1);
    layer_backward(nn, 3, A[S_E2A], A[S_E2B], G[S_E2B], G[S_E2A], H / 2, W / 2);
    layer_backward(nn, 2, A[S_P1], A[S_E2A], G[S_E2A], G[S_P1], H / 2, W / 2);
    k_pool2_bwd<<<grid_for(slot_elems(nn, S_E1B)), 256, 0, nn->s>>>(G[S_P1], G[S_E1B], B, H, W, 16, 1);
    layer_backward(nn, 1, A[S_E1A], A[S_E1B], G[S_E1B], G[S_E1A], H, W);
    layer_backward(nn, 0, A[S_IN], A[S_E1A], G[S_E1A], nullptr, H, W);
}

m1_status copy_in_f(m1_nn* nn, void* dst, const void* src, size_t bytes, m1_mem mem) {
    NCK(cudaMemcpyAsync(dst, src, bytes, mem == M1_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        nn->s));
    return M1_OK;
}
m1_status copy_out_f(m1_nn* nn, void* dst, const void* src, size_t bytes, m1_mem mem) {
    NCK(cudaMemcpyAsync(dst, src, bytes, mem == M1_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        nn->s));
    return M1_OK;
}
m1_status nn_sync(m1_nn* nn) {
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(nn->s));
    return M1_OK;
}

void refresh_rounded(m1_nn* nn) {
    k_round_bf16<<<grid_for(nn->nparams), 256, 0, nn->s>>>(nn->theta, nn->theta_r, nn->theta16, nn->nparams);
}

}  // namespace

__global__ void k_logsig(const double* __restrict__ sig, long long N, double dx, float* __restrict__ out) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
        out[p] = (float)((log10(fmax(sig[p] * dx, 1e-30)) - 0.5) / 2.5);
}

// training pair from FP64 vectors: x = [r/s, logsig] (4 ch), t = tt/s (3 ch), NHWC
__global__ void k_pack_pair(const double* __restrict__ r, const double* __restrict__ tt, long long N,
                            const float* __restrict__ logsig, double scale, float* __restrict__ x,
                            float* __restrict__ t) {
    const double inv = 1.0 / scale;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            x[4 * p + c] = (float)(r[(long long)c * N + p] * inv);
            t[3 * p + c] = (float)(tt[(long long)c * N + p] * inv);
        }
        x[4 * p + 3] = logsig[p];
    }
}

namespace m1 {
void launch_logsig(const double* sig, long long N, double dx, float* out, cudaStream_t s) {
    k_logsig<<<grid_for(N), 256, 0, s>>>(sig, N, dx, out);
}
void launch_pack_pair(const double* r, const double* tt, long long N, const float* logsig, double scale, float* x,
                      float* t, cudaStream_t s) {
    k_pack_pair<<<grid_for(N), 256, 0, s>>>(r, tt, N, logsig, scale, x, t);
}
// inference inside (F)GMRES: z += scale * N(pack(v / scale)) on the context's stream
m1_status nn_apply_add(m1_nn* nn, const float* v, long long N, const float* logsig, float scale, float* z,
                       cudaStream_t s) {
    if (!nn || (long long)nn->H * nn->W != N || nn->B != 1) return M1_ERR_ARG;
    cudaStream_t keep = nn->s;
    nn->s = s;
    __nv_bfloat16* const* A = nn->act16.data();
    k_pack_input<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(v, N, logsig, scale, nn->act16[S_IN]);
    forward<__nv_bfloat16>(nn, A);
    k_unpack_add<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(nn->act16[S_OUT], N, scale, z);
    nn->s = keep;
    return cudaGetLastError() == cudaSuccess ? M1_OK : M1_ERR_CUDA;
}
int nn_height(const m1_nn* nn) { return nn->H; }
int nn_width(const m1_nn* nn) { return nn->W; }
}  // namespace m1

extern "C" {

size_t m1_nn_num_params(void) {
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += 9 * (size_t)kSpec[l].cin * kSpec[l].cout + kSpec[l].cout;
    return n;
}

m1_status m1_nn_create(int H, int W, int batch, void* stream, m1_nn** out) {
    if (!out) return M1_ERR_ARG;
    *out = nullptr;
    if (H < 4 || W < 4 || H % 4 || W % 4 || batch < 1) return M1_ERR_ARG;
    m1_nn* nn = new (std::nothrow) m1_nn();
    if (!nn) return M1_ERR_NOMEM;
    nn->H = H;
    nn->W = W;
    nn->B = batch;
    nn->s = (cudaStream_t)stream;
    long long off = 0, maxw = 0;
    for (int l = 0; l < kLayers; ++l) {
        nn->woff[l] = off;
        off += 9LL * kSpec[l].cin * kSpec[l].cout;
        nn->boff[l] = off;
        off += kSpec[l].cout;
        maxw = std::max(maxw, 9LL * kSpec[l].cin * kSpec[l].cout + kSpec[l].cout);
    }
    nn->nparams = off;
    auto fail_free = [&](m1_status st) {
        m1_nn_destroy(nn);
        return st;
    };
#define NAL(p, cnt)                                                                            \
    do {                                                                                       \
        if (cudaMalloc((void**)&(p), sizeof(*(p)) * (size_t)(cnt)) != cudaSuccess) return fail_free(M1_ERR_NOMEM); \
    } while (0)
    NAL(nn->theta, off);
    NAL(nn->theta_r, off);
    NAL(nn->theta16, off);
    NAL(nn->grad, off);
    NAL(nn->adam_m, off);
    NAL(nn->adam_v, off);
    NAL(nn->wflip, maxw);
    nn->dwpart_size = (long long)kDwGrid * maxw;
    NAL(nn->dwpart, nn->dwpart_size);
    NAL(nn->loss_dev, batch);
    nn->act.assign(S_COUNT, nullptr);
    nn->act16.assign(S_COUNT, nullptr);
    nn->gact.assign(S_COUNT, nullptr);
    for (int sl = 0; sl < S_COUNT; ++sl) {
        NAL(nn->act[sl], slot_elems(nn, sl));
        NAL(nn->act16[sl], slot_elems(nn, sl));
        NAL(nn->gact[sl], slot_elems(nn, sl));
    }
#undef NAL
    if (cudaMallocHost((void**)&nn->loss_host, sizeof(double) * batch) != cudaSuccess) return fail_free(M1_ERR_NOMEM);
    if (cudaMemsetAsync(nn->theta, 0, sizeof(float) * off, nn->s) != cudaSuccess ||
        cudaMemsetAsync(nn->adam_m, 0, sizeof(float) * off, nn->s) != cudaSuccess ||
        cudaMemsetAsync(nn->adam_v, 0, sizeof(float) * off, nn->s) != cudaSuccess)
        return fail_free(M1_ERR_CUDA);
    refresh_rounded(nn);
    if (cudaStreamSynchronize(nn->s) != cudaSuccess) return fail_free(M1_ERR_CUDA);
    *out = nn;
    return M1_OK;
}

m1_status m1_nn_destroy(m1_nn* nn) {
    if (!nn) return M1_OK;
    cudaStreamSynchronize(nn->s);
    void* p[] = {nn->theta, nn->theta_r, nn->theta16, nn->grad, nn->adam_m, nn->adam_v, nn->wflip, nn->dwpart,
                 nn->loss_dev};
    for (void* q : p)
        if (q) cudaFree(q);
    for (auto* q : nn->act)
        if (q) cudaFree(q);
    for (auto* q : nn->act16)
        if (q) cudaFree(q);
    for (auto* q : nn->gact)
        if (q) cudaFree(q);
    if (nn->loss_host) cudaFreeHost(nn->loss_host);
    delete nn;
    return M1_OK;
}

m1_status m1_nn_set_params(m1_nn* nn, const float* theta, m1_mem mem) {
    if (!nn || !theta) return M1_ERR_ARG;
    m1_status st = copy_in_f(nn, nn->theta, theta, sizeof(float) * nn->nparams, mem);
    if (st != M1_OK) return st;
    NCK(cudaMemsetAsync(nn->adam_m, 0, sizeof(float) * nn->nparams, nn->s));
    NCK(cudaMemsetAsync(nn->adam_v, 0, sizeof(float) * nn->nparams, nn->s));
    nn->adam_t = 0;
    refresh_rounded(nn);
    return nn_sync(nn);
}

m1_status m1_nn_get_params(const m1_nn* cnn, float* theta, m1_mem mem) {
    m1_nn* nn = const_cast<m1_nn*>(cnn);
    if (!nn || !theta) return M1_ERR_ARG;
    m1_status st = copy_out_f(nn, theta, nn->theta, sizeof(float) * nn->nparams, mem);
    if (st != M1_OK) return st;
    return nn_sync(nn);
}

m1_status m1_nn_forward(m1_nn* nn, const float* x, float* y, int bf16, m1_mem mem) {
    if (!nn || !x || !y) return M1_ERR_ARG;
    const long long nin = slot_elems(nn, S_IN), nout = slot_elems(nn, S_OUT);
    m1_status st = copy_in_f(nn, nn->act[S_IN], x, sizeof(float) * nin, mem);
    if (st != M1_OK) return st;
    if (bf16) {
        k_round_bf16<<<grid_for(nin), 256, 0, nn->s>>>(nn->act[S_IN], nn->gact[S_IN], nn->act16[S_IN], nin);
        forward<__nv_bfloat16>(nn, nn->act16.data());
        k_widen<<<grid_for(nout), 256, 0, nn->s>>>(nn->act16[S_OUT], nn->act[S_OUT], nout);
    } else {
        forward<float>(nn, nn->act.data());
    }
    st = copy_out_f(nn, y, nn->act[S_OUT], sizeof(float) * nout, mem);
    if (st != M1_OK) return st;
    return nn_sync(nn);
}

m1_status m1_nn_loss_grad(m1_nn* nn, const float* x, const float* t, double* loss, float* grad, m1_mem mem) {
    if (!nn || !x || !t) return M1_ERR_ARG;
    const long long nin = slot_elems(nn, S_IN), nout = slot_elems(nn, S_OUT);
    m1_status st = copy_in_f(nn, nn->act[S_IN], x, sizeof(float) * nin, mem);
    if (st != M1_OK) return st;
    st = copy_in_f(nn, nn->act[S_T], t, sizeof(float) * nout, mem);
    if (st != M1_OK) return st;
    forward<float>(nn, nn->act.data());
    k_loss<<<nn->B, 256, 0, nn->s>>>(nn->act[S_OUT], nn->act[S_T], nout / nn->B, nn->B, nn->gact[S_OUT], nn->loss_dev);
    backward(nn);
    NCK(cudaMemcpyAsync(nn->loss_host, nn->loss_dev, sizeof(double) * nn->B, cudaMemcpyDeviceToHost, nn->s));
    if (grad) {
        st = copy_out_f(nn, grad, nn->grad, sizeof(float) * nn->nparams, mem);
        if (st != M1_OK) return st;
    }
    st = nn_sync(nn);
    if (st != M1_OK) return st;
    if (loss) {
        double L = 0.0;
        for (int b = 0; b < nn->B; ++b) L += nn->loss_host[b];
        *loss = L;
    }
    return M1_OK;
}

m1_status m1_nn_train(m1_nn* nn, const float* X, const float* T, int npairs, const m1_train_opts* o,
                      m1_train_info* info, m1_mem mem) {
    if (!nn || !X || !T || !o || npairs < nn->B) return M1_ERR_ARG;
    const long long per_in = slot_elems(nn, S_IN) / nn->B, per_out = slot_elems(nn, S_OUT) / nn->B;
    const int steps_per_epoch = npairs / nn->B;
    double first = -1.0, last = 0.0;
    unsigned long long seed = o->seed ? o->seed : 1ull;
    std::vector<int> order(npairs);
    for (int i = 0; i < npairs; ++i) order[i] = i;
    int step = 0;
    for (int ep = 0; ep < o->epochs; ++ep) {
        // SplitMix64-driven Fisher-Yates shuffle of the pair order (host)
        for (int i = npairs - 1; i > 0; --i) {
            seed += 0x9E3779B97F4A7C15ull;
            unsigned long long z = seed;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const int jx = (int)(z % (unsigned long long)(i + 1));
            std::swap(order[i], order[jx]);
        }
        double ep_loss = 0.0;
        for (int sidx = 0; sidx < steps_per_epoch; ++sidx, ++step) {
            for (int b = 0; b < nn->B; ++b) {
                const int pidx = order[sidx * nn->B + b];
                m1_status st = copy_in_f(nn, nn->act[S_IN] + b * per_in, X + (long long)pidx * per_in,
                                         sizeof(float) * per_in, mem);
                if (st != M1_OK) return st;
                st = copy_in_f(nn, nn->act[S_T] + b * per_out, T + (long long)pidx * per_out, sizeof(float) * per_out,
                               mem);
                if (st != M1_OK) return st;
            }
            forward<float>(nn, nn->act.data());
            k_loss<<<nn->B, 256, 0, nn->s>>>(nn->act[S_OUT], nn->act[S_T], per_out, nn->B, nn->gact[S_OUT],
                                             nn->loss_dev);
            backward(nn);
            nn->adam_t += 1;
            const float lr = (float)(o->lr * (o->lr_decay > 0.0 ? pow(o->lr_decay, (double)ep) : 1.0));
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - powf(b1, (float)nn->adam_t), c2 = 1.f - powf(b2, (float)nn->adam_t);
            k_adam<<<grid_for(nn->nparams), 256, 0, nn->s>>>(nn->theta, nn->theta16, nn->grad, nn->adam_m, nn->adam_v,
                                                             nn->nparams, lr, b1, b2, 1e-8f, c1, c2);
            refresh_rounded(nn);
            NCK(cudaMemcpyAsync(nn->loss_host, nn->loss_dev, sizeof(double) * nn->B, cudaMemcpyDeviceToHost, nn->s));
            m1_status st = nn_sync(nn);
            if (st != M1_OK) return st;
            double L = 0.0;
            for (int b = 0; b < nn->B; ++b) L += nn->loss_host[b];
            if (!(L == L)) return nn_fail(nn, M1_ERR_NONFINITE, "non-finite training loss");
            if (first < 0.0) first = L;
            ep_loss += L;
        }
        last = ep_loss / std::max(steps_per_epoch, 1);
    }
    if (info) {
        info->steps = step;
        info->first_loss = first;
        info->final_loss = last;
    }
    return M1_OK;
}

const char* m1_nn_last_error(const m1_nn* nn) { return nn ? nn->err.c_str() : "null network"; }

}  // extern "C"
