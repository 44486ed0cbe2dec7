// m1_unet.cu — the learned preconditioner network: a 3-level 2D U-Net
// (63,875 parameters), its forward and backward kernels, loss, Adam, and the
// packing between Krylov vectors and network tensors.
//
// Inputs (7 channels): the Krylov vector (E, F_x, F_y) scaled by s, the
// normalised log opacity, and the linearisation state of the Jacobian: the
// reduced flux f = F / (cE) (two channels, clamped to [-1, 1]) and the
// normalised log energy (log10 E + 3) / 3.
//
// Layers (all 3x3 convolutions, stride 1, zero padding, weights W[ky][kx][ci][co]):
//   e1a 7->16, e1b 16->16 | pool | e2a 16->32, e2b 32->32 | pool |
//   e3a 32->32, e3b 32->32 | up, cat(e2b) | d2a 64->32, d2b 32->16 | up, cat(e1b) |
//   d1a 32->16, d1b 16->3 (linear); ReLU after every other convolution.
// Tensors are NHWC. Activations are stored in FP32 for training and in BF16
// for inference; weights are FP32 masters with a BF16 copy (the forward pass
// always uses BF16-rounded weights); every product is accumulated in FP32.
//
// Two convolution kernels:
//   - k_conv3x3_tc, the default: an implicit GEMM on the tensor cores
//     (mma.sync m16n8k16, BF16 operands, FP32 accumulation). A CTA stages a
//     16 x 16-pixel tile plus its halo (activations rounded to BF16) and the
//     layer's weights in shared memory; each warp multiplies two 16-pixel rows
//     (M) by all output channels (N), K = 9 taps x input channels, A fragments
//     by ldmatrix from a padded pixel stride (no bank conflicts).
//   - k_conv3x3, FP32 on the CUDA cores (FP32 activations and products): the
//     precise path for gradient checks (m1_nn_set_tensor_cores(nn, 0)).
// The backward data pass is the same convolution on the flipped, transposed
// weights; the weight gradient is a per-CTA partial sum over pixel tiles on
// the CUDA cores, reduced in a fixed order.
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
constexpr int kCin0 = 7;  // input channels
const LayerSpec kSpec[kLayers] = {
    {"e1a", kCin0, 16, true},  {"e1b", 16, 16, true}, {"e2a", 16, 32, true}, {"e2b", 32, 32, true},
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

// ------------------------------------------------------------------ tensor-core convolution
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                               unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                            const void* smem_ptr) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem_ptr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// Shared memory of k_conv3x3_tc<CINP, COUTP>: the 18 x 18 halo tile with a pixel
// stride of CINP + 8 BF16 (16-byte rows for ldmatrix, consecutive pixels 16
// bytes apart modulo 128: conflict-free), then the weights as [tap][co][ci] with
// the same ci stride.
__host__ __device__ constexpr int tc_smem_bytes(int cinp, int coutp) {
    return (18 * 18 * (cinp + 8) + 9 * coutp * (cinp + 8)) * 2;
}

// y[b,i,j,co] = bias[co] + sum x[b,i+dy-1,j+dx-1,ci] w[dy][dx][ci][co] with BF16
// operands and FP32 accumulation; optional ReLU and multiplicative mask (mask > 0).
// CINP >= cin and COUTP >= cout are the padded GEMM sizes (multiples of 16 and 8).
// Grid: (ceil(W/16), ceil(H/16), B), 256 threads; warp w owns tile rows 2w, 2w+1.
template <int CINP, int COUTP, class Tin, class Tout>
__global__ void __launch_bounds__(256) k_conv3x3_tc(const Tin* __restrict__ x, int cin,
                                                    const __nv_bfloat16* __restrict__ w16,
                                                    const float* __restrict__ bias, Tout* __restrict__ y, int cout,
                                                    int H, int W, int relu, const float* __restrict__ mask) {
    static_assert(CINP % 16 == 0 && COUTP % 8 == 0, "GEMM tile sizes");
    constexpr int XS = CINP + 8;
    constexpr int NT = COUTP / 8;
    extern __shared__ __align__(16) unsigned char tc_smem[];
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(tc_smem);
    __nv_bfloat16* ws = xs + 18 * 18 * XS;
    const int j0 = blockIdx.x * 16, i0 = blockIdx.y * 16, b = blockIdx.z;
    const long long img = (long long)b * H * W;
    for (int t = threadIdx.x; t < 18 * 18 * CINP; t += 256) {
        const int c = t % CINP, px = (t / CINP) % 18, py = t / (CINP * 18);
        const int gi = i0 + py - 1, gj = j0 + px - 1;
        float v = 0.f;
        if (c < cin && gi >= 0 && gi < H && gj >= 0 && gj < W) v = ld(x, (img + (long long)gi * W + gj) * cin + c);
        xs[(py * 18 + px) * XS + c] = __float2bfloat16(v);
    }
    for (int t = threadIdx.x; t < 9 * COUTP * CINP; t += 256) {
        const int ci = t % CINP, co = (t / CINP) % COUTP, tap = t / (CINP * COUTP);
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (ci < cin && co < cout) v = w16[((long long)tap * cin + ci) * cout + co];
        ws[(tap * COUTP + co) * XS + ci] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int mi = lane >> 3, rr = lane & 7;  // ldmatrix: this lane's matrix and row
    const int apx = ((mi & 1) ? 8 : 0) + rr, ach = (mi >> 1) ? 8 : 0;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
        for (int kc = 0; kc < CINP / 16; ++kc) {
            unsigned bfr[NT][2];
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const __nv_bfloat16* wr = ws + (tap * COUTP + n * 8 + g) * XS + kc * 16 + 2 * tq;
                bfr[n][0] = *reinterpret_cast<const unsigned*>(wr);
                bfr[n][1] = *reinterpret_cast<const unsigned*>(wr + 8);
            }
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int row = warp * 2 + m;
                unsigned a0, a1, a2, a3;
                ldmatrix_x4(a0, a1, a2, a3, xs + ((row + dy) * 18 + apx + dx) * XS + kc * 16 + ach);
#pragma unroll
                for (int n = 0; n < NT; ++n) mma_bf16_16816(acc[m][n], a0, a1, a2, a3, bfr[n][0], bfr[n][1]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int i = i0 + warp * 2 + m;
        if (i >= H) continue;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // c0,c1: pixel g; c2,c3: pixel g + 8
                const int j = j0 + g + 8 * h;
                if (j >= W) continue;
                const long long o = (img + (long long)i * W + j) * cout;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int co = n * 8 + 2 * tq + e;
                    if (co < cout) {
                        float v = acc[m][n][2 * h + e] + (bias ? bias[co] : 0.f);
                        if (relu) v = fmaxf(v, 0.f);
                        if (mask) v = mask[o + co] > 0.f ? v : 0.f;
                        st(y, o + co, v);
                    }
                }
            }
        }
    }
}

// BF16 flipped weights for the backward data pass on the tensor cores
__global__ void k_flip_weights16(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int cin,
                                 int cout) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 9 * cin * cout) return;
    const int co = t % cout, ci = (t / cout) % cin, tap = t / (cout * cin);
    wt[((long long)(8 - tap) * cout + co) * cin + ci] = w[t];
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

// mean squared error per output element, L = (1/B) sum_b ||y_b - t_b||^2 / per
// (per = H W 3; the pairs' inputs have unit RMS in their residual channels),
// and its gradient dy = 2 (y - t) / per / B
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, long long per, int B,
                       float* __restrict__ gy, double* __restrict__ loss) {
    __shared__ double red[8];
    const int b = blockIdx.x;
    double num = 0.0;
    for (long long k = threadIdx.x; k < per; k += blockDim.x) {
        const double d = (double)y[b * per + k] - (double)t[b * per + k];
        num += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = num;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += red[q];
        loss[b] = a / (double)per / B;
    }
    const float sc = (float)(2.0 / (double)per / B);
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

// the scale of a vector whose squared norm the device holds: its RMS sqrt(n2 / n),
// or 1 for a zero vector (the network's input is then zero as well)
__device__ __forceinline__ float rms_scale(const double* n2, double inv_n) {
    const double q = n2[0] * inv_n;
    return q > 0.0 ? (float)sqrt(q) : 1.f;
}

// network input from a component-major Krylov vector v (E, Fx, Fy; N = H*W
// each): x = [v / s, static] in NHWC (7 channels), s = scale (or, with n2 set,
// the RMS of v from its squared norm n2[0] over n entries), static the four
// planes of the opacity and state channels (k_nn_static)
template <class T>
__global__ void k_pack_input(const float* __restrict__ v, long long N, const float* __restrict__ stat, float scale,
                             const double* __restrict__ n2, double inv_n, T* __restrict__ x) {
    const float inv = 1.f / (n2 ? rms_scale(n2, inv_n) : scale);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        st(x, kCin0 * p + 0, v[p] * inv);
        st(x, kCin0 * p + 1, v[N + p] * inv);
        st(x, kCin0 * p + 2, v[2 * N + p] * inv);
#pragma unroll
        for (int c = 0; c < 4; ++c) st(x, kCin0 * p + 3 + c, stat[c * N + p]);
    }
}

// z (component-major) += scale * (y - y0) (NHWC, 3 channels; y0 may be null;
// with n2 set the scale is the RMS of k_pack_input's vector)
template <class T>
__global__ void k_unpack_add(const T* __restrict__ y, const float* __restrict__ y0, long long N, float scale,
                             const double* __restrict__ n2, double inv_n, float* __restrict__ z) {
    if (n2) scale = rms_scale(n2, inv_n);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = ld(y, 3 * p + c) - (y0 ? y0[3 * p + c] : 0.f);
            z[c * N + p] += scale * v;
        }
    }
}

// y0 = the network's output (FP32, NHWC) for a zero residual: the part of N
// that does not depend on the Krylov vector
template <class T>
__global__ void k_copy_out(const T* __restrict__ y, long long n, float* __restrict__ y0) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        y0[k] = ld(y, k);
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
    __nv_bfloat16* wflip16 = nullptr;  // the same in BF16 (tensor-core backward data pass)
    int tc = 1;                    // convolutions on the tensor cores (1) or FP32 CUDA cores (0)
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
        case S_IN: return f * kCin0;
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

template <int CINP, int COUTP, class Tin, class Tout>
void conv_tc_launch(m1_nn* nn, const Tin* x, int cin, const __nv_bfloat16* w16, const float* b, Tout* y, int cout,
                    int H, int W, int relu, const float* mask) {
    constexpr int bytes = tc_smem_bytes(CINP, COUTP);
    static bool attr_set = false;  // per instantiation; the attribute is a property of the function
    if (!attr_set) {
        cudaFuncSetAttribute(k_conv3x3_tc<CINP, COUTP, Tin, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        attr_set = true;
    }
    dim3 grid((W + 15) / 16, (H + 15) / 16, nn->B);
    k_conv3x3_tc<CINP, COUTP, Tin, Tout><<<grid, 256, bytes, nn->s>>>(x, cin, w16, b, y, cout, H, W, relu, mask);
}

// the tensor-core convolution with the smallest GEMM tile that holds (cin, cout)
template <class Tin, class Tout>
void conv_tc(m1_nn* nn, const Tin* x, int cin, const __nv_bfloat16* w16, const float* b, Tout* y, int cout, int H,
             int W, int relu, const float* mask) {
#define TC_CASE(CI, CO)                                                                     \
    if (cin <= CI && cout <= CO) {                                                         \
        conv_tc_launch<CI, CO, Tin, Tout>(nn, x, cin, w16, b, y, cout, H, W, relu, mask); \
        return;                                                                             \
    }
    TC_CASE(16, 8)
    TC_CASE(16, 16)
    TC_CASE(16, 32)
    TC_CASE(32, 16)
    TC_CASE(32, 32)
    TC_CASE(32, 64)
    TC_CASE(64, 32)
#undef TC_CASE
}

// forward pass; T = float (training, keeps every activation) or bf16 (inference)
template <class T>
void forward(m1_nn* nn, T* const* A) {
    const int H = nn->H, W = nn->W, B = nn->B;
    const float* th = nn->theta_r;
    auto L = [&](int l, const T* in, T* out, int H_, int W_) {
        if (nn->tc)
            conv_tc<T, T>(nn, in, kSpec[l].cin, nn->theta16 + nn->woff[l], th + nn->boff[l], out, kSpec[l].cout, H_,
                          W_, kSpec[l].relu ? 1 : 0, nullptr);
        else
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
        if (nn->tc) {
            k_flip_weights16<<<(int)((nw + 255) / 256), 256, 0, nn->s>>>(nn->theta16 + nn->woff[l], nn->wflip16, ci,
                                                                          co);
            conv_tc<float, float>(nn, gout, co, nn->wflip16, nullptr, gin, ci, H, W, 0, nullptr);
        } else {
            k_flip_weights<<<(int)((nw + 255) / 256), 256, 0, nn->s>>>(nn->theta_r + nn->woff[l], nn->wflip, ci, co);
            conv<float, float>(nn, gout, co, nn->wflip, nullptr, gin, ci, H, W, 0, nullptr);
        }
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

// The four input planes that do not depend on the Krylov vector, from the
// linearisation state U (E, F_x, F_y component-major, FP64 or FP32):
// stat[0] = logsig, stat[1..2] = F / (c max(E, 1e-30)) clamped to [-1, 1],
// stat[3] = (log10 max(E, 1e-30) + 3) / 3.
template <class R>
__global__ void k_nn_static(const R* __restrict__ U, long long N, double c, const float* __restrict__ logsig,
                            float* __restrict__ stat) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const double E = fmax((double)U[p], 1e-30);
        const double inv = 1.0 / (c * E);
        stat[p] = logsig[p];
        stat[N + p] = (float)fmin(fmax((double)U[N + p] * inv, -1.0), 1.0);
        stat[2 * N + p] = (float)fmin(fmax((double)U[2 * N + p] * inv, -1.0), 1.0);
        stat[3 * N + p] = (float)((log10(E) + 3.0) / 3.0);
    }
}

// training pair from FP64 vectors: x = [r/s, static] (7 ch), t = tt/s (3 ch), NHWC
__global__ void k_pack_pair(const double* __restrict__ r, const double* __restrict__ tt, long long N,
                            const float* __restrict__ stat, double scale, float* __restrict__ x,
                            float* __restrict__ t) {
    const double inv = 1.0 / scale;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            x[kCin0 * p + c] = (float)(r[(long long)c * N + p] * inv);
            t[3 * p + c] = (float)(tt[(long long)c * N + p] * inv);
        }
        for (int c = 0; c < 4; ++c) x[kCin0 * p + 3 + c] = stat[(long long)c * N + p];
    }
}

namespace m1 {
void launch_logsig(const double* sig, long long N, double dx, float* out, cudaStream_t s) {
    k_logsig<<<grid_for(N), 256, 0, s>>>(sig, N, dx, out);
}
void launch_pack_pair(const double* r, const double* tt, long long N, const float* stat, double scale, float* x,
                      float* t, cudaStream_t s) {
    k_pack_pair<<<grid_for(N), 256, 0, s>>>(r, tt, N, stat, scale, x, t);
}
void launch_nn_static_f64(const double* U, long long N, double c, const float* logsig, float* stat, cudaStream_t s) {
    k_nn_static<double><<<grid_for(N), 256, 0, s>>>(U, N, c, logsig, stat);
}
void launch_nn_static_f32(const float* U, long long N, double c, const float* logsig, float* stat, cudaStream_t s) {
    k_nn_static<float><<<grid_for(N), 256, 0, s>>>(U, N, c, logsig, stat);
}
// inference inside (F)GMRES: z += scale * (N(pack(v / scale, static)) - y0) on the
// context's stream, y0 from nn_null_response (null: not subtracted)
m1_status nn_apply_add(m1_nn* nn, const float* v, long long N, const float* stat, const float* y0, float scale,
                       float* z, cudaStream_t s) {
    if (!nn || (long long)nn->H * nn->W != N || nn->B != 1) return M1_ERR_ARG;
    cudaStream_t keep = nn->s;
    nn->s = s;
    __nv_bfloat16* const* A = nn->act16.data();
    k_pack_input<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(v, N, stat, scale, nullptr, 0.0, nn->act16[S_IN]);
    forward<__nv_bfloat16>(nn, A);
    k_unpack_add<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(nn->act16[S_OUT], y0, N, scale, nullptr, 0.0, z);
    nn->s = keep;
    return cudaGetLastError() == cudaSuccess ? M1_OK : M1_ERR_CUDA;
}
// the same with the scale taken on the device: the RMS of v from its squared norm n2[0] (3N entries)
m1_status nn_apply_add_rms(m1_nn* nn, const float* v, long long N, const float* stat, const float* y0,
                           const double* n2, float* z, cudaStream_t s) {
    if (!nn || (long long)nn->H * nn->W != N || nn->B != 1 || !n2) return M1_ERR_ARG;
    cudaStream_t keep = nn->s;
    nn->s = s;
    const double inv_n = 1.0 / (3.0 * (double)N);
    __nv_bfloat16* const* A = nn->act16.data();
    k_pack_input<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(v, N, stat, 1.f, n2, inv_n, nn->act16[S_IN]);
    forward<__nv_bfloat16>(nn, A);
    k_unpack_add<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(nn->act16[S_OUT], y0, N, 1.f, n2, inv_n, z);
    nn->s = keep;
    return cudaGetLastError() == cudaSuccess ? M1_OK : M1_ERR_CUDA;
}
// y0 (3N floats, NHWC) = N(pack(0, static)): the network's response to a zero
// residual at this state, subtracted in every application so that the learned
// correction of a zero vector is zero (flexible GMRES would otherwise see the
// same field added to every preconditioned vector)
m1_status nn_null_response(m1_nn* nn, const float* zero3, long long N, const float* stat, float* y0, cudaStream_t s) {
    if (!nn || (long long)nn->H * nn->W != N || nn->B != 1) return M1_ERR_ARG;
    cudaStream_t keep = nn->s;
    nn->s = s;
    k_pack_input<__nv_bfloat16><<<grid_for(N), 256, 0, s>>>(zero3, N, stat, 1.f, nullptr, 0.0, nn->act16[S_IN]);
    forward<__nv_bfloat16>(nn, nn->act16.data());
    k_copy_out<__nv_bfloat16><<<grid_for(3 * N), 256, 0, s>>>(nn->act16[S_OUT], 3 * N, y0);
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
    NAL(nn->wflip16, maxw);
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
    void* p[] = {nn->theta, nn->theta_r, nn->theta16, nn->grad, nn->adam_m, nn->adam_v, nn->wflip, nn->wflip16,
                 nn->dwpart, nn->loss_dev};
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

m1_status m1_nn_set_tensor_cores(m1_nn* nn, int on) {
    if (!nn) return M1_ERR_ARG;
    nn->tc = on ? 1 : 0;
    return M1_OK;
}

const char* m1_nn_last_error(const m1_nn* nn) { return nn ? nn->err.c_str() : "null network"; }

}  // extern "C"
