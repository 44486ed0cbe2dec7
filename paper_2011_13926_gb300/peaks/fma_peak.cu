// fma_peak.cu — FP64 and FP32 FMA throughput probe (the ALU rooflines of the
// FP64 stencil kernels). Eight independent FMA chains per thread, 16 blocks per
// SM x 152 SMs, timed with CUDA events. Build: nvcc -gencode
// arch=compute_103a,code=sm_103a -O3 -o fma_peak fma_peak.cu
#include <cstdio>
#include <cuda_runtime.h>
template <class T> __global__ void k(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <class T> double run(const char* name, int iters) {
  int blocks = 152 * 16, threads = 256;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  k<T><<<blocks, threads>>>(out, 16, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  k<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8 * (double)iters * blocks * threads;
  printf("%s: %.3f ms, %.2f TFLOP/s (err %s)\n", name, ms, flops / ms / 1e9, cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
  return flops / ms / 1e9;
}
int main() { run<double>("fp64_fma", 4096); run<float>("fp32_fma", 65536); return 0; }
