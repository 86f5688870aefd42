// Standalone probe of the FP64 and FP32 FMA throughput of the GPU (not part
// of the library): 8 independent FMA chains per thread, 8 CTAs of 256 threads
// per SM, timed with CUDA events.  These figures are the arithmetic peaks the
// benchmark reports FP64-bound kernels against.
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a -o alu_peak_probe alu_peak_probe.cu
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T> void run(const char* name, int iters) {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  int blocks = p.multiProcessorCount * 8, threads = 256;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  fma_loop<T><<<blocks, threads>>>(out, 10, (T)0.999, (T)1e-3);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0);
  fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-3);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  printf("%s: %.3f ms  %.2f TFLOP/s  err=%s\n", name, ms, flops / ms / 1e9, cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("name=%s sm=%d.%d SMs=%d L2=%d B smemPerBlockOptin=%zu regsPerSM=%d busw=%d\n",
    p.name, p.major, p.minor, p.multiProcessorCount, p.l2CacheSize, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor, p.memoryBusWidth);
  run<double>("fp64", 200);
  run<double>("fp64", 400);
  run<float>("fp32", 4000);
  run<float>("fp32", 8000);
  return 0;
}
