// Arithmetic-pipe probe: FP64 FMA, FP32 FMA and FP64 mma.sync (DMMA) throughput on GPU 0.
// Build: python -m paper_2607_00199_b300.build --probe ; run: _build/peak_probe
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<typename T>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void dmma_kernel(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 0.5;
  double c[4][2];
  for (int k = 0; k < 4; ++k) { c[k][0] = 0; c[k][1] = 0; }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(a), "d"(b));
    }
  }
  double s = 0; for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void tf32_mma_kernel(float *out, int iters) {
  unsigned a0 = 0x3f800000u + threadIdx.x, a1 = a0, a2 = a0, a3 = a0, b0 = 0x3f000000u, b1 = b0;
  float c[4][4];
  for (int k = 0; k < 4; ++k) for (int j = 0; j < 4; ++j) c[k][j] = 0.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                     : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  float s = 0; for (int k = 0; k < 4; ++k) for (int j = 0; j < 4; ++j) s += c[k][j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void bf16_mma_kernel(float *out, int iters) {
  unsigned a0 = 0x3f803f80u + threadIdx.x, a1 = a0, a2 = a0, a3 = a0, b0 = 0x3f003f00u, b1 = b0;
  float c[4][4];
  for (int k = 0; k < 4; ++k) for (int j = 0; j < 4; ++j) c[k][j] = 0.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                     : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  float s = 0; for (int k = 0; k < 4; ++k) for (int j = 0; j < 4; ++j) s += c[k][j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  printf("device %s SMs %d cc %d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
  int nsm = p.multiProcessorCount;
  double* d; CK(cudaMalloc(&d, sizeof(double) * nsm * 64 * 1024));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int blocksPerSM : {4, 8}) {
    int threads = 256, blocks = nsm * blocksPerSM, iters = 2000;
    fma_kernel<double><<<blocks, threads>>>(d, 10, 1.0000001, 1e-9);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    fma_kernel<double><<<blocks, threads>>>(d, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    printf("fp64 fma: blocks/SM %d  %.3f ms  %.3f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
  }
  {
    int threads = 256, blocks = nsm * 8, iters = 20000;
    float* f = (float*)d;
    fma_kernel<float><<<blocks, threads>>>(f, 10, 1.0000001f, 1e-9f);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    fma_kernel<float><<<blocks, threads>>>(f, iters, 1.0000001f, 1e-9f);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    printf("fp32 fma: %.3f ms  %.3f TFLOP/s\n", ms, flops / ms / 1e9);
  }
  for (int blocksPerSM : {4, 8}) {
    int threads = 128, blocks = nsm * blocksPerSM, iters = 200;
    dmma_kernel<<<blocks, threads>>>(d, 2);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    dmma_kernel<<<blocks, threads>>>(d, iters);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * 8 * 4 * 16.0 * iters * blocks * (threads / 32);
    printf("dmma m8n8k4: blocks/SM %d %.3f ms  %.3f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
  }
  for (int blocksPerSM : {4, 8}) {
    int threads = 128, blocks = nsm * blocksPerSM, iters = 2000;
    tf32_mma_kernel<<<blocks, threads>>>((float *)d, 2);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    tf32_mma_kernel<<<blocks, threads>>>((float *)d, iters);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 16 * 8 * 8 * 16.0 * iters * blocks * (threads / 32);
    printf("mma.sync tf32 m16n8k8: blocks/SM %d %.3f ms  %.1f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
  }
  for (int blocksPerSM : {4, 8}) {
    int threads = 128, blocks = nsm * blocksPerSM, iters = 2000;
    bf16_mma_kernel<<<blocks, threads>>>((float *)d, 2);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    bf16_mma_kernel<<<blocks, threads>>>((float *)d, iters);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 16 * 8 * 16 * 16.0 * iters * blocks * (threads / 32);
    printf("mma.sync bf16 m16n8k16: blocks/SM %d %.3f ms  %.1f TFLOP/s\n", blocksPerSM, ms, flops / ms / 1e9);
  }
  CK(cudaFree(d));
  return 0;
}
