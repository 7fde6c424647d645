// unit_rates.cu -- per-SM throughput of the instruction classes the force
// path's arithmetic design depends on, measured on the GPU at hand: FP32 FMA,
// FP64 add and FMA, int->float and float->double conversions, MUFU reciprocal,
// warp shuffles, and scattered FP64 / FP32 atomic adds to global memory.
// Built and run by unit_rates.py; not part of the library.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s line %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)
constexpr int IT = 2048;
__global__ void k_ffma(float* out, float a, float b) {
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < IT; ++i) {
    x0 = fmaf(x0,a,b); x1 = fmaf(x1,a,b); x2 = fmaf(x2,a,b); x3 = fmaf(x3,a,b);
    x4 = fmaf(x4,a,b); x5 = fmaf(x5,a,b); x6 = fmaf(x6,a,b); x7 = fmaf(x7,a,b);
  }
  float s = x0+x1+x2+x3+x4+x5+x6+x7; if (s == 12345.f) out[threadIdx.x] = s;
}
__global__ void k_dadd(double* out, double a) {
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < IT/8; ++i) {
    x0 += a; x1 += a; x2 += a; x3 += a; x4 += a; x5 += a; x6 += a; x7 += a;
  }
  double s = x0+x1+x2+x3+x4+x5+x6+x7; if (s == 12345.) out[threadIdx.x] = s;
}
__global__ void k_dfma(double* out, double a, double b) {
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < IT/8; ++i) {
    x0 = fma(x0,a,b); x1 = fma(x1,a,b); x2 = fma(x2,a,b); x3 = fma(x3,a,b);
    x4 = fma(x4,a,b); x5 = fma(x5,a,b); x6 = fma(x6,a,b); x7 = fma(x7,a,b);
  }
  double s = x0+x1+x2+x3+x4+x5+x6+x7; if (s == 12345.) out[threadIdx.x] = s;
}
__global__ void k_i2f(float* out, int a) {
  int i0 = threadIdx.x * 7919; float s0=0, s1=0, s2=0, s3=0;
  for (int i = 0; i < IT; ++i) {
    int v = i0 + i * a;
    s0 += __int2float_rn(v); s1 += __int2float_rn(v ^ 0x5555); s2 += __int2float_rn(v + 77777); s3 += __int2float_rn(v * 3);
  }
  float s = s0+s1+s2+s3; if (s == 12345.f) out[threadIdx.x] = s;
}
__global__ void k_rcp(float* out, float a) {
  float x0=threadIdx.x+1.f, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i = 0; i < IT; ++i) {
    x0 = __fdividef(1.f, x0) + a; x1 = __fdividef(1.f, x1) + a; x2 = __fdividef(1.f, x2) + a; x3 = __fdividef(1.f, x3) + a;
  }
  float s = x0+x1+x2+x3; if (s == 12345.f) out[threadIdx.x] = s;
}
__global__ void k_f2d(double* out, float a) {
  float x = threadIdx.x; double s0=0, s1=0, s2=0, s3=0;
  for (int i = 0; i < IT/8; ++i) {
    x += a;
    s0 = (double)x; s1 = (double)(x+1.f); s2 = (double)(x+2.f); s3 = (double)(x+3.f);
    if (s0 + s1 + s2 + s3 == 12345.) out[0] = 1;
  }
}
__global__ void k_shfl(float* out, float a) {
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i = 0; i < IT; ++i) {
    x0 = __shfl_xor_sync(0xffffffffu, x0, 1) + a; x1 = __shfl_xor_sync(0xffffffffu, x1, 2) + a;
    x2 = __shfl_xor_sync(0xffffffffu, x2, 4) + a; x3 = __shfl_xor_sync(0xffffffffu, x3, 8) + a;
  }
  float s = x0+x1+x2+x3; if (s == 12345.f) out[threadIdx.x] = s;
}
__global__ void k_red64(double* acc, int n, int stride) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = 0; i < 64; ++i) {
    unsigned idx = ((unsigned)(t * 2654435761u) + i * stride) % (unsigned)n;
    atomicAdd(&acc[idx], 1.0);
  }
}
__global__ void k_red32(float* acc, int n, int stride) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = 0; i < 64; ++i) {
    unsigned idx = ((unsigned)(t * 2654435761u) + i * stride) % (unsigned)n;
    atomicAdd(&acc[idx], 1.0f);
  }
}
int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int sms = p.multiProcessorCount; int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("device %s sms %d clockrate_khz %d cc %d.%d\n", p.name, sms, clk, p.major, p.minor);
  float* fo; double* dout; CK(cudaMalloc(&fo, 1<<20)); CK(cudaMalloc(&dout, 1<<20));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  int blocks = sms * 8, threads = 256; double nthr = (double)blocks * threads;
  auto timeit = [&](const char* name, auto launch, double ops_per_thread) {
    launch(); cudaDeviceSynchronize();
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) { cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms; }
    double rate = nthr * ops_per_thread / (best * 1e-3);
    printf("%-8s %.3f ms  %.3e ops/s  per_SM_per_clk@2070MHz %.2f\n", name, best, rate, rate / sms / 2.07e9);
  };
  timeit("ffma", [&]{ k_ffma<<<blocks, threads>>>(fo, 0.999f, 0.001f); }, IT * 8.0);
  timeit("dadd", [&]{ k_dadd<<<blocks, threads>>>(dout, 0.001); }, IT / 8 * 8.0);
  timeit("dfma", [&]{ k_dfma<<<blocks, threads>>>(dout, 0.999, 0.001); }, IT / 8 * 8.0);
  timeit("i2f", [&]{ k_i2f<<<blocks, threads>>>(fo, 3); }, IT * 4.0);
  timeit("rcp", [&]{ k_rcp<<<blocks, threads>>>(fo, 0.5f); }, IT * 4.0);
  timeit("f2d", [&]{ k_f2d<<<blocks, threads>>>(dout, 0.5f); }, IT / 8 * 4.0);
  timeit("shfl", [&]{ k_shfl<<<blocks, threads>>>(fo, 0.5f); }, IT * 4.0);
  int n = 1 << 20; CK(cudaMemset(dout, 0, 8 * (size_t)n > (1<<20) ? (1<<20) : 8*(size_t)n));
  double* acc; CK(cudaMalloc(&acc, 8 * (size_t)n)); CK(cudaMemset(acc, 0, 8 * (size_t)n));
  timeit("red64", [&]{ k_red64<<<blocks, threads>>>(acc, n, 1); }, 64.0);
  float* acc32; CK(cudaMalloc(&acc32, 4 * (size_t)n)); CK(cudaMemset(acc32, 0, 4 * (size_t)n));
  timeit("red32", [&]{ k_red32<<<blocks, threads>>>(acc32, n, 1); }, 64.0);
  CK(cudaGetLastError()); CK(cudaDeviceSynchronize());
  printf("done\n");
  return 0;
}
