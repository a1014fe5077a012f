// mdx_measure_peaks: arithmetic-throughput probes that give the roofline
// denominators of the benchmark's compute-bound kernels (not part of the
// detection path).
//
//   FP32 FFMA  the tree searches' partial distances (Eq. 4 / Eq. inc) are
//              FP32 FMAs; the probe runs 8 independent FFMA chains per
//              thread on every SM.
//   FP64 DFMA  the QR's panel (Householder reflectors, Sec. III-B) is FP64
//              FMA work; 8 independent DFMA chains per thread.
//   FP64 MMA   the QR's trailing updates are mma.sync m8n8k4 FP64 tiles; the
//              probe runs 4 independent accumulator chains per warp and
//              changes the A and B operand values before every MMA with an
//              integer XOR of their lowest mantissa bit (an ALU-pipe op), so
//              the hardware sees fresh operands each time, as in the QR.  A
//              loop that feeds the same operands reads several times higher
//              and does not describe real tiles.
// Flops count an FMA as two; an m8n8k4 MMA as 2 * 8 * 8 * 4 = 512.
#include <cuda_runtime.h>

#include "mdx_internal.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_probe(int iters, float seed, float* sink) {
  float a[kChains];
  const float b = 1.0f - 1e-7f * (threadIdx.x & 7), c = 1e-7f * seed;
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = seed + 0.01f * j + 1e-6f * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(256) dfma_probe(int iters, double seed, double* sink) {
  double a[kChains];
  const double b = 1.0 - 1e-12 * (threadIdx.x & 7), c = 1e-12 * seed;
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = seed + 0.01 * j + 1e-9 * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.678) sink[blockIdx.x] = s;
}

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ double flip_lsb(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ 1ll);
}

__global__ void __launch_bounds__(256) dmma_probe(int iters, double seed, double* sink) {
  double acc[4][2];
  double a[4], b[4];
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    acc[j][0] = acc[j][1] = 0.0;
    a[j] = 1e-3 * (seed + lane + 3 * j);
    b[j] = 1e-3 * (seed - lane + 5 * j);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[j] = flip_lsb(a[j]);
      b[j] = flip_lsb(b[j]);
      dmma(acc[j][0], acc[j][1], a[j], b[j]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += acc[j][0] + acc[j][1];
  if (s == 12345.678) sink[blockIdx.x] = s;
}

template <typename F>
cudaError_t time_ms(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  launch();  // warm-up
  cudaEventRecord(e0, s);
  launch();
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" mdx_status mdx_measure_peaks(int device, double* out, void* stream) {
  if (!out) return MDX_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return MDX_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return MDX_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 4, threads = 256;
  double* sink = nullptr;
  mdx_status st = MDX_OK;
  float ms[3] = {0, 0, 0};
  const int it32 = 1 << 18, it64 = 1 << 12, itmma = 1 << 11;
  if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) {
    cudaSetDevice(prev);
    return MDX_ENOMEM;
  }
  cudaError_t e = time_ms([&] { ffma_probe<<<blocks, threads, 0, s>>>(it32, 1.5f, (float*)sink); }, s, &ms[0]);
  if (e == cudaSuccess) e = time_ms([&] { dfma_probe<<<blocks, threads, 0, s>>>(it64, 1.5, sink); }, s, &ms[1]);
  if (e == cudaSuccess) e = time_ms([&] { dmma_probe<<<blocks, threads, 0, s>>>(itmma, 1.5, sink); }, s, &ms[2]);
  if (e != cudaSuccess) st = MDX_ECUDA;
  cudaFree(sink);
  cudaSetDevice(prev);
  if (st != MDX_OK) return st;
  const double thr = (double)blocks * threads;
  out[0] = 2.0 * kChains * thr * it32 / (ms[0] * 1e-3) / 1e12;
  out[1] = 2.0 * kChains * thr * it64 / (ms[1] * 1e-3) / 1e12;
  out[2] = 512.0 * 4 * (thr / 32) * itmma / (ms[2] * 1e-3) / 1e12;
  out[3] = ms[0] + ms[1] + ms[2];
  return MDX_OK;
}
