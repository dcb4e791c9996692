// Measured arithmetic peaks for the roofline of ALU-bound kernels.
//
// The FP32 filter of the diameter engine is bound by FP32 arithmetic, not by
// memory, so its roofline needs the rate at which this GPU retires FP32 fused
// multiply-adds; the plain FP64 kernels need the FP64 rate.  This file
// measures both: one full wave of blocks runs eight independent
// multiply-add chains per thread in registers (x <- x a + b with |a| < 1, so
// the values settle at b / (1 - a) and never overflow), with no memory
// traffic, and the host times the second of two identical launches with CUDA
// events.  A multiply-add counts as two flops; a packed f32x2 multiply-add as
// four.
#include "rad_internal.cuh"

namespace rad {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// kind 0: scalar FP32 multiply-adds; kind 2: FP64 multiply-adds.  The store
// is never taken (the chains settle near 1), it only keeps them live.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T a, T b, T* sink) {
  pdl_enter();  // the timed launch starts after the warm-up launch has finished
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x & 7) * (T)0.125 + (T)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s < (T)-1) sink[0] = s;
}

// kind 1: packed f32x2 multiply-adds (two FP32 lanes per instruction).
__global__ void __launch_bounds__(kProbeThreads) k_fma2_probe(int iters, float a, float b, float* sink) {
  pdl_enter();
  unsigned long long x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    const float v = (float)(threadIdx.x & 7) * 0.125f + (float)k;
    x[k] = pack2(v, v + 0.5f);
  }
  const unsigned long long A = pack2(a, a), B = pack2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma2(x[k], A, B);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += __uint_as_float((unsigned int)x[k]) + __uint_as_float((unsigned int)(x[k] >> 32));
  if (s < -1.f) sink[0] = s;
}

template <typename K, typename... Args>
rad_status timed_wave(const char* name, K kernel, cudaStream_t st, float* ms, Args... args) {
  const int grid = wave_grid(kernel, kProbeThreads, 1ll << 30);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RAD_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("cudaEventCreate failed");
    return RAD_ERR_CUDA;
  }
  rad_status rs = RAD_OK;
  auto run = [&]() -> rad_status {
    RAD_LAUNCH(name, kernel, grid, kProbeThreads, 0, st, args...);  // warm-up: clocks and caches
    RAD_CUDA(cudaEventRecord(e0, st));
    RAD_LAUNCH(name, kernel, grid, kProbeThreads, 0, st, args...);
    RAD_CUDA(cudaEventRecord(e1, st));
    RAD_CUDA(cudaEventSynchronize(e1));
    RAD_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return RAD_OK;
  };
  rs = run();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rs;
}

}  // namespace
}  // namespace rad

extern "C" rad_status rad_peak_probe(int kind, double* tflops, void* stream) {
  using namespace rad;
  if (!tflops || kind < RAD_PROBE_FP32 || kind > RAD_PROBE_FP64) {
    set_error("rad_peak_probe: unknown kind or NULL output");
    return RAD_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf sink;
  RAD_TRY(sink.reserve(16));
  float ms = 0.f;
  int grid = 0, iters = 0;
  double flops_per_step = 0.0;  // per thread and loop iteration
  rad_status rs = RAD_OK;
  if (kind == RAD_PROBE_FP32) {
    iters = 1 << 16;
    flops_per_step = 2.0 * kChains;
    grid = wave_grid(k_fma_probe<float>, kProbeThreads, 1ll << 30);
    rs = timed_wave("probe_fp32", k_fma_probe<float>, st, &ms, iters, 0.9990234375f, 0.0009765625f,
                    sink.as<float>());
  } else if (kind == RAD_PROBE_FP32X2) {
    iters = 1 << 15;
    flops_per_step = 4.0 * kChains;
    grid = wave_grid(k_fma2_probe, kProbeThreads, 1ll << 30);
    rs = timed_wave("probe_fp32x2", k_fma2_probe, st, &ms, iters, 0.9990234375f, 0.0009765625f,
                    sink.as<float>());
  } else {
    iters = 1 << 11;
    flops_per_step = 2.0 * kChains;
    grid = wave_grid(k_fma_probe<double>, kProbeThreads, 1ll << 30);
    rs = timed_wave("probe_fp64", k_fma_probe<double>, st, &ms, iters, 0.9990234375, 0.0009765625,
                    sink.as<double>());
  }
  sink.release();
  if (rs != RAD_OK) return rs;
  if (!(ms > 0.f)) {
    set_error("rad_peak_probe: no elapsed time measured");
    return RAD_ERR_INTERNAL;
  }
  const double flops = (double)grid * kProbeThreads * (double)iters * flops_per_step;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return RAD_OK;
}
