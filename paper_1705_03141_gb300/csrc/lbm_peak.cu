// FP32 CUDA-core throughput of the device, measured: the ALU roof beside the
// HBM roof for the stepping kernels, whose arithmetic is FP32 FMA/ADD/MUL on
// the CUDA cores (no tensor-core contraction on this path).
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (hides the FMA latency)

// Every thread runs kChains dependent chains x <- x*a + b for `iters` iterations;
// the final values are stored so that nothing is dead code.
__global__ void __launch_bounds__(256) k_fma_scalar(float* __restrict__ out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same with Blackwell's packed FP32x2 FMA: kChains/2 float2 chains, the
// same FLOPs per iteration.
__global__ void __launch_bounds__(256) k_fma_packed(float* __restrict__ out, int iters, float a, float b) {
  float2 x[kChains / 2];
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) x[j] = make_float2((float)(threadIdx.x + 2 * j) * 1e-3f, (float)(threadIdx.x + 2 * j + 1) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) s += x[j].x + x[j].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

lbm_status lbm_measure_fp32_peak(void* cuda_stream, int packed, double* tflops) {
  if (!tflops) return LBM_EINVAL;
  *tflops = 0.0;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  const int threads = 256, blocks = sms * 8, iters = 1 << 15;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * threads * blocks) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lbm_status st = LBM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = LBM_ECUDA;
  float best = 0.f;
  for (int rep = 0; rep < 4 && st == LBM_OK; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(e0, s);
    if (packed)
      k_fma_packed<<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-4f);
    else
      k_fma_scalar<<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-4f);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = LBM_ECUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (st == LBM_OK && best > 0.f)
    *tflops = 2.0 * kChains * (double)iters * threads * blocks / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  cudaGetLastError();
  return st;
}

}  // extern "C"
