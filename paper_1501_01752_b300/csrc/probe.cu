// Arithmetic-throughput probes: the measured FMA rate of this GPU, the ALU
// roofline denominator of the FP64 product and of the double-float residual
// (the copy bandwidth and the tensor rate are measured elsewhere; nothing on
// this path uses tensor cores).  Each thread runs PROBE_CHAINS independent
// FMA chains (enough to cover the pipe latency), one wave of blocks per SM
// slot; the chains' sum is stored so that no FMA can be dropped.
#include <cuda_runtime.h>

#include "../../include/gsm.h"
#include "common.cuh"

namespace gsm {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(T *out, int iters, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed FP32 pairs: one fma.rn.f32x2 is two FP32 FMAs
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma2(float2 *out, int iters, float a, float b) {
  float2 x[PROBE_CHAINS];
  const float2 A = make_float2(a, a), Bv = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = make_float2((float)threadIdx.x, (float)c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = f2::fma(x[c], A, Bv);
  }
  float2 s = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s = f2::add(s, x[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace gsm

using namespace gsm;

// kind 0: FP64 FMA, 1: FP32 FMA, 2: packed FP32 pair FMA (fma.rn.f32x2).
extern "C" gsm_status gsm_probe_fma(int device, void *cuda_stream, int kind, double *tflops) {
  if (!tflops || kind < 0 || kind > 2) return GSM_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GSM_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device);
  const int blocks = sms * (per_sm / PROBE_THREADS);
  const int iters = kind == 0 ? 2048 : 16384;
  void *out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * 8) != cudaSuccess) {
    cudaGetLastError();
    return GSM_ERR_NOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    if (kind == 0)
      k_probe_fma<double><<<blocks, PROBE_THREADS, 0, st>>>((double *)out, iters, 0.999999, 1e-7);
    else if (kind == 1)
      k_probe_fma<float><<<blocks, PROBE_THREADS, 0, st>>>((float *)out, iters, 0.999999f, 1e-7f);
    else
      k_probe_fma2<<<blocks, PROBE_THREADS, 0, st>>>((float2 *)out, iters, 0.999999f, 1e-7f);
  };
  launch();   // warm-up
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GSM_ERR_CUDA;
  }
  const double fma_per_launch = (double)blocks * PROBE_THREADS * PROBE_CHAINS * iters * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fma_per_launch / (best * 1e-3) / 1e12;
  return GSM_OK;
}
