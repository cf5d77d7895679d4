// ib_measure_peak: throughput probes of this GPU for the rooflines the
// benchmark reports next to the HBM one (no counterpart in the paper).
//
//   IB_PEAK_FP64_FMA, IB_PEAK_FP32_FMA: fused multiply-adds of independent
//     register chains (8 per thread, enough warps per SM to fill the pipe),
//     reported as FLOP/s (2 per FMA).  The FP64 one is the ceiling of the FP64
//     right-hand side and line solves, whose throughput is bound by the FP64
//     pipe rather than by HBM.
//   IB_PEAK_L2_ATOMIC: float atomic adds whose results are not returned
//     (reductions), each warp instruction on 32 consecutive floats of a 16 MB
//     buffer that stays in L2, reported as atomic updates per second: the
//     ceiling of spreading (Step 2b), which is bound by L2 atomics.
// Each probe runs 3 warm-up and 5 timed launches (CUDA events on the given
// stream) and reports the best.  It allocates and frees its own scratch and
// synchronises the stream.
#include <cuda_runtime.h>

#include "../../include/ib_gb300.h"

int ib_internal_fail(int code, const char *msg);

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(T *out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == T(-1)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_red(float *buf, unsigned mask, int iters) {
  const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  unsigned base = warp * 32u * 977u;
  for (int i = 0; i < iters; ++i) {
    atomicAdd(buf + ((base + 32u * (unsigned)i + lane) & mask), 1.0f);
  }
}

}  // namespace

extern "C" int ib_measure_peak(int kind, void *stream, double *value) {
  if (!value) return ib_internal_fail(IB_ERR_ARG, "ib_measure_peak: null value");
  if (kind != IB_PEAK_FP64_FMA && kind != IB_PEAK_FP32_FMA && kind != IB_PEAK_L2_ATOMIC)
    return ib_internal_fail(IB_ERR_ARG, "ib_measure_peak: unknown kind");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return ib_internal_fail(IB_ERR_CUDA, cudaGetErrorString(e));
  const unsigned nbuf = 1u << 22;  // 16 MB of floats
  void *buf = nullptr;
  if ((e = cudaMalloc(&buf, nbuf * sizeof(float))) != cudaSuccess) return ib_internal_fail(IB_ERR_OOM, "ib_measure_peak");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 0.0;
  const int blocks = sms * 8, threads = 256;
  const int iters = kind == IB_PEAK_FP64_FMA ? 256 : (kind == IB_PEAK_FP32_FMA ? 8192 : 512);
  double work = (double)blocks * threads * iters;  // FMAs per chain, or atomics
  if (kind != IB_PEAK_L2_ATOMIC) work *= 2.0 * kChains;
  if ((e = cudaMemsetAsync(buf, 0, nbuf * sizeof(float), s)) == cudaSuccess && (e = cudaEventCreate(&e0)) == cudaSuccess &&
      (e = cudaEventCreate(&e1)) == cudaSuccess) {
    for (int rep = 0; rep < 8 && e == cudaSuccess; ++rep) {
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
      if (kind == IB_PEAK_FP64_FMA)
        k_peak_fma<double><<<blocks, threads, 0, s>>>((double *)buf, iters, 0.999999, 1e-9);
      else if (kind == IB_PEAK_FP32_FMA)
        k_peak_fma<float><<<blocks, threads, 0, s>>>((float *)buf, iters, 0.999999f, 1e-9f);
      else
        k_peak_red<<<blocks, threads, 0, s>>>((float *)buf, nbuf - 1, iters);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (rep >= 3 && ms > 0.f && work / (ms * 1e-3) > best) best = work / (ms * 1e-3);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return ib_internal_fail(IB_ERR_CUDA, cudaGetErrorString(e));
  *value = best;
  return IB_OK;
}
