// shf_fma_peak: the FP32 or FP64 fused multiply-add rate of the current GPU,
// measured.  It is the ceiling of the arithmetic roofline against which the
// transform passes of the step are read (they are bound by instruction issue
// and memory latency as much as by HBM bytes).  Not a step of the method.
#include <cuda_runtime.h>

#include "../../include/shf.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (hide the pipe latency)
constexpr int kUnroll = 16;      // FMAs per chain per loop iteration
constexpr int kThreads = 256;

// Each thread runs kChains independent recurrences a <- a * b + c.  With
// 0 < b < 1 the values settle at c / (1 - b), so nothing overflows; b and c
// are kernel arguments, so nothing folds at compile time.  The final test is
// false for every input the host passes and only keeps the chains live.
template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(-1)) out[blockIdx.x] = s;
}

template <class T>
int fma_peak_t(int ctas, double* flops_per_s) {
  T* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SHF_ECUDA;
  if (cudaMalloc(&out, ctas * sizeof(T)) != cudaSuccess) return SHF_ENOMEM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    const T b = T(0.999), c = T(1e-3);
    int iters = 64;
    float ms = 0.f;
    bool ok = true;
    // warm-up, then grow the loop until one launch takes at least 20 ms
    for (int pass = 0; pass < 8 && ok; ++pass) {
      cudaEventRecord(e0, st);
      k_fma_chains<T><<<ctas, kThreads, 0, st>>>(out, iters, b, c);
      cudaEventRecord(e1, st);
      ok = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (!ok || (pass > 0 && ms >= 20.f)) break;
      const double grow = ms > 0.f ? 25.0 / ms : 16.0;
      const double next = iters * (grow < 16.0 ? (grow > 1.0 ? grow : 1.0) : 16.0);
      iters = next > (1 << 24) ? (1 << 24) : (int)next;
    }
    if (ok && ms > 0.f) {
      const double fmas = (double)ctas * kThreads * iters * kUnroll * kChains;
      *flops_per_s = 2.0 * fmas / (ms * 1e-3);
      rc = SHF_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int shf_fma_peak(int precision, int device, double* flops_per_s) {
  if (!flops_per_s || (precision != SHF_FP32 && precision != SHF_FP64)) return SHF_EINVAL;
  *flops_per_s = 0.0;
  int prev = 0, ndev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaGetDeviceCount(&ndev) != cudaSuccess) return SHF_ECUDA;
  if (device < 0 || device >= ndev) return SHF_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return SHF_ECUDA;
  int sms = 0, per_sm = 0;
  int rc = SHF_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess) {
    // a whole number of resident waves: every SM runs the same number of CTAs
    cudaError_t e = precision == SHF_FP32
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<float>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<double>, kThreads, 0);
    if (e == cudaSuccess && per_sm > 0) {
      const int ctas = sms * per_sm * 4;
      rc = precision == SHF_FP32 ? fma_peak_t<float>(ctas, flops_per_s) : fma_peak_t<double>(ctas, flops_per_s);
    }
  }
  cudaSetDevice(prev);
  return rc;
}
