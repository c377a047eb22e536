// shf_mass_static: the mean of a caller-owned device field without any device
// allocation.  It runs the same two reductions as shf_mass (per-CTA Neumaier
// partials over the same number of CTAs, then a fold of the partials in CTA
// order), so both return the same bits for the same field; the partials live
// in a fixed file-scope device array instead of a lazily allocated buffer, and
// the fold runs on the device so that only three doubles come back.
#include <cmath>
#include <cstdint>

#include "../../include/shf.h"
#include "shf_internal.cuh"

using namespace shf;

namespace {

constexpr int kStaticMassCtas = 1024;   // CTAs of the partial pass; equal to shf_mass's
constexpr int kStaticMaxSide = 4096;    // largest nx and ny accepted (the largest grid)
// [0, 3*kStaticMassCtas): (sum, compensation, non-finite count) per CTA;
// [3*kStaticMassCtas, +3): the folded (sum, compensation, non-finite count).
constexpr int kResultSlot = 3 * kStaticMassCtas;
constexpr int kStaticSlots = kResultSlot + 3;   // 24,600 bytes per device

static __device__ __align__(256) double g_mass_scratch[kStaticSlots];

// Fold the partials in CTA order with the same Neumaier steps, in the same
// order, as shf_mass's host-side fold: one thread, so the result is fixed.
__global__ void k_fold_mass_partials(const double* __restrict__ part, int ctas, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double s = 0.0, c = 0.0, nf = 0.0;
  for (int b = 0; b < ctas; ++b) {
    const double v = part[3 * b];
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
    c += part[3 * b + 1];
    nf += part[3 * b + 2];
  }
  out[0] = s;
  out[1] = c;
  out[2] = nf;
}

template <class T>
int mass_static_t(const void* d_field, long long count, cudaStream_t st, double* res) {
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_mass_scratch) != cudaSuccess || !sym) return SHF_ECUDA;
  double* scratch = static_cast<double*>(sym);
  // The partial slots are all written by the partial pass before the fold
  // reads them; only the result slot is reset (to NaN bytes) so that a failed
  // pass can never hand back a previous call's result.
  if (cudaMemsetAsync(scratch + kResultSlot, 0xFF, 3 * sizeof(double), st) != cudaSuccess) return SHF_ECUDA;
  const int ctas = launch_mass_partials<T>(static_cast<const T*>(d_field), count, scratch, kStaticMassCtas, st);
  if (cudaGetLastError() != cudaSuccess) return SHF_ECUDA;
  k_fold_mass_partials<<<1, 32, 0, st>>>(scratch, ctas, scratch + kResultSlot);
  if (cudaGetLastError() != cudaSuccess) return SHF_ECUDA;
  if (cudaMemcpyAsync(res, scratch + kResultSlot, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SHF_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SHF_ECUDA;
  return SHF_OK;
}

}  // namespace

extern "C" int shf_mass_static(const void* d_field, int precision, int nx, int ny, void* cuda_stream,
                               double* mean_phi) {
  if (!mean_phi || !d_field) return SHF_EINVAL;
  if (precision != SHF_FP32 && precision != SHF_FP64) return SHF_EINVAL;
  if (nx < 1 || ny < 1 || nx > kStaticMaxSide || ny > kStaticMaxSide) return SHF_EINVAL;
  const size_t esize = precision == SHF_FP64 ? sizeof(double) : sizeof(float);
  if (reinterpret_cast<uintptr_t>(d_field) % esize != 0) return SHF_EINVAL;
  *mean_phi = NAN;

  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, d_field) != cudaSuccess) {
    cudaGetLastError();
    return SHF_ECUDA;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return SHF_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return SHF_ECUDA;
  if (attr.device != prev && cudaSetDevice(attr.device) != cudaSuccess) return SHF_ECUDA;

  double res[3] = {NAN, NAN, NAN};
  const long long count = (long long)nx * ny;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int rc = precision == SHF_FP64 ? mass_static_t<double>(d_field, count, st, res)
                                       : mass_static_t<float>(d_field, count, st, res);
  if (attr.device != prev) cudaSetDevice(prev);
  if (rc != SHF_OK) return rc;
  if (res[2] > 0.0 || !(res[2] == res[2])) return SHF_ENONFINITE;
  *mean_phi = (res[0] + res[1]) / ((double)nx * (double)ny);
  return SHF_OK;
}
