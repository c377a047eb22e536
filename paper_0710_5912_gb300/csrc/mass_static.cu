// shf_mass_static: the mean of a caller-owned device field without any device
// allocation.  It runs the same two reductions as shf_mass (per-CTA partials
// over the same number of CTAs, then the same fixed-order fold of the
// partials on the device), so both return the same bits for the same field;
// the partials live in a fixed file-scope device array instead of the grid's
// lazily allocated scratch, and only three doubles come back.
#include <cmath>
#include <cstdint>
#include <mutex>

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

// Device address of g_mass_scratch on each device, looked up once per device
// (with that device current) by the first call that runs there.  In host code
// the name g_mass_scratch is only a host-side stand-in, so kernels get this
// address, never the name.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {};

// the scratch address on the current device `dev`; nullptr if the lookup fails
double* scratch_on(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* sym = nullptr;
    if (cudaGetSymbolAddress(&sym, g_mass_scratch) != cudaSuccess || !sym) return nullptr;
    g_addr[dev] = static_cast<double*>(sym);
  }
  return g_addr[dev];
}

template <class T>
int mass_static_t(double* scratch, const void* d_field, long long count, cudaStream_t st, double* res) {
  // The partial slots are all written by the partial pass before the fold
  // reads them; only the result slot is reset (to NaN bytes) so that a failed
  // pass can never hand back a previous call's result.
  if (cudaMemsetAsync(scratch + kResultSlot, 0xFF, 3 * sizeof(double), st) != cudaSuccess) return SHF_ECUDA;
  const int ctas = launch_mass_partials<T>(static_cast<const T*>(d_field), count, scratch, kStaticMassCtas, st);
  if (cudaGetLastError() != cudaSuccess) return SHF_ECUDA;
  launch_mass_fold(scratch, ctas, scratch + kResultSlot, st);
  if (cudaGetLastError() != cudaSuccess) return SHF_ECUDA;
  if (cudaMemcpyAsync(res, scratch + kResultSlot, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SHF_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SHF_ECUDA;
  return SHF_OK;
}

}  // namespace

extern "C" int shf_mass_static(const void* d_field, int precision, int nx, int ny, void* cuda_stream,
                               double* mean_phi) {
  if (!mean_phi) return SHF_EINVAL;
  *mean_phi = NAN;
  if (!d_field) return SHF_EINVAL;
  if (precision != SHF_FP32 && precision != SHF_FP64) return SHF_EINVAL;
  if (nx < 1 || ny < 1 || nx > kStaticMaxSide || ny > kStaticMaxSide) return SHF_EINVAL;
  const size_t esize = precision == SHF_FP64 ? sizeof(double) : sizeof(float);
  if (reinterpret_cast<uintptr_t>(d_field) % esize != 0) return SHF_EINVAL;
  // a launch error left pending by earlier work on this thread is cleared
  // here, so that the check after this call's launches reports only its own
  cudaGetLastError();

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
  double* scratch = scratch_on(attr.device);
  int rc = SHF_ECUDA;
  if (scratch)
    rc = precision == SHF_FP64 ? mass_static_t<double>(scratch, d_field, count, st, res)
                               : mass_static_t<float>(scratch, d_field, count, st, res);
  if (attr.device != prev) cudaSetDevice(prev);
  if (rc != SHF_OK) return rc;
  if (res[2] > 0.0 || !(res[2] == res[2])) return SHF_ENONFINITE;
  *mean_phi = (res[0] + res[1]) / ((double)nx * (double)ny);
  return SHF_OK;
}
