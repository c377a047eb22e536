// Diagnostics and data movement: precision conversion, the mass of phi
// (compensated double-precision sums) and the structure factor S(q) with its
// moments (Section VI, Eq. L_structure).  All reductions are deterministic:
// fixed per-thread order, fixed tree order in the CTA, fixed order over CTAs.
#include "shf_internal.cuh"

namespace shf {

// Neumaier's compensated summation (improved Kahan): sum holds the running
// sum, comp the accumulated rounding error of every addition.
__device__ __forceinline__ void neumaier_add(double& sum, double& comp, double v) {
  const double t = sum + v;
  if (fabs(sum) >= fabs(v)) comp += (sum - t) + v;
  else comp += (v - t) + sum;
  sum = t;
}

// Deterministic block reduction of NV (sum, comp) pairs (and plain values)
// through warp shuffles and one shared-memory round.  Result valid in thread 0.
template <int NV>
__device__ void block_reduce_pairs(double (&s)[NV], double (&c)[NV], double* sh /* 2*NV*32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double os = __shfl_down_sync(0xffffffffu, s[v], off);
      const double oc = __shfl_down_sync(0xffffffffu, c[v], off);
      if (lane < off) {
        neumaier_add(s[v], c[v], os);
        c[v] += oc;
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sh[(2 * v) * 32 + warp] = s[v];
      sh[(2 * v + 1) * 32 + warp] = c[v];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      s[v] = sh[(2 * v) * 32];
      c[v] = sh[(2 * v + 1) * 32];
      for (int w = 1; w < nw; ++w) {
        neumaier_add(s[v], c[v], sh[(2 * v) * 32 + w]);
        c[v] += sh[(2 * v + 1) * 32 + w];
      }
    }
  }
}

template <class T>
__global__ void k_convert_in(const double* __restrict__ src, T* __restrict__ dst, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}
template <class T>
__global__ void k_convert_out(const T* __restrict__ src, double* __restrict__ dst, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}

// Knuth's TwoSum: s + e equals a + b exactly (round to nearest, no overflow),
// with s = fl(a + b); explicit round-to-nearest additions keep the compiler
// from reordering it.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
// 1 if x is NaN or +-Inf (all exponent bits set), from the bits alone
__device__ __forceinline__ unsigned nonfinite_bit(float x) {
  return (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u;
}

// FP32 fields: out[3*cta + 0..2] = (sum, compensation, non-finite count) over
// this CTA's grid-stride share of f.  A thread reads 16-byte vectors, eight
// per group of 32 values (one from each of eight consecutive grid strides, all
// in flight at once), and adds each group with a tree of Knuth's TwoSum in
// FP32: the group's rounded sum goes into a double accumulator (one FP64
// addition per 32 values, the FP64 pipe being narrow on this part) and the
// exact rounding errors of the tree into a float one.  Each double addition
// rounds at most half an ulp of the thread's running sum, so the thread total
// is within a few 1e-16 of its exact sum relative to its magnitude; threads
// and CTAs are then combined with Neumaier's compensated sum.  Fixed order
// throughout: for one field and launch shape the result is always the same
// bits.
constexpr int kMassVec = 8;   // 16-byte vectors per group
__device__ __forceinline__ float mass_group(const float4 (&v)[kMassVec], float& err, unsigned& bad) {
  float s[2 * kMassVec];
  float e = 0.f;
#pragma unroll
  for (int k = 0; k < kMassVec; ++k) {
    bad |= nonfinite_bit(v[k].x) | nonfinite_bit(v[k].y) | nonfinite_bit(v[k].z) | nonfinite_bit(v[k].w);
    float e0, e1;
    s[2 * k] = two_sum(v[k].x, v[k].y, e0);
    s[2 * k + 1] = two_sum(v[k].z, v[k].w, e1);
    e += e0 + e1;
  }
#pragma unroll
  for (int w = 2 * kMassVec; w > 1; w >>= 1) {        // pairwise tree, fixed order
#pragma unroll
    for (int k = 0; k < w / 2; ++k) {
      float ek;
      s[k] = two_sum(s[2 * k], s[2 * k + 1], ek);
      e += ek;
    }
  }
  err += e;
  return s[0];
}
__global__ void __launch_bounds__(256) k_mass_partials_f32(const float* __restrict__ f, long long count,
                                                           double* __restrict__ out) {
  __shared__ double sh[2 * 2 * 32];
  double acc4[4] = {0.0, 0.0, 0.0, 0.0};                // groups g go to acc4[g mod 4]: short FP64 chains
  float tail = 0.f;
  unsigned bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = (reinterpret_cast<uintptr_t>(f) & 15) == 0 ? count / 4 : 0;
  const float4* f4 = reinterpret_cast<const float4*>(f);
  long long e = tid;
  int g = 0;
  for (; e + (kMassVec - 1) * stride < n4; e += kMassVec * stride, ++g) {
    float4 v[kMassVec];
#pragma unroll
    for (int k = 0; k < kMassVec; ++k) v[k] = __ldcs(f4 + e + k * stride);
    const double h = (double)mass_group(v, tail, bad);
    switch (g & 3) {
      case 0: acc4[0] += h; break;
      case 1: acc4[1] += h; break;
      case 2: acc4[2] += h; break;
      default: acc4[3] += h; break;
    }
  }
  double acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
  for (; e < n4; e += stride) {                        // the last partial group
    const float4 a = __ldcs(f4 + e);
    bad |= nonfinite_bit(a.x) | nonfinite_bit(a.y) | nonfinite_bit(a.z) | nonfinite_bit(a.w);
    float e0, e1, e2;
    const float s01 = two_sum(a.x, a.y, e0), s23 = two_sum(a.z, a.w, e1);
    const float h = two_sum(s01, s23, e2);
    acc += (double)h;
    tail += (e0 + e1) + e2;
  }
  for (long long k = 4 * n4 + tid; k < count; k += stride) {   // the rest (or an unaligned field)
    const float v = f[k];
    bad |= nonfinite_bit(v);
    acc += (double)v;
  }
  // the CTA's sum: Neumaier over the lanes (fixed tree), then over the warps
  // in order; the non-finite flags by an integer OR (no FP64 work for them)
  double s = acc, c = (double)tail;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double os = __shfl_down_sync(0xffffffffu, s, off), oc = __shfl_down_sync(0xffffffffu, c, off);
    if (lane < off) {
      neumaier_add(s, c, os);
      c += oc;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  __shared__ unsigned shbad[32];
  if (lane == 0) {
    sh[warp] = s;
    sh[32 + warp] = c;
    shbad[warp] = bad;
  }
  __syncthreads();
  if (warp == 0) {                                     // the warps' sums in a fixed pairwise tree
    const int nw = (blockDim.x + 31) >> 5;
    s = lane < nw ? sh[lane] : 0.0;
    c = lane < nw ? sh[32 + lane] : 0.0;
    unsigned b = lane < nw ? shbad[lane] : 0u;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double os = __shfl_down_sync(0xffffffffu, s, off), oc = __shfl_down_sync(0xffffffffu, c, off);
      if (lane < off) {
        neumaier_add(s, c, os);
        c += oc;
      }
    }
    b = __reduce_or_sync(0xffffffffu, b);
    if (lane == 0) {
      out[3 * blockIdx.x + 0] = s;
      out[3 * blockIdx.x + 1] = c;
      out[3 * blockIdx.x + 2] = b ? 1.0 : 0.0;
    }
  }
}

// FP64 fields: out[3*cta + 0..2] = (sum, compensation, non-finite count) over
// this CTA's grid-stride share of f, one Neumaier addition per value.
template <class T>
__global__ void __launch_bounds__(256) k_mass_partials(const T* __restrict__ f, long long count,
                                                       double* __restrict__ out) {
  __shared__ double sh[2 * 2 * 32];
  double s[2] = {0.0, 0.0}, c[2] = {0.0, 0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = (double)f[e];
    if (isfinite(v)) neumaier_add(s[0], c[0], v);
    else s[1] += 1.0;
  }
  block_reduce_pairs<2>(s, c, sh);
  if (threadIdx.x == 0) {
    out[3 * blockIdx.x + 0] = s[0];
    out[3 * blockIdx.x + 1] = c[0];
    out[3 * blockIdx.x + 2] = s[1] + c[1];
  }
}

// Fold of the per-CTA mass partials into out[0..2] = (sum, compensation,
// non-finite count), in a fixed two-level order: lane l of one warp folds
// partials [l G, (l + 1) G) in order (G = ceil(ctas / 32)) with Neumaier's
// steps, then the 32 lane results meet in a fixed pairwise tree.  Every caller
// (shf_mass, shf_sync, shf_mass_static) uses this one fold, so they agree
// bit for bit on the same field.
__global__ void k_mass_fold(const double* __restrict__ part, int ctas, double* __restrict__ out) {
  const int lane = threadIdx.x;
  const int G = (ctas + 31) / 32;
  double s = 0.0, c = 0.0, nf = 0.0;
  for (int b = lane * G; b < (lane + 1) * G && b < ctas; ++b) {
    neumaier_add(s, c, part[3 * b]);
    c += part[3 * b + 1];
    nf += part[3 * b + 2];
  }
  // the 32 lane results in a fixed pairwise tree (short FP64 dependency chains)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double os = __shfl_down_sync(0xffffffffu, s, off), oc = __shfl_down_sync(0xffffffffu, c, off);
    const double on = __shfl_down_sync(0xffffffffu, nf, off);
    if (lane < off) {
      neumaier_add(s, c, os);
      c += oc;
      nf += on;
    }
  }
  if (lane == 0) {
    out[0] = s;
    out[1] = c;
    out[2] = nf;
  }
}

// Row transform of a real field, two rows per FFT (z = f_{2p} + i f_{2p+1}).
template <class T>
__global__ void __launch_bounds__(512) k_sf_rows(const T* __restrict__ f, cplx<T>* __restrict__ xs,
                                                  int log2nx, int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = 1 << log2nx, mx = nx - 1, half = nx >> 1;
  const int Tf = nx >> 3;
  const int inst = threadIdx.x / Tf, tid = threadIdx.x - inst * Tf;
  const int ipc = blockDim.x / Tf;
  const int j0 = 2 * (blockIdx.x * ipc + inst);
  C* z = reinterpret_cast<C*>(smem_raw) + (size_t)inst * nx;
  for (int q = 0; q < 8; ++q) {
    const int i = tid + q * Tf;
    z[i] = C{f[(size_t)j0 * nx + i], f[(size_t)(j0 + 1) * nx + i]};
  }
  C* const b1[1] = {z};
  fft_smem<false, 1>(b1, log2nx, tid, tw);
  for (int q = 0; q < 4; ++q) {
    const int k = tid + q * Tf;
    const C zk = z[k], zc = cconj(z[(-k) & mx]);
    xs[(size_t)j0 * half + k] = C{(zk.x + zc.x) * T(0.5), (zk.y + zc.y) * T(0.5)};
    xs[(size_t)(j0 + 1) * half + k] = C{(zk.y - zc.y) * T(0.5), -(zk.x - zc.x) * T(0.5)};
  }
}

// Column transforms of the x-spectral phi, then per-CTA partial moments of
// S = |phi_hat|^2 / (nx ny)^2 over the laboratory wavevector magnitude
// k = |(q_x, q_y - s q_x)|, half-spectrum weight 2 for m > 0, k = 0 and the
// Nyquist row excluded; optional per-CTA bins of width dk = 2 pi / (ny dx).
// Partials per CTA (kSfMoments): sum S, sum k S, sum S/k, and for the tensor
// of Eq. L_matrix sum q_cx^2 S, sum q_cx q_cy S, sum q_cy^2 S, sum S with
// k = 0 included.
template <class T>
__global__ void __launch_bounds__(512) k_sf_cols(const cplx<T>* __restrict__ xs, int log2nx, int log2ny,
                                                  double dx, double s, const cplx<T>* __restrict__ tw,
                                                  double* __restrict__ partials, int nbins,
                                                  double* __restrict__ bin_partials) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[2 * kSfMoments * 32];
  const int nx = 1 << log2nx, ny = 1 << log2ny, half = nx >> 1;
  const int Tc = ny >> 3;
  const int col = threadIdx.x / Tc, tid = threadIdx.x - col * Tc;
  const int ncol = blockDim.x / Tc;
  const int log2ncol = 31 - __clz(ncol);
  const int m0 = blockIdx.x * ncol;
  C* sm = reinterpret_cast<C*>(smem_raw);
  double* Sw = reinterpret_cast<double*>(sm + ncol * ny);     // weighted S per mode
  int* bin = reinterpret_cast<int*>(Sw + ncol * ny);
  for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
    const int c = e & (ncol - 1), n = e >> log2ncol;
    sm[c * ny + n] = xs[(size_t)n * half + m0 + c];
  }
  C* const b1[1] = {sm + col * ny};
  fft_smem<false, 1>(b1, log2ny, tid, tw);
  const int m = m0 + col;
  const double two_pi = 6.283185307179586476925286766559;
  const double qx = two_pi * m / (nx * dx);
  const double norm = 1.0 / ((double)nx * (double)ny);
  const double dk = two_pi / (ny * dx);
  double acc_s[kSfMoments], acc_c[kSfMoments];
  for (int v = 0; v < kSfMoments; ++v) acc_s[v] = acc_c[v] = 0.0;
  for (int q = 0; q < 8; ++q) {
    const int n = tid + q * Tc;
    const int idx = col * ny + n;
    double w = 0.0;
    int b = -1;
    if (n != (ny >> 1)) {
      const int ns = n < (ny >> 1) ? n : n - ny;
      const double qy = two_pi * ns / (ny * dx);
      const double ky = qy - s * qx;
      const C X = sm[idx];
      const double re = (double)X.x * norm, im = (double)X.y * norm;
      const double S = (m == 0 ? 1.0 : 2.0) * (re * re + im * im);
      neumaier_add(acc_s[3], acc_c[3], qx * qx * S);
      neumaier_add(acc_s[4], acc_c[4], qx * ky * S);
      neumaier_add(acc_s[5], acc_c[5], ky * ky * S);
      neumaier_add(acc_s[6], acc_c[6], S);
      if (!(m == 0 && n == 0)) {
        const double k = sqrt(qx * qx + ky * ky);
        neumaier_add(acc_s[0], acc_c[0], S);
        neumaier_add(acc_s[1], acc_c[1], k * S);
        neumaier_add(acc_s[2], acc_c[2], S / k);
        w = S;
        const double fb = floor(k / dk);
        b = (fb < (double)nbins) ? (int)fb : -1;
      }
    }
    if (nbins > 0) {
      Sw[idx] = w;
      bin[idx] = b;
    }
  }
  block_reduce_pairs<kSfMoments>(acc_s, acc_c, sh);
  if (threadIdx.x == 0) {
    for (int v = 0; v < kSfMoments; ++v) partials[kSfMoments * blockIdx.x + v] = acc_s[v] + acc_c[v];
  }
  if (nbins > 0) {
    __syncthreads();
    for (int bb = threadIdx.x; bb < nbins; bb += blockDim.x) {
      double sum = 0.0, comp = 0.0;
      for (int e = 0; e < ncol * ny; ++e)
        if (bin[e] == bb) neumaier_add(sum, comp, Sw[e]);
      bin_partials[(size_t)blockIdx.x * nbins + bb] = sum + comp;
    }
  }
}

// Column sums of a rows x cols array, each column summed over rows in order.
__global__ void k_reduce_rows(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double sum = 0.0, comp = 0.0;
  for (int r = 0; r < rows; ++r) neumaier_add(sum, comp, in[(size_t)r * cols + c]);
  out[c] = sum + comp;
}

// ----------------------------------------------------------------- launchers
template <class T>
void launch_convert_in(const double* src, T* dst, long long count, cudaStream_t st) {
  const int thr = 256;
  long long ctas = (count + thr - 1) / thr;
  if (ctas > 4096) ctas = 4096;
  k_convert_in<T><<<(int)ctas, thr, 0, st>>>(src, dst, count);
}
template <class T>
void launch_convert_out(const T* src, double* dst, long long count, cudaStream_t st) {
  const int thr = 256;
  long long ctas = (count + thr - 1) / thr;
  if (ctas > 4096) ctas = 4096;
  k_convert_out<T><<<(int)ctas, thr, 0, st>>>(src, dst, count);
}
template <class T>
int launch_mass_partials(const T* f, long long count, double* out, int max_ctas, cudaStream_t st) {
  const int thr = 256;
  // FP32: at least 256 values per thread, so that few threads take part in the
  // FP64 reductions (this part's FP64 pipe is narrow); FP64: one per thread
  const long long per = sizeof(T) == 4 ? 256 : 1;
  long long ctas = (count + thr * per - 1) / (thr * per);
  if (ctas > max_ctas) ctas = max_ctas;
  if (ctas < 1) ctas = 1;
  if constexpr (sizeof(T) == 4) k_mass_partials_f32<<<(int)ctas, thr, 0, st>>>(f, count, out);
  else k_mass_partials<T><<<(int)ctas, thr, 0, st>>>(f, count, out);
  return (int)ctas;
}
void launch_mass_fold(const double* partials, int ctas, double* out, cudaStream_t st) {
  k_mass_fold<<<1, 32, 0, st>>>(partials, ctas, out);
}
template <class T>
void launch_sf_rows(const T* phi, cplx<T>* xs, int log2nx, int log2ny, const cplx<T>* tw, const RowCfg& c,
                    cudaStream_t st) {
  k_sf_rows<T><<<c.ctas, c.threads, c.smem, st>>>(phi, xs, log2nx, log2ny, tw);
}
template <class T>
void launch_sf_cols(const cplx<T>* xs, int log2nx, int log2ny, double dx, double s, const cplx<T>* tw,
                    const ColCfg& c, double* partials, int nbins, double* bin_partials, cudaStream_t st) {
  k_sf_cols<T><<<c.ctas, c.threads, c.smem, st>>>(xs, log2nx, log2ny, dx, s, tw, partials, nbins,
                                                  bin_partials);
}
void launch_reduce_rows(const double* in, int rows, int cols, double* out, cudaStream_t st) {
  k_reduce_rows<<<(cols + 127) / 128, 128, 0, st>>>(in, rows, cols, out);
}

template <class T>
void set_diag_smem_limits() {
  const int lim = 220 * 1024;   // dynamic part; leaves room for static shared memory
  cudaFuncSetAttribute(k_sf_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_sf_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

#define SHF_DIAG_INST(T)                                                                                   \
  template void launch_convert_in<T>(const double*, T*, long long, cudaStream_t);                          \
  template void launch_convert_out<T>(const T*, double*, long long, cudaStream_t);                         \
  template int launch_mass_partials<T>(const T*, long long, double*, int, cudaStream_t);                   \
  template void launch_sf_rows<T>(const T*, cplx<T>*, int, int, const cplx<T>*, const RowCfg&,             \
                                  cudaStream_t);                                                           \
  template void launch_sf_cols<T>(const cplx<T>*, int, int, double, double, const cplx<T>*, const ColCfg&, \
                                  double*, int, double*, cudaStream_t);                                    \
  template void set_diag_smem_limits<T>();

SHF_DIAG_INST(float)
SHF_DIAG_INST(double)

}  // namespace shf
