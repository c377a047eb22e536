// Device helpers shared by the step kernels (step_kernels.cu: stencils and
// dispatch; step_rows.cu: row transforms; step_cols.cu: column passes).
#pragma once
#include <type_traits>

#include "shf_internal.cuh"

namespace shf {

// minimum resident CTAs per SM requested from the compiler (caps registers)
template <class T> constexpr int min_ctas() { return sizeof(T) == 8 ? 1 : 2; }

template <class T> struct Layout;
template <> struct Layout<float> { static constexpr int LC = 1; };   // 2 complex floats = 16 B
template <> struct Layout<double> { static constexpr int LC = 0; };  // 1 complex double = 16 B

// cells by which row j moves at a wrap: ((K1 - K0) r j) mod nx
__device__ __forceinline__ int remap_shift(long long dK, int r, int j, int nx) {
  long long v = ((dK * r) % nx) * j % nx;
  if (v < 0) v += nx;
  return (int)v;
}

// x-spectral element (j, m) in the tiled layout
__device__ __forceinline__ size_t xs_idx(int j, int m, int ny, int LC) {
  return ((((size_t)(m >> LC) * ny) + j) << LC) | (size_t)(m & ((1 << LC) - 1));
}

// Strain s, wrap flag and the weights of the sheared y-derivative (Eq. p1y):
// D_y^s f = [w0 (f(i, j+1) - f(i, j-1)) + w1 (f(i+d, j+1) - f(i-d, j-1))] / 2h,
// w1 = |s|/2, w0 = 1 - w1, d = -2 for s >= 0 and +2 for s < 0.
template <class T>
struct Shear {
  T s, w0, w1;
  int d;
  long long dK;   // K(n+1) - K(n): nonzero when the strain wraps during the step
  // next = false: s = s(t^n) (stage 1); next = true: s = s(t^{n+1}) (stages 2-3)
  __device__ __forceinline__ Shear(const StepState& S, bool next) {
    s = (T)(next ? S.s1 : S.s0);
    w1 = (s < T(0) ? -s : s) * T(0.5);
    w0 = T(1) - w1;
    d = s >= T(0) ? -2 : 2;
    dK = S.dK;
  }
};

// one thread: the StepState of member D for the step starting at n
__device__ __forceinline__ void step_state_set(const MemberDesc& D, long long n) {
  double s0, s1;
  long long K0, K1;
  strain_dev(n, D.gdot, D.dt, D.ratio, s0, K0);
  strain_dev(n + 1, D.gdot, D.dt, D.ratio, s1, K1);
  StepState* S = D.st;
  S->n = n;
  S->dK = K1 - K0;
  S->s0 = s0;
  S->s1 = s1;
}


// One step of Kahan's compensated summation: returns the new running sum of
// s + x; c carries the excess of the additions so far (the exact sum is the
// returned value minus c).  Explicit round-to-nearest operations keep the
// compiler from simplifying it.
__device__ __forceinline__ float kahan_add(float s, float x, float& c) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  return t;
}

// ---- double-float arithmetic: a value carried as hi + lo, |lo| at most half
// an ulp of hi (Dekker's and Knuth's error-free transformations; the product's
// rounding error by one fused multiply-add).  About 44 significant bits.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_of(double v) {
  const float h = (float)v;
  return F2{h, (float)(v - (double)h)};
}
// Knuth's TwoSum: a + b = s + e exactly
__device__ __forceinline__ F2 two_sum_f(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return F2{s, e};
}
// Dekker's FastTwoSum (|a| >= |b| or a = 0): renormalises a pair
__device__ __forceinline__ F2 fast_two_sum_f(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  const F2 s = two_sum_f(a.hi, b.hi);
  return fast_two_sum_f(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ F2 df_neg(F2 a) { return F2{-a.hi, -a.lo}; }
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum_f(p, e);
}
// acc += x without renormalising (the low parts gather the rounding errors;
// renormalise with fast_two_sum_f once the sum is complete)
__device__ __forceinline__ void df_acc(F2& acc, F2 x) {
  const F2 s = two_sum_f(acc.hi, x.hi);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, x.lo));
}

// ---------------------------------------------------------------- stencils
// four consecutive reals at a 16-byte-aligned address
template <class T>
struct Quad {
  T v[4];
};
__device__ __forceinline__ Quad<float> ld4(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  return Quad<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return Quad<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ Quad<float> ldg4(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return Quad<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<double> ldg4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return Quad<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}
// two reals at an address aligned to two elements
__device__ __forceinline__ void ldg2(const float* p, float& a, float& b) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ldg2(const double* p, double& a, double& b) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// The advective increment of omega alone, -dt (D_y psi D_x omega - D_x psi
// D_y omega) (Eq. advective), written in place of omega* when omega is carried
// in spectral form (MemberDesc::wspec).  One expression for the tile and the
// streamed stencil, so both give the same bits.
template <class T>
__device__ __forceinline__ T advect_incr(T dt, T dyp, T dxf, T dxp, T dyf) {
  return -(dt * (dyp * dxf - dxp * dyf));
}

// a b - c d with a single rounding of the result (Kahan's algorithm with two
// fused multiply-adds): w = c d rounded, e = w - c d exactly, f = a b - w
// rounded once, result f + e.  The body-force curl is a small difference of
// two products of derivatives; this keeps its rounding relative to the result
// instead of to the products.  Sign-symmetric, so phi -> -phi stays exact.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = __fmaf_rn(-c, d, w);
  const float f = __fmaf_rn(a, b, -w);
  return __fadd_rn(f, e);
}
__device__ __forceinline__ double diff_of_products(double a, double b, double c, double d) {
  const double w = __dmul_rn(c, d);
  const double e = __fma_rn(-c, d, w);
  const double f = __fma_rn(a, b, -w);
  return __dadd_rn(f, e);
}

// Eight reals of a tile row, cols c .. c+7 (c a multiple of 4): the stencil
// row of a 4-point block whose first point sits at c + 2.
template <class T>
struct Row8 {
  T v[8];
};
template <class T>
__device__ __forceinline__ Row8<T> ld8(const T* p) {
  const Quad<T> a = ld4(p), b = ld4(p + 4);
  return Row8<T>{{a.v[0], a.v[1], a.v[2], a.v[3], b.v[0], b.v[1], b.v[2], b.v[3]}};
}

// Six reals of a tile row, cols c - 1 .. c + 4 (c a multiple of 4), read as
// pairs at c - 2 and c + 4 and a quad at c: the stencil row of a 4-point
// block of second differences whose first point sits at c.
template <class T>
struct Six {
  T v[6];
};
__device__ __forceinline__ Six<float> ld6(const float* p) {
  const float2 l = *reinterpret_cast<const float2*>(p - 2);
  const float4 m = *reinterpret_cast<const float4*>(p);
  const float2 r = *reinterpret_cast<const float2*>(p + 4);
  return Six<float>{{l.y, m.x, m.y, m.z, m.w, r.x}};
}
__device__ __forceinline__ Six<double> ld6(const double* p) {
  const double2 l = *reinterpret_cast<const double2*>(p - 2);
  const double2 m0 = reinterpret_cast<const double2*>(p)[0], m1 = reinterpret_cast<const double2*>(p)[1];
  const double2 r = *reinterpret_cast<const double2*>(p + 4);
  return Six<double>{{l.y, m0.x, m0.y, m1.x, m1.y, r.x}};
}

// Derivatives at the 4 points (centre index p + 2) of rows U (j+1), C (j),
// Dn (j-1): D_x f = (f(i+1) - f(i-1)) / 2h and Eq. p1y's sheared D_y^s f =
// [w0 (f(i, j+1) - f(i, j-1)) + w1 (f(i+d, j+1) - f(i-d, j-1))] / 2h, with
// d = -2 for s >= 0 (NEG = false) and d = +2 for s < 0 (NEG = true).
template <bool NEG, class T>
__device__ __forceinline__ void grad4(const Row8<T>& U, const Row8<T>& C, const Row8<T>& Dn, T w0, T w1, T inv2h,
                                      T (&dx)[4], T (&dy)[4]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    dx[p] = (C.v[p + 3] - C.v[p + 1]) * inv2h;
    const T up = NEG ? U.v[p + 4] : U.v[p];         // f(i+d, j+1)
    const T dn = NEG ? Dn.v[p] : Dn.v[p + 4];       // f(i-d, j-1)
    dy[p] = (w0 * (U.v[p + 2] - Dn.v[p + 2]) + w1 * (up - dn)) * inv2h;
  }
}


// ---- asynchronous global -> shared copies (cp.async; the wait is a hardware
// instruction, not a spin loop)
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ask L2 for `bytes` (a multiple of 16) at p (16-byte aligned): a bulk
// prefetch issued by one thread, holding no register or shared memory
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// ---- tensor-memory-accelerator (TMA) loads completed on an mbarrier
// (PTX cp.async.bulk.tensor / mbarrier).  A CTA is a cluster of one, so a
// shared::cta address is a valid shared::cluster destination.
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes initialised mbarriers visible to the async proxy (before the CTA barrier that publishes them)
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// waits for the phase of the given parity to complete, giving up after
// kMbarSpins polls (each poll may suspend the thread for a while in hardware);
// false means the copies never arrived
constexpr long long kMbarSpins = 1ll << 24;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (long long i = 0; i < kMbarSpins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// a tensor map written to global memory by the host: acquire it for the tensormap proxy
__device__ __forceinline__ void tmap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(tmap) : "memory");
}
// contiguous global -> shared bulk copy (16-byte aligned, a multiple of 16
// bytes) whose bytes complete the transaction count of bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// tiled 3D TMA load of one box at coordinates (c0, c1, c2) into dst; its
// bytes complete the transaction count of bar
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// bytes (a multiple of 16, both ends 16-byte aligned) from src to dst
__device__ __forceinline__ void copy_async(void* dst, const void* src, int bytes, int t, int nthr) {
  char* d = static_cast<char*>(dst);
  const char* s = static_cast<const char*>(src);
  for (int off = t * 16; off < bytes; off += nthr * 16) cp_async16(d + off, s + off);
}

// Half spectra of two real rows a, b from Z = FFT(a + i b) held in a padded
// buffer: A[m] = (Z[m] + conj Z[N-m]) / 2, B[m] = (Z[m] - conj Z[N-m]) / (2i).
template <class C>
__device__ __forceinline__ void split_pair(const C* z, int m, int mx, C& A, C& B) {
  using T = decltype(z[0].x);
  const C zk = z[pad16(m)];
  const C zc = cconj(z[pad16((-m) & mx)]);
  A = C{(zk.x + zc.x) * T(0.5), (zk.y + zc.y) * T(0.5)};
  B = C{(zk.y - zc.y) * T(0.5), -(zk.x - zc.x) * T(0.5)};
}

// One 32-byte global store (sm_100+ 256-bit access; p 32-byte aligned): a
// whole sector in one request.  The row passes' chunk writes land 64 KB apart,
// so two 16-byte stores per chunk cost two L2 requests each; this is 19%
// faster for the forward row pass at 4096^2.
__device__ __forceinline__ void st_global_v8(float* p, float4 a, float4 b) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
               "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
               : "memory");
}

// Z holds FFT(row j0 + i row j0+1) of one field: both half spectra -> dst.
// A thread writes whole chunks of the pair: 2 CL elements = 32 contiguous
// bytes (a full sector), as one 32-byte store in FP32 (j0 even and ny even
// keep it 32-byte aligned).
template <int LC, class C>
__device__ __forceinline__ void write_pair_rows(const C* z, C* dst, int j0, int nx, int ny, int t, int Tthreads) {
  constexpr int CL = 1 << LC;
  const int mx = nx - 1;
  const int nchunk = (nx >> 1) >> LC;
  for (int cb = t; cb < nchunk; cb += Tthreads) {
    C* p = dst + ((((size_t)cb * ny) + j0) << LC);
    C A[CL], B[CL];
#pragma unroll
    for (int c = 0; c < CL; ++c) split_pair(z, (cb << LC) + c, mx, A[c], B[c]);
    if constexpr (CL == 2) {
      st_global_v8(reinterpret_cast<float*>(p), make_float4(A[0].x, A[0].y, A[1].x, A[1].y),
                   make_float4(B[0].x, B[0].y, B[1].x, B[1].y));
    } else {
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        p[c] = A[c];
        p[CL + c] = B[c];
      }
    }
  }
}

// v[q] = Z[t + T q] from a padded buffer (the register layout of fft_reg)
template <int P, class C>
__device__ __forceinline__ void smem_to_reg(C (&v)[P], const C* Z, int log2N, int t) {
  const int T = 1 << (log2N - log2_points<P>());
#pragma unroll
  for (int q = 0; q < P; ++q) v[q] = Z[pad16(t + q * T)];
}

// Number of loop iterations of a persistent CTA: every instance of the CTA runs
// the same count (the loop body has barriers); an instance whose item is past
// the end idles through its last iteration.
__device__ __forceinline__ int persistent_iters(int nitems, int ipc) {
  const int stride = gridDim.x * ipc;
  const int first = blockIdx.x * ipc;
  return first < nitems ? (nitems - first + stride - 1) / stride : 0;
}

// Calls f(std::integral_constant<int, L>{}) for L = ln, the log2 of a transform
// length in [4, LOG2_NMAX]: the transform kernels are compiled per length.
template <class F>
inline void with_log2n(int ln, F&& f) {
  switch (ln) {
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: f(std::integral_constant<int, 9>{}); break;
    case 10: f(std::integral_constant<int, 10>{}); break;
    case 11: f(std::integral_constant<int, 11>{}); break;
    default: f(std::integral_constant<int, 12>{}); break;
  }
}

}  // namespace shf
