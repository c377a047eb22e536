// Block-level complex FFTs for the row and column passes.
//
// The paper's transforms (Appendix B: real <-> reciprocal space "x -> q_x and
// y -> q_y", done with a CPU library) are done here by a hand-written
// Stockham auto-sort FFT: every stage reads R values at stride N/R, applies the
// stage twiddles, performs a radix-R DFT in registers and writes the results to
// their auto-sorted positions, so the output comes out in natural order with no
// bit reversal.
//
// - fft_reg (the step kernels): each thread holds P = 8 (or 16)
//   complex values in registers; a stage is radix P (one butterfly per
//   thread), or radix 8 / 4 / 2 for the last stage; stages exchange through a
//   padded shared buffer.  Twiddles come from per-stage tables (below), copied
//   once per CTA into shared memory in a compact per-length form.
// - fft_smem (the structure-factor diagnostics): in-place in shared memory,
//   8 values per thread per stage, twiddles from one table
//   W[k] = exp(+2 pi i k / NMAX) read with stride NMAX / N.
//
// Conventions (shared with the host code): forward uses exp(-2 pi i jk / N),
// inverse uses exp(+2 pi i jk / N) without scaling.  All tables are computed on
// the host in double precision and rounded once to the working precision.
#pragma once
#include <cuda_runtime.h>

namespace shf {

constexpr int LOG2_NMAX = 12;          // largest supported transform: 4096 points
constexpr int NMAX = 1 << LOG2_NMAX;

template <class T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <class T> using cplx = typename cplx_of<T>::type;

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) { return C{a.x * s, a.y * s}; }

// multiply by sigma*i, sigma = +1 (inverse) or -1 (forward)
template <bool INV, class C> __device__ __forceinline__ C mul_si(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

template <bool INV, class C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// X_k = sum_r v_r w^{rk}, w = sigma*i
template <bool INV, class C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  C s02 = cadd(v0, v2), d02 = csub(v0, v2);
  C s13 = cadd(v1, v3), d13 = csub(v1, v3);
  C wd = mul_si<INV>(d13);
  v0 = cadd(s02, s13);
  v2 = csub(s02, s13);
  v1 = cadd(d02, wd);
  v3 = csub(d02, wd);
}

// radix 8 as two radix-4 DFTs (even / odd inputs) joined by powers of
// w8 = exp(sigma 2 pi i / 8) = (1 + sigma i) / sqrt(2)
template <bool INV, class C>
__device__ __forceinline__ void dft8(C* v) {
  using T = decltype(v[0].x);
  const T c = T(0.70710678118654752440084436210484904);  // 1/sqrt(2)
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const T sg = INV ? T(1) : T(-1);
  // w8^1 * o1 = c (1 + sigma i) o1
  C t1 = C{c * (o1.x - sg * o1.y), c * (o1.y + sg * o1.x)};
  // w8^2 * o2 = sigma i o2
  C t2 = mul_si<INV>(o2);
  // w8^3 * o3 = c (-1 + sigma i) o3
  C t3 = C{c * (-o3.x - sg * o3.y), c * (-o3.y + sg * o3.x)};
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

// radix 16 as 4 x 4: radix-4 DFTs over n1 (n = 4 n1 + n2), the factors
// w16^{n2 k1}, w16 = exp(sigma 2 pi i / 16), then radix-4 DFTs over n2;
// X[k1 + 4 k2] lands in v[k1 + 4 k2]
template <bool INV, class C>
__device__ __forceinline__ C w16_times(C x, int e) {
  using T = decltype(x.x);
  const T c1 = T(0.92387953251128675612818318939678828682), s1 = T(0.38268343236508977172845998403039886676);
  const T r2 = T(0.70710678118654752440084436210484903928);
  const T sg = INV ? T(1) : T(-1);                     // sign of the imaginary part of w16
  T cr, ci;                                            // w16^e = cr + i sg ci
  switch (e) {
    case 1: cr = c1; ci = s1; break;
    case 2: cr = r2; ci = r2; break;
    case 3: cr = s1; ci = c1; break;
    case 4: return mul_si<INV>(x);
    case 6: cr = -r2; ci = r2; break;
    case 9: cr = -c1; ci = -s1; break;
    default: return x;
  }
  const T wi = sg * ci;
  return C{x.x * cr - x.y * wi, x.x * wi + x.y * cr};
}
template <bool INV, class C>
__device__ __forceinline__ void dft16(C* v) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);   // -> v[4 k1 + n2]
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[4 * k1 + n2] = w16_times<INV>(v[4 * k1 + n2], n2 * k1);
  C o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a = v[4 * k1], b = v[4 * k1 + 1], c = v[4 * k1 + 2], d = v[4 * k1 + 3];
    dft4<INV>(a, b, c, d);
    o[k1] = a;
    o[k1 + 4] = b;
    o[k1 + 8] = c;
    o[k1 + 12] = d;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = o[q];
}

template <bool INV, class C>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int idx) {
  C w = __ldg(tw + idx);
  return INV ? w : cconj(w);
}

// One Stockham stage of radix R = 2^LR on NB buffers: each thread does 8/R
// butterflies j = tid + b*T (T = N/8 threads per instance), reading inputs at
// j + r*N/R and writing the radix-R outputs to ((j - k) R + k) + r Ns with
// k = j mod Ns, Ns being the length of the sub-transforms already done.
template <bool INV, int NB, int LR, class C>
__device__ __forceinline__ void fft_stage(C* const (&buf)[NB], int log2N, int log2Ns, int tid,
                                          const C* __restrict__ tw) {
  constexpr int R = 1 << LR;
  constexpr int B = 8 >> LR;
  const int N = 1 << log2N;
  const int T = N >> 3;
  const int stride = N >> LR;
  C v[NB][8];
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][b * R + r] = buf[q][tid + b * T + r * stride];
  __syncthreads();
  const int Ns = 1 << log2Ns;
  const int twShift = LOG2_NMAX - log2Ns - LR;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = tid + b * T;
    const int k = j & (Ns - 1);
    const int base = ((j - k) << LR) + k;
    if (log2Ns > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C w = twiddle<INV>(tw, (k * r) << twShift);
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q][b * R + r] = cmul(v[q][b * R + r], w);
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (LR == 3) {
        dft8<INV>(&v[q][b * R]);
      } else if (LR == 2) {
        dft4<INV>(v[q][b * R], v[q][b * R + 1], v[q][b * R + 2], v[q][b * R + 3]);
      } else {
        dft2<INV>(v[q][b * R], v[q][b * R + 1]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) buf[q][base + r * Ns] = v[q][b * R + r];
    }
  }
  __syncthreads();
}

// In-place FFT of NB buffers of length N = 2^log2N (N >= 8) held in shared
// memory.  tid in [0, N/8) is this thread's index within its FFT instance;
// every thread of the CTA must call this (it contains __syncthreads), and all
// instances in the CTA must share N.  The routine starts with a barrier, so
// the caller's writes to the buffers need no barrier of their own, and it
// ends with one, so the results may be read right away.
template <bool INV, int NB, class C>
__device__ void fft_smem(C* const (&buf)[NB], int log2N, int tid, const C* __restrict__ tw) {
  __syncthreads();
  int log2Ns = 0;
  while (log2N - log2Ns >= 3) {
    fft_stage<INV, NB, 3>(buf, log2N, log2Ns, tid, tw);
    log2Ns += 3;
  }
  if (log2N - log2Ns == 2) fft_stage<INV, NB, 2>(buf, log2N, log2Ns, tid, tw);
  else if (log2N - log2Ns == 1) fft_stage<INV, NB, 1>(buf, log2N, log2Ns, tid, tw);
}

// ---------------------------------------------------------------------------
// Register-resident FFT (P = 8 points per thread).
//
// Thread t of an instance (0 <= t < T = N/P) holds v[q] = x[t + T q],
// q = 0..P-1.  Each Stockham stage is radix P except possibly the last (radix
// 4 or 2 when log2 N is not a multiple of log2 P).  A stage's butterflies
// j = t + b T (b < P/R) read x[j + r N/R] = v[b + r P/R] -- exactly the
// register layout -- so the first stage needs no exchange, and the last
// stage's outputs (positions j + r N/R) land in that same layout, so the
// transform ends in registers with v[q] = X[t + T q].  Only the stages in
// between exchange through shared memory.  Exchange buffers are padded by one
// element per 16 (index i -> i + i/16), which keeps the scatter of the early
// stages free of bank conflicts.  The column passes use eight points per
// thread (P = 16 with one mode per instance measured no faster there); the
// FP32 row passes use sixteen, one exchange fewer, which measured faster.
constexpr int kP = 8;
constexpr int kLogP = 3;

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// elements of a padded exchange buffer for an N-point transform
__host__ __device__ constexpr int padded_len(int N) { return N + N / 16; }

// Per-stage twiddle tables.  A stage of radix R = 2^LR after sub-transforms of
// length Ns = 2^a multiplies input r of butterfly k = j mod Ns by W_L^{k r},
// L = Ns R.  The table holds, for each (a, LR) with a + LR <= 12, the pair
// (exp(+2 pi i k / L), exp(+2 pi i 2k / L)) for k = 0..Ns-1 at entries
// [2 (stage_table_offset(a, LR) + k)], [.. + 1]: one 16-byte load (FP32) per
// butterfly, and the warp's loads are one contiguous run.  The other factors
// are products of these two (at most two roundings deep): w3 = w1 w2,
// w4 = w2 w2, w5 = w4 w1, w6 = w4 w2, w7 = w4 w3.
__host__ __device__ constexpr int stage_table_offset(int a, int LR) {
  return 4 * ((1 << a) - 1) + (LR - 1) * (1 << a);
}
// complex entries of the whole table (pairs for a = 0..11, LR = 1..4)
__host__ __device__ constexpr int stage_table_len() { return 2 * 4 * ((1 << 12) - 1); }

// Compact per-length tables in shared memory.  A register transform with
// 2^LP points per thread multiplies by twiddles only in its stages a = LP,
// 2 LP, ... (a = log2 Ns < log2 N; the last one of radix 2^(log2 N - a) <=
// 2^LP).  The compact table holds the Ns pairs of exactly these stages, in
// stage order: stage a starts at pair (2^a - 2^LP) / (2^LP - 1), the sum of
// the earlier stages' 2^b.  Each transform kernel copies it from the global
// table once per CTA, so the butterflies read their pair from shared memory.
__host__ __device__ constexpr int compact_stage_offset(int a, int LP) {
  return a < LP ? 0 : ((1 << a) - (1 << LP)) / ((1 << LP) - 1);
}
// pairs of the compact table of an N = 2^log2N transform
__host__ __device__ constexpr int compact_stage_pairs(int log2N, int LP) {
  return compact_stage_offset(((log2N - 1) / LP) * LP + LP, LP);
}
template <class C>
__device__ __forceinline__ void stage_tables_to_smem(C* dst, const C* __restrict__ tw, int log2N, int LP, int tid,
                                                     int nthr) {
  for (int a = LP; a < log2N; a += LP) {
    const int LR = log2N - a < LP ? log2N - a : LP;
    const C* src = tw + 2 * stage_table_offset(a, LR);
    C* d = dst + 2 * compact_stage_offset(a, LP);
    for (int i = tid; i < (2 << a); i += nthr) d[i] = __ldg(src + i);
  }
}

__device__ __forceinline__ void load_pair(const float2* p, float2& w1, float2& w2) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  w1 = float2{x.x, x.y};
  w2 = float2{x.z, x.w};
}
__device__ __forceinline__ void load_pair(const double2* p, double2& w1, double2& w2) {
  w1 = p[0];
  w2 = p[1];
}

// the R factors W_L^{k r}, r = 0..R-1, of butterfly k of a stage, from the
// compact table of a transform with 2^LP points per thread
template <int R, int LP, class C>
__device__ __forceinline__ void load_stage_factors(const C* tab, int log2Ns, int k, C (&f)[R]) {
  C w1, w2;
  load_pair(tab + 2 * (compact_stage_offset(log2Ns, LP) + k), w1, w2);
  f[1] = w1;
  if (R > 2) {
    f[2] = w2;
    f[3] = cmul(w1, w2);
  }
  if (R > 4) {
    f[4] = cmul(w2, w2);
    f[5] = cmul(f[4], w1);
    f[6] = cmul(f[4], w2);
    f[7] = cmul(f[4], f[3]);
  }
  if (R > 8) {                                          // w8 = w4 w4, w(8+r) = w8 wr
    f[8] = cmul(f[4], f[4]);
#pragma unroll
    for (int r = 1; r < 8; ++r) f[8 + r] = cmul(f[8], f[r]);
  }
}

template <bool INV, int LR, class C>
__device__ __forceinline__ void dft_radix(C* v) {
  if (LR == 4) dft16<INV>(v);
  else if (LR == 3) dft8<INV>(v);
  else if (LR == 2) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft2<INV>(v[0], v[1]);
}

// One stage on the register layout.  LAST: keep the outputs in registers;
// otherwise scatter them to buf (padded), barrier, gather the next stage's
// inputs, barrier (so the buffer can be written again).  The barrier is the
// CTA's (CtaSync) or, for a transform owned by a whole-warp subset of the CTA,
// a named barrier of that subset (NamedSync), so that several transforms in
// one CTA need not wait for each other.
template <int P> constexpr int log2_points() { return P == 16 ? 4 : 3; }

struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct NamedSync {
  int id, nthreads;                                    // barrier 1..15, a multiple of 32 threads
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
  }
};

template <bool INV, int LR, bool LAST, int P, class C, class Sync = CtaSync>
__device__ __forceinline__ void fft_reg_stage(C (&v)[P], int log2N, int log2Ns, int t, C* buf, const C* twt,
                                              const Sync& sync = Sync{}) {
  constexpr int R = 1 << LR;
  constexpr int B = P >> LR;
  const int T = 1 << (log2N - log2_points<P>());
  const int Ns = 1 << log2Ns;
  C w[R];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = t + b * T;
    const int k = j & (Ns - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = v[b + r * B];
    if (log2Ns > 0) {
      C f[R];
      load_stage_factors<R, log2_points<P>()>(twt, log2Ns, k, f);
#pragma unroll
      for (int r = 1; r < R; ++r) w[r] = cmul(w[r], INV ? f[r] : cconj(f[r]));
    }
    dft_radix<INV, LR>(w);
    if (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b + r * B] = w[r];
    } else {
      const int base = ((j - k) << LR) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad16(base + r * Ns)] = w[r];
    }
  }
  if (!LAST) {
    sync();
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = buf[pad16(t + q * T)];
    sync();
  }
}

// Transform of N = 2^log2N points (16 <= N <= NMAX) held as v[q] = x[t + T q].
// buf: this instance's padded exchange buffer (padded_len(N) elements); tw:
// the compact stage table of this length and P (compact_stage_offset) in
// shared memory.  All threads of the CTA must call it (barriers) with the same
// log2N.
template <bool INV, int P, class C, class Sync = CtaSync>
__device__ __forceinline__ void fft_reg(C (&v)[P], int log2N, int t, C* buf, const C* tw, const Sync& sync = Sync{}) {
  constexpr int LP = log2_points<P>();
  int log2Ns = 0;
  while (log2N - log2Ns > LP) {
    fft_reg_stage<INV, LP, false>(v, log2N, log2Ns, t, buf, tw, sync);
    log2Ns += LP;
  }
  switch (log2N - log2Ns) {
    case 4: if constexpr (P == 16) fft_reg_stage<INV, 4, true>(v, log2N, log2Ns, t, buf, tw, sync); break;
    case 3: fft_reg_stage<INV, 3, true>(v, log2N, log2Ns, t, buf, tw, sync); break;
    case 2: fft_reg_stage<INV, 2, true>(v, log2N, log2Ns, t, buf, tw, sync); break;
    default: fft_reg_stage<INV, 1, true>(v, log2N, log2Ns, t, buf, tw, sync); break;
  }
}

// v[q] = X[t + T q] -> buf (padded, natural order), followed by a barrier.
template <int P, class C>
__device__ __forceinline__ void reg_to_smem(const C (&v)[P], int log2N, int t, C* buf) {
  const int T = 1 << (log2N - log2_points<P>());
#pragma unroll
  for (int q = 0; q < P; ++q) buf[pad16(t + q * T)] = v[q];
  __syncthreads();
}

}  // namespace shf
