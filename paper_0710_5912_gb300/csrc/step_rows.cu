// Row (x) passes of a step, compiled per row length nx = 2^LN: k_stage1_rows
// (the stage-1 stencil fused with the row transforms of phi*, f, omega*),
// k_rowfwd (mode 1: the stage-2 stencil fused with g's row transform; mode 2:
// omega's row transform that seeds w_hat) and k_rowinv (rowinv_phi,
// rowinv_flow; TMA-loaded row pairs).  See step_kernels.cu for the step's
// kernels and the x-spectral layout.
#include "step_common.cuh"

namespace shf {

// ============================================ low row modes of g (FP32 members)
// The coefficients m = 0..lowm of the row DFT of g, accurate to the rounding
// of g itself.  The flow solve divides g_hat by k^2 (or k^4), and at the
// smallest k the force's spectrum is small against its mean square, so the
// rounding of an FP32 transform (about eps times the RMS of g_hat at every
// mode) would dominate psi there.  The first radix-16 stage of the register
// FFT already holds, for thread t, y_t[r] = sum_q z(t + T q) W_16^{rq} with
// z = g(row 2p) + i g(row 2p + 1) and T = N / 16, and
//   Z[m] = sum_t W_N^{m t} y_t[m mod 16],
//   Z[N - m] = sum_t conj(W_N^{m t}) y_t[(16 - m) mod 16];
// each thread forms its terms in FP32 (one radix-16 DFT, one twiddle product)
// and the T terms of each coefficient are added with Kahan's compensated
// summation in two fixed-order levels through the (then idle) exchange
// buffer, which holds exactly 2 (2 kLowM + 1) floats per thread.  The two
// rows' coefficients A[m] = (Z[m] + conj Z[N-m]) / 2 and
// B[m] = (Z[m] - conj Z[N-m]) / (2i) go to low_rows.
// Part 1, each thread's terms: stage holds the item's two real rows (a at
// [0, N), b at [N, 2N)), so z(t + T q) = (a, b)[t + T q]; Zb: this instance's
// exchange buffer as floats; tws: the compact P = 16 stage table of this
// length.  No barrier: the caller's next barrier publishes the terms.
template <int LN>
__device__ __forceinline__ void low_row_terms(const float* stage, float* Zb, const float2* tws, int t,
                                              const MemberDesc& D) {
  constexpr int log2nx = LN;
  constexpr int N = 1 << LN;
  const int lowm = D.lowm;
  constexpr int Tc = N / 16;                           // threads per instance
  float2 u[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) u[q] = float2{stage[t + q * Tc], stage[N + t + q * Tc]};
  dft16<false>(u);                                     // u[r] = y_t[r]
  // W_N^t and W_N^{2t} (forward sign) from the last stage's pairs
  float2 w1 = float2{1.f, 0.f}, w2 = float2{1.f, 0.f};
  if (log2nx > 4) {
    constexpr int a_last = ((log2nx - 1) / 4) * 4;
    float2 e1, e2;
    load_pair(tws + 2 * (compact_stage_offset(a_last, 4) + t), e1, e2);
    w1 = cconj(e1);
    w2 = cconj(e2);
  }
  float2 w[kLowM + 1];
  w[0] = float2{1.f, 0.f};
  w[1] = w1;
  w[2] = w2;
  w[3] = cmul(w1, w2);
  w[4] = cmul(w2, w2);
  w[5] = cmul(w[4], w1);
  w[6] = cmul(w[4], w2);
  w[7] = cmul(w[4], w[3]);
  w[8] = cmul(w[4], w[4]);
  // value slots: 2 m, 2 m + 1 = Z[m] (m = 0..lowm); 2 (lowm + m) .. +1 = Z[N - m] (m = 1..lowm)
#pragma unroll
  for (int m = 0; m <= kLowM; ++m) {
    if (m > lowm) break;
    const float2 zm = cmul(w[m], u[m & 15]);
    Zb[(2 * m) * Tc + t] = zm.x;
    Zb[(2 * m + 1) * Tc + t] = zm.y;
    if (m > 0) {
      const float2 zn = cmul(cconj(w[m]), u[(16 - m) & 15]);
      Zb[(2 * (lowm + m)) * Tc + t] = zn.x;
      Zb[(2 * (lowm + m) + 1) * Tc + t] = zn.y;
    }
  }
}

// Part 2, after a barrier: the compensated sums and the rows' coefficients.
// All threads of the CTA call it (barriers).
template <int LN>
__device__ __forceinline__ void low_row_reduce(float* Zb, int t, const MemberDesc& D, int p, bool active,
                                               int log2ny) {
  const int lowm = D.lowm;
  const int nv = 2 * (2 * lowm + 1);                   // real values per thread
  constexpr int Tc = (1 << LN) / 16;                   // threads per instance
  // level 1 (long rows): value k's Tc terms in G groups, one (sum, compensation) each
  constexpr int kSlots = (2 * (2 * kLowM + 1) + Tc - 1) / Tc;
  const int G = Tc >= 2 * nv ? Tc / nv : 1;
  if (G > 1) {
    const int per = (Tc + G - 1) / G;
    float s = 0.f, c = 0.f;
    const bool has = t < nv * G;
    if (has) {
      const int k = t / G, gi = t - k * G;
      const int t0 = gi * per, t1 = min(Tc, t0 + per);
      for (int tt = t0; tt < t1; ++tt) s = kahan_add(s, Zb[k * Tc + tt], c);
    }
    __syncthreads();
    if (has) {
      Zb[2 * t] = s;
      Zb[2 * t + 1] = c;
    }
    __syncthreads();
  }
  // level 2: value k = t + i Tc folds its G partials (or its Tc terms) in order
  float tot[kSlots];
#pragma unroll
  for (int i = 0; i < kSlots; ++i) {
    const int k = t + i * Tc;
    float s = 0.f, c = 0.f;
    if (k < nv) {
      if (G > 1) {
        for (int gi = 0; gi < G; ++gi) {
          s = kahan_add(s, Zb[2 * (k * G + gi)], c);
          s = kahan_add(s, -Zb[2 * (k * G + gi) + 1], c);
        }
      } else {
        for (int tt = 0; tt < Tc; ++tt) s = kahan_add(s, Zb[k * Tc + tt], c);
      }
    }
    tot[i] = __fsub_rn(s, c);                          // Kahan's c is the excess added
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSlots; ++i)
    if (t + i * Tc < nv) Zb[t + i * Tc] = tot[i];
  __syncthreads();
  for (int m = t; active && m <= lowm; m += Tc) {     // short rows have fewer threads than modes
    const float zr = Zb[2 * m], zi = Zb[2 * m + 1];
    const float nr = m ? Zb[2 * (lowm + m)] : zr, ni = m ? Zb[2 * (lowm + m) + 1] : zi;
    float2* lr = static_cast<float2*>(D.low_rows) + ((size_t)m << log2ny);
    lr[2 * p] = float2{0.5f * (zr + nr), 0.5f * (zi - ni)};
    lr[2 * p + 1] = float2{0.5f * (zi + ni), -0.5f * (zr - nr)};
  }
  __syncthreads();
}

// ===================================================== stage-2 stencil of a row pair
// mu = -a phi + b phi^3 - kappa L_s phi (Appendix B item 2: 3-point second
// differences, the 4-point cross difference) and the body-force curl
// g = c_force (D_x phi D_y^s mu - D_y^s phi D_x mu) at s = s^{n+1} (Eqs.
// vortNum, G), for rows j0, j0 + 1, written as two real rows into buf.  A
// thread takes columns x0 .. x0 + 3 (x0 = 4k) and walks phi's rows j0 - 2 ..
// j0 + 3 straight from global memory (the item's rows were prefetched into
// L2), forming mu of rows j0 - 1 .. j0 + 2 at x0 - 2 .. x0 + 5 as each phi
// row arrives; only three phi rows and three mu rows are live at a time.

// columns x0 - 4 .. x0 + 7 of a global row (x0 a multiple of 4), periodic
template <class T>
struct Row12 {
  T v[12];
};
template <class T>
__device__ __forceinline__ Row12<T> ld12_row(const T* row, int x0, int mx) {
  const Quad<T> a = ldg4(row + ((x0 - 4) & mx)), b = ldg4(row + x0), c = ldg4(row + ((x0 + 4) & mx));
  return Row12<T>{{a.v[0], a.v[1], a.v[2], a.v[3], b.v[0], b.v[1], b.v[2], b.v[3], c.v[0], c.v[1], c.v[2], c.v[3]}};
}
// the middle eight (x0 - 2 .. x0 + 5)
template <class T>
__device__ __forceinline__ Row8<T> mid8(const Row12<T>& r) {
  return Row8<T>{{r.v[2], r.v[3], r.v[4], r.v[5], r.v[6], r.v[7], r.v[8], r.v[9]}};
}
template <class T>
struct MuConsts {
  T a, b, kxx, kxy, kyy;
};
// mu at x0 - 2 .. x0 + 5 of the row whose phi is C (U above, Dn below)
template <class T>
__device__ __forceinline__ Row8<T> mu8(const Row12<T>& U, const Row12<T>& C, const Row12<T>& Dn,
                                       const MuConsts<T>& k) {
  Row8<T> m;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T pc = C.v[c + 2];
    const T sxx = C.v[c + 3] - T(2) * pc + C.v[c + 1];          // unscaled second differences
    const T syy = U.v[c + 2] - T(2) * pc + Dn.v[c + 2];
    const T sxy = U.v[c + 3] - Dn.v[c + 3] - U.v[c + 1] + Dn.v[c + 1];
    const T klap = k.kxx * sxx - k.kxy * sxy + k.kyy * syy;      // kappa L_s phi
    m.v[c] = pc * (k.b * (pc * pc) - k.a) - klap;
  }
  return m;
}
template <bool NEG, class T>
__device__ __forceinline__ void stage2_pair(const MemberDesc& D, const T* __restrict__ phi, T* buf, int j0,
                                            int log2nx, int my, const Shear<T>& sc, int t, int Tf) {
  const int nx = 1 << log2nx, mx = nx - 1;
  const T cxx = T(1) + sc.s * sc.s, cxy = T(2) * sc.s;
  const T kappa = (T)D.kappa;
  const MuConsts<T> k{(T)D.a, (T)D.b, kappa * cxx * (T)D.inv_h2, kappa * cxy * (T)D.inv_4h2, kappa * (T)D.inv_h2};
  const T inv2h = (T)D.inv_2h, cf = (T)D.c_force;
  auto row = [&](int j) { return phi + ((size_t)(j & my) << log2nx); };
  for (int q = t; q < (nx >> 2); q += Tf) {
    const int x0 = 4 * q;
    Row12<T> p0 = ld12_row(row(j0 - 2), x0, mx), p1 = ld12_row(row(j0 - 1), x0, mx), p2 = ld12_row(row(j0), x0, mx);
    Row12<T> p3 = ld12_row(row(j0 + 1), x0, mx);
    const Row8<T> m0 = mu8(p2, p1, p0, k);             // mu rows j0 - 1, j0, j0 + 1, j0 + 2
    Row8<T> m1 = mu8(p3, p2, p1, k);
    const Row12<T> p4 = ld12_row(row(j0 + 2), x0, mx);
    Row8<T> m2 = mu8(p4, p3, p2, k);
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      // row j0 + o: phi rows (o + 1, o + 2, o + 3) of p0 .. p4, mu rows (o, o + 1, o + 2) of m0 .. m3
      T dxp[4], dyp[4], dxm[4], dym[4];
      if (o == 0) {
        grad4<NEG>(mid8(p3), mid8(p2), mid8(p1), sc.w0, sc.w1, inv2h, dxp, dyp);
        grad4<NEG>(m2, m1, m0, sc.w0, sc.w1, inv2h, dxm, dym);
      } else {
        const Row12<T> p5 = ld12_row(row(j0 + 3), x0, mx);
        const Row8<T> m3 = mu8(p5, p4, p3, k);
        grad4<NEG>(mid8(p4), mid8(p3), mid8(p2), sc.w0, sc.w1, inv2h, dxp, dyp);
        grad4<NEG>(m3, m2, m1, sc.w0, sc.w1, inv2h, dxm, dym);
      }
      T r[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) r[p] = cf * diff_of_products(dxp[p], dym[p], dyp[p], dxm[p]);
      st4(buf + o * nx + x0, r[0], r[1], r[2], r[3]);
    }
  }
}

// ====================================================== forward row transforms
// Work items: one per row pair p = rows (2p, 2p+1).  Mode 1 is stage 2: the
// stage-2 stencil of the pair (stage2_pair) computed straight into the
// staging buffer, then its row transform -> xs_g, plus the low row modes of g
// (FP32 inertial, P = 16); g itself never reaches HBM.  Mode 2: omega ->
// xs_w (the row half of the transform that seeds w_hat), staged with
// asynchronous copies.  Each item holds the two real rows (a, b) in shared
// memory and transforms a + i b, so every output chunk of the pair is one
// whole 32-byte piece.  (Stage 1's row transforms are fused with its
// stencil: k_stage1_rows.)
template <class T, int LN, int P, int MODE>
__global__ void __launch_bounds__(rowfwd_cta_threads(P), rowfwd_min_ctas<T>(P)) k_rowfwd(const MemberDesc* __restrict__ descs, int log2ny,
                                                               const cplx<T>* __restrict__ tw) {
  constexpr int mode = MODE;
  constexpr int log2nx = LN;
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tf = nx / P;
  const int ipc = blockDim.x / Tf;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int nitems = mode == 2 && !D.wspec ? 0 : ny >> 1;
  const int stride = gridDim.x * ipc;
  unsigned char* base = smem_raw + (size_t)inst * rowfwd_inst_bytes(nx, sizeof(T));
  T* stage = reinterpret_cast<T*>(base);
  C* Z = reinterpret_cast<C*>(base + 2 * (size_t)nx * sizeof(T));
  const T* src = mode == 1 ? static_cast<const T*>(D.phi) : static_cast<const T*>(D.omega);
  C* tws = reinterpret_cast<C*>(smem_raw + (size_t)ipc * rowfwd_inst_bytes(nx, sizeof(T)));
  stage_tables_to_smem(tws, tw, log2nx, log2_points<P>(), threadIdx.x, blockDim.x);
  const Shear<T> sc(*D.st, true);                      // stage 2: s^{n+1}
  const int my = ny - 1;

  auto issue = [&](int w) {                            // mode 2: stage omega's two rows
    if (w < nitems) {
      const T* ra = src + ((size_t)(2 * w) << log2nx);
      copy_async(stage, ra, nx * (int)sizeof(T), t, Tf);
      copy_async(stage + nx, ra + nx, nx * (int)sizeof(T), t, Tf);
    }
    cp_async_commit();
  };
  auto prefetch = [&](int w) {                         // mode 1: ask L2 for phi's rows 2w - 2 .. 2w + 3
    if (w < nitems && t < 6) l2_prefetch(src + ((size_t)((2 * w - 2 + t) & my) << log2nx), (unsigned)(nx * sizeof(T)));
  };

  const int iters = persistent_iters(nitems, ipc);
  int w = blockIdx.x * ipc + inst;
  if (MODE == 1) prefetch(w);
  else issue(w);
  for (int it = 0; it < iters; ++it, w += stride) {
    const bool active = w < nitems;
    const int p = w;
    if constexpr (MODE == 1) {
      const int j0 = 2 * (active ? w : 0);
      if (sc.d > 0) stage2_pair<true>(D, src, stage, j0, log2nx, my, sc, t, Tf);
      else stage2_pair<false>(D, src, stage, j0, log2nx, my, sc, t, Tf);
      __syncthreads();                                 // the pair's g complete
      prefetch(w + stride);                            // the next item's rows, during the transform
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    if constexpr (sizeof(T) == 4 && P == 16 && MODE == 1) {   // the force's low row modes, part 1
      if (D.low == 1) low_row_terms<LN>(reinterpret_cast<const float*>(stage), reinterpret_cast<float*>(Z), tws, t, D);
    }
    C v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = t + q * Tf;
      v[q] = C{stage[i], stage[nx + i]};
    }
    __syncthreads();                                    // stage free
    if (MODE == 2) issue(w + stride);                   // next item streams in during the transform
    if constexpr (sizeof(T) == 4 && P == 16 && MODE == 1) {
      if (D.low == 1) low_row_reduce<LN>(reinterpret_cast<float*>(Z), t, D, p, active, log2ny);
    }
    fft_reg<false>(v, log2nx, t, Z, tws);
    reg_to_smem(v, log2nx, t, Z);
    if (active) write_pair_rows<LC>(Z, static_cast<C*>(mode == 1 ? D.xs_g : D.xs_w), 2 * p, nx, ny, t, Tf);
    __syncthreads();                                    // Z reads done before the next transform
  }
  cp_async_wait_all();
}

// ===================================== stage 1 fused with its row transforms
// Per row pair p (rows j0 = 2p, j1 = 2p + 1), item 1 + item 2's advection at
// s = s^n (Eq. advective with the Eq. p1y stencils) and the row transforms
// of what it makes, with no HBM round trip in between:
//   phi* = phi - dt J(psi, phi): written out (the base of phi's increment)
//     and row-transformed -> xs_phi, nyq_phi;
//   f = phi^3 (the pre-advection phi) -> xs_f;
//   inertial members: omega* = omega - dt J(psi, omega) (written out, the base
//     of omega's increment) -> xs_w, nyq_omega; or, with w_hat, the increment
//     a = -dt J(psi, omega) alone -> xs_w.  At a wrap these are taken at the
//     relabelled positions (row j shifted by the wrap's cells).
// One stencil pass per item reads the four rows j0 - 1 .. j1 + 1 of phi, psi
// and omega straight from global memory (the halo rows come from L2), a
// thread making 4 x 2 outputs of each field per column group of 4, and writes
// the two pairs into the instance's two padded buffers; each buffer then feeds
// the register FFT and serves as its exchange buffer.  The next item's rows
// are prefetched into L2 while the current one is transformed.

// columns x0 - 2 .. x0 + 5 of a global row (x0 a multiple of 4), periodic
template <class T>
__device__ __forceinline__ Row8<T> ld8_row(const T* row, int x0, int mx) {
  T l0, l1, r0, r1;
  ldg2(row + ((x0 - 2) & mx), l0, l1);
  const Quad<T> q = ldg4(row + x0);
  ldg2(row + ((x0 + 4) & mx), r0, r1);
  return Row8<T>{{l0, l1, q.v[0], q.v[1], q.v[2], q.v[3], r0, r1}};
}

// the stencils of both rows of the pair, both fields in one pass over their
// inputs (psi's derivatives shared): bufp <- phi* = phi - dt J(psi, phi)
// (also to gphi when not null); inertial: bufw <- omega - dt J(psi, omega),
// or the increment alone (INCR), at the rows' relabelling cells sh0, sh1
// (also to gom when not null)
template <bool NEG, bool INCR, bool OMEGA, class T>
__device__ __forceinline__ void stage1_pair(const T* phi, const T* psi, const T* om, T* bufp, T* bufw, T* gphi,
                                            T* gom, int j0, int log2nx, int my, const Shear<T>& sc, T dt,
                                            T inv2h, int t, int Tf, int sh0, int sh1) {
  const int nx = 1 << log2nx, mx = nx - 1;
  auto row = [&](const T* a, int j) { return a + ((size_t)(j & my) << log2nx); };
  for (int k = t; k < (nx >> 2); k += Tf) {
    const int x0 = 4 * k;
    Row8<T> pD = ld8_row(row(phi, j0 - 1), x0, mx), pC = ld8_row(row(phi, j0), x0, mx);
    Row8<T> sD = ld8_row(row(psi, j0 - 1), x0, mx), sC = ld8_row(row(psi, j0), x0, mx);
    Row8<T> oD, oC;
    if (OMEGA) {
      oD = ld8_row(row(om, j0 - 1), x0, mx);
      oC = ld8_row(row(om, j0), x0, mx);
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const int j = j0 + o;
      const Row8<T> pU = ld8_row(row(phi, j + 1), x0, mx), sU = ld8_row(row(psi, j + 1), x0, mx);
      Row8<T> oU;
      if (OMEGA) oU = ld8_row(row(om, j + 1), x0, mx);
      T dxp[4], dyp[4];
      grad4<NEG>(sU, sC, sD, sc.w0, sc.w1, inv2h, dxp, dyp);
      {
        T dxf[4], dyf[4];
        grad4<NEG>(pU, pC, pD, sc.w0, sc.w1, inv2h, dxf, dyf);
        T r[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) r[p] = pC.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
        st4(bufp + o * nx + x0, r[0], r[1], r[2], r[3]);
        if (gphi) st4(gphi + ((size_t)j << log2nx) + x0, r[0], r[1], r[2], r[3]);
      }
      if (OMEGA) {
        T dxf[4], dyf[4];
        grad4<NEG>(oU, oC, oD, sc.w0, sc.w1, inv2h, dxf, dyf);
        T r[4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
          r[p] = INCR ? advect_incr(dt, dyp[p], dxf[p], dxp[p], dyf[p])
                      : oC.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
        T* brow = bufw + o * nx;
        const int sh = o ? sh1 : sh0;
        if (sh == 0) {
          st4(brow + x0, r[0], r[1], r[2], r[3]);
          if (gom) st4(gom + ((size_t)j << log2nx) + x0, r[0], r[1], r[2], r[3]);
        } else {
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            brow[(x0 + p + sh) & mx] = r[p];
            if (gom) gom[((size_t)j << log2nx) + ((x0 + p + sh) & mx)] = r[p];
          }
        }
        oD = oC;
        oC = oU;
      }
      pD = pC;
      pC = pU;
      sD = sC;
      sC = sU;
    }
  }
}

template <class T, int LN, int P>
__global__ void __launch_bounds__(rowfwd_cta_threads(P), rowfwd_min_ctas<T>(P))
    k_stage1_rows(const MemberDesc* __restrict__ descs, int log2ny, const cplx<T>* __restrict__ tw) {
  constexpr int log2nx = LN;
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, my = ny - 1;
  const int Tf = nx / P;
  const int ipc = blockDim.x / Tf;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int nitems = ny >> 1;
  const int stride = gridDim.x * ipc;
  // two padded buffers per instance: phi*'s pair, then omega*'s (or a's)
  const size_t one = stage1_inst_bytes(nx, sizeof(T));
  T* bufp = reinterpret_cast<T*>(smem_raw + (size_t)inst * 2 * one);
  T* bufw = reinterpret_cast<T*>(smem_raw + (size_t)inst * 2 * one + one);
  C* tws = reinterpret_cast<C*>(smem_raw + (size_t)ipc * 2 * one);
  stage_tables_to_smem(tws, tw, log2nx, log2_points<P>(), threadIdx.x, blockDim.x);
  const T* phi = static_cast<const T*>(D.phi);
  const T* psi = static_cast<const T*>(D.psi);
  const T* om = static_cast<const T*>(D.omega);
  const Shear<T> sc(*D.st, false);                     // s^n
  const T dt = (T)D.dt, inv2h = (T)D.inv_2h;
  const bool inertial = !D.stokes;
  const bool wrap = D.remap && sc.dK != 0;

  // ask L2 for item w's input rows (j0 - 1 .. j1 + 1 of phi, psi, omega)
  auto prefetch = [&](int w) {
    if (w < nitems && t < 4) {
      const int j = (2 * w - 1 + t) & my;
      const unsigned bytes = (unsigned)nx * sizeof(T);
      l2_prefetch(phi + ((size_t)j << log2nx), bytes);
      l2_prefetch(psi + ((size_t)j << log2nx), bytes);
      if (inertial) l2_prefetch(om + ((size_t)j << log2nx), bytes);
    }
  };
  // the row pair staged in buf (complete: the caller synchronised) -> FFT ->
  // both half spectra into dst (and the pair's Nyquist coefficients into nyq,
  // when not null); buf is the exchange buffer; ends with a barrier
  auto transform_pair = [&](T* buf, bool active, C* dst, T* nyq, int p) {
    C v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = t + q * Tf;
      v[q] = C{buf[i], buf[nx + i]};
    }
    __syncthreads();                                   // buf becomes the exchange buffer
    C* Z = reinterpret_cast<C*>(buf);
    fft_reg<false>(v, log2nx, t, Z, tws);
    reg_to_smem(v, log2nx, t, Z);
    if (active) {
      write_pair_rows<LC>(Z, dst, 2 * p, nx, ny, t, Tf);
      if (nyq && t == 0) {
        const C zn = Z[pad16(nx >> 1)];
        nyq[2 * p] = zn.x;
        nyq[2 * p + 1] = zn.y;
      }
    }
    __syncthreads();                                   // Z read before buf is written again
  };

  const int iters = persistent_iters(nitems, ipc);
  int w = blockIdx.x * ipc + inst;
  prefetch(w);
  for (int it = 0; it < iters; ++it, w += stride) {
    const bool active = w < nitems;
    const int p = active ? w : 0, j0 = 2 * p;
    // phi* (not relabelled: phi's wrap is applied to phi^{n+1}) and omega* or a
    T* gphi = active ? static_cast<T*>(D.phi_star) : (T*)nullptr;
    if (inertial) {
      const int sh0 = wrap ? remap_shift(sc.dK, D.ratio, j0, nx) : 0;
      const int sh1 = wrap ? remap_shift(sc.dK, D.ratio, j0 + 1, nx) : 0;
      T* gom = (active && !D.wspec) ? static_cast<T*>(D.omega_star) : (T*)nullptr;
      if (D.wspec) {
        if (sc.d > 0) stage1_pair<true, true, true>(phi, psi, om, bufp, bufw, gphi, gom, j0, log2nx, my, sc, dt, inv2h, t, Tf, sh0, sh1);
        else stage1_pair<false, true, true>(phi, psi, om, bufp, bufw, gphi, gom, j0, log2nx, my, sc, dt, inv2h, t, Tf, sh0, sh1);
      } else {
        if (sc.d > 0) stage1_pair<true, false, true>(phi, psi, om, bufp, bufw, gphi, gom, j0, log2nx, my, sc, dt, inv2h, t, Tf, sh0, sh1);
        else stage1_pair<false, false, true>(phi, psi, om, bufp, bufw, gphi, gom, j0, log2nx, my, sc, dt, inv2h, t, Tf, sh0, sh1);
      }
    } else {
      if (sc.d > 0) stage1_pair<true, false, false>(phi, psi, om, bufp, bufw, gphi, (T*)nullptr, j0, log2nx, my, sc, dt, inv2h, t, Tf, 0, 0);
      else stage1_pair<false, false, false>(phi, psi, om, bufp, bufw, gphi, (T*)nullptr, j0, log2nx, my, sc, dt, inv2h, t, Tf, 0, 0);
    }
    __syncthreads();                                   // both staged pairs complete
    prefetch(w + stride);                              // the next item's rows, during the transforms
    transform_pair(bufp, active, static_cast<C*>(D.xs_phi), static_cast<T*>(D.nyq_phi), p);
    // f = phi^3 of the pre-advection pair, in the FFT's register layout (the rows are in L1/L2)
    {
      C v[P];
      const T* ra = phi + ((size_t)j0 << log2nx);
      const T* rb = ra + nx;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int i = t + q * Tf;
        const T a = ra[i], b = rb[i];
        v[q] = C{(a * a) * a, (b * b) * b};
      }
      C* Z = reinterpret_cast<C*>(bufp);
      fft_reg<false>(v, log2nx, t, Z, tws);
      reg_to_smem(v, log2nx, t, Z);
      if (active) write_pair_rows<LC>(Z, static_cast<C*>(D.xs_f), j0, nx, ny, t, Tf);
      __syncthreads();
    }
    if (inertial)
      transform_pair(bufw, active, static_cast<C*>(D.xs_w), D.wspec ? (T*)nullptr : static_cast<T*>(D.nyq_omega), p);
  }
}

// one 16-byte shared-memory word as complex values (two floats pairs, or one double pair)
__device__ __forceinline__ void load16(const float2* p, float2 (&v)[2]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = float2{x.x, x.y};
  v[1] = float2{x.z, x.w};
}
__device__ __forceinline__ void load16(const double2* p, double2 (&v)[1]) { v[0] = *p; }

// ====================================================== inverse row transforms
// Work items: mode 0 (phi): row pairs of the phi increment; mode 1 (flow): per
// row pair, item 0 = psi, item 1 = the omega increment (inertial members).  The
// item's 32-byte chunks stream into the staging buffer during the previous
// transform; Z[k] = A[k] + i B[k], Z[N-k] = conj A[k] + i conj B[k] (A, B the
// two rows), Z[0] from the real parts, Z[N/2] = minus the staged field's row
// Nyquist coefficients / nx.
// P = 16 (FP32): 256-thread CTAs, two per SM (128 registers), and the
// increment bases are loaded after the transform to keep registers free.
template <class T, int LN, int P, int MODE>
__global__ void __launch_bounds__(rowfwd_cta_threads(P), P == 16 ? 2 : min_ctas<T>()) k_rowinv(
    const MemberDesc* __restrict__ descs, int log2ny, const cplx<T>* __restrict__ tw) {
  constexpr int mode = MODE;
  constexpr int log2nx = LN;
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  constexpr int CL = 1 << LC;
  constexpr int H = 16 / sizeof(C);                     // complex values per 16 bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1;
  const int Tf = nx / P;
  const int ipc = blockDim.x / Tf;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int nsub = (mode == 1 && !D.stokes) ? 2 : 1;
  const int nitems = (ny >> 1) * nsub;
  const int stride = gridDim.x * ipc;
  const int nchunk = (nx >> 1) >> LC;
  unsigned char* base = smem_raw + (size_t)inst * rowinv_inst_bytes(nx, sizeof(T));
  // staged chunks: row j0's chunk cb at stage[CL cb], row j1's at stage[CL (nchunk + cb)],
  // so that consecutive threads touch consecutive 16-byte words
  C* stage = reinterpret_cast<C*>(base);
  C* Z = stage + nx;
  C* tws = reinterpret_cast<C*>(smem_raw + (size_t)ipc * rowinv_inst_bytes(nx, sizeof(T)));
  stage_tables_to_smem(tws, tw, log2nx, log2_points<P>(), threadIdx.x, blockDim.x);

  // FP32 rows of >= 1024 points with tensor maps: one thread per instance loads
  // the item's row pair with TMA boxes of {4 floats, 2 rows, 256 chunks} (the
  // staged layout is then [chunk][row][16 bytes]); else every thread gathers
  // its chunks with 16-byte asynchronous copies ([row][chunk][16 bytes])
  constexpr int kBox = 256;
  const bool tma = sizeof(T) == 4 && P == 16 && D.tmap != nullptr && nchunk % kBox == 0 &&
                   (smem_addr(smem_raw) & 127u) == 0;   // uniform; TMA destinations 128-byte aligned
  // the instances' mbarriers sit after the twiddle table (kRowinvBarBytes of
  // the launch's dynamic shared memory), so that no static shared memory
  // shifts the 128-byte alignment of the staging buffers the TMA writes
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(
      smem_raw + (size_t)ipc * rowinv_inst_bytes(nx, sizeof(T)) + stage_table_bytes(log2nx, log2_points<P>(), sizeof(T)));
  unsigned long long* bar = bars + (inst & 3);
  unsigned phase = 0;
  const char* tmaps = static_cast<const char*>(D.tmap);
  if (tma && t == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
    for (int k = 0; k < 3; ++k) tmap_acquire(tmaps + 128 * k);
  }
  __syncthreads();

  auto issue = [&](int w) {
    if (w < nitems) {
      const int sub = w % nsub;
      const int j0 = 2 * (w / nsub);
      if (tma) {
        if (t == 0) {
          const char* tm = tmaps + 128 * (mode == 0 ? 0 : (sub == 0 ? 1 : 2));
          fence_proxy_async_smem();                     // the stage's earlier reads come first
          mbar_arrive_expect_tx(bar, (unsigned)(2 * nchunk * 16));
          for (int k = 0; k < nchunk / kBox; ++k) tma_load_3d(stage + 2 * CL * kBox * k, tm, 0, j0, kBox * k, bar);
        }
      } else {
        const C* src = static_cast<const C*>(mode == 0 ? D.xs_phi : (sub == 0 ? D.xs_g : D.xs_w));
        for (int cb = t; cb < nchunk; cb += Tf) {
          const C* g = src + ((((size_t)cb * ny) + j0) << LC);
          cp_async16(stage + CL * cb, g);
          cp_async16(stage + CL * (nchunk + cb), g + H);
        }
      }
      // the item's increment bases, read after its transform: into L2 now
      const bool base = mode == 0 || (sub == 1 && !D.wspec);
      if (P == 16 && base && t == 0) {
        const T* bs = static_cast<const T*>(mode == 0 ? D.phi_star : D.omega_star) + ((size_t)j0 << log2nx);
        l2_prefetch(bs, 2 * nx * (unsigned)sizeof(T));
      }
    }
    cp_async_commit();
  };

  const long long dK = (mode == 0 && D.remap) ? D.st->dK : 0;
  const T rn = T(1) / T(nx);
  const int iters = persistent_iters(nitems, ipc);
  int w = blockIdx.x * ipc + inst;
  issue(w);
  for (int it = 0; it < iters; ++it, w += stride) {
    const bool active = w < nitems;
    const int p = w / nsub, sub = w - p * nsub;
    const int j0 = 2 * p, j1 = j0 + 1;
    // phi increment, psi, omega increment; with w_hat, omega is a whole-field
    // transform like psi (kind 3)
    const int kind = mode == 0 ? 0 : (sub == 0 ? 1 : (D.wspec ? 3 : 2));
    C zn = C{T(0), T(0)};
    if (active && (kind == 0 || kind == 2)) {
      const T* nq = static_cast<const T*>(kind == 0 ? D.nyq_phi : D.nyq_omega);
      zn = C{-nq[j0] * rn, -nq[j1] * rn};
    }
    bool ok = true;
    if (tma) {
      if (active) {
        ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
      }
    } else {
      cp_async_wait_all();
    }
    if (!__syncthreads_and(ok)) {                       // the item's copies never arrived: flag it and stop
      if (threadIdx.x == 0) atomicOr(D.err, 1);
      return;
    }
    for (int cb = t; cb < nchunk; cb += Tf) {
      C Av[CL], Bv[CL];
      load16(stage + (tma ? 2 * CL * cb : CL * cb), Av);
      load16(stage + (tma ? 2 * CL * cb + CL : CL * (nchunk + cb)), Bv);
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        const int k = (cb << LC) + c;
        const C A = Av[c], B = Bv[c];
        if (k == 0) {
          Z[pad16(0)] = C{A.x, B.x};
          Z[pad16(nx >> 1)] = zn;
        } else {
          Z[pad16(k)] = C{A.x - B.y, A.y + B.x};
          Z[pad16(nx - k)] = C{A.x + B.y, B.x - A.y};
        }
      }
    }
    __syncthreads();                                    // Z complete, stage free
    issue(w + stride);
    C v[P];
    smem_to_reg(v, Z, log2nx, t);
    __syncthreads();                                    // Z becomes the exchange buffer
    // the real-space base of the increment (phi* or omega*): loaded before the
    // transform with 8 points per thread, after it with 16 (registers)
    T b0[P], b1[P];
    auto load_bases = [&]() {
      if (active && (kind == 0 || kind == 2)) {
        const T* bs = static_cast<const T*>(kind == 0 ? D.phi_star : D.omega_star);
#pragma unroll
        for (int q = 0; q < P; ++q) {
          b0[q] = bs[((size_t)j0 << log2nx) + t + q * Tf];
          b1[q] = bs[((size_t)j1 << log2nx) + t + q * Tf];
        }
      }
    };
    if (P == 8) load_bases();
    fft_reg<true>(v, log2nx, t, Z, tws);
    if (P == 16) load_bases();
    if (active) {
      if (kind == 1 || kind == 3) {
        T* out = static_cast<T*>(kind == 1 ? D.psi : D.omega);
#pragma unroll
        for (int q = 0; q < P; ++q) {
          out[((size_t)j0 << log2nx) + t + q * Tf] = v[q].x;
          out[((size_t)j1 << log2nx) + t + q * Tf] = v[q].y;
        }
      } else {
        T* out = static_cast<T*>(kind == 0 ? D.phi : D.omega);
        const int sh0 = (kind == 0 && dK) ? remap_shift(dK, D.ratio, j0, nx) : 0;
        const int sh1 = (kind == 0 && dK) ? remap_shift(dK, D.ratio, j1, nx) : 0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int i = t + q * Tf;
          out[((size_t)j0 << log2nx) + ((i + sh0) & mx)] = b0[q] + v[q].x;
          out[((size_t)j1 << log2nx) + ((i + sh1) & mx)] = b1[q] + v[q].y;
        }
      }
    }
  }
  cp_async_wait_all();
  // the next step's state; no CTA of this launch reads it
  if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_state_set(D, D.st->n + 1);
}

// ----------------------------------------------------------------- launchers
// the row kernels by variant P (points per thread; FP64 has P = 8 only) and
// mode (0: phi, 1: g or flow), each compiled separately
// the forward row kernels by P and mode (1: g, 2: omega into xs_w)
template <class T, int LN>
const void* rowfwd_fn(int P, int mode) {
  if constexpr (sizeof(T) == 4) {
    if (P == 16) return mode == 1 ? (const void*)k_rowfwd<T, LN, 16, 1> : (const void*)k_rowfwd<T, LN, 16, 2>;
  }
  return mode == 1 ? (const void*)k_rowfwd<T, LN, 8, 1> : (const void*)k_rowfwd<T, LN, 8, 2>;
}
template <class T, int LN>
const void* rowinv_fn(int P, int mode) {
  if constexpr (sizeof(T) == 4) {
    if (P == 16) return mode == 0 ? (const void*)k_rowinv<T, LN, 16, 0> : (const void*)k_rowinv<T, LN, 16, 1>;
  }
  return mode == 0 ? (const void*)k_rowinv<T, LN, 8, 0> : (const void*)k_rowinv<T, LN, 8, 1>;
}

template <class T, int LN>
const void* stage1_fn(int P) {
  if constexpr (sizeof(T) == 4) {
    if (P == 16) return (const void*)k_stage1_rows<T, LN, 16>;
  }
  return (const void*)k_stage1_rows<T, LN, 8>;
}

template <class T>
void launch_row_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                       const LaunchCfg& c, cudaStream_t st) {
  if (kind == KIND_STAGE1) {
    const dim3 grid(c.grid_x, nmem);
    with_log2n(log2nx, [&](auto L) {
      constexpr int LN = decltype(L)::value;
      const MemberDesc* dd = d;
      const cplx<T>* tt = tw;
      void* args[] = {(void*)&dd, (void*)&log2ny, (void*)&tt};
      cudaLaunchKernel(stage1_fn<T, LN>(c.variant), grid, dim3(c.threads), args, c.smem, st);
    });
    return;
  }
  const dim3 grid(c.grid_x, nmem);
  const bool fwd = kind == KIND_STAGE2 || kind == KIND_ROWFWD_OMEGA;
  const int mode = fwd ? (kind == KIND_ROWFWD_OMEGA ? 2 : 1) : (kind == KIND_ROWINV_PHI ? 0 : 1);
  with_log2n(log2nx, [&](auto L) {
    constexpr int LN = decltype(L)::value;
    const void* f = fwd ? rowfwd_fn<T, LN>(c.variant, mode) : rowinv_fn<T, LN>(c.variant, mode);
    const MemberDesc* dd = d;
    const cplx<T>* tt = tw;
    void* args[] = {(void*)&dd, (void*)&log2ny, (void*)&tt};
    cudaLaunchKernel(f, grid, dim3(c.threads), args, c.smem, st);
  });
}

template <class T>
int row_kernel_occupancy(int kind, int log2nx, int variant, int threads, size_t smem) {
  int nb = 0;
  if (kind == KIND_STAGE1) {
    with_log2n(log2nx, [&](auto L) {
      constexpr int LN = decltype(L)::value;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage1_fn<T, LN>(variant), threads, smem) != cudaSuccess)
        nb = 1;
    });
    return nb < 1 ? 1 : nb;
  }
  const bool fwd = kind == KIND_STAGE2;
  const int mode = fwd ? 1 : (kind == KIND_ROWINV_PHI ? 0 : 1);
  with_log2n(log2nx, [&](auto L) {
    constexpr int LN = decltype(L)::value;
    const void* f = fwd ? rowfwd_fn<T, LN>(variant, mode) : rowinv_fn<T, LN>(variant, mode);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) nb = 1;
  });
  return nb < 1 ? 1 : nb;
}

template <class T>
void set_row_smem_limits(int lim) {
  for (int ln = 4; ln <= LOG2_NMAX; ++ln)
    with_log2n(ln, [&](auto L) {
      constexpr int LN = decltype(L)::value;
      for (int P : {8, 16})
        cudaFuncSetAttribute(stage1_fn<T, LN>(P), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      for (int P : {8, 16})
        for (int mode : {0, 1, 2}) {
          if (mode > 0)
            cudaFuncSetAttribute(rowfwd_fn<T, LN>(P, mode), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
          if (mode < 2)
            cudaFuncSetAttribute(rowinv_fn<T, LN>(P, mode), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        }
    });
}

#define SHF_ROW_INST(T)                                                                                   \
  template void launch_row_kernel<T>(int, const MemberDesc*, int, int, int, const cplx<T>*, const LaunchCfg&, \
                                     cudaStream_t);                                                        \
  template int row_kernel_occupancy<T>(int, int, int, int, size_t);                                        \
  template void set_row_smem_limits<T>(int);

SHF_ROW_INST(float)
SHF_ROW_INST(double)

}  // namespace shf
