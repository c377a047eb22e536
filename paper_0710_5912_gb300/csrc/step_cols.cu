// Column (y) passes of a step, compiled per column length ny = 2^LN: in FP32
// k_colpass_chunk (ny >= 512: a two-mode chunk per CTA, one 16-point
// instance per mode) and k_colpass_single (shorter columns: one mode per
// instance), both with radix-16 stages; in FP64 k_colpass (one mode per
// 16-byte chunk, 8 points per thread).  The force's low modes (k_lowmode_cols)
// are here too.  See step_kernels.cu for the step's kernels and the
// x-spectral layout.
#include "step_common.cuh"

namespace shf {

// ============================================================ column passes
// Work items: columns m = 0..nx/2-1, one column per instance (ny/8 threads).
// The two input columns of the next item stream into the staging buffer while
// the current one is transformed.  mode 0: phi (inputs phi*, f -> increment
// of phi); mode 1: flow (g, omega* -> psi, increment of omega; Stokes: g ->
// psi).
template <class T>
__device__ __forceinline__ void stage_column(cplx<T>* st, const cplx<T>* __restrict__ src, int m, int ny, int t,
                                             int Tc) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  if (LC == 0) {
    copy_async(st, src + (size_t)m * ny, ny * (int)sizeof(C), t, Tc);
  } else {
    for (int n = t; n < ny; n += Tc) cp_async8(st + n, src + xs_idx(n, m, ny, LC));
  }
}

// Constants of the column-pass multipliers (Appendix B item 1 for mode 0;
// Eq. forOmega with the Poisson solve, or the Stokes solve, for mode 1).
template <class T>
struct ColConsts {
  T norm, qyu, caM, cbM, ckM, cnu, dt;
  double qx_unit, s_d;
  int ny;
  bool stokes;
  __device__ __forceinline__ ColConsts(const MemberDesc& D, int mode, int ny_)
      : norm((T)D.inv_nxny), qyu((T)D.qy_unit), caM((T)D.c_dt_aM), cbM((T)D.c_dt_bM), ckM((T)D.c_hdt_kM),
        cnu((T)D.c_hdt_nu), dt((T)D.dt), qx_unit(D.qx_unit),
        s_d(mode == 0 ? D.st->s0 : D.st->s1),        // s^n for phi, s^{n+1} for flow
        ny(ny_), stokes(D.stokes != 0) {}
};

// Quotients of the multipliers: FP32 takes the hardware reciprocal
// (__fdividef, within 2 ulp; the divisors here lie in [1e-12, 1e3]), FP64 the
// IEEE quotient.
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double quot(double a, double b) { return a / b; }

// The multiplier at mode (m, row nn) of the column transform, in place, for a
// compile-time pass kind (0: phi; 1: inertial flow; 2: Stokes flow):
// kind 0: va = phi*_hat -> increment of phi_hat (x norm), vb = f_hat;
// kinds 1-2: va = g_hat -> psi_hat (x norm), vb = omega*_hat -> increment (x norm).
// qx = m q_unit and sqx = s q_x, both formed in double.
template <int KIND, class T>
__device__ __forceinline__ void col_multiply_k(const ColConsts<T>& K, int m, T qx, T sqx, int nn, cplx<T>& va,
                                               cplx<T>& vb) {
  using C = cplx<T>;
  const int ns = nn < (K.ny >> 1) ? nn : nn - K.ny;
  const T ky = (T)ns * K.qyu - sqx;
  const T k2 = qx * qx + ky * ky;
  const bool nyq_row = nn == (K.ny >> 1);
  const T norm = K.norm;
  if (KIND == 0) {
    const C P = va, F = vb;
    if (nyq_row) {
      va = C{-P.x * norm, -P.y * norm};                 // Nyquist row of phi^{n+1} -> 0
    } else {
      const T c4 = K.ckM * (k2 * k2);
      const T aa = K.caM * k2 - T(2) * c4;
      const T bbm = K.cbM * k2;
      const T inv = quot(norm, T(1) + c4);
      va = C{(aa * P.x - bbm * F.x) * inv, (aa * P.y - bbm * F.y) * inv};
    }
  } else {
    const bool zero = nyq_row || (m == 0 && nn == 0);
    const C G = va;
    if (KIND == 2) {
      const T inv = zero ? T(0) : quot(norm, k2 * k2);
      va = C{G.x * inv, G.y * inv};
    } else {
      const C Wv = vb;
      if (zero) {
        va = C{T(0), T(0)};
        vb = C{-Wv.x * norm, -Wv.y * norm};             // omega^{n+1} -> 0 there
      } else {
        const T cc = K.cnu * k2;
        const T inv = quot(T(1), T(1) + cc);
        const C dw = C{(-T(2) * cc * Wv.x + K.dt * G.x) * inv, (-T(2) * cc * Wv.y + K.dt * G.y) * inv};
        const T ik = quot(norm, k2);
        va = C{(Wv.x + dw.x) * ik, (Wv.y + dw.y) * ik};
        vb = C{dw.x * norm, dw.y * norm};
      }
    }
  }
}
// FP32 inertial members: omega carried in 2D spectral form (w_hat).  At mode
// (m, row nn): va = g_hat, vb = the transform of the advective increment A,
// Wn = omega_hat^n (relabelled at a wrap).  omega* = Wn + A and Eq. forOmega
// in increment form, omega^{n+1} = omega* + (dt g - 2 C omega*) / (1 + C),
// C = dt nu k^2 / 2, then psi = omega^{n+1} / k^2.  Returns omega^{n+1}
// (unnormalised, the new w_hat); va <- psi_hat norm, vb <- omega^{n+1} norm,
// the inputs of the inverse column transforms.  Every mode is stored as its
// own FP32 number from step to step, so each keeps its own relative
// precision; the real omega of the stencils is derived from w_hat.
__device__ __forceinline__ float2 col_multiply_wspec(const ColConsts<float>& K, int m, float qx, float sqx, int nn,
                                                     float2& va, float2& vb, float2 Wn) {
  const int ns = nn < (K.ny >> 1) ? nn : nn - K.ny;
  const float ky = (float)ns * K.qyu - sqx;
  const float k2 = qx * qx + ky * ky;
  if (nn == (K.ny >> 1) || (m == 0 && nn == 0)) {     // Nyquist row and k = 0: omega = psi = 0
    va = float2{0.f, 0.f};
    vb = float2{0.f, 0.f};
    return float2{0.f, 0.f};
  }
  const float2 G = va, A = vb;
  const float2 Ws = float2{Wn.x + A.x, Wn.y + A.y};
  const float cc = K.cnu * k2;
  const float inv = quot(1.f, 1.f + cc);
  const float2 W1 = float2{Ws.x + (K.dt * G.x - 2.f * cc * Ws.x) * inv, Ws.y + (K.dt * G.y - 2.f * cc * Ws.y) * inv};
  const float ik = quot(K.norm, k2);
  va = float2{W1.x * ik, W1.y * ik};
  vb = float2{W1.x * K.norm, W1.y * K.norm};
  return W1;
}

// FP32: g_hat at (m, row nn) from low_hat when the mode lies in the low window
// (the force's transform there carries the rounding of the row transform's
// compensated low modes only, see low_row_modes in step_rows.cu)
__device__ __forceinline__ void low_override(const MemberDesc& D, int m, int nn, int ny, float2& v) {
  if (m > D.lowm) return;
  const int ns = nn < (ny >> 1) ? nn : nn - ny;
  if (ns < -D.lown || ns > D.lown) return;
  v = static_cast<const float2*>(D.low_hat)[m * (2 * D.lown + 1) + ns + D.lown];
}

// the same with the kind chosen at run time (mode 0 or 1, and K.stokes)
template <class T>
__device__ __forceinline__ void col_multiply(int mode, const ColConsts<T>& K, int m, T qx, T sqx, int nn,
                                             cplx<T>& va, cplx<T>& vb) {
  if (mode == 0) col_multiply_k<0>(K, m, qx, sqx, nn, va, vb);
  else if (K.stokes) col_multiply_k<2>(K, m, qx, sqx, nn, va, vb);
  else col_multiply_k<1>(K, m, qx, sqx, nn, va, vb);
}

template <class T, int LN>
__global__ void __launch_bounds__(512, min_ctas<T>()) k_colpass(const MemberDesc* __restrict__ descs, int log2nx,
                                                                const cplx<T>* __restrict__ tw, int mode) {
  constexpr int log2ny = LN;
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tc = ny >> kLogP;
  const int ipc = blockDim.x / Tc;
  const int inst = threadIdx.x / Tc, t = threadIdx.x - inst * Tc;
  const int nitems = nx >> 1;
  const int stride = gridDim.x * ipc;
  const bool stokes = D.stokes != 0;
  const bool two = mode == 0 || !stokes;                // second input column
  unsigned char* base = smem_raw + (size_t)inst * colpass_inst_bytes(ny, sizeof(T));
  C* st0 = reinterpret_cast<C*>(base);
  C* st1 = st0 + ny;
  C* buf = st1 + ny;
  C* in0 = static_cast<C*>(mode == 0 ? D.xs_phi : D.xs_g);
  C* in1 = static_cast<C*>(mode == 0 ? D.xs_f : D.xs_w);
  C* tws = reinterpret_cast<C*>(smem_raw + (size_t)ipc * colpass_inst_bytes(ny, sizeof(T)));
  stage_tables_to_smem(tws, tw, log2ny, kLogP, threadIdx.x, blockDim.x);

  auto issue = [&](int m) {
    if (m < nitems) {
      stage_column<T>(st0, in0, m, ny, t, Tc);
      if (two) stage_column<T>(st1, in1, m, ny, t, Tc);
    }
    cp_async_commit();
  };

  const ColConsts<T> K(D, mode, ny);

  const int iters = persistent_iters(nitems, ipc);
  int m = blockIdx.x * ipc + inst;
  issue(m);
  for (int it = 0; it < iters; ++it, m += stride) {
    const bool active = m < nitems;
    cp_async_wait_all();
    __syncthreads();
    C va[kP], vb[kP];
    const int mm = active ? m : 0;
#pragma unroll
    for (int q = 0; q < kP; ++q) va[q] = st0[t + q * Tc];
    if (two) {
#pragma unroll
      for (int q = 0; q < kP; ++q) vb[q] = st1[t + q * Tc];
    }
    __syncthreads();                                    // stage free
    issue(m + stride);
    fft_reg<false>(va, log2ny, t, buf, tws);
    if (two) fft_reg<false>(vb, log2ny, t, buf, tws);
    const double qx_d = mm * K.qx_unit;
    const T qx = (T)qx_d;
    const T sqx = (T)(K.s_d * qx_d);                    // s q_x formed in double
#pragma unroll
    for (int q = 0; q < kP; ++q) col_multiply<T>(mode, K, mm, qx, sqx, t + q * Tc, va[q], vb[q]);
    fft_reg<true>(va, log2ny, t, buf, tws);
    if (active) {
#pragma unroll
      for (int q = 0; q < kP; ++q) in0[xs_idx(t + q * Tc, m, ny, LC)] = va[q];
    }
    if (mode == 1 && !stokes) {
      fft_reg<true>(vb, log2ny, t, buf, tws);
      if (active) {
#pragma unroll
        for (int q = 0; q < kP; ++q) in1[xs_idx(t + q * Tc, m, ny, LC)] = vb[q];
      }
    }
  }
  cp_async_wait_all();
}

// Error-free transformations in FP32 (Knuth's TwoSum; the product's error by
// one fused multiply-add) for the double-float sums of k_lowmode_cols.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float ph, float pl) {
  const float s = __fadd_rn(hi, ph);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pl));
}
// a (b_hi + b_lo) as hi + lo: the rounded product, its exact error and the
// product with the low part
__device__ __forceinline__ void ff_mul(float a, float bh, float bl, float& ph, float& pl) {
  ph = __fmul_rn(a, bh);
  pl = __fmaf_rn(a, bl, __fmaf_rn(a, bh, -ph));
}

// The column DFT of the low row modes of g (FP32 members):
//   low_hat[m][n + lown] = sum_j low_rows[m][j] exp(-2 pi i n j / ny),
// m <= lowm, |n| <= lown.  Each term is the product of an FP32 coefficient
// (a double-float one for the exact Stokes rows, low == 2, whose low part
// adds one fused multiply-add) with a double-float twiddle, formed without
// rounding error to about 2^-48,
// and the four real sums (Re r cos, Im r sin, Im r cos, Re r sin) are
// double-float sums (TwoSum), so the result carries essentially only the
// rounding of the coefficients themselves.  A CTA holds one output; its
// eight warps share the rows in eighths (lanes coalesced along j, each lane's
// rows loaded at once); lanes and warps are folded in a fixed order, as float
// pairs.
constexpr int kLowColsWarps = 8;
// U rows per lane per round, all their loads in flight at once; the launcher
// takes U = ny / 256 (one round per warp), 1..16
template <int U>
__global__ void __launch_bounds__(kLowColsWarps * 32) k_lowmode_cols(const MemberDesc* __restrict__ descs,
                                                                     int log2ny, const float4* __restrict__ twff) {
  const MemberDesc& D = descs[blockIdx.y];
  if (!D.low) return;                                  // uniform per CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int o = blockIdx.x;
  const int nn = 2 * D.lown + 1;
  if (o >= (D.lowm + 1) * nn) return;                  // uniform per CTA
  const int m = o / nn, ns = o - m * nn - D.lown;
  const int ny = 1 << log2ny;
  const int tshift = LOG2_NMAX - log2ny;
  const int step = ns & (ny - 1);
  const int rows = ny / kLowColsWarps > 0 ? ny / kLowColsWarps : 1;
  const int j0 = warp * rows, j1 = min(ny, j0 + rows);
  const float2* lr = static_cast<const float2*>(D.low_rows) + ((size_t)m << log2ny);
  // low parts of the coefficients (low == 2: exact Stokes rows), else none
  const float2* lrl = D.low == 2 ? lr + ((size_t)(kLowM + 1) << log2ny) : nullptr;
  float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
  for (int jb = j0; jb < j1; jb += 32 * U) {
    float2 r[U], rl[U];
    float4 w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = jb + u * 32 + lane;
      const bool in = j < j1;
      r[u] = in ? lr[j] : float2{0.f, 0.f};
      rl[u] = in && lrl ? lrl[j] : float2{0.f, 0.f};
      w[u] = in ? __ldg(twff + (((step * j) & (ny - 1)) << tshift)) : float4{1.f, 0.f, 0.f, 0.f};
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float ph, pl;
      ff_mul(r[u].x, w[u].x, w[u].y, ph, pl);          // Re r cos
      ff_add(h[0], l[0], ph, __fmaf_rn(rl[u].x, w[u].x, pl));
      ff_mul(r[u].y, w[u].z, w[u].w, ph, pl);          // Im r sin
      ff_add(h[1], l[1], ph, __fmaf_rn(rl[u].y, w[u].z, pl));
      ff_mul(r[u].y, w[u].x, w[u].y, ph, pl);          // Im r cos
      ff_add(h[2], l[2], ph, __fmaf_rn(rl[u].y, w[u].x, pl));
      ff_mul(r[u].x, w[u].z, w[u].w, ph, pl);          // Re r sin
      ff_add(h[3], l[3], ph, __fmaf_rn(rl[u].x, w[u].z, pl));
    }
  }
  // fold the lanes pairwise in a fixed tree, every sum kept as a float pair
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float oh = __shfl_down_sync(0xffffffffu, h[k], off), ol = __shfl_down_sync(0xffffffffu, l[k], off);
      if (lane < off) ff_add(h[k], l[k], oh, ol);
    }
  }
  __shared__ float part[kLowColsWarps][8];
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      part[warp][k] = h[k];
      part[warp][4 + k] = l[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {                              // the warps in order
    float H[4] = {0.f, 0.f, 0.f, 0.f}, L[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < kLowColsWarps; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) ff_add(H[k], L[k], part[q][k], part[q][4 + k]);
    // r conj(w): Re = Re r cos + Im r sin, Im = Im r cos - Re r sin
    ff_add(H[0], L[0], H[1], L[1]);
    ff_add(H[2], L[2], -H[3], -L[3]);
    static_cast<float2*>(D.low_hat)[o] = float2{__fadd_rn(H[0], L[0]), __fadd_rn(H[2], L[2])};
  }
}

void launch_lowmode_cols(const MemberDesc* d, int nmem, int log2ny, const float4* twff, cudaStream_t st) {
  const int outs = (kLowM + 1) * (2 * kLowN + 1);
  const dim3 grid(outs, nmem);
  const int u = (1 << log2ny) / (kLowColsWarps * 32);
  if (u >= 16) k_lowmode_cols<16><<<grid, kLowColsWarps * 32, 0, st>>>(d, log2ny, twff);
  else if (u >= 8) k_lowmode_cols<8><<<grid, kLowColsWarps * 32, 0, st>>>(d, log2ny, twff);
  else if (u >= 4) k_lowmode_cols<4><<<grid, kLowColsWarps * 32, 0, st>>>(d, log2ny, twff);
  else if (u >= 2) k_lowmode_cols<2><<<grid, kLowColsWarps * 32, 0, st>>>(d, log2ny, twff);
  else k_lowmode_cols<1><<<grid, kLowColsWarps * 32, 0, st>>>(d, log2ny, twff);
}

// The FP32 column pass on single mode columns (ny < 512): item m = one mode,
// its ny rows staged with 8-byte copies from the two-mode chunk layout,
// transformed with 16 points per thread (radix-16 stages), multiplied,
// transformed back and stored 8 bytes per row.  Several instances share a
// CTA.  Kinds: 0: phi; 1: inertial flow with w_hat; 2: Stokes flow; 4:
// omega's forward column transform into w_hat (3: mixed, chosen per CTA).
template <int LN, int KIND>
__device__ __forceinline__ void colpass_single_body(const MemberDesc& D, int log2nx, const float2* __restrict__ tw,
                                                    unsigned char* smem_raw) {
  constexpr int log2ny = LN;
  constexpr int P = 16;
  constexpr bool two = KIND == 0 || KIND == 1;          // second input field
  using T = float;
  using C = float2;
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tc = ny / P;
  const int ipc = blockDim.x / Tc;
  const int inst = threadIdx.x / Tc, t = threadIdx.x - inst * Tc;
  const int nitems = KIND == 4 && !D.wspec ? 0 : nx >> 1;
  const int stride = gridDim.x * ipc;
  unsigned char* base = smem_raw + (size_t)inst * colsingle_inst_bytes(ny);
  C* st0 = reinterpret_cast<C*>(base);
  C* st1 = st0 + ny;
  C* buf = st1 + ny;
  C* in0 = static_cast<C*>(KIND == 0 ? D.xs_phi : (KIND == 4 ? D.xs_w : D.xs_g));
  C* in1 = static_cast<C*>(KIND == 0 ? D.xs_f : D.xs_w);
  C* what = static_cast<C*>(D.w_hat);
  // a wrap during the step relabels omega_hat^n: (m, n) <- (m, n + m dK)
  const int dK = (KIND == 1 && D.remap) ? (int)(D.st->dK & (ny - 1)) : 0;
  C* tws = reinterpret_cast<C*>(smem_raw + (size_t)ipc * colsingle_inst_bytes(ny));
  stage_tables_to_smem(tws, tw, log2ny, 4, threadIdx.x, blockDim.x);

  auto issue = [&](int m) {
    if (m < nitems) {
      for (int n = t; n < ny; n += Tc) {
        cp_async8(st0 + n, in0 + xs_idx(n, m, ny, 1));
        if (two) cp_async8(st1 + n, in1 + xs_idx(n, m, ny, 1));
      }
    }
    cp_async_commit();
  };

  const ColConsts<T> K(D, KIND == 0 ? 0 : 1, ny);
  const int iters = persistent_iters(nitems, ipc);
  int m = blockIdx.x * ipc + inst;
  issue(m);
  for (int it = 0; it < iters; ++it, m += stride) {
    const bool active = m < nitems;
    cp_async_wait_all();
    __syncthreads();
    C a[P], b[P];                                       // the two fields of mode m, rows t + q Tc
#pragma unroll
    for (int q = 0; q < P; ++q) a[q] = st0[t + q * Tc];
    if (two) {
#pragma unroll
      for (int q = 0; q < P; ++q) b[q] = st1[t + q * Tc];
    }
    __syncthreads();                                    // stage free
    issue(m + stride);
    fft_reg<false>(a, log2ny, t, buf, tws);
    if (two) fft_reg<false>(b, log2ny, t, buf, tws);
    const int mm = active ? m : 0;
    if (KIND == 4) {                                    // omega's 2D transform: the new w_hat
      if (active) {
#pragma unroll
        for (int q = 0; q < P; ++q) what[xs_idx(t + q * Tc, mm, ny, 1)] = a[q];
      }
      continue;
    }
    if ((KIND == 1 || KIND == 2) && D.low && mm <= D.lowm) {   // the force's low modes
#pragma unroll
      for (int q = 0; q < P; ++q) low_override(D, mm, t + q * Tc, ny, a[q]);
    }
    const double q_d = mm * K.qx_unit;
    const T qx = (T)q_d;
    const T sqx = (T)(K.s_d * q_d);                     // s q_x formed in double
    if (KIND == 1) {
      if (dK) {                                         // stage omega_hat^n so that rows can be relabelled
#pragma unroll
        for (int q = 0; q < P; ++q) buf[pad16(t + q * Tc)] = what[xs_idx(t + q * Tc, mm, ny, 1)];
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int nn = t + q * Tc;
        const C Wn = dK ? buf[pad16((nn + mm * dK) & (ny - 1))] : what[xs_idx(nn, mm, ny, 1)];
        const C Nw = col_multiply_wspec(K, mm, qx, sqx, nn, a[q], b[q], Wn);
        if (active) what[xs_idx(nn, mm, ny, 1)] = Nw;
      }
      if (dK) __syncthreads();                          // buf is the exchange buffer again
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) col_multiply_k<KIND>(K, mm, qx, sqx, t + q * Tc, a[q], b[q]);
    }
    fft_reg<true>(a, log2ny, t, buf, tws);
    if (active) {
#pragma unroll
      for (int q = 0; q < P; ++q) in0[xs_idx(t + q * Tc, mm, ny, 1)] = a[q];
    }
    if (KIND == 1) {
      fft_reg<true>(b, log2ny, t, buf, tws);
      if (active) {
#pragma unroll
        for (int q = 0; q < P; ++q) in1[xs_idx(t + q * Tc, mm, ny, 1)] = b[q];
      }
    }
  }
  cp_async_wait_all();
}

// The FP32 column pass on whole two-mode chunks for long columns (ny >= 512):
// the CTA stages a chunk's ny 16-byte rows of each input field (whole
// sectors), and two 16-point instances of ny/16 threads each take one mode,
// transform, multiply and transform back on their own exchange buffers,
// synchronising on their own named barriers (1 and 2), so neither waits for
// the other's stages.  The results of the two modes meet in the (then idle)
// exchange buffers and leave as whole 16-byte rows; the CTA synchronises only
// there and at the item boundaries.  Kinds as colpass_single_body.
template <int LN, int KIND>
__device__ __forceinline__ void colpass_chunk_body(const MemberDesc& D, int log2nx, const float2* __restrict__ tw,
                                                   unsigned char* smem_raw) {
  constexpr int log2ny = LN;
  constexpr int ny = 1 << LN;
  constexpr int P = 16;
  constexpr int Tc = ny / P;                            // threads of one mode's instance (>= 32)
  constexpr bool two = KIND == 0 || KIND == 1;
  using T = float;
  using C = float2;
  const int nx = 1 << log2nx;
  const int sub = threadIdx.x / Tc, t = threadIdx.x - sub * Tc;
  const NamedSync sync{1 + sub, Tc};
  const int nitems = KIND == 4 && !D.wspec ? 0 : nx >> 2;
  const int stride = gridDim.x;
  float4* st0 = reinterpret_cast<float4*>(smem_raw);
  float4* st1 = st0 + ny;
  C* buf = reinterpret_cast<C*>(st1 + ny) + (size_t)sub * padded_len(ny);
  // after the transforms the two exchange buffers together hold one chunk's
  // ny 16-byte rows: the two modes' results meet there and leave as whole rows
  float4* ost = reinterpret_cast<float4*>(st1 + ny);
  C* in0 = static_cast<C*>(KIND == 0 ? D.xs_phi : (KIND == 4 ? D.xs_w : D.xs_g));
  C* in1 = static_cast<C*>(KIND == 0 ? D.xs_f : D.xs_w);
  C* what = static_cast<C*>(D.w_hat);
  const int dK = (KIND == 1 && D.remap) ? (int)(D.st->dK & (ny - 1)) : 0;
  C* tws = reinterpret_cast<C*>(smem_raw + colchunk_cta_bytes(ny));
  stage_tables_to_smem(tws, tw, log2ny, 4, threadIdx.x, blockDim.x);

  // mode sub's values v[q] (rows t + q Tc) of chunk cb -> dst as whole 16-byte rows
  auto store_rows = [&](const C (&v)[P], C* dst, int cb, bool active) {
    __syncthreads();                                   // both modes' transforms are done with the buffers
#pragma unroll
    for (int q = 0; q < P; ++q) reinterpret_cast<C*>(ost + t + q * Tc)[sub] = v[q];
    __syncthreads();
    if (active) {
      float4* o = reinterpret_cast<float4*>(dst) + (size_t)cb * ny;
      for (int n = threadIdx.x; n < ny; n += blockDim.x) o[n] = ost[n];
    }
    __syncthreads();                                   // ost is the exchange buffers again
  };

  // each field's chunk is one contiguous run of ny 16-byte rows: one thread
  // stages it with a bulk copy completed on the CTA's mbarrier (after the
  // twiddle table, kColBarBytes of the launch's dynamic shared memory)
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + colchunk_cta_bytes(ny) +
                                                                  stage_table_bytes(log2ny, 4, sizeof(float)));
  unsigned phase = 0;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int cb) {
    if (cb < nitems && threadIdx.x == 0) {
      fence_proxy_async_smem();                         // the stage's earlier reads come first
      mbar_arrive_expect_tx(bar, (two ? 2u : 1u) * ny * 16u);
      bulk_g2s(st0, reinterpret_cast<const float4*>(in0) + (size_t)cb * ny, ny * 16u, bar);
      if (two) bulk_g2s(st1, reinterpret_cast<const float4*>(in1) + (size_t)cb * ny, ny * 16u, bar);
      // the inertial flow pass reads the chunk's omega_hat^n in its multiply: into L2 now
      if (KIND == 1 && D.wspec) l2_prefetch(reinterpret_cast<const float4*>(what) + (size_t)cb * ny, ny * 16u);
    }
  };

  const ColConsts<T> K(D, KIND == 0 ? 0 : 1, ny);
  const int iters = persistent_iters(nitems, 1);
  int cb = blockIdx.x;
  issue(cb);
  for (int it = 0; it < iters; ++it, cb += stride) {
    const bool active = cb < nitems;
    bool ok = true;
    if (active) {
      ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
    }
    if (!__syncthreads_and(ok)) {                       // the chunk never arrived: flag it and stop
      if (threadIdx.x == 0) atomicOr(D.err, 1);
      return;
    }
    C a[P], b[P];                                       // mode 2 cb + sub of the two fields
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const float4 x = st0[t + q * Tc];
      a[q] = sub ? C{x.z, x.w} : C{x.x, x.y};
    }
    if (two) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const float4 x = st1[t + q * Tc];
        b[q] = sub ? C{x.z, x.w} : C{x.x, x.y};
      }
    }
    __syncthreads();                                    // stage free
    issue(cb + stride);
    fft_reg<false>(a, log2ny, t, buf, tws, sync);
    if (two) fft_reg<false>(b, log2ny, t, buf, tws, sync);
    const int mm = active ? 2 * cb + sub : sub;
    if (KIND == 4) {                                    // omega's 2D transform: the new w_hat
      store_rows(a, what, cb, active);
      continue;
    }
    if ((KIND == 1 || KIND == 2) && D.low && mm <= D.lowm) {   // the force's low modes
#pragma unroll
      for (int q = 0; q < P; ++q) low_override(D, mm, t + q * Tc, ny, a[q]);
    }
    const double q_d = mm * K.qx_unit;
    const T qx = (T)q_d;
    const T sqx = (T)(K.s_d * q_d);                     // s q_x formed in double
    if (KIND == 1) {
      if (dK) {                                         // stage omega_hat^n so that rows can be relabelled
#pragma unroll
        for (int q = 0; q < P; ++q) buf[pad16(t + q * Tc)] = what[xs_idx(t + q * Tc, mm, ny, 1)];
        sync();
      }
      C Nw[P];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int nn = t + q * Tc;
        const C Wn = dK ? buf[pad16((nn + mm * dK) & (ny - 1))] : what[xs_idx(nn, mm, ny, 1)];
        Nw[q] = col_multiply_wspec(K, mm, qx, sqx, nn, a[q], b[q], Wn);
      }
      store_rows(Nw, what, cb, active);                 // the new omega_hat
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) col_multiply_k<KIND>(K, mm, qx, sqx, t + q * Tc, a[q], b[q]);
    }
    fft_reg<true>(a, log2ny, t, buf, tws, sync);
    store_rows(a, in0, cb, active);
    if (KIND == 1) {
      fft_reg<true>(b, log2ny, t, buf, tws, sync);
      store_rows(b, in1, cb, active);
    }
  }
  cp_async_wait_all();
}
constexpr int colchunk_threads(int ln) { return 2 * ((1 << ln) / 16); }
template <int LN, int KIND>
__global__ void __launch_bounds__(colchunk_threads(LN), 1) k_colpass_chunk(const MemberDesc* __restrict__ descs,
                                                                           int log2nx, const float2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  if (KIND != 3) colpass_chunk_body<LN, KIND>(D, log2nx, tw, smem_raw);
  else if (D.stokes) colpass_chunk_body<LN, 2>(D, log2nx, tw, smem_raw);
  else colpass_chunk_body<LN, 1>(D, log2nx, tw, smem_raw);
}
template <int LN, int KIND>
__global__ void __launch_bounds__(256, 2) k_colpass_single(const MemberDesc* __restrict__ descs, int log2nx,
                                                           const float2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  if (KIND != 3) colpass_single_body<LN, KIND>(D, log2nx, tw, smem_raw);
  else if (D.stokes) colpass_single_body<LN, 2>(D, log2nx, tw, smem_raw);
  else colpass_single_body<LN, 1>(D, log2nx, tw, smem_raw);
}

// the FP32 column kernels of a length: the chunk kernel for ny >= 512, else
// the single-mode kernel
template <int LN>
const void* colpass_fp32_fn(int kind) {
  if constexpr (LN >= 9) {
    switch (kind) {
      case 0: return (const void*)k_colpass_chunk<LN, 0>;
      case 1: return (const void*)k_colpass_chunk<LN, 1>;
      case 2: return (const void*)k_colpass_chunk<LN, 2>;
      case 4: return (const void*)k_colpass_chunk<LN, 4>;
      default: return (const void*)k_colpass_chunk<LN, 3>;
    }
  } else {
    switch (kind) {
      case 0: return (const void*)k_colpass_single<LN, 0>;
      case 1: return (const void*)k_colpass_single<LN, 1>;
      case 2: return (const void*)k_colpass_single<LN, 2>;
      case 4: return (const void*)k_colpass_single<LN, 4>;
      default: return (const void*)k_colpass_single<LN, 3>;
    }
  }
}

// ----------------------------------------------------------------- launchers
template <class T>
void launch_col_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                       const LaunchCfg& c, cudaStream_t st) {
  const dim3 grid(c.grid_x, nmem);
  const int mode = kind == KIND_COLPASS_PHI ? 0 : 1;
  with_log2n(log2ny, [&](auto L) {
    constexpr int LN = decltype(L)::value;
    if constexpr (sizeof(T) == 4) {
      // variant of the flow pass: 1 inertial members, 2 Stokes, 3 mixed; 4: seeding w_hat
      const int k = kind == KIND_COLPASS_WINIT ? 4 : (mode == 0 ? 0 : (c.variant >= 1 && c.variant <= 3 ? c.variant : 3));
      const MemberDesc* dd = d;
      const float2* tt = tw;
      void* args[] = {(void*)&dd, (void*)&log2nx, (void*)&tt};
      cudaLaunchKernel(colpass_fp32_fn<LN>(k), grid, dim3(c.threads), args, c.smem, st);
    } else
      k_colpass<T, LN><<<grid, c.threads, c.smem, st>>>(d, log2nx, tw, mode);
  });
}

template <class T>
int col_kernel_occupancy(int log2ny, int threads, size_t smem) {
  int nb = 0;
  with_log2n(log2ny, [&](auto L) {
    constexpr int LN = decltype(L)::value;
    const void* f;
    if constexpr (sizeof(T) == 4) f = colpass_fp32_fn<LN>(3);
    else f = (const void*)k_colpass<T, LN>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) nb = 1;
  });
  return nb < 1 ? 1 : nb;
}

template <class T>
void set_col_smem_limits(int lim) {
  for (int ln = 4; ln <= LOG2_NMAX; ++ln)
    with_log2n(ln, [&](auto L) {
      constexpr int LN = decltype(L)::value;
      if constexpr (sizeof(T) == 4) {
        for (int k = 0; k < 5; ++k)
          cudaFuncSetAttribute(colpass_fp32_fn<LN>(k), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      } else
        cudaFuncSetAttribute(k_colpass<T, LN>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    });
}

#define SHF_COL_INST(T)                                                                                   \
  template void launch_col_kernel<T>(int, const MemberDesc*, int, int, int, const cplx<T>*, const LaunchCfg&, \
                                     cudaStream_t);                                                        \
  template int col_kernel_occupancy<T>(int, int, size_t);                                                  \
  template void set_col_smem_limits<T>(int);

SHF_COL_INST(float)
SHF_COL_INST(double)

}  // namespace shf
