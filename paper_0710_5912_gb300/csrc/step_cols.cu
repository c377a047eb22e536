// Column (y) passes of a step: k_colpass_pair (FP32, two-mode chunks) and
// k_colpass (FP64, one mode per chunk), compiled per column length ny = 2^LN.
// See step_kernels.cu for the step's kernels and the x-spectral layout.
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

// The FP32 column pass body for one compile-time kind (0: phi; 1: inertial flow; 2:
// Stokes flow), so no per-point branch on the mode or the member's regime.
template <int LN, int KIND>
__device__ __forceinline__ void colpass_pair_body(const MemberDesc& D, int log2nx, const float2* __restrict__ tw,
                                                  unsigned char* smem_raw) {
  constexpr int log2ny = LN;
  constexpr bool two = KIND != 2;                       // second input field
  using T = float;
  using C = float2;
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tc = ny >> kLogP;
  const int ipc = blockDim.x / Tc;
  const int inst = threadIdx.x / Tc, t = threadIdx.x - inst * Tc;
  const int nitems = nx >> 2;
  const int stride = gridDim.x * ipc;
  unsigned char* base = smem_raw + (size_t)inst * colpass_inst_bytes(ny, sizeof(T));
  float4* st0 = reinterpret_cast<float4*>(base);
  float4* st1 = st0 + ny;
  float4* buf = st1 + ny;
  float4* in0 = static_cast<float4*>(KIND == 0 ? D.xs_phi : D.xs_g);
  float4* in1 = static_cast<float4*>(KIND == 0 ? D.xs_f : D.xs_w);
  float2* tws = reinterpret_cast<float2*>(smem_raw + (size_t)ipc * colpass_inst_bytes(ny, sizeof(T)));
  stage_tables_to_smem(tws, tw, log2ny, kLogP, threadIdx.x, blockDim.x);

  auto issue = [&](int cb) {
    if (cb < nitems) {
      copy_async(st0, in0 + (size_t)cb * ny, ny * 16, t, Tc);
      if (two) copy_async(st1, in1 + (size_t)cb * ny, ny * 16, t, Tc);
    }
    cp_async_commit();
  };

  const ColConsts<T> K(D, KIND == 0 ? 0 : 1, ny);
  const int iters = persistent_iters(nitems, ipc);
  int cb = blockIdx.x * ipc + inst;
  issue(cb);
  for (int it = 0; it < iters; ++it, cb += stride) {
    const bool active = cb < nitems;
    cp_async_wait_all();
    __syncthreads();
    C a0[kP], b0[kP], a1[kP], b1[kP];                   // a: mode 2cb, b: mode 2cb+1; 0/1: the two fields
#pragma unroll
    for (int q = 0; q < kP; ++q) {
      const float4 x = st0[t + q * Tc];
      a0[q] = C{x.x, x.y};
      b0[q] = C{x.z, x.w};
    }
    if (two) {
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        const float4 x = st1[t + q * Tc];
        a1[q] = C{x.x, x.y};
        b1[q] = C{x.z, x.w};
      }
    }
    __syncthreads();                                    // stage free
    issue(cb + stride);
    fft_reg2<false>(a0, b0, log2ny, t, buf, tws);
    if (two) fft_reg2<false>(a1, b1, log2ny, t, buf, tws);
    const int m0 = active ? 2 * cb : 0, m1 = m0 + 1;
    const double qa_d = m0 * K.qx_unit, qb_d = m1 * K.qx_unit;
    const T qa = (T)qa_d, qb = (T)qb_d;
    const T sqa = (T)(K.s_d * qa_d), sqb = (T)(K.s_d * qb_d);   // s q_x formed in double
#pragma unroll
    for (int q = 0; q < kP; ++q) {
      col_multiply_k<KIND>(K, m0, qa, sqa, t + q * Tc, a0[q], a1[q]);
      col_multiply_k<KIND>(K, m1, qb, sqb, t + q * Tc, b0[q], b1[q]);
    }
    fft_reg2<true>(a0, b0, log2ny, t, buf, tws);
    if (active) {
      float4* o = in0 + (size_t)cb * ny;
#pragma unroll
      for (int q = 0; q < kP; ++q) o[t + q * Tc] = make_float4(a0[q].x, a0[q].y, b0[q].x, b0[q].y);
    }
    if (KIND == 1) {
      fft_reg2<true>(a1, b1, log2ny, t, buf, tws);
      if (active) {
        float4* o = in1 + (size_t)cb * ny;
#pragma unroll
        for (int q = 0; q < kP; ++q) o[t + q * Tc] = make_float4(a1[q].x, a1[q].y, b1[q].x, b1[q].y);
      }
    }
  }
  cp_async_wait_all();
}

// FP32 column pass over whole chunks: item cb = the two modes m = 2cb, 2cb+1,
// whose ny rows are one contiguous 16-byte-per-row run in the x-spectral
// layout.  Both columns are staged with 16-byte copies, transformed in lock
// step (shared twiddles, 16-byte exchanges) and written back as whole 16-byte
// rows, so no sector is touched twice.  The kind is uniform per CTA (one
// member per blockIdx.y).
// KIND 0-2 as colpass_pair_body; KIND 3: flow for a launch whose members mix
// both regimes (the body is chosen per CTA).  One kernel per kind, so each
// gets its own register allocation.
template <int LN, int KIND>
__global__ void __launch_bounds__(512, 1) k_colpass_pair(const MemberDesc* __restrict__ descs, int log2nx,
                                                        const float2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  if (KIND != 3) colpass_pair_body<LN, KIND>(D, log2nx, tw, smem_raw);
  else if (D.stokes) colpass_pair_body<LN, 2>(D, log2nx, tw, smem_raw);
  else colpass_pair_body<LN, 1>(D, log2nx, tw, smem_raw);
}
template <int LN>
const void* colpass_pair_fn(int kind) {
  switch (kind) {
    case 0: return (const void*)k_colpass_pair<LN, 0>;
    case 1: return (const void*)k_colpass_pair<LN, 1>;
    case 2: return (const void*)k_colpass_pair<LN, 2>;
    default: return (const void*)k_colpass_pair<LN, 3>;
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
      // variant of the flow pass: 1 inertial members, 2 Stokes, 3 mixed
      const int k = mode == 0 ? 0 : (c.variant >= 1 && c.variant <= 3 ? c.variant : 3);
      switch (k) {
        case 0: k_colpass_pair<LN, 0><<<grid, c.threads, c.smem, st>>>(d, log2nx, tw); break;
        case 1: k_colpass_pair<LN, 1><<<grid, c.threads, c.smem, st>>>(d, log2nx, tw); break;
        case 2: k_colpass_pair<LN, 2><<<grid, c.threads, c.smem, st>>>(d, log2nx, tw); break;
        default: k_colpass_pair<LN, 3><<<grid, c.threads, c.smem, st>>>(d, log2nx, tw); break;
      }
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
    if constexpr (sizeof(T) == 4) f = colpass_pair_fn<LN>(3);
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
        for (int k = 0; k < 4; ++k)
          cudaFuncSetAttribute(colpass_pair_fn<LN>(k), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
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
