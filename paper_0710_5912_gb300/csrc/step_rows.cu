// Row (x) transforms of a step: k_rowfwd (rowfwd_phi, rowfwd_g) and k_rowinv
// (rowinv_phi, rowinv_flow), compiled per row length nx = 2^LN.  See
// step_kernels.cu for the step's kernels and the x-spectral layout.
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

// ====================================================== forward row transforms
// Work items: mode 0 (phi): per row pair p = rows (2p, 2p+1), item 0 = phi*,
// item 1 = f = phi^3, item 2 = omega* (inertial members; with w_hat, the
// advective increment of omega); mode 1 (g): one item per row pair, plus the
// low row modes of g (FP32, P = 16); mode 2: omega's row pairs into xs_w (the
// row half of the transform that seeds w_hat).  Each item stages the two real
// rows (a, b) in shared memory and transforms a + i b (for f the staged phi
// rows are cubed on the fly), so every output chunk of the pair is one whole
// 32-byte piece.
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
  const int nsub = mode == 0 ? (D.stokes ? 2 : 3) : 1;
  const int nitems = mode == 2 && !D.wspec ? 0 : (ny >> 1) * nsub;
  const int stride = gridDim.x * ipc;
  unsigned char* base = smem_raw + (size_t)inst * rowfwd_inst_bytes(nx, sizeof(T));
  T* stage = reinterpret_cast<T*>(base);
  C* Z = reinterpret_cast<C*>(base + 2 * (size_t)nx * sizeof(T));
  const T* phis = static_cast<const T*>(D.phi_star);
  const T* phi = static_cast<const T*>(D.phi);
  const T* oms = static_cast<const T*>(D.omega_star);
  const T* gb = static_cast<const T*>(D.gbuf);
  C* tws = reinterpret_cast<C*>(smem_raw + (size_t)ipc * rowfwd_inst_bytes(nx, sizeof(T)));
  stage_tables_to_smem(tws, tw, log2nx, log2_points<P>(), threadIdx.x, blockDim.x);

  auto issue = [&](int w) {
    if (w < nitems) {
      const int p = w / nsub, sub = w - p * nsub;
      const T *ra, *rb;
      if (mode >= 1) {
        const T* src = mode == 1 ? gb : static_cast<const T*>(D.omega);
        ra = src + ((size_t)(2 * p) << log2nx);
        rb = src + ((size_t)(2 * p + 1) << log2nx);
      } else if (sub < 2) {
        const T* src = sub == 0 ? phis : phi;             // phi* pair, or phi pair (cubed on the fly)
        ra = src + ((size_t)(2 * p) << log2nx);
        rb = src + ((size_t)(2 * p + 1) << log2nx);
      } else {
        ra = oms + ((size_t)(2 * p) << log2nx);
        rb = oms + ((size_t)(2 * p + 1) << log2nx);
      }
      copy_async(stage, ra, nx * (int)sizeof(T), t, Tf);
      copy_async(stage + nx, rb, nx * (int)sizeof(T), t, Tf);
    }
    cp_async_commit();
  };

  const int iters = persistent_iters(nitems, ipc);
  int w = blockIdx.x * ipc + inst;
  issue(w);
  for (int it = 0; it < iters; ++it, w += stride) {
    const bool active = w < nitems;
    const int p = w / nsub, sub = w - p * nsub;
    const bool cube = mode == 0 && sub == 1;
    cp_async_wait_all();
    __syncthreads();
    if constexpr (sizeof(T) == 4 && P == 16 && MODE == 1) {   // the force's low row modes, part 1
      if (D.low) low_row_terms<LN>(reinterpret_cast<const float*>(stage), reinterpret_cast<float*>(Z), tws, t, D);
    }
    C v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = t + q * Tf;
      const T a = stage[i], bb = stage[nx + i];
      v[q] = cube ? C{(a * a) * a, (bb * bb) * bb} : C{a, bb};
    }
    __syncthreads();                                    // stage free
    issue(w + stride);                                  // next item streams in during the transform
    if constexpr (sizeof(T) == 4 && P == 16 && MODE == 1) {
      if (D.low) low_row_reduce<LN>(reinterpret_cast<float*>(Z), t, D, p, active, log2ny);
    }
    fft_reg<false>(v, log2nx, t, Z, tws);
    reg_to_smem(v, log2nx, t, Z);
    if (active) {
      if (mode >= 1) {
        write_pair_rows<LC>(Z, static_cast<C*>(mode == 1 ? D.xs_g : D.xs_w), 2 * p, nx, ny, t, Tf);
      } else if (sub < 2) {
        write_pair_rows<LC>(Z, static_cast<C*>(sub == 0 ? D.xs_phi : D.xs_f), 2 * p, nx, ny, t, Tf);
        if (sub == 0 && t == 0) {                        // phi*'s row Nyquist coefficients
          const C zn = Z[pad16(nx >> 1)];
          static_cast<T*>(D.nyq_phi)[2 * p] = zn.x;
          static_cast<T*>(D.nyq_phi)[2 * p + 1] = zn.y;
        }
      } else {
        write_pair_rows<LC>(Z, static_cast<C*>(D.xs_w), 2 * p, nx, ny, t, Tf);
        if (t == 0) {
          const C zn = Z[pad16(nx >> 1)];
          static_cast<T*>(D.nyq_omega)[2 * p] = zn.x;
          static_cast<T*>(D.nyq_omega)[2 * p + 1] = zn.y;
        }
      }
    }
    __syncthreads();                                    // Z reads done before the next transform
  }
  cp_async_wait_all();
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

  auto issue = [&](int w) {
    if (w < nitems) {
      const int sub = w % nsub;
      const C* src = static_cast<const C*>(mode == 0 ? D.xs_phi : (sub == 0 ? D.xs_g : D.xs_w));
      const int j0 = 2 * (w / nsub);
      for (int cb = t; cb < nchunk; cb += Tf) {
        const C* g = src + ((((size_t)cb * ny) + j0) << LC);
        cp_async16(stage + CL * cb, g);
        cp_async16(stage + CL * (nchunk + cb), g + H);
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
    cp_async_wait_all();
    __syncthreads();
    for (int cb = t; cb < nchunk; cb += Tf) {
      C Av[CL], Bv[CL];
      load16(stage + CL * cb, Av);
      load16(stage + CL * (nchunk + cb), Bv);
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
template <class T, int LN>
const void* rowfwd_fn(int P, int mode) {
  if constexpr (sizeof(T) == 4) {
    if (P == 16)
      return mode == 0 ? (const void*)k_rowfwd<T, LN, 16, 0>
                       : (mode == 1 ? (const void*)k_rowfwd<T, LN, 16, 1> : (const void*)k_rowfwd<T, LN, 16, 2>);
  }
  return mode == 0 ? (const void*)k_rowfwd<T, LN, 8, 0>
                   : (mode == 1 ? (const void*)k_rowfwd<T, LN, 8, 1> : (const void*)k_rowfwd<T, LN, 8, 2>);
}
template <class T, int LN>
const void* rowinv_fn(int P, int mode) {
  if constexpr (sizeof(T) == 4) {
    if (P == 16) return mode == 0 ? (const void*)k_rowinv<T, LN, 16, 0> : (const void*)k_rowinv<T, LN, 16, 1>;
  }
  return mode == 0 ? (const void*)k_rowinv<T, LN, 8, 0> : (const void*)k_rowinv<T, LN, 8, 1>;
}

template <class T>
void launch_row_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                       const LaunchCfg& c, cudaStream_t st) {
  const dim3 grid(c.grid_x, nmem);
  const bool fwd = kind == KIND_ROWFWD_PHI || kind == KIND_ROWFWD_G || kind == KIND_ROWFWD_OMEGA;
  const int mode = (kind == KIND_ROWFWD_PHI || kind == KIND_ROWINV_PHI) ? 0 : (kind == KIND_ROWFWD_OMEGA ? 2 : 1);
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
  const bool fwd = kind == KIND_ROWFWD_PHI || kind == KIND_ROWFWD_G;
  const int mode = (kind == KIND_ROWFWD_PHI || kind == KIND_ROWINV_PHI) ? 0 : 1;
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
        for (int mode : {0, 1, 2}) {
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
