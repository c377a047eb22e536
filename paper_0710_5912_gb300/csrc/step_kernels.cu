// Kernels of one time step (Appendix B of arXiv:0710.5912), templated on the
// working precision T (float or double).  A step is eight launches per grid
// size:
//
//   stencil1     item 1 + item 2's advection at s = s^n (Eq. advective with the
//                Eq. p1y stencils): phi* = phi - dt J(psi, phi) and omega* =
//                omega - dt J(psi, omega), real; omega* is written at the
//                relabelled positions when the strain wraps during the step.
//   rowfwd_phi   row (x) transforms of (phi*, f = phi^3) per row and of the
//                omega* row pair -> x-spectral buffers, plus each row's real
//                Nyquist coefficient of phi* and omega*.
//   colpass_phi  column (y) transforms of phi*, f; the Cahn-Hilliard update of
//                item 1 in the paper's increment form
//                  phi^{n+1} = phi* + (1 + D4/2)^-1 (-D2 phi* - D4 phi* + D2 f),
//                Nyquist modes of phi^{n+1} zeroed; the increment back along y.
//   rowinv_phi   phi^{n+1} = phi* + row inverse of the increment (minus phi*'s
//                Nyquist column), written at the relabelled positions at a wrap.
//   stencil2     mu = -a phi + b phi^3 - kappa lap_c phi and the body-force curl
//                F = d_x phi d_y mu - d_y phi d_x mu at s = s^{n+1} (Eq. G);
//                g = -F/rho, or -F/eta for Stokes, real.
//   rowfwd_g     row transforms of g row pairs.
//   colpass_flow column transforms; Crank-Nicolson vorticity update in increment
//                form omega^{n+1} = omega* + (1 - C/2)^-1 (C omega* + g) and the
//                Poisson solve psi = omega / k^2 (items 2-3), or the Stokes solve
//                psi = g / k^4; inverse column transforms.
//   rowinv_flow  psi rows, and omega^{n+1} = omega* + row inverse of the
//                increment; advances the step counter.
//
// Transforming only the increments keeps the FP32 rounding of a step
// proportional to the change of the field instead of to the field itself.
//
// Execution: the stencils run on 2D tiles; the transform kernels are
// persistent -- every instance walks its work items (row pairs or columns) with
// a grid stride and, while transforming one item, streams the next item's
// input into a shared-memory staging buffer with cp.async, so the loads in
// flight hold shared memory rather than registers.  The FFT itself keeps 8
// points per thread in registers (fft_block.cuh).
//
// Layout: real fields ny x nx row-major.  x-spectral buffers hold, for each row
// j, the modes m = 0..nx/2-1 of the row's real DFT (the Nyquist column is
// carried separately as one real per row), tiled in chunks of CL = 2^LC
// adjacent modes: element (j, m) sits at ((m >> LC) ny + j) CL + (m & (CL-1)),
// so a chunk of a row pair is 32 contiguous bytes and a column is one strided
// run.  The 1/(nx ny) of the inverse transforms is applied in the column passes.
// Each launch covers a batch of members of one size (one descriptor each).
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

__global__ void k_step_state_init(const MemberDesc* __restrict__ descs, int nmem) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nmem) step_state_set(descs[r], descs[r].st->n);
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

// Z holds FFT(row j0 + i row j0+1) of one field: both half spectra -> dst.
// A thread writes whole chunks of the pair: 2 CL elements = 32 contiguous
// bytes (a full sector), as two 16-byte stores in FP32.
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
      reinterpret_cast<float4*>(p)[0] = make_float4(A[0].x, A[0].y, A[1].x, A[1].y);
      reinterpret_cast<float4*>(p)[1] = make_float4(B[0].x, B[0].y, B[1].x, B[1].y);
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
template <class C>
__device__ __forceinline__ void smem_to_reg(C (&v)[kP], const C* Z, int log2N, int t) {
  const int T = 1 << (log2N - kLogP);
#pragma unroll
  for (int q = 0; q < kP; ++q) v[q] = Z[pad16(t + q * T)];
}

// Number of loop iterations of a persistent CTA: every instance of the CTA runs
// the same count (the loop body has barriers); an instance whose item is past
// the end idles through its last iteration.
__device__ __forceinline__ int persistent_iters(int nitems, int ipc) {
  const int stride = gridDim.x * ipc;
  const int first = blockIdx.x * ipc;
  return first < nitems ? (nitems - first + stride - 1) / stride : 0;
}

// ============================================================== stencils
// 2D tiles of TX x TY outputs (TX = min(nx, 128), a template constant so that
// every tile index is divided by a constant; TY = 8), 256 threads.
constexpr int kTY = 8;

// stage-1 stencil: inputs phi, psi (and omega) with halo x +-2, y +-1
template <class T, int TX>
__global__ void __launch_bounds__(256) k_stencil1(const MemberDesc* __restrict__ descs, int log2nx, int log2ny) {
  constexpr int W = TX + 4;
  __shared__ T sh[3][kTY + 2][W];
  const MemberDesc& D = descs[blockIdx.z];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * kTY;
  const bool stokes = D.stokes != 0;
  const Shear<T> sc(*D.st, false);                      // s^n
  const T dt = (T)D.dt, inv2h = (T)D.inv_2h;
  const T* __restrict__ f0 = static_cast<const T*>(D.phi);
  const T* __restrict__ f1 = static_cast<const T*>(D.psi);
  const T* __restrict__ f2 = static_cast<const T*>(D.omega);
  for (int e = threadIdx.x; e < (kTY + 2) * W; e += blockDim.x) {
    const int r = e / W, c = e - r * W;
    const size_t g = ((size_t)((y0 - 1 + r) & my) << log2nx) + ((x0 - 2 + c) & mx);
    sh[0][r][c] = __ldg(f0 + g);
    sh[1][r][c] = __ldg(f1 + g);
    if (!stokes) sh[2][r][c] = __ldg(f2 + g);
  }
  __syncthreads();
  T* phis = static_cast<T*>(D.phi_star);
  T* oms = static_cast<T*>(D.omega_star);
  const bool wrap = D.remap && sc.dK != 0;
  for (int e = threadIdx.x; e < kTY * TX; e += blockDim.x) {
    const int ly = e / TX, lx = e - ly * TX;
    const int r = ly + 1, c = lx + 2;
    const int y = y0 + ly, x = x0 + lx;
    auto dxf = [&](int f) { return (sh[f][r][c + 1] - sh[f][r][c - 1]) * inv2h; };
    auto dyf = [&](int f) {
      return (sc.w0 * (sh[f][r + 1][c] - sh[f][r - 1][c]) +
              sc.w1 * (sh[f][r + 1][c + sc.d] - sh[f][r - 1][c - sc.d])) * inv2h;
    };
    const T dxpsi = dxf(1), dypsi = dyf(1);
    const T pc = sh[0][r][c];
    phis[((size_t)y << log2nx) + x] = pc - dt * (dypsi * dxf(0) - dxpsi * dyf(0));
    if (!stokes) {
      const T ws = sh[2][r][c] - dt * (dypsi * dxf(2) - dxpsi * dyf(2));
      const int sh_y = wrap ? remap_shift(sc.dK, D.ratio, y, nx) : 0;
      oms[((size_t)y << log2nx) + ((x + sh_y) & mx)] = ws;
    }
  }
}

// stage-2 stencil: mu on a halo tile (x +-2, y +-1) from phi (x +-3, y +-2),
// then g = c_force (d_x phi d_y mu - d_y phi d_x mu)
template <class T, int TX>
__global__ void __launch_bounds__(256) k_stencil2(const MemberDesc* __restrict__ descs, int log2nx, int log2ny) {
  constexpr int WP = TX + 6, WM = TX + 4;
  __shared__ T sp[kTY + 4][WP];
  __shared__ T sm[kTY + 2][WM];
  const MemberDesc& D = descs[blockIdx.z];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * kTY;
  const Shear<T> sc(*D.st, true);                        // s^{n+1}
  const T a = (T)D.a, b = (T)D.b, kappa = (T)D.kappa;
  const T inv2h = (T)D.inv_2h, ih2 = (T)D.inv_h2, i4h2 = (T)D.inv_4h2;
  const T cxx = T(1) + sc.s * sc.s, cxy = T(2) * sc.s;
  const T cf = (T)D.c_force;
  const T* __restrict__ phi = static_cast<const T*>(D.phi);
  for (int e = threadIdx.x; e < (kTY + 4) * WP; e += blockDim.x) {
    const int r = e / WP, c = e - r * WP;
    sp[r][c] = __ldg(phi + ((size_t)((y0 - 2 + r) & my) << log2nx) + ((x0 - 3 + c) & mx));
  }
  __syncthreads();
  // mu (Appendix B item 2: 3-point second differences, 4-point cross difference)
  for (int e = threadIdx.x; e < (kTY + 2) * WM; e += blockDim.x) {
    const int r = e / WM, c = e - r * WM;
    const int pr = r + 1, pcc = c + 1;
    const T pc = sp[pr][pcc];
    const T dxx = (sp[pr][pcc + 1] - T(2) * pc + sp[pr][pcc - 1]) * ih2;
    const T dyy = (sp[pr + 1][pcc] - T(2) * pc + sp[pr - 1][pcc]) * ih2;
    const T dxy = (sp[pr + 1][pcc + 1] - sp[pr - 1][pcc + 1] - sp[pr + 1][pcc - 1] + sp[pr - 1][pcc - 1]) * i4h2;
    const T lap = cxx * dxx - cxy * dxy + dyy;
    sm[r][c] = -a * pc + b * ((pc * pc) * pc) - kappa * lap;
  }
  __syncthreads();
  T* g = static_cast<T*>(D.gbuf);
  for (int e = threadIdx.x; e < kTY * TX; e += blockDim.x) {
    const int ly = e / TX, lx = e - ly * TX;
    const int rp = ly + 2, cp = lx + 3, rm = ly + 1, cm = lx + 2;
    const T dxphi = (sp[rp][cp + 1] - sp[rp][cp - 1]) * inv2h;
    const T dyphi = (sc.w0 * (sp[rp + 1][cp] - sp[rp - 1][cp]) +
                     sc.w1 * (sp[rp + 1][cp + sc.d] - sp[rp - 1][cp - sc.d])) * inv2h;
    const T dxmu = (sm[rm][cm + 1] - sm[rm][cm - 1]) * inv2h;
    const T dymu = (sc.w0 * (sm[rm + 1][cm] - sm[rm - 1][cm]) +
                    sc.w1 * (sm[rm + 1][cm + sc.d] - sm[rm - 1][cm - sc.d])) * inv2h;
    g[((size_t)(y0 + ly) << log2nx) + x0 + lx] = cf * (dxphi * dymu - dyphi * dxmu);
  }
}

// ====================================================== forward row transforms
// Work items: mode 0 (phi): per row pair p = rows (2p, 2p+1), item 0 = phi*,
// item 1 = f = phi^3, item 2 = omega* (inertial members); mode 1 (g): one item
// per row pair.  Each item stages the two real rows (a, b) in shared memory and
// transforms a + i b (for f the staged phi rows are cubed on the fly), so every
// output chunk of the pair is one whole 32-byte piece.
template <class T>
__global__ void __launch_bounds__(512, min_ctas<T>()) k_rowfwd(const MemberDesc* __restrict__ descs, int log2nx, int log2ny,
                                                const cplx<T>* __restrict__ tw, int mode) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tf = nx >> kLogP;
  const int ipc = blockDim.x / Tf;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int nsub = mode == 0 ? (D.stokes ? 2 : 3) : 1;
  const int nitems = (ny >> 1) * nsub;
  const int stride = gridDim.x * ipc;
  unsigned char* base = smem_raw + (size_t)inst * rowfwd_inst_bytes(nx, sizeof(T));
  T* stage = reinterpret_cast<T*>(base);
  C* Z = reinterpret_cast<C*>(base + 2 * (size_t)nx * sizeof(T));
  const T* phis = static_cast<const T*>(D.phi_star);
  const T* phi = static_cast<const T*>(D.phi);
  const T* oms = static_cast<const T*>(D.omega_star);
  const T* gb = static_cast<const T*>(D.gbuf);

  auto issue = [&](int w) {
    if (w < nitems) {
      const int p = w / nsub, sub = w - p * nsub;
      const T *ra, *rb;
      if (mode == 1) {
        ra = gb + ((size_t)(2 * p) << log2nx);
        rb = gb + ((size_t)(2 * p + 1) << log2nx);
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
    C v[kP];
#pragma unroll
    for (int q = 0; q < kP; ++q) {
      const int i = t + q * Tf;
      const T a = stage[i], bb = stage[nx + i];
      v[q] = cube ? C{(a * a) * a, (bb * bb) * bb} : C{a, bb};
    }
    __syncthreads();                                    // stage free
    issue(w + stride);                                  // next item streams in during the transform
    fft_reg<false>(v, log2nx, t, Z, tw);
    reg_to_smem(v, log2nx, t, Z);
    if (active) {
      if (mode == 1) {
        write_pair_rows<LC>(Z, static_cast<C*>(D.xs_g), 2 * p, nx, ny, t, Tf);
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

// The multiplier at mode (m, row nn) of the column transform, in place:
// mode 0: va = phi*_hat -> increment of phi_hat (x norm), vb = f_hat;
// mode 1: va = g_hat -> psi_hat (x norm), vb = omega*_hat -> increment (x norm).
// qx = m q_unit and sqx = s q_x, both formed in double.
template <class T>
__device__ __forceinline__ void col_multiply(int mode, const ColConsts<T>& K, int m, T qx, T sqx, int nn,
                                             cplx<T>& va, cplx<T>& vb) {
  using C = cplx<T>;
  const int ns = nn < (K.ny >> 1) ? nn : nn - K.ny;
  const T ky = (T)ns * K.qyu - sqx;
  const T k2 = qx * qx + ky * ky;
  const bool nyq_row = nn == (K.ny >> 1);
  const T norm = K.norm;
  if (mode == 0) {
    const C P = va, F = vb;
    if (nyq_row) {
      va = C{-P.x * norm, -P.y * norm};                 // Nyquist row of phi^{n+1} -> 0
    } else {
      const T c4 = K.ckM * (k2 * k2);
      const T aa = K.caM * k2 - T(2) * c4;
      const T bbm = K.cbM * k2;
      const T inv = norm / (T(1) + c4);
      va = C{(aa * P.x - bbm * F.x) * inv, (aa * P.y - bbm * F.y) * inv};
    }
  } else {
    const bool zero = nyq_row || (m == 0 && nn == 0);
    const C G = va;
    if (K.stokes) {
      const T inv = zero ? T(0) : norm / (k2 * k2);
      va = C{G.x * inv, G.y * inv};
    } else {
      const C Wv = vb;
      if (zero) {
        va = C{T(0), T(0)};
        vb = C{-Wv.x * norm, -Wv.y * norm};             // omega^{n+1} -> 0 there
      } else {
        const T cc = K.cnu * k2;
        const T inv = T(1) / (T(1) + cc);
        const C dw = C{(-T(2) * cc * Wv.x + K.dt * G.x) * inv, (-T(2) * cc * Wv.y + K.dt * G.y) * inv};
        const T ik = norm / k2;
        va = C{(Wv.x + dw.x) * ik, (Wv.y + dw.y) * ik};
        vb = C{dw.x * norm, dw.y * norm};
      }
    }
  }
}

template <class T>
__global__ void __launch_bounds__(512, min_ctas<T>()) k_colpass(const MemberDesc* __restrict__ descs, int log2nx, int log2ny,
                                                 const cplx<T>* __restrict__ tw, int mode) {
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
    fft_reg<false>(va, log2ny, t, buf, tw);
    if (two) fft_reg<false>(vb, log2ny, t, buf, tw);
    const double qx_d = mm * K.qx_unit;
    const T qx = (T)qx_d;
    const T sqx = (T)(K.s_d * qx_d);                    // s q_x formed in double
#pragma unroll
    for (int q = 0; q < kP; ++q) col_multiply<T>(mode, K, mm, qx, sqx, t + q * Tc, va[q], vb[q]);
    fft_reg<true>(va, log2ny, t, buf, tw);
    if (active) {
#pragma unroll
      for (int q = 0; q < kP; ++q) in0[xs_idx(t + q * Tc, m, ny, LC)] = va[q];
    }
    if (mode == 1 && !stokes) {
      fft_reg<true>(vb, log2ny, t, buf, tw);
      if (active) {
#pragma unroll
        for (int q = 0; q < kP; ++q) in1[xs_idx(t + q * Tc, m, ny, LC)] = vb[q];
      }
    }
  }
  cp_async_wait_all();
}

// FP32 column pass over whole chunks: item cb = the two modes m = 2cb, 2cb+1,
// whose ny rows are one contiguous 16-byte-per-row run in the x-spectral
// layout.  Both columns are staged with 16-byte copies, transformed in lock
// step (shared twiddles, 16-byte exchanges) and written back as whole 16-byte
// rows, so no sector is touched twice.
__global__ void __launch_bounds__(512, 1) k_colpass_pair(const MemberDesc* __restrict__ descs, int log2nx,
                                                        int log2ny, const float2* __restrict__ tw, int mode) {
  using T = float;
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tc = ny >> kLogP;
  const int ipc = blockDim.x / Tc;
  const int inst = threadIdx.x / Tc, t = threadIdx.x - inst * Tc;
  const int nitems = nx >> 2;
  const int stride = gridDim.x * ipc;
  const bool stokes = D.stokes != 0;
  const bool two = mode == 0 || !stokes;                // second input field
  unsigned char* base = smem_raw + (size_t)inst * colpass_inst_bytes(ny, sizeof(T));
  float4* st0 = reinterpret_cast<float4*>(base);
  float4* st1 = st0 + ny;
  float4* buf = st1 + ny;
  float4* in0 = static_cast<float4*>(mode == 0 ? D.xs_phi : D.xs_g);
  float4* in1 = static_cast<float4*>(mode == 0 ? D.xs_f : D.xs_w);

  auto issue = [&](int cb) {
    if (cb < nitems) {
      copy_async(st0, in0 + (size_t)cb * ny, ny * 16, t, Tc);
      if (two) copy_async(st1, in1 + (size_t)cb * ny, ny * 16, t, Tc);
    }
    cp_async_commit();
  };

  const ColConsts<T> K(D, mode, ny);
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
    fft_reg2<false>(a0, b0, log2ny, t, buf, tw);
    if (two) fft_reg2<false>(a1, b1, log2ny, t, buf, tw);
    const int m0 = active ? 2 * cb : 0, m1 = m0 + 1;
    const double qa_d = m0 * K.qx_unit, qb_d = m1 * K.qx_unit;
    const T qa = (T)qa_d, qb = (T)qb_d;
    const T sqa = (T)(K.s_d * qa_d), sqb = (T)(K.s_d * qb_d);   // s q_x formed in double
#pragma unroll
    for (int q = 0; q < kP; ++q) {
      col_multiply<T>(mode, K, m0, qa, sqa, t + q * Tc, a0[q], a1[q]);
      col_multiply<T>(mode, K, m1, qb, sqb, t + q * Tc, b0[q], b1[q]);
    }
    fft_reg2<true>(a0, b0, log2ny, t, buf, tw);
    if (active) {
      float4* o = in0 + (size_t)cb * ny;
#pragma unroll
      for (int q = 0; q < kP; ++q) o[t + q * Tc] = make_float4(a0[q].x, a0[q].y, b0[q].x, b0[q].y);
    }
    if (mode == 1 && !stokes) {
      fft_reg2<true>(a1, b1, log2ny, t, buf, tw);
      if (active) {
        float4* o = in1 + (size_t)cb * ny;
#pragma unroll
        for (int q = 0; q < kP; ++q) o[t + q * Tc] = make_float4(a1[q].x, a1[q].y, b1[q].x, b1[q].y);
      }
    }
  }
  cp_async_wait_all();
}

// ====================================================== inverse row transforms
// Work items: mode 0 (phi): row pairs of the phi increment; mode 1 (flow): per
// row pair, item 0 = psi, item 1 = the omega increment (inertial members).  The
// item's 32-byte chunks stream into the staging buffer during the previous
// transform; Z[k] = A[k] + i B[k], Z[N-k] = conj A[k] + i conj B[k] (A, B the
// two rows), Z[0] from the real parts, Z[N/2] = minus the staged field's row
// Nyquist coefficients / nx.
template <class T>
__global__ void __launch_bounds__(512, min_ctas<T>()) k_rowinv(const MemberDesc* __restrict__ descs, int log2nx, int log2ny,
                                                const cplx<T>* __restrict__ tw, int mode) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  constexpr int CL = 1 << LC;
  constexpr int H = 16 / sizeof(C);                     // complex values per 16 bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1;
  const int Tf = nx >> kLogP;
  const int ipc = blockDim.x / Tf;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int nsub = (mode == 1 && !D.stokes) ? 2 : 1;
  const int nitems = (ny >> 1) * nsub;
  const int stride = gridDim.x * ipc;
  const int nchunk = (nx >> 1) >> LC;
  unsigned char* base = smem_raw + (size_t)inst * rowinv_inst_bytes(nx, sizeof(T));
  C* stage = reinterpret_cast<C*>(base);               // chunk cb at stage[2 CL cb]
  C* Z = stage + nx;

  auto issue = [&](int w) {
    if (w < nitems) {
      const int sub = w % nsub;
      const C* src = static_cast<const C*>(mode == 0 ? D.xs_phi : (sub == 0 ? D.xs_g : D.xs_w));
      const int j0 = 2 * (w / nsub);
      for (int cb = t; cb < nchunk; cb += Tf) {
        const C* g = src + ((((size_t)cb * ny) + j0) << LC);
        cp_async16(stage + 2 * CL * cb, g);
        cp_async16(stage + 2 * CL * cb + H, g + H);
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
    const int kind = mode == 0 ? 0 : (sub == 0 ? 1 : 2);   // phi increment, psi, omega increment
    C zn = C{T(0), T(0)};
    if (active && kind != 1) {
      const T* nq = static_cast<const T*>(kind == 0 ? D.nyq_phi : D.nyq_omega);
      zn = C{-nq[j0] * rn, -nq[j1] * rn};
    }
    cp_async_wait_all();
    __syncthreads();
    for (int cb = t; cb < nchunk; cb += Tf) {
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        const int k = (cb << LC) + c;
        const C A = stage[2 * CL * cb + c], B = stage[2 * CL * cb + CL + c];
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
    C v[kP];
    smem_to_reg(v, Z, log2nx, t);
    __syncthreads();                                    // Z becomes the exchange buffer
    // the real-space base of the increment (phi* or omega*), loaded before the transform
    T b0[kP], b1[kP];
    if (active && kind != 1) {
      const T* bs = static_cast<const T*>(kind == 0 ? D.phi_star : D.omega_star);
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        b0[q] = bs[((size_t)j0 << log2nx) + t + q * Tf];
        b1[q] = bs[((size_t)j1 << log2nx) + t + q * Tf];
      }
    }
    fft_reg<true>(v, log2nx, t, Z, tw);
    if (active) {
      if (kind == 1) {
        T* out = static_cast<T*>(D.psi);
#pragma unroll
        for (int q = 0; q < kP; ++q) {
          out[((size_t)j0 << log2nx) + t + q * Tf] = v[q].x;
          out[((size_t)j1 << log2nx) + t + q * Tf] = v[q].y;
        }
      } else {
        T* out = static_cast<T*>(kind == 0 ? D.phi : D.omega);
        const int sh0 = (kind == 0 && dK) ? remap_shift(dK, D.ratio, j0, nx) : 0;
        const int sh1 = (kind == 0 && dK) ? remap_shift(dK, D.ratio, j1, nx) : 0;
#pragma unroll
        for (int q = 0; q < kP; ++q) {
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
void launch_step_state_init(const MemberDesc* d, int nmem, cudaStream_t st) {
  k_step_state_init<<<(nmem + 127) / 128, 128, 0, st>>>(d, nmem);
}

template <class T>
void launch_step_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                        const LaunchCfg& c, cudaStream_t st) {
  switch (kind) {
    case KIND_STENCIL1:
      switch (log2nx) {
        case 4: k_stencil1<T, 16><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
        case 5: k_stencil1<T, 32><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
        case 6: k_stencil1<T, 64><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
        default: k_stencil1<T, 128><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
      }
      break;
    case KIND_ROWFWD_PHI:
      k_rowfwd<T><<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 0);
      break;
    case KIND_COLPASS_PHI:
      if constexpr (sizeof(T) == 4)
        k_colpass_pair<<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 0);
      else
        k_colpass<T><<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 0);
      break;
    case KIND_ROWINV_PHI:
      k_rowinv<T><<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 0);
      break;
    case KIND_STENCIL2:
      switch (log2nx) {
        case 4: k_stencil2<T, 16><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
        case 5: k_stencil2<T, 32><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
        case 6: k_stencil2<T, 64><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
        default: k_stencil2<T, 128><<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny); break;
      }
      break;
    case KIND_ROWFWD_G:
      k_rowfwd<T><<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 1);
      break;
    case KIND_COLPASS_FLOW:
      if constexpr (sizeof(T) == 4)
        k_colpass_pair<<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 1);
      else
        k_colpass<T><<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 1);
      break;
    default:
      k_rowinv<T><<<dim3(c.grid_x, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, 1);
      break;
  }
}

// CTAs of a persistent kind that fit on one SM at (threads, smem)
template <class T>
int step_kernel_occupancy(int kind, int threads, size_t smem) {
  int nb = 0;
  const void* f = nullptr;
  switch (kind) {
    case KIND_ROWFWD_PHI:
    case KIND_ROWFWD_G: f = (const void*)k_rowfwd<T>; break;
    case KIND_COLPASS_PHI:
    case KIND_COLPASS_FLOW:
      f = sizeof(T) == 4 ? (const void*)k_colpass_pair : (const void*)k_colpass<T>;
      break;
    default: f = (const void*)k_rowinv<T>; break;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) nb = 1;
  return nb < 1 ? 1 : nb;
}

template <class T>
void set_step_smem_limits() {
  const int lim = 220 * 1024;   // dynamic part; leaves room for static shared memory
  cudaFuncSetAttribute(k_rowfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_colpass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (sizeof(T) == 4) cudaFuncSetAttribute(k_colpass_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_rowinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

#define SHF_INST(T)                                                                                      \
  template void launch_step_kernel<T>(int, const MemberDesc*, int, int, int, const cplx<T>*,             \
                                      const LaunchCfg&, cudaStream_t);                                    \
  template int step_kernel_occupancy<T>(int, int, size_t);                                                \
  template void set_step_smem_limits<T>();

SHF_INST(float)
SHF_INST(double)

}  // namespace shf
