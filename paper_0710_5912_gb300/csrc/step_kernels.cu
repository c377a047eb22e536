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
// 2D tiles of TX x TY outputs (TX = min(nx, 128), TY = min(ny, 32)); each
// thread makes a 4 x 4 block of outputs (4 consecutive x in 4 rows), reading
// its stencil rows from the shared tile with 16-byte loads.  The sign of s
// selects one of two compiled bodies (the diagonal of Eq. p1y lies on one side).

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

// Fill rows [0, H) of NF tiles (tile column c <-> x0 - OFF + c, OFF = 2 or 6,
// width TX + 2 OFF) from NF fields at rows y0 - HY + r (periodic).  Interior
// quads are 16-byte global loads; the OFF halo columns on each side are pairs.
template <class T, int TX, int OFF, int H, int NF>
__device__ __forceinline__ void fill_tiles(T* tile, const T* const* src, int x0, int yb, int log2nx, int my,
                                           int tid, int nthr) {
  constexpr int QX = TX / 4, W = TX + 2 * OFF, HP = OFF / 2;   // HP halo pairs per side
  constexpr int SLOTS = QX + 2 * HP;
  const int mx = (1 << log2nx) - 1;
  for (int e = tid; e < NF * H * SLOTS; e += nthr) {
    const int f = e / (H * SLOTS);
    const int rem = e - f * (H * SLOTS);
    const int r = rem / SLOTS, k = rem - r * SLOTS;
    const T* row = src[f] + ((size_t)((yb + r) & my) << log2nx);
    T* trow = tile + ((size_t)f * H + r) * W;
    if (k < QX) {
      const Quad<T> q = ldg4(row + x0 + 4 * k);
      T* d = trow + OFF + 4 * k;
      if (OFF % 4 == 0) {
        st4(d, q.v[0], q.v[1], q.v[2], q.v[3]);
      } else {
        st2(d, q.v[0], q.v[1]);
        st2(d + 2, q.v[2], q.v[3]);
      }
    } else {
      const int h = k - QX;                               // 0 .. 2 HP - 1
      const int side = h / HP, j = h - side * HP;         // left (0) or right (1) halo, pair j
      const int c = side == 0 ? 2 * j : OFF + TX + 2 * j;
      const int x = (x0 - OFF + c) & mx;                  // even, so the pair is contiguous
      T a, b;
      ldg2(row + x, a, b);
      st2(trow + c, a, b);
    }
  }
}

// stage-1 stencil: phi* = phi - dt J(psi, phi), omega* = omega - dt J(psi, omega)
// (Eq. advective with J(A, B) = D_y^s A D_x B - D_x A D_y^s B), tiles of
// phi, psi (and omega) with halo x +-2, y +-1.  At a wrap omega* is stored
// remapped (row j shifted by the wrap's cells).
template <bool NEG, class T, int TX, int TY>
__device__ __forceinline__ void stencil1_body(const MemberDesc& D, const T* tiles, const Shear<T>& sc, int x0,
                                              int y0, int log2nx) {
  constexpr int QX = TX / 4, W = TX + 4, H = TY + 2;
  const int nx = 1 << log2nx, mx = nx - 1;
  const int q = threadIdx.x % QX, g = threadIdx.x / QX;
  const bool stokes = D.stokes != 0;
  const bool wrap = D.remap && sc.dK != 0;
  const T dt = (T)D.dt, inv2h = (T)D.inv_2h;
  T* phis = static_cast<T*>(D.phi_star);
  T* oms = static_cast<T*>(D.omega_star);
  const T* t0 = tiles;                 // phi
  const T* t1 = tiles + H * W;         // psi
  const T* t2 = tiles + 2 * H * W;     // omega
  const int x = x0 + 4 * q;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int tr = 4 * g + 1 + o;      // tile row of output row y0 + 4 g + o
    const int y = y0 + 4 * g + o;
    T dxp[4], dyp[4];
    grad4<NEG>(ld8(t1 + (tr + 1) * W + 4 * q), ld8(t1 + tr * W + 4 * q), ld8(t1 + (tr - 1) * W + 4 * q), sc.w0,
               sc.w1, inv2h, dxp, dyp);
    {
      const Row8<T> C = ld8(t0 + tr * W + 4 * q);
      T dxf[4], dyf[4];
      grad4<NEG>(ld8(t0 + (tr + 1) * W + 4 * q), C, ld8(t0 + (tr - 1) * W + 4 * q), sc.w0, sc.w1, inv2h, dxf, dyf);
      T r[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) r[p] = C.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
      st4(phis + ((size_t)y << log2nx) + x, r[0], r[1], r[2], r[3]);
    }
    if (!stokes) {
      const Row8<T> C = ld8(t2 + tr * W + 4 * q);
      T dxf[4], dyf[4];
      grad4<NEG>(ld8(t2 + (tr + 1) * W + 4 * q), C, ld8(t2 + (tr - 1) * W + 4 * q), sc.w0, sc.w1, inv2h, dxf, dyf);
      T r[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) r[p] = C.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
      T* orow = oms + ((size_t)y << log2nx);
      if (!wrap) {
        st4(orow + x, r[0], r[1], r[2], r[3]);
      } else {
        const int sh_y = remap_shift(sc.dK, D.ratio, y, nx);
#pragma unroll
        for (int p = 0; p < 4; ++p) orow[(x + p + sh_y) & mx] = r[p];
      }
    }
  }
}

template <class T, int TX, int TY>
__global__ void __launch_bounds__(256) k_stencil1(const MemberDesc* __restrict__ descs, int log2nx, int log2ny) {
  constexpr int H = TY + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];   // stencil1_smem_bytes
  T* tiles = reinterpret_cast<T*>(smem_raw);
  const MemberDesc& D = descs[blockIdx.z];
  const int my = (1 << log2ny) - 1;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const Shear<T> sc(*D.st, false);                      // s^n
  const T* src[3] = {static_cast<const T*>(D.phi), static_cast<const T*>(D.psi), static_cast<const T*>(D.omega)};
  if (D.stokes) fill_tiles<T, TX, 2, H, 2>(tiles, src, x0, y0 - 1, log2nx, my, threadIdx.x, blockDim.x);
  else fill_tiles<T, TX, 2, H, 3>(tiles, src, x0, y0 - 1, log2nx, my, threadIdx.x, blockDim.x);
  __syncthreads();
  if (sc.d > 0) stencil1_body<true, T, TX, TY>(D, tiles, sc, x0, y0, log2nx);
  else stencil1_body<false, T, TX, TY>(D, tiles, sc, x0, y0, log2nx);
}

// stage-2 stencil: mu = -a phi + b phi^3 - kappa L_s phi (Appendix B item 2:
// 3-point second differences, 4-point cross difference) on a tile with halo
// x +-2, y +-1 from phi (halo x +-6 loaded, y +-2), then
// g = c_force (D_x phi D_y^s mu - D_y^s phi D_x mu) (Eqs. vortNum, G).
template <bool NEG, class T, int TX, int TY>
__device__ __forceinline__ void stencil2_body(const MemberDesc& D, const T* tp, T* tm, const Shear<T>& sc, int x0,
                                              int y0, int log2nx) {
  constexpr int QX = TX / 4, W = TX + 12, HP = TY + 4, HM = TY + 2;
  constexpr int NQ = QX + 1;                  // mu quads per row: tile cols 4 .. TX + 7
  const int tid = threadIdx.x, nthr = blockDim.x;
  const T a = (T)D.a, b = (T)D.b, kappa = (T)D.kappa;
  const T ih2 = (T)D.inv_h2, i4h2 = (T)D.inv_4h2, inv2h = (T)D.inv_2h;
  const T cxx = T(1) + sc.s * sc.s, cxy = T(2) * sc.s;
  // mu tile row rm <-> y0 - 1 + rm <-> phi tile row rm + 1; mu quad at tile col 4 (k + 1)
  for (int e = tid; e < HM * NQ; e += nthr) {
    const int rm = e / NQ, k = e - rm * NQ;
    const int c = 4 * (k + 1);
    const T* pr = tp + (rm + 1) * W;
    const Quad<T> Cl = ld4(pr + c - 4), Cc = ld4(pr + c), Cr = ld4(pr + c + 4);
    const Quad<T> Ul = ld4(pr + W + c - 4), Uc = ld4(pr + W + c), Ur = ld4(pr + W + c + 4);
    const Quad<T> Dl = ld4(pr - W + c - 4), Dc = ld4(pr - W + c), Dr = ld4(pr - W + c + 4);
    const T cw[6] = {Cl.v[3], Cc.v[0], Cc.v[1], Cc.v[2], Cc.v[3], Cr.v[0]};
    const T uw[6] = {Ul.v[3], Uc.v[0], Uc.v[1], Uc.v[2], Uc.v[3], Ur.v[0]};
    const T dw[6] = {Dl.v[3], Dc.v[0], Dc.v[1], Dc.v[2], Dc.v[3], Dr.v[0]};
    T m[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const T pc = cw[p + 1];
      const T dxx = (cw[p + 2] - T(2) * pc + cw[p]) * ih2;
      const T dyy = (uw[p + 1] - T(2) * pc + dw[p + 1]) * ih2;
      const T dxy = (uw[p + 2] - dw[p + 2] - uw[p] + dw[p]) * i4h2;
      const T lap = cxx * dxx - cxy * dxy + dyy;
      m[p] = -a * pc + b * ((pc * pc) * pc) - kappa * lap;
    }
    st4(tm + rm * W + c, m[0], m[1], m[2], m[3]);
  }
  __syncthreads();
  const int q = tid % QX, g = tid / QX;
  const T cf = (T)D.c_force;
  T* gout = static_cast<T*>(D.gbuf);
  const int x = x0 + 4 * q;
  // the 8-wide rows of output block (cols x - 2 .. x + 5) start at tile col 4 q + 4
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int y = y0 + 4 * g + o;
    const int rp = 4 * g + 2 + o, rmu = 4 * g + 1 + o;   // phi and mu tile rows of y
    T dxp[4], dyp[4], dxm[4], dym[4];
    grad4<NEG>(ld8(tp + (rp + 1) * W + 4 * q + 4), ld8(tp + rp * W + 4 * q + 4), ld8(tp + (rp - 1) * W + 4 * q + 4),
               sc.w0, sc.w1, inv2h, dxp, dyp);
    grad4<NEG>(ld8(tm + (rmu + 1) * W + 4 * q + 4), ld8(tm + rmu * W + 4 * q + 4),
               ld8(tm + (rmu - 1) * W + 4 * q + 4), sc.w0, sc.w1, inv2h, dxm, dym);
    T r[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) r[p] = cf * (dxp[p] * dym[p] - dyp[p] * dxm[p]);
    st4(gout + ((size_t)y << log2nx) + x, r[0], r[1], r[2], r[3]);
  }
}

template <class T, int TX, int TY>
__global__ void __launch_bounds__(256) k_stencil2(const MemberDesc* __restrict__ descs, int log2nx, int log2ny) {
  constexpr int W = TX + 12, HP = TY + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];   // stencil2_smem_bytes
  T* tp = reinterpret_cast<T*>(smem_raw);                     // phi tile, HP x W
  T* tm = tp + HP * W;                                        // mu tile, (TY + 2) x W
  const MemberDesc& D = descs[blockIdx.z];
  const int my = (1 << log2ny) - 1;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const Shear<T> sc(*D.st, true);                       // s^{n+1}
  const T* src[1] = {static_cast<const T*>(D.phi)};
  fill_tiles<T, TX, 6, HP, 1>(tp, src, x0, y0 - 2, log2nx, my, threadIdx.x, blockDim.x);
  __syncthreads();
  if (sc.d > 0) stencil2_body<true, T, TX, TY>(D, tp, tm, sc, x0, y0, log2nx);
  else stencil2_body<false, T, TX, TY>(D, tp, tm, sc, x0, y0, log2nx);
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

// stencil tiles: TX = min(nx, 128) columns, TY = min(ny, 32) rows,
// (TX / 4) (TY / 4) threads
template <class T, int TX, int TY>
void launch_stencil_t(int which, const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c,
                      cudaStream_t st) {
  const dim3 grid(c.grid_x, c.grid_y, nmem);
  if (which == 0) k_stencil1<T, TX, TY><<<grid, c.threads, c.smem, st>>>(d, log2nx, log2ny);
  else k_stencil2<T, TX, TY><<<grid, c.threads, c.smem, st>>>(d, log2nx, log2ny);
}
template <class T, int TX, int TY>
void stencil_smem_limits_t(int lim) {
  cudaFuncSetAttribute(k_stencil1<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_stencil2<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}
template <class T, int TY>
void stencil_smem_limits_ty(int lim) {
  stencil_smem_limits_t<T, 16, TY>(lim);
  stencil_smem_limits_t<T, 32, TY>(lim);
  stencil_smem_limits_t<T, 64, TY>(lim);
  stencil_smem_limits_t<T, 128, TY>(lim);
}
template <class T, int TY>
void launch_stencil_ty(int which, const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c,
                       cudaStream_t st) {
  switch (log2nx) {
    case 4: launch_stencil_t<T, 16, TY>(which, d, nmem, log2nx, log2ny, c, st); break;
    case 5: launch_stencil_t<T, 32, TY>(which, d, nmem, log2nx, log2ny, c, st); break;
    case 6: launch_stencil_t<T, 64, TY>(which, d, nmem, log2nx, log2ny, c, st); break;
    default: launch_stencil_t<T, 128, TY>(which, d, nmem, log2nx, log2ny, c, st); break;
  }
}
template <class T>
void launch_stencil(int which, const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c,
                    cudaStream_t st) {
  if (log2ny >= 5) launch_stencil_ty<T, 32>(which, d, nmem, log2nx, log2ny, c, st);
  else launch_stencil_ty<T, 16>(which, d, nmem, log2nx, log2ny, c, st);
}

template <class T>
void launch_step_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                        const LaunchCfg& c, cudaStream_t st) {
  switch (kind) {
    case KIND_STENCIL1:
      launch_stencil<T>(0, d, nmem, log2nx, log2ny, c, st);
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
      launch_stencil<T>(1, d, nmem, log2nx, log2ny, c, st);
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
  stencil_smem_limits_ty<T, 16>(lim);
  stencil_smem_limits_ty<T, 32>(lim);
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
