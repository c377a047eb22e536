// Kernels of one time step (Appendix B of arXiv:0710.5912), templated on the
// working precision T (float or double).  A step is eight launches per grid
// size:
//
//   stencil1     item 1 + item 2's advection at s = s^n (Eq. advective with the
//                Eq. p1y stencils): phi* = phi - dt J(psi, phi) and omega* =
//                omega - dt J(psi, omega), real (FP32 inertial members: the
//                increment -dt J(psi, omega) alone, see step_cols.cu); omega*
//                is written at the relabelled positions when the strain wraps
//                during the step.
//   rowfwd_phi   row (x) transforms of the phi*, f = phi^3 and omega* row
//                pairs -> x-spectral buffers, plus each row's real Nyquist
//                coefficient of phi* and omega*.
//   colpass_phi  column (y) transforms of phi*, f; the Cahn-Hilliard update of
//                item 1 in the paper's increment form
//                  phi^{n+1} = phi* + (1 + D4/2)^-1 (-D2 phi* - D4 phi* + D2 f),
//                Nyquist modes of phi^{n+1} zeroed; the increment back along y.
//   rowinv_phi   phi^{n+1} = phi* + row inverse of the increment (minus phi*'s
//                Nyquist column), written at the relabelled positions at a wrap.
//   stencil2     mu = -a phi + b phi^3 - kappa lap_c phi and the body-force curl
//                F = d_x phi d_y mu - d_y phi d_x mu at s = s^{n+1} (Eq. G);
//                g = -F/rho, or -F/eta for Stokes, real.
//   rowfwd_g     row transforms of g row pairs (FP32: plus the low row modes
//                of g with compensated sums).
//   lowmode      FP32: the column DFT of those low row modes.
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
// This file holds the stencils and the launch dispatch; the transform kernels
// are in step_rows.cu and step_cols.cu (compiled per transform length).
//
// Execution: the FP32 stage-1 stencil (nx >= 128) streams row strips through
// registers; the other stencils run on 2D tiles, 4 x 4 outputs per thread; the
// transform kernels are persistent -- every instance walks its work items (row
// pairs or column chunks) with a grid stride and, while transforming one item,
// streams the next item's input into a shared-memory staging buffer with
// cp.async, so the loads in flight hold shared memory rather than registers.
// The FFT keeps 8 (or, in the FP32 row passes, 16) points per thread in
// registers (fft_block.cuh).
//
// Layout: real fields ny x nx row-major.  x-spectral buffers hold, for each row
// j, the modes m = 0..nx/2-1 of the row's real DFT (the Nyquist column is
// carried separately as one real per row), tiled in chunks of CL = 2^LC
// adjacent modes: element (j, m) sits at ((m >> LC) ny + j) CL + (m & (CL-1)),
// so a chunk of a row pair is 32 contiguous bytes and a column is one strided
// run.  The 1/(nx ny) of the inverse transforms is applied in the column passes.
// Each launch covers a batch of members of one size (one descriptor each).
#include "step_common.cuh"

namespace shf {

__global__ void k_step_state_init(const MemberDesc* __restrict__ descs, int nmem) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nmem) step_state_set(descs[r], descs[r].st->n);
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

// Fill rows [0, H) of NF tiles (tile column c <-> x0 - OFF + c, OFF = 2 or 6,
// width TX + 2 OFF) from NF fields at rows y0 - HY + r (periodic), with
// asynchronous copies (all of a thread's copies are in flight at once) of two
// reals each: the interior in pairs, the OFF halo columns on each side as
// pairs.  Returns after the copies have landed (this thread's; the caller
// then synchronises the CTA).
template <class T>
__device__ __forceinline__ void cp_async_pair(T* dst, const T* src) {
  if (sizeof(T) == 4) cp_async8(dst, src);
  else cp_async16(dst, src);
}
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
      const T* g = row + x0 + 4 * k;
      T* d = trow + OFF + 4 * k;
      cp_async_pair(d, g);
      cp_async_pair(d + 2, g + 2);
    } else {
      const int h = k - QX;                               // 0 .. 2 HP - 1
      const int side = h / HP, j = h - side * HP;         // left (0) or right (1) halo, pair j
      const int c = side == 0 ? 2 * j : OFF + TX + 2 * j;
      const int x = (x0 - OFF + c) & mx;                  // even, so the pair is contiguous
      cp_async_pair(trow + c, row + x);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
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
      if (D.wspec) {
#pragma unroll
        for (int p = 0; p < 4; ++p) r[p] = advect_incr(dt, dyp[p], dxf[p], dxp[p], dyf[p]);
      } else {
#pragma unroll
        for (int p = 0; p < 4; ++p) r[p] = C.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
      }
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
  // kappa and the difference scalings folded into the three Laplacian weights
  const T kxx = kappa * cxx * ih2, kxy = kappa * cxy * i4h2, kyy = kappa * ih2;
  // mu tile row rm <-> y0 - 1 + rm <-> phi tile row rm + 1; mu quad at tile col 4 (k + 1).
  // Work unit: one quad column k over RPT consecutive mu rows, with a three-row
  // window of phi (one new phi row per mu row).
  constexpr int NT = QX * (TY / 4);                    // threads of the CTA
  constexpr int RG = NT / NQ;                          // row groups
  constexpr int RPT = (HM + RG - 1) / RG;              // mu rows per unit
  if (tid < NQ * RG) {
    const int k = tid % NQ, rg = tid / NQ;
    const int c = 4 * (k + 1);
    const int r0 = rg * RPT;
    Six<T> Dn = ld6(tp + r0 * W + c), Cn = ld6(tp + (r0 + 1) * W + c);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {                     // a fixed trip count, so the window stays in registers
      const int rm = r0 + i;
      if (rm >= HM) break;
      const Six<T> Un = ld6(tp + (rm + 2) * W + c);
      T m[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const T pc = Cn.v[p + 1];
        const T sxx = Cn.v[p + 2] - T(2) * pc + Cn.v[p];          // unscaled second differences
        const T syy = Un.v[p + 1] - T(2) * pc + Dn.v[p + 1];
        const T sxy = Un.v[p + 2] - Dn.v[p + 2] - Un.v[p] + Dn.v[p];
        const T klap = kxx * sxx - kxy * sxy + kyy * syy;          // kappa L_s phi
        m[p] = pc * (b * (pc * pc) - a) - klap;
      }
      st4(tm + rm * W + c, m[0], m[1], m[2], m[3]);
      Dn = Cn;
      Cn = Un;
    }
  }
  __syncthreads();
  const int q = tid % QX, g = tid / QX;
  const T cf = (T)D.c_force;
  T* gout = static_cast<T*>(D.gbuf);
  const int x = x0 + 4 * q;
  // the 8-wide rows of output block (cols x - 2 .. x + 5) start at tile col 4 q + 4;
  // output row y0 + 4 g + o is phi tile row 4 g + 2 + o and mu tile row 4 g + 1 + o
  const T* pcol = tp + 4 * q + 4;
  const T* mcol = tm + 4 * q + 4;
  Row8<T> pD = ld8(pcol + (4 * g + 1) * W), pC = ld8(pcol + (4 * g + 2) * W);
  Row8<T> mD = ld8(mcol + (4 * g) * W), mC = ld8(mcol + (4 * g + 1) * W);
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int y = y0 + 4 * g + o;
    const Row8<T> pU = ld8(pcol + (4 * g + 3 + o) * W), mU = ld8(mcol + (4 * g + 2 + o) * W);
    T dxp[4], dyp[4], dxm[4], dym[4];
    grad4<NEG>(pU, pC, pD, sc.w0, sc.w1, inv2h, dxp, dyp);
    grad4<NEG>(mU, mC, mD, sc.w0, sc.w1, inv2h, dxm, dym);
    T r[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) r[p] = cf * diff_of_products(dxp[p], dym[p], dyp[p], dxm[p]);
    st4(gout + ((size_t)y << log2nx) + x, r[0], r[1], r[2], r[3]);
    pD = pC;
    pC = pU;
    mD = mC;
    mC = mU;
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

// ------------------------------------------------- streamed stage-1 stencil
// FP32, nx >= 128: the stage-1 stencil without shared tiles.  A warp owns a
// 128-column segment (4 columns per lane) and walks a strip of consecutive
// rows, keeping the rows j - 1, j, j + 1 of each field in registers: each row
// is one 16-byte load per lane, the x +-2 halo comes from the neighbouring
// lanes by shuffles (lanes 0 and 31 load theirs), the loads of row j + 2 are
// issued before row j is computed, and lane 0 asks L2 for the warp's row
// segments kStreamPrefetch rows ahead (bulk prefetch).  The grid holds exactly
// the resident CTAs, and the rows are split evenly over the warps, so every
// warp streams about the same number of rows in one wave.  Same arithmetic,
// in the same order, as k_stencil1.
constexpr int kStreamPrefetch = 4;      // rows of L2 prefetch ahead (measured best of 2..16)
constexpr int kStreamThreads = 128;     // four warps per CTA

struct RawRow {
  float4 q;       // this lane's four columns
  float2 l, r;    // lane 0: the two columns left of the segment; lane 31: the two right of it
};
__device__ __forceinline__ RawRow load_raw(const float* rowp, int x, int lane, int mx) {
  RawRow w;
  w.q = __ldg(reinterpret_cast<const float4*>(rowp + x));
  w.l = lane == 0 ? __ldg(reinterpret_cast<const float2*>(rowp + ((x - 2) & mx))) : float2{0.f, 0.f};
  w.r = lane == 31 ? __ldg(reinterpret_cast<const float2*>(rowp + ((x + 4) & mx))) : float2{0.f, 0.f};
  return w;
}
// columns x - 2 .. x + 5 of a row from the lanes' quads
__device__ __forceinline__ Row8<float> widen(const RawRow& w, int lane) {
  const unsigned full = 0xffffffffu;
  float l0 = __shfl_up_sync(full, w.q.z, 1), l1 = __shfl_up_sync(full, w.q.w, 1);
  float r0 = __shfl_down_sync(full, w.q.x, 1), r1 = __shfl_down_sync(full, w.q.y, 1);
  if (lane == 0) {
    l0 = w.l.x;
    l1 = w.l.y;
  }
  if (lane == 31) {
    r0 = w.r.x;
    r1 = w.r.y;
  }
  return Row8<float>{{l0, l1, w.q.x, w.q.y, w.q.z, w.q.w, r0, r1}};
}

template <bool NEG, bool STOKES>
__device__ __forceinline__ void stencil1_stream_body(const MemberDesc& D, const Shear<float>& sc, int x, int y0,
                                                     int nrows, int log2nx, int my, int lane) {
  using T = float;
  const int nx = 1 << log2nx, mx = nx - 1;
  const bool wrap = D.remap && sc.dK != 0;
  const T dt = (T)D.dt, inv2h = (T)D.inv_2h;
  const T* ph = static_cast<const T*>(D.phi);
  const T* ps = static_cast<const T*>(D.psi);
  const T* om = static_cast<const T*>(D.omega);
  T* phis = static_cast<T*>(D.phi_star);
  T* oms = static_cast<T*>(D.omega_star);
  auto rp = [&](const T* f, int y) { return f + ((size_t)(y & my) << log2nx); };
  Row8<T> pD = widen(load_raw(rp(ph, y0 - 1), x, lane, mx), lane), pC = widen(load_raw(rp(ph, y0), x, lane, mx), lane);
  Row8<T> sD = widen(load_raw(rp(ps, y0 - 1), x, lane, mx), lane), sC = widen(load_raw(rp(ps, y0), x, lane, mx), lane);
  Row8<T> oD, oC;
  if (!STOKES) {
    oD = widen(load_raw(rp(om, y0 - 1), x, lane, mx), lane);
    oC = widen(load_raw(rp(om, y0), x, lane, mx), lane);
  }
  RawRow pN = load_raw(rp(ph, y0 + 1), x, lane, mx), sN = load_raw(rp(ps, y0 + 1), x, lane, mx), oN;
  if (!STOKES) oN = load_raw(rp(om, y0 + 1), x, lane, mx);
#pragma unroll 2
  for (int j = 0; j < nrows; ++j) {
    const int y = y0 + j;
    if (lane == 0) {                                    // the warp's 512-byte segments, rows ahead
      l2_prefetch(rp(ph, y + kStreamPrefetch) + x, 512);
      l2_prefetch(rp(ps, y + kStreamPrefetch) + x, 512);
      if (!STOKES) l2_prefetch(rp(om, y + kStreamPrefetch) + x, 512);
    }
    const Row8<T> pU = widen(pN, lane), sU = widen(sN, lane);
    Row8<T> oU;
    if (!STOKES) oU = widen(oN, lane);
    if (j + 1 < nrows) {                                // row y + 2 in flight while row y is computed
      pN = load_raw(rp(ph, y + 2), x, lane, mx);
      sN = load_raw(rp(ps, y + 2), x, lane, mx);
      if (!STOKES) oN = load_raw(rp(om, y + 2), x, lane, mx);
    }
    T dxp[4], dyp[4];
    grad4<NEG>(sU, sC, sD, sc.w0, sc.w1, inv2h, dxp, dyp);
    {
      T dxf[4], dyf[4];
      grad4<NEG>(pU, pC, pD, sc.w0, sc.w1, inv2h, dxf, dyf);
      T r[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) r[p] = pC.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
      st4(phis + ((size_t)y << log2nx) + x, r[0], r[1], r[2], r[3]);
    }
    if (!STOKES) {
      T dxf[4], dyf[4];
      grad4<NEG>(oU, oC, oD, sc.w0, sc.w1, inv2h, dxf, dyf);
      T r[4];
      if (D.wspec) {
#pragma unroll
        for (int p = 0; p < 4; ++p) r[p] = advect_incr(dt, dyp[p], dxf[p], dxp[p], dyf[p]);
      } else {
#pragma unroll
        for (int p = 0; p < 4; ++p) r[p] = oC.v[p + 2] - dt * (dyp[p] * dxf[p] - dxp[p] * dyf[p]);
      }
      T* orow = oms + ((size_t)y << log2nx);
      if (!wrap) {
        st4(orow + x, r[0], r[1], r[2], r[3]);
      } else {
        const int sh_y = remap_shift(sc.dK, D.ratio, y, nx);
#pragma unroll
        for (int p = 0; p < 4; ++p) orow[(x + p + sh_y) & mx] = r[p];
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

// grid (nx / 128, G, members); warp w of CTA (bx, by) streams strip
// s = 4 by + w of the 4 G equal strips of rows
__global__ void __launch_bounds__(kStreamThreads, 4) k_stencil1_stream(const MemberDesc* __restrict__ descs,
                                                                       int log2nx, int log2ny) {
  const MemberDesc& D = descs[blockIdx.z];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ny = 1 << log2ny, my = ny - 1;
  const int x = blockIdx.x * 128 + 4 * lane;
  const int S = gridDim.y * (kStreamThreads / 32), s = blockIdx.y * (kStreamThreads / 32) + w;
  const int y0 = (int)(((long long)s * ny) / S), y1 = (int)(((long long)(s + 1) * ny) / S);
  const Shear<float> sc(*D.st, false);                  // s^n
  if (D.stokes) {
    if (sc.d > 0) stencil1_stream_body<true, true>(D, sc, x, y0, y1 - y0, log2nx, my, lane);
    else stencil1_stream_body<false, true>(D, sc, x, y0, y1 - y0, log2nx, my, lane);
  } else {
    if (sc.d > 0) stencil1_stream_body<true, false>(D, sc, x, y0, y1 - y0, log2nx, my, lane);
    else stencil1_stream_body<false, false>(D, sc, x, y0, y1 - y0, log2nx, my, lane);
  }
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
// the tile height TY (16 or 32, at most ny) is the launch's variant; variant
// kStencilStream selects the streamed FP32 stage-1 stencil
template <class T>
void launch_stencil(int which, const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c,
                    cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (which == 0 && c.variant == kStencilStream) {
      k_stencil1_stream<<<dim3(c.grid_x, c.grid_y, nmem), c.threads, 0, st>>>(d, log2nx, log2ny);
      return;
    }
  }
  if (c.variant == 32) launch_stencil_ty<T, 32>(which, d, nmem, log2nx, log2ny, c, st);
  else launch_stencil_ty<T, 16>(which, d, nmem, log2nx, log2ny, c, st);
}

template <class T>
void launch_step_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                        const LaunchCfg& c, cudaStream_t st) {
  switch (kind) {
    case KIND_STENCIL1: launch_stencil<T>(0, d, nmem, log2nx, log2ny, c, st); break;
    case KIND_STENCIL2: launch_stencil<T>(1, d, nmem, log2nx, log2ny, c, st); break;
    case KIND_COLPASS_PHI:
    case KIND_COLPASS_FLOW: launch_col_kernel<T>(kind, d, nmem, log2nx, log2ny, tw, c, st); break;
    default: launch_row_kernel<T>(kind, d, nmem, log2nx, log2ny, tw, c, st); break;
  }
}

// CTAs of a persistent kind that fit on one SM at (threads, smem); log2n is the
// kind's transform length (log2 nx for row kinds, log2 ny for column kinds)
template <class T>
int step_kernel_occupancy(int kind, int log2n, int variant, int threads, size_t smem) {
  if (kind == KIND_COLPASS_PHI || kind == KIND_COLPASS_FLOW) return col_kernel_occupancy<T>(log2n, threads, smem);
  return row_kernel_occupancy<T>(kind, log2n, variant, threads, smem);
}

int stencil1_stream_occupancy() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stencil1_stream, kStreamThreads, 0) != cudaSuccess) nb = 1;
  return nb < 1 ? 1 : nb;
}

template <class T>
void set_step_smem_limits() {
  const int lim = 220 * 1024;   // dynamic part; leaves room for static shared memory
  set_row_smem_limits<T>(lim);
  set_col_smem_limits<T>(lim);
  stencil_smem_limits_ty<T, 16>(lim);
  stencil_smem_limits_ty<T, 32>(lim);
}

#define SHF_INST(T)                                                                                      \
  template void launch_step_kernel<T>(int, const MemberDesc*, int, int, int, const cplx<T>*,             \
                                      const LaunchCfg&, cudaStream_t);                                    \
  template int step_kernel_occupancy<T>(int, int, int, int, size_t);                                      \
  template void set_step_smem_limits<T>();

SHF_INST(float)
SHF_INST(double)

}  // namespace shf
