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

// ======================================= exact low row modes of the Stokes force
// The Stokes solve psi_hat = g_hat / (eta k^4) (Eq. equationNew) multiplies
// the force's lowest modes by up to (L / 2 pi)^4.  There the curl F is a small
// residue of much larger products, and the FP32 rounding of F at every point
// (about eps |F|, spread over all modes) would outweigh it: psi's lowest modes
// need F itself beyond FP32.  This kernel forms, for members with D.low == 2
// (FP32 Stokes), the row DFT coefficients m = 0..lowm of
//   g = c_force (D_x phi D_y^s mu - D_y^s phi D_x mu)
// with F evaluated in double-float from the FP32 phi^{n+1} and an FP32 mu
// (mu as the stage-2 stencil forms it): the differences of two FP32 values
// are exact as pairs, the Eq. p1y weights w0 = 1 - |s|/2, w1 = |s|/2 come from
// the FP64 strain, and every product and sum carries its rounding error.
// The DFT terms F W^{m x} use the double-float twiddle table and are summed
// as double-float pairs; the threads' sums are folded in a fixed order.  The
// result, hi and lo planes of low_rows, feeds k_lowmode_cols like the
// compensated sums of the row pass do for the other FP32 members.
// Work: a CTA takes a tile of up to 32 rows x 64 columns.  phi (halo 2 rows,
// 3 columns) and mu (halo 1 row, 2 columns) of the tile sit in shared memory;
// lane r of every warp owns row j0 + r and its warp's slice of the columns,
// so a thread sums its own row and the twiddle W^{m x} is the same for the
// whole warp (one broadcast load).  The 8 warps' sums of a row are folded in
// warp order; with several column tiles per row the CTAs park their sums in
// a scratch area and the last CTA of a row block to finish (an atomic
// counter; nothing waits) folds them in tile order into low_rows.
constexpr int kLxRows = 32;     // rows per CTA: one per lane
constexpr int kLxCols = 64;     // columns per CTA
constexpr int kLxWarps = 8;
constexpr int kLxValues = 2 * (kLowMExact + 1);   // Re and Im of m = 0..kLowMExact
__host__ __device__ constexpr int lowexact_cols(int nx) { return nx < kLxCols ? nx : kLxCols; }
__host__ __device__ constexpr int lowexact_rows(int ny) { return ny < kLxRows ? ny : kLxRows; }
__host__ __device__ constexpr int lowexact_pitch_phi(int xt) { return (xt + 6) | 1; }
__host__ __device__ constexpr int lowexact_pitch_mu(int xt) { return (xt + 4) | 1; }
__host__ __device__ constexpr int lowexact_smem_floats(int nx, int ny) {
  return (lowexact_rows(ny) + 4) * lowexact_pitch_phi(lowexact_cols(nx)) +
                 (lowexact_rows(ny) + 2) * lowexact_pitch_mu(lowexact_cols(nx)) >
                 2 * kLxValues * kLxWarps * kLxRows
             ? (lowexact_rows(ny) + 4) * lowexact_pitch_phi(lowexact_cols(nx)) +
                   (lowexact_rows(ny) + 2) * lowexact_pitch_mu(lowexact_cols(nx))
             : 2 * kLxValues * kLxWarps * kLxRows;
}
// acc += F w for an FP32-pair F and a double-float w: the product's rounding
// error by fused multiply-adds, the low parts added unnormalised
__device__ __forceinline__ void df_acc_prod(F2& acc, F2 F, float wh, float wl) {
  const float p = __fmul_rn(F.hi, wh);
  float e = __fmaf_rn(F.hi, wh, -p);
  e = __fmaf_rn(F.hi, wl, e);
  e = __fmaf_rn(F.lo, wh, e);
  const F2 s = two_sum_f(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__global__ void __launch_bounds__(kLxWarps * 32) k_lowrows_exact(const MemberDesc* __restrict__ descs, int log2nx,
                                                                 int log2ny, const float4* __restrict__ twff) {
  const MemberDesc& D = descs[blockIdx.z];
  if (D.low != 2) return;                              // uniform per CTA
  extern __shared__ __align__(16) float sm[];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1;
  const int XT = lowexact_cols(nx), RT = lowexact_rows(ny);
  const int PP = lowexact_pitch_phi(XT), PM = lowexact_pitch_mu(XT);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int x0 = blockIdx.x * XT, j0 = blockIdx.y * RT;
  const float* phi = static_cast<const float*>(D.phi);
  float* tp = sm;                                      // phi rows j0 - 2 + r, cols x0 - 3 + c
  float* tm = sm + (RT + 4) * PP;                      // mu rows j0 - 1 + r, cols x0 - 2 + c
  for (int e = tid; e < (RT + 4) * (XT + 6); e += nt) {
    const int r = e / (XT + 6), c = e - r * (XT + 6);
    tp[r * PP + c] = __ldg(phi + ((size_t)((j0 - 2 + r) & my) << log2nx) + ((x0 - 3 + c) & mx));
  }
  __syncthreads();
  const Shear<float> sc(*D.st, true);                  // s^{n+1}
  {                                                    // mu in FP32, as the stage-2 stencil forms it
    const float a = (float)D.a, b = (float)D.b, kappa = (float)D.kappa;
    const float cxx = 1.f + sc.s * sc.s, cxy = 2.f * sc.s;
    const float kxx = kappa * cxx * (float)D.inv_h2, kxy = kappa * cxy * (float)D.inv_4h2,
                kyy = kappa * (float)D.inv_h2;
    for (int e = tid; e < (RT + 2) * (XT + 4); e += nt) {
      const int r = e / (XT + 4), c = e - r * (XT + 4);
      const float* pc_ = tp + (r + 1) * PP + (c + 1);  // the centre in the phi tile
      const float pc = pc_[0];
      const float sxx = pc_[1] - 2.f * pc + pc_[-1];
      const float syy = pc_[PP] - 2.f * pc + pc_[-PP];
      const float sxy = pc_[PP + 1] - pc_[-PP + 1] - pc_[PP - 1] + pc_[-PP - 1];
      const float klap = kxx * sxx - kxy * sxy + kyy * syy;
      tm[r * PM + c] = pc * (b * (pc * pc) - a) - klap;
    }
  }
  __syncthreads();
  const double s1 = D.st->s1;
  const double w1d = 0.5 * (s1 < 0.0 ? -s1 : s1);
  const F2 W0 = f2_of(1.0 - w1d), W1 = f2_of(w1d);
  const F2 KF = f2_of(D.c_force * D.inv_2h * D.inv_2h);
  const int dd = sc.d;                                 // the diagonal's x offset at row j + 1
  const int lowm = D.lowm, nv = 2 * (lowm + 1);
  const int tshift = LOG2_NMAX - log2nx;
  const int lane = tid & 31, warp = tid >> 5;
  const int cw = XT / kLxWarps > 0 ? XT / kLxWarps : 1;        // columns per warp
  const int c0 = warp * cw, c1 = min(XT, c0 + cw);
  F2 acc[kLxValues];
#pragma unroll
  for (int k = 0; k < kLxValues; ++k) acc[k] = F2{0.f, 0.f};
  if (lane < RT) {
    const float* prow = tp + (lane + 2) * PP + 3;     // phi row j, col 0 of the tile
    const float* mrow = tm + (lane + 1) * PM + 2;     // mu row j
    for (int c = c0; c < c1; ++c) {
      const float* p = prow + c;
      const float* q = mrow + c;
      const F2 dxp = two_sum_f(p[1], -p[-1]);
      const F2 dxm = two_sum_f(q[1], -q[-1]);
      const F2 dyp = df_add(df_mul(W0, two_sum_f(p[PP], -p[-PP])), df_mul(W1, two_sum_f(p[PP + dd], -p[-PP - dd])));
      const F2 dym = df_add(df_mul(W0, two_sum_f(q[PM], -q[-PM])), df_mul(W1, two_sum_f(q[PM + dd], -q[-PM - dd])));
      const F2 F = df_mul(df_add(df_mul(dxp, dym), df_neg(df_mul(dyp, dxm))), KF);
      df_acc(acc[0], F);
      const int x = x0 + c;
#pragma unroll
      for (int m = 1; m <= kLowMExact; ++m) {
        if (m > lowm) break;
        const float4 w = __ldg(twff + (((m * x) & mx) << tshift));   // cos, sin of 2 pi m x / nx as pairs
        df_acc_prod(acc[2 * m], F, w.x, w.y);
        df_acc_prod(acc[2 * m + 1], F, -w.z, -w.w);
      }
    }
  }
  __syncthreads();                                     // tiles no longer read: the fold reuses them
  float* red = sm;                                     // value v, warp w, lane r: [(2 v) W + w] 32 + r
#pragma unroll
  for (int v = 0; v < kLxValues; ++v) {
    if (v >= nv) break;
    const F2 r = fast_two_sum_f(acc[v].hi, acc[v].lo);
    red[((2 * v) * kLxWarps + warp) * 32 + lane] = r.hi;
    red[((2 * v + 1) * kLxWarps + warp) * 32 + lane] = r.lo;
  }
  __syncthreads();
  // item e < RT nv: row r = e mod RT, value v = e / RT, the warps in order
  const int nxb = gridDim.x;
  float2* lrh = static_cast<float2*>(D.low_rows);
  float2* lrl = lrh + ((size_t)(kLowM + 1) << log2ny);
  float2* part = lrl + ((size_t)(kLowM + 1) << log2ny);           // [tile][v][row] (hi, lo)
  int* cnt = reinterpret_cast<int*>(part + ((size_t)nxb * kLxValues << log2ny));
  for (int e = tid; e < RT * nv; e += nt) {
    const int r = e % RT, v = e / RT;
    F2 sum{0.f, 0.f};
    for (int w = 0; w < kLxWarps; ++w)
      sum = df_add(sum, F2{red[((2 * v) * kLxWarps + w) * 32 + r], red[((2 * v + 1) * kLxWarps + w) * 32 + r]});
    const int j = j0 + r, m = v >> 1;
    if (nxb == 1) {
      reinterpret_cast<float*>(lrh + ((size_t)m << log2ny) + j)[v & 1] = sum.hi;
      reinterpret_cast<float*>(lrl + ((size_t)m << log2ny) + j)[v & 1] = sum.lo;
    } else {
      part[(((size_t)blockIdx.x * kLxValues + v) << log2ny) + j] = float2{sum.hi, sum.lo};
    }
  }
  if (nxb == 1) return;
  __threadfence();                                     // this tile's sums visible before it is counted
  __syncthreads();
  __shared__ int last;
  if (tid == 0) last = atomicAdd(cnt + blockIdx.y, 1) == nxb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = tid; e < RT * nv; e += nt) {
    const int r = e % RT, v = e / RT;
    const int j = j0 + r, m = v >> 1;
    F2 tot{0.f, 0.f};
    for (int xb = 0; xb < nxb; ++xb) {
      const float2 pv = __ldcg(part + (((size_t)xb * kLxValues + v) << log2ny) + j);
      tot = df_add(tot, F2{pv.x, pv.y});
    }
    reinterpret_cast<float*>(lrh + ((size_t)m << log2ny) + j)[v & 1] = tot.hi;
    reinterpret_cast<float*>(lrl + ((size_t)m << log2ny) + j)[v & 1] = tot.lo;
  }
  if (tid == 0) cnt[blockIdx.y] = 0;                   // ready for the next step
}

// ----------------------------------------------------------------- launchers
void launch_lowrows_exact(const MemberDesc* d, int nmem, int log2nx, int log2ny, const float4* twff,
                          cudaStream_t st) {
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const size_t smem = (size_t)lowexact_smem_floats(nx, ny) * sizeof(float);
  const dim3 grid(nx / lowexact_cols(nx), ny / lowexact_rows(ny), nmem);
  k_lowrows_exact<<<grid, kLxWarps * 32, smem, st>>>(d, log2nx, log2ny, twff);
}
size_t lowrows_bytes(int nx, int ny) {
  // hi and lo planes of the coefficients, the exact path's per-tile sums and
  // its row-block counters
  return 2 * (size_t)(kLowM + 1) * ny * sizeof(float2) +
         (size_t)(nx / lowexact_cols(nx)) * kLxValues * ny * sizeof(float2) +
         (size_t)(ny / lowexact_rows(ny)) * sizeof(int);
}
void launch_step_state_init(const MemberDesc* d, int nmem, cudaStream_t st) {
  k_step_state_init<<<(nmem + 127) / 128, 128, 0, st>>>(d, nmem);
}

// stencil tiles: TX = min(nx, 128) columns, TY = min(ny, 32) rows,
// (TX / 4) (TY / 4) threads
template <class T, int TX, int TY>
void launch_stencil_t(const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c, cudaStream_t st) {
  const dim3 grid(c.grid_x, c.grid_y, nmem);
  k_stencil2<T, TX, TY><<<grid, c.threads, c.smem, st>>>(d, log2nx, log2ny);
}
template <class T, int TX, int TY>
void stencil_smem_limits_t(int lim) {
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
void launch_stencil_ty(const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c, cudaStream_t st) {
  switch (log2nx) {
    case 4: launch_stencil_t<T, 16, TY>(d, nmem, log2nx, log2ny, c, st); break;
    case 5: launch_stencil_t<T, 32, TY>(d, nmem, log2nx, log2ny, c, st); break;
    case 6: launch_stencil_t<T, 64, TY>(d, nmem, log2nx, log2ny, c, st); break;
    default: launch_stencil_t<T, 128, TY>(d, nmem, log2nx, log2ny, c, st); break;
  }
}
// the stage-2 stencil; the tile height TY (16 or 32, at most ny) is the launch's variant
template <class T>
void launch_stencil(const MemberDesc* d, int nmem, int log2nx, int log2ny, const LaunchCfg& c, cudaStream_t st) {
  if (c.variant == 32) launch_stencil_ty<T, 32>(d, nmem, log2nx, log2ny, c, st);
  else launch_stencil_ty<T, 16>(d, nmem, log2nx, log2ny, c, st);
}

template <class T>
void launch_step_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                        const LaunchCfg& c, cudaStream_t st) {
  switch (kind) {
    case KIND_STENCIL2: launch_stencil<T>(d, nmem, log2nx, log2ny, c, st); break;
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

template <class T>
void set_step_smem_limits() {
  const int lim = 220 * 1024;   // dynamic part; leaves room for static shared memory
  set_row_smem_limits<T>(lim);
  set_col_smem_limits<T>(lim);
  stencil_smem_limits_ty<T, 16>(lim);
  stencil_smem_limits_ty<T, 32>(lim);
  if (sizeof(T) == 4) cudaFuncSetAttribute(k_lowrows_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

#define SHF_INST(T)                                                                                      \
  template void launch_step_kernel<T>(int, const MemberDesc*, int, int, int, const cplx<T>*,             \
                                      const LaunchCfg&, cudaStream_t);                                    \
  template int step_kernel_occupancy<T>(int, int, int, int, size_t);                                      \
  template void set_step_smem_limits<T>();

SHF_INST(float)
SHF_INST(double)

}  // namespace shf
