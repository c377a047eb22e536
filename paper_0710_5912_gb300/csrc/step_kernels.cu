// Kernels of one time step (Appendix B of arXiv:0710.5912), templated on the
// working precision T (float or double).  A step is seven launches per grid
// size (six for FP64):
//
//   stage1       item 1 + item 2's advection at s = s^n (Eq. advective with the
//                Eq. p1y stencils), fused with the row (x) transforms of what
//                it makes: phi* = phi - dt J(psi, phi) (written out, the base
//                of phi's increment) -> xs_phi; f = phi^3 -> xs_f; omega* =
//                omega - dt J(psi, omega), or for FP32 inertial members the
//                increment -dt J(psi, omega) alone (omega is carried as its 2D
//                transform w_hat, step_cols.cu) -> xs_w, at the relabelled
//                positions when the strain wraps during the step
//                (k_stage1_rows, step_rows.cu).
//   colpass_phi  column (y) transforms of phi*, f; the Cahn-Hilliard update of
//                item 1 in the paper's increment form
//                  phi^{n+1} = phi* + (1 + D4/2)^-1 (-D2 phi* - D4 phi* + D2 f),
//                Nyquist modes of phi^{n+1} zeroed; the increment back along y.
//   rowinv_phi   phi^{n+1} = phi* + row inverse of the increment (minus phi*'s
//                Nyquist column), written at the relabelled positions at a wrap.
//   stage2       mu = -a phi + b phi^3 - kappa lap_c phi and the body-force curl
//                F = d_x phi d_y mu - d_y phi d_x mu at s = s^{n+1} (Eq. G);
//                g = -F/rho, or -F/eta for Stokes, computed straight into the
//                row transform of g (k_rowfwd mode 1; FP32 inertial: plus the
//                low row modes of g with compensated sums).
//   lowmode      FP32: the column DFT of the low row modes of g (for Stokes
//                members, first the exact low row modes, k_lowrows_exact
//                below).
//   colpass_flow column transforms; Crank-Nicolson vorticity update
//                omega^{n+1} = omega* + (dt g - 2C omega*) / (1 + C) with
//                C = dt (eta / rho) k^2 / 2, and the Poisson solve
//                psi = omega / k^2 (items 2-3), or the Stokes solve
//                psi = g / k^4; inverse column transforms.
//   rowinv_flow  psi rows and omega^{n+1}; advances the step counter.
//
// Transforming only the increments keeps the FP32 rounding of a step
// proportional to the change of the field instead of to the field itself.
//
// This file holds the exact low-mode kernel of the Stokes force, the state
// seeding and the launch dispatch; the transform kernels (with the fused
// stencils) are in step_rows.cu and step_cols.cu, compiled per transform
// length.  The transform kernels are persistent -- every instance walks its
// work items (row pairs or column chunks) with a grid stride and, while
// transforming one item, streams the next item's input into shared memory
// (cp.async) or L2 (bulk prefetch).  The FFT keeps 8 (FP64) or 16 (FP32)
// points per thread in registers (fft_block.cuh).
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
// Work: a CTA takes up to 32 rows x 64 columns of the first half of the rows
// and the same columns shifted by nx / 2, folded before the DFT: since
// W^{m (x + nx/2)} = (-1)^m W^{m x}, the terms of both are
// (F(x) + F(x + nx/2)) W^{m x} for even m and (F(x) - F(x + nx/2)) W^{m x}
// for odd m, half the products.  phi (halo 2 rows, 3 columns) and mu (halo 1
// row, 2 columns) of both tiles sit in shared memory; lane r of every warp owns
// row j0 + r and its warp's slice of the columns, so a thread sums its own row
// and the twiddle W^{m x} is the same for the whole warp (one broadcast load).  The 8 warps' sums of a row are folded in
// warp order; with several column tiles per row the CTAs park their sums in
// a scratch area and the last CTA of a row block to finish (an atomic
// counter; nothing waits) folds them in tile order into low_rows.
constexpr int kLxRows = 32;     // rows per CTA: one per lane
constexpr int kLxCols = 64;     // columns per CTA
constexpr int kLxWarps = 8;
constexpr int kLxValues = 2 * (kLowMExact + 1);   // Re and Im of m = 0..kLowMExact
// a CTA's tile covers XT columns of the first half of the rows and the same
// columns shifted by nx / 2 (the DFT folds them: W^{m (x + nx/2)} = (-1)^m W^{m x})
__host__ __device__ constexpr int lowexact_cols(int nx) { return nx / 2 < kLxCols ? nx / 2 : kLxCols; }
__host__ __device__ constexpr int lowexact_rows(int ny) { return ny < kLxRows ? ny : kLxRows; }
__host__ __device__ constexpr int lowexact_pitch_phi(int xt) { return (xt + 6) | 1; }
__host__ __device__ constexpr int lowexact_pitch_mu(int xt) { return (xt + 4) | 1; }
__host__ __device__ constexpr int lowexact_tile_floats(int nx, int ny) {   // one phi tile and its mu tile
  return (lowexact_rows(ny) + 4) * lowexact_pitch_phi(lowexact_cols(nx)) +
         (lowexact_rows(ny) + 2) * lowexact_pitch_mu(lowexact_cols(nx));
}
__host__ __device__ constexpr int lowexact_smem_floats(int nx, int ny) {
  return 2 * lowexact_tile_floats(nx, ny) > 2 * kLxValues * kLxWarps * kLxRows ? 2 * lowexact_tile_floats(nx, ny)
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
  // half h = 0, 1: phi rows j0 - 2 + r, cols x0 + h nx/2 - 3 + c; mu rows
  // j0 - 1 + r, cols x0 + h nx/2 - 2 + c
  const int TF = lowexact_tile_floats(nx, ny);
  for (int e = tid; e < 2 * (RT + 4) * (XT + 6); e += nt) {
    const int h = e / ((RT + 4) * (XT + 6)), e1 = e - h * (RT + 4) * (XT + 6);
    const int r = e1 / (XT + 6), c = e1 - r * (XT + 6);
    sm[h * TF + r * PP + c] =
        __ldg(phi + ((size_t)((j0 - 2 + r) & my) << log2nx) + ((x0 + h * (nx >> 1) - 3 + c) & mx));
  }
  __syncthreads();
  const Shear<float> sc(*D.st, true);                  // s^{n+1}
  {                                                    // mu in FP32, as the stage-2 stencil forms it
    const float a = (float)D.a, b = (float)D.b, kappa = (float)D.kappa;
    const float cxx = 1.f + sc.s * sc.s, cxy = 2.f * sc.s;
    const float kxx = kappa * cxx * (float)D.inv_h2, kxy = kappa * cxy * (float)D.inv_4h2,
                kyy = kappa * (float)D.inv_h2;
    for (int e = tid; e < 2 * (RT + 2) * (XT + 4); e += nt) {
      const int h = e / ((RT + 2) * (XT + 4)), e1 = e - h * (RT + 2) * (XT + 4);
      const int r = e1 / (XT + 4), c = e1 - r * (XT + 4);
      const float* pc_ = sm + h * TF + (r + 1) * PP + (c + 1);   // the centre in half h's phi tile
      const float pc = pc_[0];
      const float sxx = pc_[1] - 2.f * pc + pc_[-1];
      const float syy = pc_[PP] - 2.f * pc + pc_[-PP];
      const float sxy = pc_[PP + 1] - pc_[-PP + 1] - pc_[PP - 1] + pc_[-PP - 1];
      const float klap = kxx * sxx - kxy * sxy + kyy * syy;
      sm[h * TF + (RT + 4) * PP + r * PM + c] = pc * (b * (pc * pc) - a) - klap;
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
  // F at (row j, col x) of half h in double-float, p and q pointing at phi and mu there
  auto curl = [&](const float* p, const float* q) {
    const F2 dxp = two_sum_f(p[1], -p[-1]);
    const F2 dxm = two_sum_f(q[1], -q[-1]);
    const F2 dyp = df_add(df_mul(W0, two_sum_f(p[PP], -p[-PP])), df_mul(W1, two_sum_f(p[PP + dd], -p[-PP - dd])));
    const F2 dym = df_add(df_mul(W0, two_sum_f(q[PM], -q[-PM])), df_mul(W1, two_sum_f(q[PM + dd], -q[-PM - dd])));
    return df_mul(df_add(df_mul(dxp, dym), df_neg(df_mul(dyp, dxm))), KF);
  };
  if (lane < RT) {
    const float* prow = sm + (lane + 2) * PP + 3;                // phi row j, col 0 of half 0's tile
    const float* mrow = sm + (RT + 4) * PP + (lane + 1) * PM + 2;   // mu row j
    for (int c = c0; c < c1; ++c) {
      const F2 Fa = curl(prow + c, mrow + c);                    // x
      const F2 Fb = curl(prow + TF + c, mrow + TF + c);          // x + nx / 2
      const F2 E = df_add(Fa, Fb), O = df_add(Fa, df_neg(Fb));   // for even and odd m
      df_acc(acc[0], E);
      const int x = x0 + c;
#pragma unroll
      for (int m = 1; m <= kLowMExact; ++m) {
        if (m > lowm) break;
        const float4 w = __ldg(twff + (((m * x) & mx) << tshift));   // cos, sin of 2 pi m x / nx as pairs
        const F2 G = (m & 1) ? O : E;
        df_acc_prod(acc[2 * m], G, w.x, w.y);
        df_acc_prod(acc[2 * m + 1], G, -w.z, -w.w);
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
  const dim3 grid((nx / 2) / lowexact_cols(nx), ny / lowexact_rows(ny), nmem);
  k_lowrows_exact<<<grid, kLxWarps * 32, smem, st>>>(d, log2nx, log2ny, twff);
}
size_t lowrows_bytes(int nx, int ny) {
  // hi and lo planes of the coefficients, the exact path's per-tile sums and
  // its row-block counters
  return 2 * (size_t)(kLowM + 1) * ny * sizeof(float2) +
         (size_t)((nx / 2) / lowexact_cols(nx)) * kLxValues * ny * sizeof(float2) +
         (size_t)(ny / lowexact_rows(ny)) * sizeof(int);
}
void launch_step_state_init(const MemberDesc* d, int nmem, cudaStream_t st) {
  k_step_state_init<<<(nmem + 127) / 128, 128, 0, st>>>(d, nmem);
}

template <class T>
void launch_step_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                        const LaunchCfg& c, cudaStream_t st) {
  switch (kind) {
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
