// Kernels of one time step (Appendix B of arXiv:0710.5912), templated on the
// working precision T (float or double).  A step is six launches:
//
//   stage1       item 1 + item 2's advection at s = s^n: phi* = phi - dt J(psi, phi),
//                omega* = omega - dt J(psi, omega) (Eq. advective with the Eq. p1y
//                stencils), f = phi^3; phi*, omega* are kept in real space and
//                their row (x) transforms, with f's, go to x-spectral buffers.
//   colpass_phi  column (y) transforms of phi*, f and the Cahn-Hilliard update
//                of item 1 in the paper's increment form
//                  phi^{n+1} = phi* + (1 + D4/2)^-1 (-D2 phi* - D4 phi* + D2 f),
//                Nyquist modes of phi^{n+1} zeroed; the increment is transformed
//                back along y.
//   rowinv_phi   inverse row transform of the increment, phi^{n+1} = phi* + inc
//                (minus phi*'s Nyquist column); at a strain wrap the row-shift
//                remap is applied as a permutation of the writes.
//   stage2       mu = -a phi + b phi^3 - kappa lap_c phi and the body-force curl
//                F = d_x phi d_y mu - d_y phi d_x mu at s = s^{n+1} (Eq. G), g =
//                -F/rho (or -F/eta for Stokes), row transform.
//   colpass_flow column transforms; Crank-Nicolson vorticity update in increment
//                form omega^{n+1} = omega* + (1 - C/2)^-1 (C omega* + g) and the
//                Poisson solve psi = omega / k^2 (items 2-3), or the Stokes solve
//                psi = g / k^4; inverse column transforms.
//   rowinv_flow  inverse row transforms: psi, and omega^{n+1} = omega* + inc;
//                advances the step counter.
//
// Transforming only the increments keeps the FP32 rounding of every step
// proportional to the change of the field instead of to the field itself.
//
// Layout: real fields ny x nx row-major.  x-spectral buffers hold, for each row
// j, the modes m = 0..nx/2-1 of the row's real DFT (the Nyquist column is
// carried separately as one real per row), tiled in chunks of CL = 2^LC
// adjacent modes: element (j, m) sits at ((m >> LC) ny + j) CL + (m & (CL-1)),
// so a column pass reads whole chunks contiguously and a pair of rows writes
// 2 CL adjacent values.  The 1/(nx ny) of the inverse transforms is applied in
// the column passes.  Each launch covers a batch of members (blockIdx.y).
#include "shf_internal.cuh"

namespace shf {

template <class T>
__device__ __forceinline__ T ldf(const T* __restrict__ f, int i, int j, int mx, int my, int l2x) {
  return __ldg(f + (((j & my) << l2x) | (i & mx)));
}

// Sheared y-derivative of Eq. p1y: the vertical central difference blended
// (weight |s|/2) with the difference across the diagonal pair two cells away;
// d = -2 for s >= 0 (pair (i-2, j+1), (i+2, j-1)), d = +2 for s < 0.
template <class T>
__device__ __forceinline__ T dy_sheared(const T* __restrict__ f, int i, int j, int mx, int my, int l2x,
                                        T w0, T w1, int d, T inv2h) {
  const T vert = ldf(f, i, j + 1, mx, my, l2x) - ldf(f, i, j - 1, mx, my, l2x);
  const T diag = ldf(f, i + d, j + 1, mx, my, l2x) - ldf(f, i - d, j - 1, mx, my, l2x);
  return (w0 * vert + w1 * diag) * inv2h;
}

template <class T>
__device__ __forceinline__ T dx_central(const T* __restrict__ f, int i, int j, int mx, int my, int l2x,
                                        T inv2h) {
  return (ldf(f, i + 1, j, mx, my, l2x) - ldf(f, i - 1, j, mx, my, l2x)) * inv2h;
}

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

// Writes the half spectra of rows (j0, j0+1) split from Z = FFT(a + i b):
//   pair_of_rows = true : z0 holds (row j0, row j0+1) of one field -> dst
//   pair_of_rows = false: z0 holds (field1, field2) of row j0 and z1 of row j0+1
//                         -> field1 to dst, field2 to dst2
// Each thread writes whole chunks: 2 CL adjacent elements (rows j0 and j0+1).
template <int LC, class C>
__device__ __forceinline__ void write_pair_rows(const C* z0, const C* z1, bool pair_of_rows, C* dst, C* dst2,
                                                int j0, int nx, int ny, int t, int Tthreads) {
  constexpr int CL = 1 << LC;
  const int mx = nx - 1;
  const int nchunk = (nx >> 1) >> LC;
  for (int cb = t; cb < nchunk; cb += Tthreads) {
    C r0[CL], r1[CL], s0[CL], s1[CL];
#pragma unroll
    for (int c = 0; c < CL; ++c) {
      const int m = (cb << LC) + c;
      if (pair_of_rows) {
        split_pair(z0, m, mx, r0[c], r1[c]);
      } else {
        split_pair(z0, m, mx, r0[c], s0[c]);
        split_pair(z1, m, mx, r1[c], s1[c]);
      }
    }
    C* p = dst + ((((size_t)cb * ny) + j0) << LC);
#pragma unroll
    for (int c = 0; c < CL; ++c) {
      p[c] = r0[c];
      p[CL + c] = r1[c];
    }
    if (!pair_of_rows) {
      C* p2 = dst2 + ((((size_t)cb * ny) + j0) << LC);
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        p2[c] = s0[c];
        p2[CL + c] = s1[c];
      }
    }
  }
}

// Launch bounds: row kernels run 256 threads; the minimum CTAs per SM caps
// registers so that several CTAs (as many as shared memory allows) co-reside.
// Column kernels run up to 512 threads in float and 256 in double.
template <class T> constexpr int col_threads() { return sizeof(T) == 8 ? 256 : 512; }
template <class T> constexpr int min_ctas(int fp32, int fp64) { return sizeof(T) == 8 ? fp64 : fp32; }

template <class T> struct Layout;
template <> struct Layout<float> { static constexpr int LC = 1; };   // 2 complex floats = 16 B
template <> struct Layout<double> { static constexpr int LC = 0; };  // 1 complex double = 16 B

// ---- asynchronous global -> shared copies of single elements (cp.async)
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Tile of NF fields x R rows (r0 .. r0+R-1) x W columns (x0 .. x0+W-1), all
// indices periodic, element (f, r, x) at tile[(f R + r) W + x]; issued by the
// nthreads threads of one instance.
template <class T, int NF>
__device__ __forceinline__ void load_tile_async(T* tile, const T* const (&fld)[NF], int r0, int R, int x0, int W,
                                                int mx, int my, int l2x, int t, int nthreads) {
#pragma unroll
  for (int fi = 0; fi < NF; ++fi)
    for (int r = 0; r < R; ++r) {
      const T* row = fld[fi] + ((size_t)((r0 + r) & my) << l2x);
      T* dst = tile + (fi * R + r) * W;
      for (int x = t; x < W; x += nthreads) cp_async_elem(dst + x, row + ((x0 + x) & mx));
    }
}

// Sheared y-derivative (Eq. p1y) and central x-derivative on a tile row r,
// local column x (tile row pitch W).
template <class T>
__device__ __forceinline__ T tile_dy(const T* tl, int r, int x, int W, T w0, T w1, int d, T inv2h) {
  const T vert = tl[(r + 1) * W + x] - tl[(r - 1) * W + x];
  const T diag = tl[(r + 1) * W + x + d] - tl[(r - 1) * W + x - d];
  return (w0 * vert + w1 * diag) * inv2h;
}
template <class T>
__device__ __forceinline__ T tile_dx(const T* tl, int r, int x, int W, T inv2h) {
  return (tl[r * W + x + 1] - tl[r * W + x - 1]) * inv2h;
}

// Half spectra of one row from Z = FFT(a + i b) (a, b the row of two fields):
// field a -> dstA, field b -> dstB, whole chunks of CL modes per thread.
template <int LC, class C>
__device__ __forceinline__ void write_one_row(const C* z, C* dstA, C* dstB, int j, int nx, int ny, int t,
                                              int Tthreads) {
  constexpr int CL = 1 << LC;
  const int mx = nx - 1;
  const int nchunk = (nx >> 1) >> LC;
  for (int cb = t; cb < nchunk; cb += Tthreads) {
    C* pa = dstA + ((((size_t)cb * ny) + j) << LC);
    C* pb = dstB + ((((size_t)cb * ny) + j) << LC);
#pragma unroll
    for (int c = 0; c < CL; ++c) {
      C A, B;
      split_pair(z, (cb << LC) + c, mx, A, B);
      pa[c] = A;
      pb[c] = B;
    }
  }
}

// v[q] = Z[t + T q] from a padded buffer (the register layout of fft_reg)
template <class C>
__device__ __forceinline__ void smem_to_reg(C (&v)[16], const C* Z, int log2N, int t) {
  const int T = 1 << (log2N - 4);
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = Z[pad16(t + q * T)];
}

// ----------------------------------------------------------------- stage 1
// One instance = a pair of rows (j0, j1), Tf = nx/16 threads; register q of
// thread t is point i = Tf q + t, so each q is a chunk of Tf consecutive
// points whose stencil inputs (4 rows, Tf + 4 columns) are staged in shared
// memory by cp.async, one chunk ahead.  Three passes: row j0 (phi*, f), row j1
// (phi*, f), rows j0 and j1 of omega* (inertial members only).
template <class T>
__global__ void __launch_bounds__(256, min_ctas<T>(2, 1)) k_stage1(const MemberDesc* __restrict__ descs, int log2nx,
                                                                    int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1;
  const int Tf = nx >> 4;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int j0 = 2 * (blockIdx.x * (blockDim.x / Tf) + inst), j1 = j0 + 1;
  const int W = Tf + 4;
  unsigned char* base = smem_raw + (size_t)inst * stage1_inst_bytes(nx, sizeof(T));
  C* Z = reinterpret_cast<C*>(base);
  T* tiles = reinterpret_cast<T*>(base + (size_t)padded_len(nx) * sizeof(C));
  const int tsz = 2 * 4 * W;

  const long long n = *D.n;
  double s_d, s1_d;
  long long K0, K1;
  strain_dev(n, D.gdot, D.dt, D.ratio, s_d, K0);
  strain_dev(n + 1, D.gdot, D.dt, D.ratio, s1_d, K1);
  const T s = (T)s_d;
  const T w1 = (s < T(0) ? -s : s) * T(0.5);
  const T w0 = T(1) - w1;
  const int d = s >= T(0) ? -2 : 2;
  const T dt = (T)D.dt, inv2h = (T)D.inv_2h;
  const bool stokes = D.stokes != 0;
  const bool wrap = D.remap && (K1 != K0);
  const T* __restrict__ phi = static_cast<const T*>(D.phi);
  const T* __restrict__ psi = static_cast<const T*>(D.psi);
  const T* __restrict__ om = static_cast<const T*>(D.omega);
  T* phis = static_cast<T*>(D.phi_star);
  T* oms = static_cast<T*>(D.omega_star);
  const int npass = stokes ? 2 : 3;

  C v[16];
#pragma unroll 1
  for (int pass = 0; pass < npass; ++pass) {
    const bool wpass = pass == 2;
    if (wpass && wrap) {
      // omega* at a wrap: evaluated at the source of every remapped position,
      // gathered through Z (a rolled loop: this path runs once per wrap)
      const int sh0 = remap_shift(K1 - K0, D.ratio, j0, nx);
      const int sh1 = remap_shift(K1 - K0, D.ratio, j1, nx);
#pragma unroll 1
      for (int p = t; p < nx; p += Tf) {
        T ws[2];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int j = j0 + jj;
          const int i = (p - (jj ? sh1 : sh0)) & mx;
          const T dxpsi = dx_central(psi, i, j, mx, my, log2nx, inv2h);
          const T dypsi = dy_sheared(psi, i, j, mx, my, log2nx, w0, w1, d, inv2h);
          const T dxw = dx_central(om, i, j, mx, my, log2nx, inv2h);
          const T dyw = dy_sheared(om, i, j, mx, my, log2nx, w0, w1, d, inv2h);
          ws[jj] = ldf(om, i, j, mx, my, log2nx) - dt * (dypsi * dxw - dxpsi * dyw);
          oms[((size_t)j << log2nx) + p] = ws[jj];
        }
        Z[pad16(p)] = C{ws[0], ws[1]};
      }
      __syncthreads();
      smem_to_reg(v, Z, log2nx, t);
      __syncthreads();
    } else {
      const T* fld[2] = {wpass ? psi : phi, wpass ? om : psi};
      load_tile_async<T, 2>(tiles, fld, j0 - 1, 4, -2, W, mx, my, log2nx, t, Tf);
      cp_async_commit();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (q + 1 < 16) {
          load_tile_async<T, 2>(tiles + ((q + 1) & 1) * tsz, fld, j0 - 1, 4, Tf * (q + 1) - 2, W, mx, my, log2nx,
                                t, Tf);
          cp_async_commit();
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();
        const T* ta = tiles + (q & 1) * tsz;        // field 0: phi (or psi)
        const T* tb = ta + 4 * W;                   // field 1: psi (or omega)
        const int x = t + 2;
        const int i = Tf * q + t;
        if (!wpass) {
          const int r = pass + 1;                   // tile row of j0 or j1
          const T pc = ta[r * W + x];
          const T dxphi = tile_dx(ta, r, x, W, inv2h);
          const T dyphi = tile_dy(ta, r, x, W, w0, w1, d, inv2h);
          const T dxpsi = tile_dx(tb, r, x, W, inv2h);
          const T dypsi = tile_dy(tb, r, x, W, w0, w1, d, inv2h);
          const T phistar = pc - dt * (dypsi * dxphi - dxpsi * dyphi);
          phis[((size_t)(j0 + pass) << log2nx) + i] = phistar;
          v[q] = C{phistar, (pc * pc) * pc};
        } else {
          T ws[2];
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int r = jj + 1;
            const T dxpsi = tile_dx(ta, r, x, W, inv2h);
            const T dypsi = tile_dy(ta, r, x, W, w0, w1, d, inv2h);
            const T dxw = tile_dx(tb, r, x, W, inv2h);
            const T dyw = tile_dy(tb, r, x, W, w0, w1, d, inv2h);
            ws[jj] = tb[r * W + x] - dt * (dypsi * dxw - dxpsi * dyw);
            oms[((size_t)(j0 + jj) << log2nx) + i] = ws[jj];
          }
          v[q] = C{ws[0], ws[1]};
        }
        __syncthreads();                            // tile (q & 1) may now be refilled
      }
    }
    fft_reg<false>(v, log2nx, t, Z, tw);
    reg_to_smem(v, log2nx, t, Z);
    if (!wpass) {
      write_one_row<LC>(Z, static_cast<C*>(D.xs_phi), static_cast<C*>(D.xs_f), j0 + pass, nx, ny, t, Tf);
      if (t == 0) static_cast<T*>(D.nyq_phi)[j0 + pass] = Z[pad16(nx >> 1)].x;   // phi*'s row Nyquist
    } else {
      write_pair_rows<LC>(Z, Z, true, static_cast<C*>(D.xs_w), static_cast<C*>(nullptr), j0, nx, ny, t, Tf);
      if (t == 0) {
        const C zn = Z[pad16(nx >> 1)];
        static_cast<T*>(D.nyq_omega)[j0] = zn.x;
        static_cast<T*>(D.nyq_omega)[j1] = zn.y;
      }
    }
    __syncthreads();                                // Z is reused by the next pass
  }
}

// ------------------------------------------------------------ column passes
// CTA: NC = 2^log2nc adjacent columns m0..m0+NC-1 (NC a multiple of the chunk
// width); thread (c, t) with c = threadIdx.x mod NC handles column m0 + c,
// points n = t + Tc q.  Loads and stores are contiguous across the warp.
template <class T>
__global__ void __launch_bounds__(col_threads<T>()) k_colpass_phi(const MemberDesc* __restrict__ descs, int log2nx,
                                                      int log2ny, int log2nc, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int ny = 1 << log2ny;
  const int Tc = ny >> 4;
  const int c = threadIdx.x & ((1 << log2nc) - 1), t = threadIdx.x >> log2nc;
  const int m = (blockIdx.x << log2nc) + c;
  C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)c * padded_len(ny);
  C* xp = static_cast<C*>(D.xs_phi);
  const C* xf = static_cast<const C*>(D.xs_f);
  C vp[16], vf[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const size_t g = xs_idx(t + q * Tc, m, ny, LC);
    vp[q] = xp[g];
    vf[q] = xf[g];
  }
  fft_reg<false>(vp, log2ny, t, buf, tw);
  fft_reg<false>(vf, log2ny, t, buf, tw);
  double s_d;
  long long K;
  strain_dev(*D.n, D.gdot, D.dt, D.ratio, s_d, K);       // stage 1 uses s^n
  const double qx_d = m * D.qx_unit;
  const T qx = (T)qx_d;
  const T sqx = (T)(s_d * qx_d);                          // s q_x formed in double
  const T caM = (T)D.c_dt_aM, cbM = (T)D.c_dt_bM, ckM = (T)D.c_hdt_kM;
  const T norm = (T)D.inv_nxny, qyu = (T)D.qy_unit;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int nn = t + q * Tc;
    C inc;
    if (nn == (ny >> 1)) {
      inc = C{-vp[q].x * norm, -vp[q].y * norm};          // Nyquist row of phi^{n+1} -> 0
    } else {
      const int ns = nn < (ny >> 1) ? nn : nn - ny;
      const T ky = (T)ns * qyu - sqx;
      const T k2 = qx * qx + ky * ky;
      const T c4 = ckM * (k2 * k2);
      const T a = caM * k2 - T(2) * c4;
      const T b = cbM * k2;
      const T inv = norm / (T(1) + c4);
      inc = C{(a * vp[q].x - b * vf[q].x) * inv, (a * vp[q].y - b * vf[q].y) * inv};
    }
    vp[q] = inc;
  }
  fft_reg<true>(vp, log2ny, t, buf, tw);
#pragma unroll
  for (int q = 0; q < 16; ++q) xp[xs_idx(t + q * Tc, m, ny, LC)] = vp[q];
}

template <class T>
__global__ void __launch_bounds__(col_threads<T>()) k_colpass_flow(const MemberDesc* __restrict__ descs, int log2nx,
                                                       int log2ny, int log2nc, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int ny = 1 << log2ny;
  const int Tc = ny >> 4;
  const int c = threadIdx.x & ((1 << log2nc) - 1), t = threadIdx.x >> log2nc;
  const int m = (blockIdx.x << log2nc) + c;
  C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)c * padded_len(ny);
  C* xg = static_cast<C*>(D.xs_g);
  C* xw = static_cast<C*>(D.xs_w);
  const bool stokes = D.stokes != 0;
  C vg[16], vw[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) vg[q] = xg[xs_idx(t + q * Tc, m, ny, LC)];
  if (!stokes) {
#pragma unroll
    for (int q = 0; q < 16; ++q) vw[q] = xw[xs_idx(t + q * Tc, m, ny, LC)];
  }
  fft_reg<false>(vg, log2ny, t, buf, tw);
  if (!stokes) fft_reg<false>(vw, log2ny, t, buf, tw);
  double s_d;
  long long K;
  strain_dev(*D.n + 1, D.gdot, D.dt, D.ratio, s_d, K);   // stages 2-3 use s^{n+1}
  const double qx_d = m * D.qx_unit;
  const T qx = (T)qx_d;
  const T sqx = (T)(s_d * qx_d);
  const T norm = (T)D.inv_nxny, qyu = (T)D.qy_unit;
  const T cnu = (T)D.c_hdt_nu, dt = (T)D.dt;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int nn = t + q * Tc;
    const bool zero = (nn == (ny >> 1)) || (m == 0 && nn == 0);
    const int ns = nn < (ny >> 1) ? nn : nn - ny;
    const T ky = (T)ns * qyu - sqx;
    const T k2 = qx * qx + ky * ky;
    const C G = vg[q];
    if (stokes) {
      const T inv = zero ? T(0) : norm / (k2 * k2);
      vg[q] = C{G.x * inv, G.y * inv};
    } else {
      const C W = vw[q];
      C inc, ps;
      if (zero) {
        inc = C{-W.x * norm, -W.y * norm};                 // omega^{n+1} -> 0 there
        ps = C{T(0), T(0)};
      } else {
        const T cc = cnu * k2;
        const T inv = T(1) / (T(1) + cc);
        const C dw = C{(-T(2) * cc * W.x + dt * G.x) * inv, (-T(2) * cc * W.y + dt * G.y) * inv};
        const T ik = norm / k2;
        ps = C{(W.x + dw.x) * ik, (W.y + dw.y) * ik};
        inc = C{dw.x * norm, dw.y * norm};
      }
      vg[q] = ps;
      vw[q] = inc;
    }
  }
  fft_reg<true>(vg, log2ny, t, buf, tw);
#pragma unroll
  for (int q = 0; q < 16; ++q) xg[xs_idx(t + q * Tc, m, ny, LC)] = vg[q];
  if (!stokes) {
    fft_reg<true>(vw, log2ny, t, buf, tw);
#pragma unroll
    for (int q = 0; q < 16; ++q) xw[xs_idx(t + q * Tc, m, ny, LC)] = vw[q];
  }
}

// ----------------------------------------------------------- inverse rows
// Z for the inverse row transform of rows (j0, j0+1) of one x-spectral field:
// Z[k] = A[k] + i B[k] (0 < k < N/2), Z[0] = Re A[0] + i Re B[0], Z[N/2] = zn,
// Z[N-k] = conj A[k] + i conj B[k] (A = row j0, B = row j0+1).  Each thread
// loads whole 32-byte chunks (both rows of CL modes) and scatters them into the
// padded buffer; a barrier follows.
template <int LC, class C>
__device__ __forceinline__ void load_pair_rows_to_smem(C* Z, const C* __restrict__ xs, int j0, C zn, int nx,
                                                       int ny, int t, int Tthreads) {
  constexpr int CL = 1 << LC;
  const int nchunk = (nx >> 1) >> LC;
  for (int cb = t; cb < nchunk; cb += Tthreads) {
    const float4* p4 = reinterpret_cast<const float4*>(xs + ((((size_t)cb * ny) + j0) << LC));
    union { float4 f4[2]; C c[2 * CL]; } u;
    u.f4[0] = __ldg(p4);
    u.f4[1] = __ldg(p4 + 1);
#pragma unroll
    for (int c = 0; c < CL; ++c) {
      const int k = (cb << LC) + c;
      const C A = u.c[c], B = u.c[CL + c];
      if (k == 0) {
        Z[pad16(0)] = C{A.x, B.x};
        Z[pad16(nx >> 1)] = zn;
      } else {
        Z[pad16(k)] = C{A.x - B.y, A.y + B.x};
        Z[pad16(nx - k)] = C{A.x + B.y, B.x - A.y};
      }
    }
  }
  __syncthreads();
}

// Chunks of a row pair held in registers between their load and their scatter
// into Z: thread t holds chunks cb = t + Tf u, u < NCH, each 32 bytes (rows
// j0 and j0+1 of CL modes).
template <class C, int LC>
struct PairChunks {
  static constexpr int NCH = 8 >> LC;               // (nx/2 / CL) / (nx/16)
  float4 f4[NCH][2];
  __device__ __forceinline__ void load(const C* __restrict__ xs, int j0, int ny, int t, int Tf) {
#pragma unroll
    for (int u = 0; u < NCH; ++u) {
      const int cb = t + u * Tf;
      const float4* p4 = reinterpret_cast<const float4*>(xs + ((((size_t)cb * ny) + j0) << LC));
      f4[u][0] = __ldg(p4);
      f4[u][1] = __ldg(p4 + 1);
    }
  }
  // Z[k] = A[k] + i B[k], Z[N-k] = conj A[k] + i conj B[k], Z[0] real parts,
  // Z[N/2] = zn; followed by a barrier
  __device__ __forceinline__ void scatter(C* Z, C zn, int nx, int t, int Tf) const {
    constexpr int CL = 1 << LC;
#pragma unroll
    for (int u = 0; u < NCH; ++u) {
      union { float4 f[2]; C c[2 * CL]; } w;
      w.f[0] = f4[u][0];
      w.f[1] = f4[u][1];
      const int cb = t + u * Tf;
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        const int k = (cb << LC) + c;
        const C A = w.c[c], B = w.c[CL + c];
        if (k == 0) {
          Z[pad16(0)] = C{A.x, B.x};
          Z[pad16(nx >> 1)] = zn;
        } else {
          Z[pad16(k)] = C{A.x - B.y, A.y + B.x};
          Z[pad16(nx - k)] = C{A.x + B.y, B.x - A.y};
        }
      }
    }
    __syncthreads();
  }
};

// phi^{n+1} rows (j0, j1) = phi* + increment - phi*'s row Nyquist component,
// written at the remapped positions when the strain wraps during this step.
// Persistent: each instance walks row pairs with a stride of all instances of
// the grid and loads the next pair's spectrum while transforming the current.
template <class T>
__global__ void __launch_bounds__(256, min_ctas<T>(2, 1)) k_rowinv_phi(const MemberDesc* __restrict__ descs,
                                                                        int log2nx, int log2ny,
                                                                        const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1;
  const int Tf = nx >> 4;
  const int ipc = blockDim.x / Tf;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int npairs = ny >> 1;
  const int stride = gridDim.x * ipc;
  C* Z = reinterpret_cast<C*>(smem_raw) + (size_t)inst * padded_len(nx);
  long long dK = 0;
  if (D.remap) {
    double s0, s1;
    long long K0, K1;
    const long long n = *D.n;
    strain_dev(n, D.gdot, D.dt, D.ratio, s0, K0);
    strain_dev(n + 1, D.gdot, D.dt, D.ratio, s1, K1);
    dK = K1 - K0;
  }
  const T* nq = static_cast<const T*>(D.nyq_phi);
  const T rn = T(1) / T(nx);
  const C* xp = static_cast<const C*>(D.xs_phi);
  const T* phis = static_cast<const T*>(D.phi_star);
  T* phi = static_cast<T*>(D.phi);
  // every instance of the CTA runs the same number of iterations (barriers)
  const int iters = (npairs - (int)blockIdx.x * ipc + stride - 1) / stride;
  int pair = blockIdx.x * ipc + inst;
  PairChunks<C, LC> ch;
  if (pair < npairs) ch.load(xp, 2 * pair, ny, t, Tf);
  for (int it = 0; it < iters; ++it) {
    const bool active = pair < npairs;
    const int j0 = 2 * pair, j1 = j0 + 1;
    C zn = C{T(0), T(0)};
    if (active) zn = C{-nq[j0] * rn, -nq[j1] * rn};
    if (active) ch.scatter(Z, zn, nx, t, Tf);
    else __syncthreads();
    C v[16];
    smem_to_reg(v, Z, log2nx, t);
    __syncthreads();                                // Z becomes the exchange buffer
    const int next = pair + stride;
    if (next < npairs) ch.load(xp, 2 * next, ny, t, Tf);   // in flight during the FFT
    T ps0[16], ps1[16];
    if (active) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = t + q * Tf;
        ps0[q] = phis[((size_t)j0 << log2nx) + i];
        ps1[q] = phis[((size_t)j1 << log2nx) + i];
      }
    }
    fft_reg<true>(v, log2nx, t, Z, tw);
    if (active) {
      const int sh0 = dK ? remap_shift(dK, D.ratio, j0, nx) : 0;
      const int sh1 = dK ? remap_shift(dK, D.ratio, j1, nx) : 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = t + q * Tf;
        phi[((size_t)j0 << log2nx) + ((i + sh0) & mx)] = ps0[q] + v[q].x;
        phi[((size_t)j1 << log2nx) + ((i + sh1) & mx)] = ps1[q] + v[q].y;
      }
    }
    __syncthreads();                                // last exchange reads done before the next scatter
    pair = next;
  }
}

// psi rows (j0, j1) from psi_hat; for inertial members also omega^{n+1} =
// omega* + increment - omega*'s row Nyquist component.  Advances n.
template <class T>
__global__ void __launch_bounds__(256, min_ctas<T>(2, 1)) k_rowinv_flow(const MemberDesc* __restrict__ descs,
                                                                         int log2nx, int log2ny,
                                                                         const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny;
  const int Tf = nx >> 4;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int j0 = 2 * (blockIdx.x * (blockDim.x / Tf) + inst), j1 = j0 + 1;
  C* Z = reinterpret_cast<C*>(smem_raw) + (size_t)inst * padded_len(nx);
  T* psi = static_cast<T*>(D.psi);
  C v[16];
  load_pair_rows_to_smem<LC>(Z, static_cast<const C*>(D.xs_g), j0, C{T(0), T(0)}, nx, ny, t, Tf);
  smem_to_reg(v, Z, log2nx, t);
  __syncthreads();
  fft_reg<true>(v, log2nx, t, Z, tw);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int i = t + q * Tf;
    psi[((size_t)j0 << log2nx) + i] = v[q].x;
    psi[((size_t)j1 << log2nx) + i] = v[q].y;
  }
  if (!D.stokes) {
    __syncthreads();                                // last exchange reads of Z are done
    const T* nq = static_cast<const T*>(D.nyq_omega);
    const T rn = T(1) / T(nx);
    load_pair_rows_to_smem<LC>(Z, static_cast<const C*>(D.xs_w), j0, C{-nq[j0] * rn, -nq[j1] * rn}, nx, ny, t,
                               Tf);
    smem_to_reg(v, Z, log2nx, t);
    __syncthreads();
    fft_reg<true>(v, log2nx, t, Z, tw);
    const T* oms = static_cast<const T*>(D.omega_star);
    T* om = static_cast<T*>(D.omega);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = t + q * Tf;
      om[((size_t)j0 << log2nx) + i] = oms[((size_t)j0 << log2nx) + i] + v[q].x;
      om[((size_t)j1 << log2nx) + i] = oms[((size_t)j1 << log2nx) + i] + v[q].y;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *D.n += 1;
}

// ----------------------------------------------------------------- stage 2
// One instance = rows (j0, j1); per chunk q of Tf points the phi tile (6 rows
// j0-2..j1+2, Tf + 6 columns) is staged by cp.async one chunk ahead, mu is
// computed on 4 rows x (Tf + 4) columns into shared memory, then g for both
// rows.  One FFT of (g_j0 + i g_j1).
template <class T>
__global__ void __launch_bounds__(256, min_ctas<T>(3, 1)) k_stage2(const MemberDesc* __restrict__ descs, int log2nx,
                                                                    int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int LC = Layout<T>::LC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1;
  const int Tf = nx >> 4;
  const int inst = threadIdx.x / Tf, t = threadIdx.x - inst * Tf;
  const int j0 = 2 * (blockIdx.x * (blockDim.x / Tf) + inst);
  const int W = Tf + 4, W2 = Tf + 6;
  unsigned char* base = smem_raw + (size_t)inst * stage2_inst_bytes(nx, sizeof(T));
  C* Z = reinterpret_cast<C*>(base);
  T* ptile = reinterpret_cast<T*>(base + (size_t)padded_len(nx) * sizeof(C));   // 2 x 6 x W2
  T* mt = ptile + 2 * 6 * W2;                                                   // 4 x W

  double s_d;
  long long K;
  strain_dev(*D.n + 1, D.gdot, D.dt, D.ratio, s_d, K);   // s^{n+1}
  const T s = (T)s_d;
  const T w1 = (s < T(0) ? -s : s) * T(0.5);
  const T w0 = T(1) - w1;
  const int d = s >= T(0) ? -2 : 2;
  const T a = (T)D.a, b = (T)D.b, kappa = (T)D.kappa;
  const T inv2h = (T)D.inv_2h, ih2 = (T)D.inv_h2, i4h2 = (T)D.inv_4h2;
  const T cxx = T(1) + s * s, cxy = T(2) * s;
  const T cf = (T)D.c_force;
  const T* fld[1] = {static_cast<const T*>(D.phi)};

  C v[16];
  load_tile_async<T, 1>(ptile, fld, j0 - 2, 6, -3, W2, mx, my, log2nx, t, Tf);
  cp_async_commit();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (q + 1 < 16) {
      load_tile_async<T, 1>(ptile + ((q + 1) & 1) * 6 * W2, fld, j0 - 2, 6, Tf * (q + 1) - 3, W2, mx, my, log2nx, t,
                            Tf);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* pt = ptile + (q & 1) * 6 * W2;
    // mu (Appendix B item 2) on tile rows 1..4 (j0-1..j1+1), columns 1..W2-2
    for (int r = 0; r < 4; ++r) {
      for (int x = t; x < W; x += Tf) {
        const int pr = r + 1, px = x + 1;
        const T pc = pt[pr * W2 + px];
        const T dxx = (pt[pr * W2 + px + 1] - T(2) * pc + pt[pr * W2 + px - 1]) * ih2;
        const T dyy = (pt[(pr + 1) * W2 + px] - T(2) * pc + pt[(pr - 1) * W2 + px]) * ih2;
        const T dxy = (pt[(pr + 1) * W2 + px + 1] - pt[(pr - 1) * W2 + px + 1] - pt[(pr + 1) * W2 + px - 1] +
                       pt[(pr - 1) * W2 + px - 1]) * i4h2;
        const T lap = cxx * dxx - cxy * dxy + dyy;
        mt[r * W + x] = -a * pc + b * ((pc * pc) * pc) - kappa * lap;
      }
    }
    __syncthreads();
    T g[2];
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int rp = jj + 2, rm = jj + 1;           // phi tile row, mu tile row of j0 + jj
      const int xp = t + 3, xm = t + 2;
      const T dxphi = tile_dx(pt, rp, xp, W2, inv2h);
      const T dyphi = tile_dy(pt, rp, xp, W2, w0, w1, d, inv2h);
      const T dxmu = tile_dx(mt, rm, xm, W, inv2h);
      const T dymu = tile_dy(mt, rm, xm, W, w0, w1, d, inv2h);
      g[jj] = cf * (dxphi * dymu - dyphi * dxmu);
    }
    v[q] = C{g[0], g[1]};
    __syncthreads();                                // tiles may now be refilled
  }
  fft_reg<false>(v, log2nx, t, Z, tw);
  reg_to_smem(v, log2nx, t, Z);
  write_pair_rows<LC>(Z, Z, true, static_cast<C*>(D.xs_g), static_cast<C*>(nullptr), j0, nx, ny, t, Tf);
}

// ----------------------------------------------------------------- launchers
template <class T>
void launch_stage1(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw, const RowCfg& c,
                   cudaStream_t st) {
  k_stage1<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
}
template <class T>
void launch_colpass_phi(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                        const ColCfg& c, cudaStream_t st) {
  k_colpass_phi<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, c.log2cols, tw);
}
template <class T>
void launch_rowinv(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw, const RowCfg& c,
                   int mode, cudaStream_t st) {
  if (mode == 0) k_rowinv_phi<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
  else k_rowinv_flow<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
}
template <class T>
void launch_stage2(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw, const RowCfg& c,
                   cudaStream_t st) {
  k_stage2<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
}
template <class T>
void launch_colpass_flow(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                         const ColCfg& c, cudaStream_t st) {
  k_colpass_flow<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, c.log2cols, tw);
}

template <class T>
void set_step_smem_limits() {
  const int lim = 220 * 1024;   // dynamic part; leaves room for static shared memory
  cudaFuncSetAttribute(k_stage1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_colpass_phi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_colpass_flow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_rowinv_phi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_rowinv_flow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_stage2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

#define SHF_INST(T)                                                                                       \
  template void launch_stage1<T>(const MemberDesc*, int, int, int, const cplx<T>*, const RowCfg&,          \
                                 cudaStream_t);                                                            \
  template void launch_colpass_phi<T>(const MemberDesc*, int, int, int, const cplx<T>*, const ColCfg&,     \
                                      cudaStream_t);                                                       \
  template void launch_rowinv<T>(const MemberDesc*, int, int, int, const cplx<T>*, const RowCfg&, int,     \
                                 cudaStream_t);                                                            \
  template void launch_stage2<T>(const MemberDesc*, int, int, int, const cplx<T>*, const RowCfg&,          \
                                 cudaStream_t);                                                            \
  template void launch_colpass_flow<T>(const MemberDesc*, int, int, int, const cplx<T>*, const ColCfg&,    \
                                       cudaStream_t);                                                      \
  template void set_step_smem_limits<T>();

SHF_INST(float)
SHF_INST(double)

}  // namespace shf
