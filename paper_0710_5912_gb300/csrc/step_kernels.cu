// Kernels of one time step (Appendix B of arXiv:0710.5912), templated on the
// working precision T (float or double).  A step is six launches:
//
//   stage1      item 1 + item 2's advection: phi* = phi - dt J_s(psi, phi),
//               omega* = omega - dt J_s(psi, omega), f = phi^3 (Eq. advective,
//               Eq. p1y stencils, s = s^n), then the row (x) transforms of
//               phi*, f, omega* -> x-spectral buffers.
//   colpass_phi column (y) transforms of phi*, f, the per-mode Cahn-Hilliard
//               update (explicit Euler on lap_c, Crank-Nicolson on lap_c^2),
//               Nyquist modes zeroed, inverse column transform.
//   rowinv(0)   inverse row transform -> real phi^{n+1}; at a strain wrap the
//               row-shift remap is applied as a permutation of the writes.
//   stage2      mu = -a phi + b phi^3 - kappa lap_c phi and the body-force
//               curl F = d_x phi d_y mu - d_y phi d_x mu at s = s^{n+1}
//               (Eq. G), g = -F/rho (or -F/eta for Stokes), row transform.
//   colpass_flow column transforms; Crank-Nicolson vorticity update and the
//               Poisson solve psi = omega / k^2 (items 2-3), or the Stokes
//               biharmonic solve psi = g / k^4; inverse column transforms.
//   rowinv(1)   inverse row transforms -> real psi, omega; advances n.
//
// Layout: real fields ny x nx row-major; x-spectral buffers ny x (nx/2)
// complex row-major (modes m = 0..nx/2-1; the Nyquist column is dropped).
// The 1/(nx ny) normalisation of the inverse transform is applied in the
// column passes.  Each launch covers a batch of members (blockIdx.y).
#include "shf_internal.cuh"

namespace shf {

// Column passes run up to 1024 threads in float (64 registers each) and up to
// 512 in double, where a complex value needs twice the registers.
template <class T>
constexpr int col_max_threads() { return sizeof(T) == 8 ? 512 : 1024; }

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

// Split Z = FFT(a + i b) of two real rows into the half spectra of a and b:
// A[k] = (Z[k] + conj Z[N-k]) / 2, B[k] = (Z[k] - conj Z[N-k]) / (2i).
template <class C>
__device__ __forceinline__ void split_real_pair(const C* z, int k, int mx, C& A, C& B) {
  using T = decltype(z[0].x);
  const C zk = z[k];
  const C zc = cconj(z[(-k) & mx]);
  A = C{(zk.x + zc.x) * T(0.5), (zk.y + zc.y) * T(0.5)};
  B = C{(zk.y - zc.y) * T(0.5), -(zk.x - zc.x) * T(0.5)};
}

// ----------------------------------------------------------------- stage 1
template <class T>
__global__ void __launch_bounds__(512) k_stage1(const MemberDesc* __restrict__ descs, int log2nx,
                                                 int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1, half = nx >> 1;
  const int Tf = nx >> 3;
  const int inst = threadIdx.x / Tf, tid = threadIdx.x - inst * Tf;
  const int ipc = blockDim.x / Tf;
  const int pair = blockIdx.x * ipc + inst;
  const int j0 = 2 * pair;
  C* bufA = reinterpret_cast<C*>(smem_raw) + (size_t)inst * 3 * nx;
  C* bufB = bufA + nx;
  C* bufC = bufB + nx;

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

#pragma unroll 1
  for (int jj = 0; jj < 2; ++jj) {
    const int j = j0 + jj;
    C* bz = jj ? bufB : bufA;
    const int sh = wrap ? remap_shift(K1 - K0, D.ratio, j, nx) : 0;
#pragma unroll 2
    for (int q = 0; q < 8; ++q) {
      const int i = tid + q * Tf;
      const T pc = ldf(phi, i, j, mx, my, log2nx);
      const T dxpsi = dx_central(psi, i, j, mx, my, log2nx, inv2h);
      const T dypsi = dy_sheared(psi, i, j, mx, my, log2nx, w0, w1, d, inv2h);
      const T dxphi = dx_central(phi, i, j, mx, my, log2nx, inv2h);
      const T dyphi = dy_sheared(phi, i, j, mx, my, log2nx, w0, w1, d, inv2h);
      const T phistar = pc - dt * (dypsi * dxphi - dxpsi * dyphi);
      bz[i] = C{phistar, (pc * pc) * pc};
      if (!stokes) {
        const T dxw = dx_central(om, i, j, mx, my, log2nx, inv2h);
        const T dyw = dy_sheared(om, i, j, mx, my, log2nx, w0, w1, d, inv2h);
        const T wstar = ldf(om, i, j, mx, my, log2nx) - dt * (dypsi * dxw - dxpsi * dyw);
        const int ii = (i + sh) & mx;
        if (jj == 0) bufC[ii].x = wstar;
        else bufC[ii].y = wstar;
      }
    }
  }
  if (stokes) {
    C* const b2[2] = {bufA, bufB};
    fft_smem<false, 2>(b2, log2nx, tid, tw);
  } else {
    C* const b3[3] = {bufA, bufB, bufC};
    fft_smem<false, 3>(b3, log2nx, tid, tw);
  }
  C* xp = static_cast<C*>(D.xs_phi) + (size_t)j0 * half;
  C* xf = static_cast<C*>(D.xs_f) + (size_t)j0 * half;
  C* xw = static_cast<C*>(D.xs_w) + (size_t)j0 * half;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = tid + q * Tf;
    C A, B;
    split_real_pair(bufA, k, mx, A, B);
    xp[k] = A;
    xf[k] = B;
    split_real_pair(bufB, k, mx, A, B);
    xp[half + k] = A;
    xf[half + k] = B;
    if (!stokes) {
      split_real_pair(bufC, k, mx, A, B);
      xw[k] = A;
      xw[half + k] = B;
    }
  }
}

// ------------------------------------------------------------ column passes
// Coalesced transfer of C adjacent columns (all ny rows) between an x-spectral
// buffer and shared memory laid out column-major [c][n].
template <class C>
__device__ __forceinline__ void load_cols(C* sm, const C* __restrict__ g, int m0, int ncol, int log2ncol,
                                          int ny, int half) {
  for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
    const int c = e & (ncol - 1), n = e >> log2ncol;
    sm[c * ny + n] = g[(size_t)n * half + m0 + c];
  }
}
template <class C>
__device__ __forceinline__ void store_cols(const C* sm, C* __restrict__ g, int m0, int ncol, int log2ncol,
                                           int ny, int half) {
  for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
    const int c = e & (ncol - 1), n = e >> log2ncol;
    g[(size_t)n * half + m0 + c] = sm[c * ny + n];
  }
}

template <class T>
__global__ void __launch_bounds__(col_max_threads<T>()) k_colpass_phi(const MemberDesc* __restrict__ descs, int log2nx,
                                                      int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, half = nx >> 1;
  const int Tc = ny >> 3;
  const int col = threadIdx.x / Tc, tid = threadIdx.x - col * Tc;
  const int ncol = blockDim.x / Tc;
  const int log2ncol = 31 - __clz(ncol);
  const int m0 = blockIdx.x * ncol;
  C* sm = reinterpret_cast<C*>(smem_raw);
  load_cols(sm, static_cast<const C*>(D.xs_phi), m0, ncol, log2ncol, ny, half);
  load_cols(sm + ncol * ny, static_cast<const C*>(D.xs_f), m0, ncol, log2ncol, ny, half);
  C* bufP = sm + col * ny;
  C* bufF = sm + (ncol + col) * ny;
  {
    C* const b2[2] = {bufP, bufF};
    fft_smem<false, 2>(b2, log2ny, tid, tw);
  }
  double s_d;
  long long K;
  strain_dev(*D.n, D.gdot, D.dt, D.ratio, s_d, K);       // stage 1 uses s^n
  const int m = m0 + col;
  const double qx_d = m * D.qx_unit;
  const T qx = (T)qx_d;
  const T sqx = (T)(s_d * qx_d);                          // s q_x formed in double
  const T caM = (T)D.c_dt_aM, cbM = (T)D.c_dt_bM, ckM = (T)D.c_hdt_kM;
  const T norm = (T)D.inv_nxny, qyu = (T)D.qy_unit;
#pragma unroll 2
  for (int q = 0; q < 8; ++q) {
    const int nn = tid + q * Tc;
    C out = C{T(0), T(0)};
    if (nn != (ny >> 1)) {
      const int ns = nn < (ny >> 1) ? nn : nn - ny;
      const T ky = (T)ns * qyu - sqx;
      const T k2 = qx * qx + ky * ky;
      const T k4 = k2 * k2;
      const T A = T(1) + caM * k2 - ckM * k4;
      const T B = cbM * k2;
      const T inv = norm / (T(1) + ckM * k4);
      const C P = bufP[nn], F = bufF[nn];
      out = C{(A * P.x - B * F.x) * inv, (A * P.y - B * F.y) * inv};
    }
    bufP[nn] = out;
  }
  {
    C* const b1[1] = {bufP};
    fft_smem<true, 1>(b1, log2ny, tid, tw);
  }
  store_cols(sm, static_cast<C*>(D.xs_phi), m0, ncol, log2ncol, ny, half);
}

template <class T>
__global__ void __launch_bounds__(col_max_threads<T>()) k_colpass_flow(const MemberDesc* __restrict__ descs, int log2nx,
                                                       int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, half = nx >> 1;
  const int Tc = ny >> 3;
  const int col = threadIdx.x / Tc, tid = threadIdx.x - col * Tc;
  const int ncol = blockDim.x / Tc;
  const int log2ncol = 31 - __clz(ncol);
  const int m0 = blockIdx.x * ncol;
  const bool stokes = D.stokes != 0;
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* bufG = sm + col * ny;
  C* bufW = sm + (ncol + col) * ny;
  load_cols(sm, static_cast<const C*>(D.xs_g), m0, ncol, log2ncol, ny, half);
  if (!stokes) {
    load_cols(sm + ncol * ny, static_cast<const C*>(D.xs_w), m0, ncol, log2ncol, ny, half);
    C* const b2[2] = {bufG, bufW};
    fft_smem<false, 2>(b2, log2ny, tid, tw);
  } else {
    C* const b1[1] = {bufG};
    fft_smem<false, 1>(b1, log2ny, tid, tw);
  }
  double s_d;
  long long K;
  strain_dev(*D.n + 1, D.gdot, D.dt, D.ratio, s_d, K);   // stages 2-3 use s^{n+1}
  const int m = m0 + col;
  const double qx_d = m * D.qx_unit;
  const T qx = (T)qx_d;
  const T sqx = (T)(s_d * qx_d);
  const T norm = (T)D.inv_nxny, qyu = (T)D.qy_unit;
  const T cnu = (T)D.c_hdt_nu, dt = (T)D.dt;
#pragma unroll 2
  for (int q = 0; q < 8; ++q) {
    const int nn = tid + q * Tc;
    C psi = C{T(0), T(0)}, w = C{T(0), T(0)};
    if (nn != (ny >> 1) && !(m == 0 && nn == 0)) {
      const int ns = nn < (ny >> 1) ? nn : nn - ny;
      const T ky = (T)ns * qyu - sqx;
      const T k2 = qx * qx + ky * ky;
      const C G = bufG[nn];
      if (stokes) {
        const T inv = norm / (k2 * k2);
        psi = C{G.x * inv, G.y * inv};
      } else {
        const C W = bufW[nn];
        const T a = T(1) - cnu * k2;
        const T inv = norm / (T(1) + cnu * k2);
        w = C{(a * W.x + dt * G.x) * inv, (a * W.y + dt * G.y) * inv};
        const T ik = T(1) / k2;
        psi = C{w.x * ik, w.y * ik};
      }
    }
    bufG[nn] = psi;
    if (!stokes) bufW[nn] = w;
  }
  if (!stokes) {
    C* const b2[2] = {bufG, bufW};
    fft_smem<true, 2>(b2, log2ny, tid, tw);
    store_cols(sm, static_cast<C*>(D.xs_g), m0, ncol, log2ncol, ny, half);
    store_cols(sm + ncol * ny, static_cast<C*>(D.xs_w), m0, ncol, log2ncol, ny, half);
  } else {
    C* const b1[1] = {bufG};
    fft_smem<true, 1>(b1, log2ny, tid, tw);
    store_cols(sm, static_cast<C*>(D.xs_g), m0, ncol, log2ncol, ny, half);
  }
}

// ----------------------------------------------------------- inverse rows
// Two real rows a, b from their half spectra: Z[k] = A[k] + i B[k] (k < N/2),
// Z[N/2] = 0, Z[k] = conj A[N-k] + i conj B[N-k] (k > N/2); z = IFFT(Z).
// mode 0: phi, row pairs (2p, 2p+1) of xs_phi -> phi, with the wrap remap;
// mode 1: inertial members: (xs_g, xs_w) row p -> (psi, omega) row p;
//         Stokes members: row pairs of xs_g -> psi.  Mode 1 advances n.
template <class T>
__global__ void __launch_bounds__(512) k_rowinv(const MemberDesc* __restrict__ descs, int log2nx,
                                                 int log2ny, const cplx<T>* __restrict__ tw, int mode) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, half = nx >> 1;
  const int Tf = nx >> 3;
  const int inst = threadIdx.x / Tf, tid = threadIdx.x - inst * Tf;
  const int ipc = blockDim.x / Tf;
  const int p = blockIdx.x * ipc + inst;
  const bool pairs = (mode == 0) || D.stokes;
  const int count = pairs ? (ny >> 1) : ny;
  if (blockIdx.x * ipc >= count) return;           // whole CTA idle (uniform)
  const bool active = p < count;
  const C *ia, *ib;
  T *oa, *ob;
  int ra, rb, sha = 0, shb = 0;
  if (mode == 0) {
    ia = ib = static_cast<const C*>(D.xs_phi);
    oa = ob = static_cast<T*>(D.phi);
    ra = 2 * p;
    rb = 2 * p + 1;
    if (D.remap) {
      double s0, s1;
      long long K0, K1;
      const long long n = *D.n;
      strain_dev(n, D.gdot, D.dt, D.ratio, s0, K0);
      strain_dev(n + 1, D.gdot, D.dt, D.ratio, s1, K1);
      if (K1 != K0) {
        sha = remap_shift(K1 - K0, D.ratio, ra, nx);
        shb = remap_shift(K1 - K0, D.ratio, rb, nx);
      }
    }
  } else if (D.stokes) {
    ia = ib = static_cast<const C*>(D.xs_g);
    oa = ob = static_cast<T*>(D.psi);
    ra = 2 * p;
    rb = 2 * p + 1;
  } else {
    ia = static_cast<const C*>(D.xs_g);
    ib = static_cast<const C*>(D.xs_w);
    oa = static_cast<T*>(D.psi);
    ob = static_cast<T*>(D.omega);
    ra = rb = p;
  }
  C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)inst * nx;
  if (active) {
    const C* A_ = ia + (size_t)ra * half;
    const C* B_ = ib + (size_t)rb * half;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = tid + q * Tf;
      C z;
      if (k < half) {
        const C A = A_[k], B = B_[k];
        z = (k == 0) ? C{A.x, B.x} : C{A.x - B.y, A.y + B.x};
      } else if (k == half) {
        z = C{T(0), T(0)};
      } else {
        const C A = A_[nx - k], B = B_[nx - k];
        z = C{A.x + B.y, B.x - A.y};
      }
      buf[k] = z;
    }
  }
  {
    C* const b1[1] = {buf};
    fft_smem<true, 1>(b1, log2nx, tid, tw);
  }
  if (active) {
    T* a_row = oa + (size_t)ra * nx;
    T* b_row = ob + (size_t)rb * nx;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = tid + q * Tf;
      const C z = buf[i];
      a_row[(i + sha) & mx] = z.x;
      b_row[(i + shb) & mx] = z.y;
    }
  }
  if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) *D.n += 1;
}

// ----------------------------------------------------------------- stage 2
template <class T>
__global__ void __launch_bounds__(512) k_stage2(const MemberDesc* __restrict__ descs, int log2nx,
                                                 int log2ny, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const MemberDesc& D = descs[blockIdx.y];
  const int nx = 1 << log2nx, ny = 1 << log2ny, mx = nx - 1, my = ny - 1, half = nx >> 1;
  const int Tf = nx >> 3;
  const int inst = threadIdx.x / Tf, tid = threadIdx.x - inst * Tf;
  const int ipc = blockDim.x / Tf;
  const int pair = blockIdx.x * ipc + inst;
  const int j0 = 2 * pair;
  unsigned char* base = smem_raw + (size_t)inst * nx * (sizeof(C) + 4 * sizeof(T));
  C* z = reinterpret_cast<C*>(base);
  T* mu = reinterpret_cast<T*>(base + nx * sizeof(C));

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
  const T* __restrict__ phi = static_cast<const T*>(D.phi);

  // mu on rows j0-1 .. j0+2 (Appendix B item 2: 3-point second differences and
  // the 4-point cross difference)
  for (int e = tid; e < 4 * nx; e += Tf) {
    const int rr = e >> log2nx, i = e & mx, j = j0 - 1 + rr;
    const T pc = ldf(phi, i, j, mx, my, log2nx);
    const T dxx = (ldf(phi, i + 1, j, mx, my, log2nx) - T(2) * pc + ldf(phi, i - 1, j, mx, my, log2nx)) * ih2;
    const T dyy = (ldf(phi, i, j + 1, mx, my, log2nx) - T(2) * pc + ldf(phi, i, j - 1, mx, my, log2nx)) * ih2;
    const T dxy = (ldf(phi, i + 1, j + 1, mx, my, log2nx) - ldf(phi, i + 1, j - 1, mx, my, log2nx) -
                   ldf(phi, i - 1, j + 1, mx, my, log2nx) + ldf(phi, i - 1, j - 1, mx, my, log2nx)) * i4h2;
    const T lap = cxx * dxx - cxy * dxy + dyy;
    mu[e] = -a * pc + b * ((pc * pc) * pc) - kappa * lap;
  }
  __syncthreads();
#pragma unroll 1
  for (int jj = 0; jj < 2; ++jj) {
    const int j = j0 + jj;
    const T* mc = mu + (jj + 1) * nx;
    const T* mu_up = mc + nx;
    const T* mu_dn = mc - nx;
#pragma unroll 2
    for (int q = 0; q < 8; ++q) {
      const int i = tid + q * Tf;
      const T dxphi = dx_central(phi, i, j, mx, my, log2nx, inv2h);
      const T dyphi = dy_sheared(phi, i, j, mx, my, log2nx, w0, w1, d, inv2h);
      const T dxmu = (mc[(i + 1) & mx] - mc[(i - 1) & mx]) * inv2h;
      const T dymu = (w0 * (mu_up[i] - mu_dn[i]) + w1 * (mu_up[(i + d) & mx] - mu_dn[(i - d) & mx])) * inv2h;
      const T g = cf * (dxphi * dymu - dyphi * dxmu);
      if (jj == 0) z[i].x = g;
      else z[i].y = g;
    }
  }
  {
    C* const b1[1] = {z};
    fft_smem<false, 1>(b1, log2nx, tid, tw);
  }
  C* xg = static_cast<C*>(D.xs_g) + (size_t)j0 * half;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = tid + q * Tf;
    C A, B;
    split_real_pair(z, k, mx, A, B);
    xg[k] = A;
    xg[half + k] = B;
  }
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
  k_colpass_phi<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
}
template <class T>
void launch_rowinv(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw, const RowCfg& c,
                   int mode, cudaStream_t st) {
  k_rowinv<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw, mode);
}
template <class T>
void launch_stage2(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw, const RowCfg& c,
                   cudaStream_t st) {
  k_stage2<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
}
template <class T>
void launch_colpass_flow(const MemberDesc* d, int nmem, int log2nx, int log2ny, const cplx<T>* tw,
                         const ColCfg& c, cudaStream_t st) {
  k_colpass_flow<T><<<dim3(c.ctas, nmem), c.threads, c.smem, st>>>(d, log2nx, log2ny, tw);
}

template <class T>
void set_step_smem_limits() {
  const int lim = 220 * 1024;   // dynamic part; leaves room for static shared memory
  cudaFuncSetAttribute(k_stage1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_colpass_phi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_colpass_flow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_rowinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
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
