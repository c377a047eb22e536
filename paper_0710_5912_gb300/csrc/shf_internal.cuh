// Internal declarations shared by the kernels and the host orchestration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_block.cuh"

namespace shf {

// Per-member step state in device memory: the step counter n and the strain
// bookkeeping of the step that starts at n (Section V), evaluated once per
// step by a single thread (the last kernel of the previous step, or
// k_step_state_init) so that no kernel evaluates the FP64 strain per thread.
struct StepState {
  long long n;
  long long dK;     // K(n+1) - K(n): nonzero when the strain wraps during the step
  double s0, s1;    // s(t^n), s(t^{n+1})
};

// Per-member descriptor, resident in device memory (one entry per run of a
// batched launch; blockIdx.y selects the member).  All fields are row-major
// ny x nx reals; the x-spectral ("row-transformed") buffers hold, per row j,
// the modes m = 0 .. nx/2-1 of the row's real DFT in a tiled order (see
// step_kernels.cu); the Nyquist column m = nx/2 is zeroed by the scheme and
// only the row coefficient of phi* / omega* is kept, to subtract it.
struct MemberDesc {
  void* phi;
  void* psi;
  void* omega;
  void* xs_phi;   // phi* -> phi^{n+1} (x-spectral)
  void* xs_f;     // f = phi^3 (x-spectral)
  void* xs_w;     // omega* -> omega^{n+1} (x-spectral)
  void* xs_g;     // g = -F/rho or -F/eta -> psi^{n+1} (x-spectral)
  void* phi_star;    // phi* = phi^n - dt J(psi, phi) (real), base of the increment
  void* omega_star;  // omega* (real, already remapped at a wrap)
  void* nyq_phi;     // per row: the real Nyquist coefficient of phi*'s row DFT
  void* nyq_omega;   // per row: the same for omega*
  // FP32 members: vorticity carried in 2D spectral form and low modes of the
  // force computed apart (see step_cols.cu).  w_hat: the 2D DFT of omega
  // (unnormalised), nx/2 x ny complex in the column-chunk layout of the
  // column passes; low_rows: the row DFT coefficients m = 0..lowm of g's rows,
  // ny complex per m (element m ny + j), then a plane of the same shape with
  // the low parts of double-float coefficients (low == 2); low_hat: the 2D DFT of g at
  // m = 0..lowm, n = -lown..lown, (2 lown + 1) complex per m.
  void* w_hat;
  void* low_rows;
  void* low_hat;
  // FP32 members with rows of 1024 points or more: TMA tensor maps (CUtensorMap,
  // 128 bytes each, in device memory) of xs_phi, xs_g and xs_w, each viewed as
  // [nx / 4 chunk columns][ny rows][4 floats], for the inverse row passes'
  // row-pair gathers; null: those gathers use per-thread asynchronous copies
  const void* tmap;
  int* err;       // device flag of the grid: a bounded wait in a kernel gave up (SHF_ETIMEOUT)
  StepState* st;  // device step counter and strain of the current step
  // parameters and derived constants (double; cast to the working precision)
  double a, b, kappa, M, eta, rho, gdot, dt, dx;
  double c_dt_aM;        // dt a M
  double c_dt_bM;        // dt b M
  double c_hdt_kM;       // dt kappa M / 2
  double c_hdt_nu;       // dt (eta / rho) / 2      (inertial)
  double c_force;        // -1/rho (inertial) or -1/eta (Stokes), multiplies F
  double inv_2h, inv_h2, inv_4h2;
  double inv_nxny;       // 1 / (nx ny), the inverse-transform normalisation
  double qx_unit, qy_unit;  // 2 pi / (nx dx), 2 pi / (ny dx)
  int stokes;            // rho == 0
  int remap;             // 1 when the SHIFT remap is active
  int ratio;             // nx / ny
  int wspec;             // 1: omega carried as w_hat (FP32 inertial); 0: increment form on omega*
  int low;               // FP32: the low modes of g_hat come from low_hat; their row
                         // coefficients from the row pass's compensated sums (1,
                         // inertial) or from k_lowrows_exact (2, Stokes); 0: FP64
  int lowm, lown;        // the low-mode window of this size: m <= lowm, |n| <= lown
  int pad_;
};

// Low-mode window of the force (FP32): the row transform of g takes its
// coefficients m <= kLowM from the first radix-16 stage with compensated
// sums, a small column DFT takes n in [-kLowN, kLowN] from them, and the flow
// column pass uses these in place of its own transform there.  kLowM = 8 is
// the most the row pass's exchange buffer can hold (2 (2 kLowM + 1) floats
// per thread).
constexpr int kLowM = 8;
constexpr int kLowN = 16;
// FP32 Stokes members form the force itself beyond FP32 for their low modes
// (k_lowrows_exact), over m <= kLowMExact.  1/k^4 weights the FP32 rounding
// of F by k^-8 in psi's error, yet a narrower window (m <= 4) leaves psi's
// error twice as large after 200 steps: the rounding at m = 5..8 reaches the
// lowest modes through the advection of phi
constexpr int kLowMExact = 8;

// Strain sawtooth of Section V from the integer step n (same operation order
// as the host and the oracle; explicit rounding intrinsics keep the compiler
// from contracting it): total = (gdot dt) n, K = floor(total / r + 1/2),
// s = total - K r.
__device__ __forceinline__ void strain_dev(long long n, double gdot, double dt, int r, double& s,
                                           long long& K) {
  const double total = __dmul_rn(__dmul_rn(gdot, dt), (double)n);
  const double Kd = floor(__dadd_rn(__ddiv_rn(total, (double)r), 0.5));
  s = __dsub_rn(total, __dmul_rn(Kd, (double)r));
  K = (long long)Kd;
}

// Shared memory of one instance of the persistent transform kernels (rounded
// to 128 bytes so that every instance's staging buffer is 16-byte aligned):
// rowfwd stages two real rows and holds the padded FFT buffer; colpass stages
// one x-spectral chunk column of each input field plus the buffer; rowinv
// stages the 32-byte chunks of a row pair (nx complex) plus the buffer.
__host__ __device__ constexpr size_t round128(size_t b) { return (b + 127) & ~(size_t)127; }
__host__ __device__ constexpr size_t rowfwd_inst_bytes(int nx, size_t real_bytes) {
  return round128(2 * (size_t)nx * real_bytes + (size_t)padded_len(nx) * 2 * real_bytes);
}
// the FP64 column pass stages two columns of 16-byte complex doubles plus
// the padded exchange buffer
__host__ __device__ constexpr size_t colpass_inst_bytes(int ny, size_t /*real_bytes*/) {
  return round128((2 * (size_t)ny + (size_t)padded_len(ny)) * 16);
}
// the FP32 single-mode column pass: two staged columns and the padded
// exchange buffer, 8-byte complex elements
__host__ __device__ constexpr size_t colsingle_inst_bytes(int ny) {
  return round128((2 * (size_t)ny + (size_t)padded_len(ny)) * 8);
}
// the FP32 chunk column pass (ny >= 512): one CTA stages a two-mode chunk of
// two fields (16-byte rows) and holds one padded exchange buffer per mode;
// its mbarrier follows the twiddle table (kColBarBytes)
constexpr size_t kColBarBytes = 128;
__host__ __device__ constexpr size_t colchunk_cta_bytes(int ny) {
  return round128(2 * (size_t)ny * 16 + 2 * (size_t)padded_len(ny) * 8);
}
// the fused stage-1 row pass: per instance two padded buffers (phi*'s pair
// and omega*'s), each holding a row pair's stencil outputs (2 nx reals) and
// then serving as the FFT exchange buffer; stage1_inst_bytes is one buffer
__host__ __device__ constexpr size_t stage1_inst_bytes(int nx, size_t real_bytes) {
  return round128((size_t)padded_len(nx) * 2 * real_bytes);
}
// the inverse row pass's mbarriers (one per instance, at most 4 with TMA),
// after its twiddle table
constexpr size_t kRowinvBarBytes = 128;
__host__ __device__ constexpr size_t rowinv_inst_bytes(int nx, size_t real_bytes) {
  return round128(((size_t)nx + (size_t)padded_len(nx)) * 2 * real_bytes);
}
// the compact twiddle table that follows the instances of a transform kernel
// (2^LP points per thread): two complex values per pair
__host__ __device__ constexpr size_t stage_table_bytes(int log2n, int LP, size_t real_bytes) {
  return round128((size_t)compact_stage_pairs(log2n, LP) * 4 * real_bytes);
}

// Row transforms come in two variants, P = 8 points per thread (radix-8
// stages, 512-thread CTAs) and P = 16 (radix-16 stages, 256-thread CTAs, FP32
// only); the column passes use 8 points and 512 threads.  The fused stage-1
// pass's P and the stage-2 stencil tile height are tuning knobs
// (shf_autotune); the FP32 g row pass uses P = 16 (its first radix-16 stage
// yields the force's low modes) and the FP32 inverse rows P = 16 (8% faster
// than 8 in the flow pass, equal in the phi pass at 4096^2).
constexpr int rowfwd_cta_threads(int P) { return P == 16 ? 256 : 512; }
template <class T> constexpr int rowfwd_min_ctas(int P) { return P == 16 ? 3 : (sizeof(T) == 4 ? 2 : 1); }
template <class T> constexpr int rowfwd_default_points() { return sizeof(T) == 4 ? 16 : 8; }
template <class T> constexpr int rowinv_default_points() { return sizeof(T) == 4 ? 16 : 8; }

// The launches of a step, in order (KIND_LOWMODE runs for FP32 classes only).
enum StepKind {
  KIND_STAGE1 = 0,        // stage-1 stencil fused with the row transforms of phi*, f, omega*
  KIND_COLPASS_PHI = 1,
  KIND_ROWINV_PHI = 2,
  KIND_STAGE2 = 3,        // stage-2 stencil fused with the row transform of g (+ its low row modes)
  KIND_LOWMODE = 4,
  KIND_COLPASS_FLOW = 5,
  KIND_ROWINV_FLOW = 6,
  KIND_COUNT = 7
};
// Launches outside the step: the 2D transform of omega into w_hat (after
// the fields were set from outside), as a row pass and a column pass.
enum { KIND_ROWFWD_OMEGA = 100, KIND_COLPASS_WINIT = 101 };

struct LaunchCfg {
  int grid_x, grid_y;   // grid (the member index is the last grid dimension)
  int threads;
  size_t smem;          // dynamic shared memory bytes
  int inst_per_cta;     // transform instances per CTA (persistent kinds)
  int variant;          // rows: points per thread (8, 16);
                        // FP32 flow column pass: members' regime (1 inertial, 2 Stokes, 3 mixed)
};

template <class T> void launch_step_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny,
                                           const cplx<T>* tw, const LaunchCfg& c, cudaStream_t st);
template <class T> int step_kernel_occupancy(int kind, int log2n, int variant, int threads, size_t smem);
// the transform kernels by family (step_rows.cu, step_cols.cu)
template <class T> void launch_row_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny,
                                          const cplx<T>* tw, const LaunchCfg& c, cudaStream_t st);
template <class T> void launch_col_kernel(int kind, const MemberDesc* d, int nmem, int log2nx, int log2ny,
                                          const cplx<T>* tw, const LaunchCfg& c, cudaStream_t st);
template <class T> int row_kernel_occupancy(int kind, int log2nx, int variant, int threads, size_t smem);
template <class T> int col_kernel_occupancy(int log2ny, int threads, size_t smem);
template <class T> void set_row_smem_limits(int lim);
template <class T> void set_col_smem_limits(int lim);
// the column DFT of the low row modes of g (FP32 members): low_rows -> low_hat;
// twff: W[k] = exp(2 pi i k / NMAX) as (cos hi, cos lo, sin hi, sin lo)
// bytes of a member's low_rows buffer (FP32)
size_t lowrows_bytes(int nx, int ny);
void launch_lowrows_exact(const MemberDesc* d, int nmem, int log2nx, int log2ny, const float4* twff,
                          cudaStream_t st);
void launch_lowmode_cols(const MemberDesc* d, int nmem, int log2ny, const float4* twff, cudaStream_t st);

// ---- kernel launchers (step_kernels.cu / diag_kernels.cu) ----
struct RowCfg {
  int inst_per_cta;   // FFT instances per CTA
  int threads;        // inst_per_cta * nx / 8
  int ctas;           // grid.x
  size_t smem;        // dynamic shared memory bytes
};
struct ColCfg {
  int cols_per_cta;
  int log2cols;
  int threads;        // cols_per_cta * ny / 8
  int ctas;
  size_t smem;
};

template <class T> void launch_convert_in(const double* src, T* dst, long long count, cudaStream_t st);
template <class T> void launch_convert_out(const T* src, double* dst, long long count, cudaStream_t st);
// partial Neumaier sums of a real field: out[3*b + {0,1,2}] = (sum, compensation,
// non-finite count) of CTA b; returns the number of CTAs used
template <class T> int launch_mass_partials(const T* f, long long count, double* out, int max_ctas,
                                            cudaStream_t st);
// the partials folded on the device in a fixed order: out[0..2] = (sum,
// compensation, non-finite count); one warp
void launch_mass_fold(const double* partials, int ctas, double* out, cudaStream_t st);
// structure factor: row transform of phi into xs (complex ny x nx/2), then per
// partial sums per CTA of the structure-factor pass (see k_sf_cols)
constexpr int kSfMoments = 7;
// CTA partial moments (kSfMoments per CTA) and per-CTA bins
template <class T> void launch_sf_rows(const T* phi, cplx<T>* xs, int log2nx, int log2ny,
                                       const cplx<T>* tw, const RowCfg& c, cudaStream_t st);
template <class T> void launch_sf_cols(const cplx<T>* xs, int log2nx, int log2ny, double dx, double s,
                                       const cplx<T>* tw, const ColCfg& c, double* partials, int nbins,
                                       double* bin_partials, cudaStream_t st);
void launch_reduce_rows(const double* in, int rows, int cols, double* out, cudaStream_t st);
template <class T> void set_step_smem_limits();
// recompute every member's StepState from its counter (before a run of steps)
void launch_step_state_init(const MemberDesc* d, int nmem, cudaStream_t st);
template <class T> void set_diag_smem_limits();

}  // namespace shf
