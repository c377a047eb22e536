/* shf.h -- C ABI of the GB300 sheared model-H stepper.
 *
 * One time step of 2D binary-fluid phase separation with full hydrodynamics
 * under steady shear (Fielding, arXiv:0710.5912): model H (Section II, Eqs.
 * ns, vorticity, stream, streamVort, phi1, mu1) in the co-sheared frame of
 * Section V / Appendix A, where Lees-Edwards boundaries become ordinary
 * periodic ones and shear enters only through grad_c = (d_x, d_y - s(t) d_x),
 * advanced by the three-stage split step of Appendix B.  The chemical
 * potential is mu = -a phi + b phi^3 - kappa lap_c phi; the paper's case is
 * a = b = 1, kappa = M = l^2 in its units (Section IV).
 *
 * Conventions for every entry point:
 *   - return value 0 (SHF_OK) on success, a negative SHF_E* code on failure;
 *     shf_last_error(g) then holds a message (owned by the grid, valid until
 *     the next call on it).  On SHF_EINVAL the grid state is left untouched.
 *   - fields are real arrays of ny rows by nx columns, row-major (x, the
 *     index i, is contiguous; row j is the y index): f[j*nx + i] = f(x_i, y_j)
 *     with x_i = i*dx, y_j = j*dx in the co-sheared frame.
 *   - host pointers are owned by the caller and only read/written during the
 *     call; device memory is owned by the library (except bound buffers).
 *   - calls on one grid are not thread-safe; distinct grids are independent.
 *   - steps are enqueued asynchronously on the grid's stream; errors raised
 *     by the GPU surface at the next synchronising call (shf_sync, shf_get_*,
 *     shf_mass, shf_structure_factor, shf_save).
 */
#ifndef SHF_H
#define SHF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shf_grid shf_grid; /* opaque, library-owned */

enum {
  SHF_OK = 0,
  SHF_EINVAL = -1,     /* bad argument (sizes, parameters, null pointer)      */
  SHF_ENOMEM = -2,     /* device or host allocation failed                    */
  SHF_ECUDA = -3,      /* CUDA runtime error (no device, launch failure, ...) */
  SHF_ENONFINITE = -4, /* phi holds NaN/Inf after stepping (state kept)       */
  SHF_ETIMEOUT = -5,   /* a bounded device-side wait gave up                  */
  SHF_EIO = -6,        /* checkpoint file missing, truncated or corrupt       */
  SHF_ESTATE = -7      /* call not valid in this state (e.g. no params yet)   */
};

enum { SHF_FP32 = 32, SHF_FP64 = 64 };

/* Strain wrap handling (Section V: once s(t) reaches Lx/(2Ly) it is shifted by
 * -Lx/Ly).  SHIFT (default) also relabels the stored fields, row j moving by
 * j*Nx/Ny cells, so the laboratory field stays continuous; NONE only shifts s. */
enum { SHF_REMAP_SHIFT = 0, SHF_REMAP_NONE = 1 };

/* Library version (major*10000 + minor*100 + patch). */
int shf_version(void);

/* Static description of an error code. */
const char* shf_strerror(int code);

/* Message of the last failed call on g (empty string if none). */
const char* shf_last_error(const shf_grid* g);

/* Create a grid of nx by ny points with spacing dx (dx = dy), Appendix B's
 * (Lx N / Ly) x N mesh.  nx, ny: powers of two in [16, 4096] with ny dividing nx
 * (the remap shifts row j by j*nx/ny cells).  precision: SHF_FP32 (bulk float
 * arithmetic; strain, sheared-wavenumber phase and mass in double) or SHF_FP64.
 * cuda_stream: a cudaStream_t to enqueue on, or NULL for a library-owned
 * stream.  The state starts at phi = psi = omega = 0, step 0; parameters must
 * be set before stepping.  Allocates about 9 * nx * ny * sizeof(real) bytes of
 * device memory (state, phi* and omega*, four x-spectral work arrays). */
int shf_create_grid(shf_grid** out, int nx, int ny, double dx, int precision, int remap_mode,
                    void* cuda_stream);

/* Free everything the library owns for g (bound buffers are left alone).
 * Ensemble member views are freed with their ensemble. */
int shf_destroy_grid(shf_grid* g);

/* Model and run parameters (Sections II, IV and V):
 *   a, b, kappa  chemical potential mu = -a phi + b phi^3 - kappa lap phi,
 *   M            mobility (Eq. phi1),
 *   eta, rho     viscosity and density (Eq. ns); rho = 0 selects the
 *                zero-Reynolds-number (Stokes) algorithm of Appendix B,
 *   gdot         shear rate, dt time step.
 * Requires kappa, M, eta, dt > 0 and rho >= 0, all finite; a, b, gdot finite.
 * On an ensemble this sets the same parameters on every member. */
int shf_set_params(shf_grid* g, double a, double b, double kappa, double M, double eta, double rho,
                   double gdot, double dt);

/* Copy fields from host arrays (ny*nx doubles each, row-major) into the
 * device state, converting to the grid's precision.  psi / omega may be NULL
 * (taken as zero).  For Stokes runs omega is ignored. */
int shf_set_fields(shf_grid* g, const double* phi, const double* psi, const double* omega);

/* The same as shf_set_fields / shf_get_fields with float host arrays, for
 * FP32 grids only (SHF_EINVAL otherwise): the values are the grid's own, so
 * nothing is converted and half the bytes cross the host link. */
int shf_set_fields_f32(shf_grid* g, const float* phi, const float* psi, const float* omega);
int shf_get_fields_f32(shf_grid* g, float* phi, float* psi, float* omega);

/* Host-in, host-out stepping for FP32 single grids: upload the state from
 * float host arrays, advance nsteps >= 0 steps (Appendix B, as shf_step), and
 * download the new state, in one synchronising call.
 *   phi_in, psi_in, omega_in: ny*nx floats each, row-major; phi_in NULL keeps
 *     the device state (then psi_in and omega_in must be NULL too); psi_in or
 *     omega_in NULL with phi_in given are taken as zero (omega is ignored for
 *     Stokes runs), as in shf_set_fields_f32.
 *   phi_out, psi_out, omega_out: ny*nx floats each, or NULL to skip; omega_out
 *     of a Stokes run is zero-filled.
 * The download of phi overlaps the last step's flow passes: phi^{n+1} is final
 * once the phi row inverse has run (Appendix B item 1), so it is copied on a
 * second stream while the stage-2 stencil, the g transforms and the flow solve
 * (items 2-3) still run.  Host arrays in pinned memory move at the link's
 * full rate; pageable arrays work but are staged by the driver.  Errors:
 * SHF_EINVAL (ensemble or member view, FP64 grid, inputs without phi_in),
 * SHF_ESTATE (parameters not set), SHF_ECUDA. */
int shf_step_host_f32(shf_grid* g, int64_t nsteps, const float* phi_in, const float* psi_in, const float* omega_in,
                      float* phi_out, float* psi_out, float* omega_out);

/* phi = amp * (2u - 1) per point, u = (z >> 11) * 2^-53 from SplitMix64
 * (Steele, Lea & Flood 2014) started at seed, one draw per point in row-major
 * order; psi = omega = 0 (the quench of Section VII).  Also resets the step
 * counter to 0. */
int shf_init_noise(shf_grid* g, uint64_t seed, double amp);

/* Use caller-owned device buffers (ny*nx reals of the grid's precision, each
 * 16-byte aligned) as the state from now on; the current state is copied
 * into them.  omega may be NULL for a Stokes-only grid.  The caller keeps them
 * alive until shf_destroy_grid or a later bind.  Not allowed on ensembles. */
int shf_bind_device_fields(shf_grid* g, void* d_phi, void* d_psi, void* d_omega);

/* Set the step counter n (t = n dt); s and the wrap count follow from n. */
int shf_set_step(shf_grid* g, int64_t n);

/* Advance nsteps >= 0 time steps (Appendix B, items 1-3 or the Stokes
 * algorithm).  Asynchronous on the grid's stream; long runs replay a CUDA
 * graph of up to 100 steps.  On an ensemble every member advances; each grid
 * size advances on a stream of the library's own, forked from and joined back
 * to the grid's stream by events, so work queued on the grid's stream after
 * this call sees every member's new state. */
int shf_step(shf_grid* g, int64_t nsteps);

/* Advance nsteps >= 1 steps like shf_step, but launch every kernel directly
 * with a CUDA event recorded on the grid's stream before and after it, and
 * return in kernel_ms[0..6] the mean device time per step of each of the seven
 * launches of a step (stage-1 stencil with the row transforms of phi*, f,
 * omega*; phi column pass; phi row inverse; stage-2 stencil with the row
 * transform of g; the force's low modes (FP32 only, 0 for FP64); flow column
 * pass; flow row inverse), summed over size classes.  nkinds must be >= 7.
 * Synchronising; meant for measurement (per-kernel roofline), not for
 * production runs. */
int shf_profile_step(shf_grid* g, int64_t nsteps, double* kernel_ms, int nkinds);

/* Wait for queued work; returns SHF_ENONFINITE if phi holds NaN/Inf, and
 * SHF_ETIMEOUT if a kernel's bounded wait for its own asynchronous (TMA)
 * input copies gave up since the last check (the kernel then stopped early;
 * the state is not a valid step; the flag is cleared). */
int shf_sync(shf_grid* g);

/* Copy the state to host arrays (ny*nx doubles each; any may be NULL).
 * Synchronising.  For Stokes runs omega is returned as zeros. */
int shf_get_fields(shf_grid* g, double* phi, double* psi, double* omega);

/* Step counter n, time t = n dt, strain s(t^n) and wrap count K_n (Section V):
 * total = (gdot*dt)*n, K = floor(total/r + 1/2), s = total - K r, r = nx/ny. */
int shf_get_time(shf_grid* g, int64_t* n, double* t, double* s, int64_t* wraps);

/* Mean of phi with a compensated (Neumaier) double-precision sum. */
int shf_mass(shf_grid* g, double* mean_phi);

/* Structure factor S(q) = |phi_hat(q)|^2 / (nx ny)^2 on the laboratory
 * wavevectors q_c = (q_x, q_y - s q_x) at the current s, k = |q_c|, the k = 0
 * mode and the Nyquist lines excluded (Section VI, Eq. L_structure).
 * moments[5] = { sum S, sum k S, sum S/k, L_1 = 2 pi sum S / sum k S,
 *                L_s = sum S/k / sum S }.
 * S_binned (nullable, nbins <= 4096 doubles): bin b sums S over b <= k/dk < b+1
 * with dk = 2 pi / (ny dx). */
int shf_structure_factor(shf_grid* g, double* S_binned, int nbins, double moments[5]);

/* The anisotropy tensor of Eq. L_matrix (Section III) at the current state:
 * G = { G_xx, G_xy, G_yy }, G_ab = int d_a phi d_b phi / int phi^2 with the
 * laboratory derivatives (d_x, d_y - s d_x), evaluated by Parseval on the
 * modes off the Nyquist lines (k = 0 included in the denominator); units
 * 1/length^2.  lengths (nullable) = { L_par, L_perp }, the reciprocal
 * eigenvalues of D = l G with l = sqrt(kappa / a) (the paper's interfacial
 * width l when a = b = 1, kappa = l^2): L_par from the smaller eigenvalue
 * (the long principal axis), INFINITY for a zero eigenvalue.
 * SHF_ESTATE if phi is identically zero. */
int shf_gradient_tensor(shf_grid* g, double G[3], double lengths[2]);

/* Pick, per size class, the launch variants that run fastest on this GPU:
 * the fused stage-1 row pass (the stage-1 stencil with the row transforms of
 * phi*, f, omega*) with 8 or 16 points per thread (radix-8 or radix-16
 * stages; FP32 only).  The fused stage-2 row pass keeps 16 points in FP32
 * (its first stage yields the force's low modes) and 8 in FP64.
 * Each candidate's kernels are timed on the grid's own buffers; only kernels
 * that write scratch buffers run, so the state (fields, step) is unchanged and
 * results stay within the parity tolerances (the variants round differently).
 * cache_path (nullable): a JSON file of earlier choices keyed by
 * "NXxNY:fp32|fp64:inertial|stokes|mixed"; keys found there are applied
 * without trials, new ones are added.  choices (nullable, nchoices ints):
 * receives (stage1_points, stage2_points) per size class,
 * in order of first appearance among the members.  Parameters must be set.  Not for member
 * views.  SHF_EIO if the cache cannot be written.  The paper has no
 * counterpart: this is a performance knob of the implementation. */
int shf_autotune(shf_grid* g, const char* cache_path, int* choices, int nchoices);

/* Checkpoint: a header (magic, version, sizes, precision, remap mode,
 * parameters, n, CRC-32 of the payload) and phi, psi, omega in the grid's
 * precision, so that a resumed run is bit-identical to an uninterrupted one.
 * shf_load requires a grid of the same nx, ny, dx and precision (else SHF_EINVAL); a missing,
 * truncated or corrupt file gives SHF_EIO and leaves the grid untouched. */
int shf_save(shf_grid* g, const char* path);
int shf_load(shf_grid* g, const char* path);

/* Ensemble of independent runs (the paper's parameter sweeps, Table I) that
 * advance together, one batched launch per pass and per grid size (the grid
 * sizes concurrently, see shf_step).
 * nx[r], ny[r]: as for shf_create_grid; params: nruns rows of
 * (a, b, kappa, M, eta, rho, gdot, dt); dx: nruns spacings or NULL (all 1);
 * seeds: nruns SplitMix64 seeds for the quench state (amplitude amp) or NULL
 * (all fields zero).  Remap mode SHF_REMAP_SHIFT. */
int shf_create_ensemble(shf_grid** out, int nruns, const int* nx, const int* ny, const double* dx,
                        const double* params, const uint64_t* seeds, double amp, int precision,
                        void* cuda_stream);

/* A view of member r of an ensemble: usable with shf_set_fields,
 * shf_get_fields, shf_get_time, shf_mass and shf_structure_factor (not with
 * shf_step, which advances the whole ensemble).  Owned by the ensemble. */
int shf_ensemble_member(shf_grid* ens, int r, shf_grid** view);

/* Host-only helpers (no GPU needed): the strain bookkeeping of shf_get_time
 * and the SplitMix64 quench noise of shf_init_noise, written to out[count]. */
int shf_strain(int64_t n, double gdot, double dt, int nx, int ny, double* s, int64_t* wraps);
int shf_noise_fill(double* out, int64_t count, uint64_t seed, double amp);

/* Mean of a caller-owned device field, like shf_mass, for callers that cannot
 * let the library allocate device memory.  The paper has no counterpart: this
 * is a service entry point, not a step of the method.
 *   d_field: device pointer (or managed) to ny*nx reals of the given
 *     precision (SHF_FP32 or SHF_FP64), row-major, element-aligned; only read.
 *   nx, ny: 1..4096 each (any sizes, not only grid sizes); larger fields are
 *     rejected with SHF_EINVAL before any device work.
 *   cuda_stream: cudaStream_t to run on (NULL: the legacy default stream); the
 *     call synchronises it before returning.
 *   mean_phi: receives the mean; set to NaN first, so it holds NaN after any
 *     error.
 * Same reductions as shf_mass (per-CTA Neumaier partials over the same CTAs,
 * at most 1024, folded in CTA order), so for the same field both return the
 * same bits.  Allocates
 * nothing: the partials live in a fixed 24,600-byte device array of the
 * library, which every device that loads the library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the field's device current) and keeps it; make
 * that first call before any stream capture.  The array is shared by all
 * calls on a device and keeps the last call's contents (the result slot is
 * reset at the start of each call), so calls that overlap in time on one
 * device (from several host threads) race and must be serialised by the
 * caller; calls from one thread never overlap, since each returns only after
 * its stream has drained.  A launch error left pending on the calling thread
 * by earlier work is cleared on entry.  Returns SHF_EINVAL for NULL pointers,
 * a bad precision, sizes out of range, a misaligned or host pointer;
 * SHF_ECUDA for a CUDA failure; SHF_ENONFINITE (mean NaN) if the field holds
 * NaN or Inf.  No grid is involved, so shf_last_error has no message for it. */
int shf_mass_static(const void* d_field, int precision, int nx, int ny, void* cuda_stream, double* mean_phi);

/* Measured fused multiply-add rate of one GPU, the arithmetic ceiling against
 * which the transform passes are read.  Not a step of the method.
 *   precision: SHF_FP32 or SHF_FP64 (the FMA type timed).
 *   device: CUDA device ordinal; the caller's current device is restored.
 *   flops_per_s: receives 2 x FMAs per second (0 on error).
 * Runs independent FMA chains on every SM (a whole number of resident waves)
 * on a stream of its own, growing the loop until one launch lasts at least
 * 20 ms, and times that launch with CUDA events; it takes well under a second.
 * Allocates a few bytes of device memory and frees them.  Returns SHF_EINVAL
 * for a bad precision, device or NULL pointer, SHF_ENOMEM if the allocation
 * fails, SHF_ECUDA for a CUDA failure. */
int shf_fma_peak(int precision, int device, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* SHF_H */
