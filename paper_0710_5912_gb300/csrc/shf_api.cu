// Host side of the C ABI declared in include/shf.h: grid and ensemble objects,
// device memory, launch configuration, per-step orchestration (seven launches
// per step and size class, each size class of an ensemble on its own stream;
// runs of 100 steps are replayed from a captured CUDA graph), TMA tensor maps,
// conversions, diagnostics and checkpoints.
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched at run time)

#include "../../include/shf.h"
#include "shf_internal.cuh"

using namespace shf;

namespace {

constexpr int kVersion = 10000;        // 1.0.0
constexpr size_t kSmemLimit = 220 * 1024;
constexpr int kGraphSteps = 100;
constexpr int kMassCtas = 1024;

struct Member {
  int nx = 0, ny = 0, log2nx = 0, log2ny = 0;
  double dx = 1.0;
  double a = 1, b = 1, kappa = 1, M = 1, eta = 1, rho = 1, gdot = 0, dt = 0;
  bool params_set = false;
  void* phi = nullptr;
  void* psi = nullptr;
  void* omega = nullptr;
  bool bound = false;
  void* xs[4] = {nullptr, nullptr, nullptr, nullptr};
  void* phi_star = nullptr;
  void* omega_star = nullptr;
  void* nyq = nullptr;        // 2 ny reals: nyq_phi then nyq_omega
  void* w_hat = nullptr;      // FP32: omega's 2D transform (inertial), see MemberDesc
  void* low_rows = nullptr;   // FP32: low row modes of g
  void* low_hat = nullptr;    // FP32: low 2D modes of g
  void* tmap = nullptr;       // FP32, nx >= 1024: TMA tensor maps of xs_phi, xs_g, xs_w (see MemberDesc)
  StepState* d_st = nullptr;  // into the owner's step-state array
  int cls = -1, slot = -1;
};

struct SizeClass {
  int nx = 0, ny = 0, log2nx = 0, log2ny = 0;
  std::vector<int> members;
  std::vector<MemberDesc> h_desc;
  MemberDesc* d_desc = nullptr;
  LaunchCfg cfg[KIND_COUNT]{};
  RowCfg sfrows{};
  ColCfg sfcols{};
};

// cuTensorMapEncodeTiled from the driver, fetched once at run time (the
// library links the runtime only); null if the driver does not provide it
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}
// An FP32 x-spectral buffer (element (j, m) at ((m >> 1) ny + j) 2 + (m & 1)
// complex) as a 3D tensor of floats: d0 = the 4 floats of a row's two-mode
// chunk (16 bytes), d1 = the row j (stride 16 bytes), d2 = the chunk column
// (stride 16 ny bytes).  Boxes of {4, 2, 256} are one row pair's 32-byte
// pieces of 256 chunk columns; no L2 promotion (the pieces lie 16 ny bytes
// apart).
bool encode_xs_map(CUtensorMap* out, void* base, int nx, int ny) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {4, (cuuint64_t)ny, (cuuint64_t)(nx / 4)};
  const cuuint64_t strides[2] = {16, (cuuint64_t)ny * 16};
  const cuuint32_t box[3] = {4, 2, 256};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
bool pow2_in_range(int v) { return v >= 16 && v <= NMAX && (v & (v - 1)) == 0; }

}  // namespace

struct shf_grid {
  int kind = 0;                 // 0 grid, 1 ensemble, 2 member view
  shf_grid* parent = nullptr;   // views: the ensemble
  int member = 0;               // views: index into parent->members
  int precision = SHF_FP32;
  int remap_mode = SHF_REMAP_SHIFT;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Member> members;
  std::vector<SizeClass> classes;
  StepState* d_state = nullptr;   // per member: counter and strain of the current step
  int* d_err = nullptr;           // set by a kernel whose bounded wait gave up (SHF_ETIMEOUT)
  long long n = 0;
  void* d_tw = nullptr;     // W[k] = exp(2 pi i k / NMAX) (shared-memory FFTs of the diagnostics)
  void* d_twff = nullptr;   // FP32 grids: W[k] as float pairs (hi, lo) per component, float4 per k
  void* d_twr = nullptr;    // per-stage tables of the register FFT (step kernels)
  double* d_stage = nullptr;
  size_t stage_count = 0;
  double* d_scratch = nullptr;
  size_t scratch_count = 0;
  double* h_pinned = nullptr;
  size_t pinned_count = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t io_stream = nullptr;   // shf_step_host_f32: the early phi download
  std::vector<cudaStream_t> class_streams;   // ensembles: one stream per size class
  cudaEvent_t fork = nullptr;                // ensembles: class streams wait on it
  std::vector<cudaEvent_t> joins;            // ensembles: the grid's stream waits on them
  cudaEvent_t phi_done = nullptr;     // recorded after the last step's phi row inverse
  bool what_valid = false;            // FP32: w_hat holds the 2D transform of the current omega
  std::vector<shf_grid*> views;
  std::string err;
};

namespace {

int fail(shf_grid* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  return code;
}

#define SHF_CUDA(g, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((g), SHF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

shf_grid* owner(shf_grid* g) { return g->kind == 2 ? g->parent : g; }

// (cos, sin)(2 pi k / N) by reduction to the first octant, so that the table
// is exactly symmetric (W[N/4] = i, W[N/2] = -1, ...).
void unit_root(long k, long N, double* c, double* s) {
  k %= N;
  if (k < 0) k += N;
  const long q = k / (N / 4), r = k % (N / 4);
  const double two_pi = 6.283185307179586476925286766559;
  double cr, sr;
  if (8 * r > N) {
    const double th = two_pi * (double)(N / 4 - r) / (double)N;
    cr = std::sin(th);
    sr = std::cos(th);
  } else {
    const double th = two_pi * (double)r / (double)N;
    cr = std::cos(th);
    sr = std::sin(th);
  }
  switch (q) {
    case 0: *c = cr; *s = sr; break;
    case 1: *c = -sr; *s = cr; break;
    case 2: *c = -cr; *s = -sr; break;
    default: *c = sr; *s = -cr; break;
  }
}

// Diagnostic (structure factor) kernels: nx/8 or ny/8 threads per FFT.
RowCfg sf_row_cfg(int nx, int ny, size_t bytes_per_inst) {
  RowCfg c{};
  const int Tf = nx / 8;
  int ipc = 256 / Tf;
  if (ipc < 1) ipc = 1;
  if (ipc > ny / 2) ipc = ny / 2;
  while (ipc > 1 && ipc * bytes_per_inst > kSmemLimit) ipc /= 2;
  c.inst_per_cta = ipc;
  c.threads = ipc * Tf;
  c.ctas = (ny / 2) / ipc;
  c.smem = ipc * bytes_per_inst;
  return c;
}

ColCfg sf_col_cfg(int nx, int ny, size_t bytes_per_row_per_col, size_t elem) {
  ColCfg c{};
  const int Tc = ny / 8;
  int cmin = (int)(32 / elem);
  if (cmin < 1) cmin = 1;
  int C = 256 / Tc;
  if (C < cmin) C = cmin;
  if (C > nx / 2) C = nx / 2;
  while (C > 1 && ((size_t)C * ny * bytes_per_row_per_col > kSmemLimit || C * Tc > 512)) C /= 2;
  c.cols_per_cta = C;
  c.log2cols = ilog2(C);
  c.threads = C * Tc;
  c.ctas = (nx / 2) / C;
  c.smem = (size_t)C * ny * bytes_per_row_per_col;
  return c;
}

int sm_count() {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Persistent transform kernels: nfft/P threads per instance (P points per
// thread: 8, or the forward rows' variant), instances per CTA up to the kind's
// CTA size; the grid holds as many CTAs as are resident at once (occupancy
// query), shared over the members of the launch.
template <class T>
LaunchCfg persistent_cfg(int kind, int nfft, int max_inst, int items, size_t inst_bytes, int nmem, int P = kP,
                         size_t extra = 0) {
  LaunchCfg c{};
  const bool fwd = kind == KIND_STAGE1 || kind == KIND_STAGE2;
  const bool rows = fwd || kind == KIND_ROWINV_PHI || kind == KIND_ROWINV_FLOW;
  const int cta = (rows || P == 16) ? rowfwd_cta_threads(P) : 512;   // FP32 column passes: 16 points, 256 threads
  const int Tf = nfft / P;
  int log2n = 0;
  while ((1 << log2n) < nfft) ++log2n;
  const size_t tab = stage_table_bytes(log2n, P == 16 ? 4 : 3, sizeof(T));   // shared twiddle table
  int ipc = cta / Tf;
  if (ipc < 1) ipc = 1;
  if (ipc > max_inst) ipc = max_inst;
  while (ipc > 1 && ipc * inst_bytes + tab + extra > kSmemLimit) ipc /= 2;
  c.inst_per_cta = ipc;
  c.threads = ipc * Tf;
  c.smem = ipc * inst_bytes + tab + extra;
  c.variant = rows ? P : 0;
  const int work = (items + ipc - 1) / ipc;
  const int resident = step_kernel_occupancy<T>(kind, log2n, c.variant, c.threads, c.smem) * sm_count();
  int g = (resident + nmem - 1) / nmem;
  if (g > work) g = work;
  c.grid_x = g < 1 ? 1 : g;
  c.grid_y = 1;
  return c;
}

// The tuning knobs of a size class: points per thread of the fused stage-1
// row pass (8 or 16; FP64: 8) and of the fused stage-2 row pass (FP32: 16,
// whose radix-16 first stage yields the force's low modes; FP64: 8).  Zero
// means "the default".
struct Tune {
  int stage1_points = 0;
  int stage2_points = 0;
};

template <class T>
Tune resolved(const SizeClass&, Tune t) {
  if (t.stage1_points == 0 || sizeof(T) == 8) t.stage1_points = rowfwd_default_points<T>();
  t.stage2_points = rowfwd_default_points<T>();
  return t;
}

template <class T>
void configure_class_t(SizeClass& cl, Tune tune) {
  tune = resolved<T>(cl, tune);
  const size_t R = sizeof(T), Cx = 2 * R;
  const int nx = cl.nx, ny = cl.ny, nmem = (int)cl.members.size();
  cl.cfg[KIND_STAGE1] = persistent_cfg<T>(KIND_STAGE1, nx, ny / 2, ny / 2, 2 * stage1_inst_bytes(nx, R), nmem,
                                           tune.stage1_points);
  cl.cfg[KIND_STAGE2] = persistent_cfg<T>(KIND_STAGE2, nx, ny / 2, ny / 2, rowfwd_inst_bytes(nx, R), nmem,
                                           tune.stage2_points);
  // column items: single mode columns with 16 points per thread (FP32), or
  // whole 16-byte chunks of one complex double with 8 (FP64)
  const int ncol_items = nx / 2;
  const size_t colb = R == 4 ? colsingle_inst_bytes(ny) : colpass_inst_bytes(ny, R);
  const int colP = R == 4 ? 16 : kP;
  cl.cfg[KIND_COLPASS_PHI] = persistent_cfg<T>(KIND_COLPASS_PHI, ny, ncol_items, ncol_items, colb, nmem, colP);
  if (R == 4 && ny >= 512) {
    // long FP32 columns: the chunk kernel, one two-mode chunk per CTA and item
    LaunchCfg c{};
    c.inst_per_cta = 1;
    c.threads = 2 * (ny / 16);
    c.smem = colchunk_cta_bytes(ny) + stage_table_bytes(cl.log2ny, 4, R) + kColBarBytes;
    const int resident = step_kernel_occupancy<T>(KIND_COLPASS_PHI, cl.log2ny, 0, c.threads, c.smem) * sm_count();
    int g = (resident + nmem - 1) / nmem;
    if (g > nx / 4) g = nx / 4;
    c.grid_x = g < 1 ? 1 : g;
    c.grid_y = 1;
    cl.cfg[KIND_COLPASS_PHI] = c;
  }
  cl.cfg[KIND_COLPASS_FLOW] = cl.cfg[KIND_COLPASS_PHI];
  const int PI = rowinv_default_points<T>();
  cl.cfg[KIND_ROWINV_PHI] = persistent_cfg<T>(KIND_ROWINV_PHI, nx, ny / 2, ny / 2, rowinv_inst_bytes(nx, R), nmem, PI,
                                              kRowinvBarBytes);
  cl.cfg[KIND_ROWINV_FLOW] = persistent_cfg<T>(KIND_ROWINV_FLOW, nx, ny / 2, ny, rowinv_inst_bytes(nx, R), nmem, PI,
                                               kRowinvBarBytes);
  cl.sfrows = sf_row_cfg(nx, ny, nx * Cx);
  cl.sfcols = sf_col_cfg(nx, ny, Cx + 12, Cx);
}

void configure_class(SizeClass& cl, int precision, Tune tune = Tune{}) {
  if (precision == SHF_FP64) configure_class_t<double>(cl, tune);
  else configure_class_t<float>(cl, tune);
}

void host_strain(long long n, double gdot, double dt, int r, double* s, long long* K) {
  volatile double total = (gdot * dt) * (double)n;
  volatile double q = total / (double)r + 0.5;
  const double Kd = std::floor(q);
  volatile double kr = Kd * (double)r;
  *s = total - kr;
  *K = (long long)Kd;
}

MemberDesc make_desc(const shf_grid* o, const Member& m) {
  MemberDesc d{};
  d.phi = m.phi;
  d.psi = m.psi;
  d.omega = m.omega;
  d.xs_phi = m.xs[0];
  d.xs_f = m.xs[1];
  d.xs_w = m.xs[2];
  d.xs_g = m.xs[3];
  d.phi_star = m.phi_star;
  d.omega_star = m.omega_star;
  d.nyq_phi = m.nyq;
  d.nyq_omega = static_cast<char*>(m.nyq) + (size_t)m.ny * (o->precision == SHF_FP64 ? 8 : 4);
  d.st = m.d_st;
  d.a = m.a; d.b = m.b; d.kappa = m.kappa; d.M = m.M; d.eta = m.eta; d.rho = m.rho;
  d.gdot = m.gdot; d.dt = m.dt; d.dx = m.dx;
  d.c_dt_aM = (m.dt * m.a) * m.M;
  d.c_dt_bM = (m.dt * m.b) * m.M;
  d.c_hdt_kM = 0.5 * ((m.dt * m.kappa) * m.M);
  d.stokes = m.rho == 0.0 ? 1 : 0;
  d.c_hdt_nu = d.stokes ? 0.0 : 0.5 * (m.dt * (m.eta / m.rho));
  d.c_force = d.stokes ? -1.0 / m.eta : -1.0 / m.rho;
  d.inv_2h = 1.0 / (2.0 * m.dx);
  d.inv_h2 = 1.0 / (m.dx * m.dx);
  d.inv_4h2 = 1.0 / (4.0 * m.dx * m.dx);
  d.inv_nxny = 1.0 / ((double)m.nx * (double)m.ny);
  const double two_pi = 6.283185307179586476925286766559;
  d.qx_unit = two_pi / (m.nx * m.dx);
  d.qy_unit = two_pi / (m.ny * m.dx);
  d.remap = o->remap_mode == SHF_REMAP_SHIFT ? 1 : 0;
  d.ratio = m.nx / m.ny;
  const bool fp32 = o->precision == SHF_FP32;
  d.w_hat = m.w_hat;
  d.low_rows = m.low_rows;
  d.low_hat = m.low_hat;
  d.tmap = m.tmap;
  d.err = o->d_err;
  d.wspec = fp32 && !d.stokes ? 1 : 0;
  d.low = fp32 ? (m.rho > 0.0 ? 1 : 2) : 0;   // 2: Stokes, F's low row modes formed exactly
  const int lowm_max = d.low == 2 ? kLowMExact : kLowM;
  d.lowm = m.nx / 2 - 1 < lowm_max ? m.nx / 2 - 1 : lowm_max;
  d.lown = m.ny / 2 - 1 < kLowN ? m.ny / 2 - 1 : kLowN;
  return d;
}

int upload_desc(shf_grid* o, int mi) {
  Member& m = o->members[mi];
  SizeClass& cl = o->classes[m.cls];
  cl.h_desc[m.slot] = make_desc(o, m);
  SHF_CUDA(o, cudaMemcpyAsync(cl.d_desc + m.slot, &cl.h_desc[m.slot], sizeof(MemberDesc),
                              cudaMemcpyHostToDevice, o->stream));
  return SHF_OK;
}

size_t real_size(const shf_grid* o) { return o->precision == SHF_FP64 ? 8 : 4; }

int ensure_stage(shf_grid* o, size_t count) {
  if (o->stage_count >= count) return SHF_OK;
  if (o->d_stage) cudaFree(o->d_stage);
  o->d_stage = nullptr;
  o->stage_count = 0;
  if (cudaMalloc(&o->d_stage, count * sizeof(double)) != cudaSuccess)
    return fail(o, SHF_ENOMEM, "staging buffer allocation failed");
  o->stage_count = count;
  return SHF_OK;
}

int ensure_scratch(shf_grid* o, size_t count) {
  if (o->scratch_count >= count) return SHF_OK;
  if (o->d_scratch) cudaFree(o->d_scratch);
  o->d_scratch = nullptr;
  o->scratch_count = 0;
  if (cudaMalloc(&o->d_scratch, count * sizeof(double)) != cudaSuccess)
    return fail(o, SHF_ENOMEM, "scratch allocation failed");
  o->scratch_count = count;
  return SHF_OK;
}

int ensure_pinned(shf_grid* o, size_t count) {
  if (o->pinned_count >= count) return SHF_OK;
  if (o->h_pinned) cudaFreeHost(o->h_pinned);
  o->h_pinned = nullptr;
  o->pinned_count = 0;
  if (cudaMallocHost(&o->h_pinned, count * sizeof(double)) != cudaSuccess)
    return fail(o, SHF_ENOMEM, "pinned host allocation failed");
  o->pinned_count = count;
  return SHF_OK;
}

// Forget the captured graph (the next run of >= kGraphSteps steps captures
// a new one): needed when the members' parameters change, because the flow
// column pass is chosen on the host from their regimes.
int drop_graph(shf_grid* o) {
  if (!o->graph) return SHF_OK;
  SHF_CUDA(o, cudaStreamSynchronize(o->stream));
  cudaGraphExecDestroy(o->graph);
  o->graph = nullptr;
  return SHF_OK;
}

void free_all(shf_grid* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->graph) cudaGraphExecDestroy(g->graph);
  for (auto& m : g->members) {
    if (!m.bound) {
      cudaFree(m.phi);
      cudaFree(m.psi);
      cudaFree(m.omega);
    }
    for (void* p : m.xs) cudaFree(p);
    cudaFree(m.phi_star);
    cudaFree(m.omega_star);
    cudaFree(m.nyq);
    cudaFree(m.w_hat);
    cudaFree(m.low_rows);
    cudaFree(m.low_hat);
    cudaFree(m.tmap);
  }
  for (auto& cl : g->classes) cudaFree(cl.d_desc);
  cudaFree(g->d_state);
  cudaFree(g->d_err);
  cudaFree(g->d_tw);
  cudaFree(g->d_twff);
  cudaFree(g->d_twr);
  cudaFree(g->d_stage);
  cudaFree(g->d_scratch);
  if (g->h_pinned) cudaFreeHost(g->h_pinned);
  if (g->phi_done) cudaEventDestroy(g->phi_done);
  if (g->io_stream) cudaStreamDestroy(g->io_stream);
  for (auto st : g->class_streams) cudaStreamDestroy(st);
  for (auto ev : g->joins) cudaEventDestroy(ev);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  for (auto* v : g->views) delete v;
  delete g;
}

int validate_size(shf_grid* g, int nx, int ny, double dx) {
  if (!pow2_in_range(nx) || !pow2_in_range(ny))
    return fail(g, SHF_EINVAL, "nx and ny must be powers of two in [16, 4096]");
  if (nx % ny != 0) return fail(g, SHF_EINVAL, "ny must divide nx");
  if (!(dx > 0.0) || !std::isfinite(dx)) return fail(g, SHF_EINVAL, "dx must be positive and finite");
  return SHF_OK;
}

int validate_params(shf_grid* g, double a, double b, double kappa, double M, double eta, double rho, double gdot,
                    double dt) {
  const double all[8] = {a, b, kappa, M, eta, rho, gdot, dt};
  for (double v : all)
    if (!std::isfinite(v)) return fail(g, SHF_EINVAL, "parameters must be finite");
  if (!(kappa > 0) || !(M > 0) || !(eta > 0) || !(dt > 0))
    return fail(g, SHF_EINVAL, "kappa, M, eta and dt must be positive");
  if (rho < 0) return fail(g, SHF_EINVAL, "rho must be >= 0");
  return SHF_OK;
}

// Builds an object with the given member sizes; allocates everything.
int build(shf_grid* g, const std::vector<int>& nx, const std::vector<int>& ny, const std::vector<double>& dx) {
  SHF_CUDA(g, cudaGetDevice(&g->device));
  if (!g->stream) {
    SHF_CUDA(g, cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    g->own_stream = true;
  }
  if (g->precision == SHF_FP64) {
    set_step_smem_limits<double>();
    set_diag_smem_limits<double>();
  } else {
    set_step_smem_limits<float>();
    set_diag_smem_limits<float>();
  }
  SHF_CUDA(g, cudaGetLastError());
  const int nm = (int)nx.size();
  g->members.resize(nm);
  if (cudaMalloc(&g->d_state, nm * sizeof(StepState)) != cudaSuccess)
    return fail(g, SHF_ENOMEM, "counter allocation failed");
  SHF_CUDA(g, cudaMemsetAsync(g->d_state, 0, nm * sizeof(StepState), g->stream));
  if (cudaMalloc(&g->d_err, sizeof(int)) != cudaSuccess) return fail(g, SHF_ENOMEM, "flag allocation failed");
  SHF_CUDA(g, cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream));
  const size_t R = real_size(g);
  for (int r = 0; r < nm; ++r) {
    Member& m = g->members[r];
    m.nx = nx[r];
    m.ny = ny[r];
    m.log2nx = ilog2(m.nx);
    m.log2ny = ilog2(m.ny);
    m.dx = dx[r];
    m.d_st = g->d_state + r;
    const size_t bytes = (size_t)m.nx * m.ny * R;
    void** bufs[9] = {&m.phi, &m.psi, &m.omega, &m.xs[0], &m.xs[1], &m.xs[2], &m.xs[3], &m.phi_star,
                      &m.omega_star};
    for (void** p : bufs) {
      if (cudaMalloc(p, bytes) != cudaSuccess) return fail(g, SHF_ENOMEM, "field allocation failed");
      SHF_CUDA(g, cudaMemsetAsync(*p, 0, bytes, g->stream));
    }
    if (cudaMalloc(&m.nyq, 2 * (size_t)m.ny * R) != cudaSuccess)
      return fail(g, SHF_ENOMEM, "field allocation failed");
    SHF_CUDA(g, cudaMemsetAsync(m.nyq, 0, 2 * (size_t)m.ny * R, g->stream));
    if (g->precision == SHF_FP32) {
      // w_hat: nx/2 x ny complex floats (the bytes of one real field); low modes of g
      const size_t lr = lowrows_bytes(m.nx, m.ny);
      const size_t lh = (size_t)(kLowM + 1) * (2 * kLowN + 1) * sizeof(float2);
      if (cudaMalloc(&m.w_hat, bytes) != cudaSuccess || cudaMalloc(&m.low_rows, lr) != cudaSuccess ||
          cudaMalloc(&m.low_hat, lh) != cudaSuccess)
        return fail(g, SHF_ENOMEM, "field allocation failed");
      SHF_CUDA(g, cudaMemsetAsync(m.w_hat, 0, bytes, g->stream));
      SHF_CUDA(g, cudaMemsetAsync(m.low_rows, 0, lr, g->stream));
      SHF_CUDA(g, cudaMemsetAsync(m.low_hat, 0, lh, g->stream));
      if (m.nx >= 1024) {                               // TMA maps for the inverse row passes
        CUtensorMap maps[3];
        if (encode_xs_map(&maps[0], m.xs[0], m.nx, m.ny) && encode_xs_map(&maps[1], m.xs[3], m.nx, m.ny) &&
            encode_xs_map(&maps[2], m.xs[2], m.nx, m.ny)) {
          if (cudaMalloc(&m.tmap, sizeof(maps)) != cudaSuccess) return fail(g, SHF_ENOMEM, "tensor map allocation failed");
          SHF_CUDA(g, cudaMemcpy(m.tmap, maps, sizeof(maps), cudaMemcpyHostToDevice));
        }
      }
    }
    int found = -1;
    for (size_t c = 0; c < g->classes.size(); ++c)
      if (g->classes[c].nx == m.nx && g->classes[c].ny == m.ny) found = (int)c;
    if (found < 0) {
      SizeClass cl;
      cl.nx = m.nx;
      cl.ny = m.ny;
      cl.log2nx = m.log2nx;
      cl.log2ny = m.log2ny;
      g->classes.push_back(cl);
      found = (int)g->classes.size() - 1;
    }
    m.cls = found;
    m.slot = (int)g->classes[found].members.size();
    g->classes[found].members.push_back(r);
  }
  for (auto& cl : g->classes) {
    configure_class(cl, g->precision);
    cl.h_desc.resize(cl.members.size());
    if (cudaMalloc(&cl.d_desc, cl.members.size() * sizeof(MemberDesc)) != cudaSuccess)
      return fail(g, SHF_ENOMEM, "descriptor allocation failed");
  }
  if (g->classes.size() > 1) {                          // a stream per size class (enqueue_steps)
    SHF_CUDA(g, cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
    for (size_t c = 0; c < g->classes.size(); ++c) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      SHF_CUDA(g, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      g->class_streams.push_back(st);
      SHF_CUDA(g, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      g->joins.push_back(ev);
    }
  }
  for (int r = 0; r < nm; ++r) {
    int rc = upload_desc(g, r);
    if (rc) return rc;
  }
  // twiddle table W[k] = exp(2 pi i k / NMAX) and the register FFT's stage
  // tables (for each stage and butterfly k, exp(2 pi i k / L) and
  // exp(2 pi i 2k / L), L = Ns R), both computed in double and rounded once
  // to the working precision
  std::vector<double> tw(2 * NMAX);
  for (int k = 0; k < NMAX; ++k) unit_root(k, NMAX, &tw[2 * k], &tw[2 * k + 1]);
  std::vector<double> twr(2 * (size_t)stage_table_len());
  for (int a = 1; a <= 11; ++a)              // a = 0 (Ns = 1) needs no factors
    for (int lr = 1; lr <= 4 && a + lr <= LOG2_NMAX; ++lr) {
      const long Ns = 1L << a, L = Ns << lr;
      for (long k = 0; k < Ns; ++k) {
        const size_t e = 2 * ((size_t)stage_table_offset(a, lr) + k);
        unit_root(k % L, L, &twr[2 * e], &twr[2 * e + 1]);
        unit_root((2 * k) % L, L, &twr[2 * e + 2], &twr[2 * e + 3]);
      }
    }
  auto upload = [&](void** dst, const std::vector<double>& src) -> int {
    const size_t cnt = src.size() / 2;
    if (g->precision == SHF_FP64) {
      if (cudaMalloc(dst, cnt * sizeof(double2)) != cudaSuccess) return fail(g, SHF_ENOMEM, "twiddles");
      SHF_CUDA(g, cudaMemcpy(*dst, src.data(), cnt * sizeof(double2), cudaMemcpyHostToDevice));
    } else {
      std::vector<float> f(src.size());
      for (size_t i = 0; i < src.size(); ++i) f[i] = (float)src[i];
      if (cudaMalloc(dst, cnt * sizeof(float2)) != cudaSuccess) return fail(g, SHF_ENOMEM, "twiddles");
      SHF_CUDA(g, cudaMemcpy(*dst, f.data(), cnt * sizeof(float2), cudaMemcpyHostToDevice));
    }
    return SHF_OK;
  };
  int rc2 = upload(&g->d_tw, tw);
  if (rc2) return rc2;
  rc2 = upload(&g->d_twr, twr);
  if (rc2) return rc2;
  if (g->precision == SHF_FP32) {
    // the low-mode column DFT's twiddles to about 2^-48: (cos hi, cos lo, sin hi, sin lo)
    std::vector<float> ff(4 * (size_t)NMAX);
    for (int k = 0; k < NMAX; ++k)
      for (int c = 0; c < 2; ++c) {
        const double v = tw[2 * k + c];
        const float hi = (float)v;
        ff[4 * k + 2 * c] = hi;
        ff[4 * k + 2 * c + 1] = (float)(v - (double)hi);
      }
    if (cudaMalloc(&g->d_twff, ff.size() * sizeof(float)) != cudaSuccess) return fail(g, SHF_ENOMEM, "twiddles");
    SHF_CUDA(g, cudaMemcpy(g->d_twff, ff.data(), ff.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  return SHF_OK;
}

// The launches of one step for one size class, in order (kind 0..KIND_COUNT-1).
template <class T>
void launch_kind(shf_grid* o, SizeClass& cl, int kind, cudaStream_t st) {
  const cplx<T>* tw = static_cast<const cplx<T>*>(o->d_twr);
  if (kind == KIND_LOWMODE) {                           // FP32 only: the force's low 2D modes
    if (sizeof(T) == 4) {
      bool stokes = false;
      for (int r : cl.members) stokes = stokes || o->members[r].rho == 0.0;
      const float4* twff = static_cast<const float4*>(o->d_twff);
      if (stokes) launch_lowrows_exact(cl.d_desc, (int)cl.members.size(), cl.log2nx, cl.log2ny, twff, st);
      launch_lowmode_cols(cl.d_desc, (int)cl.members.size(), cl.log2ny, twff, st);
    }
    return;
  }
  LaunchCfg c = cl.cfg[kind];
  if (kind == KIND_COLPASS_FLOW) {                      // the flow pass specialised on the members' regime
    bool inertial = false, stokes = false;
    for (int r : cl.members) (o->members[r].rho > 0.0 ? inertial : stokes) = true;
    c.variant = inertial && stokes ? 3 : (stokes ? 2 : 1);
  }
  launch_step_kernel<T>(kind, cl.d_desc, (int)cl.members.size(), cl.log2nx, cl.log2ny, tw, c, st);
}
template <class T>
void launch_kind(shf_grid* o, SizeClass& cl, int kind) {
  launch_kind<T>(o, cl, kind, o->stream);
}

constexpr int kKinds = KIND_COUNT;

template <class T>
void enqueue_step(shf_grid* o) {
  for (auto& cl : o->classes)
    for (int k = 0; k < kKinds; ++k) launch_kind<T>(o, cl, k);
}

// every member's StepState from its counter; needed once before a run of
// steps (each step's last kernel then prepares the next step's state).  FP32
// grids whose fields were set from outside since their last step also get
// w_hat, omega's 2D transform, recomputed from omega (a row pass and a column
// pass; members without w_hat skip them).
void enqueue_state_init(shf_grid* o) {
  for (auto& cl : o->classes) launch_step_state_init(cl.d_desc, (int)cl.members.size(), o->stream);
  if (o->precision == SHF_FP32 && !o->what_valid) {
    for (auto& cl : o->classes) {
      const int nm = (int)cl.members.size();
      launch_row_kernel<float>(KIND_ROWFWD_OMEGA, cl.d_desc, nm, cl.log2nx, cl.log2ny,
                               static_cast<const float2*>(o->d_twr), cl.cfg[KIND_STAGE2], o->stream);
      launch_col_kernel<float>(KIND_COLPASS_WINIT, cl.d_desc, nm, cl.log2nx, cl.log2ny,
                               static_cast<const float2*>(o->d_twr), cl.cfg[KIND_COLPASS_FLOW], o->stream);
    }
    o->what_valid = true;
  }
}

// k steps.  With several size classes (an ensemble) the classes are
// independent runs: each advances on a stream of its own, forked from and
// joined back to the grid's stream by events, so that the launches of small
// classes fill the SMs the large ones leave idle (inside a graph capture these
// become parallel branches).
template <class T>
void enqueue_class_steps(shf_grid* o, SizeClass& cl, long long k, cudaStream_t st) {
  for (long long i = 0; i < k; ++i)
    for (int kind = 0; kind < kKinds; ++kind) launch_kind<T>(o, cl, kind, st);
}
void enqueue_steps(shf_grid* o, long long k) {
  if (k <= 0) return;
  if (o->class_streams.size() == o->classes.size() && o->classes.size() > 1) {
    cudaEventRecord(o->fork, o->stream);
    for (size_t c = 0; c < o->classes.size(); ++c) {
      cudaStreamWaitEvent(o->class_streams[c], o->fork, 0);
      if (o->precision == SHF_FP64) enqueue_class_steps<double>(o, o->classes[c], k, o->class_streams[c]);
      else enqueue_class_steps<float>(o, o->classes[c], k, o->class_streams[c]);
      cudaEventRecord(o->joins[c], o->class_streams[c]);
      cudaStreamWaitEvent(o->stream, o->joins[c], 0);
    }
    return;
  }
  for (long long i = 0; i < k; ++i) {
    if (o->precision == SHF_FP64) enqueue_step<double>(o);
    else enqueue_step<float>(o);
  }
}

Member* member_of(shf_grid* g) {
  if (g->kind == 2) return &g->parent->members[g->member];
  if (g->kind == 0) return &g->members[0];
  return nullptr;
}

int member_index(shf_grid* g) { return g->kind == 2 ? g->member : 0; }

// sum of mass partials in fixed order; returns (sum, nonfinite count)
template <class T>
int field_sum(shf_grid* o, const Member& m, const void* field, double* total, double* nonfinite) {
  int rc = ensure_scratch(o, 3 * kMassCtas + 3);
  if (rc) return rc;
  rc = ensure_pinned(o, 3);
  if (rc) return rc;
  const long long count = (long long)m.nx * m.ny;
  const int ctas = launch_mass_partials<T>(static_cast<const T*>(field), count, o->d_scratch, kMassCtas, o->stream);
  launch_mass_fold(o->d_scratch, ctas, o->d_scratch + 3 * kMassCtas, o->stream);
  SHF_CUDA(o, cudaGetLastError());
  SHF_CUDA(o, cudaMemcpyAsync(o->h_pinned, o->d_scratch + 3 * kMassCtas, 3 * sizeof(double),
                              cudaMemcpyDeviceToHost, o->stream));
  SHF_CUDA(o, cudaStreamSynchronize(o->stream));
  *total = o->h_pinned[0] + o->h_pinned[1];
  *nonfinite = o->h_pinned[2];
  return SHF_OK;
}

uint32_t crc32_update(uint32_t crc, const unsigned char* p, size_t len) {
  // CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bitwise
  crc = ~crc;
  for (size_t i = 0; i < len; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t nx, ny, precision, remap_mode, has_params;
  double params[9];
  int64_t n;
  uint32_t payload_crc;
  uint32_t header_crc;
};

}  // namespace

namespace {

template <class T>
int set_fields_t(shf_grid* g, const double* phi, const double* psi, const double* omega) {
  shf_grid* o = owner(g);
  o->what_valid = false;
  Member& m = *member_of(g);
  const size_t count = (size_t)m.nx * m.ny;
  const double* src[3] = {phi, psi, m.rho > 0 ? omega : nullptr};
  void* dst[3] = {m.phi, m.psi, m.omega};
  if (sizeof(T) != sizeof(double)) {
    // all copies first (the copy engine streams without waiting for the
    // conversions), then the conversions; one staging slot per field
    int rc = ensure_stage(o, 3 * count);
    if (rc) return fail(g, rc, o->err);
    for (int f = 0; f < 3; ++f)
      if (src[f])
        SHF_CUDA(g, cudaMemcpyAsync(o->d_stage + f * count, src[f], count * sizeof(double), cudaMemcpyHostToDevice,
                                    o->stream));
  }
  for (int f = 0; f < 3; ++f) {
    if (!src[f]) {
      SHF_CUDA(g, cudaMemsetAsync(dst[f], 0, count * sizeof(T), o->stream));
      continue;
    }
    if (sizeof(T) == sizeof(double)) {
      SHF_CUDA(g, cudaMemcpyAsync(dst[f], src[f], count * sizeof(double), cudaMemcpyHostToDevice, o->stream));
    } else {
      launch_convert_in<T>(o->d_stage + f * count, static_cast<T*>(dst[f]), (long long)count, o->stream);
      SHF_CUDA(g, cudaGetLastError());
    }
  }
  SHF_CUDA(g, cudaStreamSynchronize(o->stream));
  return SHF_OK;
}

template <class T>
int get_fields_t(shf_grid* g, double* phi, double* psi, double* omega) {
  shf_grid* o = owner(g);
  Member& m = *member_of(g);
  const size_t count = (size_t)m.nx * m.ny;
  double* dst[3] = {phi, psi, omega};
  const void* src[3] = {m.phi, m.psi, m.omega};
  if (sizeof(T) != sizeof(double)) {
    int rc = ensure_stage(o, 3 * count);
    if (rc) return fail(g, rc, o->err);
  }
  // conversions and copies queue back to back (one staging slot per field)
  for (int f = 0; f < 3; ++f) {
    if (!dst[f]) continue;
    if (f == 2 && m.rho == 0.0) {
      std::memset(dst[f], 0, count * sizeof(double));
      continue;
    }
    if (sizeof(T) == sizeof(double)) {
      SHF_CUDA(g, cudaMemcpyAsync(dst[f], src[f], count * sizeof(double), cudaMemcpyDeviceToHost, o->stream));
    } else {
      launch_convert_out<T>(static_cast<const T*>(src[f]), o->d_stage + f * count, (long long)count, o->stream);
      SHF_CUDA(g, cudaGetLastError());
      SHF_CUDA(g, cudaMemcpyAsync(dst[f], o->d_stage + f * count, count * sizeof(double), cudaMemcpyDeviceToHost,
                                  o->stream));
    }
  }
  SHF_CUDA(g, cudaStreamSynchronize(o->stream));
  return SHF_OK;
}

// The spectral pass over phi (row and column transforms of the current
// state) with the kSfMoments sums of k_sf_cols reduced in fixed order into
// sums[], and optionally the radial bins.
int sf_sums(shf_grid* g, double* S_binned, int nbins, double sums[kSfMoments]) {
  shf_grid* o = owner(g);
  Member& m = *member_of(g);
  SizeClass& cl = o->classes[m.cls];
  double s;
  long long K;
  host_strain(o->n, m.gdot, m.dt, m.nx / m.ny, &s, &K);
  const ColCfg& cc = cl.sfcols;
  const size_t need = (size_t)cc.ctas * kSfMoments + kSfMoments + (size_t)cc.ctas * nbins + nbins;
  int rc = ensure_scratch(o, need);
  if (rc) return fail(g, rc, o->err);
  rc = ensure_pinned(o, kSfMoments + nbins);
  if (rc) return fail(g, rc, o->err);
  double* parts = o->d_scratch;
  double* red = parts + (size_t)cc.ctas * kSfMoments;
  double* bparts = red + kSfMoments;
  double* bred = bparts + (size_t)cc.ctas * nbins;
  if (o->precision == SHF_FP64) {
    using T = double;
    const cplx<T>* tw = static_cast<const cplx<T>*>(o->d_tw);
    cplx<T>* xs = static_cast<cplx<T>*>(m.xs[1]);
    launch_sf_rows<T>(static_cast<const T*>(m.phi), xs, cl.log2nx, cl.log2ny, tw, cl.sfrows, o->stream);
    launch_sf_cols<T>(xs, cl.log2nx, cl.log2ny, m.dx, s, tw, cc, parts, nbins, bparts, o->stream);
  } else {
    using T = float;
    const cplx<T>* tw = static_cast<const cplx<T>*>(o->d_tw);
    cplx<T>* xs = static_cast<cplx<T>*>(m.xs[1]);
    launch_sf_rows<T>(static_cast<const T*>(m.phi), xs, cl.log2nx, cl.log2ny, tw, cl.sfrows, o->stream);
    launch_sf_cols<T>(xs, cl.log2nx, cl.log2ny, m.dx, s, tw, cc, parts, nbins, bparts, o->stream);
  }
  launch_reduce_rows(parts, cc.ctas, kSfMoments, red, o->stream);
  if (nbins > 0) launch_reduce_rows(bparts, cc.ctas, nbins, bred, o->stream);
  SHF_CUDA(g, cudaGetLastError());
  SHF_CUDA(g, cudaMemcpyAsync(o->h_pinned, red, kSfMoments * sizeof(double), cudaMemcpyDeviceToHost, o->stream));
  if (nbins > 0)
    SHF_CUDA(g, cudaMemcpyAsync(o->h_pinned + kSfMoments, bred, nbins * sizeof(double), cudaMemcpyDeviceToHost,
                                o->stream));
  SHF_CUDA(g, cudaStreamSynchronize(o->stream));
  for (int v = 0; v < kSfMoments; ++v) sums[v] = o->h_pinned[v];
  if (S_binned && nbins > 0) std::memcpy(S_binned, o->h_pinned + kSfMoments, nbins * sizeof(double));
  return SHF_OK;
}

}  // namespace

// ------------------------------------------------------------- autotuning
namespace {

std::string tune_key(const shf_grid* o, const SizeClass& cl) {
  bool inertial = false, stokes = false;
  for (int r : cl.members) (o->members[r].rho > 0 ? inertial : stokes) = true;
  char buf[96];
  std::snprintf(buf, sizeof(buf), "%dx%d:%s:%s", cl.nx, cl.ny, o->precision == SHF_FP64 ? "fp64" : "fp32",
                inertial && stokes ? "mixed" : (inertial ? "inertial" : "stokes"));
  return buf;
}

// cache file: a JSON object, one entry per line:
//   "NXxNY:fp32:inertial": {"stage1_points": 16, "stage2_points": 16},
std::map<std::string, Tune> read_tune_cache(const char* path) {
  std::map<std::string, Tune> m;
  if (!path) return m;
  FILE* f = std::fopen(path, "r");
  if (!f) return m;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char key[256];
    Tune t;
    if (std::sscanf(line, " \"%255[^\"]\": {\"stage1_points\": %d, \"stage2_points\": %d", key, &t.stage1_points,
                    &t.stage2_points) == 3)
      m[key] = t;
  }
  std::fclose(f);
  return m;
}

bool write_tune_cache(const char* path, const std::map<std::string, Tune>& m) {
  FILE* f = std::fopen(path, "w");
  if (!f) return false;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : m) {
    std::fprintf(f, "  \"%s\": {\"stage1_points\": %d, \"stage2_points\": %d}%s\n", kv.first.c_str(),
                 kv.second.stage1_points, kv.second.stage2_points, ++i < m.size() ? "," : "");
  }
  std::fprintf(f, "}\n");
  return std::fclose(f) == 0;
}

// mean device time (ms) of one round of the given kinds of class cl
template <class T>
int time_kinds(shf_grid* o, SizeClass& cl, const int* kinds, int nk, float* ms) {
  const int reps = 5;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SHF_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SHF_ECUDA;
  }
  for (int k = 0; k < nk; ++k) launch_kind<T>(o, cl, kinds[k]);   // warm-up
  cudaEventRecord(e0, o->stream);
  for (int r = 0; r < reps; ++r)
    for (int k = 0; k < nk; ++k) launch_kind<T>(o, cl, kinds[k]);
  cudaEventRecord(e1, o->stream);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
  *ms /= reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err == cudaSuccess ? SHF_OK : SHF_ECUDA;
}

// Time the candidate values of each knob on the class's own buffers.  Only
// kinds that write scratch (the stage-1 pass: phi*, omega*, the x-spectral
// buffers) run, so the state (phi, psi, omega, omega_hat, step) is
// untouched.
template <class T>
int tune_class(shf_grid* o, SizeClass& cl, Tune* best) {
  Tune t = resolved<T>(cl, Tune{});
  if (sizeof(T) == 4) {                                // the fused stage-1 row pass: 8 or 16 points
    const int kind = KIND_STAGE1;
    float bestms = 0.f;
    for (int P : {8, 16}) {
      Tune c = t;
      c.stage1_points = P;
      configure_class_t<T>(cl, c);
      float ms = 0.f;
      const int rc = time_kinds<T>(o, cl, &kind, 1, &ms);
      if (rc) return rc;
      if (P == 8 || ms < bestms) {
        bestms = ms;
        t.stage1_points = P;
      }
    }
  }
  *best = t;
  return SHF_OK;
}

// Enqueue nsteps steps on the grid's stream: the state seed, then graph
// replays of kGraphSteps steps and direct launches for the rest.  With
// phi_event (a single FP32 grid), the last step is launched directly and
// phi_event is recorded between its phi passes (after which phi is final) and
// its flow passes.
int run_steps(shf_grid* g, long long nsteps, cudaEvent_t phi_event) {
  if (nsteps > 0) enqueue_state_init(g);
  const bool split = phi_event && nsteps > 0;
  long long left = split ? nsteps - 1 : nsteps;
  if (left >= kGraphSteps) {
    if (!g->graph) {
      cudaGraph_t graph;
      SHF_CUDA(g, cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
      enqueue_steps(g, kGraphSteps);
      cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
      if (e != cudaSuccess) return fail(g, SHF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&g->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g->graph = nullptr;
        return fail(g, SHF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
    }
    while (left >= kGraphSteps) {
      SHF_CUDA(g, cudaGraphLaunch(g->graph, g->stream));
      left -= kGraphSteps;
    }
  }
  enqueue_steps(g, left);
  if (split) {
    for (auto& cl : g->classes)
      for (int k = 0; k <= KIND_ROWINV_PHI; ++k) launch_kind<float>(g, cl, k);
    SHF_CUDA(g, cudaEventRecord(phi_event, g->stream));
    for (auto& cl : g->classes)
      for (int k = KIND_ROWINV_PHI + 1; k < kKinds; ++k) launch_kind<float>(g, cl, k);
  }
  SHF_CUDA(g, cudaGetLastError());
  g->n += nsteps;
  return SHF_OK;
}

}  // namespace

// =========================================================================
extern "C" {

int shf_version(void) { return kVersion; }

const char* shf_strerror(int code) {
  switch (code) {
    case SHF_OK: return "ok";
    case SHF_EINVAL: return "invalid argument";
    case SHF_ENOMEM: return "out of memory";
    case SHF_ECUDA: return "CUDA error";
    case SHF_ENONFINITE: return "non-finite values in phi";
    case SHF_ETIMEOUT: return "device wait timed out";
    case SHF_EIO: return "checkpoint I/O error";
    case SHF_ESTATE: return "invalid state for this call";
    default: return "unknown error";
  }
}

const char* shf_last_error(const shf_grid* g) { return g ? g->err.c_str() : "null grid"; }

int shf_strain(int64_t n, double gdot, double dt, int nx, int ny, double* s, int64_t* wraps) {
  if (!s || !wraps || !pow2_in_range(nx) || !pow2_in_range(ny) || nx % ny) return SHF_EINVAL;
  long long K;
  host_strain(n, gdot, dt, nx / ny, s, &K);
  *wraps = K;
  return SHF_OK;
}

int shf_noise_fill(double* out, int64_t count, uint64_t seed, double amp) {
  if (!out || count < 0 || !std::isfinite(amp)) return SHF_EINVAL;
  uint64_t state = seed;
  for (int64_t k = 0; k < count; ++k) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    out[k] = amp * (2.0 * u - 1.0);
  }
  return SHF_OK;
}

int shf_create_grid(shf_grid** out, int nx, int ny, double dx, int precision, int remap_mode, void* cuda_stream) {
  if (!out) return SHF_EINVAL;
  *out = nullptr;
  shf_grid tmp;
  int rc = validate_size(&tmp, nx, ny, dx);
  if (rc) return rc;
  if (precision != SHF_FP32 && precision != SHF_FP64) return SHF_EINVAL;
  if (remap_mode != SHF_REMAP_SHIFT && remap_mode != SHF_REMAP_NONE) return SHF_EINVAL;
  shf_grid* g = new shf_grid();
  g->kind = 0;
  g->precision = precision;
  g->remap_mode = remap_mode;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  rc = build(g, {nx}, {ny}, {dx});
  if (rc) {
    free_all(g);
    return rc;
  }
  *out = g;
  return SHF_OK;
}

int shf_create_ensemble(shf_grid** out, int nruns, const int* nx, const int* ny, const double* dx,
                        const double* params, const uint64_t* seeds, double amp, int precision,
                        void* cuda_stream) {
  if (!out || nruns <= 0 || !nx || !ny || !params) return SHF_EINVAL;
  *out = nullptr;
  if (precision != SHF_FP32 && precision != SHF_FP64) return SHF_EINVAL;
  shf_grid tmp;
  std::vector<int> vx(nruns), vy(nruns);
  std::vector<double> vd(nruns);
  for (int r = 0; r < nruns; ++r) {
    vx[r] = nx[r];
    vy[r] = ny[r];
    vd[r] = dx ? dx[r] : 1.0;
    if (validate_size(&tmp, vx[r], vy[r], vd[r])) return SHF_EINVAL;
    const double* p = params + 8 * r;
    if (validate_params(&tmp, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7])) return SHF_EINVAL;
  }
  shf_grid* g = new shf_grid();
  g->kind = 1;
  g->precision = precision;
  g->remap_mode = SHF_REMAP_SHIFT;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  int rc = build(g, vx, vy, vd);
  if (rc) {
    free_all(g);
    return rc;
  }
  for (int r = 0; r < nruns; ++r) {
    Member& m = g->members[r];
    const double* p = params + 8 * r;
    m.a = p[0]; m.b = p[1]; m.kappa = p[2]; m.M = p[3]; m.eta = p[4]; m.rho = p[5]; m.gdot = p[6]; m.dt = p[7];
    m.params_set = true;
    rc = upload_desc(g, r);
    if (rc) {
      free_all(g);
      return rc;
    }
  }
  g->views.resize(nruns);
  for (int r = 0; r < nruns; ++r) {
    shf_grid* v = new shf_grid();
    v->kind = 2;
    v->parent = g;
    v->member = r;
    v->precision = precision;
    v->device = g->device;
    g->views[r] = v;
  }
  if (seeds) {
    for (int r = 0; r < nruns; ++r) {
      rc = shf_init_noise(g->views[r], seeds[r], amp);
      if (rc) {
        free_all(g);
        return rc;
      }
    }
  }
  *out = g;
  return SHF_OK;
}

int shf_ensemble_member(shf_grid* ens, int r, shf_grid** view) {
  if (!ens || !view || ens->kind != 1 || r < 0 || r >= (int)ens->views.size()) return SHF_EINVAL;
  *view = ens->views[r];
  return SHF_OK;
}

int shf_destroy_grid(shf_grid* g) {
  if (!g) return SHF_EINVAL;
  if (g->kind == 2) return fail(g, SHF_EINVAL, "member views are freed with their ensemble");
  free_all(g);
  return SHF_OK;
}

int shf_set_params(shf_grid* g, double a, double b, double kappa, double M, double eta, double rho, double gdot,
                   double dt) {
  if (!g) return SHF_EINVAL;
  int rc = validate_params(g, a, b, kappa, M, eta, rho, gdot, dt);
  if (rc) return rc;
  shf_grid* o = owner(g);
  SHF_CUDA(g, cudaSetDevice(o->device));
  std::vector<int> which;
  if (g->kind == 1) {
    for (size_t r = 0; r < o->members.size(); ++r) which.push_back((int)r);
  } else {
    which.push_back(member_index(g));
  }
  for (int r : which) {
    Member& m = o->members[r];
    m.a = a; m.b = b; m.kappa = kappa; m.M = M; m.eta = eta; m.rho = rho; m.gdot = gdot; m.dt = dt;
    m.params_set = true;
    rc = upload_desc(o, r);
    if (rc) return fail(g, rc, o->err);
  }
  rc = drop_graph(o);                                   // the flow pass kernel depends on the regimes
  if (rc) return fail(g, rc, o->err);
  o->what_valid = false;                                // a regime change makes w_hat stale
  return SHF_OK;
}


int shf_set_fields(shf_grid* g, const double* phi, const double* psi, const double* omega) {
  if (!g || !phi) return fail(g, SHF_EINVAL, "phi must not be NULL");
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view to set fields of an ensemble");
  SHF_CUDA(g, cudaSetDevice(owner(g)->device));
  return g->precision == SHF_FP64 ? set_fields_t<double>(g, phi, psi, omega)
                                  : set_fields_t<float>(g, phi, psi, omega);
}

int shf_set_fields_f32(shf_grid* g, const float* phi, const float* psi, const float* omega) {
  if (!g || !phi) return fail(g, SHF_EINVAL, "phi must not be NULL");
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view to set fields of an ensemble");
  if (g->precision != SHF_FP32) return fail(g, SHF_EINVAL, "float fields need an FP32 grid");
  shf_grid* o = owner(g);
  SHF_CUDA(g, cudaSetDevice(o->device));
  o->what_valid = false;
  Member& m = *member_of(g);
  const size_t bytes = (size_t)m.nx * m.ny * sizeof(float);
  const float* src[3] = {phi, psi, m.rho > 0 ? omega : nullptr};
  void* dst[3] = {m.phi, m.psi, m.omega};
  for (int f = 0; f < 3; ++f) {
    if (src[f]) SHF_CUDA(g, cudaMemcpyAsync(dst[f], src[f], bytes, cudaMemcpyHostToDevice, o->stream));
    else SHF_CUDA(g, cudaMemsetAsync(dst[f], 0, bytes, o->stream));
  }
  SHF_CUDA(g, cudaStreamSynchronize(o->stream));
  return SHF_OK;
}

int shf_get_fields_f32(shf_grid* g, float* phi, float* psi, float* omega) {
  if (!g) return SHF_EINVAL;
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view to read fields of an ensemble");
  if (g->precision != SHF_FP32) return fail(g, SHF_EINVAL, "float fields need an FP32 grid");
  shf_grid* o = owner(g);
  SHF_CUDA(g, cudaSetDevice(o->device));
  Member& m = *member_of(g);
  const size_t count = (size_t)m.nx * m.ny;
  float* dst[3] = {phi, psi, omega};
  const void* src[3] = {m.phi, m.psi, m.omega};
  for (int f = 0; f < 3; ++f) {
    if (!dst[f]) continue;
    if (f == 2 && m.rho == 0.0) std::memset(dst[f], 0, count * sizeof(float));
    else SHF_CUDA(g, cudaMemcpyAsync(dst[f], src[f], count * sizeof(float), cudaMemcpyDeviceToHost, o->stream));
  }
  SHF_CUDA(g, cudaStreamSynchronize(o->stream));
  return SHF_OK;
}

int shf_init_noise(shf_grid* g, uint64_t seed, double amp) {
  if (!g || !std::isfinite(amp)) return SHF_EINVAL;
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view to initialise an ensemble member");
  Member& m = *member_of(g);
  std::vector<double> phi((size_t)m.nx * m.ny);
  shf_noise_fill(phi.data(), (int64_t)phi.size(), seed, amp);
  int rc = shf_set_fields(g, phi.data(), nullptr, nullptr);
  if (rc) return rc;
  if (g->kind == 0) return shf_set_step(g, 0);
  return SHF_OK;
}

int shf_bind_device_fields(shf_grid* g, void* d_phi, void* d_psi, void* d_omega) {
  if (!g || g->kind != 0 || !d_phi || !d_psi) return fail(g, SHF_EINVAL, "bind needs a grid and phi, psi");
  Member& m = g->members[0];
  const uintptr_t al = 15;
  if (((uintptr_t)d_phi & al) || ((uintptr_t)d_psi & al) || (d_omega && ((uintptr_t)d_omega & al)))
    return fail(g, SHF_EINVAL, "bound buffers must be 16-byte aligned");
  if (!d_omega && m.rho > 0) return fail(g, SHF_EINVAL, "omega is needed for an inertial grid");
  SHF_CUDA(g, cudaSetDevice(g->device));
  const size_t bytes = (size_t)m.nx * m.ny * real_size(g);
  SHF_CUDA(g, cudaMemcpyAsync(d_phi, m.phi, bytes, cudaMemcpyDeviceToDevice, g->stream));
  SHF_CUDA(g, cudaMemcpyAsync(d_psi, m.psi, bytes, cudaMemcpyDeviceToDevice, g->stream));
  if (d_omega) SHF_CUDA(g, cudaMemcpyAsync(d_omega, m.omega, bytes, cudaMemcpyDeviceToDevice, g->stream));
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  if (!m.bound) {
    cudaFree(m.phi);
    cudaFree(m.psi);
    if (d_omega) cudaFree(m.omega);
  }
  m.phi = d_phi;
  m.psi = d_psi;
  if (d_omega) m.omega = d_omega;
  m.bound = true;
  g->what_valid = false;
  return upload_desc(g, 0);
}

int shf_set_step(shf_grid* g, int64_t n) {
  if (!g || n < 0) return SHF_EINVAL;
  if (g->kind == 2) return fail(g, SHF_EINVAL, "the step counter belongs to the ensemble");
  SHF_CUDA(g, cudaSetDevice(g->device));
  // the strain fields are recomputed on the device before the next step
  std::vector<StepState> v(g->members.size(), StepState{(long long)n, 0, 0.0, 0.0});
  SHF_CUDA(g, cudaMemcpyAsync(g->d_state, v.data(), v.size() * sizeof(StepState), cudaMemcpyHostToDevice,
                              g->stream));
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  g->n = n;
  g->what_valid = false;                                // the next step re-reads omega
  return SHF_OK;
}

int shf_step(shf_grid* g, int64_t nsteps) {
  if (!g || nsteps < 0) return SHF_EINVAL;
  if (g->kind == 2) return fail(g, SHF_EINVAL, "step the ensemble, not a member view");
  for (auto& m : g->members)
    if (!m.params_set) return fail(g, SHF_ESTATE, "shf_set_params must be called before shf_step");
  SHF_CUDA(g, cudaSetDevice(g->device));
  return run_steps(g, nsteps, nullptr);
}

int shf_step_host_f32(shf_grid* g, int64_t nsteps, const float* phi_in, const float* psi_in, const float* omega_in,
                      float* phi_out, float* psi_out, float* omega_out) {
  if (!g || nsteps < 0) return SHF_EINVAL;
  if (g->kind != 0) return fail(g, SHF_EINVAL, "shf_step_host_f32 needs a single grid");
  if (g->precision != SHF_FP32) return fail(g, SHF_EINVAL, "float fields need an FP32 grid");
  if (!phi_in && (psi_in || omega_in)) return fail(g, SHF_EINVAL, "inputs need phi_in");
  Member& m = g->members[0];
  if (!m.params_set) return fail(g, SHF_ESTATE, "shf_set_params must be called before shf_step_host_f32");
  SHF_CUDA(g, cudaSetDevice(g->device));
  if (!g->io_stream) SHF_CUDA(g, cudaStreamCreateWithFlags(&g->io_stream, cudaStreamNonBlocking));
  if (!g->phi_done) SHF_CUDA(g, cudaEventCreateWithFlags(&g->phi_done, cudaEventDisableTiming));
  const size_t bytes = (size_t)m.nx * m.ny * sizeof(float);
  if (phi_in) {
    g->what_valid = false;
    const float* src[3] = {phi_in, psi_in, m.rho > 0 ? omega_in : nullptr};
    void* dst[3] = {m.phi, m.psi, m.omega};
    for (int f = 0; f < 3; ++f) {
      if (src[f]) SHF_CUDA(g, cudaMemcpyAsync(dst[f], src[f], bytes, cudaMemcpyHostToDevice, g->stream));
      else SHF_CUDA(g, cudaMemsetAsync(dst[f], 0, bytes, g->stream));
    }
  }
  const bool early = nsteps > 0 && phi_out;
  const int rc = run_steps(g, nsteps, early ? g->phi_done : nullptr);
  if (rc) return rc;
  if (phi_out) {
    if (early) {                                        // phi is final once the last step's phi passes are done
      SHF_CUDA(g, cudaStreamWaitEvent(g->io_stream, g->phi_done, 0));
      SHF_CUDA(g, cudaMemcpyAsync(phi_out, m.phi, bytes, cudaMemcpyDeviceToHost, g->io_stream));
    } else {
      SHF_CUDA(g, cudaMemcpyAsync(phi_out, m.phi, bytes, cudaMemcpyDeviceToHost, g->stream));
    }
  }
  if (psi_out) SHF_CUDA(g, cudaMemcpyAsync(psi_out, m.psi, bytes, cudaMemcpyDeviceToHost, g->stream));
  if (omega_out) {
    if (m.rho > 0) SHF_CUDA(g, cudaMemcpyAsync(omega_out, m.omega, bytes, cudaMemcpyDeviceToHost, g->stream));
    else std::memset(omega_out, 0, bytes);
  }
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  SHF_CUDA(g, cudaStreamSynchronize(g->io_stream));
  return SHF_OK;
}

int shf_profile_step(shf_grid* g, int64_t nsteps, double* kernel_ms, int nkinds) {
  if (!g || nsteps <= 0 || !kernel_ms || nkinds < kKinds) return fail(g, SHF_EINVAL, "bad profile arguments");
  if (g->kind == 2) return fail(g, SHF_EINVAL, "step the ensemble, not a member view");
  for (auto& m : g->members)
    if (!m.params_set) return fail(g, SHF_ESTATE, "shf_set_params must be called before shf_profile_step");
  SHF_CUDA(g, cudaSetDevice(g->device));
  const size_t ncls = g->classes.size();
  const size_t nev = (size_t)nsteps * ncls * (kKinds + 1);
  std::vector<cudaEvent_t> ev(nev, nullptr);
  int rc = SHF_OK;
  for (size_t e = 0; e < nev && rc == SHF_OK; ++e)
    if (cudaEventCreate(&ev[e]) != cudaSuccess) rc = fail(g, SHF_ECUDA, "event creation failed");
  if (rc == SHF_OK) {
    enqueue_state_init(g);
    for (int64_t st = 0; st < nsteps; ++st) {
      for (size_t c = 0; c < ncls; ++c) {
        cudaEvent_t* e = &ev[((size_t)st * ncls + c) * (kKinds + 1)];
        for (int k = 0; k < kKinds; ++k) {
          cudaEventRecord(e[k], g->stream);
          if (g->precision == SHF_FP64) launch_kind<double>(g, g->classes[c], k);
          else launch_kind<float>(g, g->classes[c], k);
        }
        cudaEventRecord(e[kKinds], g->stream);
      }
    }
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(g->stream);
    if (err != cudaSuccess) rc = fail(g, SHF_ECUDA, std::string("profiled step: ") + cudaGetErrorString(err));
    g->n += nsteps;
  }
  if (rc == SHF_OK) {
    for (int k = 0; k < nkinds; ++k) kernel_ms[k] = 0.0;
    for (size_t b = 0; b < (size_t)nsteps * ncls; ++b) {
      for (int k = 0; k < kKinds; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[b * (kKinds + 1) + k], ev[b * (kKinds + 1) + k + 1]);
        kernel_ms[k] += ms;
      }
    }
    for (int k = 0; k < kKinds; ++k) kernel_ms[k] /= (double)nsteps;
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}


int shf_autotune(shf_grid* g, const char* cache_path, int* choices, int nchoices) {
  if (!g || nchoices < 0 || (nchoices > 0 && !choices)) return fail(g, SHF_EINVAL, "bad autotune arguments");
  if (g->kind == 2) return fail(g, SHF_EINVAL, "tune the ensemble, not a member view");
  for (auto& m : g->members)
    if (!m.params_set) return fail(g, SHF_ESTATE, "shf_set_params must be called before shf_autotune");
  SHF_CUDA(g, cudaSetDevice(g->device));
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  std::map<std::string, Tune> cache = read_tune_cache(cache_path);
  bool changed = false;
  enqueue_state_init(g);                                // the stencils read the step's strain
  for (size_t c = 0; c < g->classes.size(); ++c) {
    SizeClass& cl = g->classes[c];
    const std::string key = tune_key(g, cl);
    Tune t;
    auto it = cache.find(key);
    if (it != cache.end()) {
      t = it->second;
    } else {
      const int rc = g->precision == SHF_FP64 ? tune_class<double>(g, cl, &t) : tune_class<float>(g, cl, &t);
      if (rc) return fail(g, rc, "autotune: a trial launch failed");
      cache[key] = t;
      changed = true;
    }
    configure_class(cl, g->precision, t);
    if (g->precision == SHF_FP64) t = resolved<double>(cl, t);
    else t = resolved<float>(cl, t);
    if ((int)(2 * c + 1) < nchoices) {
      choices[2 * c] = t.stage1_points;
      choices[2 * c + 1] = t.stage2_points;
    }
  }
  if (g->graph) {                                       // re-captured with the new launch shapes
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  if (cache_path && changed && !write_tune_cache(cache_path, cache))
    return fail(g, SHF_EIO, std::string("autotune: cannot write ") + cache_path);
  return SHF_OK;
}

int shf_sync(shf_grid* g) {
  if (!g) return SHF_EINVAL;
  shf_grid* o = owner(g);
  SHF_CUDA(g, cudaSetDevice(o->device));
  SHF_CUDA(g, cudaStreamSynchronize(o->stream));
  SHF_CUDA(g, cudaGetLastError());
  int err = 0;
  SHF_CUDA(g, cudaMemcpy(&err, o->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    SHF_CUDA(g, cudaMemset(o->d_err, 0, sizeof(int)));
    return fail(g, SHF_ETIMEOUT, "a kernel's bounded wait for its input copies gave up");
  }
  std::vector<int> which;
  if (g->kind == 1) {
    for (size_t r = 0; r < o->members.size(); ++r) which.push_back((int)r);
  } else {
    which.push_back(member_index(g));
  }
  for (int r : which) {
    double total, nf;
    const Member& m = o->members[r];
    int rc = o->precision == SHF_FP64 ? field_sum<double>(o, m, m.phi, &total, &nf)
                                      : field_sum<float>(o, m, m.phi, &total, &nf);
    if (rc) return fail(g, rc, o->err);
    if (nf > 0) return fail(g, SHF_ENONFINITE, "phi holds non-finite values");
  }
  return SHF_OK;
}


int shf_get_fields(shf_grid* g, double* phi, double* psi, double* omega) {
  if (!g) return SHF_EINVAL;
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view to read fields of an ensemble");
  SHF_CUDA(g, cudaSetDevice(owner(g)->device));
  return g->precision == SHF_FP64 ? get_fields_t<double>(g, phi, psi, omega)
                                  : get_fields_t<float>(g, phi, psi, omega);
}

int shf_get_time(shf_grid* g, int64_t* n, double* t, double* s, int64_t* wraps) {
  if (!g) return SHF_EINVAL;
  shf_grid* o = owner(g);
  const Member& m = g->kind == 1 ? o->members[0] : *member_of(g);
  double sv;
  long long K;
  host_strain(o->n, m.gdot, m.dt, m.nx / m.ny, &sv, &K);
  if (n) *n = o->n;
  if (t) *t = (double)o->n * m.dt;
  if (s) *s = sv;
  if (wraps) *wraps = K;
  return SHF_OK;
}

int shf_mass(shf_grid* g, double* mean_phi) {
  if (!g || !mean_phi) return SHF_EINVAL;
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view for the mass of an ensemble member");
  shf_grid* o = owner(g);
  SHF_CUDA(g, cudaSetDevice(o->device));
  const Member& m = *member_of(g);
  double total, nf;
  int rc = o->precision == SHF_FP64 ? field_sum<double>(o, m, m.phi, &total, &nf)
                                    : field_sum<float>(o, m, m.phi, &total, &nf);
  if (rc) return fail(g, rc, o->err);
  *mean_phi = total / ((double)m.nx * (double)m.ny);
  if (nf > 0) {
    *mean_phi = NAN;
    return fail(g, SHF_ENONFINITE, "phi holds non-finite values");
  }
  return SHF_OK;
}


int shf_structure_factor(shf_grid* g, double* S_binned, int nbins, double moments[5]) {
  if (!g || !moments || nbins < 0 || nbins > 4096 || (nbins > 0 && !S_binned))
    return fail(g, SHF_EINVAL, "bad structure factor arguments");
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view for an ensemble member");
  SHF_CUDA(g, cudaSetDevice(owner(g)->device));
  double sums[kSfMoments];
  const int rc = sf_sums(g, S_binned, nbins, sums);
  if (rc) return rc;
  const double S0 = sums[0], S1 = sums[1], Sm1 = sums[2];
  moments[0] = S0;
  moments[1] = S1;
  moments[2] = Sm1;
  moments[3] = S1 > 0 ? 6.283185307179586476925286766559 * S0 / S1 : NAN;
  moments[4] = S0 > 0 ? Sm1 / S0 : NAN;
  return SHF_OK;
}

int shf_gradient_tensor(shf_grid* g, double G[3], double lengths[2]) {
  if (!g || !G) return fail(g, SHF_EINVAL, "bad gradient tensor arguments");
  if (g->kind == 1) return fail(g, SHF_EINVAL, "use a member view for an ensemble member");
  SHF_CUDA(g, cudaSetDevice(owner(g)->device));
  double sums[kSfMoments];
  const int rc = sf_sums(g, nullptr, 0, sums);
  if (rc) return rc;
  const double den = sums[6];
  if (!(den > 0)) {
    G[0] = G[1] = G[2] = NAN;
    if (lengths) lengths[0] = lengths[1] = NAN;
    return fail(g, SHF_ESTATE, "phi is zero: the tensor is undefined");
  }
  G[0] = sums[3] / den;
  G[1] = sums[4] / den;
  G[2] = sums[5] / den;
  if (lengths) {
    const Member& m = *member_of(g);
    const double ell = std::sqrt(m.kappa / m.a);
    const double half_tr = 0.5 * (G[0] + G[2]), rad = std::hypot(0.5 * (G[0] - G[2]), G[1]);
    const double lam_min = half_tr - rad, lam_max = half_tr + rad;
    lengths[0] = lam_min > 0 ? 1.0 / (ell * lam_min) : INFINITY;
    lengths[1] = lam_max > 0 ? 1.0 / (ell * lam_max) : INFINITY;
  }
  return SHF_OK;
}

int shf_save(shf_grid* g, const char* path) {
  if (!g || !path || g->kind != 0) return fail(g, SHF_EINVAL, "save needs a single grid and a path");
  SHF_CUDA(g, cudaSetDevice(g->device));
  const Member& m = g->members[0];
  const size_t bytes = (size_t)m.nx * m.ny * real_size(g);
  // FP32 inertial grids carry omega's 2D transform from step to step; it is
  // saved too (when current), so that a resumed run continues bit for bit
  const bool with_what = g->precision == SHF_FP32 && m.rho > 0 && g->what_valid && m.w_hat;
  const int nblocks = with_what ? 4 : 3;
  std::vector<unsigned char> payload(nblocks * bytes);
  const void* src[4] = {m.phi, m.psi, m.omega, m.w_hat};
  for (int f = 0; f < nblocks; ++f)
    SHF_CUDA(g, cudaMemcpyAsync(payload.data() + f * bytes, src[f], bytes, cudaMemcpyDeviceToHost, g->stream));
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "SHFCKPT1", 8);
  h.version = 2;
  h.nx = m.nx;
  h.ny = m.ny;
  h.precision = g->precision;
  h.remap_mode = g->remap_mode;
  h.has_params = (m.params_set ? 1 : 0) | (with_what ? 2 : 0);
  const double pv[9] = {m.a, m.b, m.kappa, m.M, m.eta, m.rho, m.gdot, m.dt, m.dx};
  std::memcpy(h.params, pv, sizeof(pv));
  h.n = g->n;
  h.payload_crc = crc32_update(0, payload.data(), payload.size());
  h.header_crc = crc32_update(0, reinterpret_cast<const unsigned char*>(&h), offsetof(CkptHeader, header_crc));
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(g, SHF_EIO, std::string("cannot open ") + path);
  bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(payload.data(), 1, payload.size(), fp) == payload.size();
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(g, SHF_EIO, "write failed");
  return SHF_OK;
}

int shf_load(shf_grid* g, const char* path) {
  if (!g || !path || g->kind != 0) return fail(g, SHF_EINVAL, "load needs a single grid and a path");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(g, SHF_EIO, std::string("cannot open ") + path);
  CkptHeader h;
  const bool got = std::fread(&h, sizeof(h), 1, fp) == 1;
  Member& m = g->members[0];
  const size_t bytes = (size_t)m.nx * m.ny * real_size(g);
  bool ok = got && std::memcmp(h.magic, "SHFCKPT1", 8) == 0 && (h.version == 1 || h.version == 2) &&
            h.header_crc == crc32_update(0, reinterpret_cast<const unsigned char*>(&h), offsetof(CkptHeader, header_crc));
  const bool with_what = ok && h.version == 2 && (h.has_params & 2) && g->precision == SHF_FP32 && m.w_hat;
  std::vector<unsigned char> payload((with_what ? 4 : 3) * bytes);
  if (ok && (h.nx != m.nx || h.ny != m.ny || h.precision != g->precision)) {
    std::fclose(fp);
    return fail(g, SHF_EINVAL, "checkpoint was written for another grid size or precision");
  }
  if (ok && h.params[8] != m.dx) {                     // the mesh spacing is fixed at creation
    std::fclose(fp);
    return fail(g, SHF_EINVAL, "checkpoint was written for another mesh spacing dx");
  }
  ok = ok && std::fread(payload.data(), 1, payload.size(), fp) == payload.size();
  unsigned char extra;
  ok = ok && std::fread(&extra, 1, 1, fp) == 0;
  std::fclose(fp);
  if (!ok || h.payload_crc != crc32_update(0, payload.data(), payload.size()))
    return fail(g, SHF_EIO, "checkpoint truncated or corrupt");
  SHF_CUDA(g, cudaSetDevice(g->device));
  void* dst[4] = {m.phi, m.psi, m.omega, m.w_hat};
  for (int f = 0; f < (with_what ? 4 : 3); ++f)
    SHF_CUDA(g, cudaMemcpyAsync(dst[f], payload.data() + f * bytes, bytes, cudaMemcpyHostToDevice, g->stream));
  SHF_CUDA(g, cudaStreamSynchronize(g->stream));
  g->remap_mode = h.remap_mode;
  if (h.has_params & 1) {
    const double* p = h.params;
    m.a = p[0]; m.b = p[1]; m.kappa = p[2]; m.M = p[3]; m.eta = p[4]; m.rho = p[5]; m.gdot = p[6]; m.dt = p[7];
    m.params_set = true;
  }
  int rc = upload_desc(g, 0);
  if (!rc) rc = drop_graph(g);                           // the parameters may have changed regime
  if (rc) return rc;
  rc = shf_set_step(g, h.n);
  // omega's 2D transform: restored from the file, or recomputed from omega at the next step
  g->what_valid = with_what && m.rho > 0;
  return rc;
}

}  // extern "C"
