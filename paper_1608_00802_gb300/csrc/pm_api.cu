// Host side of the C ABI declared in include/pm.h: arena layout, cuFFT plans,
// leapfrog weights and the order of the stages of one step
// (Veltmaat & Niemeyer, arXiv:1608.00802, Sec. II.A: (i) density, (ii) Q on
// the grid, (iii) force on each particle, inside a kick-drift-kick leapfrog).
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/pm.h"
#include "pm_internal.h"

using namespace pm;

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------- units
// hbar/m in (Mpc/h)^2 H0: (hbar c) c / (m c^2), with one code unit of
// length^2/time = (100/h) Mpc km/s.  CODATA 2018 hbar*c, IAU parsec.
double hbar_over_m(double m22, double h) {
  const double hbarc_ev_m = 1.973269804e-7, c = 299792458.0, mpc = 3.0856775814913673e22;
  double si = hbarc_ev_m * c / (m22 * 1e-22);  // m^2/s
  return si / (mpc * 1e3) / (100.0 / h);
}

// ---------------------------------------------------------------- quadrature
// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n.
struct GaussLegendre {
  static const int N = 32;
  double x[N], w[N];
  GaussLegendre() {
    for (int i = 0; i < (N + 1) / 2; ++i) {
      double z = cos(M_PI * (i + 0.75) / (N + 0.5)), pp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= N; ++j) {
          double p3 = p2;
          p2 = p1;
          p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = N * (z * p1 - p2) / (z * z - 1.0);
        double dz = p1 / pp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
      }
      x[i] = -z;
      x[N - 1 - i] = z;
      w[i] = w[N - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
  }
};
const GaussLegendre& gl() {
  static GaussLegendre g;
  return g;
}

struct Weights {
  double kg;  // int da / (a^2 H): kick weight of -grad(phi~)  (comoving dp/dt = -grad phi~ / a)
  double kq;  // int da / (a^3 H): kick weight of -grad(Q~) and drift weight (dx/dt = p / a^2)
};

Weights time_weights(const pm_config& c, double a0, double a1) {
  if (!c.cosmological) return {a1 - a0, a1 - a0};
  const GaussLegendre& g = gl();
  double mid = 0.5 * (a0 + a1), half = 0.5 * (a1 - a0), kg = 0.0, kq = 0.0;
  for (int i = 0; i < GaussLegendre::N; ++i) {
    double a = mid + half * g.x[i];
    double hub = sqrt(c.omega_m / (a * a * a) + c.omega_l);
    kg += g.w[i] / (a * a * hub);
    kq += g.w[i] / (a * a * a * hub);
  }
  return {kg * half, kq * half};
}

double half_point(const pm_config& c, double a0, double a1) {
  return c.cosmological ? sqrt(a0 * a1) : 0.5 * (a0 + a1);
}

// ---------------------------------------------------------------- layout
size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
  size_t pos[2], mom[2], keys[4], vals[3], tcount, rcnt, btot, srow, mrow, tile_cnt, row_start, rho, phi, q, spec, what,
      spec2, work, staging, hist, status, st_list, st_count, part, part_aux, red, err, ktab, green, total;
  int key_bits, passes, digit_bits, ntiles;
};

bool valid_config(const pm_config* c, std::string* why) {
  if (!c) {
    *why = "null configuration";
    return false;
  }
  if (c->n_part < 1 || c->n_part > 0x7fffffffLL) {
    *why = "n_part must be in [1, 2^31-1]";
    return false;
  }
  if (c->n_mesh < 8 || c->n_mesh > 1024 || (c->n_mesh & 1)) {
    *why = "n_mesh must be even and in [8, 1024]";
    return false;
  }
  if (c->precision != PM_FP32 && c->precision != PM_FP64) {
    *why = "precision must be PM_FP32 or PM_FP64";
    return false;
  }
  if (!(c->box > 0) || !isfinite(c->box)) {
    *why = "box must be positive";
    return false;
  }
  if (c->force_mode < 0 || c->force_mode > 2 || (c->lap != 0 && c->lap != 1)) {
    *why = "force_mode or lap out of range";
    return false;
  }
  if (c->quantum && (!(c->m22 > 0) || !(c->h > 0))) {
    *why = "m22 and h must be positive with quantum pressure on";
    return false;
  }
  if (c->cosmological && (!(c->omega_m >= 0) || !(c->omega_m + c->omega_l > 0))) {
    *why = "cosmological run needs omega_m >= 0 and omega_m + omega_l > 0";
    return false;
  }
  if (!(c->rho_floor > 0) || (c->precision == PM_FP32 && !(c->rho_floor >= 1e-30))) {
    *why = "rho_floor must be positive (at least 1e-30 with PM_FP32: a normal fp32 number)";
    return false;
  }
  if (c->fft_jit != 0 && c->fft_jit != 1) {
    *why = "fft_jit must be 0 or 1";
    return false;
  }
  if (c->kernel != PM_KERNEL_CIC && c->kernel != PM_KERNEL_SPLINE) {
    *why = "kernel must be PM_KERNEL_CIC or PM_KERNEL_SPLINE";
    return false;
  }
  if (c->kernel == PM_KERNEL_SPLINE && !(c->smooth_h >= 1.0 && c->smooth_h <= 0.25 * c->n_mesh)) {
    *why = "smooth_h must be in [1, n_mesh/4] mesh cells";
    return false;
  }
  // real-space smoothing: fp32, support within three cells, one block of n_mesh threads per mesh row
  if (c->smooth_real != 0 && (c->smooth_real != 1 || c->kernel != PM_KERNEL_SPLINE || c->precision != PM_FP32 ||
                              !(c->smooth_h <= 4.0) || c->n_mesh > 512)) {
    *why = "smooth_real needs the spline kernel, PM_FP32, smooth_h <= 4 and n_mesh <= 512";
    return false;
  }
  return true;
}

// digit histograms and tile counters of a sort
constexpr size_t hist_bytes() { return (3 * (size_t(1) << RS_MAX_BITS) + 4) * 4; }

Layout make_layout(const pm_config& c, size_t work_bytes) {
  Layout L;
  const size_t n = size_t(c.n_part), N = size_t(c.n_mesh), n3 = N * N * N;
  const size_t rsz = c.precision == PM_FP64 ? 8 : 4;
  const size_t recsz = 4 * rsz;
  int bits = 0;
  while ((size_t(1) << bits) < n3) ++bits;
  L.key_bits = bits;
  L.passes = (bits + RS_MAX_BITS - 1) / RS_MAX_BITS;
  if (L.passes < 1) L.passes = 1;
  L.digit_bits = (bits + L.passes - 1) / L.passes;
  L.ntiles = int((n + RS_TILE - 1) / RS_TILE);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  for (int k = 0; k < 2; ++k) L.pos[k] = take(n * recsz);
  for (int k = 0; k < 2; ++k) L.mom[k] = take(n * recsz);
  for (int k = 0; k < 4; ++k) L.keys[k] = take(n * 4);
  for (int k = 0; k < 3; ++k) L.vals[k] = take(n * 4);
  L.tcount = take(size_t(mover_count_words(int64_t(n))) * 8);  // movers per tile, movers before each tile
  // re-sort: stayers, movers and bucket fill per mesh row; the row scan's tile totals; stayers and movers
  // before each row
  L.rcnt = take(3 * N * N * 4);
  L.btot = take(2 * row_scan_tiles(int(N)) * 4);
  L.srow = take((N * N + 1) * 4);
  L.mrow = take((N * N + 1) * 4);
  L.tile_cnt = take(16);  // (stayers, movers) of the last re-sort
  L.row_start = take((N * N + 1) * 4);
  L.rho = take(n3 * rsz);
  L.phi = take(n3 * rsz);
  L.q = take(n3 * rsz);
  L.spec = take(N * N * (N / 2 + 1) * 2 * rsz);
  // spline kernel: its real symbol over the half spectrum and a second spectrum
  const bool spline = c.kernel == PM_KERNEL_SPLINE;
  L.what = take(spline ? N * N * (N / 2 + 1) * rsz : 0);
  L.spec2 = take(spline ? N * N * (N / 2 + 1) * 2 * rsz : 0);
  L.work = take(work_bytes);
  size_t stage = 6 * n * 8;
  if (n3 * 8 > stage) stage = n3 * 8;
  L.staging = take(stage);
  // digit histograms of all passes (radix_max stride), one tile counter per pass
  L.hist = take(hist_bytes());
  L.status = take((size_t(1) << L.digit_bits) * size_t(L.ntiles) * 8);
  size_t nkb = size_t(kick_blocks(int64_t(n), KICK_MIN_THREADS));
  size_t npart = 4 * nkb;
  if (size_t(RED_GRID) * 3 * PK_MAX_BINS > npart) npart = size_t(RED_GRID) * 3 * PK_MAX_BINS;
  L.part = take(npart * 8);
  L.st_list = take(c.precision == PM_FP32 ? stencil_list_entries(int(N)) * 4 : 4);
  L.st_count = take(size_t(stencil_max_blocks(int(N))) * 4);
  size_t aux = std::max<size_t>(MESH_GRID, size_t(stencil_max_blocks(int(N))));
  if (spec_z_supported(int(N))) aux = std::max<size_t>(aux, size_t(spec_z_tiles(int(N))));
  L.part_aux = take(2 * aux * 8);
  L.red = take(3 * PK_MAX_BINS * 8 + 64);
  L.err = take(256);
  // per-step kick weights of pm_run and of a batch run
  L.ktab = take(size_t(std::max(PM_RUN_GRAPH_MAX_STEPS, PM_BATCH_MAX_STEPS)) * sizeof(KickParams));
  // the z transform's twiddles and the Green's sin^2 table (fp32 cloud-in-cell, power-of-two meshes)
  L.green = take(c.precision == PM_FP32 && !spline && spec_z_supported(int(N)) ? N * 12 : 0);
  L.total = off;
  return L;
}

bool fft_work_bytes(const pm_config& c, size_t* out, std::string* why) {
  cufftType fwd = c.precision == PM_FP64 ? CUFFT_D2Z : CUFFT_R2C;
  cufftType inv = c.precision == PM_FP64 ? CUFFT_Z2D : CUFFT_C2R;
  size_t ws[2] = {0, 0};
  cufftType types[2] = {fwd, inv};
  for (int k = 0; k < 2; ++k) {
    cufftHandle h;
    if (cufftCreate(&h) != CUFFT_SUCCESS) {
      *why = "cufftCreate failed";
      return false;
    }
    cufftSetAutoAllocation(h, 0);
    if (c.fft_jit) cufftSetPlanPropertyInt64(h, NVFFT_PLAN_PROPERTY_INT64_PATIENT_JIT, 1);
    cufftResult r = cufftMakePlan3d(h, c.n_mesh, c.n_mesh, c.n_mesh, types[k], &ws[k]);
    cufftDestroy(h);
    if (r != CUFFT_SUCCESS) {
      *why = "cufftMakePlan3d failed (" + std::to_string(int(r)) + ")";
      return false;
    }
  }
  *out = ws[0] > ws[1] ? ws[0] : ws[1];
  return true;
}

}  // namespace

void pm::set_global_error(const char* msg) { g_create_error = msg; }

// ---------------------------------------------------------------- the handle
struct pm_sim {
  pm_config cfg;
  cudaStream_t stream;
  char* arena;
  Layout L;
  Mesh mesh;
  double dx, hbm, norm;
  int cur;  // which of pos[2]/mom[2] holds the state
  uint32_t* keys;  // sorted (current) keys
  uint32_t* keys_tmp[2];
  bool keys_marked = false;  // a drift has flagged the movers in `keys` since the last sort
  Tuning tune;                // launch shapes
  // spline kernel smoothed in real space (fp32, support within three cells):
  // the smoothed density lives in the spec2 region, and `rho` holds the
  // unsmoothed Q~ between the stencil and its smoothing
  bool direct = false;
  double taps[19 * 4];
  int taps_r2 = 27;  // largest squared offset with a nonzero weight
  int sms = 152;              // multiprocessors of the device
  bool krho_valid = false;    // the K_rho partials belong to the current Q~
  cufftHandle plan_fwd, plan_inv;
  // fp32 cloud-in-cell, power-of-two mesh: batched 2D transforms of the z planes, between which
  // one kernel does the z transforms and the Green multiplication
  cufftHandle plan2_fwd = 0, plan2_inv = 0;
  bool have_plan2 = false;
  int wg_count = MESH_GRID;  // W_g partials the last force evaluation wrote
  bool have_particles, sorted, fields_valid;
  std::string err;
  // profiler: event pairs around launches while enabled
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_stage;
  size_t prof_used = 0;
  // pm_run replays captured steps on its own stream, joined to `stream` by events
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // pinned staging of the kick table (a pageable source would serialise the
  // host with this stream); ev_tab marks the end of the last upload
  KickParams* tab_host = nullptr;
  cudaEvent_t ev_tab = nullptr;
  bool tab_pending = false;
  // captured two-step graphs, one per entry state of the record buffers
  // (cur, sorted-key buffer); every pointer they hold is fixed for the
  // simulation's lifetime, so they are kept until pm_destroy
  struct RunGraph {
    int cur = -1;
    const uint32_t* keys = nullptr;
    cudaGraphExec_t exec = nullptr;
  } run_graph[2];

  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(arena + off);
  }
  void* pos() const { return arena + L.pos[cur]; }
  void* mom() const { return arena + L.mom[cur]; }
  bool fp64() const { return cfg.precision == PM_FP64; }
  int64_t n() const { return cfg.n_part; }
  // err region: [0] error bits, [1] sort epoch, [2] device step counter; at byte 64 two
  // 64-bit counters of the incremental re-sorts and of the particles they moved
  uint32_t* errword() const { return at<uint32_t>(L.err); }
  unsigned long long* sort_stats() const { return reinterpret_cast<unsigned long long*>(arena + L.err + 64); }
  // at byte 128 the Green and quantum-pressure coefficients of this simulation
  // (doubles, written at creation), read by the launches that step a packed
  // group of simulations whose boxes and masses differ
  double* coefs() const { return reinterpret_cast<double*>(arena + L.err + 128); }
  double* part() const { return at<double>(L.part); }
  double* red() const { return at<double>(L.red); }
  double* staging() const { return at<double>(L.staging); }
};

namespace {

pm_status fail(pm_sim* s, pm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s)
    s->err = buf;
  else
    g_create_error = buf;
  return st;
}

// Records an event pair around one launch when the profiler is on.
struct ProfScope {
  pm_sim* s;
  size_t slot;
  ProfScope(pm_sim* sim, int stage) : s(sim), slot(size_t(-1)) {
    if (s->prof_on && 2 * (s->prof_used + 1) <= s->prof_ev.size()) {
      slot = s->prof_used++;
      s->prof_stage[slot] = stage;
      cudaEventRecord(s->prof_ev[2 * slot], s->stream);
    }
  }
  ~ProfScope() {
    if (slot != size_t(-1)) cudaEventRecord(s->prof_ev[2 * slot + 1], s->stream);
  }
};
#define PROF(sim, stage) ProfScope prof_scope_##__LINE__(sim, stage)

#define CU(sim, expr)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) return fail(sim, PM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)
#define CF(sim, expr)                                                                      \
  do {                                                                                     \
    cufftResult r_ = (expr);                                                               \
    if (r_ != CUFFT_SUCCESS) return fail(sim, PM_ERR_CUFFT, "%s: cufft error %d", #expr, int(r_)); \
  } while (0)

// Partials: the kick diagnostics and the power spectrum use `part`; the
// gravity-energy and K_rho sums of the last force evaluation live in
// `part_aux` (one MESH_GRID-long row each) until the next evaluation.
double* wg_part(pm_sim* s) { return s->at<double>(s->L.part_aux); }
size_t aux_len(const pm_sim* s) {
  const int N = s->cfg.n_mesh;
  size_t aux = std::max<size_t>(MESH_GRID, size_t(stencil_max_blocks(N)));
  if (spec_z_supported(N)) aux = std::max<size_t>(aux, size_t(spec_z_tiles(N)));
  return aux;
}
double* kr_part(pm_sim* s) { return wg_part(s) + aux_len(s); }
int kr_blocks(const pm_sim* s) {
  const bool tiled = !s->fp64() && s->cfg.lap == PM_LAP_COMPACT;
  return tiled ? stencil_launch_blocks(s->cfg.n_mesh, s->tune.st_ty, s->tune.st_zlen) : MESH_GRID;
}

// Incremental re-sort after a drift: the stayers are still in order, so every
// particle's place follows from the stayers and movers of its mesh row (stable
// partition with per-row counts, a scan of the rows, the movers in per-row
// buckets, the placement of each particle with its records into the other
// buffer; see pm_sort.cuh).  Same order as the full sort; also writes the row
// starts.
template <typename R>
pm_status resort_movers(pm_sim* s) {
  const Layout& L = s->L;
  const int N = s->cfg.n_mesh;
  const int nxt = s->cur ^ 1;
  CU(s, cudaMemsetAsync(s->at<uint32_t>(L.rcnt), 0, size_t(3) * N * N * 4, s->stream));
  const int stages[3] = {PM_STAGE_SORT_PARTITION, PM_STAGE_SORT_PASS, PM_STAGE_SORT_MERGE};
  for (int part = 0; part < 3; ++part) {
    PROF(s, stages[part]);
    CU(s, launch_resort<R>(part, s->keys, s->n(), s->at<uint32_t>(L.tcount), s->keys_tmp[0],
                           s->at<uint32_t>(L.vals[0]), s->keys_tmp[1], s->at<uint32_t>(L.vals[1]),
                           s->at<uint32_t>(L.keys[3]), s->at<uint32_t>(L.vals[2]), s->at<uint32_t>(L.tile_cnt),
                           s->at<uint32_t>(L.rcnt), s->at<uint32_t>(L.btot), s->at<uint32_t>(L.srow),
                           s->at<uint32_t>(L.mrow), s->at<uint32_t>(L.row_start), s->mesh, s->sort_stats(), s->keys,
                           s->pos(), s->mom(), s->arena + L.pos[nxt], s->arena + L.mom[nxt], s->sms, s->stream));
  }
  s->cur = nxt;
  s->keys_marked = false;
  s->sorted = true;
  return PM_OK;
}

template <typename R>
pm_status sort_particles(pm_sim* s) {
  if (s->keys_marked) return resort_movers<R>(s);
  const Layout& L = s->L;
  const int64_t n = s->n();
  uint32_t* hist = s->at<uint32_t>(L.hist);
  uint32_t* counters = hist + 3 * (1 << RS_MAX_BITS);
  uint64_t* status = s->at<uint64_t>(L.status);
  uint32_t* vals[2] = {s->at<uint32_t>(L.vals[0]), s->at<uint32_t>(L.vals[1])};
  CU(s, cudaMemsetAsync(hist, 0, hist_bytes(), s->stream));
  {
    PROF(s, PM_STAGE_SORT_HISTOGRAM);
    CU(s, launch_sort_histogram(s->keys, n, L.passes, L.digit_bits, L.key_bits, hist, s->errword() + 1, s->stream));
  }
  const uint32_t* kin = s->keys;
  const uint32_t* vin = nullptr;
  int tmp = 0;
  for (int p = 0; p < L.passes; ++p) {
    const int shift = p * L.digit_bits;
    const int bits = (shift + L.digit_bits <= L.key_bits) ? L.digit_bits : (L.key_bits - shift);
    const bool last = p == L.passes - 1;
    const uint32_t* dtot = hist + p * (1 << RS_MAX_BITS);
    PROF(s, PM_STAGE_SORT_PASS);
    if (!last) {
      uint32_t* kout = s->keys_tmp[tmp];
      uint32_t* vout = vals[tmp];
      CU(s, launch_sort_pass<R>(false, kin, vin, n, shift, bits, dtot, status, counters + p, s->errword() + 1, p,
                                L.ntiles, kout, vout, nullptr, nullptr, nullptr, nullptr, s->errword(), s->stream));
      kin = kout;
      vin = vout;
      tmp ^= 1;
    } else {
      // the sorted keys go to a buffer that is not the input
      uint32_t* kout = (kin == s->keys) ? s->keys_tmp[tmp] : s->keys;
      const int nxt = s->cur ^ 1;
      CU(s, launch_sort_pass<R>(true, kin, vin, n, shift, bits, dtot, status, counters + p, s->errword() + 1, p,
                                L.ntiles, kout, nullptr, s->pos(), s->mom(), s->arena + L.pos[nxt],
                                s->arena + L.mom[nxt], s->errword(), s->stream));
      if (kout != s->keys) {  // swap roles so that s->keys holds the sorted keys
        for (int k = 0; k < 2; ++k)
          if (s->keys_tmp[k] == kout) s->keys_tmp[k] = s->keys;
        s->keys = kout;
      }
      s->cur = nxt;
    }
  }
  {
    PROF(s, PM_STAGE_ROW_START);
    CU(s, launch_row_start(s->keys, n, uint32_t(s->cfg.n_mesh), s->at<uint32_t>(L.row_start), s->stream));
  }
  s->sorted = true;
  return PM_OK;
}

// where the density the stencil and the Poisson solve read lives: `rho`, or
// with the real-space spline smoothing the smoothed copy in the spec2 region
size_t density_field(const pm_sim* s) { return s->direct ? s->L.spec2 : s->L.rho; }

StencilParams stencil_params(const pm_sim* s, bool diag) {
  StencilParams sp;
  sp.step = s->cfg.lap == PM_LAP_WIDE ? 2 : 1;
  sp.rho_floor = s->cfg.rho_floor;
  sp.rho_fp64 = s->cfg.rho_fp64;
  sp.qcoef = -0.5 * s->hbm * s->hbm / ((sp.step * s->dx) * (sp.step * s->dx));
  sp.ty = s->tune.st_ty;
  sp.zlen = s->tune.st_zlen;
  sp.stages = s->tune.st_stages;
  sp.diag = diag ? 1 : 0;
  return sp;
}

// Q~ (and the K_rho partials) from the density on the mesh
template <typename R>
pm_status stencil_stage(pm_sim* s, bool diag = false) {
  const Layout& L = s->L;
  const StencilParams sp = stencil_params(s, diag);
  s->krho_valid = diag || s->fp64() || s->cfg.lap != PM_LAP_COMPACT;  // the generic kernel always sums
  PROF(s, PM_STAGE_STENCIL);
  CU(s, launch_stencil<R>(s->at<R>(density_field(s)), s->mesh, sp, s->at<R>(s->direct ? L.rho : L.q), kr_part(s),
                          s->at<uint32_t>(L.st_list), s->at<uint32_t>(L.st_count), s->errword(), s->stream));
  return PM_OK;
}

// forward and inverse transforms between a real mesh field and a spectrum
template <typename R>
pm_status fft_r2c(pm_sim* s, void* in, void* out) {
  PROF(s, PM_STAGE_FFT_R2C);
  if (s->fp64()) {
    CF(s, cufftExecD2Z(s->plan_fwd, (cufftDoubleReal*)in, (cufftDoubleComplex*)out));
  } else {
    CF(s, cufftExecR2C(s->plan_fwd, (cufftReal*)in, (cufftComplex*)out));
  }
  return PM_OK;
}

template <typename R>
pm_status fft_c2r(pm_sim* s, void* in, void* out) {
  PROF(s, PM_STAGE_FFT_C2R);
  if (s->fp64()) {
    CF(s, cufftExecZ2D(s->plan_inv, (cufftDoubleComplex*)in, (cufftDoubleReal*)out));
  } else {
    CF(s, cufftExecC2R(s->plan_inv, (cufftComplex*)in, (cufftReal*)out));
  }
  return PM_OK;
}

#define PMST(expr)                  \
  do {                              \
    pm_status st_ = (expr);         \
    if (st_ != PM_OK) return st_;   \
  } while (0)

bool spline(const pm_sim* s) { return s->cfg.kernel == PM_KERNEL_SPLINE; }

// the normalised node weights of the spline at squared distance i^2 + s (in
// cells, s = j^2 + k^2 <= 18, i <= 3) for the real-space smoothing: W(r, h)
// of Sec. II.A up to its constant, divided by its sum over the nodes
void spline_taps(double hc, double* g) {
  auto f = [&](int r2) {
    const double u = sqrt(double(r2)) / hc;
    return u <= 0.5 ? 1.0 - 6.0 * u * u + 6.0 * u * u * u : (u <= 1.0 ? 2.0 * (1.0 - u) * (1.0 - u) * (1.0 - u) : 0.0);
  };
  double sum = 0.0;
  for (int i = -3; i <= 3; ++i)
    for (int j = -3; j <= 3; ++j)
      for (int k = -3; k <= 3; ++k) sum += f(i * i + j * j + k * k);
  for (int q = 0; q < 19; ++q)
    for (int i = 0; i < 4; ++i) g[q * 4 + i] = f(i * i + q) / sum;
}

// a mesh field convolved with the spline's node weights, from `in` to `out`
// (the same offset for the spectral smoothing, which works in place)
template <typename R>
pm_status smooth_field(pm_sim* s, size_t in, size_t out) {
  if (s->direct) {
    PROF(s, PM_STAGE_GREEN);
    CU(s, launch_smooth_direct<float>(s->at<float>(in), s->at<float>(out), s->mesh, s->taps, s->taps_r2, s->stream));
    return PM_OK;
  }
  PMST(fft_r2c<R>(s, s->arena + in, s->arena + s->L.spec));
  {
    PROF(s, PM_STAGE_GREEN);
    CU(s, launch_smooth_spec<R>(s->arena + s->L.spec, s->arena + s->L.what, s->mesh, s->stream));
  }
  return fft_c2r<R>(s, s->arena + s->L.spec, s->arena + out);
}

double green_coef(const pm_sim* s) {
  const double N = s->cfg.n_mesh;
  return -1.5 * s->cfg.omega_m * s->dx * s->dx / (4.0 * N * N * N);
}

// the Green multiplication inside the z transform, between batched 2D transforms
bool green_fused(const pm_sim* s) { return s->tune.green_fused && s->have_plan2; }

// The batched 2D transforms of the N z planes (forward: the real density to
// the (ky, kx) half planes; inverse: back to the real potential), sharing the
// work area of the 3D plans, and the z kernel's tables.  Sync.
cufftResult spec_plan_setup(pm_sim* s, std::string* why) {
  if (s->have_plan2) return CUFFT_SUCCESS;
  const int N = s->cfg.n_mesh;
  if (s->fp64() || spline(s) || !spec_z_supported(N)) {
    *why = "not an fp32 cloud-in-cell simulation on a power-of-two mesh of 16..512";
    return CUFFT_NOT_SUPPORTED;
  }
  const Layout& L = s->L;
  cudaError_t ce = launch_spec_tables(s->at<float2>(L.green), s->at<float>(L.green + size_t(N) * 8), N, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) {
    *why = std::string("tables: ") + cudaGetErrorString(ce);
    return CUFFT_SETUP_FAILED;
  }
  cufftHandle h[2] = {0, 0};
  const char* step = "cufftCreate";
  cufftResult r = CUFFT_SUCCESS;
  const long long nh = N / 2 + 1;
  for (int k = 0; k < 2 && r == CUFFT_SUCCESS; ++k) {
    long long n[2] = {N, N}, re[2] = {N, N}, cx[2] = {N, nh};
    size_t w = 0;
    step = "cufftCreate";
    r = cufftCreate(&h[k]);
    if (r == CUFFT_SUCCESS) r = cufftSetAutoAllocation(h[k], 0);
    if (r == CUFFT_SUCCESS && s->cfg.fft_jit)
      r = cufftSetPlanPropertyInt64(h[k], NVFFT_PLAN_PROPERTY_INT64_PATIENT_JIT, 1);
    if (r == CUFFT_SUCCESS) {
      step = "cufftMakePlanMany64";
      r = k == 0 ? cufftMakePlanMany64(h[k], 2, n, re, 1, (long long)N * N, cx, 1, (long long)N * nh, CUFFT_R2C, N, &w)
                 : cufftMakePlanMany64(h[k], 2, n, cx, 1, (long long)N * nh, re, 1, (long long)N * N, CUFFT_C2R, N, &w);
    }
    if (r == CUFFT_SUCCESS && w > L.staging - L.work) {  // the 3D plans' area
      step = "work area";
      r = CUFFT_NO_WORKSPACE;
    }
    if (r == CUFFT_SUCCESS) r = cufftSetWorkArea(h[k], s->arena + L.work);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(h[k], s->stream);
  }
  if (r != CUFFT_SUCCESS) {
    *why = step;
    for (cufftHandle x : h)
      if (x) cufftDestroy(x);
    return r;
  }
  s->plan2_fwd = h[0];
  s->plan2_inv = h[1];
  s->have_plan2 = true;
  return CUFFT_SUCCESS;
}

// Q~ from the density, smoothed with the spline kernel (the transpose of the
// density's smoothing); diag: with the K_rho partials.  In real space the
// stencil writes the raw Q~ to `rho` and the smoothing moves it to `q`.
template <typename R>
pm_status quantum_stage(pm_sim* s, bool diag = false) {
  if (!s->cfg.quantum) return PM_OK;
  PMST(stencil_stage<R>(s, diag));
  if (s->direct)
    PMST(smooth_field<R>(s, s->L.rho, s->L.q));
  else if (spline(s))
    PMST(smooth_field<R>(s, s->L.q, s->L.q));
  return PM_OK;
}

// the K_rho partials of the current density (the steps skip them): Q~ again
// with the sums, and, with the spline kernel, smoothed again as the step
// smoothed it, so that the field the next kick reads is the same
template <typename R>
pm_status krho_stage(pm_sim* s) {
  return quantum_stage<R>(s, true);
}

// phi~ and Q~ from the density (cloud-in-cell kernel: the deposit; spline
// kernel: the already smoothed density, whose force potential is smoothed
// once more)
template <typename R>
pm_status mesh_from_density(pm_sim* s) {
  const Layout& L = s->L;
  if (green_fused(s)) {  // 2D transforms of the planes; z transforms and Green in one pass between them
    const int N = s->cfg.n_mesh;
    {
      PROF(s, PM_STAGE_FFT_R2C);
      if (s->tune.green_fused == 2)
        CU(s, launch_xy_r2c(s->at<float>(L.rho), s->arena + L.spec, s->at<float2>(L.green), N, s->stream));
      else
        CF(s, cufftExecR2C(s->plan2_fwd, s->at<cufftReal>(L.rho), (cufftComplex*)(s->arena + L.spec)));
    }
    {
      PROF(s, PM_STAGE_GREEN);
      CU(s, launch_spec_z(s->arena + L.spec, s->at<float2>(L.green), s->at<float>(L.green + size_t(N) * 8), s->mesh,
                          green_coef(s), wg_part(s), s->stream));
    }
    s->wg_count = spec_z_tiles(N);
    {
      PROF(s, PM_STAGE_FFT_C2R);
      if (s->tune.green_fused == 2)
        CU(s, launch_xy_c2r(s->arena + L.spec, s->at<float>(L.phi), s->at<float2>(L.green), N, s->stream));
      else
        CF(s, cufftExecC2R(s->plan2_inv, (cufftComplex*)(s->arena + L.spec), s->at<cufftReal>(L.phi)));
    }
    PMST(quantum_stage<R>(s));
    s->fields_valid = true;
    return PM_OK;
  }
  PMST(fft_r2c<R>(s, s->arena + density_field(s), s->arena + L.spec));
  {
    PROF(s, PM_STAGE_GREEN);
    if (spline(s))
      CU(s, launch_green_spline<R>(s->arena + L.spec, nullptr, s->arena + L.what, s->mesh, green_coef(s), wg_part(s),
                                   s->stream, 0));
    else
      CU(s, launch_green<R>(s->arena + L.spec, s->mesh, green_coef(s), wg_part(s), s->stream));
  }
  s->wg_count = MESH_GRID;
  PMST(fft_c2r<R>(s, s->arena + L.spec, s->arena + L.phi));
  PMST(quantum_stage<R>(s));
  s->fields_valid = true;
  return PM_OK;
}

// spline kernel from the cloud-in-cell density in `rho`: one forward transform
// gives the force potential and (spectral smoothing) the smoothed density
// back into `rho`; the real-space smoothing writes the smoothed density to the
// spec2 region instead
template <typename R>
pm_status spline_fields(pm_sim* s) {
  const Layout& L = s->L;
  PMST(fft_r2c<R>(s, s->arena + L.rho, s->arena + L.spec));
  {
    PROF(s, PM_STAGE_GREEN);
    CU(s, launch_green_spline<R>(s->arena + L.spec, s->direct ? nullptr : s->arena + L.spec2, s->arena + L.what,
                                 s->mesh, green_coef(s), wg_part(s), s->stream, 1));
  }
  s->wg_count = MESH_GRID;
  if (s->direct)
    PMST(smooth_field<R>(s, L.rho, L.spec2));
  else
    PMST(fft_c2r<R>(s, s->arena + L.spec2, s->arena + L.rho));
  PMST(fft_c2r<R>(s, s->arena + L.spec, s->arena + L.phi));
  PMST(quantum_stage<R>(s));
  s->fields_valid = true;
  return PM_OK;
}

// the normalised symbol of the spline's node weights (once, at creation)
template <typename R>
pm_status spline_symbol(pm_sim* s) {
  const Layout& L = s->L;
  CU(s, launch_spline_weights<R>(s->arena + L.rho, s->mesh, s->cfg.smooth_h, s->stream));
  PMST(fft_r2c<R>(s, s->arena + L.rho, s->arena + L.spec));
  CU(s, launch_spline_symbol<R>(s->arena + L.spec, s->arena + L.what, s->mesh, s->stream));
  return PM_OK;
}

template <typename R>
pm_status deposit(pm_sim* s) {
  if (!s->sorted) {
    pm_status st = sort_particles<R>(s);
    if (st != PM_OK) return st;
  }
  PROF(s, PM_STAGE_DEPOSIT);
  CU(s, launch_deposit<R>(s->pos(), s->at<uint32_t>(s->L.row_start), s->n(), s->mesh, s->norm, s->at<R>(s->L.rho),
                          s->stream, s->tune.dep_warps));
  return PM_OK;
}

template <typename R>
pm_status compute_fields(pm_sim* s) {
  pm_status st = deposit<R>(s);
  if (st != PM_OK) return st;
  return spline(s) ? spline_fields<R>(s) : mesh_from_density<R>(s);
}

// the density of Eq. (rhodis) in density_field (fields left invalid)
template <typename R>
pm_status density(pm_sim* s) {
  PMST(deposit<R>(s));
  if (spline(s)) PMST(smooth_field<R>(s, s->L.rho, density_field(s)));
  s->fields_valid = false;
  return PM_OK;
}

KickParams base_kick(const pm_sim* s) {
  KickParams kp;
  memset(&kp, 0, sizeof kp);
  kp.inv_dx = 1.0 / s->dx;
  kp.grav_kernel = s->cfg.force_mode == PM_FORCE_LAGRANGIAN;
  kp.q_kernel = s->cfg.force_mode != PM_FORCE_MESHGRAD;
  kp.quantum = s->cfg.quantum != 0;
  return kp;
}

template <typename R>
pm_status kick(pm_sim* s, const KickParams& kp, double* acc, const KickParams* kp_tab = nullptr,
               const uint32_t* step = nullptr) {
  const Layout& L = s->L;
  const bool drift = kp.drift != 0.0;
  if (drift && !s->sorted) {  // movers are marked against the sorted cells
    pm_status st = sort_particles<R>(s);
    if (st != PM_OK) return st;
  }
  // a drift counts its movers per tile (for the re-sort's partition)
  if (drift)
    CU(s, cudaMemsetAsync(s->at<uint32_t>(L.tcount), 0, size_t(mover_count_words(s->n())) * 4, s->stream));
  {
    PROF(s, PM_STAGE_KICK);
    CU(s, launch_kick<R>(s->pos(), s->mom(), s->keys, s->at<uint32_t>(L.tcount), s->n(), s->at<R>(L.phi),
                         s->at<R>(L.q), s->mesh, kp, kp_tab, step, s->part(), acc, s->errword(),
                         s->tune.kick_threads, s->stream));
  }
  if (drift) {
    s->sorted = false;
    s->fields_valid = false;
    s->keys_marked = true;
  }
  return PM_OK;
}

#define DISPATCH(s, fn, ...) ((s)->fp64() ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

// Reads (after the stream has drained) and clears the device error word.
pm_status device_errors(pm_sim* s) {
  uint32_t e = 0;
  CU(s, cudaMemcpyAsync(&e, s->errword(), 4, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaStreamSynchronize(s->stream));
  if (!e) return PM_OK;
  CU(s, cudaMemsetAsync(s->errword(), 0, 4, s->stream));
  if (e & ERR_TIMEOUT) return fail(s, PM_ERR_TIMEOUT, "a bounded device wait expired (sort look-back or stencil copy)");
  return fail(s, PM_ERR_NONFINITE, "non-finite position or momentum");
}

pm_status check(pm_sim* s) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (!s->have_particles) return fail(s, PM_ERR_STATE, "no particles set");
  return PM_OK;
}

pm_status ensure_fields(pm_sim* s) {
  if (s->fields_valid) return PM_OK;
  return DISPATCH(s, compute_fields, s);
}

// one leapfrog pass: kick by (w1, w2) and drift by d (0 = none); diag = K_v of p_sync
pm_status pass(pm_sim* s, Weights w1, Weights w2, double d, bool diag) {
  KickParams kp = base_kick(s);
  kp.cg1 = w1.kg;
  kp.cq1 = w1.kq;
  kp.cg2 = w2.kg;
  kp.cq2 = w2.kq;
  kp.drift = d / s->dx;
  kp.diag = diag;
  return DISPATCH(s, kick, s, kp, nullptr);
}

double run_a(const pm_config& c, int i, int nsteps, double a_start, double a_end) {
  if (i == nsteps) return a_end;
  const double t = double(i) / nsteps;
  return c.cosmological ? a_start * pow(a_end / a_start, t) : a_start + (a_end - a_start) * t;
}

// leapfrog weights of pm_run's step i (merged kicks): returns the kick of the
// step and updates `pending` to the closing half kick
KickParams step_params(const pm_sim* s, int i, int nsteps, double a_start, double a_end, Weights* pending) {
  const double a0 = run_a(s->cfg, i, nsteps, a_start, a_end), a1 = run_a(s->cfg, i + 1, nsteps, a_start, a_end);
  const double ah = half_point(s->cfg, a0, a1);
  const Weights w2 = time_weights(s->cfg, a0, ah);
  KickParams kp = base_kick(s);
  kp.cg1 = pending->kg;
  kp.cq1 = pending->kq;
  kp.cg2 = w2.kg;
  kp.cq2 = w2.kq;
  kp.drift = time_weights(s->cfg, a0, a1).kq / s->dx;
  *pending = time_weights(s->cfg, ah, a1);
  return kp;
}

// one captured step: table-driven kick + drift, then steps (i)-(iii), then the
// device step counter advances
pm_status table_step(pm_sim* s, const KickParams* tab, uint32_t* step) {
  KickParams kp = base_kick(s);
  kp.drift = 1.0;  // host-side marker only: the positions move, the weights come from the table
  pm_status st = DISPATCH(s, kick, s, kp, nullptr, tab, step);
  if (st != PM_OK) return st;
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  CU(s, launch_step_inc(step, s->stream));
  return PM_OK;
}

void to_public(const Tuning& t, pm_tuning* o) {
  o->stencil_rows = t.st_ty;
  o->stencil_planes = t.st_zlen;
  o->stencil_stages = t.st_stages;
  o->kick_threads = t.kick_threads;
  o->deposit_warps = t.dep_warps;
  o->green_fused = t.green_fused;
}

// drops the captured steps (they hold the launch shapes)
void drop_graphs(pm_sim* s) {
  cudaStreamSynchronize(s->stream);
  if (s->cap) cudaStreamSynchronize(s->cap);
  for (auto& g : s->run_graph) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = pm_sim::RunGraph();
  }
}

// ms per launch of `reps` back-to-back launches on the simulation's stream
// (after one untimed launch); negative on error
template <typename F>
double time_launches(pm_sim* s, int reps, F&& launch) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  double ms = -1.0;
  if (launch() == PM_OK && cudaEventRecord(e0, s->stream) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = launch() == PM_OK;
    float t = 0.0f;
    if (ok && cudaEventRecord(e1, s->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
      ms = double(t) / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

template <typename R>
pm_status autotune(pm_sim* s, int reps) {
  pm_status st = ensure_fields(s);
  if (st != PM_OK) return st;
  const int n = s->cfg.n_mesh;
  const bool prof = s->prof_on;
  s->prof_on = false;
  Tuning best = s->tune;
  // stencil tiles (fp32 compact Laplacian)
  if (!s->fp64() && s->cfg.quantum && s->cfg.lap == PM_LAP_COMPACT) {
    double tbest = -1.0;
    // register-column kernel, one-shot tiles (stages 0) and sweeping tiles (ring of 4..8 planes)
    const int tys[] = {0, 1, 2, 4, 8}, zls[] = {2, 4, 8, 16, 32, 64}, sts[] = {0, 4, 6, 8};
    for (int ty : tys)
      for (int zl : zls)
        for (int sg : sts) {
          if (ty == 0 && (zl != 8 || sg != 4)) continue;  // one register-column candidate
          if (ty > 0 && sg > 0 && zl < 8) continue;        // sweeps of fewer planes re-read too much
          if (ty > 0 && !stencil_shape_ok(n, ty, zl, sg)) continue;
          s->tune.st_ty = ty;
          s->tune.st_zlen = ty ? zl : 0;
          s->tune.st_stages = ty ? sg : 0;
          const double t = time_launches(s, reps, [&] { return stencil_stage<R>(s); });
          if (t > 0 && (tbest < 0 || t < tbest)) {
            tbest = t;
            best.st_ty = s->tune.st_ty;
            best.st_zlen = s->tune.st_zlen;
            best.st_stages = s->tune.st_stages;
          }
        }
    s->tune = best;
  }
  // deposit: warps per tile of mesh rows
  {
    double tbest = -1.0;
    for (int w : {2, 4, 8}) {
      s->tune.dep_warps = w;
      const double t = time_launches(s, reps, [&] { return deposit<R>(s); });
      if (t > 0 && (tbest < 0 || t < tbest)) {
        tbest = t;
        best.dep_warps = w;
      }
    }
    s->tune = best;
  }
  // kick: threads per block, timed with zero weights and no drift (the state is unchanged)
  {
    KickParams kp = base_kick(s);
    double tbest = -1.0;
    for (int th : {128, 256}) {
      s->tune.kick_threads = th;
      const double t = time_launches(s, reps, [&] { return kick<R>(s, kp, nullptr); });
      if (t > 0 && (tbest < 0 || t < tbest)) {
        tbest = t;
        best.kick_threads = th;
      }
    }
    s->tune = best;
  }
  s->prof_on = prof;
  // the fields (and their partial sums) again, with the chosen shapes
  s->fields_valid = false;
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  return device_errors(s);
}
}  // namespace

// ================================================================ C ABI
extern "C" {

void pm_config_default(pm_config* c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  c->precision = PM_FP32;
  c->omega_m = 0.3;
  c->omega_l = 0.7;
  c->h = 0.7;
  c->m22 = 2.5;
  c->quantum = 1;
  c->force_mode = PM_FORCE_MESHGRAD;
  c->lap = PM_LAP_COMPACT;
  c->cosmological = 1;
  c->rho_floor = 1e-6;
  c->rho_fp64 = 1e-2;
  c->kernel = PM_KERNEL_CIC;
  c->smooth_h = 3.5;
}

double pm_hbar_over_m(const pm_config* c) { return c ? hbar_over_m(c->m22, c->h) : 0.0; }

size_t pm_arena_bytes(const pm_config* c) {
  std::string why;
  if (!valid_config(c, &why)) {
    g_create_error = why;
    return 0;
  }
  size_t ws = 0;
  if (!fft_work_bytes(*c, &ws, &why)) {
    g_create_error = why;
    return 0;
  }
  return make_layout(*c, ws).total;
}

pm_status pm_create(const pm_config* c, void* dev_arena, size_t bytes, void* stream, pm_sim** out) {
  if (!out) return fail(nullptr, PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  std::string why;
  if (!valid_config(c, &why)) return fail(nullptr, PM_ERR_INVALID_ARG, "%s", why.c_str());
  if (!dev_arena || (reinterpret_cast<uintptr_t>(dev_arena) & 255))
    return fail(nullptr, PM_ERR_INVALID_ARG, "arena must be a 256-byte aligned device pointer");
  size_t ws = 0;
  if (!fft_work_bytes(*c, &ws, &why)) return fail(nullptr, PM_ERR_CUFFT, "%s", why.c_str());
  Layout L = make_layout(*c, ws);
  if (bytes < L.total) return fail(nullptr, PM_ERR_NO_MEMORY, "arena has %zu bytes, needs %zu", bytes, L.total);
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, dev_arena) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(nullptr, PM_ERR_INVALID_ARG, "arena is not device memory");
  }
  pm_sim* s = new pm_sim();
  s->cfg = *c;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  s->arena = reinterpret_cast<char*>(dev_arena);
  s->L = L;
  const int N = c->n_mesh;
  s->mesh.n = N;
  s->mesh.log2n = (N & (N - 1)) == 0 ? __builtin_ctz(unsigned(N)) : -1;
  s->mesh.n2 = uint32_t(N) * uint32_t(N);
  s->mesh.n3 = s->mesh.n2 * uint32_t(N);
  s->dx = c->box / N;
  s->hbm = hbar_over_m(c->m22, c->h);
  s->norm = double(s->mesh.n3) / double(c->n_part);  // m_p / dx^3 with m_p = L^3 / n_part
  s->cur = 0;
  s->keys = s->at<uint32_t>(L.keys[0]);
  s->keys_tmp[0] = s->at<uint32_t>(L.keys[1]);
  s->keys_tmp[1] = s->at<uint32_t>(L.keys[2]);
  s->have_particles = s->sorted = s->fields_valid = false;
  s->tune = default_tuning(N);
  {
    int dev = 0, sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sm > 0)
      s->sms = sm;
  }
  cufftType fwd = c->precision == PM_FP64 ? CUFFT_D2Z : CUFFT_R2C;
  cufftType inv = c->precision == PM_FP64 ? CUFFT_Z2D : CUFFT_C2R;
  cufftHandle* plans[2] = {&s->plan_fwd, &s->plan_inv};
  cufftType types[2] = {fwd, inv};
  for (int k = 0; k < 2; ++k) {
    size_t w = 0;
    cufftResult r = cufftCreate(plans[k]);
    if (r == CUFFT_SUCCESS) r = cufftSetAutoAllocation(*plans[k], 0);
    if (r == CUFFT_SUCCESS && c->fft_jit)
      r = cufftSetPlanPropertyInt64(*plans[k], NVFFT_PLAN_PROPERTY_INT64_PATIENT_JIT, 1);
    if (r == CUFFT_SUCCESS) r = cufftMakePlan3d(*plans[k], N, N, N, types[k], &w);
    if (r == CUFFT_SUCCESS) r = cufftSetWorkArea(*plans[k], s->arena + L.work);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(*plans[k], s->stream);
    if (r != CUFFT_SUCCESS) {
      if (k == 1) cufftDestroy(s->plan_fwd);
      delete s;
      return fail(nullptr, PM_ERR_CUFFT, "cuFFT plan setup failed (%d)", int(r));
    }
  }
  if (cudaMemsetAsync(s->errword(), 0, 256, s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->arena + L.status, 0, (size_t(1) << L.digit_bits) * size_t(L.ntiles) * 8, s->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess) {
    cufftDestroy(s->plan_fwd);
    cufftDestroy(s->plan_inv);
    delete s;
    return fail(nullptr, PM_ERR_CUDA, "stream setup failed");
  }
  {
    const double coefs[2] = {green_coef(s), stencil_params(s, false).qcoef};
    if (cudaMemcpyAsync(s->coefs(), coefs, sizeof coefs, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
      cufftDestroy(s->plan_fwd);
      cufftDestroy(s->plan_inv);
      delete s;
      return fail(nullptr, PM_ERR_CUDA, "coefficient upload failed");
    }
  }
  if (c->precision == PM_FP32) kick_stream_prepare();
  // fp32 cloud-in-cell on power-of-two meshes from 128^3: the Green multiplication inside the z
  // transform (smaller meshes keep the 3D transforms, which a packed batch class batches over its
  // members; pm_set_tuning turns it on there).  Where cuFFT refuses the 2D plans, the 3D transforms
  // and the separate pass stay.
  if (c->precision == PM_FP32 && c->kernel == PM_KERNEL_CIC && spec_z_supported(N) && N >= GREEN_FUSE_MIN_MESH) {
    std::string ignored;
    if (spec_plan_setup(s, &ignored) == CUFFT_SUCCESS) s->tune.green_fused = xy_fft_supported(N) ? 2 : 1;
  }
  if (s->cfg.kernel == PM_KERNEL_SPLINE) {
    s->direct = c->smooth_real != 0;
    spline_taps(c->smooth_h, s->taps);
    s->taps_r2 = 0;
    for (int r2 = 0; r2 <= 27; ++r2)
      if (sqrt(double(r2)) < c->smooth_h) s->taps_r2 = r2;
    pm_status st = DISPATCH(s, spline_symbol, s);
    if (st == PM_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = PM_ERR_CUDA;
    if (st != PM_OK) {
      const std::string msg = s->err;
      cufftDestroy(s->plan_fwd);
      cufftDestroy(s->plan_inv);
      delete s;
      return fail(nullptr, st, "spline kernel setup failed: %s", msg.c_str());
    }
  }
  *out = s;
  return PM_OK;
}

pm_status pm_destroy(pm_sim* s) {
  if (!s) return PM_ERR_INVALID_ARG;
  cudaStreamSynchronize(s->stream);
  if (s->cap) {
    cudaStreamSynchronize(s->cap);
    cudaStreamDestroy(s->cap);
    cudaEventDestroy(s->ev_in);
    cudaEventDestroy(s->ev_out);
    cudaEventDestroy(s->ev_tab);
    cudaFreeHost(s->tab_host);
  }
  for (auto& g : s->run_graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  cufftDestroy(s->plan_fwd);
  cufftDestroy(s->plan_inv);
  if (s->have_plan2) {
    cufftDestroy(s->plan2_fwd);
    cufftDestroy(s->plan2_inv);
  }
  delete s;
  return PM_OK;
}

pm_status pm_set_particles(pm_sim* s, const double* x, const double* p) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (!x || !p) return fail(s, PM_ERR_INVALID_ARG, "x and p must be non-null host arrays");
  const size_t bytes = size_t(s->n()) * 3 * sizeof(double);
  double* dx = s->staging();
  double* dp = dx + 3 * size_t(s->n());
  CU(s, cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s->stream));
  CU(s, cudaMemcpyAsync(dp, p, bytes, cudaMemcpyHostToDevice, s->stream));
  s->cur = 0;
  CU(s, DISPATCH(s, launch_init_particles, dx, dp, s->n(), s->mesh, 1.0 / s->dx, s->pos(), s->mom(), s->keys,
                 s->errword(), s->stream));
  s->have_particles = true;
  s->sorted = s->fields_valid = s->keys_marked = false;
  pm_status st = DISPATCH(s, sort_particles, s);
  if (st != PM_OK) return st;
  return device_errors(s);
}

pm_status pm_get_particles(pm_sim* s, double* x, double* p) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (!x || !p) return fail(s, PM_ERR_INVALID_ARG, "x and p must be non-null");
  double* dx = s->staging();
  double* dp = dx + 3 * size_t(s->n());
  CU(s, DISPATCH(s, launch_get_particles, s->pos(), s->mom(), s->n(), s->mesh, s->dx, dx, dp, s->stream));
  const size_t bytes = size_t(s->n()) * 3 * sizeof(double);
  CU(s, cudaMemcpyAsync(x, dx, bytes, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaMemcpyAsync(p, dp, bytes, cudaMemcpyDeviceToHost, s->stream));
  return device_errors(s);
}

pm_status pm_deposit(pm_sim* s, double* rho_host) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  st = DISPATCH(s, density, s);  // phi and Q no longer match rho until the mesh stages run
  if (st != PM_OK) return st;
  if (rho_host) return pm_get_field(s, PM_FIELD_RHO, rho_host);
  return PM_OK;
}

pm_status pm_forces(pm_sim* s, double a, double* acc_host) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (!acc_host) return fail(s, PM_ERR_INVALID_ARG, "acc must be non-null");
  if (s->cfg.cosmological && !(a > 0)) return fail(s, PM_ERR_INVALID_ARG, "a must be positive");
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  const double aa = s->cfg.cosmological ? a : 1.0;
  KickParams kp = base_kick(s);
  kp.cg1 = 1.0 / aa;
  kp.cq1 = 1.0 / (aa * aa);
  kp.accel_out = 1;
  double* dacc = s->staging();
  st = DISPATCH(s, kick, s, kp, dacc);
  if (st != PM_OK) return st;
  CU(s, cudaMemcpyAsync(acc_host, dacc, size_t(s->n()) * 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return device_errors(s);
}

pm_status pm_step(pm_sim* s, double a0, double a1) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (s->cfg.cosmological && !(a0 > 0 && a1 > 0)) return fail(s, PM_ERR_INVALID_ARG, "a0, a1 must be positive");
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  const double ah = half_point(s->cfg, a0, a1);
  const Weights zero = {0.0, 0.0};
  const Weights d = time_weights(s->cfg, a0, a1);
  st = pass(s, zero, time_weights(s->cfg, a0, ah), d.kq, false);
  if (st != PM_OK) return st;
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  return pass(s, time_weights(s->cfg, ah, a1), zero, 0.0, true);
}

pm_status pm_run_adaptive(pm_sim* s, double a_start, double a_end, double cfl, int32_t max_steps, double* a_steps,
                          int32_t* steps_taken) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (max_steps < 1) return fail(s, PM_ERR_INVALID_ARG, "max_steps must be >= 1");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(s, PM_ERR_INVALID_ARG, "cfl must be in (0, 1]");
  if (!(a_end > a_start)) return fail(s, PM_ERR_INVALID_ARG, "a_end must exceed a_start");
  if (s->cfg.cosmological && !(a_start > 0)) return fail(s, PM_ERR_INVALID_ARG, "a must be positive");
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  const pm_config& c = s->cfg;
  const double limit = cfl * s->dx;
  const int nkb = kick_blocks(s->n(), s->tune.kick_threads);
  Weights pending = {0.0, 0.0};  // closing half kick of the previous step
  double a = a_start;
  int32_t done = 0;
  if (a_steps) a_steps[0] = a;
  while (a < a_end && done < max_steps) {
    // the bound's inputs: max |p_sync|, max |grad phi~|, max |grad Q~| (one read-only particle pass)
    KickParams km = base_kick(s);
    km.cg1 = pending.kg;
    km.cq1 = pending.kq;
    km.maxima = 1;
    st = DISPATCH(s, kick, s, km, nullptr);
    if (st != PM_OK) return st;
    double mx[3];
    CU(s, launch_reduce_max(s->part(), nkb, 3, s->red(), s->stream));
    CU(s, cudaMemcpyAsync(mx, s->red(), sizeof mx, cudaMemcpyDeviceToHost, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    const double pmax = sqrt(mx[0]), gmax = sqrt(mx[1]), qmax = sqrt(mx[2]);
    // the drift of the step, (max|p_sync| + K_g(a, a_h) g + K_q(a, a_h) q) D(a, a1), within cfl*dx:
    // the largest a1 <= a_end, by bisection in ln a (static: in t)
    auto bound = [&](double a1) {
      const Weights wh = time_weights(c, a, half_point(c, a, a1));
      return (pmax + wh.kg * gmax + wh.kq * qmax) * time_weights(c, a, a1).kq;
    };
    auto at = [&](double f) { return c.cosmological ? a * pow(a_end / a, f) : a + (a_end - a) * f; };
    double a1 = a_end;
    if (!(bound(a_end) <= limit)) {
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (bound(at(mid)) <= limit)
          lo = mid;
        else
          hi = mid;
      }
      a1 = at(lo);
      if (!(a1 > a)) return fail(s, PM_ERR_NONFINITE, "adaptive step collapsed at a = %g", a);
    }
    // the step: closing half kick of the previous step + opening half kick + drift, then the forces at a1
    const double ah = half_point(c, a, a1);
    const Weights wo = time_weights(c, a, ah);
    KickParams kp = base_kick(s);
    kp.cg1 = pending.kg;
    kp.cq1 = pending.kq;
    kp.cg2 = wo.kg;
    kp.cq2 = wo.kq;
    kp.drift = time_weights(c, a, a1).kq / s->dx;
    st = DISPATCH(s, kick, s, kp, nullptr);
    if (st != PM_OK) return st;
    st = ensure_fields(s);
    if (st != PM_OK) return st;
    pending = time_weights(c, ah, a1);
    a = a1;
    ++done;
    if (a_steps) a_steps[done] = a;
  }
  st = pass(s, pending, Weights{0.0, 0.0}, 0.0, true);  // closing half kick: synchronised momenta
  if (st != PM_OK) return st;
  if (steps_taken) *steps_taken = done;
  return device_errors(s);
}

pm_status pm_run(pm_sim* s, int32_t nsteps, double a_start, double a_end) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (nsteps < 1) return fail(s, PM_ERR_INVALID_ARG, "nsteps must be >= 1");
  if (s->cfg.cosmological && !(a_start > 0 && a_end > 0)) return fail(s, PM_ERR_INVALID_ARG, "a must be positive");
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  Weights pending = {0.0, 0.0};  // closing half kick of the previous step
  if (nsteps >= 2 && nsteps <= PM_RUN_GRAPH_MAX_STEPS && !s->prof_on) {
    // two steps captured as a CUDA graph and replayed: the weights of every
    // step come from a device table indexed by a device step counter
    if (!s->cap) {
      CU(s, cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
      CU(s, cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
      CU(s, cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming));
      CU(s, cudaEventCreateWithFlags(&s->ev_tab, cudaEventDisableTiming));
      CU(s, cudaMallocHost(&s->tab_host, size_t(PM_RUN_GRAPH_MAX_STEPS) * sizeof(KickParams)));
    }
    if (s->tab_pending) CU(s, cudaEventSynchronize(s->ev_tab));  // the previous upload has left the buffer
    for (int i = 0; i < nsteps; ++i) s->tab_host[i] = step_params(s, i, nsteps, a_start, a_end, &pending);
    KickParams* tab_dev = s->at<KickParams>(s->L.ktab);
    uint32_t* step_dev = s->errword() + 2;
    CU(s, cudaMemcpyAsync(tab_dev, s->tab_host, size_t(nsteps) * sizeof(KickParams), cudaMemcpyHostToDevice,
                          s->stream));
    CU(s, cudaEventRecord(s->ev_tab, s->stream));
    s->tab_pending = true;
    CU(s, cudaMemsetAsync(step_dev, 0, sizeof(uint32_t), s->stream));
    CU(s, cudaEventRecord(s->ev_in, s->stream));
    CU(s, cudaStreamWaitEvent(s->cap, s->ev_in, 0));
    cudaStream_t user = s->stream;
    s->stream = s->cap;
    CF(s, cufftSetStream(s->plan_fwd, s->cap));
    CF(s, cufftSetStream(s->plan_inv, s->cap));
    if (s->have_plan2) {
      CF(s, cufftSetStream(s->plan2_fwd, s->cap));
      CF(s, cufftSetStream(s->plan2_inv, s->cap));
    }
    // graphs for the present state and for the other record buffer (the state
    // after an odd number of steps); capturing executes nothing, so the host
    // state is flipped for the second capture and restored
    cudaError_t ec = cudaSuccess;
    const int cur0 = s->cur;
    for (int v = 0; v < 2 && ec == cudaSuccess && st == PM_OK; ++v) {
      const int want = v == 0 ? cur0 : 1 - cur0;
      if (v == 1 && s->L.passes < 2) break;  // a single sort pass also swaps the key buffers
      bool have = false;
      for (auto& g : s->run_graph) have |= g.exec && g.cur == want && g.keys == s->keys;
      if (have) continue;
      auto& slot = s->run_graph[want];
      if (slot.exec) cudaGraphExecDestroy(slot.exec);
      slot = pm_sim::RunGraph();
      s->cur = want;
      const bool sorted0 = s->sorted, fields0 = s->fields_valid, marked0 = s->keys_marked;
      cudaGraph_t graph = nullptr;
      ec = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
      if (ec == cudaSuccess) {
        for (int r = 0; r < 2 && st == PM_OK; ++r) st = table_step(s, tab_dev, step_dev);
        cudaError_t ee = cudaStreamEndCapture(s->cap, &graph);
        if (st == PM_OK && ee != cudaSuccess) ec = ee;
      }
      if (ec == cudaSuccess && st == PM_OK) ec = cudaGraphInstantiate(&slot.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ec == cudaSuccess && st == PM_OK) {
        slot.cur = want;
        slot.keys = s->keys;
      }
      s->cur = cur0;
      s->sorted = sorted0;
      s->fields_valid = fields0;
      s->keys_marked = marked0;
    }
    cudaGraphExec_t exec = nullptr;
    for (auto& g : s->run_graph)
      if (g.exec && g.cur == s->cur && g.keys == s->keys) exec = g.exec;
    if (!exec && ec == cudaSuccess && st == PM_OK) ec = cudaErrorUnknown;
    for (int k = 0; ec == cudaSuccess && st == PM_OK && k < nsteps / 2; ++k) ec = cudaGraphLaunch(exec, s->cap);
    if (ec == cudaSuccess && st == PM_OK && (nsteps & 1)) st = table_step(s, tab_dev, step_dev);
    s->stream = user;
    cufftSetStream(s->plan_fwd, user);
    cufftSetStream(s->plan_inv, user);
    if (s->have_plan2) {
      cufftSetStream(s->plan2_fwd, user);
      cufftSetStream(s->plan2_inv, user);
    }
    if (st != PM_OK) return st;
    if (ec != cudaSuccess) return fail(s, PM_ERR_CUDA, "captured steps: %s", cudaGetErrorString(ec));
    // the replays leave the state as it was before them (two sorts per graph),
    // except that their stencils skipped the K_rho partials
    s->krho_valid = false;
    CU(s, cudaEventRecord(s->ev_out, s->cap));
    CU(s, cudaStreamWaitEvent(s->stream, s->ev_out, 0));
  } else {
    for (int i = 0; i < nsteps; ++i) {
      const KickParams kp = step_params(s, i, nsteps, a_start, a_end, &pending);
      st = DISPATCH(s, kick, s, kp, nullptr);
      if (st != PM_OK) return st;
      st = ensure_fields(s);
      if (st != PM_OK) return st;
    }
  }
  return pass(s, pending, Weights{0.0, 0.0}, 0.0, true);
}

pm_status pm_energy(pm_sim* s, double a, double out[6]) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (!out) return fail(s, PM_ERR_INVALID_ARG, "out must be non-null");
  st = ensure_fields(s);
  if (st != PM_OK) return st;
  // K_v and momentum of the current (synchronised) momenta
  st = pass(s, Weights{0.0, 0.0}, Weights{0.0, 0.0}, 0.0, true);
  if (st != PM_OK) return st;
  if (s->cfg.quantum && !s->krho_valid) {  // the steps skip the K_rho sums: Q~ again, with them
    st = DISPATCH(s, krho_stage, s);
    if (st != PM_OK) return st;
  }
  const int nkb = kick_blocks(s->n(), s->tune.kick_threads);
  double* red = s->red();
  CU(s, launch_reduce(s->part(), nkb, 4, red, s->stream));
  CU(s, launch_reduce(wg_part(s), s->wg_count, 1, red + 4, s->stream));
  if (s->cfg.quantum) CU(s, launch_reduce(kr_part(s), kr_blocks(s), 1, red + 5, s->stream));
  double h[6];
  CU(s, cudaMemcpyAsync(h, red, 6 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  st = device_errors(s);
  if (st != PM_OK) return st;
  const double aa = s->cfg.cosmological ? a : 1.0;
  const double box = s->cfg.box;
  const double mp = box * box * box / double(s->n());
  const double dx3 = s->dx * s->dx * s->dx;
  out[0] = 0.5 * mp * h[0] / (aa * aa);
  out[1] = 0.5 / aa * h[4] * dx3;
  out[2] = s->cfg.quantum ? 0.5 * s->hbm * s->hbm / (aa * aa) * s->dx * h[5] : 0.0;
  out[3] = mp * h[1];
  out[4] = mp * h[2];
  out[5] = mp * h[3];
  bool bad = false;
  for (int k = 0; k < 6; ++k) bad |= !isfinite(out[k]);
  if (bad) return fail(s, PM_ERR_NONFINITE, "non-finite momentum or energy");
  return PM_OK;
}

pm_status pm_power_spectrum(pm_sim* s, int32_t nbins, double* k, double* P, int64_t* nmodes) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (nbins < 1 || nbins > s->cfg.n_mesh / 2 || nbins > PK_MAX_BINS || !k || !P || !nmodes)
    return fail(s, PM_ERR_INVALID_ARG, "nbins must be in [1, N/2] with non-null outputs");
  if (spline(s)) {
    // P(k) of the particles' cloud-in-cell density (the mesh holds the smoothed one)
    st = DISPATCH(s, deposit, s);
    s->fields_valid = false;
  } else {
    st = ensure_fields(s);
  }
  if (st != PM_OK) return st;
  const Layout& L = s->L;
  if (s->fp64()) {
    CF(s, cufftExecD2Z(s->plan_fwd, s->at<cufftDoubleReal>(L.rho), (cufftDoubleComplex*)(s->arena + L.spec)));
  } else {
    CF(s, cufftExecR2C(s->plan_fwd, s->at<cufftReal>(L.rho), (cufftComplex*)(s->arena + L.spec)));
  }
  double* part = s->part();
  CU(s, DISPATCH(s, launch_power, s->arena + L.spec, s->mesh, nbins, part, s->stream));
  double* red = s->red();
  CU(s, launch_reduce(part, RED_GRID, 3 * nbins, red, s->stream));
  double* h = new double[3 * nbins];
  cudaError_t e1 = cudaMemcpyAsync(h, red, 3 * nbins * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  cudaError_t e2 = cudaStreamSynchronize(s->stream);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    delete[] h;
    return fail(s, PM_ERR_CUDA, "power spectrum copy failed");
  }
  const double N = s->cfg.n_mesh, box = s->cfg.box;
  const double kf = 2.0 * M_PI / box;
  const double norm = box * box * box / (N * N * N * N * N * N);
  for (int b = 0; b < nbins; ++b) {
    double cnt = h[b];
    nmodes[b] = int64_t(llround(cnt));
    k[b] = cnt > 0 ? kf * h[nbins + b] / cnt : NAN;
    P[b] = cnt > 0 ? norm * h[2 * nbins + b] / cnt : NAN;
  }
  delete[] h;
  return PM_OK;
}

pm_status pm_get_field(pm_sim* s, int32_t which, double* host_out) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (!host_out || which < 0 || which > 2) return fail(s, PM_ERR_INVALID_ARG, "bad field or output");
  if (which == PM_FIELD_Q && !s->cfg.quantum) return fail(s, PM_ERR_STATE, "quantum pressure is off");
  const Layout& L = s->L;
  const size_t offs[3] = {density_field(s), L.phi, L.q};
  const int64_t n3 = s->mesh.n3;
  double* d = s->staging();
  if (s->fp64()) {
    CU(s, cudaMemcpyAsync(d, s->arena + offs[which], n3 * 8, cudaMemcpyDeviceToDevice, s->stream));
  } else {
    CU(s, launch_to_double<float>(s->at<float>(offs[which]), n3, d, s->stream));
  }
  CU(s, cudaMemcpyAsync(host_out, d, n3 * 8, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaStreamSynchronize(s->stream));
  return PM_OK;
}

pm_status pm_set_density(pm_sim* s, const double* rho_host) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (!rho_host) return fail(s, PM_ERR_INVALID_ARG, "rho must be non-null");
  const int64_t n3 = s->mesh.n3;
  double* d = s->staging();
  CU(s, cudaMemcpyAsync(d, rho_host, n3 * 8, cudaMemcpyHostToDevice, s->stream));
  if (s->fp64()) {
    CU(s, cudaMemcpyAsync(s->arena + density_field(s), d, n3 * 8, cudaMemcpyDeviceToDevice, s->stream));
  } else {
    CU(s, launch_from_double<float>(d, n3, s->at<float>(density_field(s)), s->stream));
  }
  pm_status st = DISPATCH(s, mesh_from_density, s);
  if (st != PM_OK) return st;
  CU(s, cudaStreamSynchronize(s->stream));
  return PM_OK;
}

pm_status pm_get_tuning(pm_sim* s, pm_tuning* out) {
  if (!s || !out) return PM_ERR_INVALID_ARG;
  to_public(s->tune, out);
  return PM_OK;
}

pm_status pm_set_tuning(pm_sim* s, const pm_tuning* t) {
  if (!s || !t) return PM_ERR_INVALID_ARG;
  const int n = s->cfg.n_mesh;
  if (t->kick_threads != 128 && t->kick_threads != 256)
    return fail(s, PM_ERR_INVALID_ARG, "kick_threads must be 128 or 256");
  if (t->deposit_warps < 1 || t->deposit_warps > 8) return fail(s, PM_ERR_INVALID_ARG, "deposit_warps must be 1..8");
  if (!stencil_shape_ok(n, t->stencil_rows, t->stencil_planes, t->stencil_stages))
    return fail(s, PM_ERR_INVALID_ARG, "stencil shape (%d rows, %d planes, %d stages) is not valid for N = %d",
                t->stencil_rows, t->stencil_planes, t->stencil_stages, n);
  if (t->green_fused < 0 || t->green_fused > 2) return fail(s, PM_ERR_INVALID_ARG, "green_fused must be 0, 1 or 2");
  if (t->green_fused && (s->fp64() || spline(s) || !spec_z_supported(s->cfg.n_mesh)))
    return fail(s, PM_ERR_INVALID_ARG, "green_fused needs PM_FP32, the cloud-in-cell kernel and a power-of-two mesh");
  if (t->green_fused == 2 && !xy_fft_supported(s->cfg.n_mesh))
    return fail(s, PM_ERR_INVALID_ARG, "green_fused = 2 (the fused x-y transform kernels) needs a 256^3 mesh");
  drop_graphs(s);
  if (t->green_fused) {
    std::string why;
    const cufftResult r = spec_plan_setup(s, &why);
    if (r != CUFFT_SUCCESS)
      return fail(s, PM_ERR_CUFFT, "batched 2D transforms: %s failed (%d)", why.c_str(), int(r));
  }
  s->tune.green_fused = t->green_fused;
  s->tune.st_ty = t->stencil_rows;
  s->tune.st_zlen = t->stencil_rows ? t->stencil_planes : 0;
  s->tune.st_stages = t->stencil_rows ? t->stencil_stages : 0;
  s->tune.kick_threads = t->kick_threads;
  s->tune.dep_warps = t->deposit_warps;
  s->fields_valid = false;  // K_rho partials follow the stencil's block count
  return PM_OK;
}

pm_status pm_autotune(pm_sim* s, int32_t reps, pm_tuning* out) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (reps < 1) reps = 5;
  drop_graphs(s);
  st = DISPATCH(s, autotune, s, int(reps));
  if (st != PM_OK) return st;
  if (out) to_public(s->tune, out);
  return PM_OK;
}

pm_status pm_get_order(pm_sim* s, uint32_t* cell, uint32_t* id) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (!cell || !id) return fail(s, PM_ERR_INVALID_ARG, "outputs must be non-null");
  if (!s->sorted) {
    st = DISPATCH(s, sort_particles, s);
    if (st != PM_OK) return st;
  }
  uint32_t* d = reinterpret_cast<uint32_t*>(s->staging());
  CU(s, DISPATCH(s, launch_get_order, s->pos(), s->mom(), s->n(), d, d + s->n(), s->stream));
  CU(s, cudaMemcpyAsync(cell, d, size_t(s->n()) * 4, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaMemcpyAsync(id, d + s->n(), size_t(s->n()) * 4, cudaMemcpyDeviceToHost, s->stream));
  return device_errors(s);
}

pm_status pm_debug_sort_timeout(pm_sim* s, int32_t spin_limit) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (spin_limit < 1) return fail(s, PM_ERR_INVALID_ARG, "spin_limit must be >= 1");
  const Layout& L = s->L;
  const int64_t n = s->n();
  if (L.ntiles < 2) return fail(s, PM_ERR_INVALID_ARG, "needs more than %d particles", RS_TILE);
  uint32_t* hist = s->at<uint32_t>(L.hist);
  uint32_t* counters = hist + 3 * (1 << RS_MAX_BITS);
  const int bits = std::min(L.digit_bits, L.key_bits);
  CU(s, cudaMemsetAsync(hist, 0, hist_bytes(), s->stream));
  CU(s, launch_sort_histogram(s->keys, n, L.passes, L.digit_bits, L.key_bits, hist, s->errword() + 1, s->stream));
  // the first tile is never claimed: its status words stay unpublished for this pass's epoch
  const uint32_t one = 1;
  CU(s, cudaMemcpyAsync(counters, &one, sizeof one, cudaMemcpyHostToDevice, s->stream));
  CU(s, DISPATCH(s, launch_sort_pass, false, s->keys, nullptr, n, 0, bits, hist, s->at<uint64_t>(L.status), counters,
                 s->errword() + 1, 0, L.ntiles, s->keys_tmp[0], s->at<uint32_t>(L.vals[0]), nullptr, nullptr, nullptr,
                 nullptr, s->errword(), s->stream, nullptr, 1, 0, int(spin_limit)));
  return device_errors(s);
}

pm_status pm_sort_stats(pm_sim* s, int64_t* resorts, int64_t* movers) {
  if (!s || !resorts || !movers) return PM_ERR_INVALID_ARG;
  unsigned long long h[2];
  CU(s, cudaMemcpyAsync(h, s->sort_stats(), sizeof h, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaStreamSynchronize(s->stream));
  *resorts = int64_t(h[0]);
  *movers = int64_t(h[1]);
  return PM_OK;
}

// ---------------------------------------------------------------- checkpoint
namespace {
constexpr uint32_t CKPT_MAGIC = 0x4b43504du;  // "MPCK"
constexpr uint32_t CKPT_VERSION = 1;
constexpr size_t CKPT_HEADER = 256;
struct CkptHeader {
  uint32_t magic, version;
  int64_t n_part;
  int32_t n_mesh, precision, kernel, flags;  // flags: 1 sorted, 2 keys marked
  pm_tuning tuning;
  uint64_t resorts, moved;
};
static_assert(sizeof(CkptHeader) <= CKPT_HEADER, "checkpoint header fits its 256 bytes");
size_t rec_bytes(const pm_sim* s) { return s->fp64() ? 32 : 16; }
}  // namespace

size_t pm_checkpoint_bytes(const pm_sim* s) {
  if (!s) return 0;
  return CKPT_HEADER + size_t(s->n()) * (2 * rec_bytes(s) + 4);
}

pm_status pm_save(pm_sim* s, void* host, size_t bytes) {
  pm_status st = check(s);
  if (st != PM_OK) return st;
  if (!host || bytes < pm_checkpoint_bytes(s))
    return fail(s, PM_ERR_INVALID_ARG, "checkpoint buffer needs %zu bytes", pm_checkpoint_bytes(s));
  CkptHeader h;
  memset(&h, 0, sizeof h);
  h.magic = CKPT_MAGIC;
  h.version = CKPT_VERSION;
  h.n_part = s->n();
  h.n_mesh = s->cfg.n_mesh;
  h.precision = s->cfg.precision;
  h.kernel = s->cfg.kernel;
  h.flags = (s->sorted ? 1 : 0) | (s->keys_marked ? 2 : 0);
  to_public(s->tune, &h.tuning);
  unsigned long long stats[2];
  char* out = static_cast<char*>(host);
  const size_t rb = size_t(s->n()) * rec_bytes(s);
  CU(s, cudaMemcpyAsync(stats, s->sort_stats(), sizeof stats, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaMemcpyAsync(out + CKPT_HEADER, s->pos(), rb, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaMemcpyAsync(out + CKPT_HEADER + rb, s->mom(), rb, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaMemcpyAsync(out + CKPT_HEADER + 2 * rb, s->keys, size_t(s->n()) * 4, cudaMemcpyDeviceToHost, s->stream));
  CU(s, cudaStreamSynchronize(s->stream));
  h.resorts = stats[0];
  h.moved = stats[1];
  memset(out, 0, CKPT_HEADER);
  memcpy(out, &h, sizeof h);
  return PM_OK;
}

pm_status pm_load(pm_sim* s, const void* host, size_t bytes) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (!host || bytes < CKPT_HEADER) return fail(s, PM_ERR_INVALID_ARG, "checkpoint buffer too short");
  CkptHeader h;
  memcpy(&h, host, sizeof h);
  if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION)
    return fail(s, PM_ERR_INVALID_ARG, "not a checkpoint of this library version");
  if (h.n_part != s->n() || h.n_mesh != s->cfg.n_mesh || h.precision != s->cfg.precision ||
      h.kernel != s->cfg.kernel)
    return fail(s, PM_ERR_INVALID_ARG, "checkpoint of another configuration (n_part, n_mesh, precision or kernel)");
  if (bytes < pm_checkpoint_bytes(s)) return fail(s, PM_ERR_INVALID_ARG, "checkpoint buffer too short");
  pm_status st = pm_set_tuning(s, &h.tuning);  // validates the shapes and drops captured steps
  if (st != PM_OK) return st;
  const char* in = static_cast<const char*>(host);
  const size_t rb = size_t(s->n()) * rec_bytes(s);
  const unsigned long long stats[2] = {h.resorts, h.moved};
  CU(s, cudaMemcpyAsync(s->pos(), in + CKPT_HEADER, rb, cudaMemcpyHostToDevice, s->stream));
  CU(s, cudaMemcpyAsync(s->mom(), in + CKPT_HEADER + rb, rb, cudaMemcpyHostToDevice, s->stream));
  CU(s, cudaMemcpyAsync(s->keys, in + CKPT_HEADER + 2 * rb, size_t(s->n()) * 4, cudaMemcpyHostToDevice, s->stream));
  CU(s, cudaMemcpyAsync(s->sort_stats(), stats, sizeof stats, cudaMemcpyHostToDevice, s->stream));
  // sorted records: the deposit reads the row starts of the keys (integer, so the same as the re-sort's)
  if (h.flags & 1)
    CU(s, launch_row_start(s->keys, s->n(), uint32_t(s->cfg.n_mesh), s->at<uint32_t>(s->L.row_start), s->stream));
  CU(s, cudaStreamSynchronize(s->stream));
  s->have_particles = true;
  s->sorted = (h.flags & 1) != 0;
  s->keys_marked = (h.flags & 2) != 0;
  s->fields_valid = false;
  s->krho_valid = false;
  return PM_OK;
}

pm_status pm_profile_begin(pm_sim* s, int32_t capacity) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (capacity < 1) return fail(s, PM_ERR_INVALID_ARG, "capacity must be >= 1");
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  s->prof_ev.assign(2 * size_t(capacity), nullptr);
  s->prof_stage.assign(size_t(capacity), PM_STAGE_OTHER);
  for (auto& e : s->prof_ev) CU(s, cudaEventCreate(&e));
  s->prof_used = 0;
  s->prof_on = true;
  return PM_OK;
}

pm_status pm_profile_end(pm_sim* s, double* ms, int64_t* launches) {
  if (!s) return PM_ERR_INVALID_ARG;
  if (!ms || !launches) return fail(s, PM_ERR_INVALID_ARG, "outputs must be non-null");
  s->prof_on = false;
  CU(s, cudaStreamSynchronize(s->stream));
  for (int k = 0; k < PM_NSTAGES; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < s->prof_used; ++i) {
    float t = 0.f;
    CU(s, cudaEventElapsedTime(&t, s->prof_ev[2 * i], s->prof_ev[2 * i + 1]));
    ms[s->prof_stage[i]] += t;
    launches[s->prof_stage[i]] += 1;
  }
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  s->prof_ev.clear();
  s->prof_stage.clear();
  s->prof_used = 0;
  return PM_OK;
}

const char* pm_last_error(const pm_sim* s) { return s ? s->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ================================================================ batches
// Members of equal configuration (every field but the box, the axion mass and
// the cosmology) form a class.  A class's members sit in the batch arena one
// after another at a fixed stride, so every buffer of member m lies m strides
// after member 0's, and one launch steps all of them: the packed kick, re-sort,
// deposit, Green and stencil kernels take the member from a grid dimension, and
// one batched cuFFT plan per class transforms all its meshes.  Per-member
// coefficients (box, mass) come from each member's arena.  Classes that the
// packed launches do not cover (fp64, the spline kernel, the wide Laplacian, a
// stencil shape other than one-shot tiles, a single member) step member by
// member on their own streams, as in pm_run.
namespace {

struct ClassKey {
  pm_config c;
  bool operator==(const ClassKey& o) const {
    const pm_config &a = c, &b = o.c;
    return a.n_part == b.n_part && a.n_mesh == b.n_mesh && a.precision == b.precision && a.quantum == b.quantum &&
           a.force_mode == b.force_mode && a.lap == b.lap && a.cosmological == b.cosmological &&
           a.rho_floor == b.rho_floor && a.rho_fp64 == b.rho_fp64 && a.kernel == b.kernel &&
           a.smooth_h == b.smooth_h && a.fft_jit == b.fft_jit;
  }
};

bool packable(const pm_config& c) {
  return c.precision == PM_FP32 && c.kernel == PM_KERNEL_CIC && c.lap == PM_LAP_COMPACT;
}

// the batched transforms of a class: nm meshes, ms bytes apart
cufftResult class_plans(const pm_config& c, int nm, size_t ms, cufftHandle* fwd, cufftHandle* inv, size_t* work) {
  long long n[3] = {c.n_mesh, c.n_mesh, c.n_mesh};
  long long re[3] = {c.n_mesh, c.n_mesh, c.n_mesh};
  long long cx[3] = {c.n_mesh, c.n_mesh, c.n_mesh / 2 + 1};
  size_t w[2] = {0, 0};
  cufftHandle* h[2] = {fwd, inv};
  for (int k = 0; k < 2; ++k) {
    cufftResult r = cufftCreate(h[k]);
    if (r != CUFFT_SUCCESS) return r;
    // (default plans: patient JIT planning measured slower for these batched transforms)
    r = cufftSetAutoAllocation(*h[k], 0);
    if (r == CUFFT_SUCCESS)
      r = k == 0 ? cufftMakePlanMany64(*h[k], 3, n, re, 1, (long long)(ms / 4), cx, 1, (long long)(ms / 8), CUFFT_R2C,
                                       nm, &w[k])
                 : cufftMakePlanMany64(*h[k], 3, n, cx, 1, (long long)(ms / 8), re, 1, (long long)(ms / 4), CUFFT_C2R,
                                       nm, &w[k]);
    if (r != CUFFT_SUCCESS) {
      cufftDestroy(*h[k]);
      if (k == 1) cufftDestroy(*fwd);
      return r;
    }
  }
  *work = std::max(w[0], w[1]);
  return CUFFT_SUCCESS;
}

struct BatchClass {
  std::vector<int> members;  // batch indices, in arena order
  size_t off = 0, stride = 0, work_off = 0, work = 0;
  bool packed = false;
};

struct BatchLayout {
  std::vector<BatchClass> classes;
  std::vector<size_t> off, bytes;  // per member (batch index)
  size_t total = 0;
};

bool batch_layout(const pm_config* cfgs, int n, BatchLayout* L, std::string* why) {
  std::vector<ClassKey> keys;
  L->off.assign(n, 0);
  L->bytes.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const size_t b = pm_arena_bytes(&cfgs[i]);
    if (b == 0) {
      *why = "member " + std::to_string(i) + ": " + g_create_error;
      return false;
    }
    L->bytes[i] = b;
    size_t k = 0;
    while (k < keys.size() && !(keys[k] == ClassKey{cfgs[i]})) ++k;
    if (k == keys.size()) {
      keys.push_back(ClassKey{cfgs[i]});
      L->classes.emplace_back();
    }
    L->classes[k].members.push_back(i);
  }
  size_t off = 0;
  for (size_t k = 0; k < L->classes.size(); ++k) {
    BatchClass& C = L->classes[k];
    C.stride = align_up(L->bytes[C.members[0]]);
    C.off = off;
    for (size_t j = 0; j < C.members.size(); ++j) L->off[C.members[j]] = off + j * C.stride;
    off = align_up(off + C.members.size() * C.stride);
    C.packed = packable(keys[k].c) && C.members.size() >= 2;
    if (C.packed) {
      cufftHandle f, v;
      if (class_plans(keys[k].c, int(C.members.size()), C.stride, &f, &v, &C.work) != CUFFT_SUCCESS) {
        C.packed = false;  // no batched plan for this class: member by member
      } else {
        cufftDestroy(f);
        cufftDestroy(v);
        C.work_off = off;
        off = align_up(off + C.work);
      }
    }
  }
  L->total = off;
  return true;
}

}  // namespace

struct pm_batch {
  std::vector<pm_sim*> sims;          // batch order
  std::vector<cudaStream_t> streams;  // one per member (member-by-member classes)
  std::vector<cudaEvent_t> join;
  struct Class {
    std::vector<int> members;
    size_t stride = 0;
    bool packed = false;
    cufftHandle fwd = 0, inv = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t join = nullptr;
  };
  std::vector<Class> classes;
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaStream_t stream = nullptr;  // the caller's stream
  cudaStream_t cap = nullptr;     // the batch's own stream: graphs are captured and launched here
  char* arena = nullptr;
  int last_packed = 0;  // members stepped by packed launches in the last run
  std::string err;
};

namespace {

pm_status bfail(pm_batch* b, pm_status st, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_create_error = msg;
  return st;
}

// the members of a packed class step together only from one common state
bool same_state(const pm_batch::Class& C, const std::vector<pm_sim*>& sims) {
  const pm_sim* a = sims[C.members[0]];
  for (int i : C.members) {
    const pm_sim* s = sims[i];
    if (s->cur != a->cur || s->sorted != a->sorted || s->fields_valid != a->fields_valid ||
        s->keys_marked != a->keys_marked || (s->keys - s->at<uint32_t>(0)) != (a->keys - a->at<uint32_t>(0)) ||
        s->tune.st_ty != a->tune.st_ty || s->tune.st_zlen != a->tune.st_zlen ||
        s->tune.st_stages != a->tune.st_stages || s->tune.kick_threads != a->tune.kick_threads ||
        s->tune.dep_warps != a->tune.dep_warps || green_fused(s) != green_fused(a) ||
        s->tune.green_fused != a->tune.green_fused)
      return false;
  }
  if (!green_fused(a) && !C.fwd) return false;  // the class's batched 3D transforms were not planned
  const StencilParams sp = stencil_params(a, false);
  return !a->cfg.quantum || (a->tune.st_ty > 0 && a->tune.st_stages == 0 && stencil_shape_ok(a->cfg.n_mesh, sp.ty, sp.zlen, 0));
}

#define PCU(expr)                                                                                       \
  do {                                                                                                  \
    cudaError_t e_ = (expr);                                                                            \
    if (e_ != cudaSuccess) return fail(s, PM_ERR_CUDA, "packed step: %s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// One table-driven leapfrog step of every member of a packed class on
// stream `st` (the packed form of table_step): kick + drift, re-sort, deposit,
// both transforms, Green, stencil, step counters.  Member 0's pointers, the
// others a stride apart.
pm_status packed_step(pm_batch::Class& C, const std::vector<pm_sim*>& sims, cudaStream_t st) {
  pm_sim* s = sims[C.members[0]];
  const Layout& L = s->L;
  const int nm = int(C.members.size());
  const size_t ms = C.stride;
  const int64_t n = s->n();
  const int nxt = s->cur ^ 1;
  // kick + drift with the weights of the members' step counters
  KickParams kp = base_kick(s);
  kp.drift = 1.0;  // host-side marker only: the positions move, the weights come from the tables
  PCU(cudaMemset2DAsync(s->at<uint32_t>(L.tcount), ms, 0, size_t(mover_count_words(n)) * 4, size_t(nm), st));
  PCU(launch_kick<float>(s->pos(), s->mom(), s->keys, s->at<uint32_t>(L.tcount), n, s->at<float>(L.phi),
                         s->at<float>(L.q), s->mesh, kp, s->at<KickParams>(L.ktab), s->errword() + 2, s->part(),
                         nullptr, s->errword(), s->tune.kick_threads, st, nm, ms));
  // re-sort into the other record buffer (the movers' count on the device of every member)
  const int N = s->cfg.n_mesh;
  PCU(cudaMemset2DAsync(s->at<uint32_t>(L.rcnt), ms, 0, size_t(3) * N * N * 4, size_t(nm), st));
  for (int part = 0; part < 3; ++part)
    PCU(launch_resort<float>(part, s->keys, n, s->at<uint32_t>(L.tcount), s->keys_tmp[0], s->at<uint32_t>(L.vals[0]),
                             s->keys_tmp[1], s->at<uint32_t>(L.vals[1]), s->at<uint32_t>(L.keys[3]),
                             s->at<uint32_t>(L.vals[2]), s->at<uint32_t>(L.tile_cnt), s->at<uint32_t>(L.rcnt),
                             s->at<uint32_t>(L.btot), s->at<uint32_t>(L.srow), s->at<uint32_t>(L.mrow),
                             s->at<uint32_t>(L.row_start), s->mesh, s->sort_stats(), s->keys, s->pos(), s->mom(),
                             s->arena + L.pos[nxt], s->arena + L.mom[nxt], s->sms, st, nm, ms));
  // deposit, potential, quantum pressure
  PCU(launch_deposit<float>(s->arena + L.pos[nxt], s->at<uint32_t>(L.row_start), n, s->mesh, s->norm,
                            s->at<float>(L.rho), st, s->tune.dep_warps, nm, ms));
  const bool fused = green_fused(s);
  const bool own_xy = fused && s->tune.green_fused == 2;
  if (own_xy)  // the x-y transforms of every member's planes in one launch
    PCU(launch_xy_r2c(s->at<float>(L.rho), s->arena + L.spec, s->at<float2>(L.green), N, st, nm, ms));
  if (fused && !own_xy) {  // each member's own 2D transforms (the same as alone)
    for (int i : C.members) {
      pm_sim* m = sims[i];
      CF(s, cufftSetStream(m->plan2_fwd, st));
      const cufftResult r = cufftExecR2C(m->plan2_fwd, m->at<cufftReal>(L.rho), (cufftComplex*)(m->arena + L.spec));
      CF(s, cufftSetStream(m->plan2_fwd, m->stream));
      CF(s, r);
    }
  }
  if (fused) {  // the z kernel over the whole class
    PCU(launch_spec_z(s->arena + L.spec, s->at<float2>(L.green), s->at<float>(L.green + size_t(N) * 8), s->mesh,
                      green_coef(s), wg_part(s), st, s->coefs(), nm, ms));
  }
  if (own_xy) PCU(launch_xy_c2r(s->arena + L.spec, s->at<float>(L.phi), s->at<float2>(L.green), N, st, nm, ms));
  if (fused && !own_xy) {
    for (int i : C.members) {
      pm_sim* m = sims[i];
      CF(s, cufftSetStream(m->plan2_inv, st));
      const cufftResult r = cufftExecC2R(m->plan2_inv, (cufftComplex*)(m->arena + L.spec), m->at<cufftReal>(L.phi));
      CF(s, cufftSetStream(m->plan2_inv, m->stream));
      CF(s, r);
    }
  }
  if (!fused) {
    CF(s, cufftSetStream(C.fwd, st));
    CF(s, cufftSetStream(C.inv, st));
    CF(s, cufftExecR2C(C.fwd, s->at<cufftReal>(L.rho), (cufftComplex*)(s->arena + L.spec)));
    PCU(launch_green<float>(s->arena + L.spec, s->mesh, green_coef(s), wg_part(s), st, s->coefs(), nm, ms));
    CF(s, cufftExecC2R(C.inv, (cufftComplex*)(s->arena + L.spec), s->at<cufftReal>(L.phi)));
  }
  if (s->cfg.quantum)
    PCU(launch_stencil<float>(s->at<float>(L.rho), s->mesh, stencil_params(s, false), s->at<float>(L.q), kr_part(s),
                              s->at<uint32_t>(L.st_list), s->at<uint32_t>(L.st_count), s->errword(), st,
                              s->coefs() + 1, nm, ms));
  PCU(launch_step_inc(s->errword() + 2, st, nm, ms));
  for (int i : C.members) {
    pm_sim* m = sims[i];
    m->cur = nxt;
    m->keys_marked = false;
    m->sorted = true;
    m->fields_valid = true;
    m->krho_valid = false;
    m->wg_count = fused ? spec_z_tiles(N) : MESH_GRID;
  }
  return PM_OK;
}
#undef PCU

}  // namespace

extern "C" {

size_t pm_batch_arena_bytes(const pm_config* cfgs, int32_t n) {
  if (!cfgs || n < 1 || n > 4096) {
    g_create_error = "need 1..4096 member configurations";
    return 0;
  }
  BatchLayout L;
  std::string why;
  if (!batch_layout(cfgs, n, &L, &why)) {
    g_create_error = why;
    return 0;
  }
  return L.total;
}

pm_status pm_batch_create(const pm_config* cfgs, int32_t n, void* dev_arena, size_t bytes, void* stream,
                          pm_batch** out) {
  if (!out) return bfail(nullptr, PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!cfgs || n < 1 || n > 4096) return bfail(nullptr, PM_ERR_INVALID_ARG, "need 1..4096 member configurations");
  if (!dev_arena || (reinterpret_cast<uintptr_t>(dev_arena) & 255))
    return bfail(nullptr, PM_ERR_INVALID_ARG, "arena must be a 256-byte aligned device pointer");
  BatchLayout L;
  std::string why;
  if (!batch_layout(cfgs, n, &L, &why)) return bfail(nullptr, PM_ERR_INVALID_ARG, why);
  if (bytes < L.total)
    return bfail(nullptr, PM_ERR_NO_MEMORY,
                 "arena has " + std::to_string(bytes) + " bytes, needs " + std::to_string(L.total));
  pm_batch* b = new pm_batch();
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->arena = reinterpret_cast<char*>(dev_arena);
  auto cleanup = [&](pm_status st, const std::string& msg) {
    pm_batch_destroy(b);
    return bfail(nullptr, st, msg);
  };
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(PM_ERR_CUDA, "event or stream creation failed");
  b->sims.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    cudaStream_t st2;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(PM_ERR_CUDA, "stream creation failed");
    b->streams.push_back(st2);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return cleanup(PM_ERR_CUDA, "event creation failed");
    b->join.push_back(ev);
    pm_sim* s = nullptr;
    pm_status r = pm_create(&cfgs[i], b->arena + L.off[i], L.bytes[i], st2, &s);
    if (r != PM_OK) return cleanup(r, "member " + std::to_string(i) + ": " + g_create_error);
    b->sims[i] = s;
  }
  for (const BatchClass& BC : L.classes) {
    pm_batch::Class C;
    C.members = BC.members;
    C.stride = BC.stride;
    C.packed = BC.packed;
    if (cudaStreamCreateWithFlags(&C.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&C.join, cudaEventDisableTiming) != cudaSuccess) {
      b->classes.push_back(C);
      return cleanup(PM_ERR_CUDA, "class stream creation failed");
    }
    if (C.packed && !green_fused(b->sims[C.members[0]])) {  // fused members transform with their own 2D plans
      size_t w = 0;
      const pm_config& c = cfgs[C.members[0]];
      if (class_plans(c, int(C.members.size()), C.stride, &C.fwd, &C.inv, &w) != CUFFT_SUCCESS || w > BC.work ||
          cufftSetWorkArea(C.fwd, b->arena + BC.work_off) != CUFFT_SUCCESS ||
          cufftSetWorkArea(C.inv, b->arena + BC.work_off) != CUFFT_SUCCESS) {
        b->classes.push_back(C);
        return cleanup(PM_ERR_CUFFT, "batched transforms of a class could not be planned");
      }
    }
    b->classes.push_back(C);
  }
  *out = b;
  return PM_OK;
}

pm_status pm_batch_destroy(pm_batch* b) {
  if (!b) return PM_ERR_INVALID_ARG;
  for (pm_sim* s : b->sims)
    if (s) pm_destroy(s);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (auto& C : b->classes) {
    if (C.fwd) cufftDestroy(C.fwd);
    if (C.inv) cufftDestroy(C.inv);
    if (C.stream) cudaStreamDestroy(C.stream);
    if (C.join) cudaEventDestroy(C.join);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return PM_OK;
}

pm_sim* pm_batch_member(pm_batch* b, int32_t i) {
  if (!b || i < 0 || i >= int32_t(b->sims.size())) return nullptr;
  return b->sims[i];
}

pm_status pm_batch_run(pm_batch* b, int32_t nsteps, const double* a_start, const double* a_end) {
  if (!b) return PM_ERR_INVALID_ARG;
  if (!a_start || !a_end || nsteps < 1 || nsteps > PM_BATCH_MAX_STEPS)
    return bfail(b, PM_ERR_INVALID_ARG, "need a_start, a_end and 1 <= nsteps <= PM_BATCH_MAX_STEPS");
  const int n = int(b->sims.size());
  for (int i = 0; i < n; ++i) {
    pm_sim* s = b->sims[i];
    if (!s->have_particles) return bfail(b, PM_ERR_STATE, "member " + std::to_string(i) + " has no particles");
    if (s->cfg.cosmological && !(a_start[i] > 0 && a_end[i] > 0))
      return bfail(b, PM_ERR_INVALID_ARG, "member " + std::to_string(i) + ": a must be positive");
    if (s->prof_on) return bfail(b, PM_ERR_STATE, "profiling must be off during pm_batch_run");
  }
  auto member_error = [&](int i) { return bfail(b, PM_ERR_CUDA, "member " + std::to_string(i) + ": " + b->sims[i]->err); };
#define BCU(expr)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) return bfail(b, PM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  // per-member weights of every step (into each member's own table), and the closing half kicks
  std::vector<KickParams> tab(nsteps);
  std::vector<Weights> closing(n);
  BCU(cudaEventRecord(b->done, b->stream));
  BCU(cudaStreamWaitEvent(b->cap, b->done, 0));
  for (int i = 0; i < n; ++i) {
    pm_sim* s = b->sims[i];
    Weights pending = {0.0, 0.0};
    for (int k = 0; k < nsteps; ++k) tab[k] = step_params(s, k, nsteps, a_start[i], a_end[i], &pending);
    closing[i] = pending;
    // a pageable copy returns once the table is staged, so `tab` can be refilled
    BCU(cudaMemcpyAsync(s->at<KickParams>(s->L.ktab), tab.data(), size_t(nsteps) * sizeof(KickParams),
                        cudaMemcpyHostToDevice, b->cap));
    BCU(cudaMemsetAsync(s->errword() + 2, 0, sizeof(uint32_t), b->cap));
  }
  BCU(cudaEventRecord(b->fork, b->cap));
  // forces at the start of every member (outside the graph), on the member streams
  for (int i = 0; i < n; ++i) {
    BCU(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
    if (ensure_fields(b->sims[i]) != PM_OK) return member_error(i);
    BCU(cudaEventRecord(b->join[i], b->streams[i]));
    BCU(cudaStreamWaitEvent(b->cap, b->join[i], 0));
  }
  // which classes step packed this time (a common state is needed)
  std::vector<bool> packed(b->classes.size());
  b->last_packed = 0;
  for (size_t k = 0; k < b->classes.size(); ++k) {
    packed[k] = b->classes[k].packed && same_state(b->classes[k], b->sims);
    if (packed[k] && nsteps >= 2) b->last_packed += int(b->classes[k].members.size());
  }
  const int pairs = nsteps / 2;
  if (pairs > 0) {
    // capture two steps of every member (the record buffers alternate each step)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    pm_status st = PM_OK;
    if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) st = PM_ERR_CUDA;
    for (size_t k = 0; k < b->classes.size() && st == PM_OK; ++k) {
      pm_batch::Class& C = b->classes[k];
      if (packed[k]) {
        if (cudaStreamWaitEvent(C.stream, b->fork, 0) != cudaSuccess) st = PM_ERR_CUDA;
        for (int r = 0; r < 2 && st == PM_OK; ++r) st = packed_step(C, b->sims, C.stream);
        if (st == PM_OK && cudaEventRecord(C.join, C.stream) != cudaSuccess) st = PM_ERR_CUDA;
        if (st == PM_OK && cudaStreamWaitEvent(b->cap, C.join, 0) != cudaSuccess) st = PM_ERR_CUDA;
        if (st != PM_OK) b->err = "capture of a packed class failed: " + b->sims[C.members[0]]->err;
        continue;
      }
      for (int i : C.members) {
        pm_sim* s = b->sims[i];
        if (st == PM_OK && cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) st = PM_ERR_CUDA;
        for (int r = 0; r < 2 && st == PM_OK; ++r) st = table_step(s, s->at<KickParams>(s->L.ktab), s->errword() + 2);
        if (st == PM_OK && cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess) st = PM_ERR_CUDA;
        if (st == PM_OK && cudaStreamWaitEvent(b->cap, b->join[i], 0) != cudaSuccess) st = PM_ERR_CUDA;
        if (st != PM_OK) {
          b->err = "capture of member " + std::to_string(i) + " failed: " + s->err;
          break;
        }
      }
    }
    cudaError_t ec = cudaStreamEndCapture(b->cap, &graph);
    if (st != PM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return PM_ERR_CUDA;
    }
    if (ec != cudaSuccess) return bfail(b, PM_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(ec));
    ec = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return bfail(b, PM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
    for (int k = 0; k < pairs; ++k) {
      ec = cudaGraphLaunch(exec, b->cap);
      if (ec != cudaSuccess) break;
    }
    cudaGraphExecDestroy(exec);
    if (ec != cudaSuccess) return bfail(b, PM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(ec));
    for (int i = 0; i < n; ++i) b->sims[i]->krho_valid = false;  // the replayed stencils skipped K_rho
  }
  // an odd last step, then the closing half kicks, on the member streams
  BCU(cudaEventRecord(b->fork, b->cap));
  for (int i = 0; i < n; ++i) {
    pm_sim* s = b->sims[i];
    BCU(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
    if (nsteps & 1) {
      if (table_step(s, s->at<KickParams>(s->L.ktab), s->errword() + 2) != PM_OK) return member_error(i);
    }
    if (pass(s, closing[i], Weights{0.0, 0.0}, 0.0, true) != PM_OK) return member_error(i);
    BCU(cudaEventRecord(b->join[i], b->streams[i]));
    BCU(cudaStreamWaitEvent(b->cap, b->join[i], 0));
  }
  // and the caller's stream follows the batch
  BCU(cudaEventRecord(b->done, b->cap));
  BCU(cudaStreamWaitEvent(b->stream, b->done, 0));
#undef BCU
  return PM_OK;
}

pm_status pm_batch_info(const pm_batch* b, int32_t* classes, int32_t* packed_members) {
  if (!b || !classes || !packed_members) return PM_ERR_INVALID_ARG;
  *classes = int32_t(b->classes.size());
  *packed_members = b->last_packed;
  return PM_OK;
}

const char* pm_batch_last_error(const pm_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
