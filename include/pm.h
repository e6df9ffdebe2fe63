/*
 * pm.h - C ABI of the GB300 particle-mesh step with quantum pressure.
 *
 * Method: Veltmaat & Niemeyer, "Cosmological particle-in-cell simulations with
 * ultralight axion dark matter", arXiv:1608.00802, Sec. II.A and Sec. III.
 * Each step (i) deposits the particle density on a periodic mesh with a
 * kernel estimate (Eq. rhodis: the cloud-in-cell kernel, or the paper's cubic
 * spline of Sec. II.A through PM_KERNEL_SPLINE), (ii) solves
 * the gravity potential and evaluates the quantum pressure
 * Q = -(hbar^2/2m^2) lap(sqrt rho)/sqrt rho (Eq. quantumpressure, comoving
 * form Eq. comquantumpressure) with a seven-point Laplacian, (iii) turns both
 * potentials into particle forces (central mesh gradient or the kernel-gradient
 * form of Eq. equationofmotion) inside a kick-drift-kick leapfrog.
 *
 * Units: length Mpc/h, time 1/H0 (H0 = 1), mean comoving density 1 (so
 * 4 pi G rho_bar = 3/2 Omega_m and a particle weighs box^3/n_part), momentum
 * p = a^2 dx/dt.  Mesh node n sits at n*box/n_mesh; mesh arrays are
 * row-major [z][y][x] with x fastest.  Static (non-cosmological) runs use
 * a = 1 and take the time t where a cosmological run takes the scale factor.
 *
 * Memory and threads: the caller owns one device buffer (the arena, sized by
 * pm_arena_bytes) and one CUDA stream; the library sub-allocates the arena and
 * enqueues all work on that stream.  cuFFT keeps its plan tables in its own
 * device memory; everything else lives in the arena.  Host arrays stay owned
 * by the caller and are copied.  A pm_sim is used from one host thread at a
 * time.  Entry points return a pm_status and never abort; pm_last_error gives
 * the message of the last failure.  Calls marked "async" return once the
 * work is enqueued; calls marked "sync" wait for the stream.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_ABI_VERSION 1

typedef enum {
  PM_OK = 0,
  PM_ERR_INVALID_ARG = 1, /* a pointer, size or configuration value is out of range */
  PM_ERR_NO_MEMORY = 2,   /* the arena passed to pm_create is smaller than pm_arena_bytes */
  PM_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in pm_last_error) */
  PM_ERR_CUFFT = 4,       /* a cuFFT call failed */
  PM_ERR_NONFINITE = 5,   /* a NaN/Inf reached a particle or a diagnostic */
  PM_ERR_STATE = 6,       /* call out of order (e.g. no particles set yet) */
  PM_ERR_TIMEOUT = 7      /* a bounded device-side wait gave up (results of that call are invalid) */
} pm_status;

/* how a mesh potential becomes a particle force (Sec. II.A, step (iii)) */
enum {
  PM_FORCE_MESHGRAD = 0,   /* gravity and Q: central-difference mesh gradient, CIC-interpolated */
  PM_FORCE_HYBRID = 1,     /* gravity as MESHGRAD; Q by Eq. equationofmotion (sum_n Q_n grad W) */
  PM_FORCE_LAGRANGIAN = 2  /* gravity and Q by the kernel gradient: conserves the discrete energies */
};
/* seven-point Laplacian in Q (the operator named after Eq. equationofmotion) */
enum {
  PM_LAP_COMPACT = 0,      /* neighbours at +-dx; pairs with forward differences in K_rho */
  PM_LAP_WIDE = 1          /* neighbours at +-2dx; pairs with the central differences of Eq. diskpoten */
};
enum { PM_FP32 = 0, PM_FP64 = 1 };
/* Density kernel of Eq. rhodis.  SPLINE: the cubic spline W(r, h) of Sec. II.A
 * (h = smooth_h mesh cells), applied as the periodic convolution of the
 * cloud-in-cell density with W sampled at the nodes (normalised to unit sum);
 * the potentials the particles feel are convolved once more (the transpose),
 * so the kernel-gradient forces stay the derivatives of the discrete energies. */
enum { PM_KERNEL_CIC = 0, PM_KERNEL_SPLINE = 1 };
enum { PM_FIELD_RHO = 0, PM_FIELD_PHI = 1, PM_FIELD_Q = 2 };

typedef struct {
  int64_t n_part;      /* number of particles, 1 .. 2^31-1 */
  int32_t n_mesh;      /* N: the mesh has N^3 nodes; even, 8 .. 1024 */
  int32_t precision;   /* PM_FP32: int32 cell + fp32 offset positions, fp32 mesh and FFT;
                          PM_FP64: fp64 offsets, momenta, mesh and FFT */
  double box;          /* periodic box side L [Mpc/h] */
  double omega_m;      /* matter density today; 4 pi G rho_bar = 3/2 omega_m */
  double omega_l;      /* cosmological constant today */
  double h;            /* H0 / (100 km/s/Mpc), sets hbar/m in code units */
  double m22;          /* axion mass / 1e-22 eV (Sec. II.A uses 2.5) */
  int32_t quantum;     /* 0: quantum pressure off (CDM), 1: on */
  int32_t force_mode;  /* PM_FORCE_* */
  int32_t lap;         /* PM_LAP_* */
  int32_t cosmological;/* 1: comoving equations with a(t); 0: static, a = 1 */
  double rho_floor;    /* sqrt(rho) uses max(rho, rho_floor) (units of the mean); Q is
                          undefined where rho = 0 (Sec. II.A).  > 0; with PM_FP32 >= 1e-30 */
  double rho_fp64;     /* PM_FP32 only: near-empty nodes (rho below this) whose fp32 Laplacian
                          of sqrt(rho) is ill-conditioned (the six neighbours' sqrt values
                          plus 6 sqrt(rho) above 4 |Laplacian|) evaluate sqrt(rho) and Q in float-float
                          (~48-bit significand) instead of fp32; 0 disables */
  int32_t kernel;      /* PM_KERNEL_* */
  int32_t reserved;    /* 0 */
  double smooth_h;     /* PM_KERNEL_SPLINE: smoothing length h in mesh cells, 1 .. n_mesh/4
                          (the paper's cosmological runs: 3.5) */
  int32_t fft_jit;     /* 1: plan the transforms (3D, and the batched 2D ones of green_fused) in cuFFT's
                          patient JIT mode (kernels chosen and
                          linked at pm_create: a slower creation, ~6 % faster transforms at 256^3 on a
                          GB300; for long-lived simulations), 0: default plans */
  int32_t smooth_real; /* PM_KERNEL_SPLINE, PM_FP32, smooth_h <= 4, n_mesh <= 512: 1 smooths the density and Q
                          by a direct sum over the node weights in real space (each node keeps the relative
                          precision of its neighbours even where the field is near zero; slower than the
                          transforms at 256^3 on a GB300), 0: by the transforms (default) */
} pm_config;

typedef struct pm_sim pm_sim;

/* Fills a configuration with defaults (fp32, MESHGRAD, compact, quantum on,
 * cosmological, Omega_m 0.3, Omega_L 0.7, h 0.7, m22 2.5, floor 1e-6,
 * fp64 branch below 1e-2, cloud-in-cell kernel, smooth_h 3.5).  n_part,
 * n_mesh and box are left 0. */
void pm_config_default(pm_config* cfg);

/* hbar/m in code units (Mpc/h)^2 H0 for the configuration's m22 and h. */
double pm_hbar_over_m(const pm_config* cfg);

/* Device bytes the arena must hold for this configuration (includes the cuFFT
 * work area; needs a current CUDA device).  0 if the configuration is invalid. */
size_t pm_arena_bytes(const pm_config* cfg);

/* Creates a simulation in the caller's arena (>= pm_arena_bytes bytes,
 * 256-byte aligned device memory) bound to the caller's cudaStream_t `stream`
 * (NULL = legacy default stream).  Builds the cuFFT plans.  Sync. */
pm_status pm_create(const pm_config* cfg, void* dev_arena, size_t arena_bytes,
                    void* stream, pm_sim** out);

/* Destroys the cuFFT plans and the handle; the arena stays the caller's. Sync. */
pm_status pm_destroy(pm_sim* sim);

/* Loads n_part particles from host arrays x[n][3] (positions in [0, box),
 * wrapped periodically otherwise) and p[n][3] (momenta a^2 dx/dt).  The input
 * index is the particle's id.  Converts positions to an integer cell plus an
 * offset in [0,1) and sorts by cell.  Sync. */
pm_status pm_set_particles(pm_sim* sim, const double* x, const double* p);

/* Copies positions and momenta back in id order (x = (cell + offset) dx). Sync. */
pm_status pm_get_particles(pm_sim* sim, double* x, double* p);

/* Step (i): sorts the particles by cell and deposits the cloud-in-cell
 * density rho_n = sum_i m_i W(x_n - q_i)/dx^3 (Eq. rhodis) by a deterministic
 * gather.  rho_host (nullable) receives the N^3 densities (sync); otherwise
 * async. */
pm_status pm_deposit(pm_sim* sim, double* rho_host);

/* Steps (i)-(iii) at scale factor a: acc_host[n][3] (id order) receives
 * dp/dt = -grad(phi)/a - grad(Q~)/a^2 with lap7 phi = 3/2 Omega_m (rho - 1)
 * and Q~ = -(hbar/m)^2/2 lap7(sqrt rho)/sqrt rho.  Sync. */
pm_status pm_forces(pm_sim* sim, double a, double* acc_host);

/* One kick-drift-kick step from a0 to a1 (the leapfrog of Sec. II.A; half
 * point sqrt(a0 a1), or (t0+t1)/2 in static runs).  Forces at a0 are reused
 * from the previous step when valid.  Async. */
pm_status pm_step(pm_sim* sim, double a0, double a1);

/* nsteps leapfrog steps from a_start to a_end, uniform in ln a (in t for static
 * runs), with the closing half kick of each step merged into the opening half
 * kick of the next; momenta are synchronised at a_end.  For
 * 2 <= nsteps <= PM_RUN_GRAPH_MAX_STEPS (and the profiler off) two steps run as
 * one CUDA graph on an internal stream (joined to the simulation's stream by
 * events); the graphs are captured at the first such call and kept until
 * pm_destroy.  Async. */
#define PM_RUN_GRAPH_MAX_STEPS 4096
pm_status pm_run(pm_sim* sim, int32_t nsteps, double a_start, double a_end);

/* Leapfrog from a_start to a_end with adaptive steps (Sec. II.A: the time
 * step keeps every particle within one cell width per step, the quantum
 * acceleration included).  Each step first finds max|p_sync|, max|grad phi~|
 * and max|grad Q~| over the particles, then ends at the largest a1 <= a_end
 * for which (max|p_sync| + K_g(a, a_h) max|grad phi~| + K_q(a, a_h) max|grad Q~|)
 * D(a, a1) <= cfl * dx, an upper bound of every particle's drift (a_h the
 * half point, K and D the kick and drift weights); cfl in (0, 1].  Stops at
 * a_end or after max_steps steps; the momenta are synchronised at the end.
 * a_steps (nullable, max_steps + 1 doubles) receives the step boundaries,
 * steps_taken (nullable) their number.  Static runs step in t.  Sync (one
 * small device-to-host read per step). */
pm_status pm_run_adaptive(pm_sim* sim, double a_start, double a_end, double cfl, int32_t max_steps,
                          double* a_steps, int32_t* steps_taken);

/* Energies at scale factor a for the current particles (momenta synchronised):
 * out = {K_v (Eq. diskkinen), W_g = (1/2a) sum (rho-1) phi dx^3,
 *        K_rho (Eq. diskpoten; forward differences for the compact Laplacian,
 *        the printed central differences for the wide one), P_x, P_y, P_z}.
 * Reductions in fp64.  Sync. */
pm_status pm_energy(pm_sim* sim, double a, double out[6]);

/* Power spectrum of delta = rho - 1 on the CIC mesh, deconvolved by the CIC
 * window: P = (L^3/N^6) |delta_k|^2 / prod_d sinc^4(k_d dx/2), shells
 * i = 1..nbins (nbins <= N/2) of width k_f = 2 pi/L centred on i k_f, over
 * the full grid.  k[i], P[i]: shell means; nmodes[i]: mode count.  Sync. */
pm_status pm_power_spectrum(pm_sim* sim, int32_t nbins, double* k, double* P,
                            int64_t* nmodes);

/* Copies a mesh field (PM_FIELD_RHO, PM_FIELD_PHI = phi~, PM_FIELD_Q = Q~) of
 * the last force evaluation to host memory as N^3 doubles.  Sync. */
pm_status pm_get_field(pm_sim* sim, int32_t which, double* host_out);

/* Replaces the density by host values (N^3 doubles) and evaluates phi~ and Q~
 * from it, so mesh stages can be checked on prescribed fields.  Sync. */
pm_status pm_set_density(pm_sim* sim, const double* rho_host);

/* Current storage order: cell key (iz*N+iy)*N+ix and id of each slot. Sync. */
pm_status pm_get_order(pm_sim* sim, uint32_t* cell, uint32_t* id);

/* ---- launch shapes and the autotuner ---------------------------------------
 * Each simulation launches its kernels in shapes chosen for its mesh size (a
 * default from the mesh size, or measured by pm_autotune).  The mesh fields,
 * forces and particle states do not depend on the shapes; the diagnostic sums
 * of pm_energy differ only by the grouping of their partial sums. */
typedef struct {
  int32_t stencil_rows;    /* fp32 compact stencil: mesh rows per block (1, 2, 4 or 8, dividing n_mesh,
                              n_mesh a multiple of 4), the block's density arriving by bulk copies;
                              0 = the register-column kernel (any even n_mesh) */
  int32_t stencil_planes;  /* z planes per stencil block: 2..16 for one-shot tiles, 4..n_mesh for
                              sweeps (ignored when stencil_rows = 0) */
  int32_t stencil_stages;  /* 0 = one-shot tile (the block loads its whole input at once); 4..8 = a
                              sweep along z through a ring of that many planes (ignored when rows = 0) */
  int32_t kick_threads;    /* threads (particles) per interpolate+kick+drift block: 128 or 256 */
  int32_t deposit_warps;   /* warps per deposit block (each warp owns a tile of up to 2 x 4 mesh rows): 1..8 */
  int32_t green_fused;     /* PM_FP32 cloud-in-cell on a power-of-two mesh of 16..512 only: 1 transforms the
                              planes of constant z with batched 2D transforms and does the z transforms, the
                              Green multiplication and the inverse z transforms in one kernel between them
                              (the spectrum crosses device memory once instead of three times; the default
                              where it applies); 2 (256^3 meshes only, their default) does the same with
                              the x and y transforms of each plane in one kernel per direction (a cluster of
                              CTAs per plane) instead of the batched 2D cuFFT plans; 0 uses the 3D
                              transforms and a separate Green pass.  The potential agrees to fp32 rounding
                              in every mode */
} pm_tuning;

/* Current shapes. */
pm_status pm_get_tuning(pm_sim* sim, pm_tuning* out);

/* Sets the shapes (e.g. a cached autotuner result).  PM_ERR_INVALID_ARG if a
 * value is outside the ranges above or the stencil tile does not fit the mesh
 * or the 227 KB of shared memory of a block.  Drops captured steps; the next
 * force evaluation recomputes the fields.  Sync. */
pm_status pm_set_tuning(pm_sim* sim, const pm_tuning* t);

/* Times the candidate shapes of the stencil, the deposit and the kick on this
 * simulation's current state (reps launches each, after one untimed), keeps
 * the fastest of each and returns them in `out` (may be null).  Needs
 * particles (PM_ERR_STATE).  The state is not changed; the fields are
 * recomputed with the chosen shapes.  Sync. */
pm_status pm_autotune(pm_sim* sim, int32_t reps, pm_tuning* out);

/* Stages timed by the profiler (one CUDA-event pair per launch, recorded on
 * the simulation's stream).  The cuFFT stages cover one cufftExec call each. */
enum {
  PM_STAGE_SORT_HISTOGRAM = 0, PM_STAGE_SORT_PASS = 1, PM_STAGE_ROW_START = 2, PM_STAGE_DEPOSIT = 3,
  PM_STAGE_FFT_R2C = 4, PM_STAGE_GREEN = 5, PM_STAGE_FFT_C2R = 6, PM_STAGE_STENCIL = 7, PM_STAGE_KICK = 8,
  PM_STAGE_SORT_PARTITION = 9, PM_STAGE_SORT_MERGE = 10, PM_STAGE_OTHER = 11, PM_NSTAGES = 12
};

/* Test aid for the bounded device waits: runs one radix pass of the
 * particles' keys in which no block takes the first tile, so the decoupled
 * look-back of the second tile waits on a predecessor that never publishes;
 * after spin_limit polls the wait gives up and sets the timeout bit of the
 * error word instead of hanging.  Returns the status that produces
 * (PM_ERR_TIMEOUT); only scratch buffers are written, so the simulation stays
 * usable.  Needs more than 2048 particles.  Sync. */
pm_status pm_debug_sort_timeout(pm_sim* sim, int32_t spin_limit);

/* Incremental re-sorts since pm_create (one per drift of the particles) and
 * the particles they moved to another cell, summed on the device.  Sync. */
pm_status pm_sort_stats(pm_sim* sim, int64_t* resorts, int64_t* movers);

/* ---- checkpoint and resume -------------------------------------------------
 * A checkpoint holds what the steps continue from: the particle records in
 * storage order (cell, offsets, momenta, id), the sorted cell keys and their
 * flags, the re-sort statistics and the launch shapes.  The momenta a run
 * leaves are synchronised with the positions (every pm_run / pm_step ends with
 * its closing half kick), so a checkpoint taken between calls and loaded into a
 * simulation of the same n_part, n_mesh, precision and kernel (a new one, or
 * the same) continues on the same bits as the uninterrupted run: the mesh fields
 * are recomputed from the records when next needed.  The scale factor is the
 * caller's (it passes a to every call).  Layout: a 256-byte header (magic,
 * version, sizes, flags, shapes, statistics), then the position records, the
 * momentum records (16 bytes each in PM_FP32, 32 in PM_FP64) and the keys
 * (4 bytes each), host byte order. */
size_t pm_checkpoint_bytes(const pm_sim* sim);

/* Writes the checkpoint to `host` (>= pm_checkpoint_bytes bytes).  PM_ERR_STATE
 * without particles, PM_ERR_INVALID_ARG for a short buffer.  Sync. */
pm_status pm_save(pm_sim* sim, void* host, size_t bytes);

/* Replaces the simulation's particles, keys, statistics and launch shapes by a
 * checkpoint's.  PM_ERR_INVALID_ARG if the buffer is short or its header does
 * not match this simulation (magic, version, n_part, n_mesh, precision,
 * kernel); the simulation is unchanged then.  Sync. */
pm_status pm_load(pm_sim* sim, const void* host, size_t bytes);

/* Starts recording a CUDA-event pair around every launch of this handle, for
 * up to `capacity` launches (events are created here, before any timed work).
 * Async. */
pm_status pm_profile_begin(pm_sim* sim, int32_t capacity);

/* Stops recording, waits for the stream and returns per stage the summed
 * device time in ms and the number of launches (arrays of PM_NSTAGES).  Sync. */
pm_status pm_profile_end(pm_sim* sim, double* ms, int64_t* launches);

/* ---- batches of independent simulations ------------------------------------
 * A batch steps many simulations of different sizes together on one GPU (the
 * paper's runs are independent; the batch is only an execution unit).  Each
 * member is an ordinary pm_sim (use pm_batch_member with the single-simulation
 * calls: pm_set_particles, pm_energy, pm_get_particles, ...) with its own
 * stream.  Members of equal configuration apart from box, mass and cosmology
 * form a class and sit in the batch arena at a fixed stride; pm_batch_run
 * steps each class with one launch per kernel over all its members and one
 * batched cuFFT plan (see pm_batch_info), captures two leapfrog steps of all
 * classes as one CUDA graph (classes run concurrently inside it) and replays
 * it, so a step costs one graph launch.  Per-step kick and drift weights come
 * from a table in each member's arena indexed by its step counter on the
 * device. */
typedef struct pm_batch pm_batch;
#define PM_BATCH_MAX_STEPS 8192

/* Device bytes of a batch arena for n member configurations (0 if one is invalid). */
size_t pm_batch_arena_bytes(const pm_config* cfgs, int32_t n);

/* Creates n members (1 <= n <= 4096) in the caller's arena, each on a new
 * stream; `stream` is the batch's own stream (NULL = legacy default).  Sync. */
pm_status pm_batch_create(const pm_config* cfgs, int32_t n, void* dev_arena, size_t arena_bytes, void* stream,
                          pm_batch** out);

/* Destroys the members, their streams and the graph; the arena stays the caller's. Sync. */
pm_status pm_batch_destroy(pm_batch* b);

/* Member i (0-based), or NULL if out of range.  Owned by the batch. */
pm_sim* pm_batch_member(pm_batch* b, int32_t i);

/* nsteps leapfrog steps for every member, member i from a_start[i] to a_end[i]
 * (uniform in ln a, or in t for static members), the same steps as pm_run;
 * momenta are synchronised at the end.  1 <= nsteps <= PM_BATCH_MAX_STEPS.
 * Async with respect to the host; the batch stream waits for all members. */
pm_status pm_batch_run(pm_batch* b, int32_t nsteps, const double* a_start, const double* a_end);

/* Classes of the batch (members of equal configuration apart from box, mass
 * and cosmology) and the members the last pm_batch_run stepped by packed
 * launches: one launch per kernel and one batched cuFFT transform per class
 * (fp32 cloud-in-cell classes of two or more members in one common state, with
 * one-shot stencil tiles); the others step member by member. */
pm_status pm_batch_info(const pm_batch* b, int32_t* classes, int32_t* packed_members);

/* Message of the last failure of a batch call. */
const char* pm_batch_last_error(const pm_batch* b);

/* ---- allocation-free deposit ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: cudaFree synchronises the whole device and
 * cudaMalloc may block, which a latency-critical serving loop or a real-time
 * thread cannot afford, and a process that has already given its whole device
 * memory budget to fixed arenas has nothing left to allocate from.
 *
 * pm_deposit_noalloc computes the same cloud-in-cell density as pm_deposit
 * (step (i); fp32 path: cell + offset positions, stable radix sort by cell,
 * deterministic gather; the same bits as pm_deposit on the same positions)
 * from n_part positions x_dev (device memory, n_part x 3 doubles in [0, box),
 * wrapped periodically otherwise) into rho_dev (device memory, n_mesh^3
 * floats, [z][y][x], mean 1), enqueued on the cudaStream_t `stream` (NULL =
 * legacy default stream); async.  err_dev (nullable; device memory or mapped
 * pinned host memory) receives, in stream order after the deposit, the
 * call's device error bits: 0 = ok, bit 0 (1) = a non-finite position was
 * placed at 0, bit 1 (2) = a bounded wait of the sort gave up and rho_dev is
 * invalid.  The host return value cannot report these without a
 * synchronisation, which this entry point does not make.  It calls no
 * cudaMalloc, cudaFree or allocating library routine: all temporaries live
 * in one file-scope static device array of PM_NOALLOC_SCRATCH_BYTES, which
 * every GPU that loads the library holds until the process exits.  Limits:
 * 1 <= n_part <= PM_NOALLOC_MAX_PARTICLES and n_mesh even in
 * [8, PM_NOALLOC_MAX_MESH]; larger sizes return PM_ERR_INVALID_ARG and
 * pm_last_error(NULL) says which limit was exceeded.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture, and do not reset the device
 * (cudaDeviceReset) after it.  Every call reuses the same array and clears
 * what must start at zero, so calls that overlap on the GPU (other streams,
 * other host threads) race: serialise them. */
#define PM_NOALLOC_MAX_PARTICLES 65536
#define PM_NOALLOC_MAX_MESH 128
#define PM_NOALLOC_SCRATCH_BYTES (8u << 20)
pm_status pm_deposit_noalloc(const double* x_dev, int64_t n_part, int32_t n_mesh, double box, float* rho_dev,
                             uint32_t* err_dev, void* stream);

/* Message of the last failure on this handle (or of the last pm_create
 * failure when sim is NULL). */
const char* pm_last_error(const pm_sim* sim);

#ifdef __cplusplus
}
#endif
#endif /* PM_H */
