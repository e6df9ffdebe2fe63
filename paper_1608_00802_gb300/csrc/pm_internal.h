// Internal declarations shared by the host C-ABI (pm_api.cu) and the kernel
// translation units (pm_kernels_f32.cu, pm_kernels_f64.cu).
#pragma once
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

namespace pm {

// 32-byte record for the fp64 path (CUDA 13 deprecates the plain double4).
struct __align__(32) D4 {
  double x, y, z, w;
};

template <typename R> struct VT;
template <> struct VT<float> {
  using v4 = float4;
  using cplx = cufftComplex;
};
template <> struct VT<double> {
  using v4 = D4;
  using cplx = cufftDoubleComplex;
};

// Mesh geometry: N^3 nodes, node (x,y,z) at linear index (z*N + y)*N + x.
struct Mesh {
  int n;        // N
  int log2n;    // log2(N) when N is a power of two, else -1
  uint32_t n2;  // N^2
  uint32_t n3;  // N^3
};

// Leapfrog weights for one pass over the particles.  The momentum update is
//   p_sync = p - (cg1 grad phi + cq1 grad Q),  p_new = p_sync - (cg2 grad phi + cq2 grad Q)
// and the offsets (cell units) move by p_new * drift.
struct KickParams {
  double cg1, cq1, cg2, cq2;
  double drift;       // D/dx, 0 = no drift
  double inv_dx;      // 1/dx
  int grav_kernel;    // 1: gravity by the kernel gradient, 0: central mesh gradient
  int q_kernel;       // 1: Q by the kernel gradient (Eq. equationofmotion), 0: central
  int quantum;        // Q force on/off
  int diag;           // accumulate sum p_sync^2 and sum p_sync per block
  int accel_out;      // write -(cg1 grad phi + cq1 grad Q) to acc[id] and leave the state
  int maxima;         // leave the state; per-block maxima of |p_sync|^2, |grad phi|^2, |grad Q|^2
};

struct StencilParams {
  int step;           // 1 = compact Laplacian, 2 = wide
  double rho_floor;   // s = sqrt(max(rho, rho_floor))
  double rho_fp64;    // nodes below take the fp64 branch (fp32 path)
  double qcoef;       // -(hbar/m)^2 / 2 / (step*dx)^2
  // fp32 compact tiles: ty mesh rows x zlen planes per block with a ring of
  // `stages` bulk-copied planes; ty = 0 selects the register-column kernel
  int ty, zlen, stages;
  int diag;           // also write the K_rho partials (the fp32 compact kernels skip them otherwise)
};

// Launch shapes of one simulation (defaults by mesh size, or measured by the
// autotuner).  Kernel results do not depend on them; the diagnostic sums
// differ only in the grouping of their partial sums.
struct Tuning {
  int st_ty, st_zlen, st_stages;  // fp32 compact stencil tiles (see StencilParams)
  int kick_threads;               // 128 or 256
  int dep_warps;                  // warps per deposit block (one block per tile of mesh rows), 1..8
  int green_fused;                // fp32 cloud-in-cell: the Green multiplication inside the z transform
};
// smallest mesh whose simulations take the Green multiplication inside the z transform by default
constexpr int GREEN_FUSE_MIN_MESH = 128;
constexpr int KICK_MIN_THREADS = 128;

// Packed groups of simulations: member m of a group of equal configurations
// has every buffer at the same offset of its own arena, the arenas `ms` bytes
// apart, so a pointer of member 0 becomes member m's by moff(p, m * ms).
// Kernels that step a whole group take the member from a grid dimension
// (ms = 0 and one member for a single simulation).
template <typename T>
__host__ __device__ __forceinline__ T* moff(T* p, size_t off) {
  return p ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + off) : p;
}

// The Green multiplication between batched 2D transforms (fp32 cloud-in-cell,
// N a power of two in [16, 512]): one kernel transforms the half spectrum's
// columns along z, multiplies by the Green's function and transforms back;
// tiles of 16 columns, one W_g partial per tile.
bool spec_z_supported(int n);
int spec_z_tiles(int n);
// exp(-2 pi i t / N) for t < N (rounded from fp64) and sin^2(pi t / N) as k_green computes it
cudaError_t launch_spec_tables(float2* tw, float* s2, int n, cudaStream_t s);
cudaError_t launch_spec_z(void* spec, const float2* tw, const float* s2, Mesh m, double coef, double* part,
                          cudaStream_t s, const double* coefp = nullptr, int nm = 1, size_t ms = 0);

// error bits of the device error word
enum : uint32_t { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_TILE_SHIFT = 11;
static_assert(RS_TILE == (1 << RS_TILE_SHIFT), "RS_TILE is 2^RS_TILE_SHIFT");
// the drift counts its movers per tile (one word per tile), and the re-sort
// scans those counts into the movers before each tile (one more word per tile)
inline int64_t mover_count_words(int64_t n) { return (n + RS_TILE - 1) >> RS_TILE_SHIFT; }
constexpr int RS_MAX_BITS = 10;
// set in a sort key by the drift when the particle's cell changed (keys use at most 30 bits)
constexpr uint32_t KEY_MOVER = 0x80000000u;

constexpr int KICK_THREADS = 256;
constexpr int MESH_THREADS = 256;
constexpr int RED_GRID = 608;    // 4 blocks per SM on 152 SMs, fixed for deterministic reductions
constexpr int MESH_GRID = 1216;  // grid-stride mesh kernels with block partials (8 blocks per SM)
constexpr int PK_MAX_BINS = 512;

inline size_t radix_smem_bytes(int bits) {
  size_t radix = size_t(1) << bits;
  return (RS_WARPS * radix + 2 * radix + 2 * RS_TILE + 64) * sizeof(uint32_t);
}

template <typename R>
cudaError_t launch_init_particles(const double* x, const double* p, int64_t n, Mesh m, double inv_dx,
                                  void* pos, void* mom, uint32_t* keys, uint32_t* err, cudaStream_t s);
// n_dev (may be null): device word that overrides n (the grid is sized for n, which must bound it)
cudaError_t launch_sort_histogram(const uint32_t* keys, int64_t n, int passes, int digit_bits, int key_bits,
                                  uint32_t* hist, uint32_t* epoch, cudaStream_t s,
                                  const uint32_t* n_dev = nullptr);
template <typename R>
cudaError_t launch_sort_pass(bool last, const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int shift,
                             int bits, const uint32_t* digit_total, uint64_t* status, uint32_t* tile_counter,
                             const uint32_t* epoch, int pass, int ntiles, uint32_t* keys_out, uint32_t* vals_out,
                             const void* pos_in, const void* mom_in, void* pos_out, void* mom_out, uint32_t* err,
                             cudaStream_t s, const uint32_t* n_dev = nullptr, int nm = 1, size_t ms = 0,
                             int spin_limit = 0);  // polls of a look-back wait before it gives up (0: default)
// incremental re-sort after a drift (keys carry KEY_MOVER; tcount holds the
// drift's mover counts per tile and per group of tiles): stable partition
// into stayers (sk, sv) and movers (mk, mv) with per-row counts (rcnt: 3 N^2
// words, cleared before: stayers, movers, bucket fill), a scan of the row
// counts (btot: 2 ceil(N^2 / 4096) words; srow, mrow, row_start: N^2 + 1
// words), the movers in per-row buckets (bk, bv) and the placement of every
// particle: sorted keys to keys_out, records from (pos_in, mom_in) to
// (pos_out, mom_out) in sorted order.  stats (nullable): re-sorts and movers.
// part 0: the partition; 1: the rows (scan, buckets, movers' placement); 2:
// the stayers' placement (launched in this order).
template <typename R>
cudaError_t launch_resort(int part, const uint32_t* keys, int64_t n, const uint32_t* tcount, uint32_t* sk, uint32_t* sv,
                          uint32_t* mk, uint32_t* mv, uint32_t* bk, uint32_t* bv, uint32_t* counts, uint32_t* rcnt,
                          uint32_t* btot, uint32_t* srow, uint32_t* mrow, uint32_t* row_start, Mesh m,
                          unsigned long long* stats, uint32_t* keys_out, const void* pos_in, const void* mom_in,
                          void* pos_out, void* mom_out, int sms, cudaStream_t s, int nm = 1, size_t ms = 0);
inline size_t row_scan_tiles(int n_mesh) { return (size_t(n_mesh) * n_mesh + 1023) / 1024; }  // tiles of 1024 rows
cudaError_t launch_step_inc(uint32_t* step, cudaStream_t s, int nm = 1, size_t ms = 0);
// the x-y transforms of the z-planes of a 256^3 fp32 mesh, one kernel per direction (unnormalised,
// the layouts of the batched 2D R2C / C2R); tw: exp(-2 pi i t / 256), t < 256
bool xy_fft_supported(int n_mesh);
cudaError_t launch_xy_r2c(const float* rho, void* spec, const void* tw, int n_mesh, cudaStream_t s, int nm = 1,
                          size_t ms = 0);
cudaError_t launch_xy_c2r(const void* spec, float* phi, const void* tw, int n_mesh, cudaStream_t s, int nm = 1,
                          size_t ms = 0);
// row starts of sorted keys
cudaError_t launch_row_start(const uint32_t* keys, int64_t n, uint32_t n_mesh, uint32_t* row_start, cudaStream_t s);
// (nm, ms: a packed group of nm members, ms bytes apart; coefp/qcp: member
// 0's coefficient in device memory, read per member)
template <typename R>
cudaError_t launch_deposit(const void* pos, const uint32_t* row_start, int64_t n, Mesh m, double norm, R* rho,
                           cudaStream_t s, int warps = 8, int nm = 1, size_t ms = 0);
template <typename R>
cudaError_t launch_green(void* spec, Mesh m, double coef, double* part, cudaStream_t s,
                         const double* coefp = nullptr, int nm = 1, size_t ms = 0);
// cubic spline kernel: node weights, their normalised real symbol, the Green
// multiplication with the symbol (spec2 null: spec already holds rho_W^) and
// the smoothing of a transformed field
template <typename R>
cudaError_t launch_spline_weights(void* w, Mesh m, double hc, cudaStream_t s);
template <typename R>
cudaError_t launch_spline_symbol(const void* spec, void* what, Mesh m, cudaStream_t s);
template <typename R>
cudaError_t launch_green_spline(void* spec, void* spec2, const void* what, Mesh m, double coef, double* part,
                                cudaStream_t s, int smooth_in);
// the spline smoothing in real space for supports within three cells (fp32):
// g[s*4 + i] = normalised node weight at squared distance i^2 + s (s <= 18);
// maxr2: the largest squared distance with a nonzero weight
template <typename R>
cudaError_t launch_smooth_direct(const R* in, R* out, Mesh m, const double* g, int maxr2, cudaStream_t s);
template <typename R>
cudaError_t launch_smooth_spec(void* spec, const void* what, Mesh m, cudaStream_t s);
template <typename R>
cudaError_t launch_stencil(const R* rho, Mesh m, StencilParams sp, R* q, double* part, uint32_t* list,
                           uint32_t* list_count, uint32_t* err, cudaStream_t s, const double* qcp = nullptr,
                           int nm = 1, size_t ms = 0);
// fp32 stencil tiling (defined with the kernels): list length of the
// register-column kernel, blocks (= K_rho partials) of a shape and the most
// over every valid shape, shape validity and the default shape
size_t stencil_list_entries(int n);
int stencil_launch_blocks(int n, int ty, int zlen);
int stencil_max_blocks(int n);
bool stencil_shape_ok(int n, int ty, int zlen, int stages);
Tuning default_tuning(int n);
// sizes the fp32 streaming kick's grid for this device (an occupancy query;
// call outside any stream capture, before the first kick)
void kick_stream_prepare();
// updates the records in place; with a drift also the keys and the mover
// counts tcount (cleared before)
template <typename R>
cudaError_t launch_kick(void* pos, void* mom, uint32_t* keys, uint32_t* tcount, int64_t n, const R* phi, const R* q,
                        Mesh m, KickParams kp,
                        const KickParams* kp_tab, const uint32_t* step, double* part, double* acc, uint32_t* err,
                        int threads, cudaStream_t s, int nm = 1, size_t ms = 0);
template <typename R>
cudaError_t launch_power(const void* spec, Mesh m, int nbins, double* part, cudaStream_t s);
cudaError_t launch_reduce(const double* part, int nblocks, int nvals, double* out, cudaStream_t s);
// out[v] = max_b part[v*nblocks + b]
cudaError_t launch_reduce_max(const double* part, int nblocks, int nvals, double* out, cudaStream_t s);
template <typename R>
cudaError_t launch_get_particles(const void* pos, const void* mom, int64_t n, Mesh m, double dx, double* x,
                                 double* p, cudaStream_t s);
template <typename R>
cudaError_t launch_get_order(const void* pos, const void* mom, int64_t n, uint32_t* cell, uint32_t* id,
                             cudaStream_t s);
template <typename R>
cudaError_t launch_to_double(const R* f, int64_t n, double* out, cudaStream_t s);
template <typename R>
cudaError_t launch_from_double(const double* f, int64_t n, R* out, cudaStream_t s);

// stores the message that pm_last_error(NULL) returns (host side)
void set_global_error(const char* msg);

inline int kick_blocks(int64_t n, int threads = KICK_THREADS) { return int((n + threads - 1) / threads); }

}  // namespace pm
