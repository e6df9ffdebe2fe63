// fp32 instantiation of the step kernels, plus the type-independent launchers.
#include "pm_kernels.cuh"
#include "pm_sort.cuh"
#include "pm_instantiate.cuh"

namespace pm {

// the device step counters of nm members (ms bytes apart)
static __global__ void k_step_inc(uint32_t* step, int nm, size_t ms) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < nm) *moff(step, size_t(m) * ms) += 1u;
}

cudaError_t launch_step_inc(uint32_t* step, cudaStream_t s, int nm, size_t ms) {
  k_step_inc<<<unsigned((nm + 255) / 256), 256, 0, s>>>(step, nm, ms);
  return cudaGetLastError();
}

cudaError_t launch_sort_histogram(const uint32_t* keys, int64_t n, int passes, int digit_bits, int key_bits,
                                  uint32_t* hist, uint32_t* epoch, cudaStream_t s, const uint32_t* n_dev) {
  int64_t blocks = (n + RS_THREADS * 16 - 1) / (RS_THREADS * 16);
  if (blocks > 2 * 152) blocks = 2 * 152;
  if (blocks < 1) blocks = 1;
  k_sort_histogram<<<unsigned(blocks), RS_THREADS, 0, s>>>(keys, n, passes, digit_bits, key_bits, hist, epoch,
                                                            n_dev);
  return cudaGetLastError();
}

cudaError_t launch_row_start(const uint32_t* keys, int64_t n, uint32_t n_mesh, uint32_t* row_start, cudaStream_t s) {
  k_row_start<<<unsigned((n + 1 + 255) / 256), 256, 0, s>>>(keys, n, n_mesh, n_mesh * n_mesh, row_start);
  return cudaGetLastError();
}

size_t stencil_list_entries(int n) { return stencil_list_len(n); }

void kick_stream_prepare() {
  for (int fm : {KICK_FM_ANY, KICK_FM_HYBRID_Q}) {
    kick_stream_resident<float>(128, fm);
    kick_stream_resident<float>(256, fm);
  }
}

int stencil_launch_blocks(int n, int ty, int zlen) {
  if (ty <= 0) return stencil_blocks(n);
  return (n / ty) * ((n + zlen - 1) / zlen);
}

// most blocks of any valid shape: one row per block, two planes (one-shot tiles)
int stencil_max_blocks(int n) {
  const int most = n * ((n + 1) / 2);
  return most > stencil_blocks(n) ? most : stencil_blocks(n);
}

bool stencil_shape_ok(int n, int ty, int zlen, int stages) {
  if (ty == 0) return true;
  return stages == 0 ? stencil_tile_shape_ok(n, ty, zlen) : stencil_bulk_shape_ok(n, ty, zlen, stages);
}

Tuning default_tuning(int n) {
  Tuning t;
  t.kick_threads = KICK_THREADS;
  t.dep_warps = 8;
  t.green_fused = 0;
  // one-shot tiles of 4 rows x 4 planes where they fit (the multiple-of-4 meshes up to 1024)
  if (stencil_tile_shape_ok(n, 4, 4)) {
    t.st_ty = 4;
    t.st_zlen = 4;
    t.st_stages = 0;
    return t;
  }
  t.st_ty = n <= 256 ? 4 : (n <= 512 ? 2 : 1);
  t.st_zlen = n < 16 ? n : 16;
  t.st_stages = 6;
  while (t.st_ty > 0 && !stencil_bulk_shape_ok(n, t.st_ty, t.st_zlen, t.st_stages)) {
    if (t.st_stages > 4) {
      --t.st_stages;
    } else {
      t.st_ty >>= 1;
      t.st_stages = 6;
    }
  }
  if (t.st_ty == 0) t.st_zlen = t.st_stages = 0;  // the register-column kernel
  return t;
}

cudaError_t launch_reduce_max(const double* part, int nblocks, int nvals, double* out, cudaStream_t s) {
  if (nvals <= 0) return cudaSuccess;
  k_reduce_max<<<nvals, 256, 0, s>>>(part, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* part, int nblocks, int nvals, double* out, cudaStream_t s) {
  if (nvals <= 0) return cudaSuccess;
  k_reduce<<<nvals, 256, 0, s>>>(part, nblocks, out);
  return cudaGetLastError();
}

PM_INSTANTIATE(float)
template cudaError_t launch_smooth_direct<float>(const float*, float*, Mesh, const double*, int, cudaStream_t);


// ---------------------------------------------------------------- Green's function inside the z transform
bool spec_z_supported(int n) { return n >= 16 && n <= 512 && (n & (n - 1)) == 0; }
int spec_z_tiles(int n) { return n * (n / 2 + 1) / SPZ_COLS; }

cudaError_t launch_spec_tables(float2* tw, float* s2, int n, cudaStream_t s) {
  if (!spec_z_supported(n)) return cudaErrorInvalidValue;
  // the 512-point blocks take 70 KB of shared memory (set once, outside any stream capture)
  static bool done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !done[dev]) {
    const int most = 512 * int(SPZ_COLS * sizeof(float2) + sizeof(float2) + sizeof(float));
    e = cudaFuncSetAttribute(k_spec_z<32, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_spec_z<32, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  k_spec_tables<<<(n + 255) / 256, 256, 0, s>>>(tw, s2, n);
  return cudaGetLastError();
}

cudaError_t launch_spec_z(void* spec, const float2* tw, const float* s2, Mesh m, double coef, double* part,
                          cudaStream_t s, const double* coefp, int nm, size_t ms) {
  float2* sp = static_cast<float2*>(spec);
  switch (m.n) {
    case 16: return launch_spec_z_pq<4, 4>(sp, tw, s2, coef, part, s, coefp, nm, ms);
    case 32: return launch_spec_z_pq<8, 4>(sp, tw, s2, coef, part, s, coefp, nm, ms);
    case 64: return launch_spec_z_pq<8, 8>(sp, tw, s2, coef, part, s, coefp, nm, ms);
    case 128: return launch_spec_z_pq<16, 8>(sp, tw, s2, coef, part, s, coefp, nm, ms);
    case 256: return launch_spec_z_pq<16, 16>(sp, tw, s2, coef, part, s, coefp, nm, ms);
    case 512: return launch_spec_z_pq<32, 16>(sp, tw, s2, coef, part, s, coefp, nm, ms);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pm
