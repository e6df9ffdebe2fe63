// fp32 instantiation of the step kernels, plus the type-independent launchers.
#include "pm_kernels.cuh"
#include "pm_sort.cuh"

namespace pm {

static __global__ void k_step_inc(uint32_t* step) { *step += 1u; }

cudaError_t launch_step_inc(uint32_t* step, cudaStream_t s) {
  k_step_inc<<<1, 1, 0, s>>>(step);
  return cudaGetLastError();
}

cudaError_t launch_sort_histogram(const uint32_t* keys, int64_t n, int passes, int digit_bits, int key_bits,
                                  uint32_t* hist, uint32_t* epoch, cudaStream_t s) {
  int64_t blocks = (n + RS_THREADS * 16 - 1) / (RS_THREADS * 16);
  if (blocks > 2 * 152) blocks = 2 * 152;
  if (blocks < 1) blocks = 1;
  k_sort_histogram<<<unsigned(blocks), RS_THREADS, 0, s>>>(keys, n, passes, digit_bits, key_bits, hist, epoch);
  return cudaGetLastError();
}

cudaError_t launch_row_start(const uint32_t* keys, int64_t n, uint32_t n_mesh, uint32_t* row_start, cudaStream_t s) {
  k_row_start<<<unsigned((n + 1 + 255) / 256), 256, 0, s>>>(keys, n, n_mesh, n_mesh * n_mesh, row_start);
  return cudaGetLastError();
}

size_t stencil_list_entries(int n) { return stencil_list_len(n); }
int stencil_block_count(int n) { return stencil_blocks(n); }

cudaError_t launch_reduce(const double* part, int nblocks, int nvals, double* out, cudaStream_t s) {
  if (nvals <= 0) return cudaSuccess;
  k_reduce<<<nvals, 256, 0, s>>>(part, nblocks, out);
  return cudaGetLastError();
}

#define PM_INSTANTIATE(R)                                                                                         \
  template cudaError_t launch_init_particles<R>(const double*, const double*, int64_t, Mesh, double, void*, void*, \
                                                uint32_t*, uint32_t*, cudaStream_t);                              \
  template cudaError_t launch_sort_pass<R>(bool, const uint32_t*, const uint32_t*, int64_t, int, int,             \
                                           const uint32_t*, uint64_t*, uint32_t*, const uint32_t*, int, int,       \
                                           uint32_t*, uint32_t*, const void*, const void*, void*, void*,           \
                                           uint32_t*, cudaStream_t);                                              \
  template cudaError_t launch_deposit<R>(const void*, const uint32_t*, int64_t, Mesh, double, R*, cudaStream_t);           \
  template cudaError_t launch_green<R>(void*, Mesh, double, double*, cudaStream_t);                               \
  template cudaError_t launch_stencil<R>(const R*, Mesh, StencilParams, R*, double*, uint32_t*, uint32_t*,       \
                                          cudaStream_t);               \
  template cudaError_t launch_kick<R>(void*, void*, uint32_t*, int64_t, const R*, const R*, Mesh, KickParams,     \
                                      const KickParams*, const uint32_t*, double*, double*, uint32_t*,            \
                                      cudaStream_t);                                                              \
  template cudaError_t launch_power<R>(const void*, Mesh, int, double*, cudaStream_t);                            \
  template cudaError_t launch_get_particles<R>(const void*, const void*, int64_t, Mesh, double, double*, double*, \
                                               cudaStream_t);                                                     \
  template cudaError_t launch_get_order<R>(const void*, const void*, int64_t, uint32_t*, uint32_t*, cudaStream_t); \
  template cudaError_t launch_to_double<R>(const R*, int64_t, double*, cudaStream_t);                             \
  template cudaError_t launch_from_double<R>(const double*, int64_t, R*, cudaStream_t);

PM_INSTANTIATE(float)

}  // namespace pm
