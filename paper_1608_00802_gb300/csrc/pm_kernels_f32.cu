// fp32 instantiation of the step kernels, plus the type-independent launchers.
#include "pm_kernels.cuh"
#include "pm_sort.cuh"
#include "pm_instantiate.cuh"

namespace pm {

static __global__ void k_step_inc(uint32_t* step) { *step += 1u; }

cudaError_t launch_step_inc(uint32_t* step, cudaStream_t s) {
  k_step_inc<<<1, 1, 0, s>>>(step);
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

cudaError_t launch_mover_partition(const uint32_t* keys, int64_t n, uint32_t* tile_cnt, uint32_t* counts,
                                   uint32_t* s_keys, uint32_t* s_vals, uint32_t* m_keys, uint32_t* m_vals,
                                   cudaStream_t s) {
  const int ntiles = int((n + RS_TILE - 1) / RS_TILE);
  k_mover_count<<<unsigned(ntiles), RS_THREADS, 0, s>>>(keys, n, tile_cnt);
  k_mover_scan<<<1, RS_THREADS, 0, s>>>(tile_cnt, ntiles, n, counts);
  k_mover_scatter<<<unsigned(ntiles), RS_THREADS, 0, s>>>(keys, n, tile_cnt, s_keys, s_vals, m_keys, m_vals);
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

PM_INSTANTIATE(float)

}  // namespace pm
