// Stable least-significant-digit radix sort of the particles by cell key,
// hand-written (no library sort).  Keys are linear cell indices
// (iz*N + iy)*N + ix of ceil(log2 N^3) bits, split into 2..3 digits of at most
// RS_MAX_BITS bits.  Each pass is reduce-then-scan over tiles of RS_TILE keys:
//   upsweep   : per-tile digit histogram (warp-aggregated shared atomics on
//               integer counts, so the result is exact),
//   scan      : per digit, exclusive scan over tiles (one block per digit),
//   downsweep : stable rank inside the tile (warp match + per-warp counters,
//               tile order = warp, round, lane), staging in shared memory,
//               coalesced scatter.  The last pass gathers the 16/32-byte
//               particle records directly into sorted order.
// Equal keys keep their previous order, so the order after a step is the
// stable sort of the new cells with ties broken by the previous order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pm_internal.h"

namespace pm {

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

static __global__ void __launch_bounds__(RS_THREADS) k_radix_upsweep(const uint32_t* __restrict__ keys, int64_t n,
                                                              int shift, int bits, uint32_t* __restrict__ hist,
                                                              int ntiles) {
  extern __shared__ uint32_t sh_hist[];
  const int radix = 1 << bits;
  const uint32_t mask = uint32_t(radix - 1);
  for (int d = threadIdx.x; d < radix; d += blockDim.x) sh_hist[d] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t i = base + int64_t(j) * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    const uint32_t d = valid ? (__ldg(keys + i) >> shift) & mask : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&sh_hist[d], uint32_t(__popc(peers)));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[size_t(d) * ntiles + blockIdx.x] = sh_hist[d];
}

// Block-wide exclusive scan of one value per thread (RS_THREADS threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* scratch, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < RS_WARPS ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < RS_WARPS) scratch[32 + lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t warp_off = warp ? scratch[32 + warp - 1] : 0u;
  total = scratch[32 + RS_WARPS - 1];
  __syncthreads();
  return warp_off + incl - v;
}

// One block per digit: hist[d][*] <- exclusive scan over tiles; digit_total[d] <- sum.
static __global__ void __launch_bounds__(RS_THREADS) k_radix_scan(uint32_t* hist, int ntiles, uint32_t* digit_total) {
  __shared__ uint32_t scratch[64];
  uint32_t* row = hist + size_t(blockIdx.x) * ntiles;
  uint32_t carry = 0;
  for (int base = 0; base < ntiles; base += RS_THREADS * 4) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int t = base + threadIdx.x * 4 + k;
      v[k] = t < ntiles ? row[t] : 0u;
      s += v[k];
    }
    uint32_t total;
    uint32_t off = block_excl_scan(s, scratch, total) + carry;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int t = base + threadIdx.x * 4 + k;
      if (t < ntiles) row[t] = off;
      off += v[k];
    }
    carry += total;
  }
  if (threadIdx.x == 0) digit_total[blockIdx.x] = carry;
}

template <bool LAST, typename V4>
__global__ void __launch_bounds__(RS_THREADS) k_radix_downsweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, int64_t n, int shift, int bits,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ digit_total, int ntiles,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const V4* __restrict__ pos_in,
    const V4* __restrict__ mom_in, V4* __restrict__ pos_out, V4* __restrict__ mom_out) {
  extern __shared__ uint32_t smem[];
  const int radix = 1 << bits;
  const uint32_t mask = uint32_t(radix - 1);
  uint32_t* warp_cnt = smem;                          // [RS_WARPS][radix]
  uint32_t* digit_base = warp_cnt + RS_WARPS * radix;  // [radix] global start of (digit, this tile)
  uint32_t* tile_start = digit_base + radix;           // [radix] start of digit inside the tile
  uint32_t* s_keys = tile_start + radix;               // [RS_TILE]
  uint32_t* s_vals = s_keys + RS_TILE;                 // [RS_TILE]
  uint32_t* scratch = s_vals + RS_TILE;                // [64]

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile_base = int64_t(blockIdx.x) * RS_TILE;
  const int64_t rem = n - tile_base;
  const int tile_n = rem < RS_TILE ? int(rem) : RS_TILE;

  for (int d = threadIdx.x; d < RS_WARPS * radix; d += RS_THREADS) warp_cnt[d] = 0;
  // global digit starts: exclusive scan of digit_total, plus this tile's prefix
  {
    const int per = (radix + RS_THREADS - 1) / RS_THREADS;  // <= 4
    uint32_t v[4], s = 0;
    for (int k = 0; k < per; ++k) {
      int d = threadIdx.x * per + k;
      v[k] = d < radix ? __ldg(digit_total + d) : 0u;
      s += v[k];
    }
    uint32_t total;
    uint32_t off = block_excl_scan(s, scratch, total);
    for (int k = 0; k < per; ++k) {
      int d = threadIdx.x * per + k;
      if (d < radix) digit_base[d] = off + __ldg(hist + size_t(d) * ntiles + blockIdx.x);
      off += v[k];
    }
  }
  __syncthreads();

  // rank: warp w owns items [w*RS_ITEMS*32, (w+1)*RS_ITEMS*32) in rounds of 32
  uint32_t key[RS_ITEMS], rank[RS_ITEMS];
  const uint32_t lt = lanemask_lt();
  uint32_t* my_cnt = warp_cnt + warp * radix;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int li = warp * (RS_ITEMS * 32) + r * 32 + lane;
    const bool valid = li < tile_n;
    key[r] = valid ? __ldg(keys_in + tile_base + li) : 0u;
    const uint32_t d = valid ? (key[r] >> shift) & mask : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? my_cnt[d] : 0u;
    __syncwarp();
    const uint32_t within = __popc(peers & lt);
    if (valid && within == 0) my_cnt[d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + within;
  }
  __syncthreads();
  // per digit: exclusive scan over warps; tile total per digit
  for (int d = threadIdx.x; d < radix; d += RS_THREADS) {
    uint32_t run = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t t = warp_cnt[w * radix + d];
      warp_cnt[w * radix + d] = run;
      run += t;
    }
    tile_start[d] = run;
  }
  __syncthreads();
  {
    const int per = (radix + RS_THREADS - 1) / RS_THREADS;
    uint32_t v[4], s = 0;
    for (int k = 0; k < per; ++k) {
      int d = threadIdx.x * per + k;
      v[k] = d < radix ? tile_start[d] : 0u;
      s += v[k];
    }
    uint32_t total;
    uint32_t off = block_excl_scan(s, scratch, total);
    for (int k = 0; k < per; ++k) {
      int d = threadIdx.x * per + k;
      if (d < radix) tile_start[d] = off;
      off += v[k];
    }
  }
  __syncthreads();
  // stage in tile-sorted order
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int li = warp * (RS_ITEMS * 32) + r * 32 + lane;
    if (li < tile_n) {
      const uint32_t d = (key[r] >> shift) & mask;
      const uint32_t p = tile_start[d] + warp_cnt[warp * radix + d] + rank[r];
      s_keys[p] = key[r];
      s_vals[p] = vals_in ? __ldg(vals_in + tile_base + li) : uint32_t(tile_base + li);
    }
  }
  __syncthreads();
  for (int li = threadIdx.x; li < tile_n; li += RS_THREADS) {
    const uint32_t k = s_keys[li];
    const uint32_t d = (k >> shift) & mask;
    const uint32_t dest = digit_base[d] + uint32_t(li) - tile_start[d];
    keys_out[dest] = k;
    if (LAST) {
      const uint32_t src = s_vals[li];
      pos_out[dest] = pos_in[src];
      mom_out[dest] = mom_in[src];
    } else {
      vals_out[dest] = s_vals[li];
    }
  }
}

// row_start[r] = first sorted slot whose mesh row (key / N = z*N + y) is >= r,
// for r = 0..N^2.  Each slot i fills the rows between the row of slot i-1 and
// its own (rows are rarely empty, so almost every thread writes once or not
// at all).
static __global__ void k_row_start(const uint32_t* __restrict__ keys, int64_t n, uint32_t n_mesh, uint32_t nrows,
                                   uint32_t* row_start) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int64_t prev = i == 0 ? -1 : int64_t(__ldg(keys + i - 1) / n_mesh);
  const int64_t cur = i == n ? int64_t(nrows) : int64_t(__ldg(keys + i) / n_mesh);
  for (int64_t r = prev + 1; r <= cur; ++r) row_start[r] = uint32_t(i);
}

// Fixed-order fp64 reduction of per-block partials: out[v] = sum_b part[v*nblocks + b].
static __global__ void k_reduce(const double* __restrict__ part, int nblocks, double* out) {
  __shared__ double sh[256];
  const double* row = part + size_t(blockIdx.x) * nblocks;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += row[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

template <typename R>
cudaError_t launch_radix_downsweep(bool last, const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int shift,
                                   int bits, const uint32_t* hist, const uint32_t* digit_total, int ntiles,
                                   uint32_t* keys_out, uint32_t* vals_out, const void* pos_in, const void* mom_in,
                                   void* pos_out, void* mom_out, cudaStream_t s) {
  using V4 = typename VT<R>::v4;
  const size_t smem = radix_smem_bytes(bits);
  if (last) {
    auto k = k_radix_downsweep<true, V4>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k<<<ntiles, RS_THREADS, smem, s>>>(keys_in, vals_in, n, shift, bits, hist, digit_total, ntiles, keys_out,
                                       vals_out, (const V4*)pos_in, (const V4*)mom_in, (V4*)pos_out, (V4*)mom_out);
  } else {
    auto k = k_radix_downsweep<false, V4>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k<<<ntiles, RS_THREADS, smem, s>>>(keys_in, vals_in, n, shift, bits, hist, digit_total, ntiles, keys_out,
                                       vals_out, nullptr, nullptr, nullptr, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace pm
