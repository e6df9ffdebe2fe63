// Stable least-significant-digit radix sort of the particles by cell key,
// hand-written (no library sort).  Keys are linear cell indices
// (iz*N + iy)*N + ix of ceil(log2 N^3) bits, split into passes of at most
// RS_MAX_BITS bits.
//   k_sort_histogram : one read of the keys gives the digit histograms of all
//                      passes (warp-aggregated shared atomics on integers).
//   k_sort_pass      : one kernel per pass.  Each block takes the next tile
//                      (RS_TILE keys, tile ids from an atomic counter), ranks
//                      its keys stably (warp match + per-warp counters, tile
//                      order = warp, round, lane), publishes its per-digit
//                      counts, and finds the global start of each digit for its
//                      tile by decoupled look-back over the status words of
//                      the preceding tiles (Merrill & Garland's single-pass
//                      scan, as used by Onesweep, Adinets & Merrill 2022).  The
//                      keys are then staged in shared memory and scattered
//                      with coalesced stores; the last pass gathers the 16/32
//                      byte particle records straight into sorted order.
// Status words are 64-bit: epoch (16 bits) | flag (16) | count (32); a new
// epoch per pass makes old words invalid without clearing them.  Every wait
// on a predecessor is bounded: after RS_SPIN_LIMIT polls the kernel sets
// ERR_TIMEOUT in the error word and goes on, so a fault cannot hang the GPU.
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

constexpr uint64_t RS_FLAG_AGG = 1ull << 32;
constexpr uint64_t RS_FLAG_PREFIX = 2ull << 32;
constexpr int RS_SPIN_LIMIT = 1 << 18;
constexpr int RS_LOOKBACK = 8;  // predecessors read per look-back round

__device__ __forceinline__ uint64_t rs_word(uint32_t epoch, uint64_t flag, uint32_t v) {
  return (uint64_t(epoch) << 48) | flag | uint64_t(v);
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

// Digit histograms of every pass: hist[p * radix_max + d].
// Block 0 also advances the sort's epoch word: the passes of this sort use
// epochs base .. base + passes - 1, never 0 and never those of the previous
// sort, so status words left by earlier sorts (or by an earlier replay of a
// captured graph) are never mistaken for current ones.
static __global__ void __launch_bounds__(RS_THREADS) k_sort_histogram(const uint32_t* __restrict__ keys, int64_t n,
                                                                      int passes, int digit_bits, int key_bits,
                                                                      uint32_t* __restrict__ hist,
                                                                      uint32_t* __restrict__ epoch,
                                                                      const uint32_t* __restrict__ n_dev) {
  __shared__ uint32_t sh[3 * (1 << RS_MAX_BITS)];
  if (n_dev) n = *n_dev;  // element count known on the device only
  if (blockIdx.x == 0 && threadIdx.x == 0) *epoch = (*epoch + uint32_t(passes)) % 65530u + 1u;
  const int radix = 1 << digit_bits;
  for (int i = threadIdx.x; i < passes * radix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? __ldg(keys + i) : 0u;
    for (int p = 0; p < passes; ++p) {
      const int shift = p * digit_bits;
      const int bits = min(digit_bits, key_bits - shift);
      const uint32_t d = valid ? (key >> shift) & ((1u << bits) - 1u) : 0xffffffffu;
      // runs of equal digits in neighbouring lanes: the first lane of a run adds its length
      const uint32_t dprev = __shfl_up_sync(0xffffffffu, d, 1);
      const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || d != dprev);
      if (valid && ((heads >> lane) & 1u)) {
        const uint32_t after = heads & ~((2u << lane) - 1u);  // run heads above this lane
        const int end = after ? __ffs(after) - 1 : 32;
        atomicAdd(&sh[p * radix + d], uint32_t(end - lane));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * radix; i += blockDim.x)
    if (sh[i]) atomicAdd(hist + (i / radix) * (1 << RS_MAX_BITS) + (i % radix), sh[i]);
}

template <bool LAST, typename V4>
__global__ void __launch_bounds__(RS_THREADS) k_sort_pass(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, int64_t n, int shift, int bits,
    const uint32_t* __restrict__ digit_total, uint64_t* status, uint32_t* tile_counter,
    const uint32_t* __restrict__ epoch_base, int pass,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const V4* __restrict__ pos_in,
    const V4* __restrict__ mom_in, V4* __restrict__ pos_out, V4* __restrict__ mom_out, uint32_t* err,
    const uint32_t* __restrict__ n_dev) {
  extern __shared__ uint32_t smem[];
  if (n_dev) n = *n_dev;  // element count known on the device only: surplus tiles exit below
  const int radix = 1 << bits;
  const uint32_t mask = uint32_t(radix - 1);
  uint32_t* warp_cnt = smem;                          // [RS_WARPS][radix]
  uint32_t* digit_base = warp_cnt + RS_WARPS * radix;  // [radix] global start of (digit, this tile)
  uint32_t* tile_start = digit_base + radix;           // [radix] start of digit inside the tile
  uint32_t* s_keys = tile_start + radix;               // [RS_TILE]
  uint32_t* s_vals = s_keys + RS_TILE;                 // [RS_TILE]
  uint32_t* scratch = s_vals + RS_TILE;                // [64] (+1: tile id)

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t epoch = *epoch_base + uint32_t(pass);
  if (threadIdx.x == 0) scratch[63] = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = scratch[63];
  const int64_t tile_base = int64_t(tile) * RS_TILE;
  if (tile_base >= n) return;  // whole block: tile ids past the data (grid sized for the largest count)
  // (cleared counters are first read after the barriers of the digit scan below)
  for (int d = threadIdx.x; d < RS_WARPS * radix; d += RS_THREADS) warp_cnt[d] = 0;
  const int64_t rem = n - tile_base;
  const int tile_n = rem < RS_TILE ? int(rem) : RS_TILE;
  const int per = (radix + RS_THREADS - 1) / RS_THREADS;  // <= 4

  // exclusive scan of the pass histogram -> global start of each digit
  {
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int d = threadIdx.x * per + k;
      v[k] = (k < per && d < radix) ? __ldg(digit_total + d) : 0u;
      sum += v[k];
    }
    uint32_t total;
    uint32_t off = block_excl_scan(sum, scratch, total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int d = threadIdx.x * per + k;
      if (k < per && d < radix) digit_base[d] = off;
      off += v[k];
    }
  }

  // stable rank: warp w owns items [w*RS_ITEMS*32, (w+1)*RS_ITEMS*32) in rounds of 32
  uint32_t key[RS_ITEMS], rank[RS_ITEMS];
  const uint32_t lt = lanemask_lt();
  uint32_t* my_cnt = warp_cnt + warp * radix;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int li = warp * (RS_ITEMS * 32) + r * 32 + lane;
    key[r] = li < tile_n ? __ldg(keys_in + tile_base + li) : 0u;
  }
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int li = warp * (RS_ITEMS * 32) + r * 32 + lane;
    const bool valid = li < tile_n;
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
  // per digit: exclusive scan over warps; the tile's count, published at once
  for (int d = threadIdx.x; d < radix; d += RS_THREADS) {
    uint32_t run = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t t = warp_cnt[w * radix + d];
      warp_cnt[w * radix + d] = run;
      run += t;
    }
    tile_start[d] = run;
    __stcg(reinterpret_cast<unsigned long long*>(status + size_t(tile) * radix + d),
           rs_word(epoch, tile == 0 ? RS_FLAG_PREFIX : RS_FLAG_AGG, run));
  }
  // decoupled look-back: sum the counts of the preceding tiles for each digit
  for (int d = threadIdx.x; d < radix; d += RS_THREADS) {
    uint32_t excl = 0;
    if (tile > 0) {
      // the status words of up to RS_LOOKBACK predecessors are read at once and
      // consumed in order (nearest first) up to the first one not yet published
      int64_t t = int64_t(tile) - 1;
      int polls = 0;
      bool done = false;
      while (!done && t >= 0) {
        uint64_t w[RS_LOOKBACK];
#pragma unroll
        for (int k = 0; k < RS_LOOKBACK; ++k)
          w[k] = t - k >= 0 ? __ldcv(reinterpret_cast<const unsigned long long*>(status + size_t(t - k) * radix + d))
                            : 0ull;
        int used = 0;
#pragma unroll
        for (int k = 0; k < RS_LOOKBACK; ++k) {
          if (done || used < k || t - k < 0) continue;  // stop at the first gap
          if (uint32_t(w[k] >> 48) == epoch && (w[k] & (RS_FLAG_AGG | RS_FLAG_PREFIX))) {
            excl += uint32_t(w[k]);
            used = k + 1;
            if (w[k] & RS_FLAG_PREFIX) done = true;
          }
        }
        t -= used;
        if (done || t < 0) break;
        if (used == 0) {
          if (++polls > RS_SPIN_LIMIT) {
            atomicOr(err, ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
      __stcg(reinterpret_cast<unsigned long long*>(status + size_t(tile) * radix + d),
             rs_word(epoch, RS_FLAG_PREFIX, excl + tile_start[d]));
    }
    digit_base[d] += excl;
  }
  __syncthreads();
  // exclusive scan of the tile counts -> start of each digit inside the tile
  {
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int d = threadIdx.x * per + k;
      v[k] = (k < per && d < radix) ? tile_start[d] : 0u;
      sum += v[k];
    }
    uint32_t total;
    uint32_t off = block_excl_scan(sum, scratch, total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int d = threadIdx.x * per + k;
      if (k < per && d < radix) tile_start[d] = off;
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
    if (dest >= uint32_t(n)) {  // only possible after a timed-out look-back: drop the element
      atomicOr(err, ERR_TIMEOUT);
      continue;
    }
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
// at all).  Rows are clamped to N^2: a key outside the mesh (a slot left
// unwritten by a sort whose look-back timed out) writes nothing past the table.
static __global__ void k_row_start(const uint32_t* __restrict__ keys, int64_t n, uint32_t n_mesh, uint32_t nrows,
                                   uint32_t* row_start, uint32_t* src) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (src && i < n) src[i] = uint32_t(i);  // the records are in sorted order
  const int64_t prev = i == 0 ? -1 : min(int64_t(__ldg(keys + i - 1) / n_mesh), int64_t(nrows));
  const int64_t cur = i == n ? int64_t(nrows) : min(int64_t(__ldg(keys + i) / n_mesh), int64_t(nrows));
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

// Maximum of per-block partials: out[v] = max_b part[v*nblocks + b].
static __global__ void k_reduce_max(const double* __restrict__ part, int nblocks, double* out) {
  __shared__ double sh[256];
  const double* row = part + size_t(blockIdx.x) * nblocks;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s = fmax(s, row[b]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// ---------------------------------------------------------------- incremental re-sort
// After a drift the kick marks particles whose cell changed ("movers") by
// setting bit 31 of their new key.  The others ("stayers") keep their key, so
// in storage order they are still sorted by (key, previous slot).  The stable
// sort by new key with ties in previous order is then: partition stably into
// stayers and movers, radix-sort the movers (usually a few per cent), and merge
// the two sequences by (key, previous slot) while gathering the records.  The
// result is identical to the full sort.
// Stable partition in one pass: block t takes tile t of RS_TILE slots.  The
// drift has already counted the movers of every tile and of every group of
// 2^RS_GROUP_SHIFT tiles (tcount), so a block finds the movers of all earlier
// tiles by summing at most one group's tile counts and the earlier groups'
// counts, with no wait on other blocks.  It writes its stayers to (s_keys,
// s_vals) and its movers, flag cleared, to (m_keys, m_vals); values are the
// previous slots.  It also accumulates the digit histograms of the movers'
// keys for every radix pass (hist[p*radix_max + d], cleared before), advances
// the sort epoch for those passes (as the histogram kernel does for a full
// sort) and, in the last tile, stores counts[0] = stayers, counts[1] = movers
// and adds one re-sort and the movers to stats (nullable).
static __global__ void __launch_bounds__(RS_THREADS) k_mover_partition(
    const uint32_t* __restrict__ keys, int64_t n, const uint32_t* __restrict__ tcount,
    uint32_t* __restrict__ s_keys, uint32_t* __restrict__ s_vals, uint32_t* __restrict__ m_keys,
    uint32_t* __restrict__ m_vals, uint32_t* __restrict__ counts, uint32_t* __restrict__ hist, int passes,
    int digit_bits, int key_bits, uint32_t* __restrict__ sort_epoch, unsigned long long* __restrict__ stats) {
  __shared__ uint32_t sh_hist[3 << RS_MAX_BITS];
  __shared__ uint32_t wm[RS_WARPS], wsum[RS_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int radix = 1 << digit_bits;
  const uint32_t ntiles = uint32_t((n + RS_TILE - 1) >> RS_TILE_SHIFT);
  const uint32_t tile = blockIdx.x;
  for (int d = threadIdx.x; d < passes * radix; d += RS_THREADS) sh_hist[d] = 0u;
  if (tile == 0 && threadIdx.x == 0) *sort_epoch = (*sort_epoch + uint32_t(passes)) % 65530u + 1u;
  const int64_t tile_base = int64_t(tile) * RS_TILE;
  const uint32_t lt = lanemask_lt();
  // movers before this tile: the earlier groups' counts, then the earlier tiles of this group
  const uint32_t grp = tile >> RS_GROUP_SHIFT, first = grp << RS_GROUP_SHIFT;
  uint32_t e = 0;
  for (uint32_t g = threadIdx.x; g < grp; g += RS_THREADS) e += __ldg(tcount + ntiles + g);
  for (uint32_t t = first + threadIdx.x; t < tile; t += RS_THREADS) e += __ldg(tcount + t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (lane == 0) wsum[warp] = e;
  // warp w owns slots [w*RS_ITEMS*32, (w+1)*RS_ITEMS*32) of the tile, in rounds of 32
  uint32_t key[RS_ITEMS], rank[RS_ITEMS], mcount = 0;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = tile_base + warp * (RS_ITEMS * 32) + r * 32 + lane;
    key[r] = i < n ? __ldg(keys + i) : 0u;
    const uint32_t b = __ballot_sync(0xffffffffu, (key[r] & KEY_MOVER) != 0);
    rank[r] = mcount + __popc(b & lt);  // movers before this slot in the warp
    mcount += __popc(b);
  }
  if (lane == 0) wm[warp] = mcount;
  __syncthreads();
  uint32_t excl = 0, total = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) {
    excl += wsum[w];
    total += wm[w];
  }
  if (tile == ntiles - 1 && threadIdx.x == 0) {
    counts[0] = uint32_t(n) - (excl + total);
    counts[1] = excl + total;
    if (stats) {  // re-sorts and moved particles so far (a diagnostic)
      stats[0] += 1ull;
      stats[1] += (unsigned long long)(excl + total);
    }
  }
  // movers in the earlier warps of the tile: lane w < warp contributes wm[w]
  uint32_t mbase = lane < warp ? wm[lane] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mbase += __shfl_xor_sync(0xffffffffu, mbase, o);
  mbase += excl;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = tile_base + warp * (RS_ITEMS * 32) + r * 32 + lane;
    if (i < n) {
      const uint32_t before = mbase + rank[r];  // movers before slot i
      if (key[r] & KEY_MOVER) {
        const uint32_t k = key[r] & ~KEY_MOVER;
        if (before < uint32_t(n)) {  // always (the counts bound the movers)
          m_keys[before] = k;
          m_vals[before] = uint32_t(i);
        }
        for (int p = 0; p < passes; ++p) {
          const int shift = p * digit_bits;
          const int bits = min(digit_bits, key_bits - shift);
          atomicAdd(&sh_hist[p * radix + ((k >> shift) & ((1u << bits) - 1u))], 1u);
        }
      } else if (uint32_t(i) >= before) {
        s_keys[uint32_t(i) - before] = key[r];
        s_vals[uint32_t(i) - before] = uint32_t(i);
      }
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < passes * radix; d += RS_THREADS)
    if (sh_hist[d]) atomicAdd(hist + (d / radix) * (1 << RS_MAX_BITS) + (d % radix), sh_hist[d]);
}

__device__ __forceinline__ bool kv_less(uint32_t ka, uint32_t va, uint32_t kb, uint32_t vb) {
  return ka < kb || (ka == kb && va < vb);
}

// number of stayers among the first d outputs of the merge (merge path)
__device__ __forceinline__ uint32_t merge_split(const uint32_t* sk, const uint32_t* sv, uint32_t ns,
                                                const uint32_t* mk, const uint32_t* mv, uint32_t nm, uint32_t d) {
  uint32_t lo = d > nm ? d - nm : 0u, hi = d < ns ? d : ns;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t j = d - 1 - mid;  // the mover compared with stayer mid
    if (kv_less(sk[mid], sv[mid], mk[j], mv[j]))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

constexpr int MG_TILE = RS_TILE;  // outputs per block
inline size_t merge_smem_bytes() { return size_t(MG_TILE) * 6 * sizeof(uint32_t); }

// Both ends of the block's output range on the merge path, found by the two
// halves of the block at once with a 128-way search: each round probes 128
// evenly spaced candidates, so about three rounds (one dependent global load
// each) narrow two million candidates to one.  Returns the number of stayers
// before output d0 (split[0]) and d1 (split[1]).
__device__ __forceinline__ void merge_split_block(const uint32_t* sk, const uint32_t* sv, uint32_t ns,
                                                  const uint32_t* mk, const uint32_t* mv, uint32_t nm, uint32_t d0,
                                                  uint32_t d1, uint32_t* lo_s, uint32_t* hi_s) {
  const int grp = threadIdx.x >> 7, t = threadIdx.x & 127;
  const uint32_t d = grp ? d1 : d0;
  if (t == 0) {
    lo_s[grp] = d > nm ? d - nm : 0u;
    hi_s[grp] = d < ns ? d : ns;
    lo_s[2 + grp] = 0u;
    hi_s[2 + grp] = 0xffffffffu;
  }
  __syncthreads();
  for (;;) {
    const uint32_t lo = lo_s[grp], hi = hi_s[grp];
    if (!__syncthreads_or(lo < hi)) break;
    // candidate a in [lo, hi): are there more than a stayers before d?  (stayer a precedes mover d-1-a)
    if (lo < hi) {
      const uint32_t a = lo + uint32_t((uint64_t(hi - lo) * uint32_t(t)) >> 7);
      const uint32_t j = d - 1 - a;
      if (kv_less(sk[a], sv[a], mk[j], mv[j]))
        atomicMax(lo_s + 2 + grp, a + 1);
      else
        atomicMin(hi_s + 2 + grp, a);
    }
    __syncthreads();
    if (t == 0 && lo < hi) {
      if (lo_s[2 + grp] > lo) lo_s[grp] = lo_s[2 + grp];
      if (hi_s[2 + grp] < hi) hi_s[grp] = hi_s[2 + grp];
      lo_s[2 + grp] = 0u;
      hi_s[2 + grp] = 0xffffffffu;
    }
    __syncthreads();
  }
}

// merge of the stayers with the sorted movers, by (key, previous slot); writes
// the sorted keys, the previous slot of every sorted index (src: the records
// stay where the drift wrote them, and the deposit and the next kick read
// them through src) and the row starts (row_start[r] = first slot whose key
// is in row r or above; row_start[N^2] = n)
static __global__ void __launch_bounds__(RS_THREADS) k_merge(
    const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv, const uint32_t* __restrict__ mk,
    const uint32_t* __restrict__ mv, const uint32_t* __restrict__ counts, int64_t n, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ src_out, uint32_t n_mesh, uint32_t* __restrict__ row_start) {
  extern __shared__ uint32_t msm[];
  uint32_t* a_k = msm;               // stayers of this tile
  uint32_t* a_v = a_k + MG_TILE;
  uint32_t* b_k = a_v + MG_TILE;     // movers of this tile
  uint32_t* b_v = b_k + MG_TILE;
  uint32_t* o_k = b_v + MG_TILE;     // merged
  uint32_t* o_v = o_k + MG_TILE;
  __shared__ uint32_t lo_s[4], hi_s[4];
  __shared__ uint32_t prev_key;
  const uint32_t ns = counts[0], nm = counts[1];
  const uint32_t d0 = blockIdx.x * uint32_t(MG_TILE);
  const uint32_t d1 = int64_t(d0) + MG_TILE < n ? d0 + uint32_t(MG_TILE) : uint32_t(n);
  merge_split_block(sk, sv, ns, mk, mv, nm, d0, d1, lo_s, hi_s);
  const uint32_t a0 = lo_s[0], a1 = lo_s[1];
  const uint32_t b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t na = a1 - a0, nb = b1 - b0;
  const uint32_t tn = d1 - d0;
  if (nb == 0) {
    // no mover falls in this tile (the common case): the stayers pass through
    for (uint32_t q = threadIdx.x; q < tn; q += RS_THREADS) {
      const uint32_t k = __ldg(sk + a0 + q);
      keys_out[d0 + q] = k;
      src_out[d0 + q] = __ldg(sv + a0 + q);
      o_k[q] = k;
    }
  } else {
    for (uint32_t t = threadIdx.x; t < na; t += RS_THREADS) {
      a_k[t] = sk[a0 + t];
      a_v[t] = sv[a0 + t];
    }
    for (uint32_t t = threadIdx.x; t < nb; t += RS_THREADS) {
      b_k[t] = mk[b0 + t];
      b_v[t] = mv[b0 + t];
    }
    __syncthreads();
    // each thread merges RS_ITEMS consecutive outputs of the tile
    const uint32_t q0 = min(uint32_t(threadIdx.x) * RS_ITEMS, tn), q1 = min(q0 + RS_ITEMS, tn);
    if (q0 < q1) {
      uint32_t ia = merge_split(a_k, a_v, na, b_k, b_v, nb, q0);
      uint32_t ib = q0 - ia;
      for (uint32_t q = q0; q < q1; ++q) {
        const bool take_a = ib >= nb || (ia < na && kv_less(a_k[ia], a_v[ia], b_k[ib], b_v[ib]));
        if (take_a) {
          o_k[q] = a_k[ia];
          o_v[q] = a_v[ia];
          ++ia;
        } else {
          o_k[q] = b_k[ib];
          o_v[q] = b_v[ib];
          ++ib;
        }
      }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < tn; q += RS_THREADS) {
      keys_out[d0 + q] = o_k[q];
      src_out[d0 + q] = o_v[q];
    }
  }
  if (threadIdx.x == 0 && d0 > 0) {
    // the key at output d0-1: the larger of the last stayer and the last mover before this tile
    uint32_t k = 0, v = 0;
    bool have = false;
    if (a0 > 0) {
      k = sk[a0 - 1];
      v = sv[a0 - 1];
      have = true;
    }
    if (b0 > 0 && (!have || kv_less(k, v, mk[b0 - 1], mv[b0 - 1]))) k = mk[b0 - 1];
    prev_key = k;
  }
  __syncthreads();
  // rows (row of output i-1, row of output i] start at i (rows clamped to N^2, as in k_row_start)
  const int64_t nrows = int64_t(n_mesh) * n_mesh;
  for (uint32_t q = threadIdx.x; q <= tn; q += RS_THREADS) {
    const uint32_t i = d0 + q;
    if (q == tn && i != uint32_t(n)) break;  // output n (the closing row starts) belongs to the last block
    const int64_t prev = i == 0 ? -1 : min(int64_t((q ? o_k[q - 1] : prev_key) / n_mesh), nrows);
    const int64_t cur = i == uint32_t(n) ? nrows : min(int64_t(o_k[q] / n_mesh), nrows);
    for (int64_t r = prev + 1; r <= cur; ++r) row_start[r] = i;
  }
}

inline cudaError_t launch_merge_impl(const uint32_t* sk, const uint32_t* sv, const uint32_t* mk, const uint32_t* mv,
                                     const uint32_t* counts, int64_t n, uint32_t* keys_out, uint32_t* src_out,
                                     uint32_t n_mesh, uint32_t* row_start, cudaStream_t s) {
  static bool done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(merge_smem_bytes()));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  const unsigned blocks = unsigned((n + MG_TILE - 1) / MG_TILE);
  k_merge<<<blocks, RS_THREADS, merge_smem_bytes(), s>>>(sk, sv, mk, mv, counts, n, keys_out, src_out, n_mesh,
                                                          row_start);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sort_pass(bool last, const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int shift,
                             int bits, const uint32_t* digit_total, uint64_t* status, uint32_t* tile_counter,
                             const uint32_t* epoch, int pass, int ntiles, uint32_t* keys_out, uint32_t* vals_out,
                             const void* pos_in, const void* mom_in, void* pos_out, void* mom_out, uint32_t* err,
                             cudaStream_t s, const uint32_t* n_dev) {
  using V4 = typename VT<R>::v4;
  const size_t smem = radix_smem_bytes(bits);
  // shared-memory limits are raised once per device (for the largest digit), outside any capture
  static bool done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !done[dev]) {
    const int most = int(radix_smem_bytes(RS_MAX_BITS));
    cudaError_t e = cudaFuncSetAttribute(k_sort_pass<true, V4>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sort_pass<false, V4>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  if (last) {
    k_sort_pass<true, V4><<<ntiles, RS_THREADS, smem, s>>>(keys_in, vals_in, n, shift, bits, digit_total, status,
                                                           tile_counter, epoch, pass, keys_out, vals_out,
                                                           (const V4*)pos_in, (const V4*)mom_in, (V4*)pos_out,
                                                           (V4*)mom_out, err, n_dev);
  } else {
    k_sort_pass<false, V4><<<ntiles, RS_THREADS, smem, s>>>(keys_in, vals_in, n, shift, bits, digit_total, status,
                                                            tile_counter, epoch, pass, keys_out, vals_out, nullptr,
                                                            nullptr, nullptr, nullptr, err, n_dev);
  }
  return cudaGetLastError();
}

}  // namespace pm
