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
constexpr int RS_PASS_BLOCKS = 1216;  // blocks of one radix pass (8 per SM on 152 SMs)
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
    const uint32_t* __restrict__ n_dev, size_t ms, int spin_limit) {
  extern __shared__ uint32_t smem[];
  if (ms) {  // member blockIdx.y of a packed group (the passes over its movers)
    const size_t o = size_t(blockIdx.y) * ms;
    keys_in = moff(keys_in, o), vals_in = moff(vals_in, o), digit_total = moff(digit_total, o);
    status = moff(status, o), tile_counter = moff(tile_counter, o), epoch_base = moff(epoch_base, o);
    keys_out = moff(keys_out, o), vals_out = moff(vals_out, o), err = moff(err, o), n_dev = moff(n_dev, o);
  }
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
  // persistent blocks: each claims tiles in order until none is left (predecessors
  // of a claimed tile are always claimed already, so the look-back ends)
  for (;;) {
    if (threadIdx.x == 0) scratch[63] = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = scratch[63];
    const int64_t tile_base = int64_t(tile) * RS_TILE;
    if (tile_base >= n) break;  // whole block: no tile left (the grid is capped below the tile count)
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
            if (++polls > spin_limit) {
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
    __syncthreads();  // shared memory is reused by the next tile
  }
}

// row_start[r] = first sorted slot whose mesh row (key / N = z*N + y) is >= r,
// for r = 0..N^2.  Each slot i fills the rows between the row of slot i-1 and
// its own (rows are rarely empty, so almost every thread writes once or not
// at all).  Rows are clamped to N^2: a key outside the mesh (a slot left
// unwritten by a sort whose look-back timed out) writes nothing past the table.
static __global__ void k_row_start(const uint32_t* __restrict__ keys, int64_t n, uint32_t n_mesh, uint32_t nrows,
                                   uint32_t* row_start) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > n) return;
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
// After a drift the kick marks the particles whose cell changed ("movers") by
// setting bit 31 of their new key and counts them per tile of RS_TILE slots
// (and per group of tiles).  The others ("stayers") keep their key, so in
// storage order they are still sorted by (key, previous slot).  The stable
// sort by new key with ties in previous order is the merge of the stayers with
// the movers by (key, previous slot), and every particle's place in it follows
// from its mesh row (key / N) alone:
//   place = (stayers in earlier rows) + (movers in earlier rows)
//         + (stayers of its row before it) + (movers of its row before it),
// and a row holds a few tens of particles.  So the re-sort is: a stable
// partition that also counts stayers and movers per row; a scan of the row
// counts (which also gives the new row starts); a scatter of the movers into
// per-row buckets; and the placement of every mover and every stayer, each
// counting the entries of its own row that precede it (a mover among its
// bucket and its row's stayers, a stayer among its row's bucket) and moving
// its records there.  No sort pass over the movers and no search over the
// whole sequence; the order is fixed by comparisons, so the result is the
// same as the full stable sort (integer atomics only count and claim bucket
// slots, whose order within a bucket does not enter the result).
// Packed groups of simulations: member blockIdx.y, pointers ms bytes apart.

__device__ __forceinline__ bool kv_less(uint32_t ka, uint32_t va, uint32_t kb, uint32_t vb) {
  return ka < kb || (ka == kb && va < vb);
}

// row of a key (z*N + y), by a shift when N is a power of two
__device__ __forceinline__ uint32_t key_row(uint32_t key, uint32_t n_mesh, int log2n) {
  return log2n >= 0 ? key >> log2n : key / n_mesh;
}

constexpr int RT_THREADS = 256, RT_ITEMS = 4, RT_TILE = RT_THREADS * RT_ITEMS;
static_assert(RT_TILE == 1024, "row_scan_tiles counts tiles of 1024 rows");
// the partition sums the earlier tiles' mover counts itself up to this many tiles (else k_tile_scan)
constexpr uint32_t PART_OWN_SCAN_TILES = 2048;

// Movers before every tile: an exclusive scan of the drift's per-tile mover
// counts (tcount[0..T)) into tcount[T..2T), by one block per simulation.
constexpr int TS_THREADS = 1024;
static __global__ void __launch_bounds__(TS_THREADS) k_tile_scan(uint32_t* tcount, uint32_t ntiles, size_t ms) {
  __shared__ uint32_t wsum[TS_THREADS / 32];
  if (ms) tcount = moff(tcount, size_t(blockIdx.y) * ms);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t per = (ntiles + TS_THREADS - 1) / TS_THREADS;
  const uint32_t t0 = threadIdx.x * per, t1 = min(t0 + per, ntiles);
  uint32_t sum = 0;
  for (uint32_t t = t0; t < t1; ++t) sum += tcount[t];
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t off = 0;
  for (int w = 0; w < warp; ++w) off += wsum[w];
  uint32_t run = off + inc - sum;
  for (uint32_t t = t0; t < t1; ++t) {
    const uint32_t c = tcount[t];
    tcount[ntiles + t] = run;
    run += c;
  }
}

// Stable partition, one block per tile of RS_TILE slots; the movers of the
// earlier tiles come from the tile scan.  It writes its stayers to (s_keys, s_vals) and its
// movers, flag cleared, to (m_keys, m_vals) (values: previous slots), adds
// its stayers and movers to the per-row counts rcnt[0][row] and rcnt[1][row]
// (cleared before; one atomic per run of equal rows in a warp for the
// stayers), and the last tile stores counts[0] = stayers, counts[1] = movers
// and adds one re-sort and the movers to stats (nullable).
static __global__ void __launch_bounds__(RS_THREADS) k_mover_partition(
    const uint32_t* __restrict__ keys, int64_t n, const uint32_t* __restrict__ tcount,
    uint32_t* __restrict__ s_keys, uint32_t* __restrict__ s_vals, uint32_t* __restrict__ m_keys,
    uint32_t* __restrict__ m_vals, uint32_t* __restrict__ counts, uint32_t* __restrict__ rcnt,
    uint32_t n_mesh, int log2n, unsigned long long* __restrict__ stats, int own_scan, size_t ms) {
  __shared__ uint32_t wm[RS_WARPS];
  if (ms) {  // member blockIdx.y of a packed group
    const size_t o = size_t(blockIdx.y) * ms;
    keys = moff(keys, o), tcount = moff(tcount, o), s_keys = moff(s_keys, o), s_vals = moff(s_vals, o);
    m_keys = moff(m_keys, o), m_vals = moff(m_vals, o), counts = moff(counts, o), rcnt = moff(rcnt, o);
    stats = moff(stats, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nrows = n_mesh * n_mesh;
  const uint32_t ntiles = uint32_t((n + RS_TILE - 1) >> RS_TILE_SHIFT);
  const uint32_t tile = blockIdx.x;
  const int64_t tile_base = int64_t(tile) * RS_TILE;
  const uint32_t lt = lanemask_lt();
  // warp w owns slots [w*RS_ITEMS*32, (w+1)*RS_ITEMS*32) of the tile, in rounds of 32; all its keys
  // are requested before anything waits on them
  uint32_t key[RS_ITEMS], rank[RS_ITEMS], mcount = 0;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = tile_base + warp * (RS_ITEMS * 32) + r * 32 + lane;
    key[r] = i < n ? __ldg(keys + i) : 0u;
  }
  // movers before this tile: the tile scan's, or (few tiles) summed here from the drift's counts
  uint32_t excl;
  if (own_scan) {
    uint32_t sum = 0;
    for (uint32_t t = threadIdx.x; t < tile; t += RS_THREADS) sum += tcount[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) wm[warp] = sum;
    __syncthreads();
    excl = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) excl += wm[w];
    __syncthreads();  // wm is reused below
  } else {
    excl = __ldg(tcount + ntiles + tile);
  }
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = tile_base + warp * (RS_ITEMS * 32) + r * 32 + lane;
    const bool mover = i < n && (key[r] & KEY_MOVER);
    const uint32_t b = __ballot_sync(0xffffffffu, mover);
    rank[r] = mcount + __popc(b & lt);  // movers before this slot in the warp
    mcount += __popc(b);
    // per-row counts: stayers by runs of equal rows in the warp, movers one by one
    const uint32_t row = key_row(key[r] & ~KEY_MOVER, n_mesh, log2n);
    const bool stayer = i < n && !mover;
    const uint32_t peers = __match_any_sync(0xffffffffu, stayer ? row : 0xffffffffu) & __ballot_sync(0xffffffffu, stayer);
    if (stayer && row < nrows && (peers & lt) == 0) atomicAdd(rcnt + row, uint32_t(__popc(peers)));
    if (mover && row < nrows) atomicAdd(rcnt + nrows + row, 1u);
  }
  if (lane == 0) wm[warp] = mcount;
  __syncthreads();
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) total += wm[w];
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
        if (before < uint32_t(n)) {  // always (the counts bound the movers)
          m_keys[before] = key[r] & ~KEY_MOVER;
          m_vals[before] = uint32_t(i);
        }
      } else if (uint32_t(i) >= before) {
        s_keys[uint32_t(i) - before] = key[r];
        s_vals[uint32_t(i) - before] = uint32_t(i);
      }
    }
  }
}

// Exclusive scans of the per-row stayer and mover counts over the N^2 rows,
// in tiles of RT_TILE rows: k_row_totals sums each tile, k_row_scan adds the
// earlier tiles' totals and scans its own, writing srow (stayers before row
// r), mrow (movers before row r) and the new row starts row_start = srow +
// mrow, with the closing entries at r = N^2.

static __global__ void __launch_bounds__(RT_THREADS) k_row_totals(const uint32_t* __restrict__ rcnt, uint32_t nrows,
                                                                  uint32_t* __restrict__ btot, size_t ms) {
  __shared__ uint32_t sh[2][32];
  if (ms) {
    const size_t o = size_t(blockIdx.y) * ms;
    rcnt = moff(rcnt, o), btot = moff(btot, o);
  }
  const uint32_t r0 = blockIdx.x * RT_TILE;
  uint32_t a = 0, b = 0;
#pragma unroll
  for (int k = 0; k < RT_ITEMS; ++k) {
    const uint32_t r = r0 + threadIdx.x + k * RT_THREADS;
    if (r < nrows) {
      a += __ldg(rcnt + r);
      b += __ldg(rcnt + nrows + r);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    sh[0][warp] = a;
    sh[1][warp] = b;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    uint32_t t = 0;
    for (int w = 0; w < RT_THREADS / 32; ++w) t += sh[threadIdx.x][w];
    btot[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

static __global__ void __launch_bounds__(RT_THREADS) k_row_scan(const uint32_t* __restrict__ rcnt, uint32_t nrows,
                                                                const uint32_t* __restrict__ btot,
                                                                uint32_t* __restrict__ srow, uint32_t* __restrict__ mrow,
                                                                uint32_t* __restrict__ row_start, size_t ms) {
  __shared__ uint32_t sh[2][32];
  __shared__ uint32_t base[2];
  if (ms) {
    const size_t o = size_t(blockIdx.y) * ms;
    rcnt = moff(rcnt, o), btot = moff(btot, o), srow = moff(srow, o), mrow = moff(mrow, o);
    row_start = moff(row_start, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nb = gridDim.x;
  // totals of the earlier tiles
  uint32_t pa = 0, pb = 0;
  for (uint32_t t = threadIdx.x; t < blockIdx.x; t += RT_THREADS) {
    pa += __ldg(btot + t);
    pb += __ldg(btot + nb + t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pa += __shfl_xor_sync(0xffffffffu, pa, o);
    pb += __shfl_xor_sync(0xffffffffu, pb, o);
  }
  if (lane == 0) {
    sh[0][warp] = pa;
    sh[1][warp] = pb;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    uint32_t t = 0;
    for (int w = 0; w < RT_THREADS / 32; ++w) t += sh[threadIdx.x][w];
    base[threadIdx.x] = t;
  }
  __syncthreads();
  // this thread's RT_ITEMS consecutive rows, then a block scan of the thread sums
  const uint32_t r0 = blockIdx.x * RT_TILE + threadIdx.x * RT_ITEMS;
  uint32_t ca[RT_ITEMS], cb[RT_ITEMS], sa = 0, sb = 0;
#pragma unroll
  for (int k = 0; k < RT_ITEMS; ++k) {
    const uint32_t r = r0 + k;
    ca[k] = r < nrows ? __ldg(rcnt + r) : 0u;
    cb[k] = r < nrows ? __ldg(rcnt + nrows + r) : 0u;
    sa += ca[k];
    sb += cb[k];
  }
  uint32_t ia = sa, ib = sb;  // inclusive warp scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ua = __shfl_up_sync(0xffffffffu, ia, o), ub = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += ua;
      ib += ub;
    }
  }
  __syncthreads();  // sh is reused
  if (lane == 31) {
    sh[0][warp] = ia;
    sh[1][warp] = ib;
  }
  __syncthreads();
  uint32_t wa = 0, wb = 0;
  for (int w = 0; w < warp; ++w) {
    wa += sh[0][w];
    wb += sh[1][w];
  }
  uint32_t xa = base[0] + wa + ia - sa, xb = base[1] + wb + ib - sb;
#pragma unroll
  for (int k = 0; k < RT_ITEMS; ++k) {
    const uint32_t r = r0 + k;
    if (r < nrows) {
      srow[r] = xa;
      mrow[r] = xb;
      row_start[r] = xa + xb;
    }
    xa += ca[k];
    xb += cb[k];
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == RT_THREADS - 1) {
    srow[nrows] = xa;
    mrow[nrows] = xb;
    row_start[nrows] = xa + xb;
  }
}

// movers into per-row buckets: bucket r holds the entries [mrow[r], mrow[r+1])
// of (bk, bv), in an order the placement does not depend on
static __global__ void __launch_bounds__(RS_THREADS) k_bucket_movers(
    const uint32_t* __restrict__ mk, const uint32_t* __restrict__ mv, const uint32_t* __restrict__ counts,
    const uint32_t* __restrict__ mrow, uint32_t* __restrict__ fill, uint32_t* __restrict__ bk,
    uint32_t* __restrict__ bv, uint32_t n_mesh, int log2n, size_t ms) {
  if (ms) {
    const size_t o = size_t(blockIdx.y) * ms;
    mk = moff(mk, o), mv = moff(mv, o), counts = moff(counts, o), mrow = moff(mrow, o), fill = moff(fill, o);
    bk = moff(bk, o), bv = moff(bv, o);
  }
  const uint32_t nm = counts[1], nrows = n_mesh * n_mesh;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nm; j += gridDim.x * blockDim.x) {
    const uint32_t k = mk[j];
    const uint32_t r = key_row(k, n_mesh, log2n);
    if (r >= nrows) continue;  // (only a corrupt key)
    const uint32_t at = mrow[r] + atomicAdd(fill + r, 1u);
    bk[at] = k;
    bv[at] = mv[j];
  }
}

// The placement, one thread per output record over all of them: thread i <
// ns (the stayers' count) takes stayer i (the sorted (sk, sv) of the
// partition), thread ns + u the mover in bucket entry u.  Every record goes
// to the place of its (key, previous slot) in its row: a stayer of row r moves
// up by the movers of the rows before it (mrow[r]) and by the bucket entries
// of its own row that sort before it, a mover lands at row_start[r] plus the
// row's stayers before it (a binary search) and the bucket entries before it.
// Consecutive stayers keep consecutive places except at the few rows that
// take movers, so the keys, the slots, the gathered records and the written
// records all stream through memory in order.  The keys go to keys_out and the
// records, gathered from their previous slots, to (pos_out, mom_out).
constexpr int PF_THREADS = 256;

template <typename V4, bool PACKED>
__global__ void __launch_bounds__(PF_THREADS) k_place(
    const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv, const uint32_t* __restrict__ bk,
    const uint32_t* __restrict__ bv, const uint32_t* __restrict__ srow, const uint32_t* __restrict__ mrow,
    const uint32_t* __restrict__ row_start, const uint32_t* __restrict__ counts, uint32_t n, uint32_t n_mesh,
    int log2n, uint32_t* __restrict__ keys_out, const V4* __restrict__ pos_in, const V4* __restrict__ mom_in,
    V4* __restrict__ pos_out, V4* __restrict__ mom_out, size_t ms) {
  if constexpr (PACKED) {
    const size_t o = size_t(blockIdx.y) * ms;
    sk = moff(sk, o), sv = moff(sv, o), bk = moff(bk, o), bv = moff(bv, o), srow = moff(srow, o);
    mrow = moff(mrow, o), row_start = moff(row_start, o), counts = moff(counts, o), keys_out = moff(keys_out, o);
    pos_in = moff(pos_in, o), mom_in = moff(mom_in, o), pos_out = moff(pos_out, o), mom_out = moff(mom_out, o);
  }
  const uint32_t ns = counts[0], nrows = n_mesh * n_mesh;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const bool stayer = i < ns;
    const uint32_t k = stayer ? __ldg(sk + i) : __ldg(bk + (i - ns));
    const uint32_t v = stayer ? __ldg(sv + i) : __ldg(bv + (i - ns));
    // the record is requested as soon as its slot is known: its load overlaps the
    // place computation instead of following it
    if (v >= n) continue;  // (only after corrupt counts)
    const V4 pr = pos_in[v], mr = mom_in[v];
    const uint32_t r = key_row(k, n_mesh, log2n);
    if (r >= nrows) continue;  // (only a corrupt key)
    const uint32_t m0 = __ldg(mrow + r), m1 = __ldg(mrow + r + 1);
    uint32_t c = 0;
    for (uint32_t u = m0; u < m1; ++u) c += kv_less(__ldg(bk + u), __ldg(bv + u), k, v) ? 1u : 0u;
    uint32_t out;
    if (stayer) {
      out = i + m0 + c;
    } else {
      const uint32_t s0 = __ldg(srow + r);
      uint32_t lo = s0, hi = __ldg(srow + r + 1);
      while (lo < hi) {  // the row's stayers before it
        const uint32_t mid = (lo + hi) >> 1;
        if (kv_less(__ldg(sk + mid), __ldg(sv + mid), k, v))
          lo = mid + 1;
        else
          hi = mid;
      }
      out = __ldg(row_start + r) + c + (lo - s0);
    }
    if (out >= n) continue;  // (only after corrupt counts)
    keys_out[out] = k;
    pos_out[out] = pr;
    mom_out[out] = mr;
  }
}

// the three parts of the re-sort: the partition, the rows (scan and
// buckets) and the placement
template <typename V4>
inline cudaError_t launch_resort_place(int part, const uint32_t* keys, int64_t n, const uint32_t* tcount, uint32_t* sk,
                                       uint32_t* sv, uint32_t* mk, uint32_t* mv, uint32_t* bk, uint32_t* bv,
                                       uint32_t* counts, uint32_t* rcnt, uint32_t* btot, uint32_t* srow, uint32_t* mrow,
                                       uint32_t* row_start, Mesh m, unsigned long long* stats, uint32_t* keys_out,
                                       const V4* pos_in, const V4* mom_in, V4* pos_out, V4* mom_out, int sms,
                                       cudaStream_t s, int nm, size_t ms) {
  const size_t o = nm > 1 ? ms : 0;
  const uint32_t N = uint32_t(m.n), nrows = N * N;
  if (part == 0) {
    const unsigned ntiles = unsigned((n + RS_TILE - 1) / RS_TILE);
    // up to PART_OWN_SCAN_TILES tiles each block sums the counts of the tiles before it
    const int own = ntiles <= PART_OWN_SCAN_TILES;
    if (!own) k_tile_scan<<<dim3(1, unsigned(nm)), TS_THREADS, 0, s>>>(const_cast<uint32_t*>(tcount), ntiles, o);
    k_mover_partition<<<dim3(ntiles, unsigned(nm)), RS_THREADS, 0, s>>>(keys, n, tcount, sk, sv, mk, mv, counts, rcnt,
                                                                       N, m.log2n, stats, own, o);
  } else if (part == 1) {
    const unsigned nb = (nrows + RT_TILE - 1) / RT_TILE;
    k_row_totals<<<dim3(nb, unsigned(nm)), RT_THREADS, 0, s>>>(rcnt, nrows, btot, o);
    k_row_scan<<<dim3(nb, unsigned(nm)), RT_THREADS, 0, s>>>(rcnt, nrows, btot, srow, mrow, row_start, o);
    // the bucket scatter runs over the device's mover count: a grid of resident blocks shared by the members
    int64_t cap = int64_t(16) * sms / nm;
    if (cap < 1) cap = 1;
    const int64_t need = (n + RS_THREADS - 1) / RS_THREADS;
    const unsigned mg = unsigned(need < cap ? need : cap);
    k_bucket_movers<<<dim3(mg, unsigned(nm)), RS_THREADS, 0, s>>>(mk, mv, counts, mrow, rcnt + 2 * nrows, bk, bv, N,
                                                                  m.log2n, o);
  } else {
    // a grid of resident blocks shared by the members, striding over the records
    int64_t cap = int64_t(8) * sms / nm;
    if (cap < 1) cap = 1;
    const int64_t need = (n + PF_THREADS - 1) / PF_THREADS;
    const dim3 grid(unsigned(need < cap ? need : cap), unsigned(nm));
    if (nm > 1)
      k_place<V4, true><<<grid, PF_THREADS, 0, s>>>(sk, sv, bk, bv, srow, mrow, row_start, counts, uint32_t(n), N,
                                                    m.log2n, keys_out, pos_in, mom_in, pos_out, mom_out, o);
    else
      k_place<V4, false><<<grid, PF_THREADS, 0, s>>>(sk, sv, bk, bv, srow, mrow, row_start, counts, uint32_t(n), N,
                                                     m.log2n, keys_out, pos_in, mom_in, pos_out, mom_out, 0);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_resort(int part, const uint32_t* keys, int64_t n, const uint32_t* tcount, uint32_t* sk,
                          uint32_t* sv, uint32_t* mk, uint32_t* mv, uint32_t* bk, uint32_t* bv, uint32_t* counts,
                          uint32_t* rcnt, uint32_t* btot, uint32_t* srow, uint32_t* mrow, uint32_t* row_start, Mesh m,
                          unsigned long long* stats, uint32_t* keys_out, const void* pos_in, const void* mom_in,
                          void* pos_out, void* mom_out, int sms, cudaStream_t s, int nm, size_t ms) {
  using V4 = typename VT<R>::v4;
  return launch_resort_place<V4>(part, keys, n, tcount, sk, sv, mk, mv, bk, bv, counts, rcnt, btot, srow, mrow,
                                 row_start, m, stats, keys_out, (const V4*)pos_in, (const V4*)mom_in, (V4*)pos_out,
                                 (V4*)mom_out, sms, s, nm, ms);
}

template <typename R>
cudaError_t launch_sort_pass(bool last, const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int shift,
                             int bits, const uint32_t* digit_total, uint64_t* status, uint32_t* tile_counter,
                             const uint32_t* epoch, int pass, int ntiles, uint32_t* keys_out, uint32_t* vals_out,
                             const void* pos_in, const void* mom_in, void* pos_out, void* mom_out, uint32_t* err,
                             cudaStream_t s, const uint32_t* n_dev, int nm, size_t ms, int spin_limit) {
  if (spin_limit < 1) spin_limit = RS_SPIN_LIMIT;
  using V4 = typename VT<R>::v4;
  if (nm > 1 && (last || !n_dev)) return cudaErrorInvalidValue;  // packed groups: mover passes only
  const size_t o = nm > 1 ? ms : 0;
  // persistent blocks (they claim tiles until none is left): at most RS_PASS_BLOCKS in all
  int per = RS_PASS_BLOCKS / nm;
  if (per < 1) per = 1;
  const dim3 grid = dim3(unsigned(ntiles < per ? ntiles : per), unsigned(nm), 1u);
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
    k_sort_pass<true, V4><<<grid, RS_THREADS, smem, s>>>(keys_in, vals_in, n, shift, bits, digit_total, status,
                                                         tile_counter, epoch, pass, keys_out, vals_out,
                                                         (const V4*)pos_in, (const V4*)mom_in, (V4*)pos_out,
                                                         (V4*)mom_out, err, n_dev, o, spin_limit);
  } else {
    k_sort_pass<false, V4><<<grid, RS_THREADS, smem, s>>>(keys_in, vals_in, n, shift, bits, digit_total, status,
                                                          tile_counter, epoch, pass, keys_out, vals_out, nullptr,
                                                          nullptr, nullptr, nullptr, err, n_dev, o, spin_limit);
  }
  return cudaGetLastError();
}

}  // namespace pm
