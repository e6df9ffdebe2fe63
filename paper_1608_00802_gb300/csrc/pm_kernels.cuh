// Device kernels of the particle-mesh step with quantum pressure
// (Veltmaat & Niemeyer, arXiv:1608.00802, Sec. II.A), templated on the real
// type R (float: int32 cell + fp32 offset positions and fp32 mesh; double:
// the plain fp64 path).  Included by pm_kernels_f32.cu / pm_kernels_f64.cu.
//
// Particle storage (sorted by cell between steps):
//   pos[i] = {cell (bits), fx, fy, fz}   offsets in cell units, in [0,1)
//   mom[i] = {px, py, pz, id (bits)}     p = a^2 dx/dt
// None of these kernels use floating-point atomics on the step's data, so a
// step is bitwise reproducible for a fixed launch configuration.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pm_internal.h"
#include "pm_bulk.cuh"

namespace pm {

// ---------------------------------------------------------------- record access
__device__ __forceinline__ uint32_t rec_cell(const float4& r) { return __float_as_uint(r.x); }
__device__ __forceinline__ uint32_t rec_cell(const D4& r) { return (uint32_t)__double_as_longlong(r.x); }
__device__ __forceinline__ uint32_t rec_id(const float4& r) { return __float_as_uint(r.w); }
__device__ __forceinline__ uint32_t rec_id(const D4& r) { return (uint32_t)__double_as_longlong(r.w); }
__device__ __forceinline__ float4 make_pos(uint32_t c, float fx, float fy, float fz) {
  return make_float4(__uint_as_float(c), fx, fy, fz);
}
__device__ __forceinline__ D4 make_pos(uint32_t c, double fx, double fy, double fz) {
  D4 r;
  r.x = __longlong_as_double((long long)c);
  r.y = fx;
  r.z = fy;
  r.w = fz;
  return r;
}
__device__ __forceinline__ float4 make_mom(float px, float py, float pz, uint32_t id) {
  return make_float4(px, py, pz, __uint_as_float(id));
}
__device__ __forceinline__ D4 make_mom(double px, double py, double pz, uint32_t id) {
  D4 r;
  r.x = px;
  r.y = py;
  r.z = pz;
  r.w = __longlong_as_double((long long)id);
  return r;
}
template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ D4 ldg<D4>(const D4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  D4 r;
  r.x = a.x;
  r.y = a.y;
  r.z = b.x;
  r.w = b.y;
  return r;
}

// Typed math: each call names its precision, so that fp32 code never takes
// an fp64 routine (fp64 runs at a small fraction of the fp32 rate here).
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ float r_floor(float x) { return floorf(x); }
__device__ __forceinline__ double r_floor(double x) { return ::floor(x); }
__device__ __forceinline__ bool r_finite(float x) { return isfinite(x); }
__device__ __forceinline__ bool r_finite(double x) { return isfinite(x); }

// ---------------------------------------------------------------- float-float
// Extended precision from pairs of fp32 numbers (error-free transformations of
// Dekker 1971 / Knuth TAOCP 4.2.2): value = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits on the fp32 pipes.  Used where the method asks for
// more than fp32 (near-empty nodes, diagnostic sums) because fp64 throughput
// is a small fraction of fp32 throughput on this GPU.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // needs |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  return fast_two_sum(p, fmaf(a.lo, b, e));
}
// Hardware approximations of 1/sqrt(x) and 1/x (a few ulp) with subnormal
// inputs and results flushed to zero; the stencils call them only on floored
// densities (normal fp32 numbers, rho_floor >= 1e-30) and their square roots.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The square root starts from the hardware approximation (a few ulp) and is
// refined by one Newton step whose residual is formed exactly with fma, which
// brings it to float-float accuracy.
__device__ __forceinline__ ff ff_sqrt(float x) {  // x > 0, normal
  const float rs = rsqrt_ftz(x);
  const float s = x * rs;
  const float r = fmaf(-s, s, x);  // x - s^2, exact
  return fast_two_sum(s, r * (0.5f * rs));
}
// fp32 quotient of two float-float numbers: the fp32 quotient from the
// hardware reciprocal, refined by one Newton correction whose residual
// a - q b is formed in float-float.  The result is rounded to fp32, and one
// correction already brings it to about that rounding.
__device__ __forceinline__ float ff_quot(ff a, ff b) {
  const float inv = rcp_ftz(b.hi);
  const float q1 = a.hi * inv;
  const ff r = ff_sub(a, ff_mul_f(b, q1));
  return fmaf(r.hi, inv, q1);
}
__device__ __forceinline__ ff ff_shfl_down(ff v, int o) {
  return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ void split_cell(uint32_t c, const Mesh& m, int& x, int& y, int& z) {
  if (m.log2n >= 0) {
    uint32_t mask = uint32_t(m.n) - 1u;
    x = int(c & mask);
    y = int((c >> m.log2n) & mask);
    z = int(c >> (2 * m.log2n));
  } else {
    uint32_t q = c / uint32_t(m.n);
    x = int(c - q * uint32_t(m.n));
    z = int(q / uint32_t(m.n));
    y = int(q - uint32_t(z) * uint32_t(m.n));
  }
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV fp32 values per thread: float-float inside each warp, fp64
// across warps and blocks (fixed order, so the sums are reproducible).
template <int NV>
__device__ __forceinline__ void block_sum_store_ff(const ff (&v)[NV], double* part, int nblocks, int bid) {
  __shared__ double shf[32][NV];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    ff s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
    if (lane == 0) shf[warp][k] = double(s.hi) + double(s.lo);
  }
  __syncthreads();
  if (tid == 0) {
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += shf[w][k];
      part[k * nblocks + bid] = s;
    }
  }
}

template <int NV>
__device__ __forceinline__ void block_sum_store(float (&v)[NV], double* part, int nblocks, int bid = -1) {
  ff f[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) f[k] = ff{v[k], 0.0f};
  block_sum_store_ff<NV>(f, part, nblocks, bid < 0 ? int(blockIdx.x) : bid);
}

// sum of squared forward differences of one node, rounded the same way in
// every kernel (explicit fused multiply-adds)
__device__ __forceinline__ float krho_term(float dx, float dy, float dz) {
  return fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
}

// running float-float sum of fp32 terms (the error of each addition is kept)
__device__ __forceinline__ void ff_accumulate(ff& a, float v) {
  const ff t = two_sum(a.hi, v);
  a.hi = t.hi;
  a.lo += t.lo;
}

// Block sum of NV doubles (fixed order); thread 0 gets the totals.
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* part, int nblocks) {
  __shared__ double sh[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w][k];
      part[k * nblocks + blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------- load + cell keys
template <typename R>
__global__ void k_init_particles(const double* __restrict__ x, const double* __restrict__ p, int64_t n, Mesh m,
                                 double inv_dx, typename VT<R>::v4* pos, typename VT<R>::v4* mom,
                                 uint32_t* keys, uint32_t* err) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  R f[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double u = x[3 * i + d] * inv_dx;
    if (!isfinite(u)) {
      atomicOr(err, ERR_NONFINITE);
      u = 0.0;
    }
    double fl = floor(u);
    double fr = u - fl;
    int64_t ci = (int64_t)fl;
    R o = R(fr);
    if (o >= R(1)) {  // rounding of the offset to R reached 1: carry into the cell
      o = R(0);
      ci += 1;
    }
    ci %= m.n;
    if (ci < 0) ci += m.n;
    c[d] = int(ci);
    f[d] = o;
  }
  uint32_t cell = (uint32_t(c[2]) * uint32_t(m.n) + uint32_t(c[1])) * uint32_t(m.n) + uint32_t(c[0]);
  pos[i] = make_pos(cell, f[0], f[1], f[2]);
  // p null: particles at rest (the allocation-free deposit needs no momenta)
  mom[i] = p ? make_mom(R(p[3 * i]), R(p[3 * i + 1]), R(p[3 * i + 2]), uint32_t(i))
             : make_mom(R(0), R(0), R(0), uint32_t(i));
  keys[i] = cell;
}

// ---------------------------------------------------------------- cloud-in-cell deposit
// e / d for every 32-bit e, by the multiply-high method for invariant divisors
// (Granlund & Montgomery 1994): mul = 2^32 (2^l - d) / d + 1, l = ceil(log2 d)
struct DivU32 {
  uint32_t mul;
  int l;
};
inline DivU32 divu32_make(uint32_t d) {
  int l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  DivU32 r;
  r.mul = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  r.l = l;
  return r;
}
__device__ __forceinline__ uint32_t divu32(uint32_t e, DivU32 dv) {
  if (dv.l == 0) return e;
  const uint32_t t = __umulhi(dv.mul, e);
  return (t + ((e - t) >> 1)) >> (dv.l - 1);
}

// rho_n = norm * sum_i W(x_n - q_i): Eq. (rhodis) with the cloud-in-cell
// tent, no floating-point atomics.  A warp owns a tile of TY x TZ mesh rows
// (rows y0 .. y0 + TY - 1 of the planes z0 .. z0 + TZ - 1) and keeps them in
// shared memory (N + 1 slots per row, slot N = node 0 seen from cell N - 1).
// A particle of source row (z', y') adds to the rows (z' + dz, y' + dy),
// dz, dy in {0, 1}, so the warp reads the source rows y0 - 1 .. y0 + TY - 1
// of the planes z0 - 1 .. z0 + TZ - 1: each particle (TY + 1)(TZ + 1)/(TY TZ)
// times (1.875 for 2 x 4, against 2.5 for a column of four rows of one y).
// The source rows of one plane follow each other in the sorted order (a
// "chain"; the periodic seam at y = 0 splits it), so the warp takes a chain
// in full batches of 32 records that run across row boundaries.  In a batch:
//  - equal cells (adjacent after the sort) are summed first by a segmented
//    warp scan in a fixed tree order, and only the run's last lane adds;
//  - the f_x weight of cell t goes to node t + 1, which is the 1 - f_x node
//    of cell t + 1, so the f_x adds and the 1 - f_x adds are separated by
//    __syncwarp;
//  - source rows y' and y' + 1 share the destination row y' + 1, so the adds
//    run in two phases: dy = 0 (each source row to its own row), then dy = 1
//    (to the next row); within a phase no two source rows meet.
// The warp alone writes its rows, in a fixed order of chains, batches and
// phases, so the result is reproducible.
constexpr int DEP_WARPS = 8;

// slots of a deposit row: N + 1 rounded up to 16 bytes
template <typename R>
__host__ __device__ inline int deposit_stride_of(int n) {
  const int q = 16 / int(sizeof(R));
  return (n + 1 + q - 1) / q * q;
}

template <typename R, int TY, int TZ, bool PACKED>
__global__ void __launch_bounds__(DEP_WARPS * 32) k_deposit(const typename VT<R>::v4* __restrict__ pos,
                                                            const uint32_t* __restrict__ row_start, uint32_t np,
                                                            Mesh m, DivU32 dvn, R norm, R* __restrict__ rho,
                                                            size_t ms) {
  using V4 = typename VT<R>::v4;
  static_assert((TY + 1) * (TZ + 1) <= 32, "one source row per lane");
  if constexpr (PACKED) {  // member blockIdx.y of a packed group
    const size_t o = size_t(blockIdx.y) * ms;
    pos = moff(pos, o), row_start = moff(row_start, o), rho = moff(rho, o);
  }
  extern __shared__ __align__(16) unsigned char dep_smem[];
  const int n = m.n, stride = deposit_stride_of<R>(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int span_y = nw * TY, tiles_y = (n + span_y - 1) / span_y;
  const int y0 = int(blockIdx.x % unsigned(tiles_y)) * span_y + warp * TY, z0 = int(blockIdx.x / unsigned(tiles_y)) * TZ;
  if (y0 >= n) return;
  const int ty = min(TY, n - y0), tz = min(TZ, n - z0);
  R* acc = reinterpret_cast<R*>(dep_smem) + warp * (TY * TZ * stride);  // [TZ][TY][N + 1], this warp's
  for (int i = lane; i < TY * TZ * stride * int(sizeof(R)) / 16; i += 32)
    reinterpret_cast<float4*>(acc)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  __syncwarp();
  // the (tz + 1)(ty + 1) source rows, one per lane: plane slot sz (plane z0 - 1 + sz), row slot ly
  // (row y0 - 1 + ly).  A lane whose row does not follow the previous lane's in memory heads a chain,
  // which runs up to the next head.
  const int nr = (tz + 1) * (ty + 1);
  const int sz_l = lane / (ty + 1), ly_l = lane - sz_l * (ty + 1);
  bool head = false;
  uint32_t b = 0, e = 0, base = 0;
  if (lane < nr) {
    const int yr = wrap(y0 - 1 + ly_l, n);
    const uint32_t srow = uint32_t(wrap(z0 - 1 + sz_l, n)) * uint32_t(n) + uint32_t(yr);
    b = __ldg(row_start + srow);
    e = min(__ldg(row_start + srow + 1), np);
    head = ly_l == 0 || yr != wrap(y0 - 2 + ly_l, n) + 1;
    base = srow * uint32_t(n);
  }
  const uint32_t heads = __ballot_sync(0xffffffffu, head);
  const uint32_t later = heads & ~((2u << lane) - 1u);
  const int last = (later ? __ffs(later) - 1 : nr) - 1;                  // the chain's last row (head lanes)
  const uint32_t ce = __shfl_sync(0xffffffffu, e, last < 0 ? 0 : last);  // the chain's end
  const int crows = last - lane + 1;                                     // rows in the chain
  uint32_t todo = __ballot_sync(0xffffffffu, head && b < ce);            // nonempty chains, in order
  if (todo) {
    int k = __ffs(todo) - 1;
    todo &= todo - 1;
    uint32_t j = __shfl_sync(0xffffffffu, b, k), en = __shfl_sync(0xffffffffu, ce, k);
    V4 rec = {};
    if (j + lane < en) rec = ldg(pos + j + lane);
    // batches of 32 records, the next batch's records loaded while the current one is added
    for (;;) {
      int k2 = k;
      uint32_t j2 = j + 32, e2 = en, todo2 = todo;
      bool more = true;
      if (j2 >= en) {
        if (todo2) {
          k2 = __ffs(todo2) - 1;
          todo2 &= todo2 - 1;
          j2 = __shfl_sync(0xffffffffu, b, k2), e2 = __shfl_sync(0xffffffffu, ce, k2);
        } else {
          more = false;
        }
      }
      V4 rec2 = {};
      if (more && j2 + lane < e2) rec2 = ldg(pos + j2 + lane);
      const int sz = __shfl_sync(0xffffffffu, sz_l, k), ly0 = __shfl_sync(0xffffffffu, ly_l, k);
      const int nrc = __shfl_sync(0xffffffffu, crows, k);
      const uint32_t cbase = __shfl_sync(0xffffffffu, base, k);
      bool valid = j + lane < en;
      uint32_t key = 0x80000000u + uint32_t(lane);  // invalid lanes: unique keys
      int x = 0, ly = 0;
      R v[2][2][2];  // [dy][dz][0: 1 - f_x to node x, 1: f_x to node x + 1]
      if (valid) {
        const uint32_t rel = rec_cell(rec) - cbase;
        const uint32_t off = divu32(rel, dvn);
        // a record outside the chain's rows (only after a sort whose look-back
        // timed out, which the error word reports) is skipped, not written out of bounds
        valid = off < uint32_t(nrc);
        if (valid) key = rel, ly = ly0 + int(off), x = int(rel - off * uint32_t(n));
      }
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const R wz = dz ? rec.w : R(1) - rec.w;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const R w = (dy ? rec.z : R(1) - rec.z) * wz;
          v[dy][dz][1] = rec.y * w;
          v[dy][dz][0] = (R(1) - rec.y) * w;
        }
      }
      const uint32_t kp = __shfl_up_sync(0xffffffffu, key, 1);
      const uint32_t runs = __ballot_sync(0xffffffffu, lane == 0 || kp != key);
      if (runs != 0xffffffffu) {  // some cell holds several particles of the batch
        // length of the run that starts at this lane (0 elsewhere), and the longest; the scan stops
        // after the steps the longest run needs (the skipped steps would add nothing)
        const uint32_t above = runs & ~((2u << lane) - 1u);
        const int len = ((runs >> lane) & 1u) ? (above ? __ffs(above) - 1 : 32) - lane : 0;
        const int longest = int(__reduce_max_sync(0xffffffffu, uint32_t(len)));
        for (int off = 1; off < longest; off <<= 1) {
          R u[2][2][2];
#pragma unroll
          for (int a = 0; a < 8; ++a) (&u[0][0][0])[a] = __shfl_up_sync(0xffffffffu, (&v[0][0][0])[a], off);
          // lane - off is in this lane's run iff no run starts in (lane - off, lane]
          const uint32_t span = lane >= off ? ((2u << lane) - 1u) & ~((2u << (lane - off)) - 1u) : 0u;
          if (lane >= off && !(runs & span)) {
#pragma unroll
            for (int a = 0; a < 8; ++a) (&v[0][0][0])[a] += (&u[0][0][0])[a];
          }
        }
      }
      const bool add = valid && (lane == 31 || ((runs >> (lane + 1)) & 1u));
      // planes sz - 1 (dz = 0) and sz (dz = 1); the edge plane slots of the tile have one of the two,
      // and the chain's slot is the same for the whole warp, so the adds branch on it instead of
      // issuing the missing half predicated off
      auto adds = [&](auto h0, auto h1) {
        constexpr bool H0 = decltype(h0)::value, H1 = decltype(h1)::value;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int ry = ly - 1 + dy;  // destination row of this phase
          const bool okr = add && unsigned(ry) < unsigned(ty);
          if (!__any_sync(0xffffffffu, okr)) continue;  // a batch within the chain's first or last row
          const int a0 = ((sz - 1) * TY + ry) * stride + x, a1 = a0 + TY * stride;
          if (H0 && okr) acc[a0 + 1] += v[dy][0][1];
          if (H1 && okr) acc[a1 + 1] += v[dy][1][1];
          __syncwarp();
          if (H0 && okr) acc[a0] += v[dy][0][0];
          if (H1 && okr) acc[a1] += v[dy][1][0];
          __syncwarp();
        }
      };
      if (sz >= 1 && sz < tz)
        adds(std::true_type{}, std::true_type{});
      else if (sz >= 1)
        adds(std::true_type{}, std::false_type{});
      else
        adds(std::false_type{}, std::true_type{});
      if (!more) break;
      k = k2, j = j2, en = e2, todo = todo2, rec = rec2;
    }
  }
  for (int lz = 0; lz < tz; ++lz) {
    for (int ry = 0; ry < ty; ++ry) {
      R* a = acc + (lz * TY + ry) * stride;
      if (lane == 0) a[0] += a[n];
      __syncwarp();
      R* out = rho + (size_t(z0 + lz) * n + size_t(y0 + ry)) * n;
      if constexpr (sizeof(R) == 4) {
        if ((n & 3) == 0) {  // 16-byte loads and stores
          for (int i = 4 * lane; i < n; i += 128) {
            const float4 q = *reinterpret_cast<const float4*>(a + i);
            *reinterpret_cast<float4*>(out + i) = make_float4(q.x * norm, q.y * norm, q.z * norm, q.w * norm);
          }
          continue;
        }
      }
      for (int i = lane; i < n; i += 32) out[i] = a[i] * norm;
    }
  }
}

// ---------------------------------------------------------------- Green's function
__device__ __forceinline__ float sinpi_sq(float t) {
  float s = sinpif(t);
  return s * s;
}
__device__ __forceinline__ double sinpi_sq(double t) {
  double s = sinpi(t);
  return s * s;
}

// phi^_k = coef * rho^_k / sum_d sin^2(pi j_d / N), coef = -(3/2) Om dx^2 / (4 N^3):
// the exact periodic inverse of the compact seven-point Laplacian with the
// inverse-FFT normalisation folded in; k = 0 set to zero.  Also accumulates
// sum_n rho_n phi_n = sum_k w_k G_k |rho^_k|^2 (Parseval over the half spectrum,
// w = 1 on the x = 0 and x = N/2 planes, 2 elsewhere) for W_g.
// phi^ = -(3/2) Omega_m rho^ / kappa^2 in place over the half spectrum, with
// kappa^2 = (4/dx^2) sum_d sin^2(k_d dx/2) the exact symbol of the seven-point
// Laplacian (the comoving Poisson equation of Sec. II), and the Parseval
// partial of W_g.  Flat over the n^2 (n/2+1) complex values: every lane busy,
// four independent loads in flight per thread.
template <typename R>
__device__ __forceinline__ void green_one(typename VT<R>::cplx& v, uint32_t e, uint32_t nh, DivU32 dv, const Mesh& m,
                                          const R* s2, R coef, R& wsum) {
  const uint32_t n = uint32_t(m.n);
  const uint32_t row = divu32(e, dv), jx = e - row * nh;
  uint32_t jz, jy;
  if (m.log2n >= 0) {
    jz = row >> m.log2n;
    jy = row & (n - 1u);
  } else {
    jz = row / n;
    jy = row - jz * n;
  }
  const R syz = s2[jy] + s2[jz];
  const R s = syz + s2[jx];
  const R g = (row == 0 && jx == 0) ? R(0) : coef / s;
  const R re = v.x, im = v.y;
  const R w = (jx == 0 || jx == n / 2) ? R(1) : R(2);
  wsum += w * g * (re * re + im * im);
  v.x = re * g;
  v.y = im * g;
}

// coefp (nullable): the coefficient in device memory (member 0's, ms bytes
// apart), used instead of coef by the packed groups, whose members differ in box
template <typename R, bool PACKED>
__global__ void __launch_bounds__(MESH_THREADS) k_green(typename VT<R>::cplx* spec, Mesh m, R coef, DivU32 dv,
                                                        double* part, const double* coefp, size_t ms) {
  if constexpr (PACKED) {  // member blockIdx.y of a packed group
    const size_t o = size_t(blockIdx.y) * ms;
    spec = moff(spec, o), part = moff(part, o);
    coef = R(*moff(coefp, o));
  }
  extern __shared__ __align__(16) unsigned char green_smem[];
  R* s2 = reinterpret_cast<R*>(green_smem);  // sin^2(pi j / N), j = 0..N-1
  const uint32_t n = uint32_t(m.n), nh = n / 2 + 1;
  const R inv_n = R(1) / R(n);
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) s2[j] = sinpi_sq(R(j) * inv_n);
  __syncthreads();
  R wsum = R(0);
  const uint32_t total = m.n2 * nh, stride = gridDim.x * blockDim.x;
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < total; e += 4 * stride) {
    typename VT<R>::cplx v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = spec[e + k * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      green_one<R>(v[k], e + k * stride, nh, dv, m, s2, coef, wsum);
      spec[e + k * stride] = v[k];
    }
  }
  for (; e < total; e += stride) {
    typename VT<R>::cplx v = spec[e];
    green_one<R>(v, e, nh, dv, m, s2, coef, wsum);
    spec[e] = v;
  }
  R acc[1] = {wsum};
  block_sum_store<1>(acc, part, gridDim.x);
}

// ---------------------------------------------------------------- Green's function inside the z transform
// With the x and y transforms done plane by plane (batched 2D cuFFT), the z
// transform, the Green multiplication and the inverse z transform of one
// column of the half spectrum need nothing but that column: one kernel does
// all three in shared memory, so the spectrum crosses HBM once (read + write)
// between the two 2D transforms instead of three times (3D forward's last
// pass, k_green, 3D inverse's first pass).
//
// A z column of N = P Q points is transformed in two steps (the four-step
// factorisation, n = j + P m, k = k1 + Q k2):
//   X[k1 + Q k2] = sum_j W_P^{j k2} W_N^{j k1} sum_m x[j + P m] W_Q^{m k1},
// so thread j does a Q-point DFT over m and the twiddle W_N^{j k1}, and, after
// one exchange through shared memory, thread k1 a P-point DFT over j.  The
// inverse runs the same steps backwards with conjugate twiddles; the thread
// that ends the forward transform holds X[k1 + Q k2] for every k2, so it
// multiplies by G and starts the inverse without an exchange.  A block owns 16
// adjacent columns of the flattened (ky, kx) plane (128 contiguous bytes per z
// row: every global access is a full segment).

// exp(2 pi i t / 32) for t < 32: the twiddles of the in-register DFTs
__device__ constexpr float kCos32[32] = {
    1.0f,          0.980785251f,  0.923879504f,  0.831469595f,  0.707106769f,  0.555570245f,  0.382683426f,
    0.195090324f,  0.0f,          -0.195090324f, -0.382683426f, -0.555570245f, -0.707106769f, -0.831469595f,
    -0.923879504f, -0.980785251f, -1.0f,         -0.980785251f, -0.923879504f, -0.831469595f, -0.707106769f,
    -0.555570245f, -0.382683426f, -0.195090324f, 0.0f,          0.195090324f,  0.382683426f,  0.555570245f,
    0.707106769f,  0.831469595f,  0.923879504f,  0.980785251f};
__device__ constexpr float kSin32[32] = {
    0.0f,          0.195090324f,  0.382683426f,  0.555570245f,  0.707106769f,  0.831469595f,  0.923879504f,
    0.980785251f,  1.0f,          0.980785251f,  0.923879504f,  0.831469595f,  0.707106769f,  0.555570245f,
    0.382683426f,  0.195090324f,  0.0f,          -0.195090324f, -0.382683426f, -0.555570245f, -0.707106769f,
    -0.831469595f, -0.923879504f, -0.980785251f, -1.0f,         -0.980785251f, -0.923879504f, -0.831469595f,
    -0.707106769f, -0.555570245f, -0.382683426f, -0.195090324f};

__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// a * exp(-+2 pi i t / 32) (forward: minus), t < 16 known at compile time after unrolling
template <bool INV>
__device__ __forceinline__ float2 twiddle32(float2 a, int t) {
  if (t == 0) return a;
  if (t == 8) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);  // times +i / -i
  constexpr float h = 0.707106769f;                                           // cos(pi / 4)
  if (t == 4) return INV ? make_float2(h * (a.x - a.y), h * (a.x + a.y)) : make_float2(h * (a.x + a.y), h * (a.y - a.x));
  if (t == 12)
    return INV ? make_float2(-h * (a.x + a.y), h * (a.x - a.y)) : make_float2(h * (a.y - a.x), -h * (a.x + a.y));
  return cmul(a, make_float2(kCos32[t], INV ? kSin32[t] : -kSin32[t]));
}

// In-register DFT of M <= 32 points, radix-2 decimation in frequency: natural
// order in, bit-reversed order out (a[bitrev(k)] = X[k]); INV: exp(+2 pi i nk/M).
template <int M, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&a)[M]) {
#pragma unroll
  for (int len = M; len >= 2; len >>= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int b = 0; b < M; b += len) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 u = a[b + j], v = a[b + j + half];
        a[b + j] = make_float2(u.x + v.x, u.y + v.y);
        a[b + j + half] = twiddle32<INV>(make_float2(u.x - v.x, u.y - v.y), j * (32 / len));
      }
    }
  }
}

template <int M>
__host__ __device__ constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 1; b < M; b <<= 1) {
    r <<= 1;
    if (k & b) r |= 1;
  }
  return r;
}

constexpr int SPZ_COLS = 16;  // z columns per block (16 complex = 128 bytes per z row)
#ifndef PM_SPZ_MINB
#define PM_SPZ_MINB 4  // resident blocks of up to 256 threads the z kernel is compiled for
#endif

// exp(-2 pi i t / N) from fp64 sincospi, and k_green's sin^2(pi t / N)
static __global__ void k_spec_tables(float2* tw, float* s2, int n) {
  const float inv_n = 1.0f / float(n);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    double sv, cv;
    sincospi(2.0 * double(t) / double(n), &sv, &cv);
    tw[t] = make_float2(float(cv), float(-sv));
    s2[t] = sinpi_sq(float(t) * inv_n);
  }
}

// z transform, phi^ = G rho^ (with k_green's arithmetic and Parseval partial
// of W_g), inverse z transform, over 16 columns of the flattened (ky, kx)
// half plane per block; N = P Q, P >= Q, 16 P threads.  coefp (packed
// groups): the coefficient in device memory, member blockIdx.y, ms bytes apart.
template <int P, int Q, bool PACKED>
__global__ void __launch_bounds__(SPZ_COLS * P, SPZ_COLS * P <= 256 ? PM_SPZ_MINB : 1) k_spec_z(float2* __restrict__ spec, const float2* __restrict__ twg,
                                                         const float* __restrict__ s2g, float coef, double* part,
                                                         const double* coefp, size_t ms) {
  constexpr int N = P * Q, T = SPZ_COLS * P;
  constexpr uint32_t NH = N / 2 + 1, PLANE = uint32_t(N) * NH;
  if constexpr (PACKED) {
    const size_t o = size_t(blockIdx.y) * ms;
    spec = moff(spec, o), part = moff(part, o);
    coef = float(*moff(coefp, o));
  }
  extern __shared__ __align__(16) unsigned char spz_smem[];
  float2* tile = reinterpret_cast<float2*>(spz_smem);  // [z][16 columns]
  float2* tw = tile + N * SPZ_COLS;
  float* s2 = reinterpret_cast<float*>(tw + N);
  const int tid = threadIdx.x;
  const uint32_t col0 = blockIdx.x * SPZ_COLS;
  // the tile by asynchronous 16-byte copies: every copy of a thread in flight at once
  for (int i = tid; i < N * 8; i += T) {
    const int r = i >> 3, q = i & 7;
    cp_async16(reinterpret_cast<float4*>(tile + r * SPZ_COLS) + q,
               reinterpret_cast<const float4*>(spec + size_t(r) * PLANE + col0) + q);
  }
  for (int i = tid; i < N; i += T) {
    tw[i] = twg[i];
    s2[i] = s2g[i];
  }
  cp_async_wait_all();
  __syncthreads();
  const int c = tid & (SPZ_COLS - 1), jt = tid / SPZ_COLS;
  {  // forward, first step: thread j, Q-point DFT over m, twiddle W_N^{j k1}
    float2 a[Q];
#pragma unroll
    for (int mm = 0; mm < Q; ++mm) a[mm] = tile[(jt + P * mm) * SPZ_COLS + c];
    dft_reg<Q, false>(a);
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1)
      tile[(jt + P * k1) * SPZ_COLS + c] = cmul(a[bitrev<Q>(k1)], tw[(jt * k1) & (N - 1)]);
  }
  __syncthreads();
  float wsum = 0.0f;
  if (jt < Q) {  // thread k1: P-point DFT over j, Green, inverse P-point DFT, conjugate twiddle
    const int k1 = jt;
    float2 b[P];
#pragma unroll
    for (int j = 0; j < P; ++j) b[j] = tile[(j + P * k1) * SPZ_COLS + c];
    dft_reg<P, false>(b);
    const uint32_t col = col0 + uint32_t(c), ky = col / NH, kx = col - ky * NH;
    const float sx = s2[kx], sy = s2[ky];
    const float w = (kx == 0 || kx == N / 2) ? 1.0f : 2.0f;
    float2 d[P];
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) {
      const int kz = k1 + Q * k2;
      float2 v = b[bitrev<P>(k2)];
      const float syz = sy + s2[kz];
      const float sum = syz + sx;
      const float g = (ky == 0 && kz == 0 && kx == 0) ? 0.0f : coef * __frcp_rn(sum);
      wsum += w * g * (v.x * v.x + v.y * v.y);
      d[k2] = make_float2(v.x * g, v.y * g);
    }
    dft_reg<P, true>(d);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const float2 t = tw[(j * k1) & (N - 1)];
      tile[(j + P * k1) * SPZ_COLS + c] = cmul(d[bitrev<P>(j)], make_float2(t.x, -t.y));
    }
  }
  __syncthreads();
  {  // inverse, second step: thread j, inverse Q-point DFT over k1
    float2 e[Q];
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) e[k1] = tile[(jt + P * k1) * SPZ_COLS + c];
    dft_reg<Q, true>(e);
#pragma unroll
    for (int mm = 0; mm < Q; ++mm) tile[(jt + P * mm) * SPZ_COLS + c] = e[bitrev<Q>(mm)];
  }
  __syncthreads();
  for (int i = tid; i < N * 8; i += T) {
    const int r = i >> 3, q = i & 7;
    reinterpret_cast<float4*>(spec + size_t(r) * PLANE + col0)[q] = reinterpret_cast<const float4*>(tile + r * SPZ_COLS)[q];
  }
  float acc[1] = {wsum};
  block_sum_store<1>(acc, part, gridDim.x);
}

// ---------------------------------------------------------------- cubic spline kernel
// The cubic spline W(r, h) of Sec. II.A on the mesh: its weights W(|x_n|, h) dx^3
// at the node offsets (periodic minimum image; with h = hc dx they are
// 8/(pi hc^3) f(r/hc), r in cells), their transform's real part divided by its
// k = 0 value (unit sum), and the multiplications by that symbol.
template <typename R>
__global__ void __launch_bounds__(MESH_THREADS) k_spline_weights(R* __restrict__ w, Mesh m, double hc) {
  const int n = m.n;
  const double c = 8.0 / (M_PI * hc * hc * hc);
  for (uint32_t node = blockIdx.x * blockDim.x + threadIdx.x; node < m.n3; node += gridDim.x * blockDim.x) {
    int x, y, z;
    split_cell(node, m, x, y, z);
    const double dx = x <= n / 2 ? x : x - n, dy = y <= n / 2 ? y : y - n, dz = z <= n / 2 ? z : z - n;
    const double u = sqrt(dx * dx + dy * dy + dz * dz) / hc;
    const double f = u <= 0.5 ? 1.0 - 6.0 * u * u + 6.0 * u * u * u : (u <= 1.0 ? 2.0 * (1.0 - u) * (1.0 - u) * (1.0 - u) : 0.0);
    w[node] = R(c * f);
  }
}

template <typename R>
__global__ void __launch_bounds__(MESH_THREADS) k_spline_symbol(const typename VT<R>::cplx* __restrict__ spec,
                                                                R* __restrict__ what, uint32_t total) {
  const R w0 = spec[0].x;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x)
    what[e] = spec[e].x / w0;
}

// The Green multiplication with the spline: spec holds rho^ (cloud-in-cell,
// smooth_in = 1) or rho_W^ (smooth_in = 0).  rho_W^ = W^ rho^ goes to spec2
// if given (normalised for the inverse transform), the force potential
// phi_S^ = W^ G rho_W^ replaces spec, and the W_g partial sums G |rho_W^|^2.
template <typename R>
__global__ void __launch_bounds__(MESH_THREADS) k_green_spline(typename VT<R>::cplx* spec,
                                                               typename VT<R>::cplx* spec2,
                                                               const R* __restrict__ what, Mesh m, R coef, R inv_n3,
                                                               DivU32 dv, double* part, int smooth_in) {
  extern __shared__ __align__(16) unsigned char gs_smem[];
  R* s2 = reinterpret_cast<R*>(gs_smem);
  const uint32_t n = uint32_t(m.n), nh = n / 2 + 1;
  const R inv_n = R(1) / R(n);
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) s2[j] = sinpi_sq(R(j) * inv_n);
  __syncthreads();
  R wsum = R(0);
  const uint32_t total = m.n2 * nh, stride = gridDim.x * blockDim.x;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const uint32_t row = divu32(e, dv), jx = e - row * nh;
    uint32_t jz, jy;
    if (m.log2n >= 0) {
      jz = row >> m.log2n;
      jy = row & (n - 1u);
    } else {
      jz = row / n;
      jy = row - jz * n;
    }
    const R syz = s2[jy] + s2[jz];
    const R sk = syz + s2[jx];
    const R g = (row == 0 && jx == 0) ? R(0) : coef / sk;
    const R wk = what[e];
    auto v = spec[e];
    if (smooth_in) {
      v.x *= wk;
      v.y *= wk;
    }
    if (spec2) {
      auto u = v;
      u.x *= inv_n3;
      u.y *= inv_n3;
      spec2[e] = u;
    }
    const R w = (jx == 0 || jx == n / 2) ? R(1) : R(2);
    wsum += w * g * (v.x * v.x + v.y * v.y);
    const R f = g * wk;
    v.x *= f;
    v.y *= f;
    spec[e] = v;
  }
  R acc[1] = {wsum};
  block_sum_store<1>(acc, part, gridDim.x);
}

// spec *= W^ / N^3 (the smoothing of a transformed field, ready for the inverse transform)
template <typename R>
__global__ void __launch_bounds__(MESH_THREADS) k_smooth_spec(typename VT<R>::cplx* spec, const R* __restrict__ what,
                                                              uint32_t total, R inv_n3) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    auto v = spec[e];
    const R f = what[e] * inv_n3;
    v.x *= f;
    v.y *= f;
    spec[e] = v;
  }
}

// The same smoothing in real space, for spline kernels whose support ends
// within three cells (h <= 4 mesh cells; the paper's runs use 3.5 and 4):
// out_n = sum_o w_o in_{n+o} over the periodic mesh with the node weights w
// (normalised to unit sum), which is the operator whose symbol the spectral
// smoothing multiplies by.  Summed in real space every output is a positive
// combination of nearby values, so it keeps their relative precision (the
// transforms' rounding is relative to the whole field's norm instead, which a
// near-empty region cannot afford).  The weight of offset (i, j, k) is
// c[i][|j|][|k|] = w(i^2 + j^2 + k^2), so with the x taps done last,
//   out(x, z) = T_0(x) + sum_{i=1..3} (T_i(x - i) + T_i(x + i)),
//   T_i(x, z) = sum_{k=-3..3} V_{|k|,i}(x, z + k),
//   V_{|k|,i}(x, p) = sum_{|j|} c[i][|j|][|k|] (in(x, y+j, p) + in(x, y-j, p)):
// one block per y row (one thread per x) and a run of z planes.  Each input
// plane p is read once per thread (its seven rows y-3..y+3), turned into the
// V values and added to the T accumulators of the seven outputs p-3..p+3,
// kept in a ring of registers; the output p-3 is then complete, and the row
// exchanges its T_i through shared memory for the x taps.  Terms with
// i^2 + j^2 + k^2 > MAXR2 are left out at compile time (their weights are 0
// when MAXR2 >= the squared support).
template <typename R>
struct SplineTaps {
  R c[4][4][4];  // c[i][|j|][|k|]
};

template <typename R, int MAXR2, int U>
__device__ __forceinline__ void smooth_plane(const R* __restrict__ in, R* __restrict__ out, const Mesh& m,
                                             const SplineTaps<R>& tp, const uint32_t (&row)[7], int p, int z0, int z1,
                                             R (&acc)[7][4], R (&v)[7], R* T, int x, int xm1, int xp1, int xm2, int xp2,
                                             int xm3, int xp3) {
  const int n = m.n;
  // v holds plane p (loaded one plane ahead); plane p + 1 is requested before p is worked on
  const R P[4] = {v[3], v[2] + v[4], v[1] + v[5], v[0] + v[6]};
  {
    const R* pl = in + size_t(wrap(p + 1, n)) * m.n2;
#pragma unroll
    for (int j = 0; j < 7; ++j) v[j] = __ldg(pl + row[j]);
  }
  // output p+3 enters the ring at slot U (slots advance by one per plane)
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[U][i] = R(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    R V[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      R a = R(0);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i * i + j * j + k * k <= MAXR2) a += tp.c[i][j][k] * P[j];
      V[i] = a;
    }
    // output p - k' with |k'| = k sits at slot (U - 3 - k') mod 7
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[(U + 4 - k + 7) % 7][i] += V[i];
      if (k) acc[(U + 4 + k) % 7][i] += V[i];
    }
  }
  // output p - 3 (slot U + 1) is complete
  const int z = p - 3;
  if (z >= z0 && z < z1) {
    const R* a = acc[(U + 1) % 7];
    T[x] = a[1];
    T[n + x] = a[2];
    T[2 * n + x] = a[3];
    __syncthreads();
    const R o = a[0] + (T[xm1] + T[xp1]) + (T[n + xm2] + T[n + xp2]) + (T[2 * n + xm3] + T[2 * n + xp3]);
    out[size_t(z) * m.n2 + row[3]] = o;
    __syncthreads();  // T is rewritten for the next output
  }
}

template <typename R, int MAXR2>
__global__ void __launch_bounds__(512) k_smooth_direct(const R* __restrict__ in, R* __restrict__ out, Mesh m,
                                                       SplineTaps<R> tp, int zc) {
  extern __shared__ __align__(16) unsigned char sd_smem[];
  R* T = reinterpret_cast<R*>(sd_smem);  // T_1, T_2, T_3 of the row
  const int n = m.n, x = threadIdx.x, y = blockIdx.x;
  const int z0 = blockIdx.y * zc, z1 = min(z0 + zc, n);
  uint32_t row[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) row[j] = uint32_t(wrap(y + j - 3, n)) * uint32_t(n) + uint32_t(x);
  const int xm1 = wrap(x - 1, n), xp1 = wrap(x + 1, n), xm2 = wrap(x - 2, n), xp2 = wrap(x + 2, n);
  const int xm3 = wrap(x - 3, n), xp3 = wrap(x + 3, n);
  R acc[7][4];
#pragma unroll
  for (int q = 0; q < 7; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[q][i] = R(0);
  R v[7];
  {
    const R* pl = in + size_t(wrap(z0 - 3, n)) * m.n2;
#pragma unroll
    for (int j = 0; j < 7; ++j) v[j] = __ldg(pl + row[j]);
  }
  // input planes z0-3 .. z1+2, seven per round so that the ring slots are compile-time
  for (int p = z0 - 3; p - 3 < z1; p += 7) {
    smooth_plane<R, MAXR2, 0>(in, out, m, tp, row, p + 0, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
    smooth_plane<R, MAXR2, 1>(in, out, m, tp, row, p + 1, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
    smooth_plane<R, MAXR2, 2>(in, out, m, tp, row, p + 2, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
    smooth_plane<R, MAXR2, 3>(in, out, m, tp, row, p + 3, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
    smooth_plane<R, MAXR2, 4>(in, out, m, tp, row, p + 4, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
    smooth_plane<R, MAXR2, 5>(in, out, m, tp, row, p + 5, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
    smooth_plane<R, MAXR2, 6>(in, out, m, tp, row, p + 6, z0, z1, acc, v, T, x, xm1, xp1, xm2, xp2, xm3, xp3);
  }
}

// ---------------------------------------------------------------- quantum-pressure stencil
// Q~_n = qcoef * sum_d [(s_{n+e_d} - s_n) + (s_{n-e_d} - s_n)] / s_n with
// s = sqrt(max(rho, floor)) and neighbours at +-step (Eq. quantumpressure with
// the seven-point Laplacian; comoving 1/a^2 applied by the kick weights).
// Also accumulates the K_rho sum of Eq. (diskpoten): compact -> sum_d
// (s_{n+e_d} - s_n)^2, wide -> (1/4) sum_d (s_{n+2e_d}... written here as
// (s_{n+step e_d} - s_{n-step e_d})^2 / 4 with step = 1 for the printed form.
template <typename R>
__device__ __forceinline__ R sfloor(R rho, R fl) {
  return r_sqrt(rho > fl ? rho : fl);
}

// Extended-precision evaluation of Q~ at one near-empty node: the seven
// square roots in float-float, the Laplacian as (sum of the six neighbours)
// - 6 s_0 in float-float, so that the cancellation between neighbours of
// nearly equal density costs no digits, and the ratio to s_0 to fp32
// rounding.
static __device__ __forceinline__ float q_ext(float r0, float rxp, float rxm, float ryp, float rym, float rzp, float rzm,
                                           float fl, float qcoef) {
  const ff t0 = ff_sqrt(fmaxf(r0, fl));
  const ff sx = ff_add(ff_sqrt(fmaxf(rxp, fl)), ff_sqrt(fmaxf(rxm, fl)));
  const ff sy = ff_add(ff_sqrt(fmaxf(ryp, fl)), ff_sqrt(fmaxf(rym, fl)));
  const ff sz = ff_add(ff_sqrt(fmaxf(rzp, fl)), ff_sqrt(fmaxf(rzm, fl)));
  const ff l = ff_sub(ff_add(ff_add(sx, sy), sz), ff_mul_f(t0, 6.0f));
  return ff_quot(l, t0) * qcoef;
}

// Which fp32 nodes are redone by q_ext.  A near-empty node (s_0 < slim) whose
// fp32 Q~ may miss by more than ~2e-6: each s is within 2^-22 of sqrt(rho)
// and the sums round at 2^-24, so the fp32 Laplacian is within ~2^-21 mag of
// the exact one, mag = sum of the six neighbours' s + 6 s_0 (the absolute
// terms of the Laplacian); its relative error is thus at
// most 2^-21 mag / |lap|, and nodes with mag > ST_KAPPA |lap| are redone
// (ST_KAPPA = 4: at most 1.9e-6 elsewhere).  Seven equal values give lap = 0
// exactly in both evaluations and are kept.  Explicitly rounded operations,
// so that every kernel takes the same decision on the same values.
constexpr float ST_KAPPA = 4.0f;
__device__ __forceinline__ bool q_needs_ext(float s0, float sxp, float sxm, float syp, float sym, float szp, float szm,
                                            float lap, float slim) {
  if (!(s0 < slim)) return false;
  if ((sxp == s0) & (sxm == s0) & (syp == s0) & (sym == s0) & (szp == s0) & (szm == s0)) return false;
  const float mag = __fadd_rn(__fadd_rn(__fadd_rn(sxp, sxm), __fadd_rn(syp, sym)),
                              __fmaf_rn(6.0f, s0, __fadd_rn(szp, szm)));
  return mag > __fmul_rn(ST_KAPPA, fabsf(lap));
}

template <typename R>
__global__ void __launch_bounds__(MESH_THREADS) k_stencil(const R* __restrict__ rho, Mesh m, StencilParams sp,
                                                          R* __restrict__ q, double* part) {
  const int n = m.n;
  R ksum = R(0);
  const R fl = R(sp.rho_floor);
  const R qc = R(sp.qcoef);
  const float slim = sp.rho_fp64 > 0 ? float(sqrt(sp.rho_fp64)) : 0.0f;  // fp32 only
  for (uint32_t node = blockIdx.x * blockDim.x + threadIdx.x; node < m.n3; node += gridDim.x * blockDim.x) {
    int x, y, z;
    split_cell(node, m, x, y, z);
    const int st = sp.step;
    const uint32_t zn = uint32_t(z) * m.n2, yn = uint32_t(y) * uint32_t(n);
    const uint32_t xp = wrap(x + st, n), xm = wrap(x - st, n);
    const uint32_t yp = uint32_t(wrap(y + st, n)) * n, ym = uint32_t(wrap(y - st, n)) * n;
    const uint32_t zp = uint32_t(wrap(z + st, n)) * m.n2, zm = uint32_t(wrap(z - st, n)) * m.n2;
    const R r0 = __ldg(rho + node);
    const R rxp = __ldg(rho + zn + yn + xp), rxm = __ldg(rho + zn + yn + xm);
    const R ryp = __ldg(rho + zn + yp + x), rym = __ldg(rho + zn + ym + x);
    const R rzp = __ldg(rho + zp + yn + x), rzm = __ldg(rho + zm + yn + x);
    R s0 = sfloor(r0, fl);
    R sxp = sfloor(rxp, fl), sxm = sfloor(rxm, fl);
    R syp = sfloor(ryp, fl), sym = sfloor(rym, fl);
    R szp = sfloor(rzp, fl), szm = sfloor(rzm, fl);
    R lap = ((sxp - s0) + (sxm - s0)) + ((syp - s0) + (sym - s0)) + ((szp - s0) + (szm - s0));
    R qv = qc * lap / s0;
    if (sizeof(R) == 4 && q_needs_ext(float(s0), float(sxp), float(sxm), float(syp), float(sym), float(szp),
                                      float(szm), float(lap), slim))
      qv = R(q_ext(float(r0), float(rxp), float(rxm), float(ryp), float(rym), float(rzp), float(rzm),
                   float(sp.rho_floor), float(sp.qcoef)));
    q[node] = qv;
    if (st == 1) {
      R a = sxp - s0, b = syp - s0, c = szp - s0;
      ksum += a * a + b * b + c * c;
    } else {
      // printed form of Eq. (diskpoten): central differences over +-dx
      const R cxp = sfloor(__ldg(rho + zn + yn + wrap(x + 1, n)), fl);
      const R cxm = sfloor(__ldg(rho + zn + yn + wrap(x - 1, n)), fl);
      const R cyp = sfloor(__ldg(rho + zn + uint32_t(wrap(y + 1, n)) * n + x), fl);
      const R cym = sfloor(__ldg(rho + zn + uint32_t(wrap(y - 1, n)) * n + x), fl);
      const R czp = sfloor(__ldg(rho + uint32_t(wrap(z + 1, n)) * m.n2 + yn + x), fl);
      const R czm = sfloor(__ldg(rho + uint32_t(wrap(z - 1, n)) * m.n2 + yn + x), fl);
      R a = cxp - cxm, b = cyp - cym, c = czp - czm;
      ksum += R(0.25) * (a * a + b * b + c * c);
    }
  }
  R acc[1] = {ksum};
  block_sum_store<1>(acc, part, gridDim.x);
}

// fp32 compact-Laplacian stencil, register columns.  A block of 32 x ST_TY
// threads (one warp per y-row of a 32-wide x strip) owns ST_TY rows and one
// of ST_ZCH chunks of z.  Each thread marches its (x, y) column along z with
// s = sqrt(max(rho, floor)) at z-1, z, z+1 in registers (the density of
// plane z+2 is fetched while plane z is computed); x-neighbours come from
// warp shuffles (the two edge lanes load theirs), y-neighbours from a
// shared-memory copy of plane z (two warps also load the halo rows).  Each
// density is read about once and its square root taken about once, at ~35
// instructions per node.  Near-empty nodes whose fp32 value is
// ill-conditioned (q_needs_ext) are collected in the block's region of `list`
// (shared-memory counter) and recomputed in float-float by the same block
// after its sweep.
#ifndef PM_ST_TY
#define PM_ST_TY 16
#endif
#ifndef PM_ST_ZCH
#define PM_ST_ZCH 8
#endif
constexpr int ST_X = 32, ST_TY = PM_ST_TY, ST_Y = ST_TY, ST_ZCH = PM_ST_ZCH;

__device__ __forceinline__ float s_of(float r, float fl) {
  const float x = fmaxf(r, fl);
  return x * rsqrt_ftz(x);
}

// the seven densities of a node: centre, x+, x-, y+, y-, z+, z-
__device__ __forceinline__ void load7(const float* __restrict__ rho, uint32_t node, const Mesh& m, float (&r)[7]) {
  int x, y, z;
  split_cell(node, m, x, y, z);
  const int n = m.n;
  const uint32_t zn = uint32_t(z) * m.n2, yn = uint32_t(y) * uint32_t(n);
  r[0] = __ldg(rho + node);
  r[1] = __ldg(rho + zn + yn + wrap(x + 1, n));
  r[2] = __ldg(rho + zn + yn + wrap(x - 1, n));
  r[3] = __ldg(rho + zn + uint32_t(wrap(y + 1, n)) * n + x);
  r[4] = __ldg(rho + zn + uint32_t(wrap(y - 1, n)) * n + x);
  r[5] = __ldg(rho + uint32_t(wrap(z + 1, n)) * m.n2 + yn + x);
  r[6] = __ldg(rho + uint32_t(wrap(z - 1, n)) * m.n2 + yn + x);
}

__device__ __forceinline__ float q_ext_at(const float* __restrict__ rho, uint32_t node, const Mesh& m, float fl,
                                          float qc) {
  float r[7];
  load7(rho, node, m, r);
  return q_ext(r[0], r[1], r[2], r[3], r[4], r[5], r[6], fl, qc);
}

// the float-float pass over a block's list of near-empty nodes, two nodes per
// thread at a time (their loads and dependent chains overlap)
__device__ __forceinline__ void q_ext_list(const float* __restrict__ rho, const uint32_t* list, uint32_t cnt,
                                           const Mesh& m, float fl, float qc, float* __restrict__ q, int tid,
                                           int nthreads) {
  uint32_t i = tid;
  for (; i + nthreads < cnt; i += 2 * nthreads) {
    const uint32_t a = list[i], b = list[i + nthreads];
    float ra[7], rb[7];
    load7(rho, a, m, ra);
    load7(rho, b, m, rb);
    const float qa = q_ext(ra[0], ra[1], ra[2], ra[3], ra[4], ra[5], ra[6], fl, qc);
    const float qb = q_ext(rb[0], rb[1], rb[2], rb[3], rb[4], rb[5], rb[6], fl, qc);
    q[a] = qa;
    q[b] = qb;
  }
  if (i < cnt) {
    const uint32_t a = list[i];
    q[a] = q_ext_at(rho, a, m, fl, qc);
  }
}

static __global__ void __launch_bounds__(ST_X * ST_TY) k_stencil_tiled(const float* __restrict__ rho, Mesh m,
                                                                        float fl, float qc, float slim, int zlen,
                                                                        float* __restrict__ q, uint32_t* list,
                                                                        uint32_t* list_count, double* part,
                                                                        int diag) {
  __shared__ float S[ST_TY + 2][ST_X];  // s of plane z, rows y0-1 .. y0+ST_TY
  __shared__ uint32_t s_cnt;
  const int n = m.n;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * ST_X + tx;
  const int x0 = blockIdx.x * ST_X, y0 = blockIdx.y * ST_Y;
  const int z0 = blockIdx.z * zlen, z1 = min(z0 + zlen, n);
  const uint32_t blin = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  uint32_t* my_list = list + size_t(blin) * (ST_X * ST_Y) * zlen;
  if (tid == 0) s_cnt = 0;
  const int x = x0 + tx, y = y0 + ty;
  const bool live = x < n && y < n;
  const int xc = min(x, n - 1), yc = min(y, n - 1);  // clamped: dead lanes read valid memory
  const uint32_t col = uint32_t(yc) * n + uint32_t(xc);
  // x-neighbours outside the warp's contiguous strip (edge lanes, or the periodic wrap)
  const bool own_xm = tx == 0, own_xp = (tx == ST_X - 1) || (x + 1 >= n);
  const uint32_t col_xm = uint32_t(yc) * n + uint32_t(wrap(xc - 1, n));
  const uint32_t col_xp = uint32_t(yc) * n + uint32_t(wrap(xc + 1, n));
  // warps 0 and 1 also carry the halo rows y0-1 and y0+ST_TY of the strip
  const bool halo = ty < 2;
  const int hy = ty == 0 ? wrap(y0 - 1, n) : wrap(min(y0 + ST_TY, n) % n, n);
  const int hslot = ty == 0 ? 0 : (min(y0 + ST_TY, n) - y0 + 1);
  const uint32_t col_h = uint32_t(hy) * n + uint32_t(xc);
  auto plane = [&](int z) { return rho + uint32_t(wrap(z, n)) * m.n2; };
  // column registers
  float sm = s_of(__ldg(plane(z0 - 1) + col), fl);
  float sc = s_of(__ldg(plane(z0) + col), fl);
  float sp = s_of(__ldg(plane(z0 + 1) + col), fl);
  float pre = __ldg(plane(z0 + 2) + col);
  float exm = own_xm ? __ldg(plane(z0) + col_xm) : 0.0f, exp_ = own_xp ? __ldg(plane(z0) + col_xp) : 0.0f;
  float eh = halo ? __ldg(plane(z0) + col_h) : 0.0f;
  ff ksum = {0.0f, 0.0f};
  for (int z = z0; z < z1; ++z) {
    // plane z into shared memory (own row and the halo rows; rows past the mesh
    // do not write, their slot may be the halo slot)
    if (y < n) S[ty + 1][tx] = sc;
    if (halo) S[hslot][tx] = s_of(eh, fl);
    const float sxm_e = s_of(exm, fl), sxp_e = s_of(exp_, fl);
    // fetch for the next plane while this one is computed
    const bool more = z + 1 < z1;
    float exm_n = 0.0f, exp_n = 0.0f, eh_n = 0.0f, pre_n = 0.0f;
    if (more) {
      const float* pl = plane(z + 1);
      if (own_xm) exm_n = __ldg(pl + col_xm);
      if (own_xp) exp_n = __ldg(pl + col_xp);
      if (halo) eh_n = __ldg(pl + col_h);
      pre_n = __ldg(plane(z + 3) + col);
    }
    __syncthreads();
    float sxm = __shfl_up_sync(0xffffffffu, sc, 1), sxp = __shfl_down_sync(0xffffffffu, sc, 1);
    if (own_xm) sxm = sxm_e;
    if (own_xp) sxp = sxp_e;
    const float sym = S[ty][tx], syp = S[ty + 2][tx];
    if (live) {
      const float dxp = sxp - sc, dyp = syp - sc, dzp = sp - sc;
      const float lap = (dxp + (sxm - sc)) + (dyp + (sym - sc)) + (dzp + (sm - sc));
      const uint32_t node = uint32_t(z) * m.n2 + col;
      q[node] = (qc * lap) * rcp_ftz(sc);
      if (diag) ff_accumulate(ksum, krho_term(dxp, dyp, dzp));
      // near-empty and ill-conditioned: redone in float-float
      if (q_needs_ext(sc, sxp, sxm, syp, sym, sp, sm, lap, slim)) my_list[atomicAdd(&s_cnt, 1u)] = node;
    }
    __syncthreads();  // S is rewritten next
    sm = sc;
    sc = sp;
    sp = s_of(pre, fl);
    pre = pre_n;
    exm = exm_n;
    exp_ = exp_n;
    eh = eh_n;
  }
  // near-empty nodes of this block, recomputed in float-float
  const uint32_t cnt = s_cnt;
  q_ext_list(rho, my_list, cnt, m, fl, qc, q, tid, ST_X * ST_TY);
  if (tid == 0) list_count[blin] = cnt;
  if (diag) {
    const ff acc[1] = {fast_two_sum(ksum.hi, ksum.lo)};
    block_sum_store_ff<1>(acc, part, gridDim.x * gridDim.y * gridDim.z, int(blin));
  }
}

// fp32 compact stencil fed by bulk copies.  A block owns `ty` whole mesh rows
// (all of x, so the periodic x-neighbours are in the tile) of `zlen`
// consecutive planes.  Thread 0 streams the density of each plane tile, with
// its two halo rows, into a ring of `stages` shared-memory slots (three bulk
// copies per plane, completed on the slot's mbarrier), so that stages-3
// planes are in flight while the threads work.  When a plane arrives its
// s = sqrt(max(rho, floor)) is taken once into a ring of three s planes; Q~ of
// plane z then reads s of z-1, z, z+1 from shared memory in float4 groups
// along x.  Ill-conditioned near-empty nodes (q_needs_ext) go to a per-plane
// list and are redone in float-float from the densities still in the ring.  Per node the arithmetic
// is that of k_stencil_tiled, so both kernels give the same bits.
constexpr int SB_THREADS = 256;
constexpr uint32_t SB_WAIT_LIMIT = 1u << 20;

inline size_t stencil_bulk_smem(int n, int ty, int stages) {
  const size_t slot = size_t(ty + 2) * n * sizeof(float);
  const size_t list = (size_t(ty) * n * sizeof(uint16_t) + 15) & ~size_t(15);
  return 16 * ((stages * 8 + 15) / 16) + (size_t(stages) + 3) * slot + list;
}

constexpr size_t SB_SMEM_MAX = 226 * 1024;  // dynamic shared memory per block, below the 227 KB opt-in

inline size_t stencil_tile_smem(int n, int ty, int tz) { return 16 + size_t(ty + 2) * (tz + 2) * n * sizeof(float); }

// one-shot tiles: ty rows x tz planes (tz <= n; the last tile of a column may be shorter)
inline bool stencil_tile_shape_ok(int n, int ty, int tz) {
  if (n % 4 || !(ty == 1 || ty == 2 || ty == 4 || ty == 8) || n % ty) return false;
  if (tz < 2 || tz > 16 || tz > n) return false;
  return stencil_tile_smem(n, ty, tz) <= SB_SMEM_MAX;
}

// the fp32 compact stencil runs as one-shot tiles with these parameters
inline bool stencil_tile_path(int n, const StencilParams& sp, bool fp32) {
  return fp32 && sp.step == 1 && sp.ty > 0 && sp.stages == 0 && stencil_tile_shape_ok(n, sp.ty, sp.zlen);
}

inline bool stencil_bulk_shape_ok(int n, int ty, int zlen, int stages) {
  if (n % 4 || !(ty == 1 || ty == 2 || ty == 4 || ty == 8) || n % ty) return false;
  if (zlen < 4 || zlen > n || stages < 4 || stages > 8) return false;
  return stencil_bulk_smem(n, ty, stages) <= SB_SMEM_MAX;
}

static __global__ void __launch_bounds__(SB_THREADS) k_stencil_bulk(const float* __restrict__ rho, Mesh m, float fl,
                                                                    float qc, float slim, int ty, int zlen,
                                                                    int stages, float* __restrict__ q,
                                                                    double* part, uint32_t* err, int diag) {
  extern __shared__ __align__(16) unsigned char sb_smem[];
  __shared__ uint32_t s_cnt;
  __shared__ int s_abort;
  const int n = m.n, lg = m.log2n;
  const int slot = (ty + 2) * n;  // floats per plane tile
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb_smem);
  float* ring = reinterpret_cast<float*>(sb_smem + 16 * ((stages * 8 + 15) / 16));
  float* sring = ring + size_t(stages) * slot;
  uint16_t* list = reinterpret_cast<uint16_t*>(sring + 3 * size_t(slot));
  const int tid = threadIdx.x;
  const int y0 = blockIdx.x * ty;
  const int z0 = blockIdx.y * zlen, z1 = min(z0 + zlen, n);
  const int nplanes = z1 - z0 + 2;  // planes z0-1 .. z1
  const uint32_t row_bytes = uint32_t(n) * 4u;
  if (tid == 0) {
    for (int k = 0; k < stages; ++k) mbar_init(bar + k, 1);
    mbar_init_fence();
    s_abort = 0;
  }
  __syncthreads();
  // plane z0-1+j into slot j % stages (thread 0 only)
  auto issue = [&](int j) {
    float* dst = ring + size_t(j % stages) * slot;
    uint64_t* b = bar + (j % stages);
    const float* pl = rho + size_t(wrap(z0 - 1 + j, n)) * m.n2;
    mbar_arrive_expect(b, uint32_t(ty + 2) * row_bytes);
    bulk_load(dst, pl + size_t(wrap(y0 - 1, n)) * n, row_bytes, b);
    bulk_load(dst + n, pl + size_t(y0) * n, uint32_t(ty) * row_bytes, b);
    bulk_load(dst + size_t(ty + 1) * n, pl + size_t(wrap(y0 + ty, n)) * n, row_bytes, b);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < stages && issued < nplanes; ++issued) issue(issued);
  // waits for plane j and takes its s into sring[j % 3]; false after a timeout
  auto take_s = [&](int j) {
    // warp 0 polls the slot's mbarrier, the block barrier publishes the plane
    if (tid < 32 && !mbar_wait(bar + (j % stages), uint32_t(j / stages) & 1u, SB_WAIT_LIMIT)) {
      if (tid == 0) atomicOr(err, ERR_TIMEOUT);
      s_abort = 1;
    }
    __syncthreads();
    if (s_abort) return;
    const float4* src = reinterpret_cast<const float4*>(ring + size_t(j % stages) * slot);
    float4* dst = reinterpret_cast<float4*>(sring + size_t(j % 3) * slot);
    for (int g = tid; g < slot / 4; g += SB_THREADS) {
      const float4 r = src[g];
      dst[g] = make_float4(s_of(r.x, fl), s_of(r.y, fl), s_of(r.z, fl), s_of(r.w, fl));
    }
  };
  take_s(0);
  take_s(1);
  ff ksum = {0.0f, 0.0f};  // K_rho terms of this thread
  const int groups = ty * n / 4;
  for (int z = z0; z < z1; ++z) {
    const int jc = z - z0 + 1;  // plane z in ring numbering
    take_s(jc + 1);
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    if (s_abort) break;
    const float* Sm = sring + size_t((jc + 2) % 3) * slot;
    const float* Sc = sring + size_t(jc % 3) * slot;
    const float* Sp = sring + size_t((jc + 1) % 3) * slot;
    for (int g = tid; g < groups; g += SB_THREADS) {
      const int e = g * 4;
      const int r = 1 + (lg >= 0 ? e >> lg : e / n), x = e - (r - 1) * n;
      const int o = r * n + x;
      const float4 c4 = *reinterpret_cast<const float4*>(Sc + o);
      const float4 ym4 = *reinterpret_cast<const float4*>(Sc + o - n);
      const float4 yp4 = *reinterpret_cast<const float4*>(Sc + o + n);
      const float4 zm4 = *reinterpret_cast<const float4*>(Sm + o);
      const float4 zp4 = *reinterpret_cast<const float4*>(Sp + o);
      const float xl = Sc[r * n + (x == 0 ? n - 1 : x - 1)], xr = Sc[r * n + (x + 4 == n ? 0 : x + 4)];
      const float sc[4] = {c4.x, c4.y, c4.z, c4.w}, sym[4] = {ym4.x, ym4.y, ym4.z, ym4.w};
      const float syp[4] = {yp4.x, yp4.y, yp4.z, yp4.w}, szm[4] = {zm4.x, zm4.y, zm4.z, zm4.w};
      const float szp[4] = {zp4.x, zp4.y, zp4.z, zp4.w};
      float qv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float sxm = k ? sc[k - 1] : xl, sxp = k < 3 ? sc[k + 1] : xr;
        const float dxp = sxp - sc[k], dyp = syp[k] - sc[k], dzp = szp[k] - sc[k];
        const float lap = (dxp + (sxm - sc[k])) + (dyp + (sym[k] - sc[k])) + (dzp + (szm[k] - sc[k]));
        qv[k] = (qc * lap) * rcp_ftz(sc[k]);
        if (diag) ff_accumulate(ksum, krho_term(dxp, dyp, dzp));
        if (q_needs_ext(sc[k], sxp, sxm, syp[k], sym[k], szp[k], szm[k], lap, slim))
          list[atomicAdd(&s_cnt, 1u)] = uint16_t(e + k);
      }
      *reinterpret_cast<float4*>(q + size_t(z) * m.n2 + size_t(y0) * n + e) = make_float4(qv[0], qv[1], qv[2], qv[3]);
    }
    __syncthreads();
    // near-empty nodes of this plane, from the densities of planes z-1, z, z+1
    const uint32_t cnt = s_cnt;
    if (cnt) {
      const float* Rm = ring + size_t((jc - 1) % stages) * slot;
      const float* Rc = ring + size_t(jc % stages) * slot;
      const float* Rp = ring + size_t((jc + 1) % stages) * slot;
      for (uint32_t i = tid; i < cnt; i += SB_THREADS) {
        const int e = list[i];
        const int r = 1 + (lg >= 0 ? e >> lg : e / n), x = e - (r - 1) * n;
        const int o = r * n + x;
        const float v = q_ext(Rc[o], Rc[r * n + (x + 1 == n ? 0 : x + 1)], Rc[r * n + (x == 0 ? n - 1 : x - 1)],
                              Rc[o + n], Rc[o - n], Rp[o], Rm[o], fl, qc);
        q[size_t(z) * m.n2 + size_t(y0) * n + e] = v;
      }
    }
    __syncthreads();  // the slot of plane z-1 and the list are free again
    if (tid == 0 && issued < nplanes) issue(issued++);
  }
  // after a timeout: let the copies still in flight land before the block exits
  if (s_abort && tid == 0)
    for (int j = (issued > stages ? issued - stages : 0); j < issued; ++j)
      mbar_wait(bar + (j % stages), uint32_t(j / stages) & 1u, SB_WAIT_LIMIT);
  if (diag) {
    const ff acc[1] = {fast_two_sum(ksum.hi, ksum.lo)};
    block_sum_store_ff<1>(acc, part, gridDim.x * gridDim.y, int(blockIdx.y * gridDim.x + blockIdx.x));
  }
}

// fp32 compact stencil, one tile per block with no sweep: a block owns `ty`
// whole rows of `tz` planes and requests its whole input tile at once (one
// mbarrier): the ty+2 rows (with the y halo) of each of its planes, and the
// ty interior rows of the two halo planes; the four corner rows of the
// (ty+2) x (tz+2) frame are no neighbour of any node in a seven-point
// stencil, so they are neither copied nor used.  The block takes s in place,
// then evaluates Q~ of the interior from shared memory.  The input of several
// resident blocks is in flight together and nothing waits on a plane-by-plane
// chain.  Ill-conditioned near-empty nodes (q_needs_ext) go to the block's
// region of a global list and are redone in float-float (densities reread
// through L2).
// Per node the arithmetic is that of k_stencil_tiled (same bits).
template <bool PACKED>
__global__ void __launch_bounds__(SB_THREADS) k_stencil_tile(const float* __restrict__ rho, Mesh m, float fl,
                                                                    float qc, float slim, int ty, int tz,
                                                                    float* __restrict__ q, uint32_t* list,
                                                                    double* part, uint32_t* err, int diag,
                                                                    const double* qcp, size_t ms) {
  if constexpr (PACKED) {  // member blockIdx.z of a packed group (coefficient from device memory, as in k_green)
    const size_t o = size_t(blockIdx.z) * ms;
    rho = moff(rho, o), q = moff(q, o), list = moff(list, o), part = moff(part, o), err = moff(err, o);
    qc = float(*moff(qcp, o));
  }
  extern __shared__ __align__(16) unsigned char st_smem[];
  __shared__ uint32_t s_cnt;
  __shared__ int s_ok;
  const int n = m.n, lg = m.log2n, lty = __ffs(ty) - 1;  // ty is a power of two
  const int row = n, plane = (ty + 2) * n;  // floats
  uint64_t* bar = reinterpret_cast<uint64_t*>(st_smem);
  float* S = reinterpret_cast<float*>(st_smem + 16);
  const int tid = threadIdx.x;
  const int y0 = blockIdx.x * ty;
  const int z0 = blockIdx.y * tz, nz = min(tz, n - z0);  // planes of this tile
  const uint32_t blin = blockIdx.y * gridDim.x + blockIdx.x;
  uint32_t* my_list = list + size_t(blin) * size_t(ty) * tz * n;
  const uint32_t row_bytes = uint32_t(n) * 4u;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
    s_cnt = 0;
    s_ok = 1;
    mbar_arrive_expect(bar, uint32_t(nz * (ty + 2) + 2 * ty) * row_bytes);
    for (int j = 0; j < nz + 2; ++j) {
      const float* pl = rho + size_t(wrap(z0 - 1 + j, n)) * m.n2;
      float* dst = S + size_t(j) * plane;
      bulk_load(dst + row, pl + size_t(y0) * n, uint32_t(ty) * row_bytes, bar);
      if (j > 0 && j <= nz) {  // the y halo rows of the tile's own planes
        bulk_load(dst, pl + size_t(wrap(y0 - 1, n)) * n, row_bytes, bar);
        bulk_load(dst + size_t(ty + 1) * row, pl + size_t(wrap(y0 + ty, n)) * n, row_bytes, bar);
      }
    }
  }
  __syncthreads();
  // warp 0 polls the mbarrier (its acquire, then the block barrier, publish
  // the copied tile to every thread); the other warps sleep at the barrier
  if (tid < 32 && !mbar_wait(bar, 0, SB_WAIT_LIMIT)) {
    if (tid == 0) atomicOr(err, ERR_TIMEOUT);
    s_ok = 0;
  }
  __syncthreads();
  if (!s_ok) {  // the copies may still land: wait for them (bounded) before the block exits
    if (tid == 0) mbar_wait(bar, 0, SB_WAIT_LIMIT);
    return;
  }
  // s in place: all rows of planes 1..nz (one contiguous span), then the
  // interior rows of halo planes 0 and nz+1
  float4* S4 = reinterpret_cast<float4*>(S);
  const int mid4 = nz * plane / 4, halo4 = ty * row / 4;
  for (int g = tid; g < mid4 + 2 * halo4; g += SB_THREADS) {
    const int h = g - mid4;
    float4* at = h < 0 ? S4 + plane / 4 + g
                       : (h < halo4 ? S4 + row / 4 + h : S4 + (nz + 1) * plane / 4 + row / 4 + (h - halo4));
    const float4 r = *at;
    *at = make_float4(s_of(r.x, fl), s_of(r.y, fl), s_of(r.z, fl), s_of(r.w, fl));
  }
  __syncthreads();
  ff ksum = {0.0f, 0.0f};
  const int rows_in = nz * ty;  // interior rows, plane-major
  const int groups = rows_in * n / 4;
  for (int g = tid; g < groups; g += SB_THREADS) {
    const int e = g * 4;                                 // interior element, (plane, row, x)
    const int ri = lg >= 0 ? e >> lg : e / n;           // interior row index
    const int x = e - ri * n;
    const int pz = ri >> lty, r = ri - (pz << lty);      // plane and row inside the tile
    const int o = (pz + 1) * plane + (r + 1) * row + x;
    const float4 c4 = *reinterpret_cast<const float4*>(S + o);
    const float4 ym4 = *reinterpret_cast<const float4*>(S + o - row);
    const float4 yp4 = *reinterpret_cast<const float4*>(S + o + row);
    const float4 zm4 = *reinterpret_cast<const float4*>(S + o - plane);
    const float4 zp4 = *reinterpret_cast<const float4*>(S + o + plane);
    const int ob = o - x;
    const float xl = S[ob + (x == 0 ? n - 1 : x - 1)], xr = S[ob + (x + 4 == n ? 0 : x + 4)];
    const float sc[4] = {c4.x, c4.y, c4.z, c4.w}, sym[4] = {ym4.x, ym4.y, ym4.z, ym4.w};
    const float syp[4] = {yp4.x, yp4.y, yp4.z, yp4.w}, szm[4] = {zm4.x, zm4.y, zm4.z, zm4.w};
    const float szp[4] = {zp4.x, zp4.y, zp4.z, zp4.w};
    const uint32_t node0 = uint32_t(z0 + pz) * m.n2 + uint32_t(y0 + r) * uint32_t(n) + uint32_t(x);
    float qv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float sxm = k ? sc[k - 1] : xl, sxp = k < 3 ? sc[k + 1] : xr;
      const float dxp = sxp - sc[k], dyp = syp[k] - sc[k], dzp = szp[k] - sc[k];
      const float lap = (dxp + (sxm - sc[k])) + (dyp + (sym[k] - sc[k])) + (dzp + (szm[k] - sc[k]));
      qv[k] = (qc * lap) * rcp_ftz(sc[k]);
      if (diag) ff_accumulate(ksum, krho_term(dxp, dyp, dzp));
      if (q_needs_ext(sc[k], sxp, sxm, syp[k], sym[k], szp[k], szm[k], lap, slim))
        my_list[atomicAdd(&s_cnt, 1u)] = node0 + k;
    }
    *reinterpret_cast<float4*>(q + node0) = make_float4(qv[0], qv[1], qv[2], qv[3]);
  }
  __syncthreads();
  q_ext_list(rho, my_list, s_cnt, m, fl, qc, q, tid, SB_THREADS);
  if (diag) {
    const ff acc[1] = {fast_two_sum(ksum.hi, ksum.lo)};
    block_sum_store_ff<1>(acc, part, gridDim.x * gridDim.y, int(blin));
  }
}

// ---------------------------------------------------------------- interpolate + kick + drift
// Gradient of a mesh potential at the particle, in one of two forms:
//   central : sum_c w_c (f[c+e] - f[c-e]) / 2dx over the 8 cloud-in-cell corners c
//   kernel  : grad_q sum_c f_c w_c  (Eq. equationofmotion; 8 corner values)
struct Stencil {
  uint32_t xi[4];  // x - 1, x, x + 1, x + 2 (wrapped)
  uint32_t yi[4];  // rows times N
  uint32_t zi[4];  // planes times N^2
};

template <typename R>
__device__ __forceinline__ void grad_kernel(const R* __restrict__ f, const Stencil& s, const R (&wx)[2],
                                            const R (&wy)[2], const R (&wz)[2], R inv_dx, R (&g)[3]) {
  R c[2][2][2];
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) c[dz][dy][dx] = __ldg(f + (s.zi[dz + 1] + s.yi[dy + 1] + s.xi[dx + 1]));
  R gx = 0, gy = 0, gz = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      gx += wz[a] * wy[b] * (c[a][b][1] - c[a][b][0]);
      gy += wz[a] * wx[b] * (c[a][1][b] - c[a][0][b]);
      gz += wy[a] * wx[b] * (c[1][a][b] - c[0][a][b]);
    }
  g[0] = gx * inv_dx;
  g[1] = gy * inv_dx;
  g[2] = gz * inv_dx;
}

template <typename R>
__device__ __forceinline__ void grad_central(const R* __restrict__ f, const Stencil& s, const R (&wx)[2],
                                             const R (&wy)[2], const R (&wz)[2], R inv_dx, R (&g)[3]) {
  // the 32 distinct nodes: the inner 2x2x2 cube and its two-sided extensions
  // along each axis, each loaded once
  R c[2][2][2], ex[2][2][2], ey[2][2][2], ez[2][2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
      for (int d = 0; d < 2; ++d) c[a][b][d] = __ldg(f + (s.zi[a + 1] + s.yi[b + 1] + s.xi[d + 1]));
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        ex[a][b][e] = __ldg(f + (s.zi[a + 1] + s.yi[b + 1] + s.xi[3 * e]));
        ey[a][b][e] = __ldg(f + (s.zi[a + 1] + s.yi[3 * e] + s.xi[b + 1]));
        ez[a][b][e] = __ldg(f + (s.zi[3 * e] + s.yi[a + 1] + s.xi[b + 1]));
      }
    }
  R gx = 0, gy = 0, gz = 0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const R u0 = ex[dz][dy][0], u1 = c[dz][dy][0], u2 = c[dz][dy][1], u3 = ex[dz][dy][1];
      gx += wz[dz] * wy[dy] * (wx[0] * (u2 - u0) + wx[1] * (u3 - u1));
    }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const R u0 = ey[dz][dx][0], u1 = c[dz][0][dx], u2 = c[dz][1][dx], u3 = ey[dz][dx][1];
      gy += wz[dz] * wx[dx] * (wy[0] * (u2 - u0) + wy[1] * (u3 - u1));
    }
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const R u0 = ez[dy][dx][0], u1 = c[0][dy][dx], u2 = c[1][dy][dx], u3 = ez[dy][dx][1];
      gz += wy[dy] * wx[dx] * (wz[0] * (u2 - u0) + wz[1] * (u3 - u1));
    }
  const R h = R(0.5) * inv_dx;
  g[0] = gx * h;
  g[1] = gy * h;
  g[2] = gz * h;
}

template <typename R>
__device__ __forceinline__ bool finite3(R a, R b, R c) {
  return r_finite(a) && r_finite(b) && r_finite(c);
}

// Moves an offset o (cell units) into [0,1) and returns the integer carry.
template <typename R>
__device__ __forceinline__ int carry(R& o) {
  R fl = r_floor(o);
  fl = fl > R(1 << 29) ? R(1 << 29) : (fl < R(-(1 << 29)) ? R(-(1 << 29)) : fl);
  int c = int(fl);
  o -= fl;
  if (o >= R(1)) {  // o was a tiny negative number: o - floor(o) rounded to 1
    o = R(0);
    c += 1;
  }
  if (o < R(0)) o = R(0);
  return c;
}

// Per-block maxima of NV fp32 values (thread 0 writes part[k*nblocks + bid]).
template <int NV>
__device__ __forceinline__ void block_max_store(const float (&v)[NV], double* part, int nblocks, int bid) {
  __shared__ float shm[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float m[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    m[k] = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m[k] = fmaxf(m[k], __shfl_xor_sync(0xffffffffu, m[k], o));
    if (lane == 0) shm[warp][k] = m[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float r = 0.0f;
      for (int w = 0; w < nw; ++w) r = fmaxf(r, shm[w][k]);
      part[k * nblocks + bid] = double(r);
    }
  }
}

// resident 256-thread blocks per SM the kick's register budget is cut for
#ifndef PM_KICK_MINB
#define PM_KICK_MINB 4
#endif

// The leapfrog weights of a pass in the working precision (converted once
// per thread, so that the loop keeps no doubles live) and its switches.
template <typename R>
struct KickR {
  R cg1, cq1, cg2, cq2, drift, inv_dx;
  bool grav_kernel, q_kernel, quantum, has_drift;
};
template <typename R>
__device__ __forceinline__ KickR<R> kick_r(const KickParams& kp) {
  KickR<R> k;
  k.cg1 = R(kp.cg1), k.cq1 = R(kp.cq1), k.cg2 = R(kp.cg2), k.cq2 = R(kp.cq2), k.drift = R(kp.drift);
  k.inv_dx = R(kp.inv_dx);
  k.grav_kernel = kp.grav_kernel != 0, k.q_kernel = kp.q_kernel != 0, k.quantum = kp.quantum != 0;
  k.has_drift = kp.drift != 0.0;
  return k;
}

// One particle of a kick pass: gradients at the particle, kick, drift, new
// key.  MODE 0: kick (+ drift); 1: kick with the diagnostic sums of p_sync
// (dg); 2: write the accelerations only; 3: leave the state and write
// |p_sync|^2, |grad phi|^2 and |grad Q|^2 to dg (the adaptive step's bound).
// The records are updated in place; with a drift the new key goes to
// keys[i] and a particle that changed cell counts in the mover count of its
// tile of RS_TILE slots (tcount).
// FM: the force form fixed at compile time (KICK_FM_HYBRID_Q: gravity by central differences, the
// quantum force on, by the kernel gradient) or taken from kp at run time (KICK_FM_ANY)
constexpr int KICK_FM_ANY = 0, KICK_FM_HYBRID_Q = 1;
template <typename R, int MODE, int FM = KICK_FM_ANY>
__device__ __forceinline__ void kick_particle(int64_t i, typename VT<R>::v4 ps, typename VT<R>::v4 mo,
                                              typename VT<R>::v4* pos, typename VT<R>::v4* mom,
                                              uint32_t* keys, uint32_t* tcount,
                                              const R* __restrict__ phi, const R* __restrict__ qf, const Mesh& m,
                                              const KickR<R>& kp, double* acc_out, uint32_t* err, R (&dg)[4]) {
  const uint32_t cell = rec_cell(ps);
  int cx, cy, cz;
  split_cell(cell, m, cx, cy, cz);
  const int nn = m.n;
  Stencil s;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s.xi[k] = uint32_t(wrap(cx + k - 1, nn));
    s.yi[k] = uint32_t(wrap(cy + k - 1, nn)) * uint32_t(nn);
    s.zi[k] = uint32_t(wrap(cz + k - 1, nn)) * m.n2;
  }
  const R wx[2] = {R(1) - ps.y, ps.y}, wy[2] = {R(1) - ps.z, ps.z}, wz[2] = {R(1) - ps.w, ps.w};
  const R inv_dx = kp.inv_dx;
  R gp[3], gq[3] = {R(0), R(0), R(0)};
  const bool grav_kernel = FM == KICK_FM_HYBRID_Q ? false : kp.grav_kernel;
  const bool quantum = FM == KICK_FM_HYBRID_Q ? true : kp.quantum;
  const bool q_kernel = FM == KICK_FM_HYBRID_Q ? true : kp.q_kernel;
  if (grav_kernel)
    grad_kernel(phi, s, wx, wy, wz, inv_dx, gp);
  else
    grad_central(phi, s, wx, wy, wz, inv_dx, gp);
  if (quantum) {
    if (q_kernel)
      grad_kernel(qf, s, wx, wy, wz, inv_dx, gq);
    else
      grad_central(qf, s, wx, wy, wz, inv_dx, gq);
  }
  const R cg1 = kp.cg1, cq1 = kp.cq1;
  R d1[3] = {cg1 * gp[0] + cq1 * gq[0], cg1 * gp[1] + cq1 * gq[1], cg1 * gp[2] + cq1 * gq[2]};
  if (MODE == 3) {
    const R px = mo.x - d1[0], py = mo.y - d1[1], pz = mo.z - d1[2];
    dg[0] = px * px + py * py + pz * pz;
    dg[1] = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
    dg[2] = gq[0] * gq[0] + gq[1] * gq[1] + gq[2] * gq[2];
  } else if (MODE == 2) {
    const uint32_t id = rec_id(mo);
    acc_out[3 * size_t(id) + 0] = -double(d1[0]);
    acc_out[3 * size_t(id) + 1] = -double(d1[1]);
    acc_out[3 * size_t(id) + 2] = -double(d1[2]);
  } else {
    R px = mo.x - d1[0], py = mo.y - d1[1], pz = mo.z - d1[2];
    if (MODE == 1) {
      dg[0] = px * px + py * py + pz * pz;
      dg[1] = px;
      dg[2] = py;
      dg[3] = pz;
    }
    const R cg2 = kp.cg2, cq2 = kp.cq2;
    px -= cg2 * gp[0] + cq2 * gq[0];
    py -= cg2 * gp[1] + cq2 * gq[1];
    pz -= cg2 * gp[2] + cq2 * gq[2];
    uint32_t ncell = cell;
    R fx = ps.y, fy = ps.z, fz = ps.w;
    if (kp.has_drift) {
      const R dr = kp.drift;
      fx += px * dr;
      fy += py * dr;
      fz += pz * dr;
      if (!finite3(fx, fy, fz) || !finite3(px, py, pz)) {
        atomicOr(err, ERR_NONFINITE);
        fx = ps.y;
        fy = ps.z;
        fz = ps.w;
      }
      int ccx = carry(fx), ccy = carry(fy), ccz = carry(fz);
      if (ccx | ccy | ccz) {
        int64_t ix = (int64_t(cx) + ccx) % nn, iy = (int64_t(cy) + ccy) % nn, iz = (int64_t(cz) + ccz) % nn;
        ix += ix < 0 ? nn : 0;
        iy += iy < 0 ? nn : 0;
        iz += iz < 0 ? nn : 0;
        ncell = (uint32_t(iz) * uint32_t(nn) + uint32_t(iy)) * uint32_t(nn) + uint32_t(ix);
      }
    } else if (!finite3(px, py, pz)) {
      atomicOr(err, ERR_NONFINITE);
    }
    pos[i] = make_pos(ncell, fx, fy, fz);
    mom[i] = make_mom(px, py, pz, rec_id(mo));
    // the drift marks the particles that changed cell for the incremental re-sort;
    // without a drift the keys (marked or not) stay as they are
    if (kp.has_drift) {
      const bool moved = ncell != cell;
      keys[i] = ncell | (moved ? KEY_MOVER : 0u);
      // one atomic per warp with movers (the warp's 32 consecutive slots lie in one tile): when every
      // particle moves, per-particle atomics on the tile's counter serialise
      const uint32_t active = __activemask();
      const uint32_t movers = __ballot_sync(active, moved);
      if (movers && (threadIdx.x & 31) == uint32_t(__ffs(movers) - 1))
        atomicAdd(tcount + (i >> RS_TILE_SHIFT), uint32_t(__popc(movers)));
    }
  }
}

// One particle per thread, every mode (separate instantiations keep the
// common pass lean); MODE 1 and 3 write one partial per block.
template <typename R, int MODE>
__global__ void __launch_bounds__(KICK_THREADS, PM_KICK_MINB) k_kick(typename VT<R>::v4* pos, typename VT<R>::v4* mom,
                                                       uint32_t* keys, uint32_t* tcount,
                                                       int64_t n, const R* __restrict__ phi,
                                                       const R* __restrict__ qf, Mesh m, KickParams kp_arg,
                                                       const KickParams* __restrict__ kp_tab,
                                                       const uint32_t* __restrict__ step, double* part,
                                                       double* acc_out, uint32_t* err) {
  // weights by value, or (graph replay) from a per-step table indexed by a device step counter
  const KickR<R> kp = kick_r<R>(kp_tab ? kp_tab[*step] : kp_arg);
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  R dg[4] = {R(0), R(0), R(0), R(0)};
  if (i < n) kick_particle<R, MODE>(i, pos[i], mom[i], pos, mom, keys, tcount, phi, qf, m, kp, acc_out, err, dg);
  if (MODE == 1) block_sum_store<4>(dg, part, gridDim.x);
  if (MODE == 3) {
    const float mx[3] = {float(dg[0]), float(dg[1]), float(dg[2])};
    block_max_store<3>(mx, part, gridDim.x, blockIdx.x);
  }
}

// The common pass (MODE 0) as a grid-stride loop over a grid of resident
// blocks: each thread loads the records of its next particle before it works
// on the current one, so that the record loads of one particle overlap the
// mesh gathers of the previous one instead of adding a second dependent
// memory latency per particle.
#ifndef PM_KICK_STREAM_MINB
#define PM_KICK_STREAM_MINB 3  // the prefetched records need registers beyond k_kick's cap
#endif
// PACKED: the members of a packed group, member blockIdx.y (a separate
// instantiation: the member offsets cost the single pass ~20 % when present)
#ifndef PM_KICK_STREAM_HQ_MINB
#define PM_KICK_STREAM_HQ_MINB 4  // the HYBRID single pass fits 64 registers without spills
#endif
template <typename R, bool PACKED, int FM>
__global__ void __launch_bounds__(KICK_THREADS, (FM == KICK_FM_HYBRID_Q && !PACKED) ? PM_KICK_STREAM_HQ_MINB
                                                                                     : PM_KICK_STREAM_MINB) k_kick_stream(
    typename VT<R>::v4* pos, typename VT<R>::v4* mom, uint32_t* keys, uint32_t* tcount, int64_t n, const R* __restrict__ phi,
    const R* __restrict__ qf, Mesh m, KickParams kp_arg, const KickParams* __restrict__ kp_tab,
    const uint32_t* __restrict__ step, uint32_t* err, size_t ms) {
  using V4 = typename VT<R>::v4;
  if constexpr (PACKED) {
    const size_t o = size_t(blockIdx.y) * ms;
    pos = moff(pos, o), mom = moff(mom, o), keys = moff(keys, o), tcount = moff(tcount, o), phi = moff(phi, o);
    qf = moff(qf, o), kp_tab = moff(kp_tab, o), step = moff(step, o), err = moff(err, o);
  }
  const KickR<R> kp = kick_r<R>(kp_tab ? kp_tab[*step] : kp_arg);
  // 32-bit indices (n < 2^31, so i + stride < 2^32) keep the loop's registers down
  const uint32_t stride = gridDim.x * blockDim.x, nn = uint32_t(n);
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  V4 ps = pos[i], mo = mom[i];
  R dg[4];
  for (;;) {
    const uint32_t j = i + stride;
    V4 nps = ps, nmo = mo;
    if (j < nn) {
      nps = pos[j];
      nmo = mom[j];
    }
    kick_particle<R, 0, FM>(i, ps, mo, pos, mom, keys, tcount, phi, qf, m, kp, nullptr, err, dg);
    if (j >= nn) break;
    i = j;
    ps = nps;
    mo = nmo;
  }
}

// ---------------------------------------------------------------- power spectrum
template <typename R>
__global__ void __launch_bounds__(MESH_THREADS) k_power(const typename VT<R>::cplx* __restrict__ spec, Mesh m,
                                                        int nbins, double* part) {
  __shared__ double sb[3 * PK_MAX_BINS];
  for (int b = threadIdx.x; b < 3 * nbins; b += blockDim.x) sb[b] = 0.0;
  __syncthreads();
  const int n = m.n, nh = m.n / 2 + 1;
  const int64_t total = int64_t(n) * n * nh;
  const double inv_n = 1.0 / double(n);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int jx = int(e % nh);
    int64_t r = e / nh;
    int jy = int(r % n);
    int jz = int(r / n);
    int mx = jx, my = jy <= n / 2 ? jy : jy - n, mz = jz <= n / 2 ? jz : jz - n;
    double kk = sqrt(double(mx) * mx + double(my) * my + double(mz) * mz);
    int shell = int(floor(kk + 0.5));
    if (shell < 1 || shell > nbins) continue;
    auto v = spec[e];
    double p2 = double(v.x) * v.x + double(v.y) * v.y;
    // CIC window prod_d sinc^2(k_d dx/2), k_d dx/2 = pi m_d / N
    double win = 1.0;
    const int md[3] = {mx, my, mz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (md[d] != 0) {
        double t = double(md[d]) * inv_n;
        double sc = sinpi(t) / (M_PI * t);
        win *= sc * sc;
      }
    }
    double w = (jx == 0 || jx == n / 2) ? 1.0 : 2.0;
    atomicAdd(&sb[shell - 1], w);
    atomicAdd(&sb[nbins + shell - 1], w * kk);
    atomicAdd(&sb[2 * nbins + shell - 1], w * p2 / (win * win));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 3 * nbins; b += blockDim.x) part[size_t(b) * gridDim.x + blockIdx.x] = sb[b];
}

// ---------------------------------------------------------------- helpers
template <typename R>
__global__ void k_get_particles(const typename VT<R>::v4* __restrict__ pos, const typename VT<R>::v4* __restrict__ mom,
                                int64_t n, Mesh m, double dx, double* x, double* p) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto ps = pos[i];
  auto mo = mom[i];
  int cx, cy, cz;
  split_cell(rec_cell(ps), m, cx, cy, cz);
  size_t id = rec_id(mo);
  x[3 * id + 0] = (double(cx) + double(ps.y)) * dx;
  x[3 * id + 1] = (double(cy) + double(ps.z)) * dx;
  x[3 * id + 2] = (double(cz) + double(ps.w)) * dx;
  p[3 * id + 0] = double(mo.x);
  p[3 * id + 1] = double(mo.y);
  p[3 * id + 2] = double(mo.z);
}

template <typename R>
__global__ void k_get_order(const typename VT<R>::v4* __restrict__ pos, const typename VT<R>::v4* __restrict__ mom,
                            int64_t n, uint32_t* cell, uint32_t* id) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cell[i] = rec_cell(pos[i]);
  id[i] = rec_id(mom[i]);
}

template <typename R>
__global__ void k_to_double(const R* __restrict__ f, int64_t n, double* out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = double(f[i]);
}
template <typename R>
__global__ void k_from_double(const double* __restrict__ f, int64_t n, R* out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = R(f[i]);
}

// ---------------------------------------------------------------- launch wrappers
inline unsigned mesh_grid(uint32_t n3) { return (n3 + MESH_THREADS - 1) / MESH_THREADS; }

template <typename R>
cudaError_t launch_init_particles(const double* x, const double* p, int64_t n, Mesh m, double inv_dx, void* pos,
                                  void* mom, uint32_t* keys, uint32_t* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  using V4 = typename VT<R>::v4;
  k_init_particles<R><<<unsigned((n + 255) / 256), 256, 0, s>>>(x, p, n, m, inv_dx, (V4*)pos, (V4*)mom, keys, err);
  return cudaGetLastError();
}

// deposit tile of TY x TZ rows per warp: the largest of 2 x 4, 2 x 2, 1 x 2, 1 x 1 whose rows fit
// PM_DEPOSIT_WARP_BYTES of shared memory per 4-byte accumulator (4.25 KB: 2 x 2 rows of a 256^3
// fp32 mesh; measured there: 43 us against 53 us for 2 x 4 rows, whose 8.3 KB per warp leave
// too few resident warps)
#ifndef PM_DEPOSIT_WARP_BYTES
#define PM_DEPOSIT_WARP_BYTES 4352
#endif
template <typename R>
inline int deposit_shape(int n, int& ty, int& tz) {
  static const int shapes[4][2] = {{2, 4}, {2, 2}, {1, 2}, {1, 1}};
  const size_t row = size_t(deposit_stride_of<R>(n)) * sizeof(R);
  const size_t most = size_t(PM_DEPOSIT_WARP_BYTES) * sizeof(R) / 4;
  int s = 0;
  while (s < 3 && size_t(shapes[s][0] * shapes[s][1]) * row > most) ++s;
  ty = shapes[s][0], tz = shapes[s][1];
  return s;
}

template <typename R, int TY, int TZ>
cudaError_t launch_deposit_tile(const void* pos, const uint32_t* row_start, int64_t n, Mesh m, double norm, R* rho,
                                cudaStream_t s, int warps, int nm, size_t ms) {
  using V4 = typename VT<R>::v4;
  const size_t smem = size_t(warps) * TY * TZ * deposit_stride_of<R>(m.n) * sizeof(R);
  const unsigned tiles_y = unsigned((m.n + warps * TY - 1) / (warps * TY));
  const unsigned blocks = tiles_y * unsigned((m.n + TZ - 1) / TZ);
  const DivU32 dv = divu32_make(uint32_t(m.n));
  if (nm > 1)
    k_deposit<R, TY, TZ, true><<<dim3(blocks, unsigned(nm)), warps * 32, smem, s>>>(
        (const V4*)pos, row_start, uint32_t(n), m, dv, R(norm), rho, ms);
  else
    k_deposit<R, TY, TZ, false><<<blocks, warps * 32, smem, s>>>((const V4*)pos, row_start, uint32_t(n), m, dv,
                                                                 R(norm), rho, 0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_deposit(const void* pos, const uint32_t* row_start, int64_t n, Mesh m, double norm, R* rho,
                           cudaStream_t s, int warps, int nm, size_t ms) {
  if (warps < 1 || warps > DEP_WARPS) warps = DEP_WARPS;
  int ty = 1, tz = 1;
  const int shape = deposit_shape<R>(m.n, ty, tz);
  if (size_t(warps) * ty * tz * deposit_stride_of<R>(m.n) * sizeof(R) > 48 * 1024) {
    // once per device, for every tile shape, so that no attribute call falls inside a stream capture
    static bool done[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      const int most = int(DEP_WARPS * PM_DEPOSIT_WARP_BYTES * sizeof(R) / 4);
      cudaError_t e = cudaSuccess;
      void* fns[8] = {(void*)k_deposit<R, 2, 4, false>, (void*)k_deposit<R, 2, 4, true>,
                      (void*)k_deposit<R, 2, 2, false>, (void*)k_deposit<R, 2, 2, true>,
                      (void*)k_deposit<R, 1, 2, false>, (void*)k_deposit<R, 1, 2, true>,
                      (void*)k_deposit<R, 1, 1, false>, (void*)k_deposit<R, 1, 1, true>};
      for (void* f : fns)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  switch (shape) {
    case 0: return launch_deposit_tile<R, 2, 4>(pos, row_start, n, m, norm, rho, s, warps, nm, ms);
    case 1: return launch_deposit_tile<R, 2, 2>(pos, row_start, n, m, norm, rho, s, warps, nm, ms);
    case 2: return launch_deposit_tile<R, 1, 2>(pos, row_start, n, m, norm, rho, s, warps, nm, ms);
    default: return launch_deposit_tile<R, 1, 1>(pos, row_start, n, m, norm, rho, s, warps, nm, ms);
  }
}

template <typename R>
cudaError_t launch_spline_weights(void* w, Mesh m, double hc, cudaStream_t s) {
  k_spline_weights<R><<<MESH_GRID, MESH_THREADS, 0, s>>>((R*)w, m, hc);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_spline_symbol(const void* spec, void* what, Mesh m, cudaStream_t s) {
  using C = typename VT<R>::cplx;
  k_spline_symbol<R><<<MESH_GRID, MESH_THREADS, 0, s>>>((const C*)spec, (R*)what, m.n2 * uint32_t(m.n / 2 + 1));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_green_spline(void* spec, void* spec2, const void* what, Mesh m, double coef, double* part,
                                cudaStream_t s, int smooth_in) {
  using C = typename VT<R>::cplx;
  k_green_spline<R><<<MESH_GRID, MESH_THREADS, m.n * sizeof(R), s>>>(
      (C*)spec, (C*)spec2, (const R*)what, m, R(coef), R(1.0 / double(m.n3)), divu32_make(uint32_t(m.n / 2 + 1)), part,
      smooth_in);
  return cudaGetLastError();
}

// the direct smoothing (support within three cells, n_mesh <= 512: one
// thread per x of a row); zc planes per block.  g[s*4 + i] = w(i^2 + s);
// maxr2: the largest squared offset with a nonzero weight
template <typename R>
cudaError_t launch_smooth_direct(const R* in, R* out, Mesh m, const double* g, int maxr2, cudaStream_t s) {
  SplineTaps<R> tp;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) tp.c[i][j][k] = R(g[(j * j + k * k) * 4 + i]);
#ifndef PM_SD_ZC
#define PM_SD_ZC 16
#endif
  const int zc = m.n >= 2 * PM_SD_ZC ? PM_SD_ZC : m.n;
  const dim3 grid(unsigned(m.n), unsigned((m.n + zc - 1) / zc));
  const size_t smem = 3 * m.n * sizeof(R);
  if (maxr2 <= 8)
    k_smooth_direct<R, 8><<<grid, unsigned(m.n), smem, s>>>(in, out, m, tp, zc);
  else if (maxr2 <= 12)
    k_smooth_direct<R, 12><<<grid, unsigned(m.n), smem, s>>>(in, out, m, tp, zc);
  else if (maxr2 <= 15)
    k_smooth_direct<R, 15><<<grid, unsigned(m.n), smem, s>>>(in, out, m, tp, zc);
  else
    k_smooth_direct<R, 27><<<grid, unsigned(m.n), smem, s>>>(in, out, m, tp, zc);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_smooth_spec(void* spec, const void* what, Mesh m, cudaStream_t s) {
  using C = typename VT<R>::cplx;
  k_smooth_spec<R><<<MESH_GRID, MESH_THREADS, 0, s>>>((C*)spec, (const R*)what, m.n2 * uint32_t(m.n / 2 + 1),
                                                      R(1.0 / double(m.n3)));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_green(void* spec, Mesh m, double coef, double* part, cudaStream_t s, const double* coefp, int nm,
                         size_t ms) {
  using C = typename VT<R>::cplx;
  if (nm > 1)
    k_green<R, true><<<dim3(MESH_GRID, unsigned(nm)), MESH_THREADS, m.n * sizeof(R), s>>>(
        (C*)spec, m, R(coef), divu32_make(uint32_t(m.n / 2 + 1)), part, coefp, ms);
  else
    k_green<R, false><<<MESH_GRID, MESH_THREADS, m.n * sizeof(R), s>>>(
        (C*)spec, m, R(coef), divu32_make(uint32_t(m.n / 2 + 1)), part, nullptr, 0);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t launch_spec_z_pq(float2* spec, const float2* tw, const float* s2, double coef, double* part,
                             cudaStream_t s, const double* coefp, int nm, size_t ms) {
  constexpr int N = P * Q;
  const size_t smem = size_t(N) * (SPZ_COLS * sizeof(float2) + sizeof(float2) + sizeof(float));
  const unsigned tiles = unsigned(N * (N / 2 + 1) / SPZ_COLS);
  if (nm > 1)
    k_spec_z<P, Q, true><<<dim3(tiles, unsigned(nm)), SPZ_COLS * P, smem, s>>>(spec, tw, s2, float(coef), part, coefp,
                                                                             ms);
  else
    k_spec_z<P, Q, false><<<tiles, SPZ_COLS * P, smem, s>>>(spec, tw, s2, float(coef), part, nullptr, 0);
  return cudaGetLastError();
}

inline dim3 stencil_grid(int n) { return dim3((n + ST_X - 1) / ST_X, (n + ST_Y - 1) / ST_Y, ST_ZCH); }
inline int stencil_zlen(int n) { return (n + ST_ZCH - 1) / ST_ZCH; }
// entries of the near-empty node list (one region per stencil block)
inline size_t stencil_list_len(int n) {
  const dim3 g = stencil_grid(n);
  const size_t tiled = size_t(g.x) * g.y * g.z * ST_X * ST_Y * stencil_zlen(n);
  const size_t tiles = size_t(n) * n * (n + 16);  // one-shot tiles, a ragged last tile included
  return tiled > tiles ? tiled : tiles;
}
inline int stencil_blocks(int n) {
  const dim3 g = stencil_grid(n);
  return int(g.x * g.y * g.z);
}

template <typename R>
cudaError_t launch_stencil(const R* rho, Mesh m, StencilParams sp, R* q, double* part, uint32_t* list,
                           uint32_t* list_count, uint32_t* err, cudaStream_t s, const double* qcp, int nm,
                           size_t ms) {
  // a packed group steps its members in one launch of the one-shot tiles only
  if (nm > 1 && !stencil_tile_path(m.n, sp, sizeof(R) == 4)) return cudaErrorInvalidValue;
  if (sizeof(R) == 4 && sp.step == 1) {
    // fp32 compact path: shared-memory tiles, ill-conditioned near-empty nodes redone in float-float
    const float slim = sp.rho_fp64 > 0 ? float(sqrt(sp.rho_fp64)) : 0.0f;
    if (stencil_tile_path(m.n, sp, true)) {
      static bool done[64];
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64 || !done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_stencil_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(SB_SMEM_MAX));
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(k_stencil_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(SB_SMEM_MAX));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
      }
      const dim3 g(unsigned(m.n / sp.ty), unsigned((m.n + sp.zlen - 1) / sp.zlen), unsigned(nm));
      if (nm > 1)
        k_stencil_tile<true><<<g, SB_THREADS, stencil_tile_smem(m.n, sp.ty, sp.zlen), s>>>(
            (const float*)rho, m, float(sp.rho_floor), float(sp.qcoef), slim, sp.ty, sp.zlen, (float*)q, list, part,
            err, sp.diag, qcp, ms);
      else
        k_stencil_tile<false><<<g, SB_THREADS, stencil_tile_smem(m.n, sp.ty, sp.zlen), s>>>(
            (const float*)rho, m, float(sp.rho_floor), float(sp.qcoef), slim, sp.ty, sp.zlen, (float*)q, list, part,
            err, sp.diag, nullptr, 0);
      return cudaGetLastError();
    }
    if (sp.ty > 0 && stencil_bulk_shape_ok(m.n, sp.ty, sp.zlen, sp.stages)) {
      static bool done[64];  // the shared-memory opt-in, once per device (never inside a capture)
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64 || !done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_stencil_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(SB_SMEM_MAX));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
      }
      const dim3 g(unsigned(m.n / sp.ty), unsigned((m.n + sp.zlen - 1) / sp.zlen));
      k_stencil_bulk<<<g, SB_THREADS, stencil_bulk_smem(m.n, sp.ty, sp.stages), s>>>(
          (const float*)rho, m, float(sp.rho_floor), float(sp.qcoef), slim, sp.ty, sp.zlen, sp.stages, (float*)q,
          part, err, sp.diag);
      return cudaGetLastError();
    }
    const dim3 g = stencil_grid(m.n), b(ST_X, ST_TY);
    const int zlen = stencil_zlen(m.n);
    k_stencil_tiled<<<g, b, 0, s>>>((const float*)rho, m, float(sp.rho_floor), float(sp.qcoef), slim, zlen, (float*)q,
                                    list, list_count, part, sp.diag);
  } else {
    k_stencil<R><<<MESH_GRID, MESH_THREADS, 0, s>>>(rho, m, sp, q, part);
  }
  return cudaGetLastError();
}

// resident blocks of k_kick_stream on the whole GPU for a block size, queried
// once per device and block size (pm_create asks first, outside any capture);
// if the query fails, one particle per thread
template <typename R>
int kick_stream_resident(int threads, int fm = KICK_FM_ANY) {
  static int cache[64][2][2];
  int dev = 0;
  cudaGetDevice(&dev);
  const int t = threads == 128 ? 0 : 1, f = fm == KICK_FM_HYBRID_Q ? 1 : 0;
  if (dev >= 0 && dev < 64 && cache[dev][t][f] > 0) return cache[dev][t][f];
  int per_sm = 0, sms = 0, r = 1 << 30;
  const void* fn = f ? (const void*)k_kick_stream<R, false, KICK_FM_HYBRID_Q> : (const void*)k_kick_stream<R, false, KICK_FM_ANY>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && per_sm > 0 && sms > 0)
    r = per_sm * sms;
  else
    cudaGetLastError();
  if (dev >= 0 && dev < 64) cache[dev][t][f] = r;
  return r;
}
// the compile-time force form of a kick's parameters (the common HYBRID run with the quantum force)
inline int kick_fm(const KickParams& kp) {
  return (!kp.grav_kernel && kp.quantum && kp.q_kernel) ? KICK_FM_HYBRID_Q : KICK_FM_ANY;
}
inline unsigned kick_stream_blocks(int64_t n, int threads, int resident) {
  const int64_t need = (n + threads - 1) / threads;
  return unsigned(need < resident ? need : resident);
}

template <typename R>
cudaError_t launch_kick(void* pos, void* mom, uint32_t* keys, uint32_t* tcount, int64_t n, const R* phi, const R* q,
                        Mesh m, KickParams kp,
                        const KickParams* kp_tab, const uint32_t* step, double* part, double* acc, uint32_t* err,
                        int threads, cudaStream_t s, int nm, size_t ms) {
  if (n <= 0) return cudaSuccess;
  if (nm > 1) {
    // a packed group: the streaming pass of every member, resident blocks shared among them
    if constexpr (sizeof(R) == 4) {
      if (kp.maxima || kp.accel_out || kp.diag || !kp_tab) return cudaErrorInvalidValue;
      using V4 = typename VT<R>::v4;
      if (threads != 128 && threads != 256) threads = KICK_THREADS;
      const int per = kick_stream_resident<R>(threads) / nm;
      const unsigned g = kick_stream_blocks(n, threads, per > 1 ? per : 1);
      if (kick_fm(kp) == KICK_FM_HYBRID_Q)
        k_kick_stream<R, true, KICK_FM_HYBRID_Q><<<dim3(g, unsigned(nm)), threads, 0, s>>>(
            (V4*)pos, (V4*)mom, keys, tcount, n, phi, q, m, kp, kp_tab, step, err, ms);
      else
        k_kick_stream<R, true, KICK_FM_ANY><<<dim3(g, unsigned(nm)), threads, 0, s>>>(
            (V4*)pos, (V4*)mom, keys, tcount, n, phi, q, m, kp, kp_tab, step, err, ms);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  using V4 = typename VT<R>::v4;
  if (threads != 128 && threads != 256) threads = KICK_THREADS;
  const unsigned g = kick_blocks(n, threads);
  V4 *p = (V4*)pos, *mo = (V4*)mom;
  if (kp.maxima)
    k_kick<R, 3><<<g, threads, 0, s>>>(p, mo, keys, tcount, n, phi, q, m, kp, kp_tab, step, part, acc, err);
  else if (kp.accel_out)
    k_kick<R, 2><<<g, threads, 0, s>>>(p, mo, keys, tcount, n, phi, q, m, kp, kp_tab, step, part, acc, err);
  else if (kp.diag)
    k_kick<R, 1><<<g, threads, 0, s>>>(p, mo, keys, tcount, n, phi, q, m, kp, kp_tab, step, part, acc, err);
  else if constexpr (sizeof(R) == 4) {  // the fp64 records would spill in the streaming loop
    const int fm = kick_fm(kp);
    const unsigned gs = kick_stream_blocks(n, threads, kick_stream_resident<R>(threads, fm));
    if (fm == KICK_FM_HYBRID_Q)
      k_kick_stream<R, false, KICK_FM_HYBRID_Q><<<gs, threads, 0, s>>>(p, mo, keys, tcount, n, phi, q, m, kp, kp_tab,
                                                                       step, err, 0);
    else
      k_kick_stream<R, false, KICK_FM_ANY><<<gs, threads, 0, s>>>(p, mo, keys, tcount, n, phi, q, m, kp, kp_tab, step,
                                                                  err, 0);
  }
  else
    k_kick<R, 0><<<g, threads, 0, s>>>(p, mo, keys, tcount, n, phi, q, m, kp, kp_tab, step, part, acc, err);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_power(const void* spec, Mesh m, int nbins, double* part, cudaStream_t s) {
  using C = typename VT<R>::cplx;
  k_power<R><<<RED_GRID, MESH_THREADS, 0, s>>>((const C*)spec, m, nbins, part);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_get_particles(const void* pos, const void* mom, int64_t n, Mesh m, double dx, double* x, double* p,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  using V4 = typename VT<R>::v4;
  k_get_particles<R><<<unsigned((n + 255) / 256), 256, 0, s>>>((const V4*)pos, (const V4*)mom, n, m, dx, x, p);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_get_order(const void* pos, const void* mom, int64_t n, uint32_t* cell, uint32_t* id,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  using V4 = typename VT<R>::v4;
  k_get_order<R><<<unsigned((n + 255) / 256), 256, 0, s>>>((const V4*)pos, (const V4*)mom, n, cell, id);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_to_double(const R* f, int64_t n, double* out, cudaStream_t s) {
  k_to_double<R><<<RED_GRID, 256, 0, s>>>(f, n, out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_from_double(const double* f, int64_t n, R* out, cudaStream_t s) {
  k_from_double<R><<<RED_GRID, 256, 0, s>>>(f, n, out);
  return cudaGetLastError();
}

}  // namespace pm
