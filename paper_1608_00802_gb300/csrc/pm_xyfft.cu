// The x and y transforms of the z-planes of a 256^3 fp32 mesh, each direction
// in one kernel (the forward transform of the density before the z kernel,
// the inverse transform of the potential after it), in place of the batched
// 2D cuFFT plans, which read and write every plane twice.
//
// A cluster of eight CTAs owns one plane (four with PM_XY_CLUSTER=4).
// Forward (real rows -> half spectrum):
//  - CTA q transforms its 32 rows y = 32 q .. 32 q + 31 along x.  A 256-point
//    real transform is a 128-point complex one of z[m] = x[2m] + i x[2m+1]
//    (four-step, 128 = 8 x 16: thread j of a row does the 16-point DFT over
//    m of z[j + 8m] and the twiddle, after an exchange through shared memory
//    a thread does the 8-point DFTs over j of two k1), then
//      X[k] = E[k] + W^k O[k],  E = (Z[k] + Z*[128-k]) / 2,
//      O = -i (Z[k] - Z*[128-k]) / 2,  W = exp(-2 pi i / 256);
//    X[0] and X[128] are real and travel packed as X[0] + i X[128].
//  - After a cluster barrier, CTA q reads its columns (16 q .. 16 q + 15) of
//    every row from the shared memory of the CTA that owns the row.
//  - CTA q transforms its 16 columns along y (four-step, 256 = 16 x 16, as
//    in the z kernel) and writes them to the half spectrum [z][ky][kx].  The
//    packed column holds the transforms A + i B of two real sequences, so
//    A[ky] = (Y[ky] + Y*[-ky]) / 2 and B[ky] = -i (Y[ky] - Y*[-ky]) / 2 give
//    the kx = 0 and kx = 128 columns.
// Inverse (half spectrum -> real rows): the same steps backwards with
// conjugate twiddles; a row's 128-point inverse transform takes
//      Z[k] = (X[k] + X*[128-k]) + i W^-k (X[k] - X*[128-k]),
// read from the cluster's columns.  Both directions are unnormalised, like
// cuFFT's R2C and C2R.
#include <cooperative_groups.h>

#include "pm_kernels.cuh"

namespace pm {
namespace cg = cooperative_groups;

namespace {

#ifndef PM_XY_CLUSTER
#define PM_XY_CLUSTER 8  // CTAs per plane (4 or 8)
#endif
constexpr int XY_N = 256, XY_CL = PM_XY_CLUSTER, XY_ROWS = XY_N / XY_CL, XY_COLS = XY_N / 2 / XY_CL;
constexpr int XY_THREADS = XY_ROWS * 8, XY_MINB = 1024 / XY_THREADS;  // 1024 threads of 64 registers per SM
constexpr int XY_NH = XY_N / 2 + 1;  // complex values per row of the half spectrum
constexpr int XY_SROW = 136;         // a row's 128 values in the x exchange, one pad slot per 16
constexpr int XY_TSZ = XY_N * XY_COLS > XY_ROWS * XY_SROW ? XY_N * XY_COLS : XY_ROWS * XY_SROW;
constexpr size_t XY_SMEM = size_t(XY_TSZ + XY_N) * sizeof(float2);
static_assert(XY_THREADS == XY_ROWS * 8 && XY_THREADS == XY_COLS * 16, "one thread per (row, j) and (column, j)");

__device__ __forceinline__ int xy_sw(int n) { return n + (n >> 4); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// E + W^k O and the packed X[0] + i X[128] from Z[k] and Z[128 - k]
__device__ __forceinline__ float2 r2c_post(float2 z, float2 zp, float2 w, bool k0) {
  const float ex = 0.5f * (z.x + zp.x), ey = 0.5f * (z.y - zp.y);  // E = (Z + Z*p) / 2
  const float ox = 0.5f * (z.y + zp.y), oy = -0.5f * (z.x - zp.x);  // O = -i (Z - Z*p) / 2
  if (k0) return make_float2(ex + ox, ex - ox);                    // (E0 + O0) + i (E0 - O0), both real
  const float2 wo = cmul(make_float2(ox, oy), w);
  return make_float2(ex + wo.x, ey + wo.y);
}

// Z[k] = (X[k] + X*[128-k]) + i W^-k (X[k] - X*[128-k]); k = 0: X[0], X[128] from the packed value
__device__ __forceinline__ float2 c2r_pre(float2 x, float2 xp, float2 w, bool k0) {
  if (k0) return make_float2(x.x + x.y, x.x - x.y);
  const float2 e = make_float2(x.x + xp.x, x.y - xp.y);
  const float2 d = cmul(make_float2(x.x - xp.x, x.y + xp.y), conjf2(w));  // W^-k (X - X*p)
  return make_float2(e.x - d.y, e.y + d.x);
}

template <bool PACKED>
__global__ void __cluster_dims__(XY_CL, 1, 1) __launch_bounds__(XY_THREADS, XY_MINB)
    k_xy_r2c(const float* __restrict__ rho, float2* __restrict__ spec, const float2* __restrict__ twg, size_t ms) {
  if constexpr (PACKED) {  // member blockIdx.y of a packed group
    const size_t o = size_t(blockIdx.y) * ms;
    rho = moff(rho, o), spec = moff(spec, o);
  }
  extern __shared__ __align__(16) unsigned char xy_smem[];
  float2* T = reinterpret_cast<float2*>(xy_smem);
  float2* tw = T + XY_TSZ;
  cg::cluster_group cl = cg::this_cluster();
  const int q = int(cl.block_rank()), z = int(blockIdx.x) / XY_CL, tid = threadIdx.x;
  // the CTA's XY_ROWS rows by 16-byte asynchronous copies, XY_SROW complex values apart
  {
    float* R = reinterpret_cast<float*>(T);
    const float* src = rho + (size_t(z) * XY_N + size_t(XY_ROWS) * q) * XY_N;
    for (int i = tid; i < XY_ROWS * XY_N / 4; i += XY_THREADS) {
      const int row = i / (XY_N / 4), c4 = i % (XY_N / 4);
      cp_async16(R + row * 2 * XY_SROW + 4 * c4, src + row * XY_N + 4 * c4);
    }
  }
  for (int i = tid; i < XY_N; i += XY_THREADS) tw[i] = twg[i];
  cp_async_wait_all();
  __syncthreads();
  // x: thread j of row r (8 lanes per row, 4 rows per warp), the 16 values z[j + 8m]
  const int r = tid >> 3, j = tid & 7, rl = (threadIdx.x & 31) & ~7;
  float2* S = T + r * XY_SROW;
  float2 a[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) a[m] = S[j + 8 * m];
  __syncthreads();  // the rows are read: the area becomes the x exchange
  dft_reg<16, false>(a);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) S[xy_sw(j + 8 * k1)] = cmul(a[bitrev<16>(k1)], tw[(2 * j * k1) & (XY_N - 1)]);
  __syncthreads();
  float2 Z[2][8];
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // thread j now takes k1 = 2j + h: 8-point DFTs over the row's j
    const int k1 = 2 * j + h;
    float2 b[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) b[jj] = S[xy_sw(jj + 8 * k1)];
    dft_reg<8, false>(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) Z[h][k2] = b[bitrev<8>(k2)];
  }
  // Z[128 - k] of k = k1 + 16 k2 is Z[(16 - k1) + 16 (7 - k2)]: lane 8 - j's Z[0][7 - k2] for k1 = 2j > 0,
  // lane 7 - j's Z[1][7 - k2] for k1 = 2j + 1; for k1 = 0 it is this lane's Z[0][(8 - k2) mod 8]
  {
    float2 zp[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      const float2 o = Z[0][7 - k2];
      zp[k2] = make_float2(__shfl_sync(0xffffffffu, o.x, rl + ((8 - j) & 7)),
                           __shfl_sync(0xffffffffu, o.y, rl + ((8 - j) & 7)));
      if (j == 0) zp[k2] = Z[0][(8 - k2) & 7];
    }
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) Z[0][k2] = r2c_post(Z[0][k2], zp[k2], tw[2 * j + 16 * k2], j == 0 && k2 == 0);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      const float2 o = Z[1][7 - k2];
      zp[k2] = make_float2(__shfl_sync(0xffffffffu, o.x, rl + 7 - j), __shfl_sync(0xffffffffu, o.y, rl + 7 - j));
    }
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) Z[1][k2] = r2c_post(Z[1][k2], zp[k2], tw[2 * j + 1 + 16 * k2], false);
  }
  __syncthreads();  // the exchange is read: the area holds the rows' X[k], row after row
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) S[2 * j + h + 16 * k2] = Z[h][k2];
  cl.sync();
  // y: column c of the CTA's XY_COLS, thread jt; X[y][XY_COLS q + c] read from the CTA that owns row y (runs of
  // XY_COLS contiguous values)
  const int c = tid & (XY_COLS - 1), jt = tid / XY_COLS;
  float2 u[16];
#pragma unroll
  for (int mm = 0; mm < 16; ++mm) {
    const int yy = jt + 16 * mm;
    u[mm] = cl.map_shared_rank(T, yy / XY_ROWS)[(yy % XY_ROWS) * XY_SROW + XY_COLS * q + c];
  }
  cl.sync();  // no CTA reads another's rows any more: the area becomes the y exchange
  dft_reg<16, false>(u);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) T[(jt + 16 * k1) * XY_COLS + c] = cmul(u[bitrev<16>(k1)], tw[(jt * k1) & (XY_N - 1)]);
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) u[jj] = T[(jj + 16 * jt) * XY_COLS + c];
  dft_reg<16, false>(u);  // u[bitrev(k2)] = Y[jt + 16 k2]
  float2* out = spec + size_t(z) * XY_N * XY_NH;
  const int kx = XY_COLS * q + c;
  if (kx != 0) {
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) out[(jt + 16 * k2) * XY_NH + kx] = u[bitrev<16>(k2)];
  }
  if (q == 0) {  // the packed column: kx = 0 and kx = N/2
    __syncthreads();
    if (c == 0) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) T[(jt + 16 * k2) * XY_COLS] = u[bitrev<16>(k2)];
    }
    __syncthreads();
    if (c == 0) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int ky = jt + 16 * k2;
        const float2 yv = u[bitrev<16>(k2)], ym = T[((XY_N - ky) & (XY_N - 1)) * XY_COLS];
        out[ky * XY_NH] = make_float2(0.5f * (yv.x + ym.x), 0.5f * (yv.y - ym.y));
        out[ky * XY_NH + XY_N / 2] = make_float2(0.5f * (yv.y + ym.y), -0.5f * (yv.x - ym.x));
      }
    }
  }
}

template <bool PACKED>
__global__ void __cluster_dims__(XY_CL, 1, 1) __launch_bounds__(XY_THREADS, XY_MINB)
    k_xy_c2r(const float2* __restrict__ spec, float* __restrict__ phi, const float2* __restrict__ twg, size_t ms) {
  if constexpr (PACKED) {
    const size_t o = size_t(blockIdx.y) * ms;
    spec = moff(spec, o), phi = moff(phi, o);
  }
  extern __shared__ __align__(16) unsigned char xy_smem[];
  float2* T = reinterpret_cast<float2*>(xy_smem);
  float2* tw = T + XY_TSZ;
  cg::cluster_group cl = cg::this_cluster();
  const int q = int(cl.block_rank()), z = int(blockIdx.x) / XY_CL, tid = threadIdx.x;
  for (int i = tid; i < XY_N; i += XY_THREADS) tw[i] = twg[i];
  // y: column c of this CTA's XY_COLS (kx = 0 packed with kx = N/2), thread jt
  const int c = tid & (XY_COLS - 1), jt = tid / XY_COLS, kx = XY_COLS * q + c;
  const float2* in = spec + size_t(z) * XY_N * XY_NH;
  float2 u[16];
#pragma unroll
  for (int mm = 0; mm < 16; ++mm) {
    const int ky = jt + 16 * mm;
    if (kx == 0) {
      const float2 a0 = __ldcs(in + ky * XY_NH), b0 = __ldcs(in + ky * XY_NH + XY_N / 2);
      u[mm] = make_float2(a0.x - b0.y, a0.y + b0.x);  // A + i B
    } else {
      u[mm] = __ldcs(in + ky * XY_NH + kx);
    }
  }
  __syncthreads();  // twiddles
  dft_reg<16, true>(u);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1)
    T[(jt + 16 * k1) * XY_COLS + c] = cmul(u[bitrev<16>(k1)], conjf2(tw[(jt * k1) & (XY_N - 1)]));
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) u[jj] = T[(jj + 16 * jt) * XY_COLS + c];
  dft_reg<16, true>(u);  // u[bitrev(k2)] = the value of row jt + 16 k2
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) T[(jt + 16 * k2) * XY_COLS + c] = u[bitrev<16>(k2)];
  cl.sync();  // all columns transformed: each row gathers its 129 values from the cluster
  // x: thread j of row r (8 lanes per row, 4 rows per warp) reads X[k], k = j + 8m, from the CTA that owns
  // column k; X[128 - k] is lane 8 - j's X[(8 - j) + 8 (15 - m)] (j > 0) or this lane's X[8 (16 - m)] (j = 0)
  const int r = tid >> 3, j = tid & 7, y = XY_ROWS * q + r, rl = (threadIdx.x & 31) & ~7;
  const int partner = rl + ((8 - j) & 7);
  float2 a[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k = j + 8 * m;
    a[m] = cl.map_shared_rank(T, k / XY_COLS)[y * XY_COLS + (k % XY_COLS)];
  }
  {
    // m < 8 into a separate array (the partner still needs this lane's a[0..7] for its m >= 8), then
    // m >= 8 in place (nobody needs a[8..15] any more)
    float2 lo[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float2 o = a[15 - m];
      float2 xp = make_float2(__shfl_sync(0xffffffffu, o.x, partner), __shfl_sync(0xffffffffu, o.y, partner));
      if (j == 0) xp = a[(16 - m) & 15];
      lo[m] = c2r_pre(a[m], xp, tw[j + 8 * m], j == 0 && m == 0);
    }
#pragma unroll
    for (int m = 8; m < 16; ++m) {
      const float2 o = a[15 - m];
      float2 xp = make_float2(__shfl_sync(0xffffffffu, o.x, partner), __shfl_sync(0xffffffffu, o.y, partner));
      if (j == 0) xp = a[16 - m];
      a[m] = c2r_pre(a[m], xp, tw[j + 8 * m], false);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) a[m] = lo[m];
  }
  cl.sync();  // no CTA reads another's columns any more: the area becomes the x exchange
  dft_reg<16, true>(a);
  float2* S = T + r * XY_SROW;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1)
    S[xy_sw(j + 8 * k1)] = cmul(a[bitrev<16>(k1)], conjf2(tw[(2 * j * k1) & (XY_N - 1)]));
  __syncthreads();
  float2 o[2][8];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k1 = 2 * j + h;
    float2 b[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) b[jj] = S[xy_sw(jj + 8 * k1)];
    dft_reg<8, true>(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) o[h][k2] = b[bitrev<8>(k2)];  // (x[2n], x[2n+1]), n = k1 + 16 k2
  }
  __syncthreads();  // the exchange is read: the area holds the rows, then 16-byte stores
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) S[2 * j + h + 16 * k2] = o[h][k2];
  __syncthreads();
  float4* out = reinterpret_cast<float4*>(phi + (size_t(z) * XY_N + size_t(XY_ROWS) * q) * XY_N);
  const float4* src = reinterpret_cast<const float4*>(T);
  for (int i = tid; i < XY_ROWS * XY_N / 4; i += XY_THREADS) {
    const int row = i / (XY_N / 4), c4 = i % (XY_N / 4);
    out[row * (XY_N / 4) + c4] = src[row * (XY_SROW / 2) + c4];
  }
}

// the shared-memory attribute of all four kernels, once per device (so that no attribute call falls
// inside a stream capture)
cudaError_t xy_prepare() {
  static bool done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  const void* fns[4] = {(const void*)k_xy_r2c<false>, (const void*)k_xy_r2c<true>, (const void*)k_xy_c2r<false>,
                        (const void*)k_xy_c2r<true>};
  for (const void* f : fns)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(XY_SMEM));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

}  // namespace

bool xy_fft_supported(int n_mesh) { return n_mesh == XY_N; }

cudaError_t launch_xy_r2c(const float* rho, void* spec, const void* tw, int n_mesh, cudaStream_t s, int nm, size_t ms) {
  if (!xy_fft_supported(n_mesh)) return cudaErrorInvalidValue;
  cudaError_t e = xy_prepare();
  if (e != cudaSuccess) return e;
  const dim3 grid(unsigned(XY_N * XY_CL), unsigned(nm > 1 ? nm : 1));
  if (nm > 1)
    k_xy_r2c<true><<<grid, XY_THREADS, XY_SMEM, s>>>(rho, (float2*)spec, (const float2*)tw, ms);
  else
    k_xy_r2c<false><<<grid, XY_THREADS, XY_SMEM, s>>>(rho, (float2*)spec, (const float2*)tw, 0);
  return cudaGetLastError();
}

cudaError_t launch_xy_c2r(const void* spec, float* phi, const void* tw, int n_mesh, cudaStream_t s, int nm, size_t ms) {
  if (!xy_fft_supported(n_mesh)) return cudaErrorInvalidValue;
  cudaError_t e = xy_prepare();
  if (e != cudaSuccess) return e;
  const dim3 grid(unsigned(XY_N * XY_CL), unsigned(nm > 1 ? nm : 1));
  if (nm > 1)
    k_xy_c2r<true><<<grid, XY_THREADS, XY_SMEM, s>>>((const float2*)spec, phi, (const float2*)tw, ms);
  else
    k_xy_c2r<false><<<grid, XY_THREADS, XY_SMEM, s>>>((const float2*)spec, phi, (const float2*)tw, 0);
  return cudaGetLastError();
}

}  // namespace pm
