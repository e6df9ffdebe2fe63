// pm_deposit_noalloc: the cloud-in-cell deposit for callers that must not
// allocate device memory.  Some callers cannot call cudaMalloc or cudaFree:
// cudaFree synchronises the whole device and cudaMalloc may block, which a
// latency-critical serving loop or a real-time thread cannot afford, and a
// process that has already handed its whole device-memory budget to fixed
// arenas has nothing left to allocate from.  This entry point therefore keeps
// every temporary (particle records, sort keys and values, digit histograms,
// look-back status words, row starts) in one file-scope static device array
// of PM_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.  It calls no allocating routine, its own or a
// library's.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/pm.h"
#include "pm_internal.h"

using namespace pm;

namespace {

constexpr int64_t kMaxPart = PM_NOALLOC_MAX_PARTICLES;
constexpr int kMaxMesh = PM_NOALLOC_MAX_MESH;
constexpr int kMaxTiles = int((kMaxPart + RS_TILE - 1) / RS_TILE);
constexpr size_t kRadixMax = size_t(1) << RS_MAX_BITS;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// offsets inside the static scratch array
constexpr size_t kPos0 = 0;
constexpr size_t kPos1 = kPos0 + align256(kMaxPart * 16);
constexpr size_t kMom0 = kPos1 + align256(kMaxPart * 16);
constexpr size_t kMom1 = kMom0 + align256(kMaxPart * 16);
constexpr size_t kKeys0 = kMom1 + align256(kMaxPart * 16);
constexpr size_t kKeys1 = kKeys0 + align256(kMaxPart * 4);
constexpr size_t kKeys2 = kKeys1 + align256(kMaxPart * 4);
constexpr size_t kVals0 = kKeys2 + align256(kMaxPart * 4);
constexpr size_t kVals1 = kVals0 + align256(kMaxPart * 4);
constexpr size_t kHist = kVals1 + align256(kMaxPart * 4);  // 3 histograms + 4 tile counters
constexpr size_t kStatus = kHist + align256((3 * kRadixMax + 4) * 4);
constexpr size_t kRows = kStatus + align256(size_t(kMaxTiles) * kRadixMax * 8);
constexpr size_t kErr = kRows + align256((size_t(kMaxMesh) * kMaxMesh + 1) * 4);
constexpr size_t kTotal = kErr + 256;
static_assert(kTotal <= PM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds PM_NOALLOC_SCRATCH_BYTES");

static __device__ __align__(256) unsigned char g_scratch[PM_NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch per device, looked up once per device (with
// that device current) by the first call made on it.
std::mutex g_mu;
void* g_addr[64];
bool g_ready[64];

thread_local char g_msg[256];

// the call's error bits to the caller's word (device or mapped host memory)
__global__ void k_copy_error(const uint32_t* err, uint32_t* out) { *out = *err; }

// the message goes where pm_last_error(NULL) reads it
pm_status nfail(pm_status st, const char* msg) {
  set_global_error(msg);
  return st;
}

pm_status scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nfail(PM_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lock(g_mu);  // also serialises the message buffer
  if (!g_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(g_msg, sizeof g_msg, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return nfail(PM_ERR_CUDA, g_msg);
    }
    g_addr[dev] = p;
    g_ready[dev] = true;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_deposit_noalloc(const double* x_dev, int64_t n_part, int32_t n_mesh, double box, float* rho_dev,
                             uint32_t* err_dev, void* stream) {
  if (n_part < 1 || n_part > kMaxPart) {
    snprintf(g_msg, sizeof g_msg, "n_part = %lld is outside [1, %lld], the static scratch limit", (long long)n_part,
             (long long)kMaxPart);
    return nfail(PM_ERR_INVALID_ARG, g_msg);
  }
  if (n_mesh < 8 || n_mesh > kMaxMesh || (n_mesh & 1)) {
    snprintf(g_msg, sizeof g_msg, "n_mesh = %d must be even and in [8, %d], the static scratch limit", n_mesh,
             kMaxMesh);
    return nfail(PM_ERR_INVALID_ARG, g_msg);
  }
  if (!x_dev || !rho_dev || !(box > 0)) return nfail(PM_ERR_INVALID_ARG, "x, rho must be device pointers, box > 0");
  unsigned char* base = nullptr;
  pm_status st = scratch_address(&base);
  if (st != PM_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = n_part;
  Mesh m;
  m.n = n_mesh;
  m.log2n = (n_mesh & (n_mesh - 1)) == 0 ? __builtin_ctz(unsigned(n_mesh)) : -1;
  m.n2 = uint32_t(n_mesh) * uint32_t(n_mesh);
  m.n3 = m.n2 * uint32_t(n_mesh);
  int bits = 0;
  while ((uint32_t(1) << bits) < m.n3) ++bits;
  int passes = (bits + RS_MAX_BITS - 1) / RS_MAX_BITS;
  if (passes < 1) passes = 1;
  const int digit_bits = (bits + passes - 1) / passes;
  const int ntiles = int((n + RS_TILE - 1) / RS_TILE);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + kHist);
  uint32_t* counters = hist + 3 * kRadixMax;
  uint64_t* status = reinterpret_cast<uint64_t*>(base + kStatus);
  uint32_t* err = reinterpret_cast<uint32_t*>(base + kErr);
  uint32_t* keys[3] = {reinterpret_cast<uint32_t*>(base + kKeys0), reinterpret_cast<uint32_t*>(base + kKeys1),
                       reinterpret_cast<uint32_t*>(base + kKeys2)};
  uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(base + kVals0), reinterpret_cast<uint32_t*>(base + kVals1)};
  void* pos[2] = {base + kPos0, base + kPos1};
  void* mom[2] = {base + kMom0, base + kMom1};

#define NA_CU(expr)                                                                             \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      snprintf(g_msg, sizeof g_msg, "%s: %s", #expr, cudaGetErrorString(e_));                   \
      return nfail(PM_ERR_CUDA, g_msg);                                                         \
    }                                                                                           \
  } while (0)
  // the array keeps the previous call's contents: clear what must start at zero
  NA_CU(cudaMemsetAsync(hist, 0, (3 * kRadixMax + 4) * 4, s));
  NA_CU(cudaMemsetAsync(status, 0, size_t(ntiles) * (size_t(1) << digit_bits) * 8, s));
  NA_CU(cudaMemsetAsync(err, 0, 8, s));  // error word and sort epoch word
  // positions to cell + offset as pm_set_particles converts them (1/dx with dx = box/N), at rest
  NA_CU(launch_init_particles<float>(x_dev, nullptr, n, m, 1.0 / (box / n_mesh), pos[0], mom[0], keys[0], err, s));
  NA_CU(launch_sort_histogram(keys[0], n, passes, digit_bits, bits, hist, err + 1, s));
  const uint32_t* kin = keys[0];
  const uint32_t* vin = nullptr;
  int tmp = 0;
  uint32_t* sorted_keys = keys[0];
  for (int p = 0; p < passes; ++p) {
    const int shift = p * digit_bits;
    const int pb = (shift + digit_bits <= bits) ? digit_bits : (bits - shift);
    const bool last = p == passes - 1;
    if (!last) {
      NA_CU(launch_sort_pass<float>(false, kin, vin, n, shift, pb, hist + p * kRadixMax, status, counters + p, err + 1,
                                    p, ntiles, keys[1 + tmp], vals[tmp], nullptr, nullptr, nullptr, nullptr, err, s));
      kin = keys[1 + tmp];
      vin = vals[tmp];
      tmp ^= 1;
    } else {
      uint32_t* kout = (kin == keys[0]) ? keys[1 + tmp] : keys[0];
      NA_CU(launch_sort_pass<float>(true, kin, vin, n, shift, pb, hist + p * kRadixMax, status, counters + p, err + 1,
                                    p, ntiles, kout, nullptr, pos[0], mom[0], pos[1], mom[1], err, s));
      sorted_keys = kout;
    }
  }
  uint32_t* rows = reinterpret_cast<uint32_t*>(base + kRows);
  NA_CU(launch_row_start(sorted_keys, n, uint32_t(n_mesh), rows, s));
  NA_CU(launch_deposit<float>(pos[1], rows, n, m, double(m.n3) / double(n), rho_dev, s));
  if (err_dev) {
    k_copy_error<<<1, 1, 0, s>>>(err, err_dev);
    NA_CU(cudaGetLastError());
  }
#undef NA_CU
  return PM_OK;
}

}  // extern "C"
