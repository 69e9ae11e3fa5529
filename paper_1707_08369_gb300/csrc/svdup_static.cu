// svdup_static.cu -- secular roots for callers that cannot allocate device memory.
//
// svdup_secular needs a handle, and a handle allocates (its status word at create, its
// workspace on first use).  Some callers cannot do that: code that runs inside a host
// application whose memory pool has already claimed the device memory it is allowed,
// plug-ins that are not permitted to call the CUDA allocator, and latency-critical loops
// where cudaMalloc/cudaFree would synchronise the device.  svdup_secular_static gives
// them the same roots with its scratch in a fixed array of this library's device memory.
//
// The array below is a file-scope __device__ variable: every GPU that loads the library
// holds it (SVDUP_SECULAR_STATIC_MAX_K bounds its size) until the process exits.  In
// host code its name is only a host-side stand-in, so its device address is looked up
// with cudaGetSymbolAddress, once per device, on that device's first call.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "svdup_internal.cuh"

using namespace svdup;

namespace {

constexpr int kMaxK = SVDUP_SECULAR_STATIC_MAX_K;
// Slots of the scratch array, each a multiple of 256 bytes: rho and k (one 256-byte
// slot), then dc, z2c, dk, tauc, dorg (doubles) and orgc (ints), kMaxK entries each.
constexpr size_t kSlot = (kMaxK * sizeof(double) + 255) / 256 * 256;
constexpr size_t kScratchDoubles = (256 + 6 * kSlot) / sizeof(double);
constexpr int kMaxDevices = 64;

std::mutex g_mu;
double* g_addr[kMaxDevices];  // device address of the array, per device ordinal

}  // namespace

static __device__ __align__(256) double g_secular_scratch[kScratchDoubles];

namespace {

// The device address of the scratch array on the current device (looked up on the
// device's first call and cached).
int scratch_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SVDUP_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_secular_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SVDUP_ECUDA;
    }
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return SVDUP_OK;
}

// rho, k and the rho > 0 orientation of the problem (the solver's input form): for
// rho < 0 the poles are reflected, d -> -d in reversed order.
// A NaN or infinity in d or z latches SVDUP_ENONFINITE in the caller's info word.
__global__ void k_static_prep(int k, const double* __restrict__ d, const double* __restrict__ z,
                              double rho, double* rhop, int* kp, double* dc, double* z2c,
                              double* dk, int* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    rhop[0] = rho;
    kp[0] = k;
  }
  if (t >= k) return;
  dk[t] = d[t];
  const int s = rho > 0.0 ? t : k - 1 - t;
  dc[t] = rho > 0.0 ? d[s] : -d[s];
  z2c[t] = z[s] * z[s];
  if (!isfinite(d[s]) || !isfinite(z[s])) latch(status, SVDUP_ENONFINITE);
}

}  // namespace

extern "C" int svdup_secular_static(void* stream, int k, const double* d, const double* z,
                                    double rho, int* org, double* tau, int* info) {
  if (k < 1 || k > kMaxK || !d || !z || !org || !tau || !info) return SVDUP_EINVAL;
  if (!(rho != 0.0) || !isfinite(rho)) return SVDUP_EINVAL;
  double* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* b = (char*)base;
  Eig e;
  memset(&e, 0, sizeof(e));
  e.N = k;
  e.rhop = (double*)b;
  e.kp = (int*)(b + sizeof(double));
  e.dc = (double*)(b + 256);
  e.z2c = (double*)(b + 256 + kSlot);
  e.dk = (double*)(b + 256 + 2 * kSlot);
  e.tauc = (double*)(b + 256 + 3 * kSlot);
  e.dorg = (double*)(b + 256 + 4 * kSlot);
  e.orgc = (int*)(b + 256 + 5 * kSlot);
  e.org = org;  // the results go straight to the caller's buffers
  e.tau = tau;
  // The status starts at zero on every call; the scratch slots are all rewritten
  // before they are read, so the previous call's contents do not matter.
  if (cudaMemsetAsync(info, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return SVDUP_ECUDA;
  }
  k_static_prep<<<(k + 255) / 256, 256, 0, st>>>(k, d, z, rho, e.rhop, e.kp, e.dc, e.z2c, e.dk,
                                                 info);
  SVDUP_COUNT_LAUNCH();
  launch_secular(st, e, info, 64);
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? SVDUP_OK : SVDUP_ECUDA;
}
