// Green's convolution without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while device allocation
// is forbidden or unsafe (inside another framework's memory pool or a
// pre-allocated sandbox with no free device memory left, allocator hooks
// that must not re-enter the allocator, or hosts that only hand out device
// pointers to buffers they already own).  For them this file offers one
// entry point that uses a file-scope device array as its scratch instead of
// a handle's workspace.  The caller passes the input and output volumes.
//
// Scratch: g_noalloc_scratch holds the two transform buffers, the Green's
// kernel spectrum, its FP64 construction buffers and the twiddles for grids
// up to NA_MAX_N^3.  Every GPU that loads the library keeps this array until
// the process exits.  In host code the array's name is only a stand-in: its
// device address comes from cudaGetSymbolAddress, once per device (again only
// when the device's context has changed), with that device current.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

namespace {

constexpr int NA_MAX_N = 32;
constexpr int NA_MAX_P = 2 * NA_MAX_N;
constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_M1 = NA_MAX_N + 1;
constexpr size_t NA_T1 = 0;
constexpr size_t NA_T2 = na_align(NA_T1 + (size_t)NA_MAX_N * NA_MAX_N * NA_MAX_P * sizeof(float2));
constexpr size_t NA_KH = na_align(NA_T2 + (size_t)NA_MAX_N * NA_MAX_P * NA_MAX_P * sizeof(float2));
constexpr size_t NA_KA = na_align(NA_KH + NA_M1 * NA_M1 * NA_M1 * sizeof(float2));
constexpr size_t NA_KB = na_align(NA_KA + NA_M1 * NA_M1 * NA_M1 * sizeof(double2));
constexpr size_t NA_COS = na_align(NA_KB + NA_M1 * NA_M1 * NA_M1 * sizeof(double2));
constexpr size_t NA_TW = na_align(NA_COS + 3 * NA_MAX_P * sizeof(double));   // one cosine table per axis
constexpr size_t NA_ERR = na_align(NA_TW + NA_MAX_P * sizeof(float2));
constexpr size_t NA_BYTES = na_align(NA_ERR + sizeof(int));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Per-device set-up state (host side).
struct NoallocDevice {
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch
  unsigned long long ctx = 0;      // unique id of the context the address was taken in
  int n = 0;                       // grid of the spectrum currently held (0: none)
  double h = 0.0, kb = 0.0;
  alignas(64) unsigned char tmap[128];
};
constexpr int NA_MAX_DEVICES = 64;
NoallocDevice g_devices[NA_MAX_DEVICES];
std::mutex g_mutex;

// Unique id of the calling thread's current context (driver entry points
// through the runtime's query, so the library does not link libcuda).  False
// when no context is current or the id cannot be read.  A device reset or a
// re-created primary context gets a new id, which sends the next call through
// the set-up again (the module, and with it the scratch array, may have moved).
bool current_context_id(unsigned long long* id) {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1 ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2)
      return false;
    get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
    get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

}  // namespace

extern "C" size_t mqnpm_noalloc_scratch_bytes(void) { return NA_BYTES; }

extern "C" int mqnpm_green_apply_noalloc(int n, double h, double kb, const float* v, float* out, int adjoint,
                                         void* stream) {
  if (n < 4 || n > NA_MAX_N || !green_supported(n)) {
    fprintf(stderr, "mqnpm_green_apply_noalloc: n = %d is outside the supported range (grid edge <= %d with a "
                    "compiled transform length 2n)\n", n, NA_MAX_N);
    return MQNPM_ERR_INVALID_ARG;
  }
  if (!v || !out || v == out || !(h > 0) || !(kb > 0)) return MQNPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return MQNPM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  NoallocDevice& d = g_devices[dev];
  unsigned long long ctx = 0;
  if (d.base == nullptr || !current_context_id(&ctx) || ctx != d.ctx) {
    // set-up of this device (first call, or a new context since the last one):
    // the device address of the scratch array, taken with the device current
    void* p = nullptr;
    d.base = nullptr;
    d.n = 0;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return MQNPM_ERR_CUDA;
    if (!current_context_id(&ctx)) return MQNPM_ERR_CUDA;
    d.base = static_cast<unsigned char*>(p);
    d.ctx = ctx;
  }
  float2* T1 = reinterpret_cast<float2*>(d.base + NA_T1);
  float2* T2 = reinterpret_cast<float2*>(d.base + NA_T2);
  float2* khat = reinterpret_cast<float2*>(d.base + NA_KH);
  float2* tw = reinterpret_cast<float2*>(d.base + NA_TW);
  int* err = reinterpret_cast<int*>(d.base + NA_ERR);
  if (d.n != n || d.h != h || d.kb != kb) {
    // set-up for this grid: spectrum, twiddles, tensor map of T2
    d.n = 0;
    const int P = 2 * n;
    std::vector<float2> twh(P);
    for (int j = 0; j < P; ++j) {
      const double a = 2.0 * M_PI * (double)j / (double)P;
      twh[j] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
    }
    if (cudaMemcpyAsync(tw, twh.data(), P * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
        build_khat_scratch(n, h, kb, khat, reinterpret_cast<double2*>(d.base + NA_KA),
                           reinterpret_cast<double2*>(d.base + NA_KB), reinterpret_cast<double*>(d.base + NA_COS),
                           s) != cudaSuccess ||
        make_t2_tensor_map(T2, n, n, n, 1, 0, d.tmap) != cudaSuccess)
      return MQNPM_ERR_CUDA;
    d.n = n;
    d.h = h;
    d.kb = kb;
  }
  GreenCall c;
  c.nx = c.ny = c.nz = n;
  c.nb = 1;
  c.adjoint = adjoint != 0;
  c.pro = PRO_PLAIN;
  c.pa.q = reinterpret_cast<const float2*>(v);
  c.epi = EPI_PLAIN;
  c.ea.out = reinterpret_cast<float2*>(out);
  c.T1 = T1;
  c.T2 = T2;
  c.khat = khat;
  c.twx = c.twy = c.twz = tw;
  c.tmap = d.tmap;
  c.err = err;
  if (green_launch(c, s) != cudaSuccess) return MQNPM_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MQNPM_ERR_CUDA;
  if (flag) {
    // the flag must start at zero for the next call
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return MQNPM_ERR_CUDA;
    return MQNPM_ERR_TIMEOUT;
  }
  return MQNPM_OK;
}
