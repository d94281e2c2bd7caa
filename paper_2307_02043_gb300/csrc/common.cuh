// Shared device helpers for the MQNPM hot path (sm_103a).
//
// Complex64 arithmetic on float2, compile-time twiddle factors, deterministic
// block reductions into FP64 partials, and a grid barrier with a bounded wait
// for cooperative (co-resident) launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>
#include <type_traits>

#define MQ_HD __host__ __device__ __forceinline__
#define MQ_D __device__ __forceinline__

// ---------------------------------------------------------------- complex64
MQ_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
MQ_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
MQ_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
MQ_HD float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// A rounded product that the compiler never contracts into a following add
// (the first butterflies of the prologue's transform): every kernel that
// scales by the contrast then rounds the same way.
MQ_HD float2 cscale(float2 a, float s) {
#ifdef __CUDA_ARCH__
  return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
#else
  return make_float2(a.x * s, a.y * s);
#endif
}
MQ_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a + s * b (s complex)
MQ_HD float2 caxpy(float2 s, float2 b, float2 a) {
  return make_float2(fmaf(s.x, b.x, fmaf(-s.y, b.y, a.x)), fmaf(s.x, b.y, fmaf(s.y, b.x, a.y)));
}
MQ_HD float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ---------------------------------------------------- compile-time sin / cos
// Twiddle factors of the in-register DFTs are evaluated by the compiler from
// Taylor series (angle reduced to |t| <= pi/4 by octant symmetry), so they
// become immediates; no runtime table and no device math library call.
namespace ctrig {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double sin_series(double t) {
  double term = t, sum = t;
  for (int i = 1; i < 16; ++i) {
    term *= -t * t / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double cos_series(double t) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 16; ++i) {
    term *= -t * t / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
// cos and sin of 2*pi*j/R, exact reduction on the rational angle j/R.
// Octant o = floor(8 j / R) and remainder give |t| <= pi/4.
struct CS { double c, s; };
constexpr CS cs_turn(long j, long R) {
  j %= R;
  if (j < 0) j += R;
  // angle = 2*pi*j/R = (pi/4) * (8j/R); split 8j = o*R + rem.
  long o = (8 * j) / R;
  long rem = 8 * j - o * R;            // 0 <= rem < R
  // t in [0, pi/4): base angle within the octant
  double t = (kPi / 4.0) * static_cast<double>(rem) / static_cast<double>(R);
  double c0 = cos_series(t), s0 = sin_series(t);
  // rotate by o * pi/4
  const double h = 0.70710678118654752440084436210484903928;  // sqrt(2)/2
  double c = c0, s = s0;
  switch (o) {
    case 0: c = c0; s = s0; break;
    case 1: c = h * (c0 - s0); s = h * (c0 + s0); break;
    case 2: c = -s0; s = c0; break;
    case 3: c = -h * (c0 + s0); s = h * (c0 - s0); break;
    case 4: c = -c0; s = -s0; break;
    case 5: c = -h * (c0 - s0); s = -h * (c0 + s0); break;
    case 6: c = s0; s = -c0; break;
    default: c = h * (c0 + s0); s = -h * (c0 - s0); break;
  }
  return CS{c, s};
}
}  // namespace ctrig

// ------------------------------------------------------------- static loops
template <class F, int... I>
MQ_D void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
MQ_D void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// -------------------------------------------------------------- reductions
MQ_D double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
MQ_D float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum K doubles over the block (blockDim.x a multiple of 32, <= 1024) in a
// fixed order; thread 0 receives the totals in out[]. scratch: >= 32*K doubles.
template <int K>
MQ_D void block_sum(double (&v)[K], double* scratch, double (&out)[K]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[warp * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += scratch[w * K + k];
      out[k] = s;
    }
  }
  __syncthreads();
}

// Sum K per-thread float partials over the block: the warp tree runs in FP32
// (GB300's FP64 rate is a small fraction of its FP32 rate), the per-warp
// results are combined in FP64 in warp order.  Thread 0 receives out[].
// scratch: >= (warps + 1) * K doubles (33 * K covers any block size).
template <int K>
MQ_D void block_sum_f(const float (&v)[K], double* scratch, double (&out)[K]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float w = warp_sumf(v[k]);
    if (lane == 0) scratch[warp * K + k] = (double)w;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += scratch[w * K + k];
    scratch[nw * K + k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = scratch[nw * K + k];
  }
  __syncthreads();
}

// Acquire load of a flag written with a release store by another block.
MQ_D unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// ------------------------------------------------------- TMA and mbarriers
// Tensor-memory-accelerator tile loads into shared memory, completed on an
// mbarrier (transaction count = bytes).  Waits are bounded: the caller gets
// `false` after `limit` polls and must report the failure instead of hanging.
MQ_D uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
MQ_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make mbarrier initialisation visible to the async (TMA) proxy
MQ_D void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
MQ_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
MQ_D void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
MQ_D bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
MQ_D bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 3D tile load: box origin (x, y, z) in elements; x * element size must be a
// multiple of 16 bytes (callers pass tile-aligned x).
MQ_D void tma_load_3d(void* dst, const void* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// ----------------------------------------------------------------- helpers
MQ_HD int ceil_div(int a, int b) { return (a + b - 1) / b; }
MQ_HD long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }
