// Quasi-Newton point of Algorithm 4.1 for k > S:
//   v_k = x - a S B^{-1} g,  B = tau* I + U U^T,
//   B^{-1} = tau*^{-1} I - tau*^{-2} U (I + U^T U / tau*)^{-1} U^T   (Woodbury, Section 4.3).
// One reduction pass forms U^T U and U^T g; a one-block kernel forms the S x S
// inverse; a last pass applies the low-rank correction.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

namespace {

constexpr int SM2 = MQNPM_MAX_S * MQNPM_MAX_S;
constexpr int OFF_G = 0;          // U^T U        (S x S, row stride S)
constexpr int OFF_M = SM2;        // (I + U^T U / tau)^{-1}
constexpr int OFF_UV = 2 * SM2;   // U^T g

template <int S>
MQ_D void block_reduce_store(float (&acc)[S], double* dst) {
  __shared__ double scratch[9 * S];   // 8 warps + totals
  double o[S];
  block_sum_f<S>(acc, scratch, o);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) dst[s] = o[s];
  }
}

// Partials of U^T U (upper triangle) and U^T g.
template <int S>
__global__ void k_gram(UPtrs U, const float* __restrict__ g, int N, double* part) {
  constexpr int NG = S * (S + 1) / 2;
  float acc[NG + S];
#pragma unroll
  for (int k = 0; k < NG + S; ++k) acc[k] = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    float u[S];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = U.u[s][i];
    int k = 0;
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int t = s; t < S; ++t) {
        acc[k] = fmaf(u[s], u[t], acc[k]);
        ++k;
      }
    const float gi = g[i];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[NG + s] = fmaf(u[s], gi, acc[NG + s]);
  }
  block_reduce_store<NG + S>(acc, part + (size_t)blockIdx.x * (NG + S));
}

// Reduce the partials; G, U^T g and M = (I + G/tau)^{-1} into scal.  One warp
// per reduced value (fixed order: deterministic); one Cholesky factorisation of
// I + G/tau, then one thread per column of M for the two triangular solves.
template <int S>
__global__ void k_gram_setup(const double* part, int nctas, double tau, double* scal) {
  constexpr int NG = S * (S + 1) / 2, NV = NG + S;
  __shared__ double tot[NV];
  __shared__ double A[S * S];
  __shared__ int ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ double rdiag[S];   // reciprocals of the factor's diagonal
  for (int k = warp; k < NV; k += nwarps) {
    // eight independent partial sums per lane keep eight loads in flight
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int c = lane;
    for (; c + 7 * 32 < nctas; c += 8 * 32) {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] += part[(size_t)(c + 32 * u) * NV + k];
    }
    for (int u = 0; c < nctas; c += 32, ++u) v[u & 7] += part[(size_t)c * NV + k];
    double t = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    t = warp_sum(t);
    if (lane == 0) tot[k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double inv_tau = 1.0 / tau;
    int k = 0;
    for (int a = 0; a < S; ++a)
      for (int b = a; b < S; ++b) {
        scal[OFF_G + a * S + b] = tot[k];
        scal[OFF_G + b * S + a] = tot[k];
        A[a * S + b] = A[b * S + a] = (a == b ? 1.0 : 0.0) + tot[k] * inv_tau;
        ++k;
      }
    for (int a = 0; a < S; ++a) scal[OFF_UV + a] = tot[NG + a];
    // lower Cholesky factor in place, one FP64 reciprocal per column (FP64
    // division is a long instruction sequence on this device)
    ok = 1;
    for (int j = 0; j < S; ++j) {
      double d = A[j * S + j];
      for (int q = 0; q < j; ++q) d -= A[j * S + q] * A[j * S + q];
      if (!(d > 0.0)) { ok = 0; break; }
      const double l = sqrt(d), rl = 1.0 / l;
      A[j * S + j] = l;
      rdiag[j] = rl;
      for (int i = j + 1; i < S; ++i) {
        double t = A[i * S + j];
        for (int q = 0; q < j; ++q) t -= A[i * S + q] * A[j * S + q];
        A[i * S + j] = t * rl;
      }
    }
  }
  __syncthreads();
  const int col = threadIdx.x;
  if (col < S) {
    double b[S];
    for (int i = 0; i < S; ++i) b[i] = (i == col) ? 1.0 : 0.0;
    if (ok) {
      for (int i = 0; i < S; ++i) {
        double t = b[i];
        for (int q = 0; q < i; ++q) t -= A[i * S + q] * b[q];
        b[i] = t * rdiag[i];
      }
      for (int i = S - 1; i >= 0; --i) {
        double t = b[i];
        for (int q = i + 1; q < S; ++q) t -= A[q * S + i] * b[q];
        b[i] = t * rdiag[i];
      }
    }
    for (int i = 0; i < S; ++i) scal[OFF_M + i * S + col] = b[i];
  }
}

// v = x - (aS/tau) g + (aS/tau^2) U M U^T g
template <int S>
__global__ void k_qn_point(const float* __restrict__ x, const float* __restrict__ g, UPtrs U, const double* scal,
                           double aS, double tau, float* __restrict__ v, int N) {
  __shared__ float coef[S];
  if (threadIdx.x < S) {
    double cs = 0.0;
    for (int t = 0; t < S; ++t) cs += scal[OFF_M + threadIdx.x * S + t] * scal[OFF_UV + t];
    coef[threadIdx.x] = (float)(aS / (tau * tau) * cs);
  }
  __syncthreads();
  const float a0 = (float)(aS / tau);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    float acc = fmaf(-a0, g[i], x[i]);
#pragma unroll
    for (int s = 0; s < S; ++s) acc = fmaf(coef[s], U.u[s][i], acc);
    v[i] = acc;
  }
}

template <int S>
cudaError_t qn_point(mqnpm_handle* h, const float* x, const float* g, const UPtrs& U, double tau, double aS, float* v) {
  cudaStream_t s = h->stream;
  const int ctas = h->wp.ctas_vec;
  k_gram<S><<<ctas, 256, 0, s>>>(U, g, (int)h->N, h->wp.gram);
  k_gram_setup<S><<<1, 256, 0, s>>>(h->wp.gram, ctas, tau, h->wp.scal);
  k_qn_point<S><<<ctas, 256, 0, s>>>(x, g, U, h->wp.scal, aS, tau, v, (int)h->N);
  h->launches += 3;
  return cudaGetLastError();
}

}  // namespace

int qn_point_impl(mqnpm_handle* h, const float* x, const float* g, const UPtrs& U, int S_eff, double tau,
                  double aS, float* v) {
  cudaError_t e;
  switch (S_eff) {
    case 1: e = qn_point<1>(h, x, g, U, tau, aS, v); break;
    case 2: e = qn_point<2>(h, x, g, U, tau, aS, v); break;
    case 3: e = qn_point<3>(h, x, g, U, tau, aS, v); break;
    case 4: e = qn_point<4>(h, x, g, U, tau, aS, v); break;
    case 5: e = qn_point<5>(h, x, g, U, tau, aS, v); break;
    case 6: e = qn_point<6>(h, x, g, U, tau, aS, v); break;
    case 7: e = qn_point<7>(h, x, g, U, tau, aS, v); break;
    case 8: e = qn_point<8>(h, x, g, U, tau, aS, v); break;
    case 9: e = qn_point<9>(h, x, g, U, tau, aS, v); break;
    case 10: e = qn_point<10>(h, x, g, U, tau, aS, v); break;
    case 11: e = qn_point<11>(h, x, g, U, tau, aS, v); break;
    case 12: e = qn_point<12>(h, x, g, U, tau, aS, v); break;
    case 13: e = qn_point<13>(h, x, g, U, tau, aS, v); break;
    case 14: e = qn_point<14>(h, x, g, U, tau, aS, v); break;
    case 15: e = qn_point<15>(h, x, g, U, tau, aS, v); break;
    case 16: e = qn_point<16>(h, x, g, U, tau, aS, v); break;
    default: return set_error(h, MQNPM_ERR_INVALID_ARG, "qn_point: S_eff out of range");
  }
  return e == cudaSuccess ? MQNPM_OK : set_cuda_error(h, e, "qn_point");
}

int woodbury_scal_count() { return 2 * SM2 + MQNPM_MAX_S; }
