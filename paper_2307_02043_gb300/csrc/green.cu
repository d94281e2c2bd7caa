// Dispatch of the Green's apply by transform length, and construction of the
// Green's kernel spectrum K_hat.
//
// Discretisation (our reading of the forward model of Section 6): with voxel h
// and background wavenumber kb,
//   (G v)_i = kb^2 sum_j w_{i-j} v_j,  offsets D in (-n, n)^3,
//   w_D = h^3 exp(j kb |D| h) / (4 pi |D| h) for D != 0,
//   w_0 = [exp(j kb a)(1 - j kb a) - 1] / kb^2, a = (3/(4 pi))^(1/3) h.
// On the periodic grid of edge P = 2n the kernel is even in every axis, so its
// DFT is a product of three 1D cosine sums over the first octant of offsets:
//   Kf(f) = k(0) + 2 sum_{d=1}^{n-1} k(d) cos(2 pi f d / P),  f = 0..n.
// These sums run in FP64 on the device; the result, scaled by 1/P^3 (the
// normalisation of the inverse transform), is rounded to complex64.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "green_passes.cuh"
#include "internal.h"
#include "mqnpm.h"

#define MQ_DISPATCH(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(320) X(384)

bool green_supported(int n) {
  switch (2 * n) {
#define MQ_CASE(P) case P:
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    return true;
    default:
      return false;
  }
}

void green_shape(int n, int tile, int* shape, size_t* smem) {
  for (int i = 0; i < 6; ++i) shape[i] = 0;
  size_t m = 0;
  switch (2 * n) {
#define MQ_CASE(P) case P: green_shape_P##P(tile, n, shape, &m); break;
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default:
      break;
  }
  if (smem) *smem = m;
}

bool green_tile_fits(int n, int tile, int device) {
  int shape[6], optin = 0;
  size_t smem = 0;
  green_shape(n, tile, shape, &smem);
  if (shape[0] <= 0 || cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
    return false;
  return smem <= (size_t)optin;
}

int green_row_ctas(int n, int tile) {
  int shape[6];
  green_shape(n, tile, shape);
  return shape[0] > 0 ? (n * n + shape[0] - 1) / shape[0] : 0;
}

int green_plane_ctas(int n, int tile) {
  int shape[6];
  green_shape(n, tile, shape);
  return shape[0] > 0 ? (n + shape[0] - 1) / shape[0] : 0;
}

int green_row_ctas_max(int n) { return std::max(green_row_ctas(n, 0), green_row_ctas(n, 1)); }

int green_col_width(int n, int tile) {   // columns per CTA of pass 3 (the tensor-map box)
  int shape[6];
  green_shape(n, tile, shape);
  return shape[4];
}

cudaError_t green_launch(const GreenCall& c, cudaStream_t s) {
  switch (2 * c.n) {
#define MQ_CASE(P) case P: return green_launch_P##P(c, s);
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------- T2 tensor map
// T2 viewed as a 3D tensor of 8-byte elements: x = kx (P), y = ky (P),
// z = slot * n + z (max_batch * n).  Pass 3 loads boxes of C x 1 x n: one
// column set of one slot.  The encoder comes from the driver through the
// runtime's entry-point query, so the library does not link libcuda.
cudaError_t make_t2_tensor_map(void* T2, int n, int max_batch, int tile, void* map_out) {
  const int P = 2 * n;
  const int C = green_col_width(n, tile);
  if (C <= 0) return cudaErrorInvalidValue;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)P, (cuuint64_t)max_batch * n};
  const cuuint64_t strides[2] = {(cuuint64_t)P * 8, (cuuint64_t)P * P * 8};
  const cuuint32_t box[3] = {(cuuint32_t)C, 1u, (cuuint32_t)n};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, T2, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ------------------------------------------------------------ K_hat build
// k[dz][dy][dx] for offsets in [0, n)^3 (FP64 complex as double2).
__global__ void k_kernel_octant(double2* k, int n, double h, double kb) {
  const long long N = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int dx = (int)(i % n), dy = (int)((i / n) % n), dz = (int)(i / ((long long)n * n));
    double re, im;
    if (dx == 0 && dy == 0 && dz == 0) {
      const double a = cbrt(3.0 / (4.0 * 3.14159265358979323846)) * h;
      double s, c;
      sincos(kb * a, &s, &c);
      // exp(j kb a) (1 - j kb a) - 1, divided by kb^2, times kb^2
      re = (c + kb * a * s) - 1.0;
      im = s - kb * a * c;
    } else {
      const double r = h * sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz);
      double s, c;
      sincos(kb * r, &s, &c);
      const double f = kb * kb * h * h * h / (4.0 * 3.14159265358979323846 * r);
      re = f * c;
      im = f * s;
    }
    k[i] = make_double2(re, im);
  }
}

// One separable even-sum pass along the fastest axis of `in` (extent n, the
// offsets), writing extent m = n+1 (the folded frequencies) as the *slowest*
// axis of `out`, so three passes rotate the axes back to [fz][fy][fx].
//   in : [a][b][d]  (d < n)      out: [f][a][b]  (f <= n)
__global__ void k_cos_pass(const double2* __restrict__ in, double2* __restrict__ out, int A, int B, int n,
                           const double* __restrict__ cosP, int P) {
  const long long total = (long long)(n + 1) * A * B;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int bb = (int)(i % B);
    const int aa = (int)((i / B) % A);
    const int f = (int)(i / ((long long)A * B));
    const double2* row = in + ((long long)aa * B + bb) * n;
    double re = row[0].x, im = row[0].y;
    for (int d = 1; d < n; ++d) {
      const double c = 2.0 * cosP[(long long)f * d % P];
      re += c * row[d].x;
      im += c * row[d].y;
    }
    out[i] = make_double2(re, im);
  }
}

__global__ void k_round_khat(const double2* __restrict__ in, float2* __restrict__ out, long long M, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)(in[i].x * scale), (float)(in[i].y * scale));
}

// The same construction with caller-provided device scratch: a, b hold
// (n+1)^3 double2 each, dcos holds P doubles.  No device allocation.
cudaError_t build_khat_scratch(int n, double h, double kb, float2* khat_out, double2* a, double2* b, double* dcos,
                               cudaStream_t s) {
  const int P = 2 * n;
  const long long m = n + 1;
  std::vector<double> cosv(P);
  for (int j = 0; j < P; ++j) cosv[j] = std::cos(2.0 * M_PI * (double)j / (double)P);
  cudaError_t e = cudaMemcpyAsync(dcos, cosv.data(), P * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int th = 256, gr = 1024;
  k_kernel_octant<<<gr, th, 0, s>>>(a, n, h, kb);
  k_cos_pass<<<gr, th, 0, s>>>(a, b, n, n, n, dcos, P);
  k_cos_pass<<<gr, th, 0, s>>>(b, a, (int)m, n, n, dcos, P);
  k_cos_pass<<<gr, th, 0, s>>>(a, b, (int)m, (int)m, n, dcos, P);
  k_round_khat<<<gr, th, 0, s>>>(b, khat_out, m * m * m, 1.0 / ((double)P * P * P));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host cosine table goes out of scope
  return e;
}

// ------------------------------------------------ truncated Green's kernel
// Transform of g_R(r) = exp(j kb r)/(4 pi r) 1[r <= R] at radial frequency s
// (Vico, Greengard and Ferrando, J. Comput. Phys. 2016).  With q = kb:
//   g_R^(s) = [-1 + e^{jqR}(cos sR - j q sin(sR)/s)] / (q^2 - s^2).
// Near s = q numerator and denominator both vanish; splitting
// e^{jqR} cos sR and e^{jqR} sin sR into e^{j(q+s)R} and e^{j(q-s)R} gives the
// cancellation-free form used for s >= q/2:
//   g_R^(s) = (1 - e^{j(q+s)R}) / (2s(q+s)) + (R/(2s)) [-(t/2) sinc^2(t/2) + j sinc(t)],
// t = (q - s)R, sinc(t) = sin(t)/t.  Below q/2 the rational form has no
// cancellation; s = 0 takes its limit (e^{jqR}(1 - jqR) - 1)/q^2.
__device__ double sinc_d(double t) { return t == 0.0 ? 1.0 : sin(t) / t; }

__device__ double2 truncated_ft(double s, double q, double R) {
  double sq, cq;
  sincos(q * R, &sq, &cq);
  if (s == 0.0) {
    // (cos qR + j sin qR)(1 - j qR) - 1
    const double re = cq + q * R * sq - 1.0, im = sq - q * R * cq;
    return make_double2(re / (q * q), im / (q * q));
  }
  if (s < 0.5 * q) {
    double ss, cs;
    sincos(s * R, &ss, &cs);
    const double br = cs, bi = -q * ss / s;               // cos sR - j q sin(sR)/s
    const double re = cq * br - sq * bi - 1.0, im = cq * bi + sq * br;
    const double den = q * q - s * s;
    return make_double2(re / den, im / den);
  }
  double sp, cp;
  sincos((q + s) * R, &sp, &cp);
  const double a = 1.0 / (2.0 * s * (q + s));
  const double t = (q - s) * R;
  const double sh = sinc_d(0.5 * t);
  const double b = R / (2.0 * s);
  return make_double2((1.0 - cp) * a - b * 0.5 * t * sh * sh, -sp * a + b * sinc_d(t));
}

// spec[mz][my][mx] = g_R^(ds |m|) for m in [0, M)^3 (M = 2n + 1: the folded
// frequencies of the period T = 4n, the transform being radial).
__global__ void k_truncated_spectrum(double2* spec, int M, double ds, double kb, double R) {
  const long long total = (long long)M * M * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int mx = (int)(i % M), my = (int)((i / M) % M), mz = (int)(i / ((long long)M * M));
    const double s = ds * sqrt((double)mx * mx + (double)my * my + (double)mz * mz);
    spec[i] = truncated_ft(s, kb, R);
  }
}

// One even inverse-DFT pass of period T over the fastest axis of `in`
// (extent M = T/2 + 1, the folded frequencies), keeping offsets d < n, written
// as the slowest axis of `out`:  out[d][a][b] = sum_m c_m cos(2 pi m d / T) in[a][b][m],
// c_0 = c_{T/2} = 1, else 2.   in: [A][B][M]   out: [n][A][B]
__global__ void k_even_idft_pass(const double2* __restrict__ in, double2* __restrict__ out, int A, int B, int M,
                                 int n, const double* __restrict__ cosT, int T) {
  const long long total = (long long)n * A * B;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int bb = (int)(i % B);
    const int aa = (int)((i / B) % A);
    const int d = (int)(i / ((long long)A * B));
    const double2* row = in + ((long long)aa * B + bb) * M;
    double re = row[0].x + (d % 2 == 0 ? 1.0 : -1.0) * row[M - 1].x;   // m = T/2: cos(pi d)
    double im = row[0].y + (d % 2 == 0 ? 1.0 : -1.0) * row[M - 1].y;
    int j = d;   // (m d) mod T, stepped
    for (int m = 1; m < M - 1; ++m) {
      const double c = 2.0 * cosT[j];
      re += c * row[m].x;
      im += c * row[m].y;
      j += d;
      if (j >= T) j -= T;
    }
    out[i] = make_double2(re, im);
  }
}

__global__ void k_scale_d2(double2* a, long long count, double sc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    a[i] = make_double2(a[i].x * sc, a[i].y * sc);
}

// Real-space octant kb^2 w_D, D in [0, n)^3, of the truncated kernel into `a`
// ([dz][dy][dx]), from its transform sampled on the frequency grid of period
// T = 4n h and R = sqrt(3) n h: w_D = (1/T^3) sum_m g_R^(|s_m|) e^{j s_m . D h}
// (three even passes), times kb^2.  b: scratch; both hold (2n+1)^3 double2.
cudaError_t truncated_octant(int n, double h, double kb, double2* a, double2* b, double* dcosT, cudaStream_t s) {
  const int T = 4 * n, M = 2 * n + 1;
  const double R = std::sqrt(3.0) * n * h;
  std::vector<double> cosv(T);
  for (int j = 0; j < T; ++j) cosv[j] = std::cos(2.0 * M_PI * (double)j / (double)T);
  cudaError_t e = cudaMemcpyAsync(dcosT, cosv.data(), T * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int th = 256, gr = 2048;
  k_truncated_spectrum<<<gr, th, 0, s>>>(b, M, 2.0 * M_PI / (T * h), kb, R);   // b: [mz][my][mx]
  k_even_idft_pass<<<gr, th, 0, s>>>(b, a, M, M, M, n, dcosT, T);             // a: [dx][mz][my]
  k_even_idft_pass<<<gr, th, 0, s>>>(a, b, n, M, M, n, dcosT, T);             // b: [dy][dx][mz]
  k_even_idft_pass<<<gr, th, 0, s>>>(b, a, n, n, M, n, dcosT, T);             // a: [dz][dy][dx]
  k_scale_d2<<<gr, th, 0, s>>>(a, (long long)n * n * n, kb * kb / ((double)T * T * T));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host cosine table goes out of scope
  return e;
}

cudaError_t build_khat(int n, double h, double kb, float2* khat_out, cudaStream_t s, int kernel) {
  const int P = 2 * n;
  const long long m = n + 1;
  std::vector<double> cosv(P);
  for (int j = 0; j < P; ++j) cosv[j] = std::cos(2.0 * M_PI * (double)j / (double)P);
  double2 *a = nullptr, *b = nullptr;
  double* dcos = nullptr;
  const long long M = 2 * n + 1;
  const size_t big = kernel == MQNPM_KERNEL_TRUNCATED ? (size_t)M * M * M : (size_t)m * m * m;
  cudaError_t e;
  if ((e = cudaMallocAsync(&a, big * sizeof(double2), s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&b, big * sizeof(double2), s)) != cudaSuccess) { cudaFreeAsync(a, s); return e; }
  if ((e = cudaMallocAsync(&dcos, 4 * (size_t)n * sizeof(double), s)) != cudaSuccess) { cudaFreeAsync(a, s); cudaFreeAsync(b, s); return e; }
  if (kernel == MQNPM_KERNEL_TRUNCATED) e = truncated_octant(n, h, kb, a, b, dcos, s);   // a: [dz][dy][dx]
  if (e == cudaSuccess) e = cudaMemcpyAsync(dcos, cosv.data(), P * sizeof(double), cudaMemcpyHostToDevice, s);
  const int th = 256, gr = 1024;
  if (e == cudaSuccess) {
    if (kernel != MQNPM_KERNEL_TRUNCATED) k_kernel_octant<<<gr, th, 0, s>>>(a, n, h, kb);   // a: [dz][dy][dx]
    k_cos_pass<<<gr, th, 0, s>>>(a, b, n, n, n, dcos, P);             // b: [fx][dz][dy]
    k_cos_pass<<<gr, th, 0, s>>>(b, a, (int)m, n, n, dcos, P);        // a: [fy][fx][dz]
    k_cos_pass<<<gr, th, 0, s>>>(a, b, (int)m, (int)m, n, dcos, P);   // b: [fz][fy][fx]
    k_round_khat<<<gr, th, 0, s>>>(b, khat_out, m * m * m, 1.0 / ((double)P * P * P));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host cosine table goes out of scope
  }
  cudaFreeAsync(a, s);
  cudaFreeAsync(b, s);
  cudaFreeAsync(dcos, s);
  return e;
}

// A caller-provided spectrum: the first octant [fz][fy][fx] of the
// unnormalised DFT_P, complex64 on the host.  Scaled by 1/P^3 in FP64 and
// rounded once, like the library's own construction.
cudaError_t upload_khat(const float* host, int n, float2* khat_out, cudaStream_t s) {
  const int P = 2 * n;
  const size_t big = (size_t)(n + 1) * (n + 1) * (n + 1);
  const double scale = 1.0 / ((double)P * P * P);
  std::vector<float2> v(big);
  for (size_t i = 0; i < big; ++i) {
    const double re = host[2 * i], im = host[2 * i + 1];
    v[i] = make_float2((float)(re * scale), (float)(im * scale));
  }
  cudaError_t e = cudaMemcpyAsync(khat_out, v.data(), big * sizeof(float2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the staging vector goes out of scope
  return e;
}
