// Remote detector: the last z-slice of the scattered field carried a distance
// d further along z by the angular spectrum with a pupil (Section 6, remote
// detector reading):  D = F^-1 diag(H) F,  H = exp(j kz d) 1[kx^2 + ky^2 <= (na kb)^2],
// kz = sqrt(kb^2 - kx^2 - ky^2) (Im kz >= 0), F the 2D DFT of the n x n slice.
// The adjoint D^H uses conj(H).  The table holds H / n^2, so both directions
// are four unnormalised 1D DFT passes over the [b][y][x] slices: x forward,
// y forward, y inverse with the multiplier applied on load, x inverse.
//
// A slice is n^2 complex values (128 KB at n = 128) against the n^3 volumes of
// the solves, so the passes are plain per-line DFT sums (n threads per line,
// the twiddle index advanced incrementally), not the pruned FFT machinery.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

// out[line][k] = sum_j in[line][j] * W_n^{+-jk} (* mult[.] on load), lines
// along x (rows, contiguous) or along y (columns, stride n); grid (n lines, slots).
template <bool ALONG_Y, bool INV>
__global__ void k_dft_lines(const float2* __restrict__ in, float2* __restrict__ out, int n,
                            const float2* __restrict__ tw, const float2* __restrict__ mult, int conj_mult) {
  extern __shared__ float2 sm[];
  float2* line = sm;
  float2* tws = sm + n;
  const int ln = blockIdx.x;
  const size_t M = (size_t)n * n;
  const float2* src = in + (size_t)blockIdx.y * M;
  float2* dst = out + (size_t)blockIdx.y * M;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const size_t e = ALONG_Y ? (size_t)j * n + ln : (size_t)ln * n + j;
    float2 v = src[e];
    if (mult) {
      float2 m = mult[e];
      if (conj_mult) m.y = -m.y;
      v = cmul(v, m);
    }
    line[j] = v;
    tws[j] = tw[j];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    float re = 0.f, im = 0.f;
    int idx = 0;   // j k mod n
    for (int j = 0; j < n; ++j) {
      const float2 a = line[j], w = tws[idx];
      const float wy = INV ? -w.y : w.y;
      re = fmaf(a.x, w.x, fmaf(-a.y, wy, re));
      im = fmaf(a.x, wy, fmaf(a.y, w.x, im));
      idx += k;
      if (idx >= n) idx -= n;
    }
    const size_t e = ALONG_Y ? (size_t)k * n + ln : (size_t)ln * n + k;
    dst[e] = make_float2(re, im);
  }
}

// r = y_prop - y_meas(l) (or y_prop without measurements) and the per-CTA
// partial ||r||^2, laid out like the near-field detector's partials.
__global__ void k_det_finish(const float2* __restrict__ yprop, const float2* __restrict__ ymeas,
                             const int* __restrict__ illum, float2* __restrict__ out, int n, double* __restrict__ part) {
  const int b = blockIdx.y;
  const size_t M = (size_t)n * n;
  float acc = 0.f;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < M; j += (size_t)gridDim.x * blockDim.x) {
    float2 r = yprop[(size_t)b * M + j];
    if (ymeas) r = csub(r, ymeas[(size_t)illum[b] * M + j]);
    out[(size_t)b * M + j] = r;
    acc += cabs2(r);
  }
  __shared__ double scratch[33];
  const float v[1] = {acc};
  double o[1];
  block_sum_f<1>(v, scratch, o);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = o[0];
}

cudaError_t four_passes(mqnpm_handle* h, const float2* in, float2* out, int m, bool adjoint) {
  Workspace& w = h->w;
  const int n = h->n;
  const int th = n < 256 ? ((n + 31) / 32) * 32 : 256;
  const size_t smem = 2 * (size_t)n * sizeof(float2);
  const dim3 grid(n, m);
  cudaStream_t s = h->stream;
  k_dft_lines<false, false><<<grid, th, smem, s>>>(in, w.dtmp1, n, h->twn, nullptr, 0);
  k_dft_lines<true, false><<<grid, th, smem, s>>>(w.dtmp1, w.dtmp2, n, h->twn, nullptr, 0);
  k_dft_lines<true, true><<<grid, th, smem, s>>>(w.dtmp2, w.dtmp1, n, h->twn, h->Hdet, adjoint ? 1 : 0);
  k_dft_lines<false, true><<<grid, th, smem, s>>>(w.dtmp1, out, n, h->twn, nullptr, 0);
  h->launches += 4;
  return cudaGetLastError();
}

}  // namespace

cudaError_t detector_tables(mqnpm_handle* h, double distance, double na) {
  const int n = h->n;
  const double kb = h->kb, hh = h->h;
  std::vector<float2> twn(n), H((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    const double a = 2.0 * M_PI * (double)j / (double)n;
    twn[j] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
  }
  const double inv = 1.0 / ((double)n * n), kmax2 = (na * kb) * (na * kb);
  for (int fy = 0; fy < n; ++fy)
    for (int fx = 0; fx < n; ++fx) {
      const int sy = fy < (n + 1) / 2 ? fy : fy - n, sx = fx < (n + 1) / 2 ? fx : fx - n;   // DFT frequency order
      const double ky = 2.0 * M_PI * sy / (n * hh), kx = 2.0 * M_PI * sx / (n * hh);
      const double k2 = kx * kx + ky * ky;
      double re = 0.0, im = 0.0;
      if (k2 <= kmax2) {
        const double q = kb * kb - k2;
        if (q >= 0.0) {   // propagating: exp(j kz d)
          const double ph = std::sqrt(q) * distance;
          re = std::cos(ph);
          im = std::sin(ph);
        } else {          // evanescent: kz = j sqrt(-q), exp(-sqrt(-q) d)
          re = std::exp(-std::sqrt(-q) * distance);
        }
      }
      H[(size_t)fy * n + fx] = make_float2((float)(re * inv), (float)(im * inv));
    }
  cudaError_t e = cudaMemcpyAsync(h->twn, twn.data(), n * sizeof(float2), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->Hdet, H.data(), H.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host tables go out of scope
  return e;
}

cudaError_t detector_forward(mqnpm_handle* h, float2* det, int m, const float2* ym, const int* illum) {
  cudaError_t e = four_passes(h, det, h->w.dtmp2, m, false);
  if (e != cudaSuccess) return e;
  k_det_finish<<<dim3(h->w.ctas_row, m), 256, 0, h->stream>>>(h->w.dtmp2, ym, illum, det, h->n, h->w.partd);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t detector_adjoint(mqnpm_handle* h, const float2* r, float2* out, int m) {
  return four_passes(h, r, out, m, true);
}
