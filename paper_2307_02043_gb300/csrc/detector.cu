// Remote detector: the last z-slice of the scattered field carried a distance
// d further along z by the angular spectrum with a pupil (Section 6, remote
// detector reading):  D = F^-1 diag(H) F,  H = exp(j kz d) 1[kx^2 + ky^2 <= (na kb)^2],
// kz = sqrt(kb^2 - kx^2 - ky^2) (Im kz >= 0), F the 2D DFT of the ny x nx slice.
// The adjoint D^H uses conj(H).  The table holds H / (nx ny), so both
// directions are four unnormalised 1D DFT passes over the [b][y][x] slices:
// x forward, y forward, y inverse with the multiplier applied on load, x inverse.
//
// A slice is nx ny complex values (128 KB at 128 x 128) against the volumes of
// the solves, so the passes are plain per-line DFT sums (one thread per
// output, the twiddle index advanced incrementally), not the pruned FFT machinery.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

// out[line][k] = sum_j in[line][j] * W_len^{+-jk} (* mult[.] on load) on
// [ny][nx] slices: lines along x (the ny rows, length nx, contiguous) or
// along y (the nx columns, length ny, stride nx); grid (lines, slots); tw
// holds W_len^j, j < len.
template <bool ALONG_Y, bool INV>
__global__ void k_dft_lines(const float2* __restrict__ in, float2* __restrict__ out, int nx, int ny,
                            const float2* __restrict__ tw, const float2* __restrict__ mult, int conj_mult) {
  extern __shared__ float2 sm[];
  const int n = ALONG_Y ? ny : nx;   // line length
  float2* line = sm;
  float2* tws = sm + n;
  const int ln = blockIdx.x;
  const size_t M = (size_t)nx * ny;
  const float2* src = in + (size_t)blockIdx.y * M;
  float2* dst = out + (size_t)blockIdx.y * M;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const size_t e = ALONG_Y ? (size_t)j * nx + ln : (size_t)ln * nx + j;
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
    const size_t e = ALONG_Y ? (size_t)k * nx + ln : (size_t)ln * nx + k;
    dst[e] = make_float2(re, im);
  }
}

// r = y_prop - y_meas(l) (or y_prop without measurements) and the per-CTA
// partial ||r||^2, laid out like the near-field detector's partials.
__global__ void k_det_finish(const float2* __restrict__ yprop, const float2* __restrict__ ymeas,
                             const int* __restrict__ illum, float2* __restrict__ out, size_t M,
                             double* __restrict__ part) {
  const int b = blockIdx.y;
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
  const int nx = h->nx, ny = h->ny, nmax = nx > ny ? nx : ny;
  const int th = nmax < 256 ? ((nmax + 31) / 32) * 32 : 256;
  const size_t smem = 2 * (size_t)nmax * sizeof(float2);
  const dim3 gx(ny, m), gy(nx, m);   // rows along x, columns along y
  const float2* twx = h->twn;        // W_nx^j
  const float2* twy = h->twn + nx;   // W_ny^j
  cudaStream_t s = h->stream;
  k_dft_lines<false, false><<<gx, th, smem, s>>>(in, w.dtmp1, nx, ny, twx, nullptr, 0);
  k_dft_lines<true, false><<<gy, th, smem, s>>>(w.dtmp1, w.dtmp2, nx, ny, twy, nullptr, 0);
  k_dft_lines<true, true><<<gy, th, smem, s>>>(w.dtmp2, w.dtmp1, nx, ny, twy, h->Hdet, adjoint ? 1 : 0);
  k_dft_lines<false, true><<<gx, th, smem, s>>>(w.dtmp1, out, nx, ny, twx, nullptr, 0);
  h->launches += 4;
  return cudaGetLastError();
}

}  // namespace

cudaError_t detector_tables(mqnpm_handle* h, double distance, double na) {
  const int nx = h->nx, ny = h->ny;
  const double kb = h->kb, hh = h->h;
  std::vector<float2> twn(nx + ny), H((size_t)nx * ny);
  for (int j = 0; j < nx; ++j) {
    const double a = 2.0 * M_PI * (double)j / (double)nx;
    twn[j] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
  }
  for (int j = 0; j < ny; ++j) {
    const double a = 2.0 * M_PI * (double)j / (double)ny;
    twn[nx + j] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
  }
  const double inv = 1.0 / ((double)nx * ny), kmax2 = (na * kb) * (na * kb);
  for (int fy = 0; fy < ny; ++fy)
    for (int fx = 0; fx < nx; ++fx) {
      const int sy = fy < (ny + 1) / 2 ? fy : fy - ny, sx = fx < (nx + 1) / 2 ? fx : fx - nx;   // DFT frequency order
      const double ky = 2.0 * M_PI * sy / (ny * hh), kx = 2.0 * M_PI * sx / (nx * hh);
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
      H[(size_t)fy * nx + fx] = make_float2((float)(re * inv), (float)(im * inv));
    }
  cudaError_t e = cudaMemcpyAsync(h->twn, twn.data(), twn.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->Hdet, H.data(), H.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host tables go out of scope
  return e;
}

cudaError_t detector_forward(mqnpm_handle* h, float2* det, int m, const float2* ym, const int* illum) {
  cudaError_t e = four_passes(h, det, h->w.dtmp2, m, false);
  if (e != cudaSuccess) return e;
  k_det_finish<<<dim3(h->w.ctas_row, m), 256, 0, h->stream>>>(h->w.dtmp2, ym, illum, det, (size_t)h->M, h->w.partd);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t detector_adjoint(mqnpm_handle* h, const float2* r, float2* out, int m) {
  return four_passes(h, r, out, m, true);
}
