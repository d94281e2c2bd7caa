// Dispatch of the Green's apply by transform length, and construction of the
// Green's kernel spectrum K_hat.
//
// Discretisation (our reading of the forward model of Section 6): with voxel h
// and background wavenumber kb,
//   (G v)_i = kb^2 sum_j w_{i-j} v_j,  offsets D in (-nx, nx) x (-ny, ny) x (-nz, nz),
//   w_D = h^3 exp(j kb |D| h) / (4 pi |D| h) for D != 0,
//   w_0 = [exp(j kb a)(1 - j kb a) - 1] / kb^2, a = (3/(4 pi))^(1/3) h
// (or the truncated kernel below).  On the periodic grid of edges P_d = 2 n_d
// the kernel is even in every axis, so its DFT is a product of three 1D cosine
// sums over the first octant of offsets:
//   Kf(f) = k(0) + 2 sum_{d=1}^{n-1} k(d) cos(2 pi f d / P),  f = 0..n, per axis.
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

bool green_fused_supported(int nx, int ny) { return nx == ny && (2 * nx == 128 || 2 * nx == 256); }

namespace {

size_t fused_smem(int n) {
  switch (2 * n) {
    case 128: return green_fused_smem_P128();
    case 256: return green_fused_smem_P256();
    default: return 0;
  }
}

// The shape fields and shared memory of one length's passes.
bool shape_of(int n, int tile, int* shape, size_t* srow, size_t* scol, size_t* sz) {
  switch (2 * n) {
#define MQ_CASE(P) case P: green_shape_P##P(tile & 15, shape, srow, scol, sz); return true;
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default:
      return false;
  }
}

}  // namespace

void green_shape(int nx, int ny, int nz, int tile, int* shape, size_t* smem) {
  for (int i = 0; i < 6; ++i) shape[i] = 0;
  if (smem) *smem = 0;
  // the fused x/y passes exist for square planes of the default row shape;
  // their plane-input and plane-output applies use the unfused passes
  if ((tile & MQ_TILE_FUSED) && (!green_fused_supported(nx, ny) || (tile & 3) != 0)) return;
  int sx[6], sy[6], sz[6];
  size_t rx, cx, zx, ry, cy, zy, rz, cz, zz;
  if (!shape_of(nx, tile, sx, &rx, &cx, &zx) || !shape_of(ny, tile, sy, &ry, &cy, &zy) ||
      !shape_of(nz, tile, sz, &rz, &cz, &zz))
    return;
  shape[0] = sx[0];   // x passes: length Px
  shape[1] = sx[1];
  shape[2] = sy[2];   // y passes: length Py
  shape[3] = sy[3];
  shape[4] = sz[4];   // z pass: length Pz
  shape[5] = sz[5];
  if (smem) *smem = std::max(rx, std::max(cy, zz));
  if (smem && (tile & MQ_TILE_FUSED)) *smem = std::max(*smem, fused_smem(nx));
}

bool green_tile_fits(int nx, int ny, int nz, int tile, int device) {
  int shape[6], optin = 0;
  size_t smem = 0;
  green_shape(nx, ny, nz, tile, shape, &smem);
  if (shape[0] <= 0 || cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
    return false;
  return smem <= (size_t)optin;
}

int green_row_ctas(int nx, int ny, int nz, int tile) {
  int shape[6];
  green_shape(nx, ny, nz, tile, shape);
  return shape[0] > 0 ? (ny * nz + shape[0] - 1) / shape[0] : 0;
}

int green_plane_ctas(int nx, int ny, int tile) {
  int shape[6];
  green_shape(nx, ny, nx, tile, shape);   // the x-pass shape depends on nx only
  return shape[0] > 0 ? (ny + shape[0] - 1) / shape[0] : 0;
}

int green_row_ctas_max(int nx, int ny, int nz) {
  return std::max(green_row_ctas(nx, ny, nz, 0), green_row_ctas(nx, ny, nz, 1));
}

int green_col_width(int nx, int ny, int nz, int tile) {   // columns per CTA of pass 3 (the tensor-map box)
  int shape[6];
  green_shape(nx, ny, nz, tile, shape);
  return shape[4];
}

namespace {

cudaError_t pass1_any(const GreenCall& c, cudaStream_t s) {
  switch (2 * c.nx) {
#define MQ_CASE(P) case P: return green_pass1_P##P(c, s);
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t pass5_any(const GreenCall& c, cudaStream_t s) {
  switch (2 * c.nx) {
#define MQ_CASE(P) case P: return green_pass5_P##P(c, s);
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t passy_any(const GreenCall& c, bool inv, cudaStream_t s) {
  switch (2 * c.ny) {
#define MQ_CASE(P) case P: return green_passy_P##P(c, inv, s);
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t fused_any(const GreenCall& c, bool inv, cudaStream_t s) {
  switch (2 * c.nx) {
    case 128: return green_fused_P128(c, inv, s);
    case 256: return green_fused_P256(c, inv, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t pass3_any(const GreenCall& c, cudaStream_t s) {
  switch (2 * c.nz) {
#define MQ_CASE(P) case P: return green_pass3_P##P(c, s);
    MQ_DISPATCH(MQ_CASE)
#undef MQ_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// The five passes of one apply, each from the translation unit of its axis's
// transform length, with the optional pass events around them.
cudaError_t green_launch(const GreenCall& c, cudaStream_t s) {
  if (c.tile < 0 || c.tile >= MQ_TILES || !green_supported(c.nx) || !green_supported(c.ny) ||
      !green_supported(c.nz))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  // inside a stream capture the records must be external to become event-record
  // nodes of the graph; outside one they are plain records
  unsigned rec_flags = cudaEventRecordDefault;
  if (c.ev) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
  }
  auto rec = [&](int k) { return c.ev ? cudaEventRecordWithFlags(c.ev[k], s, rec_flags) : cudaSuccess; };
  // fused x/y passes (tile bit 4) for full applies; a plane input or output
  // takes the unfused passes on that side.  Their time counts as the x pass's
  // (events 1 and 2, 3 and 4 coincide).
  const bool fuse = (c.tile & MQ_TILE_FUSED) && green_fused_supported(c.nx, c.ny);
  const bool ffwd = fuse && !c.plane && !c.after_pass1, finv = fuse && !c.outplane;
  if ((e = rec(0)) != cudaSuccess) return e;
  if (ffwd) {
    if ((e = fused_any(c, false, s)) != cudaSuccess || (e = rec(1)) != cudaSuccess || (e = rec(2)) != cudaSuccess)
      return e;
  } else if ((e = pass1_any(c, s)) != cudaSuccess || (e = rec(1)) != cudaSuccess ||
             (c.after_pass1 && (e = c.after_pass1(c.after_pass1_ctx, s)) != cudaSuccess) ||
             (e = passy_any(c, false, s)) != cudaSuccess || (e = rec(2)) != cudaSuccess) {
    return e;
  }
  if ((e = pass3_any(c, s)) != cudaSuccess || (e = rec(3)) != cudaSuccess) return e;
  if (finv) {
    if ((e = rec(4)) != cudaSuccess || (e = fused_any(c, true, s)) != cudaSuccess || (e = rec(5)) != cudaSuccess)
      return e;
  } else if ((e = passy_any(c, true, s)) != cudaSuccess || (e = rec(4)) != cudaSuccess ||
             (e = pass5_any(c, s)) != cudaSuccess || (e = rec(5)) != cudaSuccess) {
    return e;
  }
  if (c.launches) *c.launches += 1 + (ffwd ? 1 : 2) + (finv ? 1 : 2) + (c.after_pass1 ? 1 : 0);
  return e;
}

// ---------------------------------------------------------- T2 tensor map
// T2 viewed as a 3D tensor of 8-byte elements: x = kx (Px), y = ky (Py),
// z = slot * nz + z (max_batch * nz).  Pass 3 loads boxes of C x 1 x nz: one
// column set of one slot.  The encoder comes from the driver through the
// runtime's entry-point query, so the library does not link libcuda.
cudaError_t make_t2_tensor_map(void* T2, int nx, int ny, int nz, int max_batch, int tile, void* map_out) {
  const int Px = 2 * nx, Py = 2 * ny;
  const int C = green_col_width(nx, ny, nz, tile);
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
  const cuuint64_t dims[3] = {(cuuint64_t)Px, (cuuint64_t)Py, (cuuint64_t)max_batch * nz};
  const cuuint64_t strides[2] = {(cuuint64_t)Px * 8, (cuuint64_t)Px * Py * 8};
  const cuuint32_t box[3] = {(cuuint32_t)C, 1u, (cuuint32_t)nz};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, T2, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ------------------------------------------------------------ K_hat build
// k[dz][dy][dx] for offsets in [0, nz) x [0, ny) x [0, nx) (FP64 complex as double2).
__global__ void k_kernel_octant(double2* k, int nx, int ny, int nz, double h, double kb) {
  const long long N = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int dx = (int)(i % nx), dy = (int)((i / nx) % ny), dz = (int)(i / ((long long)nx * ny));
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

// spec[mz][my][mx] = g_R^(|s_m|), s_m = (m_x dsx, m_y dsy, m_z dsz), m_d < M_d:
// the folded frequencies of the periods T_d (M_d = T_d/2 + 1; the transform is
// radial, so even in every axis).
__global__ void k_truncated_spectrum(double2* spec, int Mx, int My, int Mz, double dsx, double dsy, double dsz,
                                     double kb, double R) {
  const long long total = (long long)Mx * My * Mz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int mx = (int)(i % Mx), my = (int)((i / Mx) % My), mz = (int)(i / ((long long)Mx * My));
    const double sx = dsx * mx, sy = dsy * my, sz = dsz * mz;
    spec[i] = truncated_ft(sqrt(sx * sx + sy * sy + sz * sz), kb, R);
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

namespace {

// Truncation radius (the domain's diagonal, which covers every distance
// between two voxels) and the sample count T_d of each axis's period T_d h:
// 4 n_d, raised to the next even count >= n_d + R/h for an elongated domain,
// so that the periodic copies of g_R miss every offset the domain uses.
void truncated_periods(int nx, int ny, int nz, double h, double* R, int* T) {
  const double diag = std::sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
  *R = h * diag;
  const int n[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) T[d] = std::max(4 * n[d], 2 * (int)std::ceil((n[d] + diag) / 2.0));
}

std::vector<double> cos_tables(const int* len, int count) {
  std::vector<double> v;
  for (int q = 0; q < count; ++q)
    for (int j = 0; j < len[q]; ++j) v.push_back(std::cos(2.0 * M_PI * (double)j / (double)len[q]));
  return v;
}

// Real-space octant kb^2 w_D, D in [0, nz) x [0, ny) x [0, nx), of the
// truncated kernel into `a` ([dz][dy][dx]), from its transform sampled on the
// frequency grid of periods T_d h: w_D = (1 / prod T_d) sum_m g_R^(|s_m|) e^{j s_m . D h}
// (three even passes), times kb^2.  a, b: scratch of prod M_d double2 each;
// dcosT: Tx + Ty + Tz doubles.
cudaError_t truncated_octant(int nx, int ny, int nz, double h, double kb, double2* a, double2* b, double* dcosT,
                             cudaStream_t s) {
  double R;
  int T[3];
  truncated_periods(nx, ny, nz, h, &R, T);
  const int Mx = T[0] / 2 + 1, My = T[1] / 2 + 1, Mz = T[2] / 2 + 1;
  const std::vector<double> cosv = cos_tables(T, 3);
  cudaError_t e = cudaMemcpyAsync(dcosT, cosv.data(), cosv.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const double* cx = dcosT;
  const double* cy = dcosT + T[0];
  const double* cz = dcosT + T[0] + T[1];
  const int th = 256, gr = 2048;
  k_truncated_spectrum<<<gr, th, 0, s>>>(b, Mx, My, Mz, 2.0 * M_PI / (T[0] * h), 2.0 * M_PI / (T[1] * h),
                                         2.0 * M_PI / (T[2] * h), kb, R);   // b: [mz][my][mx]
  k_even_idft_pass<<<gr, th, 0, s>>>(b, a, Mz, My, Mx, nx, cx, T[0]);       // a: [dx][mz][my]
  k_even_idft_pass<<<gr, th, 0, s>>>(a, b, nx, Mz, My, ny, cy, T[1]);       // b: [dy][dx][mz]
  k_even_idft_pass<<<gr, th, 0, s>>>(b, a, ny, nx, Mz, nz, cz, T[2]);       // a: [dz][dy][dx]
  k_scale_d2<<<gr, th, 0, s>>>(a, (long long)nx * ny * nz, kb * kb / ((double)T[0] * T[1] * T[2]));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host cosine table goes out of scope
  return e;
}

// Scratch of the construction: double2 entries of each of a and b, and
// doubles of the cosine tables.
void khat_scratch_sizes(int nx, int ny, int nz, int kernel, size_t* big, size_t* ncos) {
  *big = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  *ncos = 2 * ((size_t)nx + ny + nz);
  if (kernel == MQNPM_KERNEL_TRUNCATED) {
    double R;
    int T[3];
    truncated_periods(nx, ny, nz, 1.0, &R, T);
    *big = std::max(*big, (size_t)(T[0] / 2 + 1) * (T[1] / 2 + 1) * (T[2] / 2 + 1));
    *ncos = std::max(*ncos, (size_t)T[0] + T[1] + T[2]);
  }
}

// K_hat octant [fz][fy][fx] = DFT of the P-periodic kernel / (Px Py Pz), rounded once.
cudaError_t khat_core(int nx, int ny, int nz, double h, double kb, int kernel, float2* khat_out, double2* a,
                      double2* b, double* dcos, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (kernel == MQNPM_KERNEL_TRUNCATED) e = truncated_octant(nx, ny, nz, h, kb, a, b, dcos, s);
  if (e != cudaSuccess) return e;
  const int P[3] = {2 * nx, 2 * ny, 2 * nz};
  const std::vector<double> cosv = cos_tables(P, 3);
  e = cudaMemcpyAsync(dcos, cosv.data(), cosv.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int th = 256, gr = 1024;
  if (kernel != MQNPM_KERNEL_TRUNCATED) k_kernel_octant<<<gr, th, 0, s>>>(a, nx, ny, nz, h, kb);   // a: [dz][dy][dx]
  k_cos_pass<<<gr, th, 0, s>>>(a, b, nz, ny, nx, dcos, P[0]);                        // b: [fx][dz][dy]
  k_cos_pass<<<gr, th, 0, s>>>(b, a, nx + 1, nz, ny, dcos + P[0], P[1]);             // a: [fy][fx][dz]
  k_cos_pass<<<gr, th, 0, s>>>(a, b, ny + 1, nx + 1, nz, dcos + P[0] + P[1], P[2]);  // b: [fz][fy][fx]
  k_round_khat<<<gr, th, 0, s>>>(b, khat_out, (long long)(nx + 1) * (ny + 1) * (nz + 1),
                                 1.0 / ((double)P[0] * P[1] * P[2]));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host cosine table goes out of scope
  return e;
}

}  // namespace

// The sampled kernel on a cubic grid with caller-provided device scratch: a,
// b hold (n+1)^3 double2 each, dcos holds 6n doubles.  No device allocation.
cudaError_t build_khat_scratch(int n, double h, double kb, float2* khat_out, double2* a, double2* b, double* dcos,
                               cudaStream_t s) {
  return khat_core(n, n, n, h, kb, MQNPM_KERNEL_SAMPLED, khat_out, a, b, dcos, s);
}

cudaError_t build_khat(int nx, int ny, int nz, double h, double kb, float2* khat_out, cudaStream_t s, int kernel) {
  size_t big = 0, ncos = 0;
  khat_scratch_sizes(nx, ny, nz, kernel, &big, &ncos);
  double2 *a = nullptr, *b = nullptr;
  double* dcos = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&a, big * sizeof(double2), s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&b, big * sizeof(double2), s)) != cudaSuccess) { cudaFreeAsync(a, s); return e; }
  if ((e = cudaMallocAsync(&dcos, ncos * sizeof(double), s)) != cudaSuccess) { cudaFreeAsync(a, s); cudaFreeAsync(b, s); return e; }
  e = khat_core(nx, ny, nz, h, kb, kernel, khat_out, a, b, dcos, s);
  cudaFreeAsync(a, s);
  cudaFreeAsync(b, s);
  cudaFreeAsync(dcos, s);
  return e;
}

// A caller-provided spectrum: the first octant [fz][fy][fx] of the
// unnormalised DFT_P, complex64 on the host.  Scaled by 1/(Px Py Pz) in FP64
// and rounded once, like the library's own construction.
cudaError_t upload_khat(const float* host, int nx, int ny, int nz, float2* khat_out, cudaStream_t s) {
  const size_t big = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  const double scale = 1.0 / (8.0 * (double)nx * ny * nz);
  std::vector<float2> v(big);
  for (size_t i = 0; i < big; ++i) {
    const double re = host[2 * i], im = host[2 * i + 1];
    v[i] = make_float2((float)(re * scale), (float)(im * scale));
  }
  cudaError_t e = cudaMemcpyAsync(khat_out, v.data(), big * sizeof(float2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the staging vector goes out of scope
  return e;
}
