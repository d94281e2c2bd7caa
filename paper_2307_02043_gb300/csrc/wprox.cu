// Weighted proximal mapping of c*TV + iota_C under B = tau I + U U^T
// (Eq. 4.4, Section 4.2-4.4, Theorem 3.1, Lemma 4.1, Algorithm 4.3).
//
// Accelerated projected gradient on the dual T(P) (Eq. 4.8):
//   w(R)  = v - c B^{-1} d(R) = v - (c/tau) d(R) + U gamma,
//           gamma = (c/tau^2) (I + U^T U / tau)^{-1} U^T d(R)      (Woodbury)
//   x     = prox^B_C(w) = clip(w - U beta*/tau),  phi(beta*) = 0     (Theorem 3.1)
//   P_j   = Proj(R_j + tau/(4 D c) d^T(x))                          (Lemma 4.1 step)
//   R_j+1 = P_j + (t_j - 1)/t_{j+1} (P_j - P_{j-1})
// beta* comes from semi-smooth Newton (Algorithm 4.3) with the generalised
// Jacobian H = I + tau^{-1} U^T diag(lo < z < hi) U; a step that does not
// reduce ||phi|| is halved.  The Newton loop runs inside one cooperative kernel
// (one grid barrier per evaluation of phi), so the host never waits on it.
//
// d(P) = sum_d (D^d)^T q_d with Neumann forward differences D^d; the dual field
// is stored as three planes q_x, q_y, q_z of N floats.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

namespace {

constexpr int OFF_G = 0;       // U^T U        (8 x 8)
constexpr int OFF_M = 64;      // (I + U^T U / tau)^{-1}
constexpr int OFF_UV = 128;    // U^T v
constexpr int OFF_BETA = 136;  // beta (warm start within a call)
constexpr int OFF_STAT = 160;  // [0] last newton count, [1] max, [2] total, [3] passes
constexpr int NSCAL = 176;

MQ_D size_t vidx(int n, int x, int y, int z) { return ((size_t)z * n + y) * n + x; }

// d(R) at one voxel: sum_d q_d(i - e_d)[i_d >= 1] - q_d(i)[i_d <= n-2]
MQ_D float div_at(const float* __restrict__ R, size_t N, int n, int x, int y, int z) {
  const size_t i = vidx(n, x, y, z);
  const float* qx = R;
  const float* qy = R + N;
  const float* qz = R + 2 * N;
  float s = 0.f;
  if (x > 0) s += qx[i - 1];
  if (x < n - 1) s -= qx[i];
  if (y > 0) s += qy[i - n];
  if (y < n - 1) s -= qy[i];
  if (z > 0) s += qz[i - (size_t)n * n];
  if (z < n - 1) s -= qz[i];
  return s;
}

MQ_D float clampf(float a, float lo, float hi) { return fminf(fmaxf(a, lo), hi); }

template <int TV>
MQ_D void project(float& px, float& py, float& pz) {
  if constexpr (TV == MQNPM_TV_ISO) {
    const float nr = sqrtf(px * px + py * py + pz * pz);
    if (nr > 1.f) {
      const float s = 1.f / nr;
      px *= s; py *= s; pz *= s;
    }
  } else {
    px = clampf(px, -1.f, 1.f);
    py = clampf(py, -1.f, 1.f);
    pz = clampf(pz, -1.f, 1.f);
  }
}

// ---------------------------------------------------- unweighted (U = 0)
// One fused dual step: x = clip(v - (c/tau) d(Rin)) at the voxel and its +x,+y,+z
// neighbours, gradient, projection, momentum.  Rin -> Rout (stencil reads), Pd in place.
template <int TV>
__global__ void k_dual_plain(const float* __restrict__ v, const float* __restrict__ Rin, float* __restrict__ Rout,
                             float* __restrict__ Pd, int n, float cdt, float step, float mom, float lo, float hi) {
  const size_t N = (size_t)n * n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    const float x0 = clampf(v[i] - cdt * div_at(Rin, N, n, x, y, z), lo, hi);
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (x < n - 1) gx = clampf(v[i + 1] - cdt * div_at(Rin, N, n, x + 1, y, z), lo, hi) - x0;
    if (y < n - 1) gy = clampf(v[i + n] - cdt * div_at(Rin, N, n, x, y + 1, z), lo, hi) - x0;
    if (z < n - 1) gz = clampf(v[i + (size_t)n * n] - cdt * div_at(Rin, N, n, x, y, z + 1), lo, hi) - x0;
    float px = Rin[i] + step * gx, py = Rin[N + i] + step * gy, pz = Rin[2 * N + i] + step * gz;
    project<TV>(px, py, pz);
    const float ox = Pd[i], oy = Pd[N + i], oz = Pd[2 * N + i];
    Pd[i] = px; Pd[N + i] = py; Pd[2 * N + i] = pz;
    Rout[i] = px + mom * (px - ox);
    Rout[N + i] = py + mom * (py - oy);
    Rout[2 * N + i] = pz + mom * (pz - oz);
  }
}

// x = clip(v - (c/tau) d(P))
__global__ void k_prox_plain(const float* __restrict__ v, const float* __restrict__ Pd, float* __restrict__ xo,
                             int n, float cdt, float lo, float hi) {
  const size_t N = (size_t)n * n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    xo[i] = clampf(v[i] - cdt * div_at(Pd, N, n, x, y, z), lo, hi);
  }
}

// ------------------------------------------------------ weighted (U != 0)
template <int S>
MQ_D void block_reduce_store(float (&acc)[S], double* dst) {
  __shared__ double scratch[32 * S];
  double v[S], o[S];
#pragma unroll
  for (int s = 0; s < S; ++s) v[s] = acc[s];
  block_sum<S>(v, scratch, o);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) dst[s] = o[s];
  }
}

// d = d(R); partials of U^T d.
template <int S>
__global__ void k_div_ut(const float* __restrict__ R, UPtrs U, float* __restrict__ d, int n, double* part) {
  const size_t N = (size_t)n * n * n;
  float acc[S];
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    const float dd = div_at(R, N, n, x, y, z);
    d[i] = dd;
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = fmaf(U.u[s][i], dd, acc[s]);
  }
  block_reduce_store<S>(acc, part + (size_t)blockIdx.x * S);
}

// Partials of U^T U (upper triangle) and U^T v.
template <int S>
__global__ void k_gram(UPtrs U, const float* __restrict__ v, size_t N, double* part) {
  constexpr int NG = S * (S + 1) / 2;
  float acc[NG + S];
#pragma unroll
  for (int k = 0; k < NG + S; ++k) acc[k] = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
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
    const float vi = v[i];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[NG + s] = fmaf(u[s], vi, acc[NG + s]);
  }
  block_reduce_store<NG + S>(acc, part + (size_t)blockIdx.x * (NG + S));
}

// Cholesky solve of the S x S SPD system A x = b (A row-major, overwritten).
template <int S>
MQ_D bool chol_solve(double (&A)[S * S], double (&b)[S]) {
#pragma unroll
  for (int j = 0; j < S; ++j) {
    double s = A[j * S + j];
    for (int k = 0; k < j; ++k) s -= A[j * S + k] * A[j * S + k];
    if (!(s > 0.0)) return false;
    const double l = sqrt(s);
    A[j * S + j] = l;
    for (int i = j + 1; i < S; ++i) {
      double t = A[i * S + j];
      for (int k = 0; k < j; ++k) t -= A[i * S + k] * A[j * S + k];
      A[i * S + j] = t / l;
    }
  }
  for (int i = 0; i < S; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= A[i * S + k] * b[k];
    b[i] = t / A[i * S + i];
  }
  for (int i = S - 1; i >= 0; --i) {
    double t = b[i];
    for (int k = i + 1; k < S; ++k) t -= A[k * S + i] * b[k];
    b[i] = t / A[i * S + i];
  }
  return true;
}

// Reduce the Gram partials; G, U^T v and M = (I + G/tau)^{-1} into scal.
template <int S>
__global__ void k_gram_setup(const double* part, int nctas, double tau, double* scal) {
  constexpr int NG = S * (S + 1) / 2, NV = NG + S;
  __shared__ double scratch[32 * NV];
  double v[NV], o[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int c = threadIdx.x; c < nctas; c += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += part[(size_t)c * NV + k];
  block_sum<NV>(v, scratch, o);
  if (threadIdx.x == 0) {
    int k = 0;
    for (int s = 0; s < S; ++s)
      for (int t = s; t < S; ++t) {
        scal[OFF_G + s * S + t] = o[k];
        scal[OFF_G + t * S + s] = o[k];
        ++k;
      }
    for (int s = 0; s < S; ++s) scal[OFF_UV + s] = o[NG + s];
    for (int col = 0; col < S; ++col) {
      double A[S * S], e[S];
      for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) A[i * S + j] = (i == j ? 1.0 : 0.0) + scal[OFF_G + i * S + j] / tau;
      for (int i = 0; i < S; ++i) e[i] = (i == col) ? 1.0 : 0.0;
      chol_solve<S>(A, e);
      for (int i = 0; i < S; ++i) scal[OFF_M + i * S + col] = e[i];
    }
    for (int s = 0; s < S; ++s) scal[OFF_BETA + s] = 0.0;
    for (int q = 0; q < 4; ++q) scal[OFF_STAT + q] = 0.0;
  }
}

// Deterministic cross-block sum of NV partials per block (all threads help).
template <int NV>
MQ_D void grid_partials_sum(const double* part, int nblk, double* sh_tot /*NV*/, double* sh_tmp /*blockDim*/) {
  const int groups = blockDim.x / NV;   // >= 1 (NV <= 44, blockDim = 256)
  const int t = threadIdx.x;
  double acc = 0.0;
  if (t < groups * NV) {
    const int v = t % NV, g = t / NV;
    for (int c = g; c < nblk; c += groups) acc += part[(size_t)c * NV + v];
  }
  sh_tmp[t] = acc;
  __syncthreads();
  if (t < NV) {
    double s = 0.0;
    for (int g = 0; g < groups; ++g) s += sh_tmp[g * NV + t];
    sh_tot[t] = s;
  }
  __syncthreads();
}

// Semi-smooth Newton for beta* (cooperative launch, one block per SM).
// Writes x = clip(v - (c/tau) d + U (gamma - beta*/tau)).
template <int S>
__global__ void __launch_bounds__(256)
k_ssn(const float* __restrict__ v, const float* __restrict__ d, UPtrs U, float* __restrict__ xo, size_t N,
      double c, double tau, float lo, float hi, double tol, int maxit, const double* __restrict__ part10,
      int ctas10, double* __restrict__ scal, double* __restrict__ part, unsigned* bar, int* err,
      long long limit) {
  constexpr int NG = S * (S + 1) / 2, NV = S + NG;
  __shared__ double sh_tot[NV > S ? NV : S];
  __shared__ double sh_tmp[256];
  __shared__ float sh_theta[S], sh_gamma[S];
  __shared__ int sh_done;
  __shared__ double sh_beta[S], sh_beta_acc[S];
  unsigned epoch = 0;
  const float cdt = (float)(c / tau);
  // U^T d -> gamma = (c/tau^2) M U^T d ; U^T w = U^T v - (c/tau) U^T d + G gamma
  grid_partials_sum<S>(part10, ctas10, sh_tot, sh_tmp);
  double gamma[S], utw[S], beta[S], beta_eval[S], dir[S], phi_cur[S];
  double nphi_cur = 0.0, tstep = 1.0, scale = 1.0;
  int halvings = 0, accepted = 0, passes = 0;
  {
    double utd[S];
#pragma unroll
    for (int s = 0; s < S; ++s) utd[s] = sh_tot[s];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      double g = 0.0;
#pragma unroll
      for (int t = 0; t < S; ++t) g += scal[OFF_M + s * S + t] * utd[t];
      gamma[s] = c / (tau * tau) * g;
    }
    double nrm = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      double g = scal[OFF_UV + s] - c / tau * utd[s];
#pragma unroll
      for (int t = 0; t < S; ++t) g += scal[OFF_G + s * S + t] * gamma[t];
      utw[s] = g;
      nrm += g * g;
    }
    scale = fmax(1.0, sqrt(nrm));
#pragma unroll
    for (int s = 0; s < S; ++s) {
      beta[s] = scal[OFF_BETA + s];
      beta_eval[s] = beta[s];
      dir[s] = 0.0;
      phi_cur[s] = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sh_done = 0;
  const int max_passes = maxit * 8;
  bool first = true;
  while (true) {
    if (threadIdx.x < S) {
      sh_theta[threadIdx.x] = (float)(gamma[threadIdx.x] - beta_eval[threadIdx.x] / tau);
      sh_gamma[threadIdx.x] = (float)gamma[threadIdx.x];
    }
    __syncthreads();
    float th[S], ga[S];
#pragma unroll
    for (int s = 0; s < S; ++s) { th[s] = sh_theta[s]; ga[s] = sh_gamma[s]; }
    float acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
      const float base = v[i] - cdt * d[i];
      float u[S];
      float zz = base, ww = base;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        u[s] = U.u[s][i];
        zz = fmaf(u[s], th[s], zz);
        ww = fmaf(u[s], ga[s], ww);
      }
      const float e = ww - clampf(zz, lo, hi);
      const float in = (zz > lo && zz < hi) ? 1.f : 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = fmaf(u[s], e, acc[s]);
      int k = S;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const float us = in * u[s];
#pragma unroll
        for (int t = s; t < S; ++t) { acc[k] = fmaf(us, u[t], acc[k]); ++k; }
      }
    }
    double* mypart = part + ((size_t)(passes & 1) * gridDim.x + blockIdx.x) * NV;
    block_reduce_store<NV>(acc, mypart);
    ++passes;
    if (!grid_barrier(bar, gridDim.x, epoch, err, limit)) return;
    grid_partials_sum<NV>(part + (size_t)((passes - 1) & 1) * gridDim.x * NV, gridDim.x, sh_tot, sh_tmp);
    if (threadIdx.x == 0) {
      double phi[S], H[S * S], nphi = 0.0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        phi[s] = sh_tot[s] + beta_eval[s];
        nphi += phi[s] * phi[s];
      }
      nphi = sqrt(nphi);
      bool accept = first || nphi < nphi_cur || halvings >= 30 || !isfinite(nphi_cur);
      first = false;
      int done = 0;
      if (accept) {
#pragma unroll
        for (int s = 0; s < S; ++s) { beta[s] = beta_eval[s]; phi_cur[s] = phi[s]; }
        nphi_cur = nphi;
        if (nphi <= tol * scale || accepted >= maxit || passes >= max_passes || !isfinite(nphi)) {
          done = 1;
        } else {
          int k = S;
          for (int s = 0; s < S; ++s)
            for (int t = s; t < S; ++t) {
              const double hst = sh_tot[k++] / tau;
              H[s * S + t] = hst + (s == t ? 1.0 : 0.0);
              H[t * S + s] = H[s * S + t];
            }
          double rhs[S];
#pragma unroll
          for (int s = 0; s < S; ++s) rhs[s] = -phi[s];
          if (!chol_solve<S>(H, rhs)) {
            done = 1;
          } else {
#pragma unroll
            for (int s = 0; s < S; ++s) { dir[s] = rhs[s]; beta_eval[s] = beta[s] + rhs[s]; }
            tstep = 1.0;
            halvings = 0;
            ++accepted;
          }
        }
      } else {
        tstep *= 0.5;
        ++halvings;
#pragma unroll
        for (int s = 0; s < S; ++s) beta_eval[s] = beta[s] + tstep * dir[s];
        if (passes >= max_passes) done = 1;
      }
      sh_done = done;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        sh_beta[s] = beta_eval[s];
        sh_beta_acc[s] = beta[s];
      }
    }
    __syncthreads();
    // every block took the same decision from the same reduced values
    if (sh_done) break;
#pragma unroll
    for (int s = 0; s < S; ++s) beta_eval[s] = sh_beta[s];
  }
  // final pass with the accepted beta (thread 0's decision, broadcast)
#pragma unroll
  for (int s = 0; s < S; ++s) beta[s] = sh_beta_acc[s];
  if (threadIdx.x < S) sh_theta[threadIdx.x] = (float)(gamma[threadIdx.x] - beta[threadIdx.x] / tau);
  __syncthreads();
  float th[S];
#pragma unroll
  for (int s = 0; s < S; ++s) th[s] = sh_theta[s];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    float zz = v[i] - cdt * d[i];
#pragma unroll
    for (int s = 0; s < S; ++s) zz = fmaf(U.u[s][i], th[s], zz);
    xo[i] = clampf(zz, lo, hi);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) scal[OFF_BETA + s] = beta[s];
    scal[OFF_STAT + 0] = accepted;
    scal[OFF_STAT + 1] = fmax(scal[OFF_STAT + 1], (double)accepted);
    scal[OFF_STAT + 2] += accepted;
    scal[OFF_STAT + 3] += passes;
  }
}

// P update from x (weighted case): gradient of x, projection, momentum; in place.
template <int TV>
__global__ void k_dual_update(const float* __restrict__ xw, float* __restrict__ R, float* __restrict__ Pd, int n,
                              float step, float mom) {
  const size_t N = (size_t)n * n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((size_t)n * n));
    const float x0 = xw[i];
    const float gx = x < n - 1 ? xw[i + 1] - x0 : 0.f;
    const float gy = y < n - 1 ? xw[i + n] - x0 : 0.f;
    const float gz = z < n - 1 ? xw[i + (size_t)n * n] - x0 : 0.f;
    float px = R[i] + step * gx, py = R[N + i] + step * gy, pz = R[2 * N + i] + step * gz;
    project<TV>(px, py, pz);
    const float ox = Pd[i], oy = Pd[N + i], oz = Pd[2 * N + i];
    Pd[i] = px; Pd[N + i] = py; Pd[2 * N + i] = pz;
    R[i] = px + mom * (px - ox);
    R[N + i] = py + mom * (py - oy);
    R[2 * N + i] = pz + mom * (pz - oz);
  }
}

#define CK(call)                                                \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return set_cuda_error(h, e_, #call); \
  } while (0)

template <int S>
cudaError_t launch_gram(mqnpm_handle* h, const UPtrs& U, const float* v, double tau) {
  cudaStream_t s = h->stream;
  const int ctas = h->wp.ctas_vec;
  k_gram<S><<<ctas, 256, 0, s>>>(U, v, h->N, h->wp.part);
  k_gram_setup<S><<<1, 256, 0, s>>>(h->wp.part, ctas, tau, h->wp.scal);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_div(mqnpm_handle* h, const float* R, const UPtrs& U, float* part10) {
  (void)part10;
  k_div_ut<S><<<h->wp.ctas_vec, 256, 0, h->stream>>>(R, U, h->wp.d, h->n, h->wp.part);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_ssn(mqnpm_handle* h, const float* v, const UPtrs& U, float* xo, double c, double tau) {
  cudaError_t e = cudaMemsetAsync(h->wp.barrier, 0, sizeof(unsigned), h->stream);
  if (e != cudaSuccess) return e;
  const float* pv = v;
  const float* pd = h->wp.d;
  UPtrs uu = U;
  size_t N = h->N;
  float lo = (float)h->lo, hi = (float)h->hi;
  double tol = h->newton_tol;
  int maxit = h->newton_maxit;
  const double* part10 = h->wp.part;
  int ctas10 = h->wp.ctas_vec;
  double* scal = h->wp.scal;
  double* part = h->wp.part + (size_t)ctas10 * 64;
  unsigned* bar = h->wp.barrier;
  int* err = h->wp.err;
  long long limit = 4000000000LL;   // ~2 s at 2 GHz
  void* args[] = {&pv, &pd, &uu, &xo, &N, &c, &tau, &lo, &hi, &tol, &maxit, &part10, &ctas10, &scal,
                  &part, &bar, &err, &limit};
  return cudaLaunchCooperativeKernel((void*)k_ssn<S>, dim3(h->wp.ctas), dim3(256), args, 0, h->stream);
}

template <int S>
int wprox_weighted(mqnpm_handle* h, const float* v, double tau, const UPtrs& U, double c, float* x_out,
                   const std::vector<double>& mom) {
  cudaStream_t s = h->stream;
  const int J = h->dual_iters;
  const float step = (float)(tau / (4.0 * 3.0 * c));
  CK(launch_gram<S>(h, U, v, tau));
  for (int j = 0; j < J; ++j) {
    CK(launch_div<S>(h, h->wp.R, U, nullptr));
    CK(launch_ssn<S>(h, v, U, h->wp.x, c, tau));
    if (h->tv == MQNPM_TV_ISO)
      k_dual_update<MQNPM_TV_ISO><<<h->wp.ctas_vec, 256, 0, s>>>(h->wp.x, h->wp.R, h->wp.Pd, h->n, step, (float)mom[j]);
    else
      k_dual_update<MQNPM_TV_ANISO><<<h->wp.ctas_vec, 256, 0, s>>>(h->wp.x, h->wp.R, h->wp.Pd, h->n, step, (float)mom[j]);
    CK(cudaGetLastError());
  }
  CK(launch_div<S>(h, h->wp.Pd, U, nullptr));
  CK(launch_ssn<S>(h, v, U, x_out, c, tau));
  return MQNPM_OK;
}

}  // namespace

int wprox_impl(mqnpm_handle* h, const float* v, double tau, const UPtrs& U, int S_eff, double c, float* P_warm,
               bool warm, float* x_out) {
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  const int J = h->dual_iters;
  // FGP momentum coefficients (t_1 = 1)
  std::vector<double> mom(std::max(J, 1));
  double t = 1.0;
  for (int j = 0; j < J; ++j) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    mom[j] = (t - 1.0) / tn;
    t = tn;
  }
  if (warm && P_warm) {
    CK(cudaMemcpyAsync(h->wp.Pd, P_warm, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemsetAsync(h->wp.Pd, 0, 3 * N * sizeof(float), s));
  }
  CK(cudaMemcpyAsync(h->wp.R, h->wp.Pd, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(h->wp.err, 0, sizeof(int), s));
  const float lo = (float)h->lo, hi = (float)h->hi;
  if (S_eff == 0) {
    const float cdt = (float)(c / tau);
    const float step = (float)(tau / (4.0 * 3.0 * c));
    float* Rin = h->wp.R;
    float* Rout = h->wp.R2;
    for (int j = 0; j < J; ++j) {
      if (h->tv == MQNPM_TV_ISO)
        k_dual_plain<MQNPM_TV_ISO><<<h->wp.ctas_vec, 256, 0, s>>>(v, Rin, Rout, h->wp.Pd, h->n, cdt, step, (float)mom[j], lo, hi);
      else
        k_dual_plain<MQNPM_TV_ANISO><<<h->wp.ctas_vec, 256, 0, s>>>(v, Rin, Rout, h->wp.Pd, h->n, cdt, step, (float)mom[j], lo, hi);
      std::swap(Rin, Rout);
    }
    k_prox_plain<<<h->wp.ctas_vec, 256, 0, s>>>(v, h->wp.Pd, x_out, h->n, cdt, lo, hi);
    CK(cudaGetLastError());
    h->last_newton_max = 0;
    h->last_newton_total = 0;
  } else {
    int rc;
    switch (S_eff) {
      case 1: rc = wprox_weighted<1>(h, v, tau, U, c, x_out, mom); break;
      case 2: rc = wprox_weighted<2>(h, v, tau, U, c, x_out, mom); break;
      case 3: rc = wprox_weighted<3>(h, v, tau, U, c, x_out, mom); break;
      case 4: rc = wprox_weighted<4>(h, v, tau, U, c, x_out, mom); break;
      case 5: rc = wprox_weighted<5>(h, v, tau, U, c, x_out, mom); break;
      case 6: rc = wprox_weighted<6>(h, v, tau, U, c, x_out, mom); break;
      case 7: rc = wprox_weighted<7>(h, v, tau, U, c, x_out, mom); break;
      case 8: rc = wprox_weighted<8>(h, v, tau, U, c, x_out, mom); break;
      default: return set_error(h, MQNPM_ERR_INVALID_ARG, "wprox: S_eff out of range");
    }
    if (rc != MQNPM_OK) return rc;
    double stat[4];
    int errflag = 0;
    CK(cudaMemcpyAsync(stat, h->wp.scal + OFF_STAT, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&errflag, h->wp.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->last_newton_max = (int)stat[1];
    h->last_newton_total = (int)stat[2];
    if (errflag) return set_error(h, MQNPM_ERR_TIMEOUT, "wprox: grid barrier wait gave up");
  }
  if (P_warm) CK(cudaMemcpyAsync(P_warm, h->wp.Pd, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return MQNPM_OK;
}

int wprox_scal_count() { return NSCAL; }

// Blocks per SM the cooperative Newton kernel can keep resident (worst case S = 8).
int wprox_coop_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ssn<8>, 256, 0) != cudaSuccess) return 0;
  return nb;
}

namespace {
// v = x - (aS/tau) g + (aS/tau^2) U M U^T g   (B^{-1} by Woodbury, Section 4.4);
// scal holds M and U^T g (as "U^T v") from k_gram_setup.
template <int S>
__global__ void k_qn_point(const float* __restrict__ x, const float* __restrict__ g, UPtrs U, const double* scal,
                           double aS, double tau, float* __restrict__ v, size_t N) {
  __shared__ float coef[S];
  if (threadIdx.x < S) {
    double cs = 0.0;
    for (int t = 0; t < S; ++t) cs += scal[OFF_M + threadIdx.x * S + t] * scal[OFF_UV + t];
    coef[threadIdx.x] = (float)(aS / (tau * tau) * cs);
  }
  __syncthreads();
  const float a0 = (float)(aS / tau);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    float acc = fmaf(-a0, g[i], x[i]);
#pragma unroll
    for (int s = 0; s < S; ++s) acc = fmaf(coef[s], U.u[s][i], acc);
    v[i] = acc;
  }
}

template <int S>
cudaError_t qn_point(mqnpm_handle* h, const float* x, const float* g, const UPtrs& U, double tau, double aS, float* v) {
  cudaError_t e = launch_gram<S>(h, U, g, tau);
  if (e != cudaSuccess) return e;
  k_qn_point<S><<<h->wp.ctas_vec, 256, 0, h->stream>>>(x, g, U, h->wp.scal, aS, tau, v, h->N);
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
    default: return set_error(h, MQNPM_ERR_INVALID_ARG, "qn_point: S_eff out of range");
  }
  return e == cudaSuccess ? MQNPM_OK : set_cuda_error(h, e, "qn_point");
}
