// Mini-batch data-term gradient (Section 6): Lippmann-Schwinger forward solve
// by BiCGSTAB, detector residual, adjoint solve and gradient assembly, all
// illuminations of a batch advancing in lockstep (converged slots idle).
//
// BiCGSTAB (van der Vorst 1992) per slot, on A = I - G X (forward) or
// A = I - G^H X (adjoint), with complex64 vectors and FP64 scalars:
//   p = r + beta (p - omega v);  v = A p;          alpha = rho / <rhat, v>
//   s = r - alpha v;             t = A s;          omega = <t, s> / <t, t>
//   u += alpha p + omega s;      r = s - omega t;  rho' = <rhat, r>, beta = rho'/rho * alpha/omega
// Both matrix-vector products are single Green's applies whose first pass
// forms p (or s) on the fly and whose last pass forms v (or t) and the inner
// products.  Forward start u_0 = u_in (so r_0 = G(x u_in)); adjoint start 0.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

namespace {

struct dc {
  double re, im;
};
MQ_D dc dmul(dc a, dc b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
MQ_D dc ddiv(dc a, dc b) {   // one FP64 reciprocal (division is a long sequence on this device)
  const double r = 1.0 / (b.re * b.re + b.im * b.im);
  return {(a.re * b.re + a.im * b.im) * r, (a.im * b.re - a.re * b.im) * r};
}
MQ_D bool dfinite(dc a) { return isfinite(a.re) && isfinite(a.im); }

// Deterministic sum of K partials per CTA over `nctas` CTAs of slot b.
template <int K>
MQ_D void sum_partials(const double* part, int b, int nctas, double (&out)[K]) {
  __shared__ double scratch[32 * K];
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
#pragma unroll 4
  for (int c = threadIdx.x; c < nctas; c += blockDim.x) {   // unrolled: loads of 4 CTAs in flight
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += part[((size_t)b * nctas + c) * K + k];
  }
  block_sum<K>(v, scratch, out);
}

// ||b||^2 of each slot's right-hand side from an apply's partials, kept in
// the slot state for a k_fin_init whose start is not 0 (bnorm2_fwd < 0).
__global__ void k_set_bnorm(KState* st, const double* part, int nctas) {
  const int b = blockIdx.x;
  double s[1];
  sum_partials<1>(part, b, nctas, s);
  if (threadIdx.x == 0) st[b].bnorm2 = s[0];
}

// Slot state of a solve whose first residual r_0 has its partials in part.
// bnorm2_fwd > 0: ||b||^2 for every slot; == 0: ||r_0||^2 (a start at 0);
// < 0: the value k_set_bnorm (or an earlier k_fin_init) left in the slot
// state.  keep_inactive: slots already stopped keep their state (their
// partials were not recomputed).
__global__ void k_fin_init(KState* st, const double* part, int nctas, double tol2, double bnorm2_fwd,
                           int keep_inactive) {
  const int b = blockIdx.x;
  if (keep_inactive && !st[b].active) return;
  double s[1];
  sum_partials<1>(part, b, nctas, s);
  if (threadIdx.x == 0) {
    const double bkept = st[b].bnorm2;
    KState k;
    memset(&k, 0, sizeof(k));
    k.rho_re = s[0];
    k.alpha_re = 1.0;
    k.omega_re = 1.0;
    k.beta_re = 0.0;   // the first iteration takes p_1 = r_0 (iters == 0)
    k.rnorm2 = s[0];
    k.bnorm2 = bnorm2_fwd > 0.0 ? bnorm2_fwd : bnorm2_fwd < 0.0 ? bkept : s[0];
    k.tol2 = tol2;
    k.iters = 0;
    if (!isfinite(s[0])) {
      k.status = KSTATUS_NONFINITE;
      k.active = 0;
    } else if (k.bnorm2 == 0.0 || k.rnorm2 <= tol2 * k.bnorm2) {
      k.status = KSTATUS_CONVERGED;
      k.active = 0;
    } else {
      k.status = KSTATUS_RUNNING;
      k.active = 1;
    }
    st[b] = k;
  }
}

__global__ void k_fin_alpha(KState* st, const double* part5, int nctas) {
  const int b = blockIdx.x;
  if (!st[b].active) return;
  double s[2];
  sum_partials<2>(part5, b, nctas, s);
  if (threadIdx.x == 0) {
    KState& k = st[b];
    const dc rv{s[0], s[1]};
    const dc rho{k.rho_re, k.rho_im};
    if (!(rv.re * rv.re + rv.im * rv.im > 0.0) || !dfinite(rv)) {
      k.status = dfinite(rv) ? KSTATUS_BREAKDOWN : KSTATUS_NONFINITE;
      k.active = 0;
      return;
    }
    const dc a = ddiv(rho, rv);
    k.alpha_re = a.re;
    k.alpha_im = a.im;
  }
}

// The half step of a BiCGSTAB iteration, between pass 1 and pass 2 of its
// second apply: a slot whose s = r - alpha v already meets the tolerance
// takes x += alpha p, r = s (omega = 0, conv_pending) and is marked active = 2,
// so the remaining passes of that apply skip it; k_fin_rho retires it.
__global__ void k_fin_s(KState* st, const double* part1, int nctas) {
  const int b = blockIdx.x;
  if (st[b].active != 1) return;
  double s1[1];
  sum_partials<1>(part1, b, nctas, s1);
  if (threadIdx.x == 0) {
    KState& k = st[b];
    if (s1[0] <= k.tol2 * k.bnorm2) {
      k.conv_pending = 1;
      k.omega_re = 0.0;
      k.omega_im = 0.0;
      k.active = 2;
    }
  }
}

__global__ void k_fin_omega(KState* st, const double* part1, const double* part5, int nctas) {
  const int b = blockIdx.x;
  if (st[b].active != 1) return;   // 2: retired at the half step, omega = 0 already
  double s1[1], s5[3];
  sum_partials<1>(part1, b, nctas, s1);
  sum_partials<3>(part5, b, nctas, s5);
  if (threadIdx.x == 0) {
    KState& k = st[b];
    if (s1[0] <= k.tol2 * k.bnorm2) {          // ||s|| small: x += alpha p, r = s
      k.conv_pending = 1;
      k.omega_re = 0.0;
      k.omega_im = 0.0;
      return;
    }
    if (!(s5[2] > 0.0) || !isfinite(s5[2]) || !isfinite(s5[0])) {
      k.status = isfinite(s5[2]) ? KSTATUS_BREAKDOWN : KSTATUS_NONFINITE;
      k.active = 0;
      return;
    }
    const double r = 1.0 / s5[2];
    k.omega_re = s5[0] * r;
    k.omega_im = s5[1] * r;
  }
}

// xs += alpha p + omega s ;  r = s - omega t ; partials <rhat, r>, ||r||^2
__global__ void k_update(const KState* __restrict__ st, float2* __restrict__ xs, float2* __restrict__ r,
                         const float2* __restrict__ p, const float2* __restrict__ sv,
                         const float2* __restrict__ tv, const float2* __restrict__ rhat, size_t N,
                         double* __restrict__ partu) {
  const int b = blockIdx.y;
  if (!st[b].active) return;
  const float2 alpha = make_float2((float)st[b].alpha_re, (float)st[b].alpha_im);
  const float2 omega = make_float2((float)st[b].omega_re, (float)st[b].omega_im);
  const float2 nomega = make_float2(-omega.x, -omega.y);
  const size_t off = (size_t)b * N;
  const bool half = st[b].conv_pending != 0;   // converged at s: x += alpha p, r = s (t not read)
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const size_t j = off + i;
    const float2 s = sv[j];
    float2 x = xs[j];
    x = caxpy(alpha, p[j], x);
    if (!half) x = caxpy(omega, s, x);
    xs[j] = x;
    const float2 rn = half ? s : caxpy(nomega, tv[j], s);
    r[j] = rn;
    const float2 d = cmulc(rhat[j], rn);
    a0 += d.x;
    a1 += d.y;
    a2 += cabs2(rn);
  }
  __shared__ double scratch[33 * 3];
  const float v[3] = {a0, a1, a2};
  double out[3];
  block_sum_f<3>(v, scratch, out);
  if (threadIdx.x == 0) {
    double* q = partu + ((size_t)b * gridDim.x + blockIdx.x) * 3;
    q[0] = out[0];
    q[1] = out[1];
    q[2] = out[2];
  }
}

__global__ void k_fin_rho(KState* st, const double* partu, int nctas, int maxit, int* nactive) {
  const int b = blockIdx.x;
  if (!st[b].active) return;
  double s[3];
  sum_partials<3>(partu, b, nctas, s);
  if (threadIdx.x == 0) {
    KState& k = st[b];
    k.iters += 1;
    k.rnorm2 = s[2];
    const dc rho_new{s[0], s[1]};
    if (!isfinite(s[2]) || !dfinite(rho_new)) {
      k.status = KSTATUS_NONFINITE;
      k.active = 0;
    } else if (k.conv_pending || s[2] <= k.tol2 * k.bnorm2) {
      k.status = KSTATUS_CONVERGED;
      k.active = 0;
    } else if (k.iters >= maxit) {
      k.status = KSTATUS_MAXIT;
      k.active = 0;
    } else {
      const dc rho{k.rho_re, k.rho_im};
      const dc alpha{k.alpha_re, k.alpha_im}, omega{k.omega_re, k.omega_im};
      if (!(rho.re * rho.re + rho.im * rho.im > 0.0) || !(omega.re * omega.re + omega.im * omega.im > 0.0)) {
        k.status = KSTATUS_BREAKDOWN;
        k.active = 0;
      } else {
        const dc beta = dmul(ddiv(rho_new, rho), ddiv(alpha, omega));
        k.beta_re = beta.re;
        k.beta_im = beta.im;
        k.rho_re = rho_new.re;
        k.rho_im = rho_new.im;
      }
    }
    if (k.active) atomicAdd(nactive, 1);
  }
}

// End of one pass through the device-side Krylov loop: keep looping while a
// slot is active.  k_fin_rho retires every slot at krylov_maxit iterations, so
// the loop ends by itself; `loops` counts the passes and caps them at `cap`
// as well (a bound that does not rely on the slot bookkeeping).
__global__ void k_loop_cond(cudaGraphConditionalHandle cond, const int* nactive, int* loops, int cap) {
  const int done = *loops + 1;
  *loops = done;
  cudaGraphSetConditional(cond, (*nactive > 0 && done < cap) ? 1u : 0u);
}

// u_in of illumination l at voxel i of an nx x ny x nz grid (d = (nx, ny, nz));
// axis tables [l][nx + ny + nz].
MQ_D float2 incident_at(const float2* tab, int l, int3 d, size_t i) {
  const int x = (int)(i % d.x), y = (int)((i / d.x) % d.y), z = (int)(i / ((size_t)d.x * d.y));
  const float2* t = tab + (size_t)l * (d.x + d.y + d.z);
  return cmul(cmul(t[x], t[d.x + y]), t[d.x + d.y + z]);
}

__global__ void k_init_uin(float2* u, const float2* tab, const int* illum, int3 n, size_t N) {
  const int b = blockIdx.y;
  const int l = illum[b];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    u[(size_t)b * N + i] = incident_at(tab, l, n, i);
}

// Start fields of a warm-started forward solve: the field stored for the
// slot's illumination where there is one (fwarm[b]), else u_in.
__global__ void k_init_u_warm(float2* u, float2* const* fwarm, const float2* tab, const int* illum, int3 n, size_t N) {
  const int b = blockIdx.y;
  const int l = illum[b];
  const float2* src = fwarm[b];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    u[(size_t)b * N + i] = src ? src[i] : incident_at(tab, l, n, i);
}

// u += r on the slots still iterating (the fixed-point step u_1 = u_0 + r_0).
__global__ void k_add_residual(float2* u, const float2* __restrict__ r, const KState* st, size_t N) {
  const int b = blockIdx.y;
  if (!st[b].active) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    u[(size_t)b * N + i] = cadd(u[(size_t)b * N + i], r[(size_t)b * N + i]);
}

// Keep each slot's converged field for its illumination's next solve
// (fstore[b]; slots without a destination keep nothing).
__global__ void k_store_field(float2* const* fstore, const float2* __restrict__ u, size_t N) {
  const int b = blockIdx.y;
  float2* dst = fstore[b];
  if (dst == nullptr) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = u[(size_t)b * N + i];
}

// Detector of the LS field: usc = (u - u_in) on z = n-1; r_det = usc - y (or usc if y == NULL).
__global__ void k_detect_ls(const float2* u, const float2* tab, const int* illum, const float2* ymeas,
                            float2* out, int3 n, size_t N, double* part) {
  const int b = blockIdx.y;
  const int l = illum[b];
  const size_t M = (size_t)n.x * n.y;
  const size_t base = (size_t)(n.z - 1) * M;
  float acc = 0.f;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < M; j += (size_t)gridDim.x * blockDim.x) {
    const size_t i = base + j;
    float2 r = csub(u[(size_t)b * N + i], incident_at(tab, l, n, i));
    if (ymeas) r = csub(r, ymeas[(size_t)l * M + j]);
    out[(size_t)b * M + j] = r;
    acc += cabs2(r);
  }
  __shared__ double scratch[33];
  const float v[1] = {acc};
  double o[1];
  block_sum_f<1>(v, scratch, o);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = o[0];
}

// grad[i] (+)= scale * sum_b Re(conj(u_b[i]) z_b[i]); u_b = u_in(l_b) when u == NULL (Born).
__global__ void k_grad(const float2* __restrict__ u, const float2* __restrict__ zsol, const float2* tab,
                       const int* illum, int nb, int3 n, size_t N, float scale, float* grad, int accumulate) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = 0; b < nb; ++b) {
      const float2 uu = u ? u[(size_t)b * N + i] : incident_at(tab, illum[b], n, i);
      const float2 zz = zsol[(size_t)b * N + i];
      acc = fmaf(uu.x, zz.x, fmaf(uu.y, zz.y, acc));
    }
    const float g = scale * acc;
    grad[i] = accumulate ? grad[i] + g : g;
  }
}

// Gradient assembly per segment of consecutive slots (blockIdx.y = segment):
// seg.grad[i] (+)= seg.scale * sum_{b in [b0, b1)} Re(conj(u_b[i]) z_b[i]),
// u_b = u_in(l_b) when u == NULL (Born).
__global__ void k_grad_seg(const float2* __restrict__ u, const float2* __restrict__ zsol, const float2* tab,
                           const int* illum, int3 n, size_t N, const GradSeg* segs) {
  const GradSeg sg = segs[blockIdx.y];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = sg.b0; b < sg.b1; ++b) {
      const float2 uu = u ? u[(size_t)b * N + i] : incident_at(tab, illum[b], n, i);
      const float2 zz = zsol[(size_t)b * N + i];
      acc = fmaf(uu.x, zz.x, fmaf(uu.y, zz.y, acc));
    }
    const float g = sg.scale * acc;
    sg.grad[i] = sg.accumulate ? sg.grad[i] + g : g;
  }
}

// Sum of nb*nctas partials (one per CTA) into out[0] (deterministic).
__global__ void k_sum_all(const double* part, int count, double* out) {
  __shared__ double scratch[32];
  double v[1] = {0.0}, o[1];
  for (int i = threadIdx.x; i < count; i += blockDim.x) v[0] += part[i];
  block_sum<1>(v, scratch, o);
  if (threadIdx.x == 0) out[0] = o[0];
}

// FP64 dot products of s = a - b (b may be NULL) and m = c - d (d may be NULL):
// partials of <s,s>, <s,m>, <m,m>.
__global__ void k_dots3(const float* a, const float* b, const float* c, const float* d, size_t N, double* part) {
  float ss = 0.f, sm = 0.f, mm = 0.f;
  double dss = 0.0, dsm = 0.0, dmm = 0.0;
  int cnt = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float s = b ? a[i] - b[i] : a[i];
    const float m = c ? (d ? c[i] - d[i] : c[i]) : 0.f;
    ss = fmaf(s, s, ss);
    sm = fmaf(s, m, sm);
    mm = fmaf(m, m, mm);
    if (++cnt == 16) {
      dss += ss; dsm += sm; dmm += mm;
      ss = sm = mm = 0.f;
      cnt = 0;
    }
  }
  dss += ss; dsm += sm; dmm += mm;
  __shared__ double scratch[32 * 3];
  double v[3] = {dss, dsm, dmm}, o[3];
  block_sum<3>(v, scratch, o);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = o[0];
    part[blockIdx.x * 3 + 1] = o[1];
    part[blockIdx.x * 3 + 2] = o[2];
  }
}
__global__ void k_sum3(const double* part, int nctas, double* out) {
  double s[3];
  sum_partials<3>(part, 0, nctas, s);
  if (threadIdx.x == 0) {
    out[0] = s[0];
    out[1] = s[1];
    out[2] = s[2];
  }
}

__global__ void k_scale_real(const float* a, float* out, size_t N, float s) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] * s;
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return set_cuda_error(h, e_, #call); \
  } while (0)

cudaError_t glaunch_ev(mqnpm_handle* h, GreenCall c, cudaStream_t s, cudaEvent_t* ev) {
  c.ev = ev;
  c.launches = &h->launches;
  c.tile = h->tile;
  c.tmap = h->w.t2map;
  c.err = h->w.gerr;
  return green_launch(c, s);
}

// The pass timers cover the full applies only: a plane-input apply (the
// adjoint lift) skips most of passes 1-3 and a plane-output apply (first-Born
// data) most of passes 3-5, so counting their slots at the full algorithmic
// bytes would overstate the bandwidth figures.
cudaError_t glaunch(mqnpm_handle* h, GreenCall c, cudaStream_t s) {
  return glaunch_ev(h, c, s, (c.plane || c.outplane) ? nullptr : profile_slot(h, c.nb));
}

GreenCall base_call(mqnpm_handle* h, int nb, bool adjoint) {
  GreenCall c;
  c.nx = h->nx;
  c.ny = h->ny;
  c.nz = h->nz;
  c.nb = nb;
  c.adjoint = adjoint;
  c.T1 = h->w.T1;
  c.T2 = h->w.T2;
  c.khat = h->khat;
  c.twx = h->twx;
  c.twy = h->twy;
  c.twz = h->twz;
  c.st = nullptr;
  c.part_pro = h->w.part1;
  c.part_epi = h->w.part5;
  return c;
}

struct FinSArgs {
  KState* st;
  const double* part1;
  int nctas, nb;
};
cudaError_t fin_s_launch(void* ctx, cudaStream_t s) {
  const FinSArgs* a = static_cast<const FinSArgs*>(ctx);
  k_fin_s<<<a->nb, 256, 0, s>>>(a->st, a->part1, a->nctas);
  return cudaGetLastError();
}

// One BiCGSTAB iteration of the nb slots on stream s; evA and evB receive the
// pass boundaries of its two Green's applies (or are null).
int iteration_body(mqnpm_handle* h, int nb, const float* x, float2* xs, bool adjoint, cudaStream_t s,
                   cudaEvent_t* evA, cudaEvent_t* evB) {
  Workspace& w = h->w;
  const size_t N = h->N;
  GreenCall c = base_call(h, nb, adjoint);
  c.st = w.st;
  c.pro = PRO_BICG_P;
  c.pa.x = x;
  c.pa.xs = x ? nullptr : w.xslot;   // x == NULL: each slot's own contrast (shared launches)
  c.pa.w = w.p;
  c.pa.r = w.r;
  c.pa.v = w.v;
  c.epi = EPI_V;
  c.ea.out = w.v;
  c.ea.a = w.p;
  c.ea.rhat = w.rhat;
  CK(glaunch_ev(h, c, s, evA));
  k_fin_alpha<<<nb, 256, 0, s>>>(w.st, w.part5, w.ctas_row);
  c.pro = PRO_BICG_S;
  c.pa.w = w.s;
  c.epi = EPI_T;
  c.ea.out = w.t;
  c.ea.a = w.s;
  FinSArgs fs{w.st, w.part1, w.ctas_row, nb};
  c.after_pass1 = fin_s_launch;        // ||s|| from pass 1: retire converged slots before pass 2
  c.after_pass1_ctx = &fs;
  CK(glaunch_ev(h, c, s, evB));
  k_fin_omega<<<nb, 256, 0, s>>>(w.st, w.part1, w.part5, w.ctas_row);
  k_update<<<dim3(w.ctas_upd, nb), 256, 0, s>>>(w.st, xs, w.r, w.p, w.s, w.t, w.rhat, N, w.partu);
  CK(cudaMemsetAsync(w.nactive, 0, sizeof(int), s));
  k_fin_rho<<<nb, 256, 0, s>>>(w.st, w.partu, w.ctas_upd, h->krylov_maxit, w.nactive);
  CK(cudaGetLastError());
  h->launches += 4;   // fin_alpha, fin_omega, update, fin_rho
  return MQNPM_OK;
}

// The whole solve as one graph: a conditional WHILE node whose body is one
// BiCGSTAB iteration followed by k_loop_cond, so the iterations of all slots
// run without a host round trip; the caller reads the slot states once at the
// end.  Event records are not allowed in a conditional body, so this form is
// used only when the pass timers are off.
int loop_graph(mqnpm_handle* h, int nb, const float* x, float2* xs, bool adjoint, cudaGraphExec_t* exec_out,
               long long* kernels_out) {
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
  cudaGraphNode_t node = nullptr;
  cudaGraphNodeParams params = {};
  params.type = cudaGraphNodeTypeConditional;
  params.conditional.handle = cond;
  params.conditional.type = cudaGraphCondTypeWhile;
  params.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &params);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return set_cuda_error(h, e, "conditional node of the Krylov loop");
  }
  cudaGraph_t body = params.conditional.phGraph_out[0];
  cudaStream_t cs = h->capture_stream;
  const long long before = h->launches;
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  int rc = MQNPM_OK;
  if (e == cudaSuccess) {
    rc = iteration_body(h, nb, x, xs, adjoint, cs, nullptr, nullptr);
    k_loop_cond<<<1, 1, 0, cs>>>(cond, h->w.nactive, h->w.loops, h->krylov_maxit + 1);
    cudaGraph_t captured = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = ee;
  }
  *kernels_out = h->launches - before + 1;
  h->launches = before;
  if (rc == MQNPM_OK && e == cudaSuccess) e = cudaGraphInstantiate(exec_out, graph, 0);
  cudaGraphDestroy(graph);
  if (rc != MQNPM_OK) return rc;
  if (e != cudaSuccess) return set_cuda_error(h, e, "capture of the device-side Krylov loop");
  return MQNPM_OK;
}

void destroy_graph(KrylovGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (cudaEvent_t& e : g.ev)
    if (e) cudaEventDestroy(e);
  g = KrylovGraph{};
}

// The iteration of this batch shape as a replayable CUDA graph, captured on a
// private stream at first use (the caller's stream may be the legacy default
// stream, which cannot be captured).  The graph ends with the copy of the
// active-slot count to the host.
int iteration_graph(mqnpm_handle* h, int nb, const float* x, float2* xs, bool adjoint, bool loop,
                    KrylovGraph** out) {
  for (KrylovGraph& g : h->graphs)
    if (g.nb == nb && g.adjoint == adjoint && g.x == x && g.xs == xs && g.prof == h->prof.on && g.loop == loop) {
      *out = &g;
      return MQNPM_OK;
    }
  if (!h->capture_stream) CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  if (h->graphs.size() >= 8) {   // a few shapes at a time: drop the oldest
    destroy_graph(h->graphs.front());
    h->graphs.erase(h->graphs.begin());
  }
  KrylovGraph g;
  g.nb = nb;
  g.adjoint = adjoint;
  g.x = x;
  g.xs = xs;
  g.prof = h->prof.on;
  g.loop = loop;
  if (loop) {
    const int rc = loop_graph(h, nb, x, xs, adjoint, &g.exec, &g.kernels);
    if (rc != MQNPM_OK) {
      destroy_graph(g);
      return rc;
    }
    h->graphs.push_back(g);
    *out = &h->graphs.back();
    return MQNPM_OK;
  }
  if (g.prof)
    for (cudaEvent_t& e : g.ev) CK(cudaEventCreate(&e));
  cudaStream_t cs = h->capture_stream;
  const long long before = h->launches;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  int rc = iteration_body(h, nb, x, xs, adjoint, cs, g.prof ? g.ev : nullptr, g.prof ? g.ev + 6 : nullptr);
  cudaError_t e = cudaMemcpyAsync(h->w.h_nactive, h->w.nactive, sizeof(int), cudaMemcpyDeviceToHost, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  g.kernels = h->launches - before;
  h->launches = before;
  if (rc == MQNPM_OK && e == cudaSuccess && ee == cudaSuccess)
    e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != MQNPM_OK || e != cudaSuccess || ee != cudaSuccess) {
    destroy_graph(g);
    if (rc != MQNPM_OK) return rc;
    return set_cuda_error(h, e != cudaSuccess ? e : ee, "capture of the BiCGSTAB iteration");
  }
  h->graphs.push_back(g);
  *out = &h->graphs.back();
  return MQNPM_OK;
}

// Run BiCGSTAB iterations for the nb slots initialised by k_fin_init; the
// host reads the number of active slots after every iteration.
int krylov_iterate(mqnpm_handle* h, int nb, const float* x, float2* xs, bool adjoint) {
  Workspace& w = h->w;
  cudaStream_t s = h->stream;
  if (!h->direct_launches && !h->prof.on) {
    // the whole loop on the device: one graph launch, no host round trip
    KrylovGraph* g = nullptr;
    const int rc = iteration_graph(h, nb, x, xs, adjoint, true, &g);
    if (rc != MQNPM_OK) return rc;
    CK(cudaMemsetAsync(w.loops, 0, sizeof(int), s));
    CK(cudaGraphLaunch(g->exec, s));
    CK(cudaMemcpyAsync(w.h_loops, w.loops, sizeof(int), cudaMemcpyDeviceToHost, s));
    h->pending_loop_kernels = g->kernels;   // counted once the stream has been synchronised
    return MQNPM_OK;
  }
  if (!h->direct_launches) {
    KrylovGraph* g = nullptr;
    const int rc = iteration_graph(h, nb, x, xs, adjoint, false, &g);
    if (rc != MQNPM_OK) return rc;
    for (int it = 0; it < h->krylov_maxit; ++it) {
      CK(cudaGraphLaunch(g->exec, s));
      h->launches += g->kernels;
      CK(cudaStreamSynchronize(s));
      if (g->prof) {   // pass times of the two applies of this replay
        for (int a = 0; a < 2; ++a)
          for (int p = 0; p < 5; ++p) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, g->ev[6 * a + p], g->ev[6 * a + p + 1]));
            h->prof.acc_ms[p] += ms;
          }
        h->prof.acc_slots += 2 * (long long)nb;
        h->prof.acc_calls += 2;
      }
      if (*w.h_nactive == 0) break;
    }
    return MQNPM_OK;
  }
  for (int it = 0; it < h->krylov_maxit; ++it) {
    const int rc = iteration_body(h, nb, x, xs, adjoint, s, profile_slot(h, nb), profile_slot(h, nb));
    if (rc != MQNPM_OK) return rc;
    if ((it + 1) % h->check_every == 0 || it + 1 == h->krylov_maxit) {
      CK(cudaMemcpyAsync(w.h_nactive, w.nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*w.h_nactive == 0) break;
    }
  }
  return MQNPM_OK;
}

// Read back slot states; returns the worst status as an mqnpm code.
int collect_states(mqnpm_handle* h, int nb, int* iters_out, int stride, int offset) {
  std::vector<KState> ks(nb);
  cudaError_t e = cudaMemcpyAsync(ks.data(), h->w.st, nb * sizeof(KState), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return set_cuda_error(h, e, "collect_states");
  if (h->pending_loop_kernels) {   // kernels of the device-side loop: per pass times passes
    h->launches += h->pending_loop_kernels * (long long)*h->w.h_loops;
    h->pending_loop_kernels = 0;
  }
  int code = MQNPM_OK;
  for (int b = 0; b < nb; ++b) {
    if (iters_out) iters_out[b * stride + offset] = ks[b].iters;
    if (ks[b].status == KSTATUS_NONFINITE) code = MQNPM_ERR_NONFINITE;
    else if ((ks[b].status == KSTATUS_MAXIT || ks[b].status == KSTATUS_BREAKDOWN) && code == MQNPM_OK)
      code = MQNPM_ERR_NOT_CONVERGED;
  }
  return code;
}

}  // namespace

// Forward LS solve for nb slots: u = (I - G X)^{-1} u_in.  The staged tables
// of the chunk give each slot its start field (fwarm) and the place its
// converged field is kept (fstore); warm selects the warm-start form of the
// first residual.  forward_refine_steps (1 by default): a warm start u_0 is
// refined by fixed-point steps u_1 = u_0 + r_0 before BiCGSTAB (one more
// apply each; r_1 = G(x r_0) is smaller than r_0 by about the scattering
// strength, so a stored field from a nearby contrast then needs fewer
// BiCGSTAB iterations).  The stopping rule is ||r|| <= tol ||u_in|| either
// way.  x == NULL: each slot's own contrast (xslot).
static int forward_ls(mqnpm_handle* h, int nb, const float* x, bool warm, bool store, int* iters, int stride,
                      int offset) {
  Workspace& w = h->w;
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  GreenCall c = base_call(h, nb, false);
  c.pa.xs = x ? nullptr : w.xslot;
  if (warm) {
    // warm start: u_0 = the stored field (or u_in), r_0 = u_in - u_0 + G(x u_0)
    k_init_u_warm<<<dim3(w.ctas_vec, nb), 256, 0, s>>>(w.u, w.fwarm, h->tab, w.illum, h->dims(), N);
    c.pro = PRO_CONTRAST;
    c.pa.x = x;
    c.pa.q = w.u;
    c.epi = EPI_INIT_WARM;
    c.ea.a = w.u;
    c.ea.tab = h->tab;
    c.ea.illum = w.illum;
  } else {
    k_init_uin<<<dim3(w.ctas_vec, nb), 256, 0, s>>>(w.u, h->tab, w.illum, h->dims(), N);
    c.pro = PRO_BORN;                    // r_0 = u_in - A u_in = G(x u_in)
    c.pa.x = x;
    c.pa.tab = h->tab;
    c.pa.illum = w.illum;
    c.epi = EPI_INIT;
  }
  c.ea.out = w.r;
  c.ea.out2 = w.rhat;
  CK(glaunch(h, c, s));
  k_fin_init<<<nb, 256, 0, s>>>(w.st, w.part5, w.ctas_row, h->krylov_tol * h->krylov_tol, (double)N, 0);
  CK(cudaGetLastError());
  h->launches += 2;   // init, fin_init
  for (int step = 0; warm && step < h->forward_refine_steps; ++step) {
    // a fixed-point step on the slots still above the tolerance:
    // u_1 = u_0 + r_0, r_1 = u_in - (I - G X) u_1 = G(x r_0), in place in r
    k_add_residual<<<dim3(w.ctas_vec, nb), 256, 0, s>>>(w.u, w.r, w.st, N);
    GreenCall c1 = base_call(h, nb, false);
    c1.st = w.st;                        // slots already converged are skipped
    c1.pro = PRO_CONTRAST;
    c1.pa.x = x;
    c1.pa.xs = x ? nullptr : w.xslot;
    c1.pa.q = w.r;
    c1.epi = EPI_INIT;
    c1.ea.out = w.r;
    c1.ea.out2 = w.rhat;
    CK(glaunch(h, c1, s));
    k_fin_init<<<nb, 256, 0, s>>>(w.st, w.part5, w.ctas_row, h->krylov_tol * h->krylov_tol, -1.0, 1);
    CK(cudaGetLastError());
    h->launches += 2;   // add_residual, fin_init
  }
  int rc = krylov_iterate(h, nb, x, w.u, false);
  if (rc != MQNPM_OK) return rc;
  if (store) {
    k_store_field<<<dim3(w.ctas_vec, nb), 256, 0, s>>>(w.fstore, w.u, N);
    CK(cudaGetLastError());
    h->launches += 1;
  }
  return collect_states(h, nb, iters, stride, offset);
}

// Adjoint solve for nb slots: z = (I - G^H X)^{-1} b, b = G^H S^T r_det.
// adjoint_from_b: started at z_0 = b (the first term of z's Neumann series,
// as u_in starts a cold forward solve): r_0 = b - (I - G^H X) b = G^H (x b),
// one more apply that saves about one BiCGSTAB iteration (two applies) at
// contrasts up to about 0.04.  Otherwise started at z_0 = 0 (r_0 = b).  The
// stopping rule is ||r|| <= tol ||b|| either way.
static int adjoint_ls(mqnpm_handle* h, int nb, const float* x, int* iters, int stride, int offset) {
  Workspace& w = h->w;
  cudaStream_t s = h->stream;
  if (!h->adjoint_from_b) CK(cudaMemsetAsync(w.zs, 0, (size_t)nb * h->N * sizeof(float2), s));
  GreenCall c = base_call(h, nb, true);
  c.pro = PRO_LIFT;
  c.plane = true;                      // S^T r: nonzero on the detector plane only
  c.pa.rdet = w.rdet;
  if (h->remote) {                     // S^T D^H r_det
    CK(detector_adjoint(h, w.rdet, w.rlift, nb));
    c.pa.rdet = w.rlift;
  }
  if (!h->adjoint_from_b) {            // r_0 = b = G^H S^T r_det (start z_0 = 0)
    c.epi = EPI_INIT;
    c.ea.out = w.r;
    c.ea.out2 = w.rhat;
    CK(glaunch(h, c, s));
    k_fin_init<<<nb, 256, 0, s>>>(w.st, w.part5, w.ctas_row, h->krylov_tol * h->krylov_tol, 0.0, 0);
    CK(cudaGetLastError());
    h->launches += 1;
    const int rc = krylov_iterate(h, nb, x, w.zs, true);
    if (rc != MQNPM_OK) return rc;
    return collect_states(h, nb, iters, stride, offset);
  }
  c.epi = EPI_INIT;                    // z_0 = b = G^H S^T r_det, and ||b||^2
  c.ea.out = w.zs;
  c.ea.out2 = w.rhat;
  CK(glaunch(h, c, s));
  k_set_bnorm<<<nb, 256, 0, s>>>(w.st, w.part5, w.ctas_row);
  GreenCall c0 = base_call(h, nb, true);
  c0.pro = PRO_CONTRAST;               // r_0 = G^H (x z_0)
  c0.pa.x = x;
  c0.pa.xs = x ? nullptr : w.xslot;
  c0.pa.q = w.zs;
  c0.epi = EPI_INIT;
  c0.ea.out = w.r;
  c0.ea.out2 = w.rhat;
  CK(glaunch(h, c0, s));
  k_fin_init<<<nb, 256, 0, s>>>(w.st, w.part5, w.ctas_row, h->krylov_tol * h->krylov_tol, -1.0, 0);
  CK(cudaGetLastError());
  h->launches += 2;
  int rc = krylov_iterate(h, nb, x, w.zs, true);
  if (rc != MQNPM_OK) return rc;
  return collect_states(h, nb, iters, stride, offset);
}


// Stage the per-slot tables of one chunk (pinned staging, then the device
// copies): illuminations, contrasts (shared launches only), warm-start and
// store fields, gradient segments.  Waits for the previous chunk's copies.
int stage_chunk(mqnpm_handle* h, const ChunkTables& t) {
  Workspace& w = h->w;
  const int m = t.m;
  if (m < 1 || m > h->max_batch || (int)t.segs.size() < 1 || (int)t.segs.size() > m)
    return set_error(h, MQNPM_ERR_INVALID_ARG, "stage_chunk: bad chunk");
  CK(cudaStreamSynchronize(h->stream));
  for (int b = 0; b < m; ++b) {
    w.h_illum[b] = t.illum[b];
    w.h_xslot[b] = t.x.empty() ? nullptr : t.x[b];
    w.h_fwarm[b] = t.warm.empty() ? nullptr : t.warm[b];
    w.h_fstore[b] = t.store.empty() ? nullptr : t.store[b];
  }
  for (size_t q = 0; q < t.segs.size(); ++q) w.h_segs[q] = t.segs[q];
  cudaStream_t s = h->stream;
  CK(cudaMemcpyAsync(w.illum, w.h_illum, m * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.xslot, w.h_xslot, m * sizeof(const float*), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.fwarm, w.h_fwarm, m * sizeof(float2*), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.fstore, w.h_fstore, m * sizeof(float2*), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.segs, w.h_segs, t.segs.size() * sizeof(GradSeg), cudaMemcpyHostToDevice, s));
  return MQNPM_OK;
}

namespace {

// The tables of chunk [c0, c0 + m) of one handle's illumination list: every
// slot reads the handle's contrast, the handle's stored fields (warm start)
// and adds into one gradient.
ChunkTables handle_chunk(mqnpm_handle* h, const int* illum, int c0, int m, double scale, float* grad) {
  ChunkTables t;
  t.m = m;
  t.illum.assign(illum + c0, illum + c0 + m);
  if (h->ufield) {
    t.warm.resize(m);
    t.store.resize(m);
    for (int b = 0; b < m; ++b) {
      const int l = t.illum[b];
      t.store[b] = h->ufield + (size_t)l * h->N;
      t.warm[b] = h->have_field[l] ? t.store[b] : nullptr;
    }
  }
  t.segs.push_back(GradSeg{0, m, c0 > 0 ? 1 : 0, (float)scale, grad});
  return t;
}

}  // namespace

// Forward fields and detector residuals of one staged chunk (slots [0, m));
// the residual norm of segment q lands in w.h_scal[q] after the next
// synchronisation (nseg > 1 only for LS without a remote detector).
int chunk_forward(mqnpm_handle* h, const float* x, int m, int* it_chunk, float2* det_out, const float2* ym,
                  bool warm, bool store, const std::vector<GradSeg>& segs) {
  Workspace& w = h->w;
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  int worst = MQNPM_OK;
  int parts = m * w.ctas_row;          // detector partials to sum
  const int nseg = (int)segs.size();
  if (nseg > 1 && (h->model != MQNPM_MODEL_LS || h->remote))
    return set_error(h, MQNPM_ERR_UNSUPPORTED, "per-segment losses need the LS model and the slice detector");
  if (h->model == MQNPM_MODEL_LS) {
    int rc = forward_ls(h, m, x, warm, store, it_chunk, 2, 0);
    if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE) return rc;
    if (rc != MQNPM_OK) worst = rc;
    k_detect_ls<<<dim3(w.ctas_row, m), 256, 0, s>>>(w.u, h->tab, w.illum, h->remote ? nullptr : ym, det_out,
                                                     h->dims(), N, w.partd);
  } else {
    GreenCall c = base_call(h, m, false);
    c.pro = PRO_BORN;
    c.outplane = true;                 // only the detector plane of G(x u_in) is used
    c.pa.x = x;
    c.pa.xs = x ? nullptr : w.xslot;
    c.pa.tab = h->tab;
    c.pa.illum = w.illum;
    c.epi = EPI_DETECT;
    c.ea.out2 = det_out;
    c.ea.ymeas = h->remote ? nullptr : ym;
    c.ea.illum = w.illum;
    c.part_epi = w.partd;
    CK(glaunch(h, c, s));
    parts = m * green_plane_ctas(h->nx, h->ny, h->tile);   // the plane pass 5 writes fewer partials
  }
  CK(cudaGetLastError());
  if (h->remote) {                     // D(slice) - y; the partials are rewritten per row CTA
    CK(detector_forward(h, det_out, m, ym, w.illum));
    parts = m * w.ctas_row;
  }
  if (nseg == 1) {
    k_sum_all<<<1, 256, 0, s>>>(w.partd, parts, w.dscal);
  } else {   // LS: partials [slot][ctas_row], one sum per segment of slots
    for (int q = 0; q < nseg; ++q)
      k_sum_all<<<1, 256, 0, s>>>(w.partd + (size_t)segs[q].b0 * w.ctas_row, (segs[q].b1 - segs[q].b0) * w.ctas_row,
                                  w.dscal + q);
  }
  CK(cudaMemcpyAsync(w.h_scal, w.dscal, nseg * sizeof(double), cudaMemcpyDeviceToHost, s));
  h->launches += (h->model == MQNPM_MODEL_LS ? 1 : 0) + nseg;
  return worst;
}


// Adjoint solves and gradient assembly of one staged chunk from the fields
// and residuals in the workspace (into the staged gradient segments).
int chunk_adjoint(mqnpm_handle* h, const float* x, int m, int* it_chunk, int nseg) {
  Workspace& w = h->w;
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  int worst = MQNPM_OK;
  if (h->model == MQNPM_MODEL_LS) {
    int rc = adjoint_ls(h, m, x, it_chunk, 2, 1);
    if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE) return rc;
    if (rc != MQNPM_OK) worst = rc;
    k_grad_seg<<<dim3(w.ctas_vec, nseg), 256, 0, s>>>(w.u, w.zs, h->tab, w.illum, h->dims(), N, w.segs);
  } else {
    GreenCall c = base_call(h, m, true);
    c.pro = PRO_LIFT;
    c.plane = true;
    c.pa.rdet = w.rdet;
    if (h->remote) {
      CK(detector_adjoint(h, w.rdet, w.rlift, m));
      c.pa.rdet = w.rlift;
    }
    c.epi = EPI_PLAIN;
    c.ea.out = w.zs;
    CK(glaunch(h, c, s));
    k_grad_seg<<<dim3(w.ctas_vec, nseg), 256, 0, s>>>(nullptr, w.zs, h->tab, w.illum, h->dims(), N, w.segs);
  }
  CK(cudaGetLastError());
  h->launches += 1;
  return worst;
}

int check_tile_waits(mqnpm_handle* h) {
  int gerr = 0;
  CK(cudaMemcpy(&gerr, h->w.gerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (gerr) return set_error(h, MQNPM_ERR_TIMEOUT, "a bounded wait for a transform tile load gave up");
  return MQNPM_OK;
}


int grad_batch_impl(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, float* grad,
                    double* loss, int* iters, bool want_grad, float2* y_out) {
  Workspace& w = h->w;
  const size_t M = (size_t)h->M;
  double total = 0.0;
  int worst = MQNPM_OK;
  h->fields_valid = false;
  h->last_iters.assign(2 * nb, 0);
  for (int c0 = 0; c0 < nb; c0 += h->max_batch) {
    const int m = std::min(h->max_batch, nb - c0);
    const ChunkTables t = handle_chunk(h, illum, c0, m, scale, grad);
    int rc = stage_chunk(h, t);
    if (rc != MQNPM_OK) return rc;
    int* it_chunk = h->last_iters.data() + 2 * c0;
    float2* det_out = y_out ? y_out + (size_t)c0 * M : w.rdet;
    const float2* ym = y_out ? nullptr : h->ymeas;
    rc = chunk_forward(h, x, m, it_chunk, det_out, ym, h->ufield != nullptr, h->ufield != nullptr, t.segs);
    if (h->ufield)
      for (int b = 0; b < m; ++b) h->have_field[t.illum[b]] = (rc == MQNPM_ERR_NONFINITE) ? 0 : 1;
    if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE) return rc;
    if (rc != MQNPM_OK) worst = rc;
    if (!y_out && want_grad) {
      rc = chunk_adjoint(h, x, m, it_chunk, 1);
      if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE) return rc;
      if (rc != MQNPM_OK) worst = rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    total += 0.5 * w.h_scal[0];
  }
  if (loss) *loss = scale * total;
  if (iters) std::memcpy(iters, h->last_iters.data(), 2 * nb * sizeof(int));
  const int rc = check_tile_waits(h);
  return rc != MQNPM_OK ? rc : worst;
}

// Data term without the gradient; a single chunk keeps its fields for
// grad_fields_impl.
int loss_batch_impl(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, double* loss,
                    int* iters) {
  const int rc = grad_batch_impl(h, x, illum, nb, scale, nullptr, loss, nullptr, false, nullptr);
  if (iters)
    for (int b = 0; b < nb; ++b) iters[b] = h->last_iters[2 * b];
  if ((rc == MQNPM_OK || rc == MQNPM_ERR_NOT_CONVERGED) && nb <= h->max_batch) {
    h->fields_valid = true;
    h->fields_x = x;
    h->fields_illum.assign(illum, illum + nb);
  }
  return rc;
}

// Gradient of the data term, reusing the fields of the last loss_batch_impl
// when allowed and they match (same x pointer and illuminations).
int grad_fields_impl(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, float* grad,
                     bool reuse, int* reused) {
  const bool match = reuse && h->fields_valid && h->fields_x == x && (int)h->fields_illum.size() == nb &&
                     std::equal(illum, illum + nb, h->fields_illum.begin());
  if (reused) *reused = match ? 1 : 0;
  if (!match) return grad_batch_impl(h, x, illum, nb, scale, grad, nullptr, nullptr, true, nullptr);
  h->fields_valid = false;   // the adjoint solve reuses the Krylov workspace
  std::vector<int> it(2 * nb, 0);
  int rc = stage_chunk(h, handle_chunk(h, illum, 0, nb, scale, grad));
  if (rc != MQNPM_OK) return rc;
  rc = chunk_adjoint(h, x, nb, it.data(), 1);
  if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE) return rc;
  CK(cudaStreamSynchronize(h->stream));
  const int rt = check_tile_waits(h);
  return rt != MQNPM_OK ? rt : rc;
}

cudaError_t vec_reduce(mqnpm_handle* h, int /*kind*/, const float* a, const float* b, const float* c,
                       const float* d, double* host_out) {
  cudaStream_t s = h->stream;
  const int ctas = h->w.ctas_vec;
  k_dots3<<<ctas, 256, 0, s>>>(a, b, c, d, h->N, h->w.partu);
  k_sum3<<<1, 256, 0, s>>>(h->w.partu, ctas, h->w.dscal);
  h->launches += 2;
  cudaError_t e = cudaMemcpyAsync(h->w.h_scal, h->w.dscal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) std::memcpy(host_out, h->w.h_scal, 3 * sizeof(double));
  return e;
}

int lipschitz_impl(mqnpm_handle* h, const int* illum, int nb, double scale, const float* start, int iters,
                   double* alpha_out) {
  Workspace& w = h->w;
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  float* q = h->vq;   // current unit vector
  float* a = h->g;    // operator output
  double d3[3];
  h->fields_valid = false;   // the power steps reuse the slot workspace
  CK(vec_reduce(h, 0, start, nullptr, nullptr, nullptr, d3));
  if (!(d3[0] > 0.0)) return set_error(h, MQNPM_ERR_INVALID_ARG, "lipschitz: zero start vector");
  k_scale_real<<<w.ctas_vec, 256, 0, s>>>(start, q, N, (float)(1.0 / std::sqrt(d3[0])));
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    for (int c0 = 0; c0 < nb; c0 += h->max_batch) {
      const int m = std::min(h->max_batch, nb - c0);
      CK(cudaStreamSynchronize(s));
      for (int b = 0; b < m; ++b) w.h_illum[b] = illum[c0 + b];
      CK(cudaMemcpyAsync(w.illum, w.h_illum, m * sizeof(int), cudaMemcpyHostToDevice, s));
      GreenCall c = base_call(h, m, false);
      c.pro = PRO_BORN;                 // S G (q u_in)
      c.outplane = true;
      c.pa.x = q;
      c.pa.tab = h->tab;
      c.pa.illum = w.illum;
      c.epi = EPI_DETECT;
      c.ea.out2 = w.rdet;
      c.ea.ymeas = nullptr;
      c.ea.illum = w.illum;
      c.part_epi = w.partd;
      CK(glaunch(h, c, s));
      GreenCall c2 = base_call(h, m, true);
      c2.pro = PRO_LIFT;                // G^H S^T (.)
      c2.plane = true;
      c2.pa.rdet = w.rdet;
      if (h->remote) {                  // J = D S G(. u_in): D, then D^H before the lift
        CK(detector_forward(h, w.rdet, m, nullptr, w.illum));
        CK(detector_adjoint(h, w.rdet, w.rlift, m));
        c2.pa.rdet = w.rlift;
      }
      c2.epi = EPI_PLAIN;
      c2.ea.out = w.zs;
      CK(glaunch(h, c2, s));
      k_grad<<<w.ctas_vec, 256, 0, s>>>(nullptr, w.zs, h->tab, w.illum, m, h->dims(), N, (float)scale, a, c0 > 0);
      CK(cudaGetLastError());
    }
    CK(vec_reduce(h, 0, q, nullptr, a, nullptr, d3));   // <q,q>, <q,a>, <a,a>
    lam = d3[1] / d3[0];
    if (!(d3[2] > 0.0)) break;
    k_scale_real<<<w.ctas_vec, 256, 0, s>>>(a, q, N, (float)(1.0 / std::sqrt(d3[2])));
  }
  *alpha_out = lam;
  return MQNPM_OK;
}
