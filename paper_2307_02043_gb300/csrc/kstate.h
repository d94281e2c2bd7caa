// Device-resident state of one BiCGSTAB solve (one slot of a mini-batch) and
// the argument blocks of the fused Green's-apply prologues/epilogues.
#pragma once
#include <cuda_runtime.h>

struct KState {
  double rho_re, rho_im;        // rho_i = <rhat, r_{i-1}>
  double alpha_re, alpha_im;
  double omega_re, omega_im;
  double beta_re, beta_im;
  double bnorm2;                // ||b||^2
  double rnorm2;                // ||r||^2 (recursive residual)
  double tol2;                  // tol^2
  int active;                   // 1 while iterating; 2 from the half step that met the
                                // tolerance to the end of that iteration
  int iters;
  int status;                   // KSTATUS_*
  int conv_pending;             // ||s|| met the tolerance in this iteration
};

enum {
  KSTATUS_RUNNING = 0,
  KSTATUS_CONVERGED = 1,
  KSTATUS_BREAKDOWN = 2,
  KSTATUS_MAXIT = 3,
  KSTATUS_NONFINITE = 4,
};

// What pass 1 feeds into the transform.
enum ProKind {
  PRO_PLAIN = 0,     // q[b]
  PRO_CONTRAST = 1,  // x * q[b]
  PRO_BORN = 2,      // x * u_in(l_b)
  PRO_BICG_P = 3,    // p = r + beta (p - omega v); write p; x * p
  PRO_BICG_S = 4,    // s = r - alpha v; write s; x * s; partial ||s||^2
  PRO_LIFT = 5,      // S^T r_det (last z-slice)
};
// What pass 5 does with g = (G q)(voxel).
enum EpiKind {
  EPI_PLAIN = 0,        // out[b] = g
  EPI_V = 1,            // v = p - g; partial <rhat, v>
  EPI_T = 2,            // t = s - g; partials <t, s>, ||t||^2
  EPI_INIT = 3,         // r = rhat = g; partial ||g||^2
  EPI_DETECT = 4,       // z = n-1: r_det = g - y_meas(l_b); partial ||r_det||^2
  EPI_INIT_WARM = 5,    // r = rhat = u_in(l_b) - u + g (start u); partial ||r||^2
};

struct ProArgs {
  const float* x;        // contrast (N), shared by every slot
  const float* const* xs;  // or per slot: contrast of slot b's volume (when non-null)
  const float2* q;       // input vector [b][N]
  float2* w;             // vector written by the prologue [b][N]
  const float2* r;       // [b][N]
  const float2* v;       // [b][N]
  const float2* tab;     // incident-field axis tables [l][3][n]
  const int* illum;      // illumination index of slot b
  const float2* rdet;    // [b][n*n]
};

struct EpiArgs {
  float2* out;           // [b][N]
  const float2* a;       // p or s [b][N]
  const float2* rhat;    // [b][N]
  float2* out2;          // second output (rhat for EPI_INIT, r_det for EPI_DETECT)
  const float2* ymeas;   // [L][n*n]
  const int* illum;
  const float2* tab;     // incident-field axis tables [l][3][n]
};

// One run of consecutive slots whose gradients add into one output (the
// illuminations of one volume): grad (+)= scale * sum_{b0 <= b < b1} Re(conj(u_b) z_b).
struct GradSeg {
  int b0, b1;
  int accumulate;        // add to grad (1) or overwrite it (0)
  float scale;
  float* grad;
};
