// The whole weighted proximal mapping (Eq. 4.4) as one cooperative kernel.
//
// Phases, separated by grid-wide barriers (deterministic reductions: the last
// block to arrive sums the per-block partials in block order and releases the
// others; every wait is bounded):
//   G  (U != 0, once)  G = U^T U, U^T v; every block forms M = (I + G/tau)^{-1}.
//   per dual iteration j = 1..J, then once more on P_J:
//   A  d = d(R) and U^T d              -> gamma = (c/tau^2) M U^T d   (Woodbury)
//   N  semi-smooth Newton on phi(beta) = U^T(w - clip(w - U beta/tau)) + beta
//      (Theorem 3.1, Algorithm 4.3): each evaluation also writes
//      x = clip(w - U beta/tau) speculatively, so the accepted evaluation leaves x.
//   X  (U = 0) x = clip(v - (c/tau) d(R))
//   D  P_j = Proj(R_j + tau/(4 D c) grad x),  R_{j+1} = P_j + mom_j (P_j - P_{j-1})
// At 128^3 the working set (v, d, x, U, R, P) stays resident in the 129 MB L2
// across phases, so most of the traffic after the first touch is L2 traffic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

namespace {

constexpr int WP_THREADS = 256;
constexpr int NVMAX = 44;     // S + S(S+1)/2 for S = 8
constexpr int ILP_FOR(int S) { return S <= 4 ? 4 : 1; }

struct WpArgs {
  const float* v;
  UPtrs U;
  float* R;
  float* Pd;
  float* d;
  float* x;
  float* xout;
  const float* mom;
  double* part;       // [gridDim.x][NVMAX]
  double* tot;        // [NVMAX]
  unsigned* count;    // arrivals (monotonic)
  unsigned* gen;      // released barrier generation
  int* err;
  double* stat;       // [0] last newton count, [1] max, [2] total, [3] evaluations
  int n, N, J;
  double tau, c;
  float lo, hi, step;
  double tol;
  int maxit;
  long long limit;
  long long* trace;   // optional: (phase tag, ns) after every barrier, recorded by block 0
  int trace_cap;
};

MQ_D float clampf(float a, float lo, float hi) { return fminf(fmaxf(a, lo), hi); }

MQ_D void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier with an optional sum of NV doubles per block (held in blk[]
// by thread 0).  The totals land in sh_tot (shared) for every thread.
MQ_D long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Partials are stored value-major, part[k * gridDim.x + b], so that the last
// block reads each value's partials with coalesced, independent loads: warp w
// reduces the values k = w, w + nwarps, ... (lane sums a fixed stripe of
// blocks, then a fixed shuffle tree), which keeps the order deterministic.
template <int NV>
MQ_D bool grid_reduce(const double* blk, double* sh_tot, const WpArgs& a, unsigned& epoch, int tag) {
  __shared__ int s_last, s_ok;
  __syncthreads();
  if (threadIdx.x < NV) a.part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = blk[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(a.count, 1u);
    s_last = (old == (epoch + 1) * gridDim.x - 1) ? 1 : 0;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    if constexpr (NV > 0) {
      __threadfence();
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const int nb = gridDim.x;
      for (int k = warp; k < NV; k += nw) {
        const double* p = a.part + (size_t)k * nb;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int b = lane;
        for (; b + 96 < nb; b += 128) {
          a0 += __ldcg(p + b);
          a1 += __ldcg(p + b + 32);
          a2 += __ldcg(p + b + 64);
          a3 += __ldcg(p + b + 96);
        }
        for (; b < nb; b += 32) a0 += __ldcg(p + b);
        const double s = warp_sum((a0 + a1) + (a2 + a3));
        if (lane == 0) a.tot[k] = s;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_u32(a.gen, epoch + 1);
    }
  } else if (threadIdx.x == 0) {
    const long long t0 = clock64();
    while (ld_acquire_u32(a.gen) < epoch + 1) {
      if (*((volatile int*)a.err) != 0) { s_ok = 0; break; }
      if (clock64() - t0 > a.limit) { atomicExch(a.err, 1); s_ok = 0; break; }
      __nanosleep(32);
    }
  }
  __syncthreads();
  epoch += 1;
  if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && (int)epoch < a.trace_cap) {
    a.trace[2 * epoch] = tag;
    a.trace[2 * epoch + 1] = globaltimer();
  }
  if (!s_ok) return false;
  if constexpr (NV > 0) {
    if (threadIdx.x < NV) sh_tot[threadIdx.x] = __ldcg(a.tot + threadIdx.x);
    __syncthreads();
  }
  return true;
}

MQ_D void coords(int i, int n, int& x, int& y, int& z) {
  const int r = i / n;
  x = i - r * n;
  z = r / n;
  y = r - z * n;
}

// d(R) at voxel i = (x, y, z): sum_d q_d(i - e_d)[i_d >= 1] - q_d(i)[i_d <= n-2]
MQ_D float div_at(const float* __restrict__ R, int N, int n, int i, int x, int y, int z) {
  const float* qx = R;
  const float* qy = R + N;
  const float* qz = R + 2 * (size_t)N;
  float s = 0.f;
  if (x > 0) s += qx[i - 1];
  if (x < n - 1) s -= qx[i];
  if (y > 0) s += qy[i - n];
  if (y < n - 1) s -= qy[i];
  if (z > 0) s += qz[i - n * n];
  if (z < n - 1) s -= qz[i];
  return s;
}

template <int TV>
MQ_D void project(float& px, float& py, float& pz) {
  if constexpr (TV == MQNPM_TV_ISO) {
    const float nr2 = px * px + py * py + pz * pz;
    if (nr2 > 1.f) {
      const float s = rsqrtf(nr2);
      px *= s; py *= s; pz *= s;
    }
  } else {
    px = clampf(px, -1.f, 1.f);
    py = clampf(py, -1.f, 1.f);
    pz = clampf(pz, -1.f, 1.f);
  }
}

template <int S>
MQ_D bool chol_solve(double (&A)[S * S], double (&b)[S]) {
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

// M = (I + G/tau)^{-1} column by column (S x S, FP64).  Called by one thread;
// kept out of line so its scratch does not cost the streaming loops registers.
template <int S>
__device__ __noinline__ void form_woodbury(const double* G, double tau, double* M) {
  for (int col = 0; col < S; ++col) {
    double A[S * S], e[S];
    for (int i = 0; i < S; ++i)
      for (int j = 0; j < S; ++j) A[i * S + j] = (i == j ? 1.0 : 0.0) + G[i * S + j] / tau;
    for (int i = 0; i < S; ++i) e[i] = (i == col) ? 1.0 : 0.0;
    chol_solve<S>(A, e);
    for (int i = 0; i < S; ++i) M[i * S + col] = e[i];
  }
}

// State of one semi-smooth Newton solve, held in shared memory.
template <int S>
struct NewtonState {
  double* beta;        // accepted iterate
  double* beta_eval;   // point evaluated by the next pass
  double* dir;         // Newton direction from beta
  double* phi_cur;     // phi(beta)
  double* nphi_cur;
  double* tstep;
  int* halvings;
  int* accepted;
  bool* first;
  int* accepted_last;
};

// One decision of Algorithm 4.3 after phi and H were evaluated at beta_eval
// (tot = [phi - beta_eval (S values), upper triangle of U^T diag(inner) U]).
// Accept the trial if it reduces ||phi|| (or halving is exhausted), stop at
// ||phi|| <= tol_abs, else take the Newton step H^{-1} phi from the accepted
// point; a rejected trial is halved.  Returns 1 when the solve is finished.
template <int S>
__device__ __noinline__ int newton_decide(NewtonState<S> ns, const double* tot, double tau, double tol_abs, int maxit,
                                          bool out_of_evals) {
  double phi[S], nphi = 0.0;
  for (int s = 0; s < S; ++s) {
    phi[s] = tot[s] + ns.beta_eval[s];
    nphi += phi[s] * phi[s];
  }
  nphi = sqrt(nphi);
  const bool accept = *ns.first || nphi < *ns.nphi_cur || *ns.halvings >= 30 || !isfinite(*ns.nphi_cur);
  *ns.first = false;
  *ns.accepted_last = accept ? 1 : 0;
  if (!accept) {
    *ns.tstep *= 0.5;
    *ns.halvings += 1;
    for (int s = 0; s < S; ++s) ns.beta_eval[s] = ns.beta[s] + *ns.tstep * ns.dir[s];
    return out_of_evals ? 1 : 0;
  }
  for (int s = 0; s < S; ++s) {
    ns.beta[s] = ns.beta_eval[s];
    ns.phi_cur[s] = phi[s];
  }
  *ns.nphi_cur = nphi;
  if (nphi <= tol_abs || *ns.accepted >= maxit || out_of_evals || !isfinite(nphi)) return 1;
  double H[S * S];
  int k = S;
  for (int s = 0; s < S; ++s)
    for (int t = s; t < S; ++t) {
      const double hst = tot[k++] / tau + (s == t ? 1.0 : 0.0);
      H[s * S + t] = hst;
      H[t * S + s] = hst;
    }
  double rhs[S];
  for (int s = 0; s < S; ++s) rhs[s] = -phi[s];
  if (!chol_solve<S>(H, rhs)) return 1;
  for (int s = 0; s < S; ++s) {
    ns.dir[s] = rhs[s];
    ns.beta_eval[s] = ns.beta[s] + rhs[s];
  }
  *ns.tstep = 1.0;
  *ns.halvings = 0;
  *ns.accepted += 1;
  return 0;
}

// Block-level sum of K floats per thread into thread 0's out[] (FP64).
template <int K>
MQ_D void block_partial(const float (&acc)[K], double (&out)[K]) {
  __shared__ double scratch[33 * (K > 0 ? K : 1)];
  block_sum_f<K>(acc, scratch, out);
}

template <int S, int TV>
__global__ void __launch_bounds__(WP_THREADS, 2) k_wprox(WpArgs a) {
  constexpr int NG = S * (S + 1) / 2;
  constexpr int NV = S + NG;
  constexpr int ILP = ILP_FOR(S);
  __shared__ double sG[S > 0 ? S * S : 1], sM[S > 0 ? S * S : 1], sUv[S > 0 ? S : 1];
  __shared__ double sGamma[S > 0 ? S : 1], sUtw[S > 0 ? S : 1], sBeta[S > 0 ? S : 1], sBetaEval[S > 0 ? S : 1];
  __shared__ double sTot[NVMAX];
  __shared__ float sTheta[S > 0 ? S : 1], sGam[S > 0 ? S : 1];
  __shared__ int sDone, sAcceptedLast;
  __shared__ double sScale;
  const int n = a.n, N = a.N;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const float cdt = (float)(a.c / a.tau);
  unsigned epoch = 0;
  __shared__ double blk[NVMAX];
  if (a.trace && blockIdx.x == 0 && threadIdx.x == 0) a.trace[1] = globaltimer();

  // ---------------------------------------------------------------- phase G
  if constexpr (S > 0) {
    float acc[NG + S];
#pragma unroll
    for (int k = 0; k < NG + S; ++k) acc[k] = 0.f;
    for (int i0 = tid; i0 < N; i0 += ILP * stride) {
#pragma unroll
      for (int q = 0; q < ILP; ++q) {
        const int i = i0 + q * stride;
        if (i < N) {
          float u[S];
#pragma unroll
          for (int s = 0; s < S; ++s) u[s] = a.U.u[s][i];
          const float vi = a.v[i];
          int k = 0;
#pragma unroll
          for (int s = 0; s < S; ++s)
#pragma unroll
            for (int t = s; t < S; ++t) {
              acc[k] = fmaf(u[s], u[t], acc[k]);
              ++k;
            }
#pragma unroll
          for (int s = 0; s < S; ++s) acc[NG + s] = fmaf(u[s], vi, acc[NG + s]);
        }
      }
    }
    double o[NG + S];
    block_partial<NG + S>(acc, o);
    if (threadIdx.x == 0)
      for (int k = 0; k < NG + S; ++k) blk[k] = o[k];
    if (!grid_reduce<NG + S>(blk, sTot, a, epoch, 1)) return;
    if (threadIdx.x == 0) {
      int k = 0;
      for (int s = 0; s < S; ++s)
        for (int t = s; t < S; ++t) {
          sG[s * S + t] = sTot[k];
          sG[t * S + s] = sTot[k];
          ++k;
        }
      for (int s = 0; s < S; ++s) sUv[s] = sTot[NG + s];
      form_woodbury<S>(sG, a.tau, sM);
      for (int s = 0; s < S; ++s) sBeta[s] = 0.0;
    }
    __syncthreads();
  }

  int newton_max = 0, newton_total = 0, evals = 0, last_newton = 0;
  for (int j = 0; j <= a.J; ++j) {
    const bool final_eval = (j == a.J);
    const float* src = final_eval ? a.Pd : a.R;
    float* xw = final_eval ? a.xout : a.x;
    if constexpr (S == 0) {
      // ------------------------------------------------------------ phase X
      for (int i0 = tid; i0 < N; i0 += ILP * stride) {
#pragma unroll
        for (int q = 0; q < ILP; ++q) {
          const int i = i0 + q * stride;
          if (i < N) {
            int x, y, z;
            coords(i, n, x, y, z);
            xw[i] = clampf(a.v[i] - cdt * div_at(src, N, n, i, x, y, z), a.lo, a.hi);
          }
        }
      }
      if (!final_eval && !grid_reduce<0>(nullptr, nullptr, a, epoch, 2)) return;
    } else {
      // ------------------------------------------------------------ phase A
      {
        float acc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = 0.f;
        for (int i0 = tid; i0 < N; i0 += ILP * stride) {
#pragma unroll
          for (int q = 0; q < ILP; ++q) {
            const int i = i0 + q * stride;
            if (i < N) {
              int x, y, z;
              coords(i, n, x, y, z);
              const float dd = div_at(src, N, n, i, x, y, z);
              a.d[i] = dd;
#pragma unroll
              for (int s = 0; s < S; ++s) acc[s] = fmaf(a.U.u[s][i], dd, acc[s]);
            }
          }
        }
        double o[S];
        block_partial<S>(acc, o);
        if (threadIdx.x == 0)
          for (int k = 0; k < S; ++k) blk[k] = o[k];
        if (!grid_reduce<S>(blk, sTot, a, epoch, 3)) return;
        if (threadIdx.x == 0) {
          double nrm = 0.0;
          for (int s = 0; s < S; ++s) {
            double g = 0.0;
            for (int t = 0; t < S; ++t) g += sM[s * S + t] * sTot[t];
            sGamma[s] = a.c / (a.tau * a.tau) * g;
          }
          for (int s = 0; s < S; ++s) {
            double g = sUv[s] - a.c / a.tau * sTot[s];
            for (int t = 0; t < S; ++t) g += sG[s * S + t] * sGamma[t];
            sUtw[s] = g;
            nrm += g * g;
          }
          sScale = fmax(1.0, sqrt(nrm));
          for (int s = 0; s < S; ++s) sBetaEval[s] = sBeta[s];
          sDone = 0;
        }
        __syncthreads();
      }
      // ------------------------------------------------------------ phase N
      // decision state (meaningful in thread 0 only)
      __shared__ double dir[S], phi_cur[S];
      __shared__ double nphi_cur, tstep;
      __shared__ int halvings, accepted;
      __shared__ bool first;
      if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { dir[s] = 0.0; phi_cur[s] = 0.0; }
        nphi_cur = 0.0;
        tstep = 1.0;
        halvings = 0;
        accepted = 0;
        first = true;
      }
      __syncthreads();
      const int max_evals = a.maxit * 8;
      int my_evals = 0;
      while (true) {
        if (threadIdx.x < S) {
          sTheta[threadIdx.x] = (float)(sGamma[threadIdx.x] - sBetaEval[threadIdx.x] / a.tau);
          sGam[threadIdx.x] = (float)sGamma[threadIdx.x];
        }
        __syncthreads();
        float th[S], ga[S];
#pragma unroll
        for (int s = 0; s < S; ++s) { th[s] = sTheta[s]; ga[s] = sGam[s]; }
        float acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.f;
        for (int i0 = tid; i0 < N; i0 += ILP * stride) {
#pragma unroll
          for (int q = 0; q < ILP; ++q) {
            const int i = i0 + q * stride;
            if (i < N) {
              const float base = a.v[i] - cdt * a.d[i];
              float u[S];
              float zz = base, ww = base;
#pragma unroll
              for (int s = 0; s < S; ++s) {
                u[s] = a.U.u[s][i];
                zz = fmaf(u[s], th[s], zz);
                ww = fmaf(u[s], ga[s], ww);
              }
              const float xc = clampf(zz, a.lo, a.hi);
              xw[i] = xc;
              const float e = ww - xc;
              const float in = (zz > a.lo && zz < a.hi) ? 1.f : 0.f;
#pragma unroll
              for (int s = 0; s < S; ++s) acc[s] = fmaf(u[s], e, acc[s]);
              int k = S;
#pragma unroll
              for (int s = 0; s < S; ++s) {
                const float us = in * u[s];
#pragma unroll
                for (int t = s; t < S; ++t) {
                  acc[k] = fmaf(us, u[t], acc[k]);
                  ++k;
                }
              }
            }
          }
        }
        double o[NV];
        block_partial<NV>(acc, o);
        if (threadIdx.x == 0)
          for (int k = 0; k < NV; ++k) blk[k] = o[k];
        if (!grid_reduce<NV>(blk, sTot, a, epoch, 4)) return;
        ++my_evals;
        if (threadIdx.x == 0) {
          NewtonState<S> ns{sBeta, sBetaEval, dir, phi_cur, &nphi_cur, &tstep, &halvings, &accepted, &first,
                            &sAcceptedLast};
          const int done = newton_decide<S>(ns, sTot, a.tau, a.tol * sScale, a.maxit, my_evals >= max_evals);
          sDone = done;
          if (done) last_newton = accepted;
        }
        __syncthreads();
        if (sDone) break;
      }
      if (threadIdx.x == 0) {
        newton_max = max(newton_max, last_newton);
        newton_total += last_newton;
      }
      evals += my_evals;
      if (!sAcceptedLast) {
        // the last evaluation was a rejected trial: write x for the accepted beta
        if (threadIdx.x < S) sTheta[threadIdx.x] = (float)(sGamma[threadIdx.x] - sBeta[threadIdx.x] / a.tau);
        __syncthreads();
        float th[S];
#pragma unroll
        for (int s = 0; s < S; ++s) th[s] = sTheta[s];
        for (int i = tid; i < N; i += stride) {
          float zz = a.v[i] - cdt * a.d[i];
#pragma unroll
          for (int s = 0; s < S; ++s) zz = fmaf(a.U.u[s][i], th[s], zz);
          xw[i] = clampf(zz, a.lo, a.hi);
        }
        if (!final_eval && !grid_reduce<0>(nullptr, nullptr, a, epoch, 5)) return;
      }
    }
    if (final_eval) break;
    // -------------------------------------------------------------- phase D
    const float mom = a.mom[j];
    for (int i0 = tid; i0 < N; i0 += ILP * stride) {
#pragma unroll
      for (int q = 0; q < ILP; ++q) {
        const int i = i0 + q * stride;
        if (i < N) {
          int x, y, z;
          coords(i, n, x, y, z);
          const float x0 = a.x[i];
          const float gx = x < n - 1 ? a.x[i + 1] - x0 : 0.f;
          const float gy = y < n - 1 ? a.x[i + n] - x0 : 0.f;
          const float gz = z < n - 1 ? a.x[i + n * n] - x0 : 0.f;
          float px = a.R[i] + a.step * gx;
          float py = a.R[(size_t)N + i] + a.step * gy;
          float pz = a.R[2 * (size_t)N + i] + a.step * gz;
          project<TV>(px, py, pz);
          const float ox = a.Pd[i], oy = a.Pd[(size_t)N + i], oz = a.Pd[2 * (size_t)N + i];
          a.Pd[i] = px;
          a.Pd[(size_t)N + i] = py;
          a.Pd[2 * (size_t)N + i] = pz;
          a.R[i] = px + mom * (px - ox);
          a.R[(size_t)N + i] = py + mom * (py - oy);
          a.R[2 * (size_t)N + i] = pz + mom * (pz - oz);
        }
      }
    }
    if (!grid_reduce<0>(nullptr, nullptr, a, epoch, 6)) return;
  }
  if (a.trace && blockIdx.x == 0 && threadIdx.x == 0) {
    a.trace[0] = epoch;                 // number of barriers passed; entry 0 also holds the start time
    if ((int)epoch + 1 < a.trace_cap) {
      a.trace[2 * (epoch + 1)] = 99;    // end of kernel
      a.trace[2 * (epoch + 1) + 1] = globaltimer();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.stat[0] = last_newton;
    a.stat[1] = newton_max;
    a.stat[2] = newton_total;
    a.stat[3] = evals;
  }
}

template <int S, int TV>
cudaError_t launch_wprox(mqnpm_handle* h, WpArgs& a) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wprox<S, TV>, WP_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int blocks = h->wp.nsm * std::min(per_sm, 2);
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((void*)k_wprox<S, TV>, dim3(blocks), dim3(WP_THREADS), args, 0, h->stream);
}

template <int TV>
cudaError_t dispatch(mqnpm_handle* h, int S, WpArgs& a) {
  switch (S) {
    case 0: return launch_wprox<0, TV>(h, a);
    case 1: return launch_wprox<1, TV>(h, a);
    case 2: return launch_wprox<2, TV>(h, a);
    case 3: return launch_wprox<3, TV>(h, a);
    case 4: return launch_wprox<4, TV>(h, a);
    case 5: return launch_wprox<5, TV>(h, a);
    case 6: return launch_wprox<6, TV>(h, a);
    case 7: return launch_wprox<7, TV>(h, a);
    case 8: return launch_wprox<8, TV>(h, a);
    default: return cudaErrorInvalidValue;
  }
}

#define CK(call)                                                \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return set_cuda_error(h, e_, #call); \
  } while (0)

}  // namespace

int wprox_impl(mqnpm_handle* h, const float* v, double tau, const UPtrs& U, int S_eff, double c, float* P_warm,
               bool warm, float* x_out) {
  if (S_eff < 0 || S_eff > MQNPM_MAX_S) return set_error(h, MQNPM_ERR_INVALID_ARG, "wprox: S_eff out of range");
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  const int J = h->dual_iters;
  if ((int)h->wp.mom_len != J) return set_error(h, MQNPM_ERR_STATE, "wprox: momentum table not initialised");
  if (warm && P_warm) {
    CK(cudaMemcpyAsync(h->wp.Pd, P_warm, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemsetAsync(h->wp.Pd, 0, 3 * N * sizeof(float), s));
  }
  CK(cudaMemcpyAsync(h->wp.R, h->wp.Pd, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(h->wp.err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(h->wp.barrier, 0, 2 * sizeof(unsigned), s));
  WpArgs a;
  a.v = v;
  a.U = U;
  a.R = h->wp.R;
  a.Pd = h->wp.Pd;
  a.d = h->wp.d;
  a.x = h->wp.x;
  a.xout = x_out;
  a.mom = h->wp.mom;
  a.part = h->wp.part;
  a.tot = h->wp.tot;
  a.count = h->wp.barrier;
  a.gen = h->wp.barrier + 1;
  a.err = h->wp.err;
  a.stat = h->wp.stat;
  a.n = h->n;
  a.N = (int)N;
  a.J = J;
  a.tau = tau;
  a.c = c;
  a.lo = (float)h->lo;
  a.hi = (float)h->hi;
  a.step = (float)(tau / (4.0 * 3.0 * c));
  a.tol = h->newton_tol;
  a.maxit = h->newton_maxit;
  a.limit = 4000000000LL;   // about 2 s at 2 GHz per wait
  a.trace = h->wp.trace;
  a.trace_cap = h->wp.trace_cap;
  cudaError_t e = h->tv == MQNPM_TV_ISO ? dispatch<MQNPM_TV_ISO>(h, S_eff, a) : dispatch<MQNPM_TV_ANISO>(h, S_eff, a);
  if (e != cudaSuccess) return set_cuda_error(h, e, "wprox launch");
  h->launches += 1;
  double stat[4];
  int errflag = 0;
  CK(cudaMemcpyAsync(stat, h->wp.stat, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&errflag, h->wp.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->last_newton_max = (int)stat[1];
  h->last_newton_total = (int)stat[2];
  if (errflag) return set_error(h, MQNPM_ERR_TIMEOUT, "wprox: grid barrier wait gave up");
  if (P_warm) CK(cudaMemcpyAsync(P_warm, h->wp.Pd, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return MQNPM_OK;
}

// Momentum table of the accelerated dual iterations: t_1 = 1,
// t_{j+1} = (1 + sqrt(1 + 4 t_j^2))/2, mom_j = (t_j - 1)/t_{j+1}.
std::vector<float> wprox_momentum(int J) {
  std::vector<float> mom(std::max(J, 1), 0.f);
  double t = 1.0;
  for (int j = 0; j < J; ++j) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    mom[j] = (float)((t - 1.0) / tn);
    t = tn;
  }
  return mom;
}

int wprox_part_len() { return NVMAX; }
