// The whole weighted proximal mapping (Eq. 4.5) as one cooperative kernel.
//
// Phases, separated by grid-wide barriers (deterministic reductions: group
// sums of the per-block partials, then every block adds the group sums in a
// fixed order; every wait is bounded):
//   G  (U != 0, once)  G = U^T U, U^T v; every block forms M = (I + G/tau)^{-1}.
//   per dual iteration j = 1..J, then once more on P_J:
//   A  d = d(R), U^T d and the first Newton evaluation, at the point that keeps
//      theta = gamma - beta/tau of the previous solve (one pass, one barrier)
//                                      -> gamma = (c/tau^2) M U^T d   (Woodbury)
//   N  semi-smooth Newton on phi(beta) = U^T(w - clip(w - U beta/tau)) + beta
//      (Theorem 3.1, Algorithm 4.3): each evaluation also writes
//      x = clip(w - U beta/tau) speculatively, so the accepted evaluation leaves x.
//   X  (U = 0) x = clip(v - (c/tau) d(R))
//   D  P_j = Proj(R_j + tau/(4 D c) grad x),  R_{j+1} = P_j + mom_j (P_j - P_{j-1})
// Every streaming loop handles four consecutive voxels per thread with 16-byte
// loads (the grid's x edge nx is a multiple of 4), so each thread keeps its whole
// working set of loads in flight.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

cudaError_t wprox_dispatch_high(mqnpm_handle* h, int S, int tv, void* args);

namespace {

constexpr int WP_THREADS = 256;
constexpr int WP_BPS = 2;        // co-resident blocks per SM the kernel is compiled and launched for
constexpr int NW = WP_THREADS / 32;
constexpr int NVMAX = 2 * MQNPM_MAX_S + MQNPM_MAX_S * (MQNPM_MAX_S + 1) / 2;   // 2S + S(S+1)/2
// Trace layout (long long pairs): pair 0 = (barriers passed, start time),
// pairs 1..TR_ACC-1 = (tag, time) per barrier, pairs from TR_ACC on hold block
// 0's accumulated times: [2 TR_ACC] dual update, [+1] work before the dual
// update, [+2] Newton evaluation pass, [+3] Newton decision (thread 0),
// [+4] divergence pass, [+5] waiting in grid barriers.
constexpr int TR_ACC = 1000;
constexpr int TR_SLOTS = 6;
// Grid barriers that carry sums reduce in two levels: groups of WP_GS
// consecutive blocks (the last block of a group to arrive sums its group's
// partials), then the last group reducer sums the group sums.  At most
// WP_MAXG groups.
constexpr int WP_GS = 16;
constexpr int WP_MAXG = 64;

struct WpArgs {
  const float* v;
  UPtrs U;
  float* R;
  float* Pd;
  float* d;
  float* x;
  float* xout;
  const float* mom;
  double* part;           // [gridDim.x][NVMAX] block partials, then 2 x [WP_MAXG][NVMAX] group sums
  unsigned* count;        // arrivals at barriers without sums (monotonic)
  unsigned* count_groups; // group sums finished (monotonic)
  unsigned* gcount;       // [WP_MAXG] arrivals per group (monotonic)
  int* err;
  double* stat;           // [0] last newton count, [1] max, [2] total, [3] evaluations
  unsigned char* status;  // per voxel: 1 if the last evaluated z was strictly inside the box
  int nx, ny, nz, N, J;
  double tau, c;
  double inv_tau, c_tau, c_tau2;   // 1/tau, c/tau, c/tau^2 (FP64 divisions are slow on the device)
  float cdt;                       // (float) c/tau
  float lo, hi, step;
  double tol;
  int maxit;
  long long limit;
  long long* trace;       // optional: (phase tag, ns) after every barrier, recorded by block 0
  int trace_cap;
};

MQ_D float clampf(float a, float lo, float hi) { return fminf(fmaxf(a, lo), hi); }

// Arrival at a grid barrier: one atomic with release semantics (the block's
// writes, made visible to thread 0 by the __syncthreads before it, are
// published with it) and acquire semantics (the arrivals before it are
// visible to the block after its next __syncthreads).  Replaces a full fence
// followed by a relaxed atomic.
MQ_D unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

MQ_D long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

MQ_D bool tracer(const WpArgs& a) { return a.trace && blockIdx.x == 0 && threadIdx.x == 0; }
// Block 0's phase accumulators and the time of the last barrier live in shared
// memory while the kernel runs (written to the trace at its end), so the
// tracing thread does no global read-modify-write on the barrier path.
MQ_D long long* tr_acc() {
  __shared__ long long acc[TR_SLOTS + 1];   // [TR_SLOTS] = time of the last barrier
  return acc;
}
MQ_D void tr_add(const WpArgs& a, int slot, long long dt) {
  if (tracer(a)) tr_acc()[slot] += dt;
}

// Four consecutive floats as an addressable array.
struct F4 {
  float v[4];
  MQ_D static F4 load(const float* p, int k4) {
    const float4 q = reinterpret_cast<const float4*>(p)[k4];
    return F4{{q.x, q.y, q.z, q.w}};
  }
  MQ_D void store(float* p, int k4) const {
    reinterpret_cast<float4*>(p)[k4] = make_float4(v[0], v[1], v[2], v[3]);
  }
  MQ_D static F4 zero() { return F4{{0.f, 0.f, 0.f, 0.f}}; }
  // read-only path: only for data no thread of the kernel writes
  MQ_D static F4 ldg(const float* p, int k4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p) + k4);
    return F4{{q.x, q.y, q.z, q.w}};
  }
};

// Per-thread staging slots in dynamic shared memory: slot j of thread t is
// wp_stage[j * WP_THREADS + t] (16 bytes; consecutive threads, consecutive
// addresses, so the 16-byte reads back are conflict-free).  cp.async copies
// land there without holding registers while in flight, so the number of
// loads a thread keeps in flight does not depend on how many registers the
// compiler leaves a pass; each thread reads back only the slots it filled,
// after its own cp.async.wait_all, so no block barrier is needed.
extern __shared__ float4 wp_stage[];
constexpr int WP_SLOTS_DUAL = 10;   // the dual update's ten streams
constexpr int WP_SU_MAX = 8;        // rows of U staged by the Newton passes (the rest are loaded directly)
// slots per thread for rank S: the dual update's ten, or the merged pass's
// staged U rows + v + six divergence loads + status
constexpr int wp_slots(int S) {
  return (S < WP_SU_MAX ? S : WP_SU_MAX) + 8 > WP_SLOTS_DUAL ? (S < WP_SU_MAX ? S : WP_SU_MAX) + 8 : WP_SLOTS_DUAL;
}

MQ_D void cp16(float4* dst, const float* src) {   // 16 bytes global -> shared, cached in L2 only
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
MQ_D void cp4(float4* dst, const float* src) {    // 4 bytes global -> the first word of a slot
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
MQ_D void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
MQ_D F4 slot4(const float4* p) {
  const float4 q = *p;
  return F4{{q.x, q.y, q.z, q.w}};
}

// Barrier counters of one launch: every block passes the same sequence of
// barriers, so these agree across blocks.
struct Epochs {
  unsigned all = 0;    // barriers passed (the released generation)
  unsigned flat = 0;   // barriers without sums
  unsigned hier = 0;   // barriers with sums
};

// Thread 0 of a block polls a monotonic arrival counter until it reaches
// target (bounded; gives up when another block reported an error).
MQ_D bool wait_count(const WpArgs& a, const unsigned* ctr, unsigned target) {
  const long long t0 = clock64();
  while (ld_acquire_u32(ctr) < target) {
    if (*((volatile int*)a.err) != 0) return false;
    if (clock64() - t0 > a.limit) {
      atomicExch(a.err, 1);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Grid-wide barrier with an optional sum of NV doubles per block (blk[],
// shared).  Every wait polls the arrival counter it waits for, so a barrier
// ends as soon as the last arrival reaches memory (no separate release word).
// NV = 0: one arrival counter.  NV > 0: each block stores its partials
// (block-major); the last block of each group of WP_GS blocks sums the
// group's partials in block order into a group sum (double-buffered by the
// barrier's parity) and counts the group as done; every block waits for all
// groups and sums the group sums itself in group order, so every block holds
// bit-identical totals in sh_tot.  Release-acquire: each block's arrival is an
// acquire-release atomic after __syncthreads, and each wait an acquire load,
// so whatever a block wrote before the barrier is visible to every block after it.
template <int NV>
MQ_D bool grid_reduce(const double* blk, double* sh_tot, const WpArgs& a, Epochs& ep, int tag) {
  __shared__ int s_role, s_ok;   // role: 1 = group reducer
  const long long t_in = tracer(a) ? globaltimer() : 0;
  __syncthreads();
  if constexpr (NV == 0) {
    if (threadIdx.x == 0) {
      atom_add_acq_rel(a.count, 1u);
      s_ok = wait_count(a, a.count, (ep.flat + 1) * gridDim.x) ? 1 : 0;
    }
    __syncthreads();
    ep.flat += 1;
  } else {
    if (threadIdx.x < NV) a.part[(size_t)blockIdx.x * NVMAX + threadIdx.x] = blk[threadIdx.x];
    __syncthreads();
    const int g = blockIdx.x / WP_GS, g0 = g * WP_GS;
    const int gsize = min(WP_GS, (int)gridDim.x - g0);
    const int ngroups = ((int)gridDim.x + WP_GS - 1) / WP_GS;
    // a block can be one barrier ahead of another still reading group sums, never two
    double* gpart = a.part + (size_t)gridDim.x * NVMAX + (size_t)(ep.hier & 1u) * WP_MAXG * NVMAX;
    if (threadIdx.x == 0) {
      const unsigned old = atom_add_acq_rel(a.gcount + g, 1u);
      s_role = (old == (ep.hier + 1) * (unsigned)gsize - 1) ? 1 : 0;
      s_ok = 1;
    }
    __syncthreads();
    if (s_role == 1) {
      if (threadIdx.x < NV) {
        double vals[WP_GS];
#pragma unroll
        for (int j = 0; j < WP_GS; ++j)
          vals[j] = (j < gsize) ? __ldcg(a.part + (size_t)(g0 + j) * NVMAX + threadIdx.x) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < WP_GS; ++j) acc += vals[j];
        gpart[(size_t)g * NVMAX + threadIdx.x] = acc;
      }
      __syncthreads();
      if (threadIdx.x == 0) atom_add_acq_rel(a.count_groups, 1u);
    }
    if (threadIdx.x == 0 && !wait_count(a, a.count_groups, (ep.hier + 1) * (unsigned)ngroups)) s_ok = 0;
    __syncthreads();
    if (s_ok && threadIdx.x < NV) {
      // all group sums of a chunk are loaded before any is added (one round
      // trip for up to 24 groups: 384 blocks)
      double acc = 0.0;
      for (int q0 = 0; q0 < ngroups; q0 += 24) {
        double vals[24];
#pragma unroll
        for (int q = 0; q < 24; ++q)
          vals[q] = (q0 + q < ngroups) ? __ldcg(gpart + (size_t)(q0 + q) * NVMAX + threadIdx.x) : 0.0;
#pragma unroll
        for (int q = 0; q < 24; ++q) acc += vals[q];
      }
      sh_tot[threadIdx.x] = acc;
    }
    __syncthreads();
    ep.hier += 1;
  }
  ep.all += 1;
  if (tracer(a)) {
    const long long t = globaltimer();
    if ((int)ep.all < TR_ACC) {
      a.trace[2 * ep.all] = tag;
      a.trace[2 * ep.all + 1] = t;
    }
    tr_acc()[5] += t - t_in;
    tr_acc()[TR_SLOTS] = t;
  }
  return s_ok != 0;
}

// Coordinates of the first of four voxels i4 = 4 k4 (nx is a multiple of 4).
MQ_D void coords4(int k4, int nx, int ny, int& x0, int& y, int& z) {
  const int i4 = 4 * k4;
  const int r = i4 / nx;
  x0 = i4 - r * nx;
  z = r / ny;
  y = r - z * ny;
}

// d(R) = sum_d q_d(i - e_d)[i_d >= 1] - q_d(i)[i_d <= n_d - 2] at four voxels,
// from the loaded values: a* = q_*(i), a*m = q_*(i - e_*) (zero where i_* = 0).
MQ_D F4 div4_of(const F4& ax, float axm, const F4& ay, const F4& aym, const F4& az, const F4& azm, int nx,
                int ny, int nz, int x0, int y, int z) {
  F4 d;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float s = (m == 0) ? axm : ax.v[m - 1];
    if (x0 + m < nx - 1) s -= ax.v[m];
    s += aym.v[m];
    if (y < ny - 1) s -= ay.v[m];
    s += azm.v[m];
    if (z < nz - 1) s -= az.v[m];
    d.v[m] = s;
  }
  return d;
}

MQ_D F4 div4(const float* __restrict__ R, int N, int nx, int ny, int nz, int k4, int x0, int y, int z) {
  const int n4 = nx / 4, nn4 = nx * ny / 4;
  const float* qx = R;
  const float* qy = R + N;
  const float* qz = R + 2 * (size_t)N;
  const F4 ax = F4::load(qx, k4), ay = F4::load(qy, k4), az = F4::load(qz, k4);
  const float axm = x0 > 0 ? qx[4 * k4 - 1] : 0.f;
  const F4 aym = y > 0 ? F4::load(qy, k4 - n4) : F4::zero();
  const F4 azm = z > 0 ? F4::load(qz, k4 - nn4) : F4::zero();
  return div4_of(ax, axm, ay, aym, az, azm, nx, ny, nz, x0, y, z);
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

// Cholesky factor of a small SPD matrix in place (lower triangle), with the
// reciprocals of the diagonal in rd.  One FP64 division and one square root per
// column: FP64 division is a long instruction sequence on this device.
template <int S>
MQ_D bool chol_factor(double (&A)[S * S], double (&rd)[S]) {
  for (int j = 0; j < S; ++j) {
    double s = A[j * S + j];
    for (int k = 0; k < j; ++k) s -= A[j * S + k] * A[j * S + k];
    if (!(s > 0.0)) return false;
    const double r = 1.0 / sqrt(s);
    A[j * S + j] = s * r;
    rd[j] = r;
    for (int i = j + 1; i < S; ++i) {
      double t = A[i * S + j];
      for (int k = 0; k < j; ++k) t -= A[i * S + k] * A[j * S + k];
      A[i * S + j] = t * r;
    }
  }
  return true;
}

// Solve (L L^T) b = b with the factor of chol_factor.
template <int S>
MQ_D void chol_apply(const double (&A)[S * S], const double (&rd)[S], double (&b)[S]) {
  for (int i = 0; i < S; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= A[i * S + k] * b[k];
    b[i] = t * rd[i];
  }
  for (int i = S - 1; i >= 0; --i) {
    double t = b[i];
    for (int k = i + 1; k < S; ++k) t -= A[k * S + i] * b[k];
    b[i] = t * rd[i];
  }
}

// The same in FP32 for the Newton direction of Algorithm 4.3: H = I + U^T D U / tau
// is symmetric positive definite with eigenvalues >= 1, and the direction only
// needs to be approximate (the step is accepted on ||phi|| evaluated in FP64).
template <int S>
MQ_D bool chol_factor_f(float (&A)[S * S], float (&rd)[S]) {
#pragma unroll
  for (int j = 0; j < S; ++j) {
    float s = A[j * S + j];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fmaf(-A[j * S + k], A[j * S + k], s);
    if (!(s > 0.f)) return false;
    const float r = rsqrtf(s);
    rd[j] = r;
#pragma unroll
    for (int i = j + 1; i < S; ++i) {
      float t = A[i * S + j];
#pragma unroll
      for (int k = 0; k < j; ++k) t = fmaf(-A[i * S + k], A[j * S + k], t);
      A[i * S + j] = t * r;
    }
  }
  return true;
}

template <int S>
MQ_D void chol_apply_f(const float (&A)[S * S], const float (&rd)[S], float (&b)[S]) {
#pragma unroll
  for (int i = 0; i < S; ++i) {
    float t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t = fmaf(-A[i * S + k], b[k], t);
    b[i] = t * rd[i];
  }
#pragma unroll
  for (int i = S - 1; i >= 0; --i) {
    float t = b[i];
#pragma unroll
    for (int k = i + 1; k < S; ++k) t = fmaf(-A[k * S + i], b[k], t);
    b[i] = t * rd[i];
  }
}

// M = (I + G/tau)^{-1} (S x S, FP64): one factorisation, S solves.  Called by
// one thread; kept out of line so its scratch does not cost the streaming loops
// registers.
template <int S>
__device__ __noinline__ void form_woodbury(const double* G, double inv_tau, double* M) {
  double A[S * S], rd[S];
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) A[i * S + j] = (i == j ? 1.0 : 0.0) + G[i * S + j] * inv_tau;
  const bool ok = chol_factor<S>(A, rd);
  for (int col = 0; col < S; ++col) {
    double e[S];
    for (int i = 0; i < S; ++i) e[i] = (i == col) ? 1.0 : 0.0;
    if (ok) chol_apply<S>(A, rd, e);
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

// One decision of Algorithm 4.3 after phi was evaluated at beta_eval
// (tot[0..S) = U^T(w - clip(z))) with hf = sum_{inner} u u^T / tau (upper
// triangle, FP32).  Accept the trial if it reduces ||phi|| (or halving is
// exhausted), stop at ||phi||^2 <= tol2, else take the Newton step -H^{-1} phi
// from the accepted point, H = I + hf; a rejected trial is halved.  The norms
// are compared squared (no FP64 square root: a long sequence on this device).
// tol2 is the squared tolerance.  Returns 1 when done.
template <int S>
__device__ __noinline__ int newton_decide(NewtonState<S> ns, const double* tot, const float* hf, double tol2,
                                          int maxit, bool out_of_evals) {
  double phi[S], nphi = 0.0;   // nphi: ||phi||^2
#pragma unroll
  for (int s = 0; s < S; ++s) {
    phi[s] = tot[s] + ns.beta_eval[s];
    nphi = fma(phi[s], phi[s], nphi);
  }
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
  if (nphi <= tol2 || *ns.accepted >= maxit || out_of_evals || !isfinite(nphi)) return 1;
  // Newton direction -H^{-1} phi, solved in FP32 (see chol_factor_f)
  float H[S * S];
  int k = 0;
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int t = s; t < S; ++t) {
      const float hst = hf[k++] + (s == t ? 1.f : 0.f);
      H[s * S + t] = hst;
      H[t * S + s] = hst;
    }
  float rhs[S], rd[S];
#pragma unroll
  for (int s = 0; s < S; ++s) rhs[s] = (float)(-phi[s]);
  if (!chol_factor_f<S>(H, rd)) return 1;
  chol_apply_f<S>(H, rd, rhs);
  for (int s = 0; s < S; ++s) {
    ns.dir[s] = (double)rhs[s];
    ns.beta_eval[s] = ns.beta[s] + (double)rhs[s];
  }
  *ns.tstep = 1.0;
  *ns.halvings = 0;
  *ns.accepted += 1;
  return 0;
}

// Block-level sum of K floats per thread into thread 0's out[] (FP64).
template <int K>
MQ_D void block_partial(const float (&acc)[K], double (&out)[K]) {
  __shared__ double scratch[(NW + 1) * (K > 0 ? K : 1)];
  block_sum_f<K>(acc, scratch, out);
}

MQ_D float dot4(const F4& a, const F4& b) {
  return fmaf(a.v[0], b.v[0], fmaf(a.v[1], b.v[1], fmaf(a.v[2], b.v[2], a.v[3] * b.v[3])));
}

// Shared state of the cooperative kernel (identical in every block).
template <int S>
struct Shared {
  static constexpr int SS = S > 0 ? S : 1;
  static constexpr int NG = S * (S + 1) / 2;
  static constexpr int NGG = NG > 0 ? NG : 1;
  WpArgs a;
  float trU[NW][SS][33];   // per-warp transpose of u for status flips
  float trSign[NW][32];
  float dH[NW][NGG];
  double Htot[NGG];        // sum_{status inner} u u^T (upper triangle)
  float Hf[NGG];           // Htot / tau* in FP32 for the Newton direction
  double G[SS * SS], M[SS * SS], Uv[SS];
  double gamma[SS], beta[SS], beta_eval[SS], dir[SS], phi_cur[SS];
  double tot[NVMAX], blk[NVMAX];
  float theta[SS], gam[SS];
  int done, accepted_last, halvings, accepted;
  double scale, nphi_cur, tstep;   // max(1, ||U^T w||^2), ||phi||^2 of the accepted point, step
  bool first;
};

// ---- phase G: block partials of U^T U (upper triangle) and U^T v into blk.
template <int S>
__device__ __noinline__ void pass_gram(Shared<S>* sh) {
  constexpr int NG = S * (S + 1) / 2;
  const WpArgs a = sh->a;   // private copy: loop loads cannot alias it, fields stay in registers
  const int N4 = a.N / 4, tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  float acc[NG + S];
#pragma unroll
  for (int k = 0; k < NG + S; ++k) acc[k] = 0.f;
  for (int k4 = tid; k4 < N4; k4 += stride) {
    F4 u[S];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = F4::load(a.U.u[s], k4);
    const F4 v4 = F4::load(a.v, k4);
    int k = 0;
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int t = s; t < S; ++t) {
        acc[k] += dot4(u[s], u[t]);
        ++k;
      }
#pragma unroll
    for (int s = 0; s < S; ++s) acc[NG + s] += dot4(u[s], v4);
  }
  double o[NG + S];
  block_partial<NG + S>(acc, o);
  if (threadIdx.x == 0)
    for (int k = 0; k < NG + S; ++k) sh->blk[k] = o[k];
}

// ---- phase X (U = 0): x = clip(v - (c/tau) d(src)).
__device__ __noinline__ void pass_x(const WpArgs* pa, const float* src, float* xw) {
  const WpArgs a = *pa;     // private copy: loop loads cannot alias it, fields stay in registers
  const int nx = a.nx, ny = a.ny, nz = a.nz, N = a.N, N4 = a.N / 4;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const float cdt = a.cdt;
  for (int k4 = tid; k4 < N4; k4 += stride) {
    int x0, y, z;
    coords4(k4, nx, ny, x0, y, z);
    const F4 dv = div4(src, N, nx, ny, nz, k4, x0, y, z);
    const F4 v4 = F4::load(a.v, k4);
    F4 xo;
#pragma unroll
    for (int m = 0; m < 4; ++m) xo.v[m] = clampf(v4.v[m] - cdt * dv.v[m], a.lo, a.hi);
    xo.store(xw, k4);
  }
}

// ---- phase N: one evaluation at theta = gamma - beta_eval/tau.  Writes
// x = clip(z) speculatively, block partials of U^T(w - clip(z)) into blk[0..S)
// and of the status flips of sum_{inner} u u^T into blk[S..S+NG).
// MERGED (the first evaluation of a dual iteration, in the divergence pass):
// d = d(src) is formed here, stored, and its U^T d partials go to
// blk[S+NG..2S+NG); gamma is not known yet, so the evaluation point is given
// by theta alone (theta of the previous solve) and the partials are
// U^T(v - (c/tau) d - clip(z)); the kernel adds G gamma once gamma is known.
template <int S, bool MERGED>
__device__ __noinline__ void pass_newton(Shared<S>* sh, const float* src, float* xw) {
  constexpr int NG = S * (S + 1) / 2;
  const WpArgs a = sh->a;   // private copy: loop loads cannot alias it, fields stay in registers
  const int nx = a.nx, ny = a.ny, nz = a.nz, N = a.N, N4 = a.N / 4;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const int gw = tid >> 5, nwt = stride >> 5;
  const float cdt = a.cdt;
  constexpr int NGL = (NG + 31) / 32;      // pairs (s, t) per lane: lane + 32 j
  int ps[NGL], pt[NGL];
#pragma unroll
  for (int j = 0; j < NGL; ++j) { ps[j] = 0; pt[j] = 0; }
  {
    int k = 0;
    for (int s = 0; s < S; ++s)
      for (int t = s; t < S; ++t) {
#pragma unroll
        for (int j = 0; j < NGL; ++j)
          if (k == lane + 32 * j) { ps[j] = s; pt[j] = t; }
        ++k;
      }
  }
  float th[S], ga[S];
#pragma unroll
  for (int s = 0; s < S; ++s) { th[s] = sh->theta[s]; ga[s] = MERGED ? 0.f : sh->gam[s]; }   // ga unused when MERGED
  float acc[S], accd[MERGED ? S : 1];
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = 0.f;
#pragma unroll
  for (int s = 0; s < (MERGED ? S : 1); ++s) accd[s] = 0.f;
  float dH[NGL];
#pragma unroll
  for (int j = 0; j < NGL; ++j) dH[j] = 0.f;
  const float* __restrict__ din = a.d;
  float* __restrict__ dout = a.d;
  const float* __restrict__ rs = src;
  float* __restrict__ xout = xw;
  uchar4* __restrict__ stat = reinterpret_cast<uchar4*>(a.status);
  constexpr int SU = S < WP_SU_MAX ? S : WP_SU_MAX;   // staged rows of U
  constexpr int SLOT_STAT = MERGED ? SU + 7 : SU + 2;
  constexpr int T = WP_THREADS;
  static_assert(SLOT_STAT < wp_slots(S), "staging slots");
  const int n4 = nx / 4, nn4 = nx * ny / 4;
  float4* st = wp_stage + threadIdx.x;
  for (int wbase = gw * 32; wbase < N4; wbase += nwt * 32) {
    const int k4 = wbase + lane;
    const bool valid = k4 < N4;
    F4 u[S];
    float sign[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid) {
      // stage SU rows of U, v, d (or the six divergence loads of src) and the
      // status word; U rows beyond SU go to registers directly
      int x0 = 0, y = 0, z = 0;
#pragma unroll
      for (int s = 0; s < SU; ++s) cp16(st + s * T, a.U.u[s] + 4 * (size_t)k4);
      cp16(st + SU * T, a.v + 4 * (size_t)k4);
      if constexpr (MERGED) {
        coords4(k4, nx, ny, x0, y, z);
        cp16(st + (SU + 1) * T, rs + 4 * (size_t)k4);
        cp16(st + (SU + 2) * T, rs + N + 4 * (size_t)k4);
        cp16(st + (SU + 3) * T, rs + 2 * (size_t)N + 4 * (size_t)k4);
        if (y > 0) cp16(st + (SU + 4) * T, rs + N + 4 * (size_t)(k4 - n4));
        if (z > 0) cp16(st + (SU + 5) * T, rs + 2 * (size_t)N + 4 * (size_t)(k4 - nn4));
        if (x0 > 0) cp4(st + (SU + 6) * T, rs + 4 * (size_t)k4 - 1);
      } else {
        cp16(st + (SU + 1) * T, din + 4 * (size_t)k4);
      }
      cp4(st + SLOT_STAT * T, reinterpret_cast<const float*>(stat + k4));
#pragma unroll
      for (int s = SU; s < S; ++s) u[s] = F4::ldg(a.U.u[s], k4);   // U is read-only in the kernel
      cp_wait_all();
#pragma unroll
      for (int s = 0; s < SU; ++s) u[s] = slot4(st + s * T);
      const F4 v4 = slot4(st + SU * T);
      F4 d4;
      if constexpr (MERGED) {
        const F4 ax = slot4(st + (SU + 1) * T), ay = slot4(st + (SU + 2) * T), az = slot4(st + (SU + 3) * T);
        const F4 aym = y > 0 ? slot4(st + (SU + 4) * T) : F4::zero();
        const F4 azm = z > 0 ? slot4(st + (SU + 5) * T) : F4::zero();
        const float axm = x0 > 0 ? reinterpret_cast<const float*>(st + (SU + 6) * T)[0] : 0.f;
        d4 = div4_of(ax, axm, ay, aym, az, azm, nx, ny, nz, x0, y, z);
        d4.store(dout, k4);
#pragma unroll
        for (int s = 0; s < S; ++s) accd[s] += dot4(u[s], d4);
      } else {
        d4 = slot4(st + (SU + 1) * T);
      }
      const uchar4 st4 = *reinterpret_cast<const uchar4*>(st + SLOT_STAT * T);
      const unsigned char old[4] = {st4.x, st4.y, st4.z, st4.w};
      unsigned char nw[4];
      F4 xo;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float base = v4.v[m] - cdt * d4.v[m];
        float zz = base, ww = base;   // MERGED: w - U gamma (gamma added to the sums later)
#pragma unroll
        for (int s = 0; s < S; ++s) {
          zz = fmaf(u[s].v[m], th[s], zz);
          if constexpr (!MERGED) ww = fmaf(u[s].v[m], ga[s], ww);
        }
        const float xc = clampf(zz, a.lo, a.hi);
        xo.v[m] = xc;
        const float e = ww - xc;
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = fmaf(u[s].v[m], e, acc[s]);
        nw[m] = (zz > a.lo && zz < a.hi) ? 1 : 0;
        if (nw[m] != old[m]) sign[m] = nw[m] ? 1.f : -1.f;
      }
      xo.store(xout, k4);
      if (sign[0] != 0.f || sign[1] != 0.f || sign[2] != 0.f || sign[3] != 0.f)
        stat[k4] = make_uchar4(nw[0], nw[1], nw[2], nw[3]);
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = F4::zero();
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      unsigned flips = __ballot_sync(0xffffffffu, sign[m] != 0.f);
      if (flips) {
#pragma unroll
        for (int s = 0; s < S; ++s) sh->trU[wib][s][lane] = u[s].v[m];
        sh->trSign[wib][lane] = sign[m];
        __syncwarp();
        while (flips) {
          const int jl = __ffs(flips) - 1;
          flips &= flips - 1;
          const float sg = sh->trSign[wib][jl];
#pragma unroll
          for (int j = 0; j < NGL; ++j)
            if (lane + 32 * j < NG) dH[j] = fmaf(sg * sh->trU[wib][ps[j]][jl], sh->trU[wib][pt[j]][jl], dH[j]);
        }
        __syncwarp();
      }
    }
  }
  double o[S];
  block_partial<S>(acc, o);
  if (threadIdx.x == 0)
    for (int k = 0; k < S; ++k) sh->blk[k] = o[k];
  if constexpr (MERGED) {
    block_partial<S>(accd, o);
    if (threadIdx.x == 0)
      for (int k = 0; k < S; ++k) sh->blk[S + NG + k] = o[k];
  }
#pragma unroll
  for (int j = 0; j < NGL; ++j)
    if (lane + 32 * j < NG) sh->dH[wib][lane + 32 * j] = dH[j];
  __syncthreads();
  if (threadIdx.x < NG) {
    double sacc = 0.0;
    for (int w = 0; w < NW; ++w) sacc += (double)sh->dH[w][threadIdx.x];
    sh->blk[S + threadIdx.x] = sacc;
  }
}

// ---- x = clip(v - (c/tau) d + U theta) for the accepted beta (after a rejected trial).
template <int S>
__device__ __noinline__ void pass_fixup(Shared<S>* sh, float* xw) {
  const WpArgs a = sh->a;   // private copy: loop loads cannot alias it, fields stay in registers
  const int N4 = a.N / 4, tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const float cdt = a.cdt;
  float th[S];
#pragma unroll
  for (int s = 0; s < S; ++s) th[s] = sh->theta[s];
  for (int k4 = tid; k4 < N4; k4 += stride) {
    const F4 v4 = F4::load(a.v, k4), d4 = F4::load(a.d, k4);
    F4 xo;
#pragma unroll
    for (int m = 0; m < 4; ++m) xo.v[m] = v4.v[m] - cdt * d4.v[m];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const F4 u4 = F4::load(a.U.u[s], k4);
#pragma unroll
      for (int m = 0; m < 4; ++m) xo.v[m] = fmaf(u4.v[m], th[s], xo.v[m]);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) xo.v[m] = clampf(xo.v[m], a.lo, a.hi);
    xo.store(xw, k4);
  }
}

// ---- phase D: P = Proj(R + step grad x), R = P + mom (P - P_prev), in place.
// The ten input streams of four voxels (x, its +y and +z neighbours and the
// next voxel in x, R and P_prev) are staged with cp.async before any is used.
template <int TV>
__device__ __noinline__ void pass_dual(const WpArgs* pa, float mom) {
  const WpArgs a = *pa;     // private copy: loop loads cannot alias it, fields stay in registers
  const int nx = a.nx, ny = a.ny, nz = a.nz, N = a.N, N4 = a.N / 4;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const int n4 = nx / 4, nn4 = nx * ny / 4;
  const float* __restrict__ xs = a.x;
  float* __restrict__ Rx = a.R;
  float* __restrict__ Ry = a.R + N;
  float* __restrict__ Rz = a.R + 2 * (size_t)N;
  float* __restrict__ Px = a.Pd;
  float* __restrict__ Py = a.Pd + N;
  float* __restrict__ Pz = a.Pd + 2 * (size_t)N;
  const float step = a.step;
  float4* st = wp_stage + threadIdx.x;
  constexpr int T = WP_THREADS;
  static_assert(WP_SLOTS_DUAL <= wp_slots(0), "staging slots");
  for (int k4 = tid; k4 < N4; k4 += stride) {
    int x0, y, z;
    coords4(k4, nx, ny, x0, y, z);
    const bool hx = x0 + 4 < nx, hy = y < ny - 1, hz = z < nz - 1;
    cp16(st, xs + 4 * (size_t)k4);
    if (hy) cp16(st + T, xs + 4 * (size_t)(k4 + n4));
    if (hz) cp16(st + 2 * T, xs + 4 * (size_t)(k4 + nn4));
    cp16(st + 3 * T, Rx + 4 * (size_t)k4);
    cp16(st + 4 * T, Ry + 4 * (size_t)k4);
    cp16(st + 5 * T, Rz + 4 * (size_t)k4);
    cp16(st + 6 * T, Px + 4 * (size_t)k4);
    cp16(st + 7 * T, Py + 4 * (size_t)k4);
    cp16(st + 8 * T, Pz + 4 * (size_t)k4);
    if (hx) cp4(st + 9 * T, xs + 4 * (size_t)k4 + 4);
    cp_wait_all();
    const F4 x4 = slot4(st);
    const F4 xy = hy ? slot4(st + T) : x4;
    const F4 xz = hz ? slot4(st + 2 * T) : x4;
    const float xnext = hx ? reinterpret_cast<const float*>(st + 9 * T)[0] : 0.f;
    F4 rx = slot4(st + 3 * T), ry = slot4(st + 4 * T), rz = slot4(st + 5 * T);
    F4 ox = slot4(st + 6 * T), oy = slot4(st + 7 * T), oz = slot4(st + 8 * T);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float xn = (m < 3) ? x4.v[m + 1] : xnext;
      const float gx = (x0 + m < nx - 1) ? xn - x4.v[m] : 0.f;
      float px = rx.v[m] + step * gx;
      float py = ry.v[m] + step * (xy.v[m] - x4.v[m]);
      float pz = rz.v[m] + step * (xz.v[m] - x4.v[m]);
      project<TV>(px, py, pz);
      rx.v[m] = px + mom * (px - ox.v[m]);
      ry.v[m] = py + mom * (py - oy.v[m]);
      rz.v[m] = pz + mom * (pz - oz.v[m]);
      ox.v[m] = px;
      oy.v[m] = py;
      oz.v[m] = pz;
    }
    ox.store(Px, k4);
    oy.store(Py, k4);
    oz.store(Pz, k4);
    rx.store(Rx, k4);
    ry.store(Ry, k4);
    rz.store(Rz, k4);
  }
}

template <int S, int TV>
__global__ void __launch_bounds__(WP_THREADS, WP_BPS) k_wprox(WpArgs args) {
  constexpr int NG = S * (S + 1) / 2;
  constexpr int NV = S + NG;
  __shared__ Shared<S> sh;
  if (threadIdx.x == 0) sh.a = args;
  __syncthreads();
  const WpArgs& a = sh.a;
  Epochs ep;
  if (tracer(a)) {
    const long long t0 = globaltimer();
    a.trace[1] = t0;
    for (int k = 0; k < TR_SLOTS; ++k) tr_acc()[k] = 0;
    tr_acc()[TR_SLOTS] = t0;
  }

  if constexpr (S > 0) {
    pass_gram<S>(&sh);
    if (!grid_reduce<NG + S>(sh.blk, sh.tot, a, ep, 1)) return;
    if (threadIdx.x == 0) {
      int k = 0;
      for (int s = 0; s < S; ++s)
        for (int t = s; t < S; ++t) {
          sh.G[s * S + t] = sh.tot[k];
          sh.G[t * S + s] = sh.tot[k];
          sh.Htot[k] = sh.tot[k];      // every voxel starts with status "inner"
          ++k;
        }
      for (int s = 0; s < S; ++s) sh.Uv[s] = sh.tot[NG + s];
      form_woodbury<S>(sh.G, a.inv_tau, sh.M);
      for (int s = 0; s < S; ++s) {
        sh.beta[s] = 0.0;
        sh.theta[s] = 0.f;   // theta of the "previous solve" before the first one
      }
    }
    __syncthreads();
  }

  int newton_max = 0, newton_total = 0, evals = 0, last_newton = 0;
  for (int j = 0; j <= a.J; ++j) {
    const bool final_eval = (j == a.J);
    const float* src = final_eval ? a.Pd : a.R;
    float* xw = final_eval ? a.xout : a.x;
    if constexpr (S == 0) {
      pass_x(&sh.a, src, xw);
      if (!final_eval && !grid_reduce<0>(nullptr, nullptr, a, ep, 2)) return;
    } else {
      // The divergence pass also takes the first Newton evaluation, at the
      // point that keeps theta = gamma - beta/tau of the previous solve
      // (beta_0 = beta_prev + tau (gamma - gamma_prev)): U^T d, the status
      // flips and U^T(v - (c/tau) d - clip(z)) in one barrier.
      long long t0 = tracer(a) ? globaltimer() : 0;
      pass_newton<S, true>(&sh, src, xw);
      if (tracer(a)) tr_add(a, 4, globaltimer() - t0);
      if (!grid_reduce<NV + S>(sh.blk, sh.tot, a, ep, 3)) return;
      const double* utd = sh.tot + NV;   // U^T d
      // S threads in parallel: gamma = c/tau^2 M U^T d, then (U^T w)_s, the
      // evaluation's U^T(w - clip(z)) = partials + (G gamma)_s, and its point
      // beta' = tau (gamma - theta)
      if (threadIdx.x < S) {
        const int s = threadIdx.x;
        double g = 0.0;
        for (int t = 0; t < S; ++t) g = fma(sh.M[s * S + t], utd[t], g);
        sh.gamma[s] = a.c_tau2 * g;
      }
      __syncthreads();
      if (threadIdx.x < S) {
        const int s = threadIdx.x;
        double gg = 0.0;
        for (int t = 0; t < S; ++t) gg = fma(sh.G[s * S + t], sh.gamma[t], gg);
        const double uw = sh.Uv[s] - a.c_tau * utd[s] + gg;
        sh.phi_cur[s] = uw * uw;   // scratch until the reset below
        sh.tot[s] += gg;
        sh.beta_eval[s] = a.tau * (sh.gamma[s] - (double)sh.theta[s]);
      }
      if (threadIdx.x < NG) {   // H's off-identity terms after the evaluation's status flips
        const double hv = sh.Htot[threadIdx.x] + sh.tot[S + threadIdx.x];
        sh.Htot[threadIdx.x] = hv;
        sh.Hf[threadIdx.x] = (float)(hv * a.inv_tau);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double nrm = 0.0;        // ||U^T w||^2
        for (int s = 0; s < S; ++s) nrm += sh.phi_cur[s];
        sh.scale = fmax(1.0, nrm);   // the stopping test compares squared norms
        for (int s = 0; s < S; ++s) {
          sh.dir[s] = 0.0;
          sh.phi_cur[s] = 0.0;
        }
        sh.nphi_cur = 0.0;
        sh.tstep = 1.0;
        sh.halvings = 0;
        sh.accepted = 0;
        sh.first = true;
        sh.done = 0;
      }
      __syncthreads();
      const int max_evals = a.maxit * 8;
      int my_evals = 1;
      if (threadIdx.x == 0) {
        t0 = tracer(a) ? globaltimer() : 0;
        NewtonState<S> ns{sh.beta, sh.beta_eval, sh.dir, sh.phi_cur, &sh.nphi_cur, &sh.tstep, &sh.halvings,
                          &sh.accepted, &sh.first, &sh.accepted_last};
        const int done = newton_decide<S>(ns, sh.tot, sh.Hf, a.tol * a.tol * sh.scale, a.maxit,
                                          my_evals >= max_evals);
        sh.done = done;
        if (done) last_newton = sh.accepted;
        if (tracer(a)) tr_add(a, 3, globaltimer() - t0);
      }
      __syncthreads();
      while (!sh.done) {
        if (threadIdx.x < S) {
          sh.theta[threadIdx.x] = (float)(sh.gamma[threadIdx.x] - sh.beta_eval[threadIdx.x] * a.inv_tau);
          sh.gam[threadIdx.x] = (float)sh.gamma[threadIdx.x];
        }
        __syncthreads();
        t0 = tracer(a) ? globaltimer() : 0;
        pass_newton<S, false>(&sh, src, xw);
        if (tracer(a)) tr_add(a, 2, globaltimer() - t0);
        if (!grid_reduce<NV>(sh.blk, sh.tot, a, ep, 4)) return;
        ++my_evals;
        if (threadIdx.x < NG) {   // the thread-parallel part of the decision: H's off-identity terms
          const double hv = sh.Htot[threadIdx.x] + sh.tot[S + threadIdx.x];
          sh.Htot[threadIdx.x] = hv;
          sh.Hf[threadIdx.x] = (float)(hv * a.inv_tau);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          t0 = tracer(a) ? globaltimer() : 0;
          NewtonState<S> ns{sh.beta, sh.beta_eval, sh.dir, sh.phi_cur, &sh.nphi_cur, &sh.tstep, &sh.halvings,
                            &sh.accepted, &sh.first, &sh.accepted_last};
          const int done = newton_decide<S>(ns, sh.tot, sh.Hf, a.tol * a.tol * sh.scale, a.maxit,
                                            my_evals >= max_evals);
          sh.done = done;
          if (done) last_newton = sh.accepted;
          if (tracer(a)) tr_add(a, 3, globaltimer() - t0);
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        newton_max = max(newton_max, last_newton);
        newton_total += last_newton;
      }
      evals += my_evals;
      if (!sh.accepted_last) {
        // the last evaluation was a rejected trial: write x for the accepted beta
        if (threadIdx.x < S) sh.theta[threadIdx.x] = (float)(sh.gamma[threadIdx.x] - sh.beta[threadIdx.x] * a.inv_tau);
        __syncthreads();
        pass_fixup<S>(&sh, xw);
        if (!final_eval && !grid_reduce<0>(nullptr, nullptr, a, ep, 5)) return;
      }
    }
    if (final_eval) break;
    long long t_pre = 0;
    if (tracer(a)) t_pre = globaltimer();
    pass_dual<TV>(&sh.a, a.mom[j]);
    if (tracer(a)) {
      // block 0's own time in the dual update and in the work since the last barrier
      const long long t_post = globaltimer();
      tr_acc()[0] += t_post - t_pre;
      tr_acc()[1] += t_pre - tr_acc()[TR_SLOTS];
    }
    if (!grid_reduce<0>(nullptr, nullptr, a, ep, 6)) return;
  }
  if (tracer(a)) {
    for (int k = 0; k < TR_SLOTS; ++k) a.trace[2 * TR_ACC + k] = tr_acc()[k];
    a.trace[0] = ep.all;                // number of barriers passed; entry 0 also holds the start time
    if ((int)ep.all + 1 < TR_ACC) {
      a.trace[2 * (ep.all + 1)] = 99;   // end of kernel
      a.trace[2 * (ep.all + 1) + 1] = globaltimer();
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
  const size_t dyn = (size_t)wp_slots(S) * WP_THREADS * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(k_wprox<S, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wprox<S, TV>, WP_THREADS, dyn);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int blocks = h->wp.nsm * std::min(per_sm, WP_BPS);
  if (blocks > WP_GS * WP_MAXG) return cudaErrorInvalidConfiguration;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((void*)k_wprox<S, TV>, dim3(blocks), dim3(WP_THREADS), args, dyn, h->stream);
}

#ifdef MQ_WP_HIGH
template <int TV>
cudaError_t dispatch_high_tv(mqnpm_handle* h, int S, WpArgs& a) {
  switch (S) {
    case 9: return launch_wprox<9, TV>(h, a);
    case 10: return launch_wprox<10, TV>(h, a);
    case 11: return launch_wprox<11, TV>(h, a);
    case 12: return launch_wprox<12, TV>(h, a);
    case 13: return launch_wprox<13, TV>(h, a);
    case 14: return launch_wprox<14, TV>(h, a);
    case 15: return launch_wprox<15, TV>(h, a);
    case 16: return launch_wprox<16, TV>(h, a);
    default: return cudaErrorInvalidValue;
  }
}

#else
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
    default: return wprox_dispatch_high(h, S, TV, &a);
  }
}
#endif

#define CK(call)                                                \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return set_cuda_error(h, e_, #call); \
  } while (0)

}  // namespace

#ifdef MQ_WP_HIGH
// Ranks 9-16, instantiated in a second compilation of this file (MQ_WP_HIGH)
// to keep each translation unit's build short.  args points to the WpArgs of
// the calling unit (the same definition, compiled from this file).
cudaError_t wprox_dispatch_high(mqnpm_handle* h, int S, int tv, void* args) {
  WpArgs& a = *static_cast<WpArgs*>(args);
  return tv == MQNPM_TV_ISO ? dispatch_high_tv<MQNPM_TV_ISO>(h, S, a) : dispatch_high_tv<MQNPM_TV_ANISO>(h, S, a);
}
#else

int wprox_impl(mqnpm_handle* h, const float* v, double tau, const UPtrs& U, int S_eff, double c, float* P_warm,
               bool warm, float* x_out) {
  if (S_eff < 0 || S_eff > MQNPM_MAX_S) return set_error(h, MQNPM_ERR_INVALID_ARG, "wprox: S_eff out of range");
  if (h->nx % 4 != 0) return set_error(h, MQNPM_ERR_UNSUPPORTED, "wprox: the x edge of the grid must be a multiple of 4");
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  const int J = h->dual_iters;
  if ((int)h->wp.mom_len != J) return set_error(h, MQNPM_ERR_STATE, "wprox: momentum table not initialised");
  // 16-byte vector access needs 16-byte aligned vectors
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!aligned(v) || !aligned(x_out) || (P_warm && !aligned(P_warm)))
    return set_error(h, MQNPM_ERR_INVALID_ARG, "wprox: vectors must be 16-byte aligned");
  for (int q = 0; q < S_eff; ++q)
    if (!aligned(U.u[q])) return set_error(h, MQNPM_ERR_INVALID_ARG, "wprox: U rows must be 16-byte aligned");
  if (warm && P_warm) {
    CK(cudaMemcpyAsync(h->wp.Pd, P_warm, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemsetAsync(h->wp.Pd, 0, 3 * N * sizeof(float), s));
  }
  CK(cudaMemcpyAsync(h->wp.R, h->wp.Pd, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(h->wp.err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(h->wp.barrier, 0, wprox_barrier_words() * sizeof(unsigned), s));
  if (S_eff > 0) CK(cudaMemsetAsync(h->wp.status, 1, N, s));
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
  a.count = h->wp.barrier;
  a.count_groups = h->wp.barrier + 1;
  a.gcount = h->wp.barrier + 2;
  a.err = h->wp.err;
  a.stat = h->wp.stat;
  a.status = h->wp.status;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.N = (int)N;
  a.J = J;
  a.tau = tau;
  a.c = c;
  a.inv_tau = 1.0 / tau;
  a.c_tau = c / tau;
  a.c_tau2 = c / (tau * tau);
  a.cdt = (float)(c / tau);
  a.lo = (float)h->lo;
  a.hi = (float)h->hi;
  a.step = (float)(tau / (4.0 * 3.0 * c));
  a.tol = h->newton_tol;
  a.maxit = h->newton_maxit;
  a.limit = h->barrier_limit;   // per wait (default about 2 s at 2 GHz)
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
int wprox_blocks_per_sm() { return WP_BPS; }
size_t wprox_part_count(int max_blocks) { return (size_t)(max_blocks + 2 * WP_MAXG) * NVMAX; }
int wprox_barrier_words() { return 2 + WP_MAXG; }
#endif
