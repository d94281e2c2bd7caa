// Fused x and y passes of the Green's apply on square planes (nx = ny = n,
// Px = Py = P = 2n): passes 1+2 (forward) and 4+5 (inverse) of the pruned
// padded convolution without the intermediate T1 / T4 arrays in HBM.
//
// One thread-block cluster of two CTAs works on one (slot, z-plane) task at a
// time (persistent over tasks).  CTA r of the pair keeps rows y in
// [r n/2, (r+1) n/2) of the plane, all P x-frequencies, in shared memory
// (128 KB at P = 256).  Forward: each CTA transforms its rows along x (pass 1's
// register DFTs and fused prologue), the pair synchronises, then each CTA
// transforms half of the kx columns along y (pass 2's register DFTs), reading
// the other half of the rows from its peer's shared memory (distributed shared
// memory), and writes T2.  Inverse: each CTA transforms half of the kx columns
// of T3 along y (pass 4), writing the kept rows y < n into its own or its
// peer's plane buffer, the pair synchronises, then each CTA transforms its rows
// along x (pass 5) with the fused epilogue.
//
// The arithmetic is pass 1/2/4/5's, operation for operation (same register
// DFTs, same twiddle values, same complex products), so the outputs are
// bit-identical to the unfused passes.  The per-CTA partial sums of the
// prologues and epilogues are formed per group of LPB lines of the unfused
// row shape (the same warps, the same FP32 warp tree and FP64 order), so the
// BiCGSTAB scalars are bit-identical too and the partials keep the unfused
// layout [slot][line / LPB][K].
#pragma once
#include <cooperative_groups.h>

#include "green_passes.cuh"

template <int P>
struct FusedShape {
  using PL = Plan<P>;
  static constexpr int R1 = PL::R1, R2 = PL::R2, T = PL::T;
  static constexpr int THREADS = 512;
  static constexpr int N = P / 2;                  // plane edge
  static constexpr int ROWS = N / 2;               // rows kept per CTA
  static constexpr int LB = THREADS / T;           // lines one pass of the threads covers
  static constexpr int LINES = LB < ROWS ? LB : ROWS;   // lines per x batch
  static constexpr int LPBV = RowShape<P, 0>::LPB; // lines per CTA of the unfused row passes
  static constexpr int PITCH = R1 + 1, PER_LINE = R2 * PITCH;   // x exchange (as the row passes)
  static constexpr int CB = THREADS / T;           // columns one pass of the threads covers
  static constexpr int C = CB < P / 2 ? CB : P / 2;   // columns per y batch
  static constexpr int EX = (LINES * PER_LINE > P * C) ? LINES * PER_LINE : P * C;   // float2
  // shared memory: linear twiddles [P], column table [R2][R1], plane [ROWS][P], exchange
  static constexpr size_t SMEM = (size_t)(P + R1 * R2 + ROWS * P + EX) * sizeof(float2);
  static constexpr bool OK = (R1 % 4 == 0) && (R2 % 4 == 0) && (R1 % T == 0) && (R2 % T == 0) &&
                             (LINES % LPBV == 0) && (ROWS % LINES == 0) && ((P / 2) % C == 0) &&
                             (LPBV * T) % 32 == 0 && SMEM <= 220 * 1024;
  static constexpr int WPV = LPBV * T / 32;        // warps per unfused row CTA
};

// Per-group-of-LPBV-lines partial sums (the unfused row pass's CTA), in its
// order: FP32 warp tree, FP64 sum over the group's warps.  nvirt groups start
// at line group vcta0.  Every thread of the block calls it.
template <int K, int WPV>
MQ_D void fused_partials(const Parts<K>& p, double* scratch, double* partials, int b, int nctas, int vcta0,
                         int nvirt) {
  if constexpr (K > 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float w = warp_sumf(p.v[k]);
      if (lane == 0) scratch[warp * K + k] = (double)w;
    }
    __syncthreads();
    if (threadIdx.x < nvirt * K) {
      const int j = threadIdx.x / K, k = threadIdx.x - (threadIdx.x / K) * K;
      double s = 0.0;
      for (int w = 0; w < WPV; ++w) s += scratch[(j * WPV + w) * K + k];
      partials[((size_t)b * nctas + vcta0 + j) * K + k] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------- forward: x (pass 1) + y (pass 2)
// T2 [b][z][ky < P][kx < P]; partials as pass 1 (nctas = ceil(n nz / LPB)).
template <int P, class Pro>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(FusedShape<P>::THREADS, 1)
k_pass12(Pro pro, float2* __restrict__ T2, int nz, int nb, const float2* __restrict__ twg,
         const KState* __restrict__ st, double* __restrict__ partials, int nctas) {
  using FS = FusedShape<P>;
  constexpr int R1 = FS::R1, R2 = FS::R2, T = FS::T, ROWS = FS::ROWS, C = FS::C, N = FS::N;
  constexpr int I1 = R2 / T, I2 = R1 / T;   // sub-DFTs per thread and stage
  constexpr int OWN = R1 / 4;               // n1 < OWN: rows of CTA 0 (y = R2 n1 + n2 < ROWS)
  static_assert(FS::OK, "fused x/y passes: unsupported length");
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  extern __shared__ float2 sm[];
  float2* twl = sm;                    // W_P^j, j < P (row passes)
  float2* twt = twl + P;               // [R2][R1] W_P^(a b) (column passes)
  float2* plane = twt + R1 * R2;       // [ROWS][P]
  float2* ex = plane + ROWS * P;
  float2* peer = cl.map_shared_rank(plane, r ^ 1);
  __shared__ double scratch[(FS::THREADS / 32) * 2 + 2];
  for (int i = threadIdx.x; i < P; i += blockDim.x) twl[i] = twg[i];
  load_twiddle_table<P>(twt, twg);
  __syncthreads();
  const int ncl = gridDim.x / 2, cid = blockIdx.x / 2;
  for (int task = cid; task < nb * nz; task += ncl) {
    const int b = task / nz, z = task - (task / nz) * nz;
    if (!slot_active(st, b)) continue;   // the same for both CTAs of the pair
    pro.begin(b);
    // ---- x transforms of this CTA's rows (pass 1)
    for (int yb = 0; yb < ROWS; yb += FS::LINES) {
      const int l = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
      const bool lv = l < FS::LINES;
      const int y = r * ROWS + yb + l;
      float2* exl = ex + l * FS::PER_LINE;
      Parts<Pro::NPART> parts;
      parts.zero();
      if (lv) {
#pragma unroll
        for (int i = 0; i < I1; ++i) {
          const int n2 = t + T * i;
          float2 a[R1];
#pragma unroll
          for (int n1 = 0; n1 < R1; ++n1) {
            a[n1] = make_float2(0.f, 0.f);
            if (n1 < R1 / 2) a[n1] = pro.load(b, R2 * n1 + n2, y, z, parts);
          }
          dft<R1, false, R1 / 2>(a);
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) exl[n2 * FS::PITCH + k1] = cmul(a[k1], twl[n2 * k1]);
        }
      }
      __syncthreads();
      if (lv) {
#pragma unroll
        for (int i = 0; i < I2; ++i) {
          const int k1 = t + T * i;
          float2 a[R2];
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) a[n2] = exl[n2 * FS::PITCH + k1];
          dft<R2, false>(a);
          float2* o = plane + (yb + l) * P;
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) o[k1 + R1 * k2] = a[k2];
        }
      }
      fused_partials<Pro::NPART, FS::WPV>(parts, scratch, partials, b, nctas, (z * N + r * ROWS + yb) / FS::LPBV,
                                          FS::LINES / FS::LPBV);
      __syncthreads();   // the exchange is reused by the next batch
    }
    cl.sync();           // both halves of the plane are complete
    // ---- y transforms of this CTA's half of the kx columns (pass 2)
    float2* dst = T2 + ((size_t)b * nz + z) * P * P;
    for (int kb = 0; kb < P / 2; kb += C) {
      const int t = threadIdx.x / C, c = threadIdx.x - (threadIdx.x / C) * C;
      const bool tv = t < T;
      const int kx = r * (P / 2) + kb + c;
      if (tv) {
#pragma unroll
        for (int i = 0; i < I1; ++i) {
          const int n2 = t + T * i;
          float2 a[R1];
#pragma unroll
          for (int n1 = 0; n1 < R1; ++n1) {
            a[n1] = make_float2(0.f, 0.f);
            if (n1 < R1 / 2) {
              const int owner = n1 / OWN;   // rows of CTA 0, then of CTA 1
              const int idx = (R2 * n1 + n2 - owner * ROWS) * P + kx;
              a[n1] = owner == r ? plane[idx] : peer[idx];   // own shared memory, or the peer's
            }
          }
          dft<R1, false, R1 / 2>(a);
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) ex[(n2 * R1 + k1) * C + c] = cmul(a[k1], twt[n2 * R1 + k1]);
        }
      }
      __syncthreads();
      if (tv) {
#pragma unroll
        for (int i = 0; i < I2; ++i) {
          const int k1 = t + T * i;
          float2 a[R2];
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) a[n2] = ex[(n2 * R1 + k1) * C + c];
          dft<R2, false>(a);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) dst[(size_t)(k1 + R1 * k2) * P + kx] = a[k2];
        }
      }
      __syncthreads();
    }
    cl.sync();           // the peer has read this plane buffer before it is overwritten
  }
}

// ---------------------------------------------- inverse: y (pass 4) + x (pass 5)
// T3 [b][z][ky < P][kx < P] in T2's storage; partials as pass 5.
template <int P, class Epi>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(FusedShape<P>::THREADS, 1)
k_pass45(Epi epi, const float2* __restrict__ T2, int nz, int nb, const float2* __restrict__ twg,
         const KState* __restrict__ st, double* __restrict__ partials, int nctas) {
  using FS = FusedShape<P>;
  constexpr int R1 = FS::R1, R2 = FS::R2, T = FS::T, ROWS = FS::ROWS, C = FS::C, N = FS::N;
  constexpr int I1 = R2 / T, I2 = R1 / T;
  constexpr int OWN = R2 / 4;               // k2 < OWN: rows y = k1 + R1 k2 of CTA 0
  static_assert(FS::OK, "fused x/y passes: unsupported length");
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  extern __shared__ float2 sm[];
  float2* twl = sm;
  float2* twt = twl + P;
  float2* plane = twt + R1 * R2;
  float2* ex = plane + ROWS * P;
  float2* peer = cl.map_shared_rank(plane, r ^ 1);
  __shared__ double scratch[(FS::THREADS / 32) * 3 + 3];
  for (int i = threadIdx.x; i < P; i += blockDim.x) twl[i] = twg[i];
  load_twiddle_table<P>(twt, twg);
  __syncthreads();
  const int ncl = gridDim.x / 2, cid = blockIdx.x / 2;
  for (int task = cid; task < nb * nz; task += ncl) {
    const int b = task / nz, z = task - (task / nz) * nz;
    if (!slot_active(st, b)) continue;
    // ---- y inverse of this CTA's half of the kx columns (pass 4): rows y < n
    const float2* src = T2 + ((size_t)b * nz + z) * P * P;
    for (int kb = 0; kb < P / 2; kb += C) {
      const int t = threadIdx.x / C, c = threadIdx.x - (threadIdx.x / C) * C;
      const bool tv = t < T;
      const int kx = r * (P / 2) + kb + c;
      if (tv) {
#pragma unroll
        for (int i = 0; i < I1; ++i) {
          const int n2 = t + T * i;
          float2 a[R1];
#pragma unroll
          for (int n1 = 0; n1 < R1; ++n1) a[n1] = src[(size_t)(R2 * n1 + n2) * P + kx];
          dft<R1, true, R1>(a);
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) ex[(n2 * R1 + k1) * C + c] = cmul(a[k1], cconj(twt[n2 * R1 + k1]));
        }
      }
      __syncthreads();
      if (tv) {
#pragma unroll
        for (int i = 0; i < I2; ++i) {
          const int k1 = t + T * i;
          float2 a[R2];
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) a[n2] = ex[(n2 * R1 + k1) * C + c];
          dft<R2, true>(a);
#pragma unroll
          for (int k2 = 0; k2 < R2 / 2; ++k2) {
            const int owner = k2 / OWN;
            const int idx = (k1 + R1 * k2 - owner * ROWS) * P + kx;
            if (owner == r) plane[idx] = a[k2];
            else peer[idx] = a[k2];
          }
        }
      }
      __syncthreads();
    }
    cl.sync();           // this CTA's rows are complete (half of them written by the peer)
    // ---- x inverse of this CTA's rows (pass 5) with the epilogue
    for (int yb = 0; yb < ROWS; yb += FS::LINES) {
      const int l = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
      const bool lv = l < FS::LINES;
      const int y = r * ROWS + yb + l;
      float2* exl = ex + l * FS::PER_LINE;
      const float2* row = plane + (yb + l) * P;
      Parts<Epi::NPART> parts;
      parts.zero();
      if (lv) {
#pragma unroll
        for (int i = 0; i < I1; ++i) {
          const int n2 = t + T * i;
          float2 a[R1];
#pragma unroll
          for (int n1 = 0; n1 < R1; ++n1) a[n1] = row[R2 * n1 + n2];
          dft<R1, true>(a);
#pragma unroll
          for (int k1 = 0; k1 < R1; ++k1) exl[n2 * FS::PITCH + k1] = cmul(a[k1], cconj(twl[n2 * k1]));
        }
      }
      __syncthreads();
      if (lv) {
#pragma unroll
        for (int i = 0; i < I2; ++i) {
          const int k1 = t + T * i;
          float2 a[R2];
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) a[n2] = exl[n2 * FS::PITCH + k1];
          dft<R2, true>(a);
#pragma unroll
          for (int k2 = 0; k2 < R2 / 2; ++k2) epi.store(b, k1 + R1 * k2, y, z, a[k2], parts);
        }
      }
      fused_partials<Epi::NPART, FS::WPV>(parts, scratch, partials, b, nctas, (z * N + r * ROWS + yb) / FS::LPBV,
                                          FS::LINES / FS::LPBV);
      __syncthreads();
    }
    cl.sync();           // the peer is done with this CTA's buffer before the next task writes it
  }
}
