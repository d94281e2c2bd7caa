// The five passes of the pruned, zero-padded Green's convolution
// (G v)|_domain = crop( IFFT_P( K_hat * FFT_P( pad_P(v) ) ) ),  P_d = 2 n_d,
// batched over the illuminations of a mini-batch (grid dimension "b").  Each
// pass is compiled for the transform length of its own axis (the template
// argument P): Px for passes 1 and 5, Py for passes 2 and 4, Pz for pass 3.
//
// Layout (complex64, x fastest everywhere):
//   volume   v [b][z][y][x]              nz*ny*nx
//   T1 / T4    [b][z][y][kx]             nz*ny*Px   (after / before the x pass)
//   T2 / T3    [b][z][ky][kx]            nz*Py*Px   (after / before the y pass)
//   K_hat octant [fz][fy][fx]            (nz+1)(ny+1)(nx+1) (K_hat is even in each axis)
// Pass 1 (x, rows)    : ny*nz lines, nx nonzero inputs -> Px outputs   + fused prologue
// Pass 2 (y, columns) : nz*Px columns, ny nonzero inputs -> Py outputs
// Pass 3 (z, columns) : Py*Px columns, forward, * K_hat, inverse, nz outputs kept
// Pass 4 (y, columns) : nz*Px columns, Py inputs -> ny outputs kept
// Pass 5 (x, rows)    : ny*nz lines, Px inputs -> nx outputs kept      + fused epilogue
// Zero rows of the padding are never read and cropped outputs never written.
// The 1/P^3 of the inverse transform is folded into K_hat.
#pragma once
#include <cuda.h>   // CUtensorMap

#include "fft.cuh"
#include "kstate.h"

// ----------------------------------------------------------- CTA shapes
// Every transform length has two row shapes (passes 1 and 5) and two column
// shapes (passes 2-4); V = 0 is the default, V = 1 the alternative the
// autotuner also times.  Where the plan's threads per line T is below R2 (T
// is limited to a common divisor of R1 and R2), the alternative gives every
// line or column R1 threads, one middle-stage DFT each (the other stage leaves
// R1 - R2 of them idle); elsewhere it halves the lines or columns per CTA, or
// doubles them where the default CTA has fewer than 128 threads.
constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

template <int P>
struct RowBase {
  using PL = Plan<P>;
  static constexpr int PITCH = PL::R1 + 1;                 // padded exchange row
  static constexpr int PER_LINE = PL::R2 * PITCH;
  static constexpr bool WIDE = PL::T < PL::R2;
  static constexpr int LPB0 = 256 / PL::T;
  static constexpr int LPB_DEF = (LPB0 * PER_LINE * 8 > 40960) ? (40960 / (PER_LINE * 8) >= 16 ? 16 : 8) : LPB0;
  static constexpr int T_ALT = WIDE ? PL::R1 : PL::T;
  // wide: the most lines, in steps that keep whole warps, with at most 320
  // threads and 48 KB of shared memory
  static constexpr int Q = 32 / gcd_c(T_ALT, 32);
  static constexpr int LPB_W0 = 320 / T_ALT < (49152 / 8 - P) / PER_LINE ? 320 / T_ALT : (49152 / 8 - P) / PER_LINE;
  static constexpr int LPB_W = (LPB_W0 / Q) * Q;
  static constexpr int LPB_ALT = WIDE ? LPB_W : (LPB_DEF * PL::T >= 128 ? LPB_DEF / 2 : 2 * LPB_DEF);
};
template <int P, int V = 0>
struct RowShape : RowBase<P> {
  static_assert(V == 0 || V == 1, "two row shapes");
  static constexpr int T = V == 0 ? Plan<P>::T : RowBase<P>::T_ALT;
  static constexpr int LPB = V == 0 ? RowBase<P>::LPB_DEF : RowBase<P>::LPB_ALT;
  static constexpr int THREADS = LPB * T;
  static_assert(LPB >= 1 && THREADS % 32 == 0, "whole warps (the partial sums reduce per warp)");
  static constexpr int SMEM = (P + LPB * RowBase<P>::PER_LINE) * 8;
};
template <int P>
struct ColBase {
  using PL = Plan<P>;
  static constexpr bool WIDE = PL::T < PL::R2;
  static constexpr int C0 = 256 / PL::T;
  static constexpr int C1 = C0 > P ? P : C0;
  static constexpr int C_DEF = (C1 * P * 8 > 40960) ? 16 : C1;
  static constexpr int C_UP = 2 * C_DEF;
  static constexpr int C_ALT = WIDE ? C_DEF
                               : (C_DEF * PL::T < 128 && C_UP <= P && P % C_UP == 0) ? C_UP : C_DEF / 2;
  static constexpr int T_ALT = WIDE ? PL::R1 : PL::T;
};
template <int P, int V = 0>
struct ColShape : ColBase<P> {
  static_assert(V == 0 || V == 1, "two column shapes");
  static constexpr int T = V == 0 ? Plan<P>::T : ColBase<P>::T_ALT;
  static constexpr int C = V == 0 ? ColBase<P>::C_DEF : ColBase<P>::C_ALT;
  static_assert(P % C == 0 && C % 2 == 0, "column tiles divide P; TMA rows of 16-byte multiples");
  static constexpr int THREADS = C * T;
  static constexpr int SMEM = (P + P * C) * 8;
};

// Co-resident CTAs per SM the x-forward pass is compiled for where its CTA
// has 256 threads and the length is at most 256: five, i.e. at most 48
// registers per thread, the occupancy this HBM-bound pass needs to keep its
// loads in flight (spill-free by ptxas; the other shapes and the x-inverse
// pass with its BiCGSTAB epilogues would spill under the cap and are left
// unbounded).
template <int P, int THREADS>
struct StreamOcc {
  static constexpr int MINB = (P <= 256 && THREADS == 256) ? 5 : 1;
};

// Per-thread FP32 partial sums, reduced per CTA into FP64 partials.
template <int K>
struct Parts {
  float v[K > 0 ? K : 1];
  MQ_D void zero() {
#pragma unroll
    for (int k = 0; k < (K > 0 ? K : 1); ++k) v[k] = 0.f;
  }
};

template <int K>
MQ_D void write_partials(const Parts<K>& p, double* partials, int b, int cta, int nctas) {
  if constexpr (K > 0) {
    __shared__ double scratch[33 * K];
    double out[K];
    block_sum_f<K>(p.v, scratch, out);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) partials[((size_t)b * nctas + cta) * K + k] = out[k];
    }
  }
}

// active == 2: the slot met the tolerance at the half step of its iteration
// and skips the rest of that iteration's second apply.
MQ_D bool slot_active(const KState* st, int b) { return st == nullptr || st[b].active == 1; }

// Twiddles W_P^(r q) as an R2 x R1 table in shared memory (r < R2, q < R1): a
// thread whose first-stage index n2 is fixed reads row n2 at compile-time
// offsets, with no per-element index arithmetic.  Only for the column passes,
// whose warps hold two values of n2 (the row passes keep a linear table: their
// warps hold sixteen, and rows 128 bytes apart would share banks).
template <int P>
MQ_D void load_twiddle_table(float2* tw, const float2* __restrict__ twg) {
  constexpr int R1 = Plan<P>::R1, R2 = Plan<P>::R2;
  for (int i = threadIdx.x; i < R1 * R2; i += blockDim.x) {
    const int r = i / R1, q = i - (i / R1) * R1;
    tw[i] = twg[r * q];
  }
}

// ------------------------------------------------------- pass 1: x forward
template <int P, int RV, class Pro>
__global__ void __launch_bounds__(RowShape<P, RV>::THREADS, StreamOcc<P, RowShape<P, RV>::THREADS>::MINB)
k_pass1(Pro pro, float2* __restrict__ T1, int ny, int nyz, const float2* __restrict__ twg,
        const KState* __restrict__ st, double* __restrict__ partials, int line0, int nlines) {
  using PL = Plan<P>;
  using SH = RowShape<P, RV>;
  constexpr int R1 = PL::R1, R2 = PL::R2, T = SH::T;
  constexpr int I1 = (R2 + T - 1) / T, I2 = (R1 + T - 1) / T;   // sub-DFTs per thread and stage
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* ex = sm + P;
  const int b = blockIdx.y;
  if (!slot_active(st, b)) return;
  pro.begin(b);
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
  const int l = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
  const int line = line0 + blockIdx.x * SH::LPB + l;   // rows [line0, line0 + nlines) of [z][y]
  const bool valid = line < line0 + nlines;
  const int z = line / ny, y = line - (line / ny) * ny;
  float2* exl = ex + l * SH::PER_LINE;
  Parts<Pro::NPART> parts;
  parts.zero();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < I1; ++i) {
    const int n2 = t + T * i;
    if (R2 % T != 0 && n2 >= R2) continue;   // idle in this stage
    float2 a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      a[n1] = make_float2(0.f, 0.f);
      if (n1 < R1 / 2 && valid) a[n1] = pro.load(b, R2 * n1 + n2, y, z, parts);
    }
    dft<R1, false, R1 / 2>(a);   // inputs n1 >= R1/2 are the zero padding
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) exl[n2 * SH::PITCH + k1] = cmul(a[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < I2; ++i) {
    const int k1 = t + T * i;
    if (R1 % T != 0 && k1 >= R1) continue;
    float2 a[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) a[n2] = exl[n2 * SH::PITCH + k1];
    dft<R2, false>(a);
    if (valid) {
      float2* o = T1 + ((size_t)b * nyz + line) * P;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) o[k1 + R1 * k2] = a[k2];
    }
  }
  write_partials<Pro::NPART>(parts, partials, b, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------- pass 5: x inverse
template <int P, int RV, class Epi>
__global__ void __launch_bounds__(RowShape<P, RV>::THREADS)
k_pass5(Epi epi, const float2* __restrict__ T4, int ny, int nyz, const float2* __restrict__ twg,
        const KState* __restrict__ st, double* __restrict__ partials, int line0, int nlines) {
  using PL = Plan<P>;
  using SH = RowShape<P, RV>;
  constexpr int R1 = PL::R1, R2 = PL::R2, T = SH::T;
  constexpr int I1 = (R2 + T - 1) / T, I2 = (R1 + T - 1) / T;   // sub-DFTs per thread and stage
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* ex = sm + P;
  const int b = blockIdx.y;
  if (!slot_active(st, b)) return;
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
  const int l = threadIdx.x / T, t = threadIdx.x - (threadIdx.x / T) * T;
  const int line = line0 + blockIdx.x * SH::LPB + l;   // rows [line0, line0 + nlines) of [z][y]
  const bool valid = line < line0 + nlines;
  const int z = line / ny, y = line - (line / ny) * ny;
  float2* exl = ex + l * SH::PER_LINE;
  const float2* src = T4 + ((size_t)b * nyz + (valid ? line : line0)) * P;
  Parts<Epi::NPART> parts;
  parts.zero();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < I1; ++i) {
    const int n2 = t + T * i;
    if (R2 % T != 0 && n2 >= R2) continue;   // idle in this stage
    float2 a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) a[n1] = valid ? src[R2 * n1 + n2] : make_float2(0.f, 0.f);
    dft<R1, true>(a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) exl[n2 * SH::PITCH + k1] = cmul(a[k1], cconj(tw[n2 * k1]));
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < I2; ++i) {
    const int k1 = t + T * i;
    if (R1 % T != 0 && k1 >= R1) continue;
    float2 a[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) a[n2] = exl[n2 * SH::PITCH + k1];
    dft<R2, true>(a);
    if (valid) {
#pragma unroll
      for (int k2 = 0; k2 < R2 / 2; ++k2) epi.store(b, k1 + R1 * k2, y, z, a[k2], parts);
    }
  }
  write_partials<Epi::NPART>(parts, partials, b, blockIdx.x, gridDim.x);
}

// ------------------------------------------------- passes 2 and 4: y columns
// P = Py; rows of px = Px values (the x pass's output pitch).  SQ: Px = Py,
// so the row pitch is the compile-time P and the column loads and stores take
// immediate offsets from one base (the cube's case).
// INV = false: T1 [b][z][y < ny][kx] -> T2 [b][z][ky < P][kx]
// INV = true : T3 [b][z][ky < P][kx] -> T4 [b][z][y < ny][kx]
template <int P, int CV, bool INV, bool SQ>
__global__ void __launch_bounds__(ColShape<P, CV>::THREADS)
k_pass_y(const float2* __restrict__ in, float2* __restrict__ out, int nz, int px_arg,
         const float2* __restrict__ twg, const KState* __restrict__ st, int z0) {
  using PL = Plan<P>;
  using SH = ColShape<P, CV>;
  constexpr int R1 = PL::R1, R2 = PL::R2, T = SH::T, C = SH::C;
  constexpr int I1 = (R2 + T - 1) / T, I2 = (R1 + T - 1) / T;   // sub-DFTs per thread and stage
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* ex = sm + P;
  const int b = blockIdx.z;
  if (!slot_active(st, b)) return;
  load_twiddle_table<P>(tw, twg);
  const int px = SQ ? P : px_arg;
  const int t = threadIdx.x / C, c = threadIdx.x - (threadIdx.x / C) * C;
  const int kx = blockIdx.x * C + c;
  const bool kv = SQ || kx < px;   // the last column tile may reach past Px
  const int z = z0 + blockIdx.y;   // planes [z0, z0 + gridDim.y)
  constexpr int len_in = INV ? P : P / 2, len_out = INV ? P / 2 : P;
  const float2* src = in + ((size_t)b * nz + z) * len_in * px + kx;
  float2* dst = out + ((size_t)b * nz + z) * len_out * px + kx;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < I1; ++i) {
    const int n2 = t + T * i;
    if (R2 % T != 0 && n2 >= R2) continue;   // idle in this stage
    float2 a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      a[n1] = make_float2(0.f, 0.f);
      if ((INV || n1 < R1 / 2) && kv) a[n1] = src[(size_t)(R2 * n1 + n2) * px];
    }
    dft<R1, INV, INV ? R1 : R1 / 2>(a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 w = tw[n2 * R1 + k1];
      ex[(n2 * R1 + k1) * C + c] = cmul(a[k1], INV ? cconj(w) : w);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < I2; ++i) {
    const int k1 = t + T * i;
    if (R1 % T != 0 && k1 >= R1) continue;
    float2 a[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) a[n2] = ex[(n2 * R1 + k1) * C + c];
    dft<R2, INV>(a);
    if (kv) {
#pragma unroll
      for (int k2 = 0; k2 < (INV ? R2 / 2 : R2); ++k2) dst[(size_t)(k1 + R1 * k2) * px] = a[k2];
    }
  }
}

// ------------------------------------- pass 3: z forward, * K_hat, z inverse
// One CTA per (kx tile of C columns, ky) column set, looping over the batch
// slots.  K_hat is even in kz, so the CTA keeps only the folded half of its
// columns' spectrum (n + 1 rows) in shared memory, read once for all slots.
// A slot's input tile (rows z < n of the C columns, 16 KB at n = 128) arrives
// by one TMA tensor copy; as soon as the first transform stage has consumed
// it, the copy of the next active slot's tile is issued into the same buffer,
// so it overlaps the remaining three stages.  In place on T2/T3
// [b][z][ky][kx]; only rows z < n are read and written.
//
// Two exchange schemes (DB): with one exchange buffer the middle stage keeps
// its inverse-stage-A results in registers until every thread has read the
// buffer (four barriers per slot; 68 KB of shared memory at P = 256, three
// CTAs per SM).  With two, the middle stage writes them straight into the
// second buffer (two barriers per slot, no register-held stage: the choice for
// lengths whose threads carry several columns of a stage, e.g. P = 192, 320).
// Two plane modes (IO) serve applies that touch one z-plane.  IO_IN: the
// adjoint right-hand side G^H S^T r, whose input is nonzero on the detector
// plane z = n - 1 only: the forward z transform of a column is then the ramp
// v W_P^{(n-1) kz} = v (-1)^kz W_P^{-kz} (P = 2n), so the first stage, the
// forward half of the middle stage and the input tile are skipped.  IO_OUT: a
// forward apply of which only the detector plane is kept (the first-Born data
// S G(x u_in)): the inverse z transform shrinks to the one output
// x[n-1] = sum_kz Y[kz] (-1)^kz W_P^kz, a per-thread sum and a column
// reduction, and only row z = n - 1 is written.
enum Pass3IO { IO_FULL = 0, IO_IN = 1, IO_OUT = 2 };

template <int P, int CV, bool DB, int IO = IO_FULL>
struct Pass3Smem {
  using SH = ColShape<P, CV>;
  static constexpr int C = SH::C;
  static constexpr int KH = P / 2 + 1;   // folded kz rows of K_hat
  static constexpr MQ_HD size_t tw_off() { return 0; }
  static constexpr MQ_HD size_t kh_off() { return P * sizeof(float2); }
  static constexpr MQ_HD size_t ex_off() { return kh_off() + (size_t)KH * C * sizeof(float2); }
  static constexpr MQ_HD size_t ex2_off() { return ex_off() + (size_t)P * C * sizeof(float2); }
  static constexpr MQ_HD size_t in_off() {   // 1 KB aligned TMA destination
    const size_t o = ex_off() + (size_t)(DB ? 2 : 1) * P * C * sizeof(float2);
    return (o + 1023) & ~(size_t)1023;
  }
  static constexpr MQ_HD size_t in_bytes(int n) { return IO == IO_IN ? 0 : (size_t)n * C * sizeof(float2); }
  static constexpr MQ_HD size_t bar_off(int n) { return in_off() + in_bytes(n); }
  static constexpr MQ_HD size_t red_off(int n) { return bar_off(n) + 16; }   // IO_OUT: column partials [T][C]
  static constexpr MQ_HD size_t red_bytes() { return IO == IO_OUT ? (size_t)SH::T * C * sizeof(float2) : 0; }
  static constexpr MQ_HD size_t bytes(int n) { return red_off(n) + red_bytes() + 1024; }   // + base alignment slack
};

// Blocks per SM the pass-3 kernel is compiled for (register cap): three when
// its shared memory allows it.
template <int P, int CV, bool DB, int IO = IO_FULL>
struct Pass3Occ {
  using SM = Pass3Smem<P, CV, DB, IO>;
  static constexpr size_t SMEM = SM::in_off() + SM::in_bytes(P / 2) + SM::red_bytes() + 1040;
  static constexpr int MIN_BLOCKS = (3 * SMEM <= 220 * 1024 && ColShape<P, CV>::THREADS <= 256) ? 3
                                    : (2 * SMEM <= 220 * 1024) ? 2 : 1;
};

// SQ: a cubic grid (Px = Py = Pz = P), whose strides and K_hat folds are
// compile-time constants; otherwise nx, ny (and so Px, Py) come at run time.
template <int P, int CV, bool DB, bool CONJ, int IO = IO_FULL, bool SQ = true>
__global__ void __launch_bounds__(ColShape<P, CV>::THREADS, Pass3Occ<P, CV, DB, IO>::MIN_BLOCKS)
k_pass3(const __grid_constant__ CUtensorMap tmap, float2* __restrict__ T2, const float2* __restrict__ khat, int nx_arg,
        int ny_arg, int nb, const float2* __restrict__ twg, const KState* __restrict__ st, int* __restrict__ err) {
  using PL = Plan<P>;
  using SH = ColShape<P, CV>;
  using SM = Pass3Smem<P, CV, DB, IO>;
  constexpr int R1 = PL::R1, R2 = PL::R2, T = SH::T, C = SH::C, KH = SM::KH;
  constexpr bool PLANE = IO == IO_IN;
  static_assert(IO == IO_FULL || R1 % 2 == 0, "plane modes: (-1)^kz = (-1)^k1 needs an even R1");
  constexpr int I1 = (R2 + T - 1) / T, I2 = (R1 + T - 1) / T;   // sub-DFTs per thread and stage
  static_assert(R1 * R2 == P && R2 % 2 == 0, "two-stage plan with an even second factor");
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  float2* tw = reinterpret_cast<float2*>(sm + SM::tw_off());   // [R2][R1]: W_P^(a b)
  float2* kh = reinterpret_cast<float2*>(sm + SM::kh_off());
  float2* ex = reinterpret_cast<float2*>(sm + SM::ex_off());
  float2* ex2 = DB ? reinterpret_cast<float2*>(sm + SM::ex2_off()) : ex;   // inverse-stage exchange
  float2* in = reinterpret_cast<float2*>(sm + SM::in_off());
  constexpr int n = P / 2;   // nz: the z extent of the domain
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SM::bar_off(n));
  const int t = threadIdx.x / C, c = threadIdx.x - (threadIdx.x / C) * C;
  const int nx = SQ ? P / 2 : nx_arg, ny = SQ ? P / 2 : ny_arg;
  const int kx0 = blockIdx.x * C, kx = kx0 + c;
  const int ky = blockIdx.y;
  const int px = 2 * nx, py = 2 * ny;
  const bool kv = SQ || kx < px;   // the last column tile may reach past Px: those columns
                                   // are zero-filled by the tile load and never stored
  const size_t zs = (size_t)px * py;
  const int mx = nx + 1, mxy = (nx + 1) * (ny + 1);   // K_hat octant strides
  const uint32_t tile_bytes = (uint32_t)SM::in_bytes(n);
  unsigned long long act = 0ull;   // active slots as a bit mask (nb <= 64)
  for (int q = 0; q < nb; ++q)
    if (slot_active(st, q)) act |= 1ull << q;
  if (act == 0ull) return;
  int b = __ffsll((long long)act) - 1;
  if (!PLANE && threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async();
    mbar_expect_tx(bar, tile_bytes);
    tma_load_3d(in, &tmap, bar, kx0, ky, b * n);
  }
  // every thread reads its twiddle row (stage 1) or column (inverse stage A)
  // at compile-time offsets from one base
  load_twiddle_table<P>(tw, twg);
  {
    const int fx = !kv ? 0 : kx <= nx ? kx : px - kx;
    const int fy = ky <= ny ? ky : py - ky;
    const float2* kcol = khat + (size_t)fy * mx + fx;
    for (int fz = t; fz < KH; fz += T) {
      float2 v = kcol[(size_t)fz * mxy];
      if (CONJ) v.y = -v.y;
      kh[fz * C + c] = v;
    }
  }
  __syncthreads();
  uint32_t phase = 0u;
  while (true) {
    int next = nb;
    float2 vplane = make_float2(0.f, 0.f);
    if constexpr (PLANE) {
      // no tile: only the previous slot's last stage must be finished with ex
      __syncthreads();
      const unsigned long long rest = act & ~((2ull << b) - 1ull);
      next = rest ? __ffsll((long long)rest) - 1 : nb;
      vplane = kv ? T2[((size_t)b * n + (n - 1)) * zs + (size_t)ky * px + kx] : make_float2(0.f, 0.f);
    } else {
      if (!mbar_wait_bounded(bar, phase, 1 << 22)) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // the copy given up on is the only one in flight: give it one more bounded wait
        mbar_wait_bounded(bar, phase, 1 << 22);
        return;
      }
      phase ^= 1u;
      // forward stage 1 (n2-threads), inputs z = R2 n1 + n2 < n from the TMA tile [z][c]
#pragma unroll
      for (int i = 0; i < I1; ++i) {
        const int n2 = t + T * i;
        if (R2 % T != 0 && n2 >= R2) continue;   // idle in this stage
        float2 a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
          a[n1] = make_float2(0.f, 0.f);
          if (n1 < R1 / 2) a[n1] = in[(R2 * n1 + n2) * C + c];
        }
        dft<R1, false, R1 / 2>(a);   // inputs n1 >= R1/2 are the zero padding
        const float2* twr = tw + n2 * R1;
        float2* exw = ex + (n2 * R1) * C + c;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) exw[k1 * C] = (k1 == 0) ? a[0] : cmul(a[k1], twr[k1]);
      }
      __syncthreads();   // the tile is consumed: fetch the next active slot's into the same buffer
      const unsigned long long rest = act & ~((2ull << b) - 1ull);
      next = rest ? __ffsll((long long)rest) - 1 : nb;
      if (next < nb && threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(bar, tile_bytes);
        tma_load_3d(in, &tmap, bar, kx0, ky, next * n);
      }
    }   // !PLANE
    // forward stage 2 (k1-threads) -> multiply -> inverse stage A (same thread).
    // K_hat row of kz = k1 + R1 k2: kz itself for k2 < R2/2, else the folded P - kz.
    float2 zb[DB ? 1 : I2][R2];
    float2 opart = make_float2(0.f, 0.f);   // IO_OUT: this thread's share of x[n-1]
#pragma unroll
    for (int i = 0; i < I2; ++i) {
      const int k1 = t + T * i;
      if (R1 % T != 0 && k1 >= R1) continue;
      float2 a[R2];
      if constexpr (PLANE) {
        // X[k1 + R1 k2] = v (-1)^k1 conj(W_P^k1) conj(W_R2^k2)
        const float2 w1 = tw[R1 + k1];   // row 1 of the table: W_P^k1
        float2 base = cmul(vplane, make_float2(w1.x, -w1.y));
        if (k1 & 1) base = make_float2(-base.x, -base.y);
        static_for<R2>([&](auto k2c) {
          constexpr int k2 = decltype(k2c)::value;
          a[k2] = tw_mul<k2, R2, true>(base);
        });
      } else {
        const float2* exr = ex + k1 * C + c;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) a[n2] = exr[n2 * R1 * C];
        dft<R2, false>(a);
      }
      const float2* khA = kh + k1 * C + c;
      const float2* khB = kh + (P - k1) * C + c;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2)
        a[k2] = cmul(a[k2], k2 < R2 / 2 ? khA[k2 * R1 * C] : khB[-k2 * R1 * C]);
      if constexpr (IO == IO_OUT) {
        // sum_k2 Y[k1 + R1 k2] (-1)^k1 W_P^k1 W_R2^k2: no inverse stage A
        float2 acc = make_float2(0.f, 0.f);
        static_for<R2>([&](auto k2c) {
          constexpr int k2 = decltype(k2c)::value;
          acc = cadd(acc, tw_mul<k2, R2, false>(a[k2]));
        });
        acc = cmul(acc, tw[R1 + k1]);
        if (k1 & 1) acc = make_float2(-acc.x, -acc.y);
        opart = cadd(opart, acc);
        continue;
      }
      dft<R2, true>(a);   // over k2 -> j1
      const float2* twc = tw + k1;
      if constexpr (DB) {
        float2* exw = ex2 + (k1 * R2) * C + c;
#pragma unroll
        for (int j1 = 0; j1 < R2; ++j1) exw[j1 * C] = (j1 == 0) ? a[0] : cmul(a[j1], cconj(twc[j1 * R1]));
      } else {
#pragma unroll
        for (int j1 = 0; j1 < R2; ++j1) zb[i][j1] = (j1 == 0) ? a[0] : cmul(a[j1], cconj(twc[j1 * R1]));
      }
    }
    if constexpr (IO == IO_OUT) {
      // column sums in a fixed thread order; the barrier also ends every
      // thread's reads of ex, so the next slot's first stage may write it
      float2* red = reinterpret_cast<float2*>(sm + SM::red_off(n));
      red[t * C + c] = opart;
      __syncthreads();
      if (t == 0 && kv) {
        float2 x = red[c];
        for (int q = 1; q < T; ++q) x = cadd(x, red[q * C + c]);
        T2[((size_t)b * n + (n - 1)) * zs + (size_t)ky * px + kx] = x;
      }
      if (next >= nb) break;
      b = next;
      continue;
    }
    __syncthreads();
    if constexpr (!DB) {
#pragma unroll
      for (int i = 0; i < I2; ++i) {
        if (R1 % T != 0 && t + T * i >= R1) continue;
        float2* exw = ex + ((t + T * i) * R2) * C + c;
#pragma unroll
        for (int j1 = 0; j1 < R2; ++j1) exw[j1 * C] = zb[i][j1];
      }
      __syncthreads();
    }
    // inverse stage B (j1-threads): outputs z = j1 + R2 j2 for j2 < R1/2
    float2* colb = T2 + (size_t)b * n * zs + (size_t)ky * px + kx;
#pragma unroll
    for (int i = 0; i < I1; ++i) {
      const int j1 = t + T * i;
      if (R2 % T != 0 && j1 >= R2) continue;
      float2 a[R1];
      const float2* exr = ex2 + j1 * C + c;
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) a[k1] = exr[k1 * R2 * C];
      dft<R1, true>(a);
      if (kv) {
        float2* col = colb + (size_t)j1 * zs;
#pragma unroll
        for (int j2 = 0; j2 < R1 / 2; ++j2) {
          *col = a[j2];
          col += (size_t)R2 * zs;
        }
      }
    }
    // one buffer: ex is free again for the next slot's first stage only after
    // this barrier.  Two buffers: the next slot's first stage writes ex, which
    // every thread finished reading before the barrier above, and its middle
    // stage writes ex2 only after the next first-stage barrier, which no thread
    // passes before finishing this stage.
    if constexpr (!DB) __syncthreads();
    if (next >= nb) break;
    b = next;
  }
}
