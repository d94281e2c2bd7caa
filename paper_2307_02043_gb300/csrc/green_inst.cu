// Instantiation of the Green's-apply passes for one transform length P.
// Compiled once per supported P with -DMQ_P=<P>.
#include "functors.cuh"
#include "internal.h"

#ifndef MQ_P
#error "compile with -DMQ_P=<transform length>"
#endif

#define MQ_CAT2(a, b) a##b
#define MQ_CAT(a, b) MQ_CAT2(a, b)

namespace {
constexpr int P = MQ_P;

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int RV, int KIND>
cudaError_t launch1(const GreenCall& c, cudaStream_t s) {
  using RS = RowShape<P, RV>;
  Pro<KIND> pro;
  pro.a = c.pa;
  pro.g = Geo{c.n};
  if constexpr (KIND == PRO_BICG_P || KIND == PRO_BICG_S) pro.st = c.st;
  auto kern = k_pass1<P, RV, Pro<KIND>>;
  cudaError_t e = set_smem(kern, RS::SMEM);
  if (e != cudaSuccess) return e;
  // a plane input needs only the rows of its plane (z = n - 1)
  const int line0 = c.plane ? (c.n - 1) * c.n : 0, nlines = c.plane ? c.n : c.n * c.n;
  dim3 grid(ceil_div(nlines, RS::LPB), c.nb);
  kern<<<grid, RS::THREADS, RS::SMEM, s>>>(pro, c.T1, c.n, c.tw, c.st, c.part_pro, line0, nlines);
  return cudaGetLastError();
}

template <int RV, int KIND>
cudaError_t launch5(const GreenCall& c, cudaStream_t s) {
  using RS = RowShape<P, RV>;
  Epi<KIND> epi;
  epi.a = c.ea;
  epi.g = Geo{c.n};
  auto kern = k_pass5<P, RV, Epi<KIND>>;
  cudaError_t e = set_smem(kern, RS::SMEM);
  if (e != cudaSuccess) return e;
  const int line0 = c.outplane ? (c.n - 1) * c.n : 0, nlines = c.outplane ? c.n : c.n * c.n;
  dim3 grid(ceil_div(nlines, RS::LPB), c.nb);
  kern<<<grid, RS::THREADS, RS::SMEM, s>>>(epi, c.T1, c.n, c.tw, c.st, c.part_epi, line0, nlines);
  return cudaGetLastError();
}

template <int RV>
cudaError_t pass1(const GreenCall& c, cudaStream_t s) {
  switch (c.pro) {
    case PRO_PLAIN: return launch1<RV, PRO_PLAIN>(c, s);
    case PRO_CONTRAST: return launch1<RV, PRO_CONTRAST>(c, s);
    case PRO_BORN: return launch1<RV, PRO_BORN>(c, s);
    case PRO_BICG_P: return launch1<RV, PRO_BICG_P>(c, s);
    case PRO_BICG_S: return launch1<RV, PRO_BICG_S>(c, s);
    case PRO_LIFT: return launch1<RV, PRO_LIFT>(c, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int RV>
cudaError_t pass5(const GreenCall& c, cudaStream_t s) {
  switch (c.epi) {
    case EPI_PLAIN: return launch5<RV, EPI_PLAIN>(c, s);
    case EPI_V: return launch5<RV, EPI_V>(c, s);
    case EPI_T: return launch5<RV, EPI_T>(c, s);
    case EPI_INIT: return launch5<RV, EPI_INIT>(c, s);
    case EPI_INIT_WARM: return launch5<RV, EPI_INIT_WARM>(c, s);
    case EPI_DETECT: return launch5<RV, EPI_DETECT>(c, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int CV, bool INV>
cudaError_t pass_y(const GreenCall& c, const float2* in, float2* out, cudaStream_t s) {
  using CS = ColShape<P, CV>;
  auto kern = k_pass_y<P, CV, INV>;
  cudaError_t e = set_smem(kern, CS::SMEM);
  if (e != cudaSuccess) return e;
  // forward y pass of a plane input, inverse y pass of a plane output: that plane only
  const bool plane = INV ? c.outplane : c.plane;
  dim3 grid(P / CS::C, plane ? 1 : c.n, c.nb);
  kern<<<grid, CS::THREADS, CS::SMEM, s>>>(in, out, c.n, c.tw, c.st, plane ? c.n - 1 : 0);
  return cudaGetLastError();
}

// one CTA per (kx tile, ky) column set; the batch is looped inside (one TMA tile buffer)
template <int CV, bool DB, bool CONJ, int IO = IO_FULL>
cudaError_t pass3(const GreenCall& c, cudaStream_t s) {
  using CS = ColShape<P, CV>;
  const CUtensorMap* tm = static_cast<const CUtensorMap*>(c.tmap);
  if (tm == nullptr || c.err == nullptr) return cudaErrorInvalidValue;
  auto kern = k_pass3<P, CV, DB, CONJ, IO>;
  const int smem = (int)Pass3Smem<P, CV, DB, IO>::bytes(c.n);
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(P / CS::C, P);
  kern<<<grid, CS::THREADS, smem, s>>>(*tm, c.T2, c.khat, c.n, c.nb, c.tw, c.st, c.err);
  return cudaGetLastError();
}

template <int YV, int ZV, bool DB>
cudaError_t columns(const GreenCall& c, cudaStream_t s, unsigned rec_flags) {
  cudaError_t e;
  if ((e = pass_y<YV, false>(c, c.T1, c.T2, s)) != cudaSuccess) return e;
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[2], s, rec_flags)) != cudaSuccess) return e;
  if (c.plane) {   // the plane input serves the adjoint lift only
    if (!c.adjoint || c.outplane) return cudaErrorInvalidValue;
    e = pass3<ZV, DB, true, IO_IN>(c, s);
  } else if (c.outplane) {   // the plane output serves the first-Born data only
    if (c.adjoint) return cudaErrorInvalidValue;
    e = pass3<ZV, DB, false, IO_OUT>(c, s);
  } else {
    e = c.adjoint ? pass3<ZV, DB, true>(c, s) : pass3<ZV, DB, false>(c, s);
  }
  if (e != cudaSuccess) return e;
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[3], s, rec_flags)) != cudaSuccess) return e;
  return pass_y<YV, true>(c, c.T2, c.T1, s);
}
}  // namespace

void MQ_CAT(green_shape_P, MQ_P)(int tile, int n, int* shape, size_t* smem) {
  shape[0] = (tile & 1) ? RowShape<P, 1>::LPB : RowShape<P, 0>::LPB;
  shape[1] = (tile & 1) ? RowShape<P, 1>::T : RowShape<P, 0>::T;
  shape[2] = (tile & 2) ? ColShape<P, 1>::C : ColShape<P, 0>::C;
  shape[3] = (tile & 2) ? ColShape<P, 1>::T : ColShape<P, 0>::T;
  shape[4] = (tile & 4) ? ColShape<P, 1>::C : ColShape<P, 0>::C;
  shape[5] = (tile & 4) ? ColShape<P, 1>::T : ColShape<P, 0>::T;
  size_t m = 0;   // the largest dynamic shared memory of the tile's five passes
  switch ((tile >> 2) & 3) {
    case 0: m = Pass3Smem<P, 0, false>::bytes(n); break;
    case 1: m = Pass3Smem<P, 1, false>::bytes(n); break;
    case 2: m = Pass3Smem<P, 0, true>::bytes(n); break;
    default: m = Pass3Smem<P, 1, true>::bytes(n); break;
  }
  const size_t ys = (tile & 2) ? ColShape<P, 1>::SMEM : ColShape<P, 0>::SMEM;
  const size_t rs = (tile & 1) ? RowShape<P, 1>::SMEM : RowShape<P, 0>::SMEM;
  *smem = m > ys ? (m > rs ? m : rs) : (ys > rs ? ys : rs);
}

cudaError_t MQ_CAT(green_launch_P, MQ_P)(const GreenCall& c, cudaStream_t s) {
  if (2 * c.n != P || c.tile < 0 || c.tile >= MQ_TILES) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  // inside a stream capture the records must be external to become event-record
  // nodes of the graph; outside one they are plain records
  unsigned rec_flags = cudaEventRecordDefault;
  if (c.ev) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
  }
  const bool row_alt = (c.tile & 1) != 0;
  const int col = (c.tile >> 1) & 7;   // bit 1: y-pass shape, bit 2: z-pass shape, bit 3: its two buffers
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[0], s, rec_flags)) != cudaSuccess) return e;
  if ((e = row_alt ? pass1<1>(c, s) : pass1<0>(c, s)) != cudaSuccess) return e;
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[1], s, rec_flags)) != cudaSuccess) return e;
  switch (col) {
    case 0: e = columns<0, 0, false>(c, s, rec_flags); break;
    case 1: e = columns<1, 0, false>(c, s, rec_flags); break;
    case 2: e = columns<0, 1, false>(c, s, rec_flags); break;
    case 3: e = columns<1, 1, false>(c, s, rec_flags); break;
    case 4: e = columns<0, 0, true>(c, s, rec_flags); break;
    case 5: e = columns<1, 0, true>(c, s, rec_flags); break;
    case 6: e = columns<0, 1, true>(c, s, rec_flags); break;
    default: e = columns<1, 1, true>(c, s, rec_flags); break;
  }
  if (e != cudaSuccess) return e;
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[4], s, rec_flags)) != cudaSuccess) return e;
  if ((e = row_alt ? pass5<1>(c, s) : pass5<0>(c, s)) != cudaSuccess) return e;
  if (c.ev) e = cudaEventRecordWithFlags(c.ev[5], s, rec_flags);
  if (c.launches) *c.launches += 5;
  return e;
}
