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
using RS = RowShape<P>;
using CS = ColShape<P>;

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int KIND>
cudaError_t launch1(const GreenCall& c, cudaStream_t s) {
  Pro<KIND> pro;
  pro.a = c.pa;
  pro.g = Geo{c.n};
  if constexpr (KIND == PRO_BICG_P || KIND == PRO_BICG_S) pro.st = c.st;
  auto kern = k_pass1<P, Pro<KIND>>;
  cudaError_t e = set_smem(kern, RS::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(c.n * c.n, RS::LPB), c.nb);
  kern<<<grid, RS::THREADS, RS::SMEM, s>>>(pro, c.T1, c.n, c.tw, c.st, c.part_pro);
  return cudaGetLastError();
}

template <int KIND>
cudaError_t launch5(const GreenCall& c, cudaStream_t s) {
  Epi<KIND> epi;
  epi.a = c.ea;
  epi.g = Geo{c.n};
  auto kern = k_pass5<P, Epi<KIND>>;
  cudaError_t e = set_smem(kern, RS::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(c.n * c.n, RS::LPB), c.nb);
  kern<<<grid, RS::THREADS, RS::SMEM, s>>>(epi, c.T1, c.n, c.tw, c.st, c.part_epi);
  return cudaGetLastError();
}
}  // namespace

int MQ_CAT(green_row_ctas_P, MQ_P)(int n) { return ceil_div(n * n, RS::LPB); }

cudaError_t MQ_CAT(green_launch_P, MQ_P)(const GreenCall& c, cudaStream_t s) {
  if (2 * c.n != P) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  // inside a stream capture the records must be external to become event-record
  // nodes of the graph; outside one they are plain records
  unsigned rec_flags = cudaEventRecordDefault;
  if (c.ev) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
  }
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[0], s, rec_flags)) != cudaSuccess) return e;
  switch (c.pro) {
    case PRO_PLAIN: e = launch1<PRO_PLAIN>(c, s); break;
    case PRO_CONTRAST: e = launch1<PRO_CONTRAST>(c, s); break;
    case PRO_BORN: e = launch1<PRO_BORN>(c, s); break;
    case PRO_BICG_P: e = launch1<PRO_BICG_P>(c, s); break;
    case PRO_BICG_S: e = launch1<PRO_BICG_S>(c, s); break;
    case PRO_LIFT: e = launch1<PRO_LIFT>(c, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[1], s, rec_flags)) != cudaSuccess) return e;
  {
    auto kern = k_pass_y<P, false>;
    if ((e = set_smem(kern, CS::SMEM)) != cudaSuccess) return e;
    dim3 grid(P / CS::C, c.n, c.nb);
    kern<<<grid, CS::THREADS, CS::SMEM, s>>>(c.T1, c.T2, c.n, c.tw, c.st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[2], s, rec_flags)) != cudaSuccess) return e;
  {
    // one CTA per (kx tile, ky) column set; the batch is looped inside (one TMA tile buffer)
    dim3 grid(P / CS::C, P);
    const int smem = (int)Pass3Smem<P>::bytes(c.n);
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(c.tmap);
    if (tm == nullptr || c.err == nullptr) return cudaErrorInvalidValue;
    if (c.adjoint) {
      auto kern = k_pass3<P, true>;
      if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
      kern<<<grid, CS::THREADS, smem, s>>>(*tm, c.T2, c.khat, c.n, c.nb, c.tw, c.st, c.err);
    } else {
      auto kern = k_pass3<P, false>;
      if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
      kern<<<grid, CS::THREADS, smem, s>>>(*tm, c.T2, c.khat, c.n, c.nb, c.tw, c.st, c.err);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[3], s, rec_flags)) != cudaSuccess) return e;
  {
    auto kern = k_pass_y<P, true>;
    if ((e = set_smem(kern, CS::SMEM)) != cudaSuccess) return e;
    dim3 grid(P / CS::C, c.n, c.nb);
    kern<<<grid, CS::THREADS, CS::SMEM, s>>>(c.T2, c.T1, c.n, c.tw, c.st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c.ev && (e = cudaEventRecordWithFlags(c.ev[4], s, rec_flags)) != cudaSuccess) return e;
  switch (c.epi) {
    case EPI_PLAIN: e = launch5<EPI_PLAIN>(c, s); break;
    case EPI_V: e = launch5<EPI_V>(c, s); break;
    case EPI_T: e = launch5<EPI_T>(c, s); break;
    case EPI_INIT: e = launch5<EPI_INIT>(c, s); break;
    case EPI_INIT_WARM: e = launch5<EPI_INIT_WARM>(c, s); break;
    case EPI_DETECT: e = launch5<EPI_DETECT>(c, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (c.ev && e == cudaSuccess) e = cudaEventRecordWithFlags(c.ev[5], s, rec_flags);
  if (c.launches) *c.launches += 5;
  return e;
}
