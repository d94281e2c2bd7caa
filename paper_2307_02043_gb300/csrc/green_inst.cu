// Instantiation of the Green's-apply passes for one transform length P.
// Compiled once per supported P with -DMQ_P=<P>.  Each entry point runs the
// passes along an axis whose transform length is P: the x passes (1 and 5)
// when Px = P, the y passes (2 and 4) when Py = P, the z pass (3) when Pz = P.
#include <algorithm>

#include "functors.cuh"
#include "green_fused.cuh"
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

Geo geo(const GreenCall& c) { return Geo{c.nx, c.ny, c.nz}; }

template <int RV, int KIND>
cudaError_t launch1(const GreenCall& c, cudaStream_t s) {
  using RS = RowShape<P, RV>;
  Pro<KIND> pro;
  pro.a = c.pa;
  pro.g = geo(c);
  if constexpr (KIND == PRO_BICG_P || KIND == PRO_BICG_S) pro.st = c.st;
  auto kern = k_pass1<P, RV, Pro<KIND>>;
  cudaError_t e = set_smem(kern, RS::SMEM);
  if (e != cudaSuccess) return e;
  // a plane input needs only the rows of its plane (z = nz - 1)
  const int line0 = c.plane ? (c.nz - 1) * c.ny : 0, nlines = c.plane ? c.ny : c.ny * c.nz;
  dim3 grid(ceil_div(nlines, RS::LPB), c.nb);
  kern<<<grid, RS::THREADS, RS::SMEM, s>>>(pro, c.T1, c.ny, c.ny * c.nz, c.twx, c.st, c.part_pro, line0, nlines);
  return cudaGetLastError();
}

template <int RV, int KIND>
cudaError_t launch5(const GreenCall& c, cudaStream_t s) {
  using RS = RowShape<P, RV>;
  Epi<KIND> epi;
  epi.a = c.ea;
  epi.g = geo(c);
  auto kern = k_pass5<P, RV, Epi<KIND>>;
  cudaError_t e = set_smem(kern, RS::SMEM);
  if (e != cudaSuccess) return e;
  const int line0 = c.outplane ? (c.nz - 1) * c.ny : 0, nlines = c.outplane ? c.ny : c.ny * c.nz;
  dim3 grid(ceil_div(nlines, RS::LPB), c.nb);
  kern<<<grid, RS::THREADS, RS::SMEM, s>>>(epi, c.T1, c.ny, c.ny * c.nz, c.twx, c.st, c.part_epi, line0, nlines);
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
  const int px = 2 * c.nx;   // the last column tile may be ragged (kx >= Px masked)
  auto kern = px == P ? k_pass_y<P, CV, INV, true> : k_pass_y<P, CV, INV, false>;
  cudaError_t e = set_smem(kern, CS::SMEM);
  if (e != cudaSuccess) return e;
  // forward y pass of a plane input, inverse y pass of a plane output: that plane only
  const bool plane = INV ? c.outplane : c.plane;
  dim3 grid(ceil_div(px, CS::C), plane ? 1 : c.nz, c.nb);
  kern<<<grid, CS::THREADS, CS::SMEM, s>>>(in, out, c.nz, px, c.twy, c.st, plane ? c.nz - 1 : 0);
  return cudaGetLastError();
}

// one CTA per (kx tile, ky) column set; the batch is looped inside (one TMA tile buffer)
template <int CV, bool DB, bool CONJ, int IO = IO_FULL>
cudaError_t pass3(const GreenCall& c, cudaStream_t s) {
  using CS = ColShape<P, CV>;
  const CUtensorMap* tm = static_cast<const CUtensorMap*>(c.tmap);
  if (tm == nullptr || c.err == nullptr) return cudaErrorInvalidValue;
  const int px = 2 * c.nx, py = 2 * c.ny;   // the last column tile may be ragged (kx >= Px masked)
  auto kern = (px == P && py == P) ? k_pass3<P, CV, DB, CONJ, IO, true> : k_pass3<P, CV, DB, CONJ, IO, false>;
  const int smem = (int)Pass3Smem<P, CV, DB, IO>::bytes(c.nz);
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(px, CS::C), py);
  kern<<<grid, CS::THREADS, smem, s>>>(*tm, c.T2, c.khat, c.nx, c.ny, c.nb, c.twz, c.st, c.err);
  return cudaGetLastError();
}

// Fused x/y passes: persistent pairs of CTAs over the (slot, z-plane) tasks,
// as many pairs as fit on the device at once.
template <class K>
int fused_pairs(K kernel, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(FusedShape<P>::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)kernel, &cfg) != cudaSuccess) return 0;
  return n;
}

template <int KIND>
cudaError_t launch12(const GreenCall& c, cudaStream_t s) {
  using FS = FusedShape<P>;
  Pro<KIND> pro;
  pro.a = c.pa;
  pro.g = geo(c);
  if constexpr (KIND == PRO_BICG_P || KIND == PRO_BICG_S) pro.st = c.st;
  auto kern = k_pass12<P, Pro<KIND>>;
  static int pairs = 0;   // per instantiation: the device's co-resident pairs
  if (pairs == 0) {
    cudaError_t e = set_smem(kern, (int)FS::SMEM);
    if (e != cudaSuccess) return e;
    pairs = fused_pairs(kern, FS::SMEM);
    if (pairs <= 0) return cudaErrorLaunchOutOfResources;
  }
  const int n = std::min(pairs, c.nb * c.nz);
  const int nctas = ceil_div(c.ny * c.nz, RowShape<P, 0>::LPB);   // pass 1's partial layout
  kern<<<2 * n, FS::THREADS, FS::SMEM, s>>>(pro, c.T2, c.nz, c.nb, c.twx, c.st, c.part_pro, nctas);
  return cudaGetLastError();
}

template <int KIND>
cudaError_t launch45(const GreenCall& c, cudaStream_t s) {
  using FS = FusedShape<P>;
  Epi<KIND> epi;
  epi.a = c.ea;
  epi.g = geo(c);
  auto kern = k_pass45<P, Epi<KIND>>;
  static int pairs = 0;
  if (pairs == 0) {
    cudaError_t e = set_smem(kern, (int)FS::SMEM);
    if (e != cudaSuccess) return e;
    pairs = fused_pairs(kern, FS::SMEM);
    if (pairs <= 0) return cudaErrorLaunchOutOfResources;
  }
  const int n = std::min(pairs, c.nb * c.nz);
  const int nctas = ceil_div(c.ny * c.nz, RowShape<P, 0>::LPB);   // pass 5's partial layout
  kern<<<2 * n, FS::THREADS, FS::SMEM, s>>>(epi, c.T2, c.nz, c.nb, c.twx, c.st, c.part_epi, nctas);
  return cudaGetLastError();
}

cudaError_t fused(const GreenCall& c, bool inv, cudaStream_t s) {
  if constexpr (FusedShape<P>::OK && (P == 128 || P == 256)) {
    if (!inv) {
      switch (c.pro) {
        case PRO_PLAIN: return launch12<PRO_PLAIN>(c, s);
        case PRO_CONTRAST: return launch12<PRO_CONTRAST>(c, s);
        case PRO_BORN: return launch12<PRO_BORN>(c, s);
        case PRO_BICG_P: return launch12<PRO_BICG_P>(c, s);
        case PRO_BICG_S: return launch12<PRO_BICG_S>(c, s);
        case PRO_LIFT: return launch12<PRO_LIFT>(c, s);
        default: return cudaErrorInvalidValue;
      }
    }
    switch (c.epi) {
      case EPI_PLAIN: return launch45<EPI_PLAIN>(c, s);
      case EPI_V: return launch45<EPI_V>(c, s);
      case EPI_T: return launch45<EPI_T>(c, s);
      case EPI_INIT: return launch45<EPI_INIT>(c, s);
      case EPI_INIT_WARM: return launch45<EPI_INIT_WARM>(c, s);
      case EPI_DETECT: return launch45<EPI_DETECT>(c, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    (void)c;
    (void)inv;
    (void)s;
    return cudaErrorNotSupported;
  }
}

template <int ZV, bool DB>
cudaError_t pass3_io(const GreenCall& c, cudaStream_t s) {
  if (c.plane) {   // the plane input serves the adjoint lift only
    if (!c.adjoint || c.outplane) return cudaErrorInvalidValue;
    return pass3<ZV, DB, true, IO_IN>(c, s);
  }
  if (c.outplane) {   // the plane output serves the first-Born data only
    if (c.adjoint) return cudaErrorInvalidValue;
    return pass3<ZV, DB, false, IO_OUT>(c, s);
  }
  return c.adjoint ? pass3<ZV, DB, true>(c, s) : pass3<ZV, DB, false>(c, s);
}
}  // namespace

void MQ_CAT(green_shape_P, MQ_P)(int tile, int* shape, size_t* smem_row, size_t* smem_col, size_t* smem_z) {
  shape[0] = (tile & 1) ? RowShape<P, 1>::LPB : RowShape<P, 0>::LPB;
  shape[1] = (tile & 1) ? RowShape<P, 1>::T : RowShape<P, 0>::T;
  shape[2] = (tile & 2) ? ColShape<P, 1>::C : ColShape<P, 0>::C;
  shape[3] = (tile & 2) ? ColShape<P, 1>::T : ColShape<P, 0>::T;
  shape[4] = (tile & 4) ? ColShape<P, 1>::C : ColShape<P, 0>::C;
  shape[5] = (tile & 4) ? ColShape<P, 1>::T : ColShape<P, 0>::T;
  switch ((tile >> 2) & 3) {   // the z pass at this length: nz = P/2
    case 0: *smem_z = Pass3Smem<P, 0, false>::bytes(P / 2); break;
    case 1: *smem_z = Pass3Smem<P, 1, false>::bytes(P / 2); break;
    case 2: *smem_z = Pass3Smem<P, 0, true>::bytes(P / 2); break;
    default: *smem_z = Pass3Smem<P, 1, true>::bytes(P / 2); break;
  }
  *smem_col = (tile & 2) ? ColShape<P, 1>::SMEM : ColShape<P, 0>::SMEM;
  *smem_row = (tile & 1) ? RowShape<P, 1>::SMEM : RowShape<P, 0>::SMEM;
}

cudaError_t MQ_CAT(green_pass1_P, MQ_P)(const GreenCall& c, cudaStream_t s) {
  if (2 * c.nx != P) return cudaErrorInvalidValue;
  return (c.tile & 1) ? pass1<1>(c, s) : pass1<0>(c, s);
}

cudaError_t MQ_CAT(green_pass5_P, MQ_P)(const GreenCall& c, cudaStream_t s) {
  if (2 * c.nx != P) return cudaErrorInvalidValue;
  return (c.tile & 1) ? pass5<1>(c, s) : pass5<0>(c, s);
}

cudaError_t MQ_CAT(green_passy_P, MQ_P)(const GreenCall& c, bool inv, cudaStream_t s) {
  if (2 * c.ny != P) return cudaErrorInvalidValue;
  if (inv) return (c.tile & 2) ? pass_y<1, true>(c, c.T2, c.T1, s) : pass_y<0, true>(c, c.T2, c.T1, s);
  return (c.tile & 2) ? pass_y<1, false>(c, c.T1, c.T2, s) : pass_y<0, false>(c, c.T1, c.T2, s);
}

cudaError_t MQ_CAT(green_pass3_P, MQ_P)(const GreenCall& c, cudaStream_t s) {
  if (2 * c.nz != P) return cudaErrorInvalidValue;
  switch ((c.tile >> 2) & 3) {   // bit 2: z-pass shape, bit 3: its two exchange buffers
    case 0: return pass3_io<0, false>(c, s);
    case 1: return pass3_io<1, false>(c, s);
    case 2: return pass3_io<0, true>(c, s);
    default: return pass3_io<1, true>(c, s);
  }
}

// Fused x/y passes of a square plane of edge P/2 (tile bit 4; P = 128, 256).
cudaError_t MQ_CAT(green_fused_P, MQ_P)(const GreenCall& c, bool inv, cudaStream_t s) {
  if (2 * c.nx != P || 2 * c.ny != P) return cudaErrorInvalidValue;
  return fused(c, inv, s);
}

size_t MQ_CAT(green_fused_smem_P, MQ_P)() {
  if constexpr (FusedShape<P>::OK && (P == 128 || P == 256)) return FusedShape<P>::SMEM;
  return 0;
}
