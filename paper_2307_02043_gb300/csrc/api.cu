// C ABI of libmqnpm: handle life cycle, data upload, and the outer loop of the
// mini-batch quasi-Newton proximal method (Algorithm 4.1) with the SR1 metric
// estimate (Algorithm 4.2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mqnpm.h"

int set_error(mqnpm_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int set_cuda_error(mqnpm_handle* h, cudaError_t e, const char* where) {
  if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return MQNPM_ERR_CUDA;
}

namespace {

#define CK(call)                                                \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return set_cuda_error(h, e_, #call); \
  } while (0)

template <class T>
int dalloc(mqnpm_handle* h, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  const size_t G = h->guard;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes + 2 * G);
  if (e != cudaSuccess) return set_cuda_error(h, e, "cudaMalloc");
  h->allocations.push_back(q);
  h->bytes += bytes + 2 * G;
  unsigned char* raw = static_cast<unsigned char*>(q);
  if (G > 0) {   // bands before and after the buffer
    if ((e = cudaMemset(raw, 0xA5, G)) != cudaSuccess || (e = cudaMemset(raw + G + bytes, 0xA5, G)) != cudaSuccess)
      return set_cuda_error(h, e, "guard bands");
    h->guards.push_back({raw, G});
    h->guards.push_back({raw + G + bytes, G});
  }
  *p = reinterpret_cast<T*>(raw + G);
  return MQNPM_OK;
}

__global__ void k_check_guards(unsigned char* const* bands, size_t len, int* bad) {
  const unsigned char* b = bands[blockIdx.x];
  int wrong = 0;
  for (size_t i = threadIdx.x; i < len; i += blockDim.x) wrong |= (b[i] != 0xA5);
  if (__syncthreads_or(wrong) && threadIdx.x == 0) bad[blockIdx.x] = 1;
}

struct Sizes {
  size_t total = 0;
};

__global__ void k_axpby(const float* x, const float* g, float a, float* out, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    out[i] = fmaf(a, g[i], x[i]);
}

// u = ((g - gbar) - tau (x - xbar)) * inv  (Algorithm 4.2, after the damping loop)
__global__ void k_sr1_u(const float* x, const float* xbar, const float* g, const float* gbar, float tau, float inv,
                        float* u, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    u[i] = ((g[i] - gbar[i]) - tau * (x[i] - xbar[i])) * inv;
}

bool finite_all(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

void profile_clear(mqnpm_handle* h) {
  for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
  h->prof.ev.clear();
  h->prof.nb.clear();
  h->prof.used = 0;
  h->prof.on = false;
  for (double& v : h->prof.acc_ms) v = 0.0;
  h->prof.acc_slots = 0;
  h->prof.acc_calls = 0;
}

}  // namespace

cudaEvent_t* profile_slot(mqnpm_handle* h, int nb) {
  Profiler& p = h->prof;
  if (!p.on || (size_t)(p.used + 1) * 6 > p.ev.size()) return nullptr;
  p.nb.push_back(nb);
  return &p.ev[6 * (size_t)p.used++];
}

extern "C" {

int mqnpm_prox_trace(mqnpm_handle* h, long long* out, int cap, int* count) {
  if (!h || !out || cap < 1 || !count) return MQNPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  const int m = std::min(cap, h->wp.trace_cap);
  CK(cudaMemcpyAsync(out, h->wp.trace, 2 * (size_t)m * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *count = (int)std::min<long long>(out[0] + 1, m - 1);
  return MQNPM_OK;
}

int mqnpm_profile_begin(mqnpm_handle* h, int max_calls) {
  if (!h || max_calls < 1) return MQNPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  profile_clear(h);
  h->prof.ev.resize(6 * (size_t)max_calls);
  for (auto& e : h->prof.ev) CK(cudaEventCreate(&e));
  h->prof.on = true;
  return MQNPM_OK;
}

int mqnpm_profile_end(mqnpm_handle* h, double* pass_ms, long long* slot_launches, int* calls) {
  if (!h || !pass_ms) return MQNPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  for (int p = 0; p < 5; ++p) pass_ms[p] = h->prof.acc_ms[p];
  long long slots = h->prof.acc_slots;
  for (int g = 0; g < h->prof.used; ++g) {
    for (int p = 0; p < 5; ++p) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->prof.ev[6 * (size_t)g + p], h->prof.ev[6 * (size_t)g + p + 1]));
      pass_ms[p] += ms;
    }
    slots += h->prof.nb[g];
  }
  if (slot_launches) *slot_launches = slots;
  if (calls) *calls = h->prof.used + h->prof.acc_calls;
  profile_clear(h);
  return MQNPM_OK;
}

const char* mqnpm_last_error(const mqnpm_handle* h) { return h ? h->err.c_str() : "null handle"; }

long long mqnpm_launch_count(const mqnpm_handle* h) { return h ? h->launches : 0; }

int mqnpm_check_guards(mqnpm_handle* h, int* corrupted) {
  if (!h || !corrupted) return MQNPM_ERR_INVALID_ARG;
  *corrupted = 0;
  if (h->guards.empty()) return MQNPM_OK;
  CK(cudaSetDevice(h->device));
  const int nb = (int)h->guards.size();
  CK(cudaMemsetAsync(h->guard_bad, 0, nb * sizeof(int), h->stream));
  k_check_guards<<<nb, 256, 0, h->stream>>>(h->guard_ptr, h->guard, h->guard_bad);
  CK(cudaGetLastError());
  std::vector<int> bad(nb);
  CK(cudaMemcpyAsync(bad.data(), h->guard_bad, nb * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int v : bad) *corrupted += v;
  return MQNPM_OK;
}

int mqnpm_debug_poke_guard(mqnpm_handle* h, int band) {
  if (!h || band < 0 || band >= (int)h->guards.size()) return MQNPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  CK(cudaMemsetAsync(h->guards[band].first + h->guards[band].second / 2, 0x00, 1, h->stream));
  return MQNPM_OK;
}

int mqnpm_tile_info(const mqnpm_handle* h, int* tile, int* shape, double* ms) {
  if (!h || !tile || !shape) return MQNPM_ERR_INVALID_ARG;
  *tile = h->tile;
  green_shape(h->nx, h->ny, h->nz, h->tile, shape);
  if (ms)
    for (int i = 0; i < MQ_TILES; ++i) ms[i] = h->tune_ms[i];
  return MQNPM_OK;
}

size_t mqnpm_workspace_bytes(const mqnpm_handle* h) { return h ? h->bytes : 0; }

int mqnpm_set_wait_limit(mqnpm_handle* h, long long cycles) {
  if (!h || cycles < 0) return set_error(h, MQNPM_ERR_INVALID_ARG, "set_wait_limit: negative limit");
  h->barrier_limit = cycles > 0 ? cycles : 4000000000LL;
  return MQNPM_OK;
}

int mqnpm_set_stream(mqnpm_handle* h, void* stream) {
  if (!h) return MQNPM_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return MQNPM_OK;
}

void mqnpm_destroy(mqnpm_handle* h) {
  if (!h) return;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  profile_clear(h);
  for (KrylovGraph& g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.ev)
      if (e) cudaEventDestroy(e);
  }
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (cudaEvent_t ev : h->step_ev)
    if (ev) cudaEventDestroy(ev);
  for (void* p : h->allocations) cudaFree(p);
  if (h->w.h_nactive) cudaFreeHost(h->w.h_nactive);
  if (h->w.h_loops) cudaFreeHost(h->w.h_loops);
  if (h->w.h_illum) cudaFreeHost(h->w.h_illum);
  if (h->w.h_xslot) cudaFreeHost(h->w.h_xslot);
  if (h->w.h_fwarm) cudaFreeHost(h->w.h_fwarm);
  if (h->w.h_fstore) cudaFreeHost(h->w.h_fstore);
  if (h->w.h_segs) cudaFreeHost(h->w.h_segs);
  if (h->w.h_scal) cudaFreeHost(h->w.h_scal);
  cudaSetDevice(dev);
  delete h;
}

}  // extern "C"

// mqnpm_create with an optional device copy source for the Green's spectrum
// (a group's engine takes its members' spectrum instead of building it again).
int create_handle(const mqnpm_config* cfg, const float2* khat_src, mqnpm_handle** out) {
  if (!out) return MQNPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return MQNPM_ERR_INVALID_ARG;
  mqnpm_handle* h = new mqnpm_handle();
  auto fail = [&](int code) {
    mqnpm_destroy(h);
    return code;
  };
  // ---- validation
  if (cfg->nx < 4 || cfg->ny < 4 || cfg->nz < 4 || cfg->L < 1 || cfg->S < 1 || cfg->S > MQNPM_MAX_S || cfg->S > cfg->L || !cfg->kdir ||
      !cfg->subset_of || !cfg->alpha || !(cfg->h > 0) || !(cfg->kb > 0) || cfg->max_batch < 1 ||
      cfg->max_batch > MQNPM_MAX_BATCH ||
      !(cfg->box_lo <= cfg->box_hi) || !(cfg->lambda >= 0) || !(cfg->step > 0) || cfg->dual_iters < 0 ||
      !(cfg->krylov_tol > 0) || cfg->krylov_maxit < 1 || (cfg->model != MQNPM_MODEL_LS && cfg->model != MQNPM_MODEL_BORN) ||
      (cfg->tv != MQNPM_TV_ISO && cfg->tv != MQNPM_TV_ANISO) || (cfg->strategy != 1 && cfg->strategy != 2) ||
      !(cfg->gamma > 0 && cfg->gamma <= 1.0) || cfg->tile < -1 || cfg->tile >= MQ_TILES ||
      !(cfg->det_na >= 0.0 && std::isfinite(cfg->det_na)) || !std::isfinite(cfg->det_distance) ||
      cfg->barrier_wait_cycles < 0 ||
      (cfg->green_kernel != MQNPM_KERNEL_SAMPLED && cfg->green_kernel != MQNPM_KERNEL_TRUNCATED) ||
      (cfg->adjoint_start != 0 && cfg->adjoint_start != 1) || (cfg->forward_start != 0 && cfg->forward_start != 1)) {
    fprintf(stderr, "mqnpm_create: invalid configuration\n");
    delete h;
    return MQNPM_ERR_INVALID_ARG;
  }
  if (!green_supported(cfg->nx) || !green_supported(cfg->ny) || !green_supported(cfg->nz)) {
    delete h;
    return MQNPM_ERR_UNSUPPORTED;
  }
  if (cfg->green_hat) {
    const size_t cnt = 2 * ((size_t)cfg->nx + 1) * ((size_t)cfg->ny + 1) * ((size_t)cfg->nz + 1);
    for (size_t i = 0; i < cnt; ++i)
      if (!std::isfinite(cfg->green_hat[i])) {
        fprintf(stderr, "mqnpm_create: green_hat holds a non-finite value\n");
        delete h;
        return MQNPM_ERR_INVALID_ARG;
      }
  }
  h->nx = cfg->nx;
  h->ny = cfg->ny;
  h->nz = cfg->nz;
  h->N = (size_t)cfg->nx * cfg->ny * cfg->nz;
  h->M = cfg->nx * cfg->ny;
  h->model = cfg->model;
  h->L = cfg->L;
  h->S = cfg->S;
  h->tv = cfg->tv;
  h->strategy = cfg->strategy;
  h->h = cfg->h;
  h->kb = cfg->kb;
  h->lambda = cfg->lambda;
  h->lo = cfg->box_lo;
  h->hi = cfg->box_hi;
  h->a = cfg->step;
  h->gamma = cfg->gamma;
  h->delta1 = cfg->delta1 > 0 ? cfg->delta1 : 1e-8;
  h->delta2 = cfg->delta2 > 0 ? cfg->delta2 : 1e-12;
  h->krylov_tol = cfg->krylov_tol;
  h->krylov_maxit = cfg->krylov_maxit;
  h->dual_iters = cfg->dual_iters;
  h->newton_tol = cfg->newton_tol > 0 ? cfg->newton_tol : 1e-6;
  h->newton_maxit = cfg->newton_maxit > 0 ? cfg->newton_maxit : 50;
  h->max_batch = cfg->max_batch;
  h->device = cfg->device;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  h->warm_start = cfg->warm_start != 0;
  h->adjoint_from_b = cfg->adjoint_start == 0;
  h->forward_refine_steps = cfg->forward_start == 0 ? 1 : 0;
  h->direct_launches = cfg->direct_launches != 0;
  h->budget = cfg->hbm_budget_bytes;
  h->guard = (cfg->guard_bytes + 255) / 256 * 256;
  if (cfg->barrier_wait_cycles > 0) h->barrier_limit = cfg->barrier_wait_cycles;
  h->green_kernel = cfg->green_kernel;
  h->kdir.assign(cfg->kdir, cfg->kdir + 3 * cfg->L);
  h->alpha.assign(cfg->alpha, cfg->alpha + cfg->S);
  h->subset_of.assign(cfg->subset_of, cfg->subset_of + cfg->L);
  if (cfg->strategy_draws && cfg->n_draws > 0) h->draws.assign(cfg->strategy_draws, cfg->strategy_draws + cfg->n_draws);
  h->subsets.assign(h->S, {});
  for (int l = 0; l < h->L; ++l) {
    const int s = h->subset_of[l];
    if (s < 0 || s >= h->S) { delete h; return MQNPM_ERR_INVALID_ARG; }
    h->subsets[s].push_back(l);
  }
  for (int s = 0; s < h->S; ++s) {
    if (h->subsets[s].empty() || !(h->alpha[s] > 0)) { delete h; return MQNPM_ERR_INVALID_ARG; }
  }
  double amax = *std::max_element(h->alpha.begin(), h->alpha.end());
  h->tau_max = cfg->tau_max > 0 ? cfg->tau_max : 1e3 * amax;
  for (int d : h->draws)
    if (d < 0 || d >= h->S) { delete h; return MQNPM_ERR_INVALID_ARG; }

  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) { set_cuda_error(h, e, "cudaSetDevice"); delete h; return MQNPM_ERR_CUDA; }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (nsm <= 0) nsm = 1;
  const size_t N = h->N, M = h->M, B = h->max_batch;
  const int nx = h->nx, ny = h->ny, nz = h->nz;
  const int Px = 2 * nx, Py = 2 * ny, Pz = 2 * nz;
  h->tile = cfg->tile;
  if (h->tile < 0) {   // autotuned below; start from the first tile that fits
    for (int t = 0; t < MQ_TILES && h->tile < 0; ++t)
      if (green_tile_fits(nx, ny, nz, t, h->device)) h->tile = t;
    if (h->tile < 0) {
      h->err = "no launch shape of the Green's passes fits the device's shared memory at this grid";
      delete h;
      return MQNPM_ERR_UNSUPPORTED;
    }
  }
  std::fill(h->tune_ms, h->tune_ms + MQ_TILES, -1.0);
  if (!green_tile_fits(nx, ny, nz, h->tile, h->device)) {
    char msg[160];
    snprintf(msg, sizeof msg, "tile %d does not run at the %d x %d x %d grid on this device (shared memory per block, "
             "or fused x/y passes without square 64 or 128 planes)", h->tile, nx, ny, nz);
    h->err = msg;
    *out = nullptr;
    delete h;
    return MQNPM_ERR_INVALID_ARG;
  }
  h->w.ctas_row = green_row_ctas_max(nx, ny, nz);   // partials sized for every tile variant
  h->w.ctas_vec = (int)std::min<long long>(ceil_div_ll((long long)N, 256LL * 8), 8LL * nsm);
  h->w.ctas_upd = (int)std::min<long long>(ceil_div_ll((long long)N, 256LL * 8), 4LL * nsm);
  if (h->w.ctas_vec < 1) h->w.ctas_vec = 1;
  if (h->w.ctas_upd < 1) h->w.ctas_upd = 1;
  h->wp.ctas_vec = h->w.ctas_vec;
  h->wp.nsm = nsm;
  const int wp_blocks = wprox_blocks_per_sm() * nsm;   // blocks of the cooperative prox kernel, at most

  // ---- budget (every device allocation of the handle)
  const size_t nkhat = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  const size_t ntab = (size_t)h->L * (nx + ny + nz);
  size_t need = 0;
  need += nkhat * 8 + (size_t)(Px + Py + Pz) * 8 + ntab * 8 + (size_t)h->L * M * 8;
  need += 8 * B * N * 8;                                   // u zs r rhat p v s t
  need += B * ((size_t)nz * ny * Px + (size_t)nz * Py * Px) * 8;   // T1, T2
  need += B * M * 8;                                       // rdet
  if (cfg->det_na > 0) need += 3 * B * M * 8 + M * 8 + (size_t)(nx + ny) * 8;   // remote detector
  need += B * (size_t)h->w.ctas_row * (1 + 3 + 1) * 8 + std::max(B * (size_t)h->w.ctas_upd, (size_t)h->w.ctas_vec) * 3 * 8;
  need += 8 * N * 4 + (size_t)(h->wp.ctas_vec * wprox_part_len() + 600) * 8 + wprox_part_count(wp_blocks) * 8;   // wprox
  need += (3 * (size_t)h->S + 2) * N * 4 + 3 * N * 4;                               // step state
  if (h->warm_start && h->model == MQNPM_MODEL_LS) need += (size_t)h->L * N * 8;     // stored fields
  if (h->budget > 0 && need > h->budget) {
    char msg[160];
    snprintf(msg, sizeof msg, "workspace of %zu bytes exceeds the budget of %zu bytes", need, h->budget);
    h->err = msg;
    *out = nullptr;
    delete h;
    return MQNPM_ERR_BUDGET;
  }

  // ---- allocations
  int rc = MQNPM_OK;
#define AL(ptr, cnt) \
  if ((rc = dalloc(h, &(ptr), (cnt))) != MQNPM_OK) return fail(rc)
  AL(h->khat, nkhat);
  AL(h->twx, (size_t)Px);
  AL(h->twy, (size_t)Py);
  AL(h->twz, (size_t)Pz);
  AL(h->tab, ntab);
  AL(h->ymeas, (size_t)h->L * M);
  Workspace& w = h->w;
  AL(w.u, B * N); AL(w.zs, B * N); AL(w.r, B * N); AL(w.rhat, B * N);
  AL(w.p, B * N); AL(w.v, B * N); AL(w.s, B * N); AL(w.t, B * N);
  AL(w.T1, B * (size_t)nz * ny * Px);
  AL(w.T2, B * (size_t)nz * Py * Px);
  AL(w.rdet, B * M);
  h->remote = cfg->det_na > 0;
  if (h->remote) {
    AL(w.dtmp1, B * M); AL(w.dtmp2, B * M); AL(w.rlift, B * M);
    AL(h->Hdet, M); AL(h->twn, (size_t)(nx + ny));
  }
  AL(w.part1, B * (size_t)w.ctas_row * 1);
  AL(w.part5, B * (size_t)w.ctas_row * 3);
  AL(w.partd, B * (size_t)w.ctas_row);
  AL(w.partu, std::max(B * (size_t)w.ctas_upd, (size_t)w.ctas_vec) * 3);
  AL(w.st, B);
  AL(w.gerr, 1);
  AL(w.illum, B);
  AL(w.xslot, B);
  AL(w.fwarm, B);
  AL(w.fstore, B);
  AL(w.segs, B);
  if (h->warm_start && h->model == MQNPM_MODEL_LS) AL(h->ufield, (size_t)h->L * N);
  h->have_field.assign(h->L, 0);
  AL(w.nactive, 1);
  AL(w.loops, 1);
  AL(w.dscal, 64);
  WproxWork& wp = h->wp;
  AL(wp.R, 3 * N); AL(wp.Pd, 3 * N); AL(wp.d, N); AL(wp.x, N);
  AL(wp.part, wprox_part_count(wp_blocks));
  AL(wp.stat, 4);
  AL(wp.gram, (size_t)wp.ctas_vec * wprox_part_len());
  AL(wp.scal, (size_t)woodbury_scal_count());
  AL(wp.barrier, (size_t)wprox_barrier_words());
  AL(wp.err, 1);
  wp.trace_cap = 1024;
  AL(wp.trace, 2 * (size_t)wp.trace_cap);
  AL(wp.status, N);
  {
    std::vector<float> mom = wprox_momentum(h->dual_iters);
    AL(wp.mom, mom.size());
    wp.mom_len = h->dual_iters;
    if ((e = cudaMemcpy(wp.mom, mom.data(), mom.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
      set_cuda_error(h, e, "momentum table");
      return fail(MQNPM_ERR_CUDA);
    }
  }
  AL(h->xbar, (size_t)h->S * N); AL(h->gbar, (size_t)h->S * N); AL(h->U, (size_t)h->S * N);
  AL(h->g, N); AL(h->vq, N); AL(h->Pwarm, 3 * N);
#undef AL
  if (!h->guards.empty()) {   // device table of the guard bands (itself unguarded)
    const size_t nb = h->guards.size();
    std::vector<unsigned char*> ptrs(nb);
    for (size_t i = 0; i < nb; ++i) ptrs[i] = h->guards[i].first;
    void* q = nullptr;
    if ((e = cudaMalloc(&q, nb * sizeof(unsigned char*))) != cudaSuccess) { set_cuda_error(h, e, "guard table"); return fail(MQNPM_ERR_CUDA); }
    h->allocations.push_back(q);
    h->guard_ptr = static_cast<unsigned char**>(q);
    if ((e = cudaMalloc(&q, nb * sizeof(int))) != cudaSuccess) { set_cuda_error(h, e, "guard flags"); return fail(MQNPM_ERR_CUDA); }
    h->allocations.push_back(q);
    h->guard_bad = static_cast<int*>(q);
    if ((e = cudaMemcpy(h->guard_ptr, ptrs.data(), nb * sizeof(unsigned char*), cudaMemcpyHostToDevice)) != cudaSuccess) {
      set_cuda_error(h, e, "guard table");
      return fail(MQNPM_ERR_CUDA);
    }
  }
  if ((e = cudaMallocHost(&w.h_nactive, sizeof(int))) != cudaSuccess) { set_cuda_error(h, e, "cudaMallocHost"); return fail(MQNPM_ERR_CUDA); }
  if ((e = cudaMallocHost(&w.h_loops, sizeof(int))) != cudaSuccess) { set_cuda_error(h, e, "cudaMallocHost"); return fail(MQNPM_ERR_CUDA); }
  if ((e = cudaMallocHost(&w.h_illum, B * sizeof(int))) != cudaSuccess) { set_cuda_error(h, e, "cudaMallocHost"); return fail(MQNPM_ERR_CUDA); }
  if ((e = cudaMallocHost(&w.h_xslot, B * sizeof(const float*))) != cudaSuccess ||
      (e = cudaMallocHost(&w.h_fwarm, B * sizeof(float2*))) != cudaSuccess ||
      (e = cudaMallocHost(&w.h_fstore, B * sizeof(float2*))) != cudaSuccess ||
      (e = cudaMallocHost(&w.h_segs, B * sizeof(GradSeg))) != cudaSuccess) {
    set_cuda_error(h, e, "cudaMallocHost");
    return fail(MQNPM_ERR_CUDA);
  }
  if ((e = cudaMallocHost(&w.h_scal, 64 * sizeof(double))) != cudaSuccess) { set_cuda_error(h, e, "cudaMallocHost"); return fail(MQNPM_ERR_CUDA); }

  // ---- tables: twiddles W_P^j per axis and incident-field axis factors
  // [l][nx + ny + nz] (x, then y, then z), built in FP64
  auto twiddles = [](int P) {
    std::vector<float2> tw(P);
    for (int j = 0; j < P; ++j) {
      const double a = 2.0 * M_PI * (double)j / (double)P;
      tw[j] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
    }
    return tw;
  };
  const std::vector<float2> twx = twiddles(Px), twy = twiddles(Py), twz = twiddles(Pz);
  std::vector<float2> tab(ntab);
  const int ext[3] = {nx, ny, nz};
  for (int l = 0; l < h->L; ++l) {
    size_t o = (size_t)l * (nx + ny + nz);
    for (int ax = 0; ax < 3; ++ax)
      for (int i = 0; i < ext[ax]; ++i, ++o) {
        const double ph = h->kb * h->kdir[3 * l + ax] * ((double)i - ext[ax] / 2.0) * h->h;
        tab[o] = make_float2((float)std::cos(ph), (float)std::sin(ph));
      }
  }
  cudaStream_t s = h->stream;
  if ((e = make_t2_tensor_map(w.T2, nx, ny, nz, (int)B, h->tile, w.t2map)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.gerr, 0, sizeof(int), s)) != cudaSuccess) {
    set_cuda_error(h, e, "tensor map of the transform buffer");
    return fail(MQNPM_ERR_CUDA);
  }
  if ((e = cudaMemcpyAsync(h->twx, twx.data(), Px * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->twy, twy.data(), Py * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->twz, twz.data(), Pz * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->tab, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = (khat_src ? cudaMemcpyAsync(h->khat, khat_src, (size_t)(nx + 1) * (ny + 1) * (nz + 1) * sizeof(float2),
                                       cudaMemcpyDeviceToDevice, s)
            : cfg->green_hat ? upload_khat(cfg->green_hat, nx, ny, nz, h->khat, s)
                             : build_khat(nx, ny, nz, h->h, h->kb, h->khat, s, h->green_kernel))) != cudaSuccess) {
    set_cuda_error(h, e, "create tables");
    return fail(MQNPM_ERR_CUDA);
  }
  if (h->remote && (e = detector_tables(h, cfg->det_distance, cfg->det_na)) != cudaSuccess) {
    set_cuda_error(h, e, "remote detector tables");
    return fail(MQNPM_ERR_CUDA);
  }
  h->tau.assign(h->alpha.begin(), h->alpha.end());
  h->has_u.assign(h->S, 0);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { set_cuda_error(h, e, "create sync"); return fail(MQNPM_ERR_CUDA); }
  if (cfg->tile < 0 && (rc = autotune_tile(h)) != MQNPM_OK) return fail(rc);
  w.ctas_row = green_row_ctas(nx, ny, nz, h->tile);
  *out = h;
  return MQNPM_OK;
}

extern "C" {

int mqnpm_create(const mqnpm_config* cfg, mqnpm_handle** out) { return create_handle(cfg, nullptr, out); }

int mqnpm_set_measurements(mqnpm_handle* h, const float* y) {
  if (!h || !y) return MQNPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  h->fields_valid = false;   // stored residuals refer to the old data
  CK(cudaMemcpyAsync(h->ymeas, y, (size_t)h->L * h->M * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
  h->have_meas = true;
  return MQNPM_OK;
}

int mqnpm_green_apply(mqnpm_handle* h, const float* v, float* out, int nb, int adjoint) {
  if (!h || !v || !out || nb < 1 || nb > h->max_batch) return set_error(h, MQNPM_ERR_INVALID_ARG, "green_apply: bad arguments");
  CK(cudaSetDevice(h->device));
  GreenCall c;
  c.nx = h->nx;
  c.ny = h->ny;
  c.nz = h->nz;
  c.nb = nb;
  c.adjoint = adjoint != 0;
  c.pro = PRO_PLAIN;
  c.pa.q = reinterpret_cast<const float2*>(v);
  c.epi = EPI_PLAIN;
  c.ea.out = reinterpret_cast<float2*>(out);
  c.T1 = h->w.T1;
  c.T2 = h->w.T2;
  c.khat = h->khat;
  c.twx = h->twx;
  c.twy = h->twy;
  c.twz = h->twz;
  c.part_pro = h->w.part1;
  c.part_epi = h->w.part5;
  c.ev = profile_slot(h, nb);
  c.launches = &h->launches;
  c.tile = h->tile;
  c.tmap = h->w.t2map;
  c.err = h->w.gerr;
  CK(green_launch(c, h->stream));
  int gerr = 0;
  CK(cudaMemcpyAsync(&gerr, h->w.gerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (gerr) return set_error(h, MQNPM_ERR_TIMEOUT, "green_apply: a bounded wait for a tile load gave up");
  return MQNPM_OK;
}

int mqnpm_forward(mqnpm_handle* h, const float* x, const int* illum, int nb, float* y_out, int* iters_out) {
  if (!h || !x || !illum || !y_out || nb < 1) return set_error(h, MQNPM_ERR_INVALID_ARG, "forward: bad arguments");
  for (int b = 0; b < nb; ++b)
    if (illum[b] < 0 || illum[b] >= h->L) return set_error(h, MQNPM_ERR_INVALID_ARG, "forward: illumination index");
  CK(cudaSetDevice(h->device));
  int rc = grad_batch_impl(h, x, illum, nb, 1.0, nullptr, nullptr, nullptr, false, reinterpret_cast<float2*>(y_out));
  if (iters_out)
    for (int b = 0; b < nb; ++b) iters_out[b] = h->last_iters[2 * b];
  return rc;
}

int mqnpm_grad_batch(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, float* grad_out,
                     double* loss_out, int* krylov_iters_out) {
  if (!h || !x || !illum || !grad_out || nb < 1) return set_error(h, MQNPM_ERR_INVALID_ARG, "grad_batch: bad arguments");
  if (!h->have_meas) return set_error(h, MQNPM_ERR_STATE, "grad_batch: measurements not set");
  for (int b = 0; b < nb; ++b)
    if (illum[b] < 0 || illum[b] >= h->L) return set_error(h, MQNPM_ERR_INVALID_ARG, "grad_batch: illumination index");
  CK(cudaSetDevice(h->device));
  return grad_batch_impl(h, x, illum, nb, scale, grad_out, loss_out, krylov_iters_out, true, nullptr);
}

int mqnpm_diagnostics(mqnpm_handle* h, const float* x_prev, const float* x_cur, int s_prime, double* out) {
  if (!h || !x_prev || !out || s_prime < 0 || s_prime >= h->S)
    return set_error(h, MQNPM_ERR_INVALID_ARG, "diagnostics: bad arguments");
  if (!h->have_meas) return set_error(h, MQNPM_ERR_STATE, "diagnostics: measurements not set");
  CK(cudaSetDevice(h->device));
  // h->g and h->vq hold a step's gradient and quasi-Newton point only within
  // mqnpm_step, so they serve as scratch here
  std::vector<int> all(h->L);
  for (int l = 0; l < h->L; ++l) all[l] = l;
  double loss = 0.0;
  int rc = grad_batch_impl(h, x_prev, all.data(), h->L, 1.0 / h->L, h->g, &loss, nullptr, true, nullptr);
  if (rc != MQNPM_OK && rc != MQNPM_ERR_NOT_CONVERGED) return rc;
  const std::vector<int>& sub = h->subsets[s_prime];
  const int rc2 = grad_batch_impl(h, x_prev, sub.data(), (int)sub.size(), (double)h->S / h->L, h->vq, nullptr,
                                  nullptr, true, nullptr);
  if (rc2 != MQNPM_OK && rc2 != MQNPM_ERR_NOT_CONVERGED) return rc2;
  double d3[3];
  CK(vec_reduce(h, 1, h->g, h->vq, x_cur ? x_cur : x_prev, x_prev, d3));
  out[0] = d3[0];
  out[1] = x_cur ? d3[2] : 0.0;
  out[2] = loss;
  return rc != MQNPM_OK ? rc : rc2;
}

int mqnpm_loss_batch(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, double* loss_out,
                     int* krylov_iters_out) {
  if (!h || !x || !illum || !loss_out || nb < 1) return set_error(h, MQNPM_ERR_INVALID_ARG, "loss_batch: bad arguments");
  if (!h->have_meas) return set_error(h, MQNPM_ERR_STATE, "loss_batch: measurements not set");
  for (int b = 0; b < nb; ++b)
    if (illum[b] < 0 || illum[b] >= h->L) return set_error(h, MQNPM_ERR_INVALID_ARG, "loss_batch: illumination index");
  CK(cudaSetDevice(h->device));
  return loss_batch_impl(h, x, illum, nb, scale, loss_out, krylov_iters_out);
}

int mqnpm_grad_fields(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, float* grad_out,
                      int reuse, int* reused_out) {
  if (!h || !x || !illum || !grad_out || nb < 1) return set_error(h, MQNPM_ERR_INVALID_ARG, "grad_fields: bad arguments");
  if (!h->have_meas) return set_error(h, MQNPM_ERR_STATE, "grad_fields: measurements not set");
  for (int b = 0; b < nb; ++b)
    if (illum[b] < 0 || illum[b] >= h->L) return set_error(h, MQNPM_ERR_INVALID_ARG, "grad_fields: illumination index");
  CK(cudaSetDevice(h->device));
  return grad_fields_impl(h, x, illum, nb, scale, grad_out, reuse != 0, reused_out);
}

int mqnpm_wprox(mqnpm_handle* h, const float* v, double tau_star, const float* U, int S_eff, double c, float* P_warm,
                float* x_out) {
  if (!h || !v || !x_out || v == x_out || !(tau_star > 0) || !(c > 0) || S_eff < 0 || S_eff > MQNPM_MAX_S ||
      (S_eff > 0 && !U))
    return set_error(h, MQNPM_ERR_INVALID_ARG, "wprox: bad arguments");
  CK(cudaSetDevice(h->device));
  UPtrs up{};
  for (int s = 0; s < S_eff; ++s) up.u[s] = U + (size_t)s * h->N;
  int rc = wprox_impl(h, v, tau_star, up, S_eff, c, P_warm, P_warm != nullptr, x_out);
  if (rc == MQNPM_OK) CK(cudaStreamSynchronize(h->stream));
  return rc;
}

int mqnpm_lipschitz(mqnpm_handle* h, const int* illum, int nb, double scale, const float* start, int iters,
                    double* alpha_out) {
  if (!h || !illum || !start || !alpha_out || nb < 1 || iters < 1) return set_error(h, MQNPM_ERR_INVALID_ARG, "lipschitz: bad arguments");
  for (int b = 0; b < nb; ++b)
    if (illum[b] < 0 || illum[b] >= h->L) return set_error(h, MQNPM_ERR_INVALID_ARG, "lipschitz: illumination index");
  CK(cudaSetDevice(h->device));
  return lipschitz_impl(h, illum, nb, scale, start, iters, alpha_out);
}

}  // extern "C"

// Subset of iteration k (Algorithm 4.1): s = k for k <= S, then s' by
// strategy I (cyclic) or II (the caller's draws).
int select_subset(mqnpm_handle* h, int k, int* sel) {
  const int S = h->S;
  if (k <= S) *sel = k - 1;
  else if (h->strategy == 1) *sel = (k - 1) % S;
  else {
    const int idx = k - S - 1;
    if (idx >= (int)h->draws.size()) return set_error(h, MQNPM_ERR_STATE, "step: strategy II draws exhausted");
    *sel = h->draws[idx];
  }
  return MQNPM_OK;
}

// Iteration k after its gradient: h->g holds grad F_{sel}(x) and loss its
// data term.  SR1 metric update (Algorithm 4.2), quasi-Newton point and the
// weighted proximal mapping (Eq. 4.5), then the bookkeeping of the step.
int finish_step(mqnpm_handle* h, float* x, int k, int sel, double loss, const std::vector<int>& its, int grad_rc,
                mqnpm_step_info* info) {
  cudaStream_t s = h->stream;
  const size_t N = h->N;
  const int S = h->S;
  int rc = MQNPM_OK;
  const std::vector<int>& sub = h->subsets[sel];
  float* xb = h->xbar + (size_t)sel * N;
  float* gb = h->gbar + (size_t)sel * N;
  int branch = -1;
  double tau_star;
  UPtrs up{};
  int S_eff = 0;
  double c;
  const int th = 256, gr = h->w.ctas_vec;
  if (k <= S) {
    // B_s = alpha_s I:  x_k = prox^{alpha_s I}_{a lam TV + iota_C}(x - (a/alpha_s) g)
    CK(cudaMemcpyAsync(xb, x, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(gb, h->g, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    h->tau[sel] = h->alpha[sel];
    h->has_u[sel] = 0;
    tau_star = h->alpha[sel];
    c = h->a * h->lambda;
    k_axpby<<<gr, th, 0, s>>>(x, h->g, (float)(-h->a / h->alpha[sel]), h->vq, N);
    CK(cudaGetLastError());
    h->launches += 1;
  } else {
    // Algorithm 4.2 on s = x - xbar_s', m = g - gbar_s'
    double d3[3];
    CK(vec_reduce(h, 1, x, xb, h->g, gb, d3));
    const double ss = d3[0], sm = d3[1], mm = d3[2];
    double tau = 0.0;
    bool rank1 = false;
    if (!finite_all(d3, 3)) return set_error(h, MQNPM_ERR_NONFINITE, "step: non-finite SR1 inner products");
    if (sm == 0.0) {
      tau = h->alpha[sel];
      branch = 1;
    } else {
      tau = std::min(mm / (h->gamma * sm), h->tau_max);
      if (tau <= 0.0) {
        tau = h->alpha[sel];
        branch = 1;
      } else {
        // ||m - tau s|| from the closed form mm - 2 tau sm + tau^2 ss
        const double qs = sm - tau * ss;
        const double qq = std::max(0.0, mm - 2.0 * tau * sm + tau * tau * ss);
        if (std::fabs(qs) <= h->delta1 * std::sqrt(ss) * std::sqrt(qq)) {
          branch = 2;
        } else {
          branch = 0;
          rank1 = true;
          while (sm - tau * ss <= h->delta2 * ss) {
            if (tau < h->delta2) {
              tau = h->alpha[sel];
              rank1 = false;
              branch = 3;
              break;
            }
            tau *= 0.5;
          }
        }
      }
    }
    if (rank1) {
      const double den = sm - tau * ss;
      k_sr1_u<<<gr, th, 0, s>>>(x, xb, h->g, gb, (float)tau, (float)(1.0 / std::sqrt(den)), h->U + (size_t)sel * N, N);
      CK(cudaGetLastError());
      h->launches += 1;
    }
    CK(cudaMemcpyAsync(xb, x, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(gb, h->g, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    h->tau[sel] = tau;
    h->has_u[sel] = rank1 ? 1 : 0;
    tau_star = 0.0;
    for (int q = 0; q < S; ++q) tau_star += h->tau[q];
    for (int q = 0; q < S; ++q)
      if (h->has_u[q]) up.u[S_eff++] = h->U + (size_t)q * N;
    c = h->a * S * h->lambda;
    // v_k = x - a S B^{-1} g, B = tau* I + U U^T
    if (S_eff == 0) {
      k_axpby<<<gr, th, 0, s>>>(x, h->g, (float)(-h->a * S / tau_star), h->vq, N);
      CK(cudaGetLastError());
      h->launches += 1;
    } else {
      rc = qn_point_impl(h, x, h->g, up, S_eff, tau_star, h->a * S, h->vq);
      if (rc != MQNPM_OK) return rc;
    }
  }
  if (!(c > 0)) {
    // lambda = 0: the proximal map reduces to the box projection under B
    c = 1e-30;
  }
  CK(cudaEventRecord(h->step_ev[2], s));
  rc = wprox_impl(h, h->vq, tau_star, up, S_eff, c, h->Pwarm, h->have_P, x);
  CK(cudaEventRecord(h->step_ev[3], s));
  if (rc != MQNPM_OK) return rc;
  h->have_P = true;
  CK(cudaStreamSynchronize(s));
  h->k = k;
  if (info) {
    info->k = k;
    info->subset = sel;
    info->loss = loss;
    info->tau_star = tau_star;
    info->rank = S_eff;
    info->sr1_branch = branch;
    int mx = 0, tot = 0;
    for (int v : its) {
      mx = std::max(mx, v);
      tot += v;
    }
    info->krylov_iters_max = mx;
    info->newton_iters_max = h->last_newton_max;
    info->krylov_iters_total = tot;
    info->n_illum = (int)sub.size();
    float t01 = 0.f, t12 = 0.f, t23 = 0.f;
    CK(cudaEventSynchronize(h->step_ev[3]));
    CK(cudaEventElapsedTime(&t01, h->step_ev[0], h->step_ev[1]));
    CK(cudaEventElapsedTime(&t12, h->step_ev[1], h->step_ev[2]));
    CK(cudaEventElapsedTime(&t23, h->step_ev[2], h->step_ev[3]));
    info->ms_gradient = t01;
    info->ms_metric = t12;
    info->ms_prox = t23;
  }
  return grad_rc;
}


int step_events(mqnpm_handle* h) {
  if (!h->step_ev[0]) {
    for (auto& ev : h->step_ev) CK(cudaEventCreate(&ev));
  }
  return MQNPM_OK;
}

extern "C" {

int mqnpm_step(mqnpm_handle* h, float* x, mqnpm_step_info* info) {
  if (!h || !x) return set_error(h, MQNPM_ERR_INVALID_ARG, "step: bad arguments");
  if (!h->have_meas) return set_error(h, MQNPM_ERR_STATE, "step: measurements not set");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const int S = h->S;
  const int k = h->k + 1;
  int sel = 0;
  int rc = select_subset(h, k, &sel);
  if (rc != MQNPM_OK) return rc;
  const std::vector<int>& sub = h->subsets[sel];
  double loss = 0.0;
  std::vector<int> its(2 * sub.size());
  if ((rc = step_events(h)) != MQNPM_OK) return rc;
  CK(cudaEventRecord(h->step_ev[0], s));
  rc = grad_batch_impl(h, x, sub.data(), (int)sub.size(), (double)S / h->L, h->g, &loss, its.data(), true, nullptr);
  CK(cudaEventRecord(h->step_ev[1], s));
  if (rc != MQNPM_OK && rc != MQNPM_ERR_NOT_CONVERGED) return rc;
  return finish_step(h, x, k, sel, loss, its, rc, info);
}

int mqnpm_step_subset(const mqnpm_handle* h, int* subset, int* illum, int* count) {
  if (!h || !count) return MQNPM_ERR_INVALID_ARG;
  int sel = 0;
  const int rc = select_subset(const_cast<mqnpm_handle*>(h), h->k + 1, &sel);
  if (rc != MQNPM_OK) return rc;
  const std::vector<int>& sub = h->subsets[sel];
  if (subset) *subset = sel;
  if (illum) std::memcpy(illum, sub.data(), sub.size() * sizeof(int));
  *count = (int)sub.size();
  return MQNPM_OK;
}

int mqnpm_step_with_gradient(mqnpm_handle* h, float* x, const float* g, double loss, mqnpm_step_info* info) {
  if (!h || !x || !g || g == x) return set_error(h, MQNPM_ERR_INVALID_ARG, "step_with_gradient: bad arguments");
  if (!std::isfinite(loss)) return set_error(h, MQNPM_ERR_NONFINITE, "step_with_gradient: non-finite loss");
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const int k = h->k + 1;
  int sel = 0;
  int rc = select_subset(h, k, &sel);
  if (rc != MQNPM_OK) return rc;
  if ((rc = step_events(h)) != MQNPM_OK) return rc;
  h->fields_valid = false;
  CK(cudaEventRecord(h->step_ev[0], s));
  CK(cudaMemcpyAsync(h->g, g, h->N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaEventRecord(h->step_ev[1], s));
  return finish_step(h, x, k, sel, loss, std::vector<int>(), MQNPM_OK, info);
}

// ---- checkpoint: header, then xbar, gbar, U (S x N floats each), P (3N floats)
struct StateHeader {
  unsigned magic;
  int nx, ny, nz, S, k, have_P, warm, L;
  int has_u[MQNPM_MAX_S];
  double tau[MQNPM_MAX_S];
};

int mqnpm_save_state(mqnpm_handle* h, void* buf, size_t* size) {
  if (!h || !size) return MQNPM_ERR_INVALID_ARG;
  const size_t N = h->N;
  const bool warm = h->ufield != nullptr;
  const size_t need = sizeof(StateHeader) + (3 * (size_t)h->S * N + 3 * N) * sizeof(float) +
                      (warm ? (size_t)h->L * (sizeof(int) + N * sizeof(float2)) : 0);
  if (!buf) {
    *size = need;
    return MQNPM_OK;
  }
  if (*size < need) return set_error(h, MQNPM_ERR_INVALID_ARG, "save_state: buffer too small");
  CK(cudaSetDevice(h->device));
  StateHeader hd{};
  hd.magic = 0x4d514e51u;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.nz = h->nz;
  hd.S = h->S;
  hd.k = h->k;
  hd.warm = warm ? 1 : 0;
  hd.L = h->L;
  hd.have_P = h->have_P ? 1 : 0;
  for (int s = 0; s < h->S; ++s) {
    hd.has_u[s] = h->has_u[s];
    hd.tau[s] = h->tau[s];
  }
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  const size_t SN = (size_t)h->S * N * sizeof(float);
  CK(cudaMemcpyAsync(p, h->xbar, SN, cudaMemcpyDeviceToHost, h->stream)); p += SN;
  CK(cudaMemcpyAsync(p, h->gbar, SN, cudaMemcpyDeviceToHost, h->stream)); p += SN;
  CK(cudaMemcpyAsync(p, h->U, SN, cudaMemcpyDeviceToHost, h->stream)); p += SN;
  CK(cudaMemcpyAsync(p, h->Pwarm, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  p += 3 * N * sizeof(float);
  if (warm) {
    std::memcpy(p, h->have_field.data(), (size_t)h->L * sizeof(int));
    p += (size_t)h->L * sizeof(int);
    CK(cudaMemcpyAsync(p, h->ufield, (size_t)h->L * N * sizeof(float2), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  *size = need;
  return MQNPM_OK;
}

int mqnpm_load_state(mqnpm_handle* h, const void* buf, size_t size) {
  if (!h || !buf) return MQNPM_ERR_INVALID_ARG;
  const size_t N = h->N;
  const bool warm = h->ufield != nullptr;
  const size_t need = sizeof(StateHeader) + (3 * (size_t)h->S * N + 3 * N) * sizeof(float) +
                      (warm ? (size_t)h->L * (sizeof(int) + N * sizeof(float2)) : 0);
  if (size < sizeof(StateHeader) || size < need) return set_error(h, MQNPM_ERR_INVALID_ARG, "load_state: buffer too small");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof hd);
  if (hd.magic != 0x4d514e51u || hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz || hd.S != h->S || hd.L != h->L || hd.warm != (warm ? 1 : 0))
    return set_error(h, MQNPM_ERR_INVALID_ARG, "load_state: state does not match this handle");
  CK(cudaSetDevice(h->device));
  const char* p = static_cast<const char*>(buf) + sizeof hd;
  const size_t SN = (size_t)h->S * N * sizeof(float);
  CK(cudaMemcpyAsync(h->xbar, p, SN, cudaMemcpyHostToDevice, h->stream)); p += SN;
  CK(cudaMemcpyAsync(h->gbar, p, SN, cudaMemcpyHostToDevice, h->stream)); p += SN;
  CK(cudaMemcpyAsync(h->U, p, SN, cudaMemcpyHostToDevice, h->stream)); p += SN;
  CK(cudaMemcpyAsync(h->Pwarm, p, 3 * N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  p += 3 * N * sizeof(float);
  if (warm) {
    std::memcpy(h->have_field.data(), p, (size_t)h->L * sizeof(int));
    p += (size_t)h->L * sizeof(int);
    CK(cudaMemcpyAsync(h->ufield, p, (size_t)h->L * N * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  h->k = hd.k;
  h->have_P = hd.have_P != 0;
  for (int s = 0; s < h->S; ++s) {
    h->has_u[s] = hd.has_u[s];
    h->tau[s] = hd.tau[s];
  }
  return MQNPM_OK;
}

}  // extern "C"
