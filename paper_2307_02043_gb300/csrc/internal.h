// Host-side declarations shared by the translation units of libmqnpm.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "kstate.h"
#include "mqnpm.h"

// One Green's apply over a batch: pass 1 (prologue) ... pass 5 (epilogue).
struct GreenCall {
  int nx = 0, ny = 0, nz = 0;  // grid; transform lengths Px = 2 nx, Py = 2 ny, Pz = 2 nz
  int nb = 0;                  // batch slots
  int pro = PRO_PLAIN;
  int epi = EPI_PLAIN;
  bool adjoint = false;        // use conj(K_hat): G^H
  ProArgs pa{};
  EpiArgs ea{};
  float2* T1 = nullptr;        // [nb][nz][ny][Px]
  float2* T2 = nullptr;        // [nb][nz][Py][Px]
  const float2* khat = nullptr;  // octant (nz+1)(ny+1)(nx+1), scaled by 1/(Px Py Pz)
  const float2* twx = nullptr;   // W_P^j, j < P, for P = Px, Py, Pz
  const float2* twy = nullptr;
  const float2* twz = nullptr;
  const KState* st = nullptr;    // slot activity (nullptr: all active)
  double* part_pro = nullptr;    // [nb][ctas1][NPART]
  double* part_epi = nullptr;    // [nb][ctas5][NPART]
  cudaEvent_t* ev = nullptr;     // optional: 6 events recorded around the 5 passes
  long long* launches = nullptr; // optional kernel-launch counter (+5 per apply)
  const void* tmap = nullptr;    // CUtensorMap of T2 for the pass-3 tile loads
  int* err = nullptr;            // device flag raised when a bounded wait gives up
  bool plane = false;            // input nonzero on the last z-plane only (the lift S^T r; G^H only)
  bool outplane = false;         // only the last z-plane of the output is needed (first-Born data; G only)
  // optional: launched right after pass 1 on the same stream; a slot it marks
  // active = 2 skips the remaining passes (the fused x/y passes are not used
  // on the forward side when it is set)
  cudaError_t (*after_pass1)(void* ctx, cudaStream_t s) = nullptr;
  void* after_pass1_ctx = nullptr;
  int tile = 0;                  // launch shapes: alternative shape of bit 0 the x passes, bit 1 the
                                 // y passes, bit 2 the z pass; bit 3 two z-pass exchange buffers;
                                 // bit 4 the fused x/y passes (square planes, P = 128 or 256)
};

constexpr int MQ_TILES = 32;     // launch-shape variants of the Green's passes
constexpr int MQ_TILE_FUSED = 16;   // tile bit: passes 1+2 and 4+5 as fused cluster kernels

// Tensor map of the pass-3 buffer T2 = [max_batch * nz][Py][Px] complex64, box C x 1 x nz
// with C the column width of the tile's z-pass shape.
cudaError_t make_t2_tensor_map(void* T2, int nx, int ny, int nz, int max_batch, int tile,
                               void* map_out /* CUtensorMap, 64 B aligned */);

// Per-pass timing (opt-in tracing): events recorded around every Green's apply.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;   // groups of 6
  int used = 0;                  // groups recorded
  std::vector<int> nb;           // batch slots of each recorded call
  double acc_ms[5] = {0, 0, 0, 0, 0};   // applies replayed inside CUDA graphs, summed per pass
  long long acc_slots = 0;
  int acc_calls = 0;
  cudaEvent_t* next();
};

// One BiCGSTAB iteration captured as a CUDA graph for a batch shape.
struct KrylovGraph {
  int nb = 0;
  bool adjoint = false, prof = false;
  bool loop = false;             // the whole solve: a conditional WHILE node around the iteration
  const float* x = nullptr;
  const float2* xs = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[12] = {};       // pass boundaries of the two applies (when profiled)
  long long kernels = 0;         // kernels per replay
};

// Number of CTAs pass 1 / pass 5 use per slot (partials layout) for a tile
// variant; green_row_ctas_max covers every variant.
int green_row_ctas(int nx, int ny, int nz, int tile);
int green_row_ctas_max(int nx, int ny, int nz);
int green_plane_ctas(int nx, int ny, int tile);   // CTAs per slot of pass 1/5 over one z-plane
// shape[6] = lines per CTA and threads per line of passes 1/5 (length Px),
// columns per CTA and threads per column of passes 2/4 (Py), then of pass 3
// (Pz) (zeros if a length is unsupported); smem = the largest dynamic shared
// memory of the tile's passes.
void green_shape(int nx, int ny, int nz, int tile, int* shape, size_t* smem = nullptr);
// Whether a tile's passes fit the device's shared memory per block (the
// column passes cover kx < Px with a ragged last tile where needed).
bool green_tile_fits(int nx, int ny, int nz, int tile, int device);
int green_col_width(int nx, int ny, int nz, int tile);   // columns per CTA of pass 3 (the tensor-map box)
bool green_supported(int n);                             // 2n is a compiled transform length
bool green_fused_supported(int nx, int ny);              // fused x/y passes exist for this plane
cudaError_t green_launch(const GreenCall& c, cudaStream_t s);

// Per-P entry points (one translation unit each): the passes along an axis
// whose transform length is P.
#define MQ_DECL(P)                                                                         \
  cudaError_t green_pass1_P##P(const GreenCall& c, cudaStream_t s);                        \
  cudaError_t green_pass5_P##P(const GreenCall& c, cudaStream_t s);                        \
  cudaError_t green_passy_P##P(const GreenCall& c, bool inv, cudaStream_t s);              \
  cudaError_t green_pass3_P##P(const GreenCall& c, cudaStream_t s);                        \
  void green_shape_P##P(int tile, int* shape, size_t* smem_row, size_t* smem_col, size_t* smem_z); \
  cudaError_t green_fused_P##P(const GreenCall& c, bool inv, cudaStream_t s);              \
  size_t green_fused_smem_P##P();
MQ_DECL(16) MQ_DECL(24) MQ_DECL(32) MQ_DECL(48) MQ_DECL(64) MQ_DECL(96) MQ_DECL(128)
MQ_DECL(192) MQ_DECL(256) MQ_DECL(320) MQ_DECL(384)
#undef MQ_DECL

// K_hat octant in FP64 by separable even (cosine) sums, rounded to complex64.
cudaError_t build_khat(int nx, int ny, int nz, double h, double kb, float2* khat_out, cudaStream_t s, int kernel);
cudaError_t upload_khat(const float* host, int nx, int ny, int nz, float2* khat_out, cudaStream_t s);
cudaError_t build_khat_scratch(int n, double h, double kb, float2* khat_out, double2* a, double2* b, double* dcos,
                               cudaStream_t s);

// ----------------------------------------------------------------- handle
struct Workspace {
  // BiCGSTAB vectors, [max_batch][N] complex64 each
  float2 *u = nullptr, *zs = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr,
         *s = nullptr, *t = nullptr;
  float2 *T1 = nullptr, *T2 = nullptr;   // transform scratch
  float2* rdet = nullptr;                // [max_batch][M]
  float2 *dtmp1 = nullptr, *dtmp2 = nullptr, *rlift = nullptr;   // remote detector: [max_batch][M] each
  double *part1 = nullptr, *part5 = nullptr, *partu = nullptr, *partd = nullptr;
  KState* st = nullptr;                  // [max_batch]
  int* illum = nullptr;                  // [max_batch]
  int* nactive = nullptr;                // device counter
  int* h_nactive = nullptr;              // pinned host mirror
  int* loops = nullptr;                  // device: iterations run by the device-side Krylov loop
  int* h_loops = nullptr;                // pinned host mirror
  int* h_illum = nullptr;                // pinned staging of slot illuminations
  const float** xslot = nullptr;         // [max_batch] contrast of each slot (shared launches)
  float2** fwarm = nullptr;              // [max_batch] field a warm start reads (NULL: u_in)
  float2** fstore = nullptr;             // [max_batch] where the converged field is kept (NULL: nowhere)
  GradSeg* segs = nullptr;               // [max_batch] gradient segments of the chunk
  const float** h_xslot = nullptr;       // pinned staging of the four tables above
  float2** h_fwarm = nullptr;
  float2** h_fstore = nullptr;
  GradSeg* h_segs = nullptr;
  double* h_scal = nullptr;              // pinned scalar staging (64 doubles)
  double* dscal = nullptr;               // device scalar scratch (64 doubles)
  int ctas_row = 0, ctas_upd = 0, ctas_vec = 0;
  int* gerr = nullptr;                   // raised by a Green's pass whose bounded wait gave up
  alignas(64) unsigned char t2map[128];  // CUtensorMap of T2
};

struct WproxWork {
  float *R = nullptr, *Pd = nullptr, *d = nullptr, *x = nullptr;
  float* mom = nullptr;         // momentum table of the dual iterations (dual_iters)
  int mom_len = 0;
  double* part = nullptr;       // per-block and per-group partials of the cooperative kernel
  double* stat = nullptr;       // [4] Newton statistics of the last call
  double* gram = nullptr;       // partials of the Woodbury Gram pass [ctas_vec][44]
  double* scal = nullptr;       // Woodbury scalars (G, M, U^T g)
  unsigned* barrier = nullptr;  // monotonic arrival counters of the grid barriers (wprox_barrier_words())
  int* err = nullptr;           // device error flag
  unsigned char* status = nullptr;  // per-voxel inner/clipped status of the Newton evaluations
  long long* trace = nullptr;   // phase trace of the last call: (tag, ns) per barrier
  int trace_cap = 0;
  int nsm = 0;
  int ctas_vec = 0;
};

struct mqnpm_handle {
  // problem: an nx x ny x nz grid (transform lengths 2 nx, 2 ny, 2 nz), M = nx ny detector values
  int nx = 0, ny = 0, nz = 0, M = 0, model = 1, L = 0, S = 0, tv = 0, strategy = 1;
  int3 dims() const { return make_int3(nx, ny, nz); }
  size_t N = 0;
  double h = 1.0, kb = 0.0, lambda = 0.0, lo = 0.0, hi = 0.0, a = 1.0, gamma = 0.8, tau_max = 0.0;
  double delta1 = 1e-8, delta2 = 1e-12, krylov_tol = 1e-6, newton_tol = 1e-6;
  int krylov_maxit = 500, dual_iters = 20, newton_maxit = 50, max_batch = 1, device = 0;
  int check_every = 1;
  long long barrier_limit = 4000000000LL;   // grid-barrier wait of the prox kernel, SM cycles
  int green_kernel = 0;                      // MQNPM_KERNEL_SAMPLED or MQNPM_KERNEL_TRUNCATED
  std::vector<double> kdir, alpha;
  std::vector<int> subset_of, draws;
  std::vector<std::vector<int>> subsets;
  cudaStream_t stream = nullptr;
  std::string err;
  size_t bytes = 0, budget = 0;
  std::vector<void*> allocations;
  size_t guard = 0;                               // guard-band bytes per side (0: none)
  std::vector<std::pair<unsigned char*, size_t>> guards;   // device guard bands
  unsigned char** guard_ptr = nullptr;            // device table of the bands (check kernel)
  int* guard_bad = nullptr;                       // device flags, one per band
  // device tables
  float2 *khat = nullptr, *tab = nullptr, *ymeas = nullptr;
  float2 *twx = nullptr, *twy = nullptr, *twz = nullptr;   // W_P^j per axis (P = 2 nx, 2 ny, 2 nz)
  bool remote = false;                    // detector behind an angular-spectrum propagation
  float2 *twn = nullptr, *Hdet = nullptr;  // W_nx^j (nx), then W_ny^j (ny); H / (nx ny) ([ky][kx], M)
  bool have_meas = false;
  Workspace w;
  WproxWork wp;
  // forward fields and residuals of the last loss-only call (for its gradient)
  bool fields_valid = false;
  const float* fields_x = nullptr;
  std::vector<int> fields_illum;
  // Krylov warm start: last forward field per illumination
  bool warm_start = false;
  bool adjoint_from_b = true;                // adjoint solves start at z_0 = b (else at 0)
  int forward_refine_steps = 1;              // fixed-point steps on a warm forward start before BiCGSTAB
  float2* ufield = nullptr;      // [L][N]
  std::vector<int> have_field;   // [L]
  // outer-loop state (Algorithm 4.1)
  int k = 0;
  float *xbar = nullptr, *gbar = nullptr, *U = nullptr, *g = nullptr, *vq = nullptr, *Pwarm = nullptr;
  std::vector<double> tau;
  std::vector<int> has_u;
  bool have_P = false;
  // diagnostics of the last calls
  std::vector<int> last_iters;   // per illumination of the last gradient: forward, adjoint
  int last_newton_max = 0, last_newton_total = 0;
  int last_status = 0;
  Profiler prof;
  bool direct_launches = false;
  int tile = 0;                            // launch shapes of the Green's passes (GreenCall::tile)
  double tune_ms[MQ_TILES] = {};   // autotuner timings (-1: not timed; set at create)
  cudaStream_t capture_stream = nullptr;   // stream the iteration graphs are captured on
  std::vector<KrylovGraph> graphs;         // captured iterations (a few batch shapes)
  long long launches = 0;        // kernels launched by this handle since creation
  long long pending_loop_kernels = 0;   // kernels per pass of the last device-side Krylov loop (not yet counted)
  cudaEvent_t step_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // phase timing of mqnpm_step
};

// mqnpm_create with the Green's spectrum copied from khat_src (device, the
// folded octant of the same grid) when it is not null (api.cu).
int create_handle(const mqnpm_config* cfg, const float2* khat_src, mqnpm_handle** out);

// Record the next profiling group for a Green's apply of nb slots (nullptr when off/full).
cudaEvent_t* profile_slot(mqnpm_handle* h, int nb);

// krylov.cu
// Per-slot tables of one chunk of solves (see stage_chunk).
struct ChunkTables {
  int m = 0;
  std::vector<int> illum;           // illumination of each slot (index into tab and ymeas)
  std::vector<const float*> x;      // contrast of each slot (empty: the call's shared x)
  std::vector<float2*> warm, store; // start field / field store of each slot (empty: none)
  std::vector<GradSeg> segs;        // runs of slots summed into one gradient each
};
int stage_chunk(mqnpm_handle* h, const ChunkTables& t);
int chunk_forward(mqnpm_handle* h, const float* x, int m, int* it_chunk, float2* det_out, const float2* ym,
                  bool warm, bool store, const std::vector<GradSeg>& segs);
int chunk_adjoint(mqnpm_handle* h, const float* x, int m, int* it_chunk, int nseg);
int check_tile_waits(mqnpm_handle* h);
int grad_batch_impl(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale,
                    float* grad, double* loss, int* iters, bool want_grad, float2* y_out);
int loss_batch_impl(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, double* loss,
                    int* iters);
int grad_fields_impl(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale, float* grad,
                     bool reuse, int* reused);
int lipschitz_impl(mqnpm_handle* h, const int* illum, int nb, double scale, const float* start,
                   int iters, double* alpha_out);
cudaError_t vec_reduce(mqnpm_handle* h, int kind, const float* a, const float* b, const float* c,
                       const float* d, double* host_out);

// wprox.cu
struct UPtrs {
  const float* u[16];
};
int wprox_impl(mqnpm_handle* h, const float* v, double tau, const UPtrs& U, int S_eff, double c,
               float* P_warm, bool warm, float* x_out);
int qn_point_impl(mqnpm_handle* h, const float* x, const float* g, const UPtrs& U, int S_eff, double tau,
                  double aS, float* v);
std::vector<float> wprox_momentum(int J);
int wprox_part_len();
int wprox_blocks_per_sm();                // co-resident blocks per SM of the cooperative prox kernel
size_t wprox_part_count(int max_blocks);   // doubles of the partials buffer
int wprox_barrier_words();                // unsigned words of the barrier counters
int woodbury_scal_count();

// detector.cu: remote detector D = F^-1 diag(H) F on the n x n slices
cudaError_t detector_tables(mqnpm_handle* h, double distance, double na);
// det (m slices) <- D(det) - y_meas(illum) (y_meas may be null), partials in w.partd
cudaError_t detector_forward(mqnpm_handle* h, float2* det, int m, const float2* ym, const int* illum);
// out <- D^H r (m slices)
cudaError_t detector_adjoint(mqnpm_handle* h, const float2* r, float2* out, int m);

// api.cu: the outer loop around a subset gradient (shared by mqnpm_step,
// mqnpm_step_with_gradient and the group step)
int select_subset(mqnpm_handle* h, int k, int* sel);
int finish_step(mqnpm_handle* h, float* x, int k, int sel, double loss, const std::vector<int>& its, int grad_rc,
                mqnpm_step_info* info);
int step_events(mqnpm_handle* h);

// tune.cu: pick the launch shapes of the Green's passes by timing
int autotune_tile(mqnpm_handle* h);

// status helpers (api.cu)
int set_cuda_error(mqnpm_handle* h, cudaError_t e, const char* where);
int set_error(mqnpm_handle* h, int code, const std::string& msg);
