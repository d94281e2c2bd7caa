/*
 * mqnpm.h -- C ABI of libmqnpm, the GB300 (sm_103a) hot path of the mini-batch
 * quasi-Newton proximal method (BQNPM, Algorithm 4.1 of "A Mini-Batch
 * Quasi-Newton Proximal Method for Constrained Total Variation Nonlinear Image
 * Reconstruction") for optical diffraction tomography.
 *
 * Problem (Eqs. 1.1-1.2, 4.1):
 *     min_{x in C}  (1/L) sum_l f_l(x) + lambda TV(x),
 *     f_l(x) = 1/2 || H_l(x) - y_l ||^2,   C = [box_lo, box_hi]^N,
 *     F_s = (S/L) sum_{l in S_s} f_l  over S non-overlapping subsets.
 *
 * Conventions shared by every call
 *   - A volume is nx*ny*nz voxels, indexed [z][y][x] with x fastest;
 *     N = nx ny nz.  Detector vectors hold the last z-slice, [y][x],
 *     M = nx ny values.
 *   - Real vectors are float32; complex vectors are interleaved (re, im)
 *     float32 pairs (the memory layout of torch.complex64).
 *   - Every pointer argument documented as "device" is a CUDA device pointer on
 *     the handle's device; "host" pointers are ordinary CPU memory.  The caller
 *     owns all buffers it passes; the library only reads or writes them during
 *     the call and keeps no reference.  The library owns its workspace, which is
 *     allocated in mqnpm_create and released by mqnpm_destroy.
 *   - All device work is ordered on the handle's stream (mqnpm_set_stream).
 *     Calls that return host values synchronise that stream before returning.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Every call returns an mqnpm_status; on failure mqnpm_last_error() gives
 *     a readable message.  MQNPM_ERR_NOT_CONVERGED still writes every output.
 */
#ifndef MQNPM_H
#define MQNPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mqnpm_status {
  MQNPM_OK = 0,
  MQNPM_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range       */
  MQNPM_ERR_BUDGET = 2,        /* the workspace would exceed hbm_budget_bytes       */
  MQNPM_ERR_CUDA = 3,          /* a CUDA runtime call failed                        */
  MQNPM_ERR_NOT_CONVERGED = 4, /* a Krylov or Newton solve hit its iteration cap    */
  MQNPM_ERR_NONFINITE = 5,     /* NaN/Inf met in a solve                            */
  MQNPM_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                */
  MQNPM_ERR_UNSUPPORTED = 7,   /* grid size without a compiled transform plan       */
  MQNPM_ERR_STATE = 8          /* call order violated (e.g. no measurements set)    */
} mqnpm_status;

enum { MQNPM_MODEL_BORN = 0, MQNPM_MODEL_LS = 1 };
enum { MQNPM_TV_ISO = 0, MQNPM_TV_ANISO = 1 };
/* Discretisation of the Green's function (Section 6; the paper defers its
 * forward model to a supplement, so both are the library's stated readings):
 * SAMPLED  w_D = h^3 g(|D| h) with the exact integral over the equal-volume
 *          sphere at D = 0;
 * TRUNCATED the truncated kernel of Vico, Greengard and Ferrando (2016): the
 *          transform of g restricted to r <= h sqrt(nx^2 + ny^2 + nz^2) (the
 *          domain's diagonal), sampled with periods T_d h along each axis,
 *          T_d = 4 n_d (raised to the next even count >= n_d + R/h for an
 *          elongated domain), which makes G v the continuous convolution of the band-limited
 *          interpolant of v (spectrally accurate for smooth v). */
enum { MQNPM_KERNEL_SAMPLED = 0, MQNPM_KERNEL_TRUNCATED = 1 };

/* Largest number of subsets S (rank of the quasi-Newton metric) supported. */
#define MQNPM_MAX_S 16
/* Largest workspace batch (illuminations solved together); larger mini-batches
 * run in chunks of max_batch. */
#define MQNPM_MAX_BATCH 64

typedef struct mqnpm_config {
  /* --- forward model (Section 6; discretisation is the library's stated reading) */
  int nx, ny, nz;          /* grid edges (x fastest); each transform length 2 n_d
                              must be one of 16,24,32,48,64,96,128,192,256,320,384
                              (else UNSUPPORTED), nx a multiple of 4 for the
                              proximal mapping                                      */
  double h;                /* voxel size (length unit)                              */
  double kb;               /* background wavenumber 2*pi/lambda_b (per unit length) */
  int model;               /* MQNPM_MODEL_LS (Lippmann-Schwinger) or _BORN          */
  int L;                   /* number of illuminations                               */
  const double* kdir;      /* host, L x 3 unit wave-vector directions (kx, ky, kz)  */
  /* --- subsets and outer loop (Algorithm 4.1) */
  int S;                   /* number of subsets, 1 <= S <= MQNPM_MAX_S              */
  const int* subset_of;    /* host, L entries in [0, S): subset of illumination l   */
  const double* alpha;     /* host, S entries alpha_s > 0 (Lipschitz constants)     */
  double step;             /* a_k (constant)                                        */
  int strategy;            /* 1: s' = mod(k, S) cyclic; 2: s' from strategy_draws   */
  const int* strategy_draws; /* host, n_draws subset indices for strategy II        */
  int n_draws;
  /* --- regulariser and constraint (Eqs. 1.2, 3.1-3.4) */
  int tv;                  /* MQNPM_TV_ISO or MQNPM_TV_ANISO                        */
  double lambda;
  double box_lo, box_hi;   /* C = [box_lo, box_hi]^N                                */
  /* --- SR1 (Algorithm 4.2) */
  double gamma;            /* in (0, 1]                                             */
  double tau_max;          /* <= 0 selects 1e3 * max_s alpha_s                      */
  double delta1, delta2;   /* <= 0 selects 1e-8 and 1e-12                           */
  /* --- inner solvers */
  double krylov_tol;       /* BiCGSTAB relative residual                            */
  int krylov_maxit;
  int dual_iters;          /* accelerated dual projected-gradient iterations J      */
  double newton_tol;       /* semi-smooth Newton tolerance (Algorithm 4.3)          */
  int newton_maxit;
  /* --- resources */
  int max_batch;           /* illuminations solved together (workspace sizing),
                              1..MQNPM_MAX_BATCH                                    */
  size_t hbm_budget_bytes; /* 0: no limit; else create fails with MQNPM_ERR_BUDGET  */
  int device;              /* CUDA device ordinal                                   */
  void* stream;            /* cudaStream_t for all work (NULL: legacy default)      */
  /* --- Krylov initial guess (the paper leaves it open) */
  int warm_start;          /* 1: each LS forward solve starts from the field last
                              computed for the same illumination (kept on the
                              device, L x N complex, and in checkpoints);
                              0: from u_in                                     */
  int direct_launches;     /* 0: a BiCGSTAB iteration (14 kernels) is captured
                              once per batch shape as a CUDA graph and replayed;
                              1: its kernels are launched one by one          */
  const float* green_hat;  /* host, (nz+1)(ny+1)(nx+1) complex64 [fz][fy][fx] or
                              NULL: the first octant of the DFT of the periodic
                              (periods 2 nx, 2 ny, 2 nz) Green's
                              kernel (even in every axis; any discretisation of
                              G, e.g. a truncated kernel), used instead of the
                              library's own (Section 6 reading)              */
  int tile;                /* launch shapes of the Green's passes: -1 picks the
                              fastest of 0..31 by timing at create (cached per
                              device, grid and batch slots); 0..31 fixes them: bits
                              0, 1, 2 select the alternative shape (lines or
                              columns per CTA, threads per line or column) of
                              the x, y and z passes, bit 3 two exchange buffers
                              in the z pass, bit 4 the fused x/y passes (pairs
                              of CTAs per z-plane in a thread-block cluster;
                              nx = ny = 64 or 128 with bits 0 and 1 clear; same
                              results bit for bit) (0 = the built-in defaults) */
  double det_distance;     /* remote detector (det_na > 0): distance from the last
                              z-slice to the detector plane, units of h        */
  double det_na;           /* 0: the detector is the last z-slice; > 0: that
                              slice propagated by the angular spectrum over
                              det_distance with the pupil kx^2 + ky^2 <=
                              (det_na kb)^2 (Section 6 reading)               */
  size_t guard_bytes;      /* debugging: 0 = off; else every workspace buffer is
                              framed by guard bands of this many bytes (rounded
                              up to 256) filled with 0xA5, checked by
                              mqnpm_check_guards                              */
  long long barrier_wait_cycles; /* longest wait of one block of the weighted
                              proximal mapping at a grid barrier, in SM clock
                              cycles, before it gives up and the call returns
                              MQNPM_ERR_TIMEOUT; 0 selects 4e9 (about 2 s)    */
  int green_kernel;        /* MQNPM_KERNEL_SAMPLED (0) or MQNPM_KERNEL_TRUNCATED;
                              ignored when green_hat is given. The truncated
                              kernel's construction at create holds two
                              (2n+1)^3 FP64 complex buffers for its duration */
  int adjoint_start;       /* LS adjoint solves (I - G^H X) z = b, b = G^H S^T r:
                              0 starts at z_0 = b (one more Green's apply for
                              r_0 = G^H(x b); at contrasts up to about 0.04 it
                              saves one BiCGSTAB iteration, two applies);
                              1 starts at z_0 = 0 (r_0 = b)                    */
  int forward_start;       /* LS forward solves started from a stored field u_s
                              (warm_start): 0 refines it by one fixed-point
                              step u_1 = u_s + r_0 before BiCGSTAB (one more
                              Green's apply, r_1 = G(x r_0); a solve whose r_1
                              meets the tolerance then takes no BiCGSTAB
                              iteration); 1 starts BiCGSTAB at u_s          */
} mqnpm_config;

typedef struct mqnpm_handle mqnpm_handle;

typedef struct mqnpm_step_info {
  int k;                   /* iteration index after the call (1-based)             */
  int subset;              /* s or s' used by the iteration (0-based)              */
  double loss;             /* F_s(x_{k-1}) of the chosen subset                     */
  double tau_star;         /* sum_s tau_s of the metric used                        */
  int rank;                /* number of rank-one terms in the metric               */
  int sr1_branch;          /* 0: rank-1 update, 1: tau<=0, 2: skip, 3: tau tiny, -1: k<=S */
  int krylov_iters_max;    /* largest BiCGSTAB iteration count in the gradient     */
  int newton_iters_max;    /* largest semi-smooth Newton count in the prox         */
  int krylov_iters_total;  /* forward + adjoint BiCGSTAB iterations, all illuminations */
  int n_illum;             /* illuminations in the subset                          */
  double ms_gradient;      /* device time of the subset gradient                   */
  double ms_metric;        /* device time of the SR1 update and quasi-Newton point */
  double ms_prox;          /* device time of the weighted proximal mapping         */
} mqnpm_step_info;

/* Create a handle: validates cfg, builds the Green's kernel spectrum (or
 * scales cfg->green_hat by 1/(8 nx ny nz) and rounds it once) and the
 * incident-field tables, and allocates the workspace for max_batch
 * illuminations.  Host arrays in cfg are copied.  Errors: INVALID_ARG (also
 * a non-finite green_hat value), UNSUPPORTED (grid), BUDGET, CUDA.  On error
 * *out is NULL. */
int mqnpm_create(const mqnpm_config* cfg, mqnpm_handle** out);

/* Release the workspace.  NULL is accepted. */
void mqnpm_destroy(mqnpm_handle* h);

/* Message of the last failure on this handle (never NULL). */
const char* mqnpm_last_error(const mqnpm_handle* h);

/* Replace the stream all later work is ordered on. */
int mqnpm_set_stream(mqnpm_handle* h, void* stream);

/* Replace barrier_wait_cycles (failure detection: no counterpart in the
 * paper).  cycles >= 0; 0 selects the default.  A wait that runs out makes
 * the next mqnpm_wprox or mqnpm_step return MQNPM_ERR_TIMEOUT with its
 * outputs unspecified; the handle stays usable and the next call starts
 * clean.  INVALID_ARG for a negative value. */
int mqnpm_set_wait_limit(mqnpm_handle* h, long long cycles);

/* Bytes of device memory the handle holds. */
size_t mqnpm_workspace_bytes(const mqnpm_handle* h);

/* Copy the measurements y_l (Eq. 1.1): device, L x M complex. */
int mqnpm_set_measurements(mqnpm_handle* h, const float* y);

/* G v or G^H v for nb volumes (the discrete Lippmann-Schwinger operator's
 * Green's convolution; adjoint != 0 selects G^H).  v, out: device, nb x N
 * complex; they must not overlap.  nb <= max_batch. */
int mqnpm_green_apply(mqnpm_handle* h, const float* v, float* out, int nb, int adjoint);

/* H_l(x) for the illuminations illum[0..nb) (Section 6: one LS solve per
 * illumination, or the first-Born field).  x: device N; illum: host nb ints;
 * y_out: device nb x M complex; iters_out: host nb ints or NULL.
 * NOT_CONVERGED if a solve hit krylov_maxit (outputs still written). */
int mqnpm_forward(mqnpm_handle* h, const float* x, const int* illum, int nb,
                  float* y_out, int* iters_out);

/* Mini-batch data-term gradient (Section 6, Eq. 4.1):
 *   grad_out = scale * sum_{l in illum} grad f_l(x),  *loss_out = scale * sum f_l(x),
 * with grad f_l = Re(conj(u_l) .* z_l), u_l the LS field (or u_in for Born) and
 * z_l = (I - G^H X)^{-1} G^H S^T (H_l(x) - y_l) (the adjoint solve).  scale = S/L
 * gives grad F_s.  x, grad_out: device N floats (may alias only if identical
 * buffers are not required afterwards: grad_out is written last).  illum: host.
 * Batches larger than max_batch are processed in chunks.  loss_out (host) and
 * krylov_iters_out (host, 2*nb ints: forward, adjoint) may be NULL.
 * Requires mqnpm_set_measurements.  NOT_CONVERGED as above. */
int mqnpm_grad_batch(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale,
                     float* grad_out, double* loss_out, int* krylov_iters_out);

/* Data term of a mini-batch without its gradient (Eq. 4.1, the forward half of
 * mqnpm_grad_batch): *loss_out = scale * sum_{l in illum} f_l(x).  x: device N
 * floats; illum, loss_out (host); krylov_iters_out: host nb ints (forward
 * solves) or NULL.  When nb <= max_batch the forward fields and detector
 * residuals stay in the workspace for a following mqnpm_grad_fields; any other
 * data-term, forward, step or lipschitz call, or new measurements, drop them.
 * Errors as mqnpm_grad_batch. */
int mqnpm_loss_batch(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale,
                     double* loss_out, int* krylov_iters_out);

/* Gradient of the same data term (the backward half): grad_out (device N
 * floats) = scale * sum grad f_l(x).  With reuse != 0, and when the workspace
 * still holds the fields of the last mqnpm_loss_batch for the same x pointer
 * and illumination list, only the adjoint solves run (the caller guarantees
 * that the contents of x did not change in between); otherwise the forward
 * fields are recomputed, chunk by chunk.  *reused_out (host, may be NULL) is 1
 * when the stored fields were used. */
int mqnpm_grad_fields(mqnpm_handle* h, const float* x, const int* illum, int nb, double scale,
                      float* grad_out, int reuse, int* reused_out);

/* Weighted proximal mapping of c*TV + iota_C under B = tau_star I + U U^T
 * (Eq. 4.5, Theorem 3.1, Lemma 4.1, Algorithm 4.3):
 *   x_out ~= argmin_{x in C} 1/2 ||x - v||_B^2 + c TV(x)
 * by cfg.dual_iters accelerated projected-gradient steps on the dual T(P).
 * v, x_out: device N floats (distinct).  U: device S_eff x N floats (row s is
 * u_s), NULL when S_eff = 0; 0 <= S_eff <= MQNPM_MAX_S.  tau_star > 0, c > 0.
 * P_warm: device 3 x N floats (components q_x, q_y, q_z) used as the starting
 * dual field and overwritten with the final one; NULL starts from zero. */
int mqnpm_wprox(mqnpm_handle* h, const float* v, double tau_star, const float* U, int S_eff,
                double c, float* P_warm, float* x_out);

/* One iteration k of Algorithm 4.1 on x (device N floats, in/out), including
 * the SR1 metric update (Algorithm 4.2) and the warm-started dual field.
 * info (host) may be NULL. */
int mqnpm_step(mqnpm_handle* h, float* x, mqnpm_step_info* info);

/* mqnpm_step in two halves, for callers that form the subset gradient
 * themselves, e.g. with its illuminations split over several GPUs and the
 * partial sums added by an all-reduce (Eq. 4.1: grad F_s = (S/L) sum over the
 * illuminations of S_s).
 * mqnpm_step_subset: the subset iteration k+1 will use (Algorithm 4.1 step 3:
 *   s = k for k <= S, else strategy I or II) in *subset (0-based, may be NULL)
 *   and its illuminations in illum (host, room for L ints, may be NULL);
 *   *count receives their number.  No device work, no state change.
 *   STATE if strategy II has run out of draws.
 * mqnpm_step_with_gradient: iteration k+1 with the caller's g = grad F_s(x)
 *   (device N floats, distinct from x) and loss = F_s(x): the SR1 update
 *   (Algorithm 4.2), quasi-Newton point and weighted proximal mapping exactly
 *   as in mqnpm_step, x updated in place.  info as mqnpm_step, with the
 *   Krylov counts 0.  NONFINITE for a non-finite loss. */
int mqnpm_step_subset(const mqnpm_handle* h, int* subset, int* illum, int* count);
int mqnpm_step_with_gradient(mqnpm_handle* h, float* x, const float* g, double loss, mqnpm_step_info* info);

/* Shared launches for several reconstructions of one grid (the request loop of
 * the serving configuration; no counterpart in the paper beyond Algorithm 4.1
 * run for each member).  A group holds count member handles with equal grid, h,
 * kb, green_kernel, tile, device, krylov_tol, krylov_maxit and
 * direct_launches, the LS model and the slice detector (else INVALID_ARG or
 * UNSUPPORTED); members keep their own L, subsets, measurements, metric
 * state, TV, box and warm-start fields, and stay usable on their own.  The
 * group allocates a shared Krylov workspace of max_slots slots (1..
 * MQNPM_MAX_BATCH, within hbm_budget_bytes when non-zero), concatenated
 * incident-field tables and measurements, and copies member 0's Green's
 * spectrum.  The group must be destroyed before its members.
 * mqnpm_group_step: iteration k+1 of Algorithm 4.1 for every member.  x:
 *   host array of count device pointers (each member's N-float iterate,
 *   in/out, distinct); info: host array of count, or NULL.  All subset
 *   gradients run as one batch of slots in chunks of max_slots (each Green's
 *   pass and BiCGSTAB iteration one launch over the slots of all members,
 *   each slot reading its own volume's contrast); then each member's SR1
 *   update, quasi-Newton point and weighted proximal mapping.  Runs on the
 *   group's stream, which becomes every member's stream.  NOT_CONVERGED as
 *   mqnpm_step (outputs written); STATE if a member has no measurements. */
typedef struct mqnpm_group mqnpm_group;
int mqnpm_group_create(mqnpm_handle* const* members, int count, int max_slots, size_t hbm_budget_bytes,
                       mqnpm_group** out);
void mqnpm_group_destroy(mqnpm_group* g);
int mqnpm_group_step(mqnpm_group* g, float* const* x, mqnpm_step_info* info);
int mqnpm_group_set_stream(mqnpm_group* g, void* stream);
size_t mqnpm_group_workspace_bytes(const mqnpm_group* g);
const char* mqnpm_group_last_error(const mqnpm_group* g);

/* alpha estimate for a subset: `iters` power steps on
 * scale * sum_{l in illum} Re(J_l^H J_l) with J_l the Born Jacobian at x = 0,
 * from the device start vector `start` (N floats); result in *alpha_out (host). */
int mqnpm_lipschitz(mqnpm_handle* h, const int* illum, int nb, double scale, const float* start,
                    int iters, double* alpha_out);

/* Convergence diagnostics of Section 6 (off the hot path: one full and one
 * subset gradient).  x_prev = x_{k-1}, x_cur = x_k (device N floats; x_cur may
 * be NULL), s_prime = the subset iteration k used (mqnpm_step_info.subset).
 * out (host, 3 doubles): out[0] = e_k^2 = ||(1/S) sum_{s != s'} (grad F_s(x_{k-1})
 * - g_s^k)||^2 with g_s^k = grad F_{s'}(x_{k-1}) (strategies I and II), computed
 * as ||grad F - grad F_{s'}||^2 with grad F = (1/L) sum_l grad f_l; out[1] =
 * ||x_k - x_{k-1}||^2 (0 without x_cur); out[2] = (1/L) sum_l f_l(x_{k-1}).
 * With warm_start the forward solves start from, and refresh, the stored
 * fields.  Requires mqnpm_set_measurements; NOT_CONVERGED as mqnpm_grad_batch. */
int mqnpm_diagnostics(mqnpm_handle* h, const float* x_prev, const float* x_cur, int s_prime, double* out);

/* Checkpoint of the outer-loop state (k, tau_s, rank flags, xbar_s, gbar_s,
 * u_s, dual field and, with warm_start, the stored forward fields).  With
 * buf == NULL, *size receives the byte count; else buf (host, *size bytes)
 * receives the state.  load restores it exactly; it rejects a state written
 * by a handle of another grid, S, L or warm_start. */
int mqnpm_save_state(mqnpm_handle* h, void* buf, size_t* size);
int mqnpm_load_state(mqnpm_handle* h, const void* buf, size_t size);

/* Opt-in tracing (no counterpart in the paper; it instruments the Green's
 * convolution of Section 6).  profile_begin records CUDA events around the five
 * transform passes of the next max_calls Green's applies on the handle's
 * stream; profile_end synchronises the stream, returns the summed device time
 * of each pass in pass_ms (host, 5 doubles: x-forward, y-forward,
 * z-forward*K_hat*z-inverse, y-inverse, x-inverse), the number of recorded
 * applies in *calls and the sum of their batch sizes in *slot_launches, and
 * stops recording.  Applies that touch one z-plane are not recorded: the
 * adjoint right-hand sides G^H S^T r (input on the detector plane) and the
 * first-Born data S G(x u_in) (only the detector plane kept). */
/* Phase trace of the last weighted proximal mapping: out (host, 2*cap
 * long longs) receives out[1] = start time (ns, GPU global timer) and, for
 * e = 1..*count, the pair (tag, time) stamped when the e-th grid barrier was
 * passed (tags: 1 Gram set-up, 2 unweighted x, 3 divergence and U^T d,
 * 4 Newton evaluation, 5 x after a rejected trial, 6 dual update, 99 end),
 * for at most 999 barriers.  With cap >= 1003, out[2000..2005] hold block 0's
 * accumulated times (ns) in the dual update, before the dual update, in the
 * Newton evaluation pass, in the Newton decision, in the divergence pass and
 * waiting in grid barriers. */
int mqnpm_prox_trace(mqnpm_handle* h, long long* out, int cap, int* count);

/* Number of CUDA kernels this handle has launched since creation. */
long long mqnpm_launch_count(const mqnpm_handle* h);

/* Guard bands (guard_bytes > 0): *corrupted receives the number of bands, of
 * the two around every workspace buffer, whose bytes are no longer 0xA5 (0 when
 * no kernel wrote outside its buffers; also 0 without guards).  Synchronises
 * the handle's stream.  mqnpm_debug_poke_guard overwrites one byte of band
 * `band` (0-based) so that a test can see the check fire; it returns
 * INVALID_ARG for a band that does not exist. */
int mqnpm_check_guards(mqnpm_handle* h, int* corrupted);
int mqnpm_debug_poke_guard(mqnpm_handle* h, int band);

/* Launch shapes the handle uses: *tile (0..31); shape (6 ints) receives the
 * lines per CTA and threads per line of the x passes, then the columns per CTA
 * and threads per column of the y passes and of the z pass; ms (32 doubles,
 * may be NULL) receives the autotuner's time of one Green's apply per tile,
 * -1 where none was taken (a fixed tile, or one whose shared memory does not
 * fit).  Returns MQNPM_OK or INVALID_ARG. */
int mqnpm_tile_info(const mqnpm_handle* h, int* tile, int* shape, double* ms);

int mqnpm_profile_begin(mqnpm_handle* h, int max_calls);
int mqnpm_profile_end(mqnpm_handle* h, double* pass_ms, long long* slot_launches, int* calls);

/* Allocation-free Green's convolution.  The paper has no counterpart: this is
 * a library service, computing for one volume and without a handle the same
 * G v / G^H v as mqnpm_green_apply.  It is for callers that cannot allocate
 * device memory: code running inside another framework's memory pool or on a
 * device whose memory is already handed out, and allocator hooks that must not
 * re-enter the allocator.  It calls no cudaMalloc/cudaFree and no allocating
 * library routine; its scratch is one file-scope device array of
 * mqnpm_noalloc_scratch_bytes() bytes (3,013,376 B, 2.9 MiB), present on every GPU
 * that loads the library until the process exits.
 *   n: grid edge, at most 32, with 2n a compiled transform length
 *      (n in {8, 12, 16, 24, 32}); larger or unsupported n returns
 *      MQNPM_ERR_INVALID_ARG and prints why on stderr.
 *   h, kb: voxel size and background wavenumber (> 0).
 *   v, out: device, n^3 complex64 each ([z][y][x], interleaved re/im), distinct.
 *   adjoint != 0 selects G^H.  stream: cudaStream_t (NULL: legacy stream).
 * Works on the current device.  Set-up: the first call on a device (and the
 * first in a new context of that device, e.g. after cudaDeviceReset) takes the
 * array's device address with cudaGetSymbolAddress, with the device current;
 * that call, and the first after n, h or kb changed, also builds the kernel
 * spectrum in the array and synchronises the stream, so make it before any
 * stream capture.  Every call synchronises the stream before it returns (it
 * reads the device error flag, which must start at zero and is reset when
 * raised).  All calls on one device share the array, which keeps the last
 * call's spectrum; calls whose GPU work overlapped would race on it.  This
 * entry point keeps its own calls apart: each holds a process-wide lock from
 * its set-up to its final synchronisation.
 * Returns MQNPM_OK, MQNPM_ERR_INVALID_ARG, MQNPM_ERR_CUDA or MQNPM_ERR_TIMEOUT
 * (a bounded wait for a tile load gave up). */
int mqnpm_green_apply_noalloc(int n, double h, double kb, const float* v, float* out, int adjoint,
                              void* stream);
size_t mqnpm_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* MQNPM_H */
