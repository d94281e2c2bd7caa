// Launch-shape autotuner of the Green's apply.
//
// Each transform length has two shapes for the x passes, two for the y
// passes and two for the z pass (lines or columns per CTA and threads per
// line or column), two exchange schemes of the z pass (one or two
// shared-memory buffers), and on square planes of edge 64 or 128 the fused
// x/y passes: up to twenty tiles that run.  The tuner times a plain apply of
// min(max_batch, 8) slots for each tile on the handle's own buffers (zero
// input: the passes do the same work for any values), round-robin over two
// rounds after one warm-up round so that clock ramp-up does not favour a late
// candidate, and keeps the tile with the smallest best time.  The choice is
// cached per (device, grid, slots) for the life of the process, so handles of
// the same shape are not re-timed.  Tiles whose shared memory does not fit
// are skipped.
#include <array>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"
#include "mqnpm.h"

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int, int, int>, std::array<double, MQ_TILES>> g_cache;

// Fastest timed tile; tiles whose shared memory does not fit carry -1.
int pick(const std::array<double, MQ_TILES>& ms) {
  int best = 0;
  for (int t = 1; t < MQ_TILES; ++t)
    if (ms[t] >= 0 && (ms[best] < 0 || ms[t] < ms[best])) best = t;
  return best;
}
}  // namespace

int autotune_tile(mqnpm_handle* h) {
  Workspace& w = h->w;
  const int nb = h->max_batch < 8 ? h->max_batch : 8;
  const auto key = std::make_tuple(h->device, h->nx, h->ny, h->nz, nb);
  std::array<double, MQ_TILES> ms{};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      ms = it->second;
      cached = true;
    }
  }
  cudaStream_t s = h->stream;
  cudaError_t e;
  if (!cached) {
    if ((e = cudaMemsetAsync(w.u, 0, (size_t)nb * h->N * sizeof(float2), s)) != cudaSuccess)
      return set_cuda_error(h, e, "autotune: input");
    GreenCall c;
    c.nx = h->nx;
    c.ny = h->ny;
    c.nz = h->nz;
    c.nb = nb;
    c.pro = PRO_PLAIN;
    c.pa.q = w.u;
    c.epi = EPI_PLAIN;
    c.ea.out = w.r;
    c.T1 = w.T1;
    c.T2 = w.T2;
    c.khat = h->khat;
    c.twx = h->twx;
    c.twy = h->twy;
    c.twz = h->twz;
    c.part_pro = w.part1;
    c.part_epi = w.part5;
    c.launches = &h->launches;
    c.err = w.gerr;
    alignas(64) unsigned char maps[MQ_TILES][128];
    bool fits[MQ_TILES];
    for (int t = 0; t < MQ_TILES; ++t) fits[t] = green_tile_fits(h->nx, h->ny, h->nz, t, h->device);
    for (int t = 0; t < MQ_TILES; ++t)
      if (fits[t] && (e = make_t2_tensor_map(w.T2, h->nx, h->ny, h->nz, h->max_batch, t, maps[t])) != cudaSuccess)
        return set_cuda_error(h, e, "autotune: tensor map");
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return set_cuda_error(h, e, "autotune: event");
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
      cudaEventDestroy(ev[0]);
      return set_cuda_error(h, e, "autotune: event");
    }
    ms.fill(1e30);
    for (int round = 0; round < 3 && e == cudaSuccess; ++round)
      for (int t = 0; t < MQ_TILES && e == cudaSuccess; ++t) {
        if (!fits[t]) continue;
        c.tile = t;
        c.tmap = maps[t];
        if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess) break;
        if ((e = green_launch(c, s)) != cudaSuccess) {
          // a fused-pass tile that cannot be launched here (no co-resident CTA
          // pair, a launch configuration the device refuses) drops out; any
          // other failure ends the tuning
          if ((t & MQ_TILE_FUSED) && round == 0 &&
              (e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidConfiguration ||
               e == cudaErrorNotSupported || e == cudaErrorInvalidValue)) {
            (void)cudaGetLastError();
            fits[t] = false;
            e = cudaSuccess;
            continue;
          }
          break;
        }
        if ((e = cudaEventRecord(ev[1], s)) != cudaSuccess || (e = cudaEventSynchronize(ev[1])) != cudaSuccess)
          break;
        float t_ms = 0.f;
        if ((e = cudaEventElapsedTime(&t_ms, ev[0], ev[1])) != cudaSuccess) break;
        if (round > 0 && (double)t_ms < ms[t]) ms[t] = t_ms;   // round 0 warms up (module load, clocks)
      }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return set_cuda_error(h, e, "autotune: timed apply");
    int gerr = 0;
    if ((e = cudaMemcpyAsync(&gerr, w.gerr, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return set_cuda_error(h, e, "autotune: error flag");
    if (gerr) return set_error(h, MQNPM_ERR_TIMEOUT, "autotune: a bounded wait for a tile load gave up");
    for (int t = 0; t < MQ_TILES; ++t)
      if (!fits[t]) ms[t] = -1.0;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = ms;
  }
  for (int t = 0; t < MQ_TILES; ++t) h->tune_ms[t] = ms[t];
  h->tile = pick(ms);
  if ((e = make_t2_tensor_map(w.T2, h->nx, h->ny, h->nz, h->max_batch, h->tile, w.t2map)) != cudaSuccess)
    return set_cuda_error(h, e, "autotune: tensor map");
  return MQNPM_OK;
}
