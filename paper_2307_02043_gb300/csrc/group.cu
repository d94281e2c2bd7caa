// Shared launches for several reconstructions on one grid.
//
// Independent volumes served together (the request loop of the serving
// configuration) run their subset gradients as one batch of slots: every
// Green's apply pass and every BiCGSTAB iteration of the group is one launch
// over the slots of all members, each slot reading its own volume's contrast
// (a per-slot pointer table), its own illumination (an index into tables
// that concatenate the members') and its own stored field.  The gradients add
// per member (one segment of consecutive slots each).  The SR1 update,
// quasi-Newton point and weighted proximal mapping of each member then run in
// turn on the member's own state (Algorithms 4.1-4.2, Eq. 4.5).
//
// The group owns an internal handle ("engine") that holds the shared Krylov
// workspace of max_slots slots, the concatenated incident-field tables and
// measurements, and a copy of member 0's Green's spectrum (copied at create,
// not built again).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "mqnpm.h"

struct mqnpm_group {
  mqnpm_handle* engine = nullptr;
  std::vector<mqnpm_handle*> members;
  std::vector<int> offset;   // first concatenated illumination of each member
  std::string err;
};

namespace {

int group_error(mqnpm_group* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  return code;
}

}  // namespace

extern "C" {

const char* mqnpm_group_last_error(const mqnpm_group* g) {
  if (!g) return "null group";
  if (!g->err.empty()) return g->err.c_str();
  return g->engine ? mqnpm_last_error(g->engine) : "";
}

void mqnpm_group_destroy(mqnpm_group* g) {
  if (!g) return;
  mqnpm_destroy(g->engine);
  delete g;
}

int mqnpm_group_create(mqnpm_handle* const* members, int count, int max_slots, size_t hbm_budget_bytes,
                       mqnpm_group** out) {
  if (!out) return MQNPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!members || count < 1 || max_slots < 1 || max_slots > MQNPM_MAX_BATCH) return MQNPM_ERR_INVALID_ARG;
  const mqnpm_handle* m0 = members[0];
  if (!m0) return MQNPM_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const mqnpm_handle* m = members[i];
    if (!m) return MQNPM_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (members[j] == m) return MQNPM_ERR_INVALID_ARG;   // a member once
    if (m->nx != m0->nx || m->ny != m0->ny || m->nz != m0->nz || m->h != m0->h || m->kb != m0->kb || m->device != m0->device || m->tile != m0->tile ||
        m->green_kernel != m0->green_kernel || m->krylov_tol != m0->krylov_tol ||
        m->krylov_maxit != m0->krylov_maxit || m->direct_launches != m0->direct_launches ||
        m->adjoint_from_b != m0->adjoint_from_b || m->forward_refine_steps != m0->forward_refine_steps)
      return MQNPM_ERR_INVALID_ARG;
    if (m->model != MQNPM_MODEL_LS || m->remote) return MQNPM_ERR_UNSUPPORTED;
  }
  mqnpm_group* g = new mqnpm_group();
  g->members.assign(members, members + count);
  std::vector<double> kdir;
  int L = 0;
  for (mqnpm_handle* m : g->members) {
    g->offset.push_back(L);
    L += m->L;
    kdir.insert(kdir.end(), m->kdir.begin(), m->kdir.end());
  }
  std::vector<int> subset_of(L, 0);
  const double alpha = 1.0;
  mqnpm_config c;
  std::memset(&c, 0, sizeof c);
  c.nx = m0->nx;
  c.ny = m0->ny;
  c.nz = m0->nz;
  c.h = m0->h;
  c.kb = m0->kb;
  c.model = MQNPM_MODEL_LS;
  c.L = L;
  c.kdir = kdir.data();
  c.S = 1;
  c.subset_of = subset_of.data();
  c.alpha = &alpha;
  c.step = 1.0;
  c.strategy = 1;
  c.tv = MQNPM_TV_ISO;
  c.lambda = 0.0;
  c.box_lo = 0.0;
  c.box_hi = 1.0;
  c.gamma = 1.0;
  c.krylov_tol = m0->krylov_tol;
  c.krylov_maxit = m0->krylov_maxit;
  c.dual_iters = 0;
  c.max_batch = max_slots;
  c.hbm_budget_bytes = hbm_budget_bytes;
  c.device = m0->device;
  c.stream = m0->stream;
  c.direct_launches = m0->direct_launches ? 1 : 0;
  c.tile = m0->tile;
  c.green_kernel = m0->green_kernel;
  c.adjoint_start = m0->adjoint_from_b ? 0 : 1;
  c.forward_start = m0->forward_refine_steps > 0 ? 0 : 1;
  // the engine takes the members' spectrum (it may come from a caller's green_hat)
  int rc = create_handle(&c, m0->khat, &g->engine);
  if (rc != MQNPM_OK) {
    delete g;
    return rc;
  }
  *out = g;
  return MQNPM_OK;
}

int mqnpm_group_set_stream(mqnpm_group* g, void* stream) {
  if (!g) return MQNPM_ERR_INVALID_ARG;
  mqnpm_set_stream(g->engine, stream);
  for (mqnpm_handle* m : g->members) mqnpm_set_stream(m, stream);
  return MQNPM_OK;
}

size_t mqnpm_group_workspace_bytes(const mqnpm_group* g) { return g ? mqnpm_workspace_bytes(g->engine) : 0; }

int mqnpm_group_step(mqnpm_group* g, float* const* x, mqnpm_step_info* info) {
  if (!g || !x) return MQNPM_ERR_INVALID_ARG;
  mqnpm_handle* E = g->engine;
  const int count = (int)g->members.size();
  for (int i = 0; i < count; ++i) {
    if (!x[i]) return group_error(g, MQNPM_ERR_INVALID_ARG, "group_step: null iterate");
    if (!g->members[i]->have_meas) return group_error(g, MQNPM_ERR_STATE, "group_step: measurements not set");
  }
  g->err.clear();
  cudaError_t e = cudaSetDevice(E->device);
  if (e != cudaSuccess) return set_cuda_error(E, e, "cudaSetDevice");
  cudaStream_t s = E->stream;
  const size_t N = E->N, M = (size_t)E->M;
  // the subset of each member's next iteration, and the slots in member order
  std::vector<int> k(count), sel(count);
  struct Slot { int member, l; };
  std::vector<Slot> slots;
  for (int i = 0; i < count; ++i) {
    mqnpm_handle* m = g->members[i];
    m->stream = s;
    k[i] = m->k + 1;
    int rc = select_subset(m, k[i], &sel[i]);
    if (rc != MQNPM_OK) return group_error(g, rc, "group_step: member " + std::to_string(i) + ": " + m->err);
    for (int l : m->subsets[sel[i]]) slots.push_back({i, l});
    if ((rc = step_events(m)) != MQNPM_OK) return rc;
    m->fields_valid = false;
  }
  // the members' current measurements, concatenated
  for (int i = 0; i < count; ++i) {
    mqnpm_handle* m = g->members[i];
    e = cudaMemcpyAsync(E->ymeas + (size_t)g->offset[i] * M, m->ymeas, (size_t)m->L * M * sizeof(float2),
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_cuda_error(E, e, "group measurements");
  }
  for (int i = 0; i < count; ++i) {
    e = cudaEventRecord(g->members[i]->step_ev[0], s);
    if (e != cudaSuccess) return set_cuda_error(E, e, "group events");
  }
  std::vector<double> loss(count, 0.0);
  std::vector<std::vector<int>> its(count);
  std::vector<char> started(count, 0);
  E->fields_valid = false;
  int worst = MQNPM_OK;
  const int total = (int)slots.size();
  for (int c0 = 0; c0 < total; c0 += E->max_batch) {
    const int cnt = std::min(E->max_batch, total - c0);
    ChunkTables t;
    t.m = cnt;
    bool warm_any = false, store_any = false;
    t.x.resize(cnt);
    t.warm.assign(cnt, nullptr);
    t.store.assign(cnt, nullptr);
    for (int b = 0; b < cnt; ++b) {
      const Slot& q = slots[c0 + b];
      mqnpm_handle* m = g->members[q.member];
      t.illum.push_back(g->offset[q.member] + q.l);
      t.x[b] = x[q.member];
      if (m->ufield) {
        t.store[b] = m->ufield + (size_t)q.l * N;
        t.warm[b] = m->have_field[q.l] ? t.store[b] : nullptr;
        store_any = true;
        warm_any = true;
      }
      if (b == 0 || slots[c0 + b - 1].member != q.member) {
        mqnpm_handle* mm = g->members[q.member];
        t.segs.push_back(GradSeg{b, b + 1, started[q.member] ? 1 : 0, (float)((double)mm->S / mm->L), mm->g});
        started[q.member] = 1;
      } else {
        t.segs.back().b1 = b + 1;
      }
    }
    int rc = stage_chunk(E, t);
    if (rc != MQNPM_OK) return rc;
    std::vector<int> it(2 * cnt, 0);
    rc = chunk_forward(E, nullptr, cnt, it.data(), E->w.rdet, E->ymeas, warm_any, store_any, t.segs);
    for (int b = 0; b < cnt; ++b) {
      const Slot& q = slots[c0 + b];
      mqnpm_handle* m = g->members[q.member];
      if (m->ufield) m->have_field[q.l] = (rc == MQNPM_ERR_NONFINITE) ? 0 : 1;
    }
    if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE || rc == MQNPM_ERR_UNSUPPORTED) return rc;
    if (rc != MQNPM_OK) worst = rc;
    rc = chunk_adjoint(E, nullptr, cnt, it.data(), (int)t.segs.size());
    if (rc == MQNPM_ERR_CUDA || rc == MQNPM_ERR_NONFINITE) return rc;
    if (rc != MQNPM_OK) worst = rc;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(E, e, "group gradient");
    for (size_t q = 0; q < t.segs.size(); ++q) {
      const int mi = slots[c0 + t.segs[q].b0].member;
      loss[mi] += 0.5 * E->w.h_scal[q];
    }
    for (int b = 0; b < cnt; ++b) {
      auto& v = its[slots[c0 + b].member];
      v.push_back(it[2 * b]);
      v.push_back(it[2 * b + 1]);
    }
  }
  int rc = check_tile_waits(E);
  if (rc != MQNPM_OK) return rc;
  for (int i = 0; i < count; ++i) {
    e = cudaEventRecord(g->members[i]->step_ev[1], s);
    if (e != cudaSuccess) return set_cuda_error(E, e, "group events");
  }
  for (int i = 0; i < count; ++i) {
    mqnpm_handle* m = g->members[i];
    const double scale = (double)m->S / m->L;
    m->last_iters = its[i];
    rc = finish_step(m, x[i], k[i], sel[i], scale * loss[i], its[i], worst, info ? info + i : nullptr);
    if (rc != MQNPM_OK && rc != MQNPM_ERR_NOT_CONVERGED)
      return group_error(g, rc, "group_step: member " + std::to_string(i) + ": " + m->err);
  }
  return worst;
}

}  // extern "C"
