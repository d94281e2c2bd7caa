// Prologues (pass 1) and epilogues (pass 5) fused into the Green's apply.
// Each reads/writes the BiCGSTAB vectors of slot b at voxel (x, y, z) and may
// accumulate per-thread FP32 partial sums (reduced per CTA in FP64).
#pragma once
#include "green_passes.cuh"

struct Geo {
  int nx, ny, nz;
  MQ_D size_t vox(int b, int x, int y, int z) const {
    return (((size_t)b * nz + z) * ny + y) * nx + x;
  }
  MQ_D size_t vox0(int x, int y, int z) const { return ((size_t)z * ny + y) * nx + x; }
};

// u_in(l, x, y, z) = ex[x] * ey[y] * ez[z] from FP64-built axis tables
// [l][nx + ny + nz].
MQ_D float2 incident(const float2* tab, int l, const Geo& g, int x, int y, int z) {
  const float2* t = tab + (size_t)l * (g.nx + g.ny + g.nz);
  return cmul(cmul(t[x], t[g.nx + y]), t[g.nx + g.ny + z]);
}

template <int KIND>
struct Pro;

template <>
struct Pro<PRO_PLAIN> {
  static constexpr int NPART = 0;
  ProArgs a;
  Geo g;
  MQ_D void begin(int) {}
  template <class Pt>
  MQ_D float2 load(int b, int x, int y, int z, Pt&) const { return a.q[g.vox(b, x, y, z)]; }
};

// Contrast of slot b: the shared one, or the slot's own (several volumes in one launch).
MQ_D const float* slot_contrast(const ProArgs& a, int b) { return a.xs ? a.xs[b] : a.x; }

template <>
struct Pro<PRO_CONTRAST> {
  static constexpr int NPART = 0;
  ProArgs a;
  Geo g;
  const float* xb;
  MQ_D void begin(int b) { xb = slot_contrast(a, b); }
  template <class Pt>
  MQ_D float2 load(int b, int x, int y, int z, Pt&) const {
    return cscale(a.q[g.vox(b, x, y, z)], xb[g.vox0(x, y, z)]);
  }
};

template <>
struct Pro<PRO_BORN> {
  static constexpr int NPART = 0;
  ProArgs a;
  Geo g;
  const float* xb;
  MQ_D void begin(int b) { xb = slot_contrast(a, b); }
  template <class Pt>
  MQ_D float2 load(int b, int x, int y, int z, Pt&) const {
    return cscale(incident(a.tab, a.illum[b], g, x, y, z), xb[g.vox0(x, y, z)]);
  }
};

template <>
struct Pro<PRO_BICG_P> {
  static constexpr int NPART = 0;
  ProArgs a;
  Geo g;
  const KState* st;
  float2 beta, omega;   // slot scalars, rounded once per thread by begin()
  bool first;
  const float* xb;
  MQ_D void begin(int b) {
    xb = slot_contrast(a, b);
    first = st[b].iters == 0;
    beta = make_float2((float)st[b].beta_re, (float)st[b].beta_im);
    omega = make_float2((float)st[b].omega_re, (float)st[b].omega_im);
  }
  template <class Pt>
  MQ_D float2 load(int b, int x, int y, int z, Pt&) const {
    const size_t i = g.vox(b, x, y, z);
    float2 pn = a.r[i];                                         // first iteration: p_1 = r_0
    if (!first) {
      const float2 pv = csub(a.w[i], cmul(omega, a.v[i]));     // p - omega v
      pn = caxpy(beta, pv, pn);                                 // r + beta (p - omega v)
    }
    a.w[i] = pn;
    return cscale(pn, xb[g.vox0(x, y, z)]);
  }
};

template <>
struct Pro<PRO_BICG_S> {
  static constexpr int NPART = 1;
  ProArgs a;
  Geo g;
  const KState* st;
  float2 alpha;         // slot scalar, rounded once per thread by begin()
  const float* xb;
  MQ_D void begin(int b) {
    xb = slot_contrast(a, b);
    alpha = make_float2((float)st[b].alpha_re, (float)st[b].alpha_im);
  }
  template <class Pt>
  MQ_D float2 load(int b, int x, int y, int z, Pt& parts) const {
    const size_t i = g.vox(b, x, y, z);
    const float2 s = caxpy(make_float2(-alpha.x, -alpha.y), a.v[i], a.r[i]);   // r - alpha v
    a.w[i] = s;
    parts.v[0] += cabs2(s);
    return cscale(s, xb[g.vox0(x, y, z)]);
  }
};

template <>
struct Pro<PRO_LIFT> {
  static constexpr int NPART = 0;
  ProArgs a;
  Geo g;
  MQ_D void begin(int) {}
  template <class Pt>
  MQ_D float2 load(int b, int x, int y, int z, Pt&) const {
    if (z != g.nz - 1) return make_float2(0.f, 0.f);
    return a.rdet[((size_t)b * g.ny + y) * g.nx + x];
  }
};

template <int KIND>
struct Epi;

template <>
struct Epi<EPI_PLAIN> {
  static constexpr int NPART = 0;
  EpiArgs a;
  Geo g;
  template <class Pt>
  MQ_D void store(int b, int x, int y, int z, float2 v, Pt&) const { a.out[g.vox(b, x, y, z)] = v; }
};

template <>
struct Epi<EPI_V> {
  static constexpr int NPART = 2;
  EpiArgs a;
  Geo g;
  template <class Pt>
  MQ_D void store(int b, int x, int y, int z, float2 gv, Pt& parts) const {
    const size_t i = g.vox(b, x, y, z);
    const float2 v = csub(a.a[i], gv);          // A p = p - G(x p)
    a.out[i] = v;
    const float2 d = cmulc(a.rhat[i], v);       // conj(rhat) v
    parts.v[0] += d.x;
    parts.v[1] += d.y;
  }
};

template <>
struct Epi<EPI_T> {
  static constexpr int NPART = 3;
  EpiArgs a;
  Geo g;
  template <class Pt>
  MQ_D void store(int b, int x, int y, int z, float2 gv, Pt& parts) const {
    const size_t i = g.vox(b, x, y, z);
    const float2 s = a.a[i];
    const float2 t = csub(s, gv);               // A s = s - G(x s)
    a.out[i] = t;
    const float2 d = cmulc(t, s);               // conj(t) s
    parts.v[0] += d.x;
    parts.v[1] += d.y;
    parts.v[2] += cabs2(t);
  }
};

template <>
struct Epi<EPI_INIT> {
  static constexpr int NPART = 1;
  EpiArgs a;
  Geo g;
  template <class Pt>
  MQ_D void store(int b, int x, int y, int z, float2 gv, Pt& parts) const {
    const size_t i = g.vox(b, x, y, z);
    a.out[i] = gv;
    a.out2[i] = gv;
    parts.v[0] += cabs2(gv);
  }
};

// Residual of a start u: r_0 = u_in - (I - G X) u = u_in - u + G(x u).
template <>
struct Epi<EPI_INIT_WARM> {
  static constexpr int NPART = 1;
  EpiArgs a;
  Geo g;
  template <class Pt>
  MQ_D void store(int b, int x, int y, int z, float2 gv, Pt& parts) const {
    const size_t i = g.vox(b, x, y, z);
    const float2 r = cadd(csub(incident(a.tab, a.illum[b], g, x, y, z), a.a[i]), gv);
    a.out[i] = r;
    a.out2[i] = r;
    parts.v[0] += cabs2(r);
  }
};

template <>
struct Epi<EPI_DETECT> {
  static constexpr int NPART = 1;
  EpiArgs a;
  Geo g;
  template <class Pt>
  MQ_D void store(int b, int x, int y, int z, float2 gv, Pt& parts) const {
    if (z != g.nz - 1) return;
    const size_t M = (size_t)g.nx * g.ny;
    const size_t j = (size_t)y * g.nx + x;
    const float2 r = a.ymeas ? csub(gv, a.ymeas[(size_t)a.illum[b] * M + j]) : gv;
    a.out2[b * M + j] = r;
    parts.v[0] += cabs2(r);
  }
};
