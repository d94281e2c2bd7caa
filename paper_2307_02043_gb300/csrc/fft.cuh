// Radix-staged FFT building blocks for the padded Green's convolution.
//
// A length-P transform is split into two register stages, P = R1 * R2
// (four-step / Cooley-Tukey):
//   X[k1 + R1 k2] = sum_{n2} W_P^{n2 k1} W_{R2}^{n2 k2} sum_{n1} x[R2 n1 + n2] W_{R1}^{n1 k1}
// Stage 1: each "n2-thread" does a DFT of length R1 on x[R2 n1 + n2] and applies
// the twiddle W_P^{n2 k1}; shared memory exchanges the R1 x R2 block; stage 2:
// each "k1-thread" does a DFT of length R2.  The in-register DFTs are themselves
// composed recursively from radix-2/3/4/5 butterflies with twiddles folded into
// compile-time constants.
#pragma once
#include "common.cuh"

// Complex sum and difference as one two-lane FP32 instruction each
// (add/sub.rn.f32x2: the same round-to-nearest result per lane as two scalar
// operations), for the butterflies whose operands are whole complex values.
MQ_D float2 padd(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
MQ_D float2 psub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Multiply by W_R^J (forward, W = exp(-2 pi i / R)) or W_R^{-J} (inverse).
template <long J, long R, bool INV>
MQ_D float2 tw_mul(float2 a) {
  constexpr long j = ((J % R) + R) % R;
  if constexpr (j == 0) {
    return a;
  } else if constexpr (2 * j == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * j == R) {            // -i (fwd) / +i (inv)
    if constexpr (INV) return make_float2(-a.y, a.x);
    else return make_float2(a.y, -a.x);
  } else if constexpr (4 * j == 3 * R) {        // +i (fwd) / -i (inv)
    if constexpr (INV) return make_float2(a.y, -a.x);
    else return make_float2(-a.y, a.x);
  } else {
    constexpr ctrig::CS cs = ctrig::cs_turn(j, R);
    constexpr float c = static_cast<float>(cs.c);
    constexpr float s = INV ? static_cast<float>(cs.s) : -static_cast<float>(cs.s);
    return cmul(a, make_float2(c, s));
  }
}

constexpr int first_factor(int R) {
  return (R % 4 == 0 && R > 4) ? 4 : (R % 2 == 0 && R > 2) ? 2 : (R % 3 == 0 && R > 3) ? 3
                                                                                           : (R % 5 == 0 && R > 5) ? 5 : R;
}

// In-place DFT of length R on registers, natural order in and out.  NZ < R
// declares a[NZ..R) zero (the zero-padded half of a pruned transform): the
// butterflies that only add those zeros are left out.
template <int R, bool INV, int NZ = R>
MQ_D void dft(float2 (&a)[R]) {
  static_assert(NZ >= 1 && NZ <= R, "NZ in [1, R]");
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2 && NZ == 1) {
    a[1] = a[0];
  } else if constexpr (R == 2) {
    float2 t = a[0];
    a[0] = padd(t, a[1]);
    a[1] = psub(t, a[1]);
  } else if constexpr (R == 4 && NZ == 1) {
    a[1] = a[0];
    a[2] = a[0];
    a[3] = a[0];
  } else if constexpr (R == 4 && NZ == 2) {
    // inputs (a0, a1, 0, 0): y_k = a0 + W^k a1
    const float2 a0 = a[0], a1 = a[1];
    const float2 r = INV ? make_float2(-a1.y, a1.x) : make_float2(a1.y, -a1.x);   // -i a1 (fwd)
    a[0] = padd(a0, a1);
    a[2] = psub(a0, a1);
    a[1] = cadd(a0, r);
    a[3] = csub(a0, r);
  } else if constexpr (R == 3) {
    constexpr float h = 0.86602540378443864676f;   // sqrt(3)/2
    float2 s = cadd(a[1], a[2]);
    float2 d = csub(a[1], a[2]);
    float2 m = make_float2(fmaf(-0.5f, s.x, a[0].x), fmaf(-0.5f, s.y, a[0].y));
    // -i*h*d (fwd) ; +i*h*d (inv)
    float2 rot = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);
    a[0] = cadd(a[0], s);
    a[1] = cadd(m, rot);
    a[2] = csub(m, rot);
  } else if constexpr (R == 4) {
    float2 s02 = padd(a[0], a[2]), d02 = psub(a[0], a[2]);
    float2 s13 = padd(a[1], a[3]), d13 = psub(a[1], a[3]);
    // -i*d13 (fwd)
    float2 r = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
    a[0] = padd(s02, s13);
    a[2] = psub(s02, s13);
    a[1] = cadd(d02, r);
    a[3] = csub(d02, r);
  } else if constexpr (R == 5) {
    constexpr ctrig::CS w1 = ctrig::cs_turn(1, 5), w2 = ctrig::cs_turn(2, 5);
    constexpr float c1 = static_cast<float>(w1.c), s1 = static_cast<float>(w1.s);
    constexpr float c2 = static_cast<float>(w2.c), s2 = static_cast<float>(w2.s);
    float2 b1 = cadd(a[1], a[4]), d1 = csub(a[1], a[4]);
    float2 b2 = cadd(a[2], a[3]), d2 = csub(a[2], a[3]);
    float2 m1 = make_float2(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
    float2 m2 = make_float2(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
    float2 e1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);   // s1 d1 + s2 d2
    float2 e2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);   // s2 d1 - s1 d2
    // fwd: y1 = m1 - i e1, y4 = m1 + i e1, y2 = m2 - i e2, y3 = m2 + i e2
    float2 ie1 = make_float2(-e1.y, e1.x), ie2 = make_float2(-e2.y, e2.x);
    a[0] = make_float2(a[0].x + b1.x + b2.x, a[0].y + b1.y + b2.y);
    if constexpr (INV) {
      a[1] = cadd(m1, ie1); a[4] = csub(m1, ie1);
      a[2] = cadd(m2, ie2); a[3] = csub(m2, ie2);
    } else {
      a[1] = csub(m1, ie1); a[4] = cadd(m1, ie1);
      a[2] = csub(m2, ie2); a[3] = cadd(m2, ie2);
    }
  } else {
    constexpr int A = first_factor(R);
    constexpr int B = R / A;
    static_assert(A * B == R && A > 1 && B > 1, "unsupported DFT length");
    float2 y[R];  // y[n2 * A + k1]
    static_for<B>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      // nonzero inputs of this sub-transform: n1 with B n1 + n2 < NZ
      constexpr int NZT0 = (NZ - n2 + B - 1) / B;
      constexpr int NZT = NZT0 < 1 ? 1 : (NZT0 > A ? A : NZT0);
      float2 t[A];
      static_for<A>([&](auto n1c) { t[decltype(n1c)::value] = a[B * decltype(n1c)::value + n2]; });
      dft<A, INV, NZT>(t);
      static_for<A>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        y[n2 * A + k1] = tw_mul<(long)n2 * k1, R, INV>(t[k1]);
      });
    });
    static_for<A>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      float2 t[B];
      static_for<B>([&](auto n2c) { t[decltype(n2c)::value] = y[decltype(n2c)::value * A + k1]; });
      dft<B, INV>(t);
      static_for<B>([&](auto k2c) { a[k1 + A * decltype(k2c)::value] = t[decltype(k2c)::value]; });
    });
  }
}

// Two-stage plan for a transform length P = R1 * R2 processed by T threads per
// line/column (T divides R1 and R2).
template <int P>
struct Plan;
template <> struct Plan<8>   { static constexpr int R1 = 4,  R2 = 2,  T = 2; };
template <> struct Plan<16>  { static constexpr int R1 = 4,  R2 = 4,  T = 4; };
template <> struct Plan<24>  { static constexpr int R1 = 6,  R2 = 4,  T = 2; };
template <> struct Plan<32>  { static constexpr int R1 = 8,  R2 = 4,  T = 4; };
template <> struct Plan<40>  { static constexpr int R1 = 10, R2 = 4,  T = 2; };
template <> struct Plan<48>  { static constexpr int R1 = 12, R2 = 4,  T = 4; };
template <> struct Plan<64>  { static constexpr int R1 = 8,  R2 = 8,  T = 8; };
template <> struct Plan<96>  { static constexpr int R1 = 12, R2 = 8,  T = 4; };
template <> struct Plan<128> { static constexpr int R1 = 16, R2 = 8,  T = 8; };
template <> struct Plan<192> { static constexpr int R1 = 16, R2 = 12, T = 4; };
template <> struct Plan<256> { static constexpr int R1 = 16, R2 = 16, T = 16; };
template <> struct Plan<320> { static constexpr int R1 = 20, R2 = 16, T = 4; };
template <> struct Plan<384> { static constexpr int R1 = 24, R2 = 16, T = 8; };
template <> struct Plan<512> { static constexpr int R1 = 32, R2 = 16, T = 16; };

// The transform lengths the library is built for (P = 2n).
#define MQNPM_FOR_EACH_P(X) X(8) X(16) X(24) X(32) X(40) X(48) X(64) X(96) X(128) X(192) X(256) X(320) X(384) X(512)
