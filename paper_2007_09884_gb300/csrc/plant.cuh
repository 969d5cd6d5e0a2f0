// plant.cuh -- device-side oculomotor plant for the 18-parameter OPMM.
//
// Model (paper Sec. 2.1 and Sec. 2.2.1, Table 1; the paper names the
// components, this is the linear six-state reading used throughout):
//   state (theta, omega, x, y, Fa, Fn) in the saccade's positive frame
//   Ta = K_SE_AG (x - theta), Tn = K_SE_ANT (y + theta), K_P = N_C_AG + N_C_ANT
//   theta' = omega
//   J omega' = Ta - Tn - B_P omega - K_P theta
//   B_AG x'  = Fa - Ta - K_LT_AG x
//   B_ANT y' = Fn - Tn - K_LT_ANT y
//   tau Fa' = Na - Fa,  tau Fn' = Nn - Fn   (pulse-step drive, Sec. 2.1)
//
// Integration: classical RK4 with h = 1 / (fs * nsub), nsub = round(1e4 / fs)
// (h ~ 0.1 ms); the substep holding the pulse end is split into two RK4 steps.
//
// GB300 formulation.  Within one input phase the plant is linear and
// time-invariant, so one RK4 step is exactly the affine map
//     s <- s* + (I + Q)(s - s*),   Q = T4(hA) - I = hA(I + hA/2(I + hA/3(I + hA/4)))
// around the phase equilibrium s*.  Q is built once per candidate in
// "increment form" (no leading identity, so slow modes keep full relative
// precision) and raised to the nsub-th power by squaring, giving one 6x6
// update per recorded sample instead of nsub x 4 derivative evaluations.  The
// matrix is block upper triangular: a 4x4 mechanical block shared by both
// phases, a 4x2 coupling and a diagonal activation block per phase.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace opmm {

// OPC vector layout: the column order of the paper's example output (Fig. 4).
enum : int {
  kSeAg = 0, kSeAnt, kLtAg, kLtAnt, kNcAg, kNcAnt, kBp, kBAg, kBAnt, kJ,
  kTacAg, kTacAnt, kTdeAg, kTdeAnt, kNcFix, kNsacAg, kNsacAnt, kPw, kNumParams
};

// Per-saccade constants in the positive (mirrored) frame.
struct SacConst {
  int L;          // samples in the window
  int onset;      // onset sample (pulse starts at onset / fs)
  int nsub;       // RK4 substeps per sample
  float fs;       // sample rate, Hz
  float h;        // RK4 step, s
  float th0;      // start fixation (th0 <= thf)
  float thf;      // end fixation
};

// Continuous-time coefficients (A matrix entries) of one candidate.
struct Coef {
  float m10, m11, m12, m13;   // omega row: theta, omega, x, y
  float m20, m22, cx;         // x row: theta, x, Fa
  float m30, m33, cy;         // y row: theta, y, Fn
  float da1, dn1;             // -1/tau of Fa, Fn during the pulse
  float da2, dn2;             // -1/tau of Fa, Fn after the pulse
  float iKa, iKn;             // 1/K_SE_AG, 1/K_SE_ANT (equilibria)
};

// Increment-form propagator of both phases: the 4x4 mechanical block m is
// shared; c1/d1 (pulse) and c2/d2 (step) are the coupling and activation
// blocks.  (I + P) acting on a phase-k deviation vector e:
//   e_m <- e_m + m e_m + ck e_f,   e_f <- e_f + dk .* e_f
struct Prop2 {
  float m[4][4];
  float c1[4][2], c2[4][2];
  float d1[2], d2[2];
};

// The reciprocals and quotients of the set-up use the fast single-precision
// division (__fdividef, within 2 ulp): it changes a coefficient by far less
// than the trajectory tolerance and saves the IEEE division sequences.
__device__ __forceinline__ void make_coef(const float* p, Coef& k) {
  const float iJ = __fdividef(1.0f, p[kJ]);
  const float iBa = __fdividef(1.0f, p[kBAg]);
  const float iBn = __fdividef(1.0f, p[kBAnt]);
  const float kp = p[kNcAg] + p[kNcAnt];
  k.m10 = -(p[kSeAg] + p[kSeAnt] + kp) * iJ;
  k.m11 = -p[kBp] * iJ;
  k.m12 = p[kSeAg] * iJ;
  k.m13 = -p[kSeAnt] * iJ;
  k.m20 = p[kSeAg] * iBa;
  k.m22 = -(p[kSeAg] + p[kLtAg]) * iBa;
  k.cx = iBa;
  k.m30 = -p[kSeAnt] * iBn;
  k.m33 = -(p[kSeAnt] + p[kLtAnt]) * iBn;
  k.cy = iBn;
  // activation/deactivation times are in ms (Table 1)
  k.da1 = __fdividef(-1000.0f, p[kTacAg]);
  k.dn1 = __fdividef(-1000.0f, p[kTdeAnt]);
  k.da2 = __fdividef(-1000.0f, p[kTdeAg]);
  k.dn2 = __fdividef(-1000.0f, p[kTacAnt]);
  k.iKa = __fdividef(1.0f, p[kSeAg]);
  k.iKn = __fdividef(1.0f, p[kSeAnt]);
}

// Substep refinement for stiff candidates.  RK4 is stable on the negative
// real axis up to |h lambda| ~ 2.78; the size of the fastest mode is estimated
// from the coefficients (no divisions) as est = B_P/J + (K_SE_AG + K_LT_AG)/B_AG
// + (K_SE_ANT + K_LT_ANT)/B_ANT + 1/tau_min.  The base step h (~0.1 ms) is
// halved until h est <= 2.5, at most kMaxRefine times; returns the number of
// halvings, or -1 when even the finest step is too large (the candidate then
// scores +inf).
constexpr int kMaxRefine = 6;

__device__ __forceinline__ int refine_shift(const Coef& k, float h) {
  const float rate = fmaxf(fmaxf(-k.da1, -k.dn1), fmaxf(-k.da2, -k.dn2));
  const float est = -(k.m11 + k.m22 + k.m33) + rate;
  int s = 0;
  while (s < kMaxRefine && !(h * est <= 2.5f)) {
    h *= 0.5f;
    ++s;
  }
  return h * est <= 2.5f ? s : -1;
}

// 2^-s for 0 <= s <= kMaxRefine, exactly (built from the exponent bits).
__device__ __forceinline__ float pow2neg(int s) { return __int_as_float((127 - s) << 23); }

// Saccade constants with the substep refined s times (h / 2^s, nsub 2^s).
__device__ __forceinline__ SacConst refined(const SacConst& sc, int s) {
  SacConst r = sc;
  r.nsub = sc.nsub << s;
  r.h = sc.h * pow2neg(s);
  return r;
}

// Rest state at fixation th with precomputed 1/K_SE.
__device__ __forceinline__ void rest_state_k(const float* p, const Coef& k, float th, float* s) {
  const float ta = fmaf(p[kNcAg], th, p[kNcFix]), tn = fmaf(-p[kNcAnt], th, p[kNcFix]);
  s[0] = th;
  s[1] = 0.0f;
  s[2] = fmaf(ta, k.iKa, th);
  s[3] = fmaf(tn, k.iKn, -th);
  s[4] = fmaf(ta, fmaf(p[kLtAg], k.iKa, 1.0f), p[kLtAg] * th);
  s[5] = fmaf(tn, fmaf(p[kLtAnt], k.iKn, 1.0f), -p[kLtAnt] * th);
}

// Equilibrium under constant active-state tensions, precomputed 1/K_SE.
__device__ __forceinline__ void drive_equilibrium_k(const float* p, const Coef& k, float fa, float fn, float* s) {
  const float ag = __fdividef(1.0f, fmaf(p[kLtAg], k.iKa, 1.0f));     // K_SE / (K_SE + K_LT)
  const float an = __fdividef(1.0f, fmaf(p[kLtAnt], k.iKn, 1.0f));
  const float kp = p[kNcAg] + p[kNcAnt];
  const float th = __fdividef(ag * fa - an * fn, kp + ag * p[kLtAg] + an * p[kLtAnt]);
  const float ta = ag * (fa - p[kLtAg] * th);
  const float tn = an * (fn + p[kLtAnt] * th);
  s[0] = th;
  s[1] = 0.0f;
  s[2] = fmaf(ta, k.iKa, th);
  s[3] = fmaf(tn, k.iKn, -th);
  s[4] = fa;
  s[5] = fn;
}

// Tension held at fixation angle th (tension slope and intercept, Sec. 2.1).
__device__ __forceinline__ float ta_eq(const float* p, float th) { return fmaf(p[kNcAg], th, p[kNcFix]); }
__device__ __forceinline__ float tn_eq(const float* p, float th) { return fmaf(-p[kNcAnt], th, p[kNcFix]); }

// Rest state at fixation angle th.
__device__ __forceinline__ void rest_state(const float* p, float th, float* s) {
  const float ta = ta_eq(p, th), tn = tn_eq(p, th);
  s[0] = th;
  s[1] = 0.0f;
  s[2] = th + ta / p[kSeAg];
  s[3] = tn / p[kSeAnt] - th;
  s[4] = ta * (1.0f + p[kLtAg] / p[kSeAg]) + p[kLtAg] * th;
  s[5] = tn * (1.0f + p[kLtAnt] / p[kSeAnt]) - p[kLtAnt] * th;
}

// Equilibrium under constant active-state tensions (fa, fn): from x' = y' = 0
// the series tensions are Ta = a_g (fa - K_LT_AG th), Tn = a_n (fn + K_LT_ANT th)
// with a = K_SE / (K_SE + K_LT); the globe balance Ta - Tn = K_P th fixes th.
__device__ __forceinline__ void drive_equilibrium(const float* p, float fa, float fn, float* s) {
  const float ag = p[kSeAg] / (p[kSeAg] + p[kLtAg]);
  const float an = p[kSeAnt] / (p[kSeAnt] + p[kLtAnt]);
  const float kp = p[kNcAg] + p[kNcAnt];
  const float th = (ag * fa - an * fn) / (kp + ag * p[kLtAg] + an * p[kLtAnt]);
  const float ta = ag * (fa - p[kLtAg] * th);
  const float tn = an * (fn + p[kLtAnt] * th);
  s[0] = th;
  s[1] = 0.0f;
  s[2] = th + ta / p[kSeAg];
  s[3] = tn / p[kSeAnt] - th;
  s[4] = fa;
  s[5] = fn;
}

// out = Zm * w for the sparse mechanical block Zm = h * A_mech, w dense 4x4
// (or 4x2 via ncol).  z: {h, h m10, h m11, h m12, h m13, h m20, h m22, h m30, h m33}
struct ZMech {
  float h, m10, m11, m12, m13, m20, m22, m30, m33;
};

template <int NC>
__device__ __forceinline__ void zm_mul(const ZMech& z, const float (&w)[4][NC], float (&o)[4][NC]) {
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const float w0 = w[0][j], w1 = w[1][j], w2 = w[2][j], w3 = w[3][j];
    o[0][j] = z.h * w1;
    o[1][j] = fmaf(z.m13, w3, fmaf(z.m12, w2, fmaf(z.m11, w1, z.m10 * w0)));
    o[2][j] = fmaf(z.m22, w2, z.m20 * w0);
    o[3][j] = fmaf(z.m33, w3, z.m30 * w0);
  }
}

// Single-substep increment propagator Q = T4(hA) - I of both phases by Horner:
// W3 = I + Z/4, W2 = I + Z W3 / 3, W1 = I + Z W2 / 2, Q = Z W1, block by block.
// Every sum of a product is written as an explicit single-rounding FMA (or
// an explicit product), so step_increment_x2 can reproduce it bit for bit.
__device__ __forceinline__ void step_increment(const Coef& k, float h, Prop2& q) {
  ZMech z;
  z.h = h;
  z.m10 = h * k.m10; z.m11 = h * k.m11; z.m12 = h * k.m12; z.m13 = h * k.m13;
  z.m20 = h * k.m20; z.m22 = h * k.m22; z.m30 = h * k.m30; z.m33 = h * k.m33;
  const float zcx = h * k.cx, zcy = h * k.cy;
  // mechanical block
  float w[4][4], t[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = (i == j ? 1.0f : 0.0f);
  // W3 = I + Zm / 4
  zm_mul<4>(z, w, t);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = (i == j ? 1.0f : 0.0f) + 0.25f * t[i][j];
  // W2 = I + Zm W3 / 3
  zm_mul<4>(z, w, t);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = __fmaf_rn(t[i][j], 1.0f / 3.0f, i == j ? 1.0f : 0.0f);
  // W1 = I + Zm W2 / 2
  zm_mul<4>(z, w, t);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = (i == j ? 1.0f : 0.0f) + 0.5f * t[i][j];
  // Qm = Zm W1
  zm_mul<4>(z, w, q.m);
  // coupling and activation blocks, per phase
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const float zda = h * (ph == 0 ? k.da1 : k.da2);
    const float zdn = h * (ph == 0 ? k.dn1 : k.dn2);
    // level 3: Wc3 = Zc / 4, Wd3 = 1 + Zd / 4
    float wc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.25f * zcx, 0.f}, {0.f, 0.25f * zcy}};
    float wda = 1.0f + 0.25f * zda, wdn = 1.0f + 0.25f * zdn;
    float tc[4][2];
    // level 2: Wc2 = (Zm Wc3 + Zc Wd3) / 3, Wd2 = 1 + Zd Wd3 / 3
    zm_mul<2>(z, wc, tc);
    tc[2][0] = fmaf(zcx, wda, tc[2][0]);
    tc[3][1] = fmaf(zcy, wdn, tc[3][1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) { wc[i][0] = tc[i][0] * (1.0f / 3.0f); wc[i][1] = tc[i][1] * (1.0f / 3.0f); }
    wda = __fmaf_rn(__fmul_rn(zda, wda), 1.0f / 3.0f, 1.0f);
    wdn = __fmaf_rn(__fmul_rn(zdn, wdn), 1.0f / 3.0f, 1.0f);
    // level 1: Wc1 = (Zm Wc2 + Zc Wd2) / 2, Wd1 = 1 + Zd Wd2 / 2
    zm_mul<2>(z, wc, tc);
    tc[2][0] = fmaf(zcx, wda, tc[2][0]);
    tc[3][1] = fmaf(zcy, wdn, tc[3][1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) { wc[i][0] = 0.5f * tc[i][0]; wc[i][1] = 0.5f * tc[i][1]; }
    wda = __fmaf_rn(0.5f * zda, wda, 1.0f);
    wdn = __fmaf_rn(0.5f * zdn, wdn, 1.0f);
    // Q: Qc = Zm Wc1 + Zc Wd1, Qd = Zd Wd1
    zm_mul<2>(z, wc, tc);
    tc[2][0] = fmaf(zcx, wda, tc[2][0]);
    tc[3][1] = fmaf(zcy, wdn, tc[3][1]);
    if (ph == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) { q.c1[i][0] = tc[i][0]; q.c1[i][1] = tc[i][1]; }
      q.d1[0] = zda * wda; q.d1[1] = zdn * wdn;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) { q.c2[i][0] = tc[i][0]; q.c2[i][1] = tc[i][1]; }
      q.d2[0] = zda * wda; q.d2[1] = zdn * wdn;
    }
  }
}

// step_increment with two columns per packed FP32 instruction: the
// mechanical block by column pairs, the coupling block's two columns as one
// pair.  Every entry gets the operations step_increment gives it, in the same
// order and with the same single roundings, so the result is the same bit
// for bit.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }

// o = Zm w for one column pair (w, o: four rows of pairs)
__device__ __forceinline__ void zm_mul_x2(const float2 (&Z)[9], const float2 (&w)[4], float2 (&o)[4]) {
  // Z: h, m10, m11, m12, m13, m20, m22, m30, m33 broadcast
  o[0] = __fmul2_rn(Z[0], w[1]);
  o[1] = __ffma2_rn(Z[4], w[3], __ffma2_rn(Z[3], w[2], __ffma2_rn(Z[2], w[1], __fmul2_rn(Z[1], w[0]))));
  o[2] = __ffma2_rn(Z[6], w[2], __fmul2_rn(Z[5], w[0]));
  o[3] = __ffma2_rn(Z[8], w[3], __fmul2_rn(Z[7], w[0]));
}

__device__ __forceinline__ void step_increment_x2(const Coef& k, float h, Prop2& q) {
  const float2 Z[9] = {bc(h), bc(h * k.m10), bc(h * k.m11), bc(h * k.m12), bc(h * k.m13),
                       bc(h * k.m20), bc(h * k.m22), bc(h * k.m30), bc(h * k.m33)};
  const float zcx = h * k.cx, zcy = h * k.cy;
  // mechanical block, column pairs jp = 0 (columns 0, 1) and 1 (columns 2, 3)
#pragma unroll
  for (int jp = 0; jp < 2; ++jp) {
    float2 id[4], w[4], t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      id[i] = f2(i == 2 * jp ? 1.0f : 0.0f, i == 2 * jp + 1 ? 1.0f : 0.0f);
      w[i] = id[i];
    }
    zm_mul_x2(Z, w, t);
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = __fadd2_rn(id[i], __fmul2_rn(bc(0.25f), t[i]));
    zm_mul_x2(Z, w, t);
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = __ffma2_rn(t[i], bc(1.0f / 3.0f), id[i]);
    zm_mul_x2(Z, w, t);
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = __fadd2_rn(id[i], __fmul2_rn(bc(0.5f), t[i]));
    zm_mul_x2(Z, w, t);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      q.m[i][2 * jp] = t[i].x;
      q.m[i][2 * jp + 1] = t[i].y;
    }
  }
  // coupling and activation blocks, per phase; the pair is (column Fa, column Fn)
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const float zda = h * (ph == 0 ? k.da1 : k.da2);
    const float zdn = h * (ph == 0 ? k.dn1 : k.dn2);
    float2 wc[4] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.25f * zcx, 0.f), f2(0.f, 0.25f * zcy)};
    float wda = 1.0f + 0.25f * zda, wdn = 1.0f + 0.25f * zdn;
    float2 tc[4];
    zm_mul_x2(Z, wc, tc);
    tc[2].x = fmaf(zcx, wda, tc[2].x);
    tc[3].y = fmaf(zcy, wdn, tc[3].y);
#pragma unroll
    for (int i = 0; i < 4; ++i) wc[i] = __fmul2_rn(tc[i], bc(1.0f / 3.0f));
    wda = __fmaf_rn(__fmul_rn(zda, wda), 1.0f / 3.0f, 1.0f);
    wdn = __fmaf_rn(__fmul_rn(zdn, wdn), 1.0f / 3.0f, 1.0f);
    zm_mul_x2(Z, wc, tc);
    tc[2].x = fmaf(zcx, wda, tc[2].x);
    tc[3].y = fmaf(zcy, wdn, tc[3].y);
#pragma unroll
    for (int i = 0; i < 4; ++i) wc[i] = __fmul2_rn(bc(0.5f), tc[i]);
    wda = __fmaf_rn(0.5f * zda, wda, 1.0f);
    wdn = __fmaf_rn(0.5f * zdn, wdn, 1.0f);
    zm_mul_x2(Z, wc, tc);
    tc[2].x = fmaf(zcx, wda, tc[2].x);
    tc[3].y = fmaf(zcy, wdn, tc[3].y);
    float (&c)[4][2] = ph == 0 ? q.c1 : q.c2;
    float (&d)[2] = ph == 0 ? q.d1 : q.d2;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[i][0] = tc[i].x;
      c[i][1] = tc[i].y;
    }
    d[0] = zda * wda;
    d[1] = zdn * wdn;
  }
}

// r = a + b + a b  (increment form of (I + a)(I + b)); r may alias neither.
__device__ __forceinline__ void prop_mul(const Prop2& a, const Prop2& b, Prop2& r) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = a.m[i][j] + b.m[i][j];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc = fmaf(a.m[i][kk], b.m[kk][j], acc);
      r.m[i][j] = acc;
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      float acc1 = fmaf(a.c1[i][f], b.d1[f], a.c1[i][f] + b.c1[i][f]);
      float acc2 = fmaf(a.c2[i][f], b.d2[f], a.c2[i][f] + b.c2[i][f]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        acc1 = fmaf(a.m[i][kk], b.c1[kk][f], acc1);
        acc2 = fmaf(a.m[i][kk], b.c2[kk][f], acc2);
      }
      r.c1[i][f] = acc1;
      r.c2[i][f] = acc2;
    }
  }
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    r.d1[f] = fmaf(a.d1[f], b.d1[f], a.d1[f] + b.d1[f]);
    r.d2[f] = fmaf(a.d2[f], b.d2[f], a.d2[f] + b.d2[f]);
  }
}

// out = (I + q)^n - I by binary powering (n >= 1).
__device__ __forceinline__ void prop_pow(const Prop2& q, int n, Prop2& out) {
  Prop2 base = q, tmp;
  bool have = false;
  while (true) {
    if (n & 1) {
      if (have) { prop_mul(out, base, tmp); out = tmp; }
      else { out = base; have = true; }
    }
    n >>= 1;
    if (!n) break;
    prop_mul(base, base, tmp);
    base = tmp;
  }
}

// Single-phase increment propagator: the mechanical block plus one phase's
// coupling and activation blocks (26 floats).
struct Prop1 {
  float m[4][4];
  float c[4][2];
  float d[2];
};

// Single-substep increment propagator of one phase (PH = 1 pulse, 2 step),
// Horner form as step_increment.
template <int PH>
__device__ __forceinline__ void step_increment1(const Coef& k, float h, Prop1& q) {
  ZMech z;
  z.h = h;
  z.m10 = h * k.m10; z.m11 = h * k.m11; z.m12 = h * k.m12; z.m13 = h * k.m13;
  z.m20 = h * k.m20; z.m22 = h * k.m22; z.m30 = h * k.m30; z.m33 = h * k.m33;
  const float zcx = h * k.cx, zcy = h * k.cy;
  const float zda = h * (PH == 1 ? k.da1 : k.da2);
  const float zdn = h * (PH == 1 ? k.dn1 : k.dn2);
  float w[4][4], t[4][4];
  float wc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.25f * zcx, 0.f}, {0.f, 0.25f * zcy}};
  float tc[4][2];
  float wda = 1.0f + 0.25f * zda, wdn = 1.0f + 0.25f * zdn;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = (i == j ? 1.0f : 0.0f);
  zm_mul<4>(z, w, t);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[i][j] = (i == j ? 1.0f : 0.0f) + 0.25f * t[i][j];
#pragma unroll
  for (int lev = 3; lev >= 2; --lev) {
    const float inv = lev == 3 ? (1.0f / 3.0f) : 0.5f;
    zm_mul<4>(z, w, t);
    zm_mul<2>(z, wc, tc);
    tc[2][0] = fmaf(zcx, wda, tc[2][0]);
    tc[3][1] = fmaf(zcy, wdn, tc[3][1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) w[i][j] = (i == j ? 1.0f : 0.0f) + t[i][j] * inv;
      wc[i][0] = tc[i][0] * inv;
      wc[i][1] = tc[i][1] * inv;
    }
    wda = 1.0f + zda * wda * inv;
    wdn = 1.0f + zdn * wdn * inv;
  }
  zm_mul<4>(z, w, q.m);
  zm_mul<2>(z, wc, q.c);
  q.c[2][0] = fmaf(zcx, wda, q.c[2][0]);
  q.c[3][1] = fmaf(zcy, wdn, q.c[3][1]);
  q.d[0] = zda * wda;
  q.d[1] = zdn * wdn;
}

// r = a + b + a b for single-phase propagators.
__device__ __forceinline__ void prop1_mul(const Prop1& a, const Prop1& b, Prop1& r) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = a.m[i][j] + b.m[i][j];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc = fmaf(a.m[i][kk], b.m[kk][j], acc);
      r.m[i][j] = acc;
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      float acc = fmaf(a.c[i][f], b.d[f], a.c[i][f] + b.c[i][f]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc = fmaf(a.m[i][kk], b.c[kk][f], acc);
      r.c[i][f] = acc;
    }
  }
#pragma unroll
  for (int f = 0; f < 2; ++f) r.d[f] = fmaf(a.d[f], b.d[f], a.d[f] + b.d[f]);
}

__device__ __forceinline__ void prop1_pow(const Prop1& q, int n, Prop1& out) {
  Prop1 base = q, tmp;
  bool have = false;
  while (true) {
    if (n & 1) {
      if (have) { prop1_mul(out, base, tmp); out = tmp; }
      else { out = base; have = true; }
    }
    n >>= 1;
    if (!n) break;
    prop1_mul(base, base, tmp);
    base = tmp;
  }
}

__device__ __forceinline__ void prop1_apply(const Prop1& q, float (&e)[6]) {
  float n[6];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float a = fmaf(q.m[i][0], e[0], e[i]);
    a = fmaf(q.m[i][1], e[1], a);
    a = fmaf(q.m[i][2], e[2], a);
    float b = q.m[i][3] * e[3];
    b = fmaf(q.c[i][0], e[4], b);
    b = fmaf(q.c[i][1], e[5], b);
    n[i] = a + b;
  }
  n[4] = fmaf(q.d[0], e[4], e[4]);
  n[5] = fmaf(q.d[1], e[5], e[5]);
#pragma unroll
  for (int i = 0; i < 6; ++i) e[i] = n[i];
}

// e <- (I + P_phase) e for a phase-1 (PH = 1) or phase-2 (PH = 2) deviation:
// one fused multiply-add per matrix element, each row a single chain (the
// search is bound by instruction issue, so no extra adds to shorten chains),
// issued column by column so that consecutive instructions share e[j].
template <int PH>
__device__ __forceinline__ void prop_apply(const Prop2& q, float (&e)[6]) {
  const float (&c)[4][2] = PH == 1 ? q.c1 : q.c2;
  const float (&d)[2] = PH == 1 ? q.d1 : q.d2;
  float n[6];
  float a0 = e[0], a1 = e[1], a2 = e[2], a3 = e[3];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float ej = e[j];
    a0 = fmaf(j < 4 ? q.m[0][j] : c[0][j - 4], ej, a0);
    a1 = fmaf(j < 4 ? q.m[1][j] : c[1][j - 4], ej, a1);
    a2 = fmaf(j < 4 ? q.m[2][j] : c[2][j - 4], ej, a2);
    a3 = fmaf(j < 4 ? q.m[3][j] : c[3][j - 4], ej, a3);
  }
  n[0] = a0;
  n[1] = a1;
  n[2] = a2;
  n[3] = a3;
  n[4] = fmaf(d[0], e[4], e[4]);
  n[5] = fmaf(d[1], e[5], e[5]);
#pragma unroll
  for (int i = 0; i < 6; ++i) e[i] = n[i];
}

// v = A w for the homogeneous deviation system of one phase.
__device__ __forceinline__ void a_apply(const Coef& k, float da, float dn, const float (&w)[6], float (&v)[6]) {
  v[0] = w[1];
  v[1] = fmaf(k.m13, w[3], fmaf(k.m12, w[2], fmaf(k.m11, w[1], k.m10 * w[0])));
  v[2] = fmaf(k.cx, w[4], fmaf(k.m22, w[2], k.m20 * w[0]));
  v[3] = fmaf(k.cy, w[5], fmaf(k.m33, w[3], k.m30 * w[0]));
  v[4] = da * w[4];
  v[5] = dn * w[5];
}

// One RK4 step of length hs on e' = A e (Horner form of T4(hs A) e).
__device__ __forceinline__ void rk4_vec(const Coef& k, float da, float dn, float hs, float (&e)[6]) {
  float w[6], v[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) w[i] = e[i];
  const float c[4] = {0.25f * hs, hs * (1.0f / 3.0f), 0.5f * hs, hs};
#pragma unroll
  for (int lev = 0; lev < 4; ++lev) {
    a_apply(k, da, dn, w, v);
#pragma unroll
    for (int i = 0; i < 6; ++i) w[i] = fmaf(c[lev], v[i], e[i]);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) e[i] = w[i];
}

// n sample intervals of one phase with the one-sample propagator, emitting
// theta_k - thf after each: e[0] + off in the pulse phase (deviation from the
// pulse equilibrium), e[0] itself in the step phase (PH = 2, whose equilibrium
// is the end fixation).  The sink is told where each block of 4 samples ends
// (the residual sink compensates per block).
template <int PH, class Sink>
__device__ __forceinline__ void run_samples(const Prop2& phi, float (&e)[6], float off, int& kk, int n,
                                            Sink& sink) {
  int i = 0;
  // one block of 4 samples per trip: unrolling further only hoists trace loads
#pragma unroll 1
  for (; i + 4 <= n; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      prop_apply<PH>(phi, e);
      sink.emit(kk++, PH == 2 ? e[0] : e[0] + off);
    }
    sink.block_end();
  }
  for (; i < n; ++i) {
    prop_apply<PH>(phi, e);
    sink.emit(kk++, PH == 2 ? e[0] : e[0] + off);
  }
}

// One phase's one-sample propagator with its rows paired for packed FP32
// (two single-precision FMAs per instruction): column j of rows 0-1 and of
// rows 2-3, and the activation diagonal.
struct PropX2 {
  float2 r01[6], r23[6];
  float2 d;
};

template <int PH>
__device__ __forceinline__ void pack_phase(const Prop2& q, PropX2& x) {
  const float (&c)[4][2] = PH == 1 ? q.c1 : q.c2;
  const float (&d)[2] = PH == 1 ? q.d1 : q.d2;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    x.r01[j] = make_float2(j < 4 ? q.m[0][j] : c[0][j - 4], j < 4 ? q.m[1][j] : c[1][j - 4]);
    x.r23[j] = make_float2(j < 4 ? q.m[2][j] : c[2][j - 4], j < 4 ? q.m[3][j] : c[3][j - 4]);
  }
  x.d = make_float2(d[0], d[1]);
}

// The same update as prop_apply with the rows taken two at a time: each
// packed FMA performs the two row FMAs that prop_apply issues one after the
// other, with the same operands in the same order, so the result is the same
// bit for bit.
__device__ __forceinline__ void prop_apply_x2(const PropX2& x, float (&e)[6]) {
  float2 a01 = make_float2(e[0], e[1]), a23 = make_float2(e[2], e[3]);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float2 ej = make_float2(e[j], e[j]);
    a01 = __ffma2_rn(x.r01[j], ej, a01);
    a23 = __ffma2_rn(x.r23[j], ej, a23);
  }
  const float2 f = make_float2(e[4], e[5]);
  const float2 nf = __ffma2_rn(x.d, f, f);
  e[0] = a01.x;
  e[1] = a01.y;
  e[2] = a23.x;
  e[3] = a23.y;
  e[4] = nf.x;
  e[5] = nf.y;
}

// run_samples with the packed update (PACK) or the scalar one.
template <int PH, bool PACK, class Sink>
__device__ __forceinline__ void run_samples_v(const Prop2& phi, float (&e)[6], float off, int& kk, int n,
                                              Sink& sink) {
  if constexpr (!PACK) {
    run_samples<PH>(phi, e, off, kk, n, sink);
  } else {
    PropX2 x;
    pack_phase<PH>(phi, x);
    int i = 0;
#pragma unroll 1
    for (; i + 4 <= n; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        prop_apply_x2(x, e);
        sink.emit(kk++, PH == 2 ? e[0] : e[0] + off);
      }
      sink.block_end();
    }
    for (; i < n; ++i) {
      prop_apply_x2(x, e);
      sink.emit(kk++, PH == 2 ? e[0] : e[0] + off);
    }
  }
}

// x <- x + y + x y (increment form of (I + x)(I + y)) in place, one block at
// a time so that only one block of y is live: the coupling blocks first (they
// read the old mechanical block of x), then the activation diagonals, then the
// mechanical block row by row.  y is x itself (SQUARE: each block is copied
// before it is overwritten) or the single-substep base in the thread's
// shared-memory slot (element i at qs[i * stride], Prop2 order).
template <bool SQUARE>
__device__ __forceinline__ void prop_mul_inplace(Prop2& x, const float* qs, int stride) {
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    float yc[4][2], yd[2];
    const int oc = ph == 0 ? 16 : 24, od = ph == 0 ? 32 : 34;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int f = 0; f < 2; ++f) yc[i][f] = SQUARE ? (ph == 0 ? x.c1[i][f] : x.c2[i][f]) : qs[(oc + 2 * i + f) * stride];
#pragma unroll
    for (int f = 0; f < 2; ++f) yd[f] = SQUARE ? (ph == 0 ? x.d1[f] : x.d2[f]) : qs[(od + f) * stride];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        const float c = ph == 0 ? x.c1[i][f] : x.c2[i][f];
        float acc = fmaf(c, yd[f], c + yc[i][f]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) acc = fmaf(x.m[i][kk], yc[kk][f], acc);
        if (ph == 0) x.c1[i][f] = acc;
        else x.c2[i][f] = acc;
      }
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      if (ph == 0) x.d1[f] = fmaf(x.d1[f], yd[f], x.d1[f] + yd[f]);
      else x.d2[f] = fmaf(x.d2[f], yd[f], x.d2[f] + yd[f]);
    }
  }
  float ym[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ym[i][j] = SQUARE ? x.m[i][j] : qs[(4 * i + j) * stride];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float a[4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) a[kk] = x.m[i][kk];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = a[j] + ym[i][j];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc = fmaf(a[kk], ym[kk][j], acc);
      x.m[i][j] = acc;
    }
  }
}

// prop_mul_inplace with two columns per packed FP32 instruction: every entry
// gets the same operations in the same order (its own add, then the FMAs over
// k = 0..3), so the result is the same bit for bit.
template <bool SQUARE>
__device__ __forceinline__ void prop_mul_inplace_x2(Prop2& x, const float* qs, int stride) {
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    float (&c)[4][2] = ph == 0 ? x.c1 : x.c2;
    float (&d)[2] = ph == 0 ? x.d1 : x.d2;
    const int oc = ph == 0 ? 16 : 24, od = ph == 0 ? 32 : 34;
    float2 yc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      yc[i] = SQUARE ? make_float2(c[i][0], c[i][1])
                     : make_float2(qs[(oc + 2 * i) * stride], qs[(oc + 2 * i + 1) * stride]);
    const float2 yd = SQUARE ? make_float2(d[0], d[1]) : make_float2(qs[od * stride], qs[(od + 1) * stride]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 ci = make_float2(c[i][0], c[i][1]);
      float2 acc = __ffma2_rn(ci, yd, __fadd2_rn(ci, yc[i]));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc = __ffma2_rn(make_float2(x.m[i][kk], x.m[i][kk]), yc[kk], acc);
      c[i][0] = acc.x;
      c[i][1] = acc.y;
    }
    const float2 dd = make_float2(d[0], d[1]);
    const float2 nd = __ffma2_rn(dd, yd, __fadd2_rn(dd, yd));
    d[0] = nd.x;
    d[1] = nd.y;
  }
  float2 ym[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jp = 0; jp < 2; ++jp)
      ym[i][jp] = SQUARE ? make_float2(x.m[i][2 * jp], x.m[i][2 * jp + 1])
                         : make_float2(qs[(4 * i + 2 * jp) * stride], qs[(4 * i + 2 * jp + 1) * stride]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float a[4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) a[kk] = x.m[i][kk];
#pragma unroll
    for (int jp = 0; jp < 2; ++jp) {
      float2 acc = __fadd2_rn(make_float2(a[2 * jp], a[2 * jp + 1]), ym[i][jp]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) acc = __ffma2_rn(make_float2(a[kk], a[kk]), ym[kk][jp], acc);
      x.m[i][2 * jp] = acc.x;
      x.m[i][2 * jp + 1] = acc.y;
    }
  }
}

// x = (I + q)^n - I for n >= 1, x holding q on entry and q stored in the slot:
// left-to-right binary powering with at most one propagator live (PACK: the
// packed products).
template <bool PACK = false>
__device__ __forceinline__ void prop_pow_slot(Prop2& x, const float* qs, int stride, int n) {
  const int msb = 31 - __clz(n);
  for (int b = msb - 1; b >= 0; --b) {
    if constexpr (PACK) {
      prop_mul_inplace_x2<true>(x, qs, stride);
      if ((n >> b) & 1) prop_mul_inplace_x2<false>(x, qs, stride);
    } else {
      prop_mul_inplace<true>(x, qs, stride);
      if ((n >> b) & 1) prop_mul_inplace<false>(x, qs, stride);
    }
  }
}

// Copy a Prop2 to / from a per-thread shared-memory slot (element i of the
// thread's copy at qs[i * stride]: consecutive threads hit consecutive banks).
__device__ __forceinline__ void prop_store(const Prop2& q, float* qs, int stride) {
  const float* f = reinterpret_cast<const float*>(&q);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(Prop2) / sizeof(float)); ++i) qs[i * stride] = f[i];
}
__device__ __forceinline__ void prop_load(Prop2& q, const float* qs, int stride) {
  float* f = reinterpret_cast<float*>(&q);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(Prop2) / sizeof(float)); ++i) f[i] = qs[i * stride];
}

// One phase of a slot's propagator (Prop2 element order: m row-major, c1,
// c2, d1, d2), read straight into the row-paired form of pack_phase.
template <int PH>
__device__ __forceinline__ void slot_load_x2(PropX2& x, const float* qs, int stride) {
  constexpr int oc = PH == 1 ? 16 : 24, od = PH == 1 ? 32 : 34;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int e0 = j < 4 ? 0 * 4 + j : oc + 0 * 2 + (j - 4), e1 = j < 4 ? 1 * 4 + j : oc + 1 * 2 + (j - 4);
    const int e2 = j < 4 ? 2 * 4 + j : oc + 2 * 2 + (j - 4), e3 = j < 4 ? 3 * 4 + j : oc + 3 * 2 + (j - 4);
    x.r01[j] = make_float2(qs[e0 * stride], qs[e1 * stride]);
    x.r23[j] = make_float2(qs[e2 * stride], qs[e3 * stride]);
  }
  x.d = make_float2(qs[od * stride], qs[(od + 1) * stride]);
}

// Bring the lanes of `mask` together before a loop whose trip count n varies
// by lane: a warp-wide maximum of n, which every lane of the mask must take
// part in (kept alive by an empty asm so that it is not removed).
__device__ __forceinline__ void converge_on(unsigned mask, int n) {
  const unsigned m = __reduce_max_sync(mask, (unsigned)n);
  asm volatile("" ::"r"(m));
}

// Walk one candidate's trajectory from the first sample after onset to the
// end of the window.  The sink receives, for each sample k > onset, the value
// dth = theta_k - thf (positive frame), and block_end() after blocks of
// samples.  Samples k <= onset sit at th0 and are handled by the caller.
// Returns the number of samples emitted; with `guard` set, -1 (nothing
// emitted) for a candidate too stiff even for the finest substep (refine_shift).
// qs (optional): a shared-memory slot that keeps the single-substep
// propagator from the set-up to the pulse-end interval instead of rebuilding it.
// pulse_end (optional): set to 1 when the pulse ends inside the window (the
// pulse-end sample was integrated substep by substep), else 0.
// SYNC: the lanes in `mask` (all of which call walk together) reconverge
// before each phase's sample loop, by a warp reduction over the loop's trip
// count, so that a warp runs each sample loop once for all of its lanes
// instead of once per group of lanes that reached it together (a plain
// __syncwarp did not keep them together); lanes that return early leave the
// mask first.
// PACK: the sample loops use the packed update (prop_apply_x2: the same
// arithmetic, two row FMAs per instruction).
template <class Sink, bool SYNC = false, bool PACK = false>
__device__ __forceinline__ int walk(const float* p, const SacConst& sc0, Sink& sink, float* qs = nullptr,
                                    int qstride = 0, bool guard = false, int* pulse_end = nullptr,
                                    unsigned mask = 0xffffffffu) {
  Coef k;
  make_coef(p, k);
  const int rs = refine_shift(k, sc0.h);
  if (SYNC) mask = __ballot_sync(mask, !(guard && rs < 0));
  if (guard && rs < 0) return -1;
  const int sh = rs < 0 ? kMaxRefine : rs;
  const int nsub = sc0.nsub << sh;            // substeps per sample, refined
  const float h = sc0.h * pow2neg(sh);        // substep, refined (exact power-of-two scale)
  const SacConst& sc = sc0;
  const int ntot = sc.L - 1 - sc.onset;
  if (ntot <= 0) return 0;
  // pulse end, in substeps after onset
  float tau = p[kPw] * sc.fs * (float)nsub * 1e-3f;
  tau = fminf(fmaxf(tau, 0.0f), 1.0e9f);
  const float jf = floorf(tau);
  const float frac = tau - jf;
  const float span = (float)ntot * (float)nsub;
  int n1, jsw = 0;
  bool sw;
  if (jf >= span) { n1 = ntot; sw = false; }
  else {
    const int J = (int)jf;
    n1 = J / nsub;
    jsw = J - n1 * nsub;
    sw = true;
  }
  float s0[6], s1[6], s2[6];
  rest_state_k(p, k, sc.th0, s0);
  drive_equilibrium_k(p, k, p[kNsacAg], p[kNsacAnt], s1);
  rest_state_k(p, k, sc.thf, s2);
  float e[6], dl[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) { e[i] = s0[i] - s1[i]; dl[i] = s1[i] - s2[i]; }
  const float off1 = s1[0] - sc.thf;
  Prop2 phi;
  if (qs) {
    if constexpr (PACK) step_increment_x2(k, h, phi);
    else step_increment(k, h, phi);
    prop_store(phi, qs, qstride);
    prop_pow_slot<PACK>(phi, qs, qstride, nsub);
  } else {
    Prop2 q;
    step_increment(k, h, q);
    prop_pow(q, nsub, phi);
  }
  int kk = sc.onset + 1;
  if (SYNC) converge_on(mask, n1);
  run_samples_v<1, PACK>(phi, e, off1, kk, n1, sink);
  if (pulse_end) *pulse_end = sw ? 1 : 0;
  if (SYNC) mask = __ballot_sync(mask, sw);
  if (sw) {
    // pulse-end interval: jsw whole substeps of the pulse phase, the split
    // substep (two RK4 steps around the switch), the rest of the step phase
    const float h1 = frac * h;
    if constexpr (PACK) {
      // the single-substep matrix of each phase straight from the slot, rows paired
      PropX2 x;
      slot_load_x2<1>(x, qs, qstride);
      for (int s = 0; s < jsw; ++s) prop_apply_x2(x, e);
      rk4_vec(k, k.da1, k.dn1, h1, e);
#pragma unroll
      for (int i = 0; i < 6; ++i) e[i] += dl[i];
      rk4_vec(k, k.da2, k.dn2, h - h1, e);
      slot_load_x2<2>(x, qs, qstride);
      for (int s = jsw + 1; s < nsub; ++s) prop_apply_x2(x, e);
    } else {
      Prop2 q;
      if (qs) prop_load(q, qs, qstride);
      else step_increment(k, h, q);
      for (int s = 0; s < jsw; ++s) prop_apply<1>(q, e);
      rk4_vec(k, k.da1, k.dn1, h1, e);
#pragma unroll
      for (int i = 0; i < 6; ++i) e[i] += dl[i];
      rk4_vec(k, k.da2, k.dn2, h - h1, e);
      for (int s = jsw + 1; s < nsub; ++s) prop_apply<2>(q, e);
    }
    sink.emit(kk++, e[0]);
    const int n2 = ntot - n1 - 1;
    if (SYNC) converge_on(mask, n2);
    run_samples_v<2, PACK>(phi, e, 0.0f, kk, n2, sink);
  }
  return ntot;
}

// Single-phase version of run_samples.
template <class Sink>
__device__ __forceinline__ void run_samples1(const Prop1& phi, float (&e)[6], float off, int& kk, int n,
                                             Sink& sink) {
  int i = 0;
  for (; i + 4 <= n; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      prop1_apply(phi, e);
      sink.emit(kk++, e[0] + off);
    }
    sink.block_end();
  }
  for (; i < n; ++i) {
    prop1_apply(phi, e);
    sink.emit(kk++, e[0] + off);
  }
}

// Register-lean walk: the same RK4 trajectory as walk(), scheduled so that
// only one phase's propagator is live at a time.  The parameters come from
// `src.load(p)`, called whenever they are needed again instead of being kept:
// the pulse phase's one-sample propagator is built first, then the
// equilibria, the pulse-phase samples, the pulse-end interval (single-substep
// matrices of both phases, the split step) and the step phase's one-sample
// propagator, built only once the pulse phase is done.
template <class PSrc, class Sink>
__device__ __forceinline__ int walk_lean(const PSrc& src, const SacConst& sc0, Sink& sink, int* pulse_end = nullptr) {
  const int ntot = sc0.L - 1 - sc0.onset;
  if (ntot <= 0) return 0;
  Prop1 phi;
  SacConst sc;
  {
    float p[kNumParams];
    src.load(p);
    Coef k;
    make_coef(p, k);
    const int rs = refine_shift(k, sc0.h);
    sc = refined(sc0, rs < 0 ? kMaxRefine : rs);
    Prop1 q;
    step_increment1<1>(k, sc.h, q);
    prop1_pow(q, sc.nsub, phi);
  }
  float e[6], dl[6], off1, frac;
  int n1, jsw = 0;
  bool sw;
  {
    float p[kNumParams];
    src.load(p);
    float tau = p[kPw] * sc.fs * (float)sc.nsub * 1e-3f;
    tau = fminf(fmaxf(tau, 0.0f), 1.0e9f);
    const float jf = floorf(tau);
    frac = tau - jf;
    const float span = (float)ntot * (float)sc.nsub;
    if (jf >= span) { n1 = ntot; sw = false; }
    else {
      const int J = (int)jf;
      n1 = J / sc.nsub;
      jsw = J - n1 * sc.nsub;
      sw = true;
    }
    Coef k;
    make_coef(p, k);
    float s0[6], s1[6], s2[6];
    rest_state_k(p, k, sc.th0, s0);
    drive_equilibrium_k(p, k, p[kNsacAg], p[kNsacAnt], s1);
    rest_state_k(p, k, sc.thf, s2);
#pragma unroll
    for (int i = 0; i < 6; ++i) { e[i] = s0[i] - s1[i]; dl[i] = s1[i] - s2[i]; }
    off1 = s1[0] - sc.thf;
  }
  int kk = sc.onset + 1;
  run_samples1(phi, e, off1, kk, n1, sink);
  if (pulse_end) *pulse_end = sw ? 1 : 0;
  if (sw) {
    {
      float p[kNumParams];
      src.load(p);
      Coef k;
      make_coef(p, k);
      {
        Prop1 q;
        step_increment1<1>(k, sc.h, q);
        for (int s = 0; s < jsw; ++s) prop1_apply(q, e);
      }
      const float h1 = frac * sc.h;
      rk4_vec(k, k.da1, k.dn1, h1, e);
#pragma unroll
      for (int i = 0; i < 6; ++i) e[i] += dl[i];
      rk4_vec(k, k.da2, k.dn2, sc.h - h1, e);
      Prop1 q;
      step_increment1<2>(k, sc.h, q);
      for (int s = jsw + 1; s < sc.nsub; ++s) prop1_apply(q, e);
      prop1_pow(q, sc.nsub, phi);
    }
    sink.emit(kk++, e[0]);
    const int n2 = ntot - n1 - 1;
    run_samples1(phi, e, 0.0f, kk, n2, sink);
  }
  return ntot;
}

}  // namespace opmm
