/*
 * opmm_oracle.c -- plain FP64 CPU oracle of the OPMM estimation path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path: every number below is typed from the paper (Table 1) or derived
 * here from the model reading written next to it.
 *
 * What it computes (paper: "Parallel Oculomotor Plant Mathematical Model for
 * Large Scale Eye Movement Simulation", arXiv 2007.09884):
 *
 *   - the 18-parameter oculomotor plant (Sec. 2.1, Sec. 2.2.1, Table 1,
 *     Fig. 1 caption).  The paper names the components but prints no
 *     equations; the reading used here is the linear six-state plant
 *     below (series elasticity, length-tension elasticity and force-velocity
 *     viscosity per muscle, globe inertia and passive viscosity, first-order
 *     active-state tension driven by a pulse-step neural signal);
 *   - a fixed-step classical RK4 integrator, h ~ 0.1 ms, with the substep
 *     that contains the pulse end split in two (model silent on integration);
 *   - an exact piecewise solver (matrix exponential per constant-input
 *     segment) used only to pin the RK4 integrator;
 *   - the optimisation error (Sec. 3.4 "OPMM output": difference between the
 *     recorded and simulated trajectory), minimised as the mean squared
 *     error and reported also as the mean absolute error;
 *   - the parallel Nelder-Mead estimator (Sec. 3.3 "Parameter estimation",
 *     Algorithm 1): all reflection, expansion, contraction and shrink points
 *     of a simplex are evaluated in one wave, then the Lagarias et al. decision
 *     is taken and the vertices sorted; exit on the distance and function
 *     tolerances or the iteration cap;
 *   - a multi-start batch of such simplices per saccade (Algorithm 1 spawns
 *     one task per saccade; the candidate budget per iteration is spread over
 *     independent simplices);
 *   - Philox4x32-10 (Salmon et al., SC'11) for the random simplex centres;
 *   - the 9-parameter model (Sec. 2.2.2, Table 2) as a map from its nine
 *     search coordinates to the 18 OPC entries, the neural control signal
 *     held at the box centre;
 *   - a Levenberg-Marquardt refinement of a fitted vector (the gradient
 *     methods Sec. 5 proposes), with a central-difference Jacobian through
 *     the same RK4 plant.
 *
 * Parity status: the plant equations are a reading of a paper that prints
 * none; agreement with the authors' own (unpublished) implementation is
 * parity unpinned.  Everything else is pinned by the tests (closed forms,
 * invariants, exact solutions, textbook optimisation problems, brute force).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define NP 18

/* OPC vector order: the column order of the paper's example output (Fig. 4):
 * SE_ag SE_ant LT_ag LT_ant PE_ag PE_ant Vis FV_ag FV_ant Inert Act_ag Act_ant
 * Deact_ag Deact_ant Step H_ag H_ant W                                      */
enum {
  KSE_AG = 0, KSE_ANT, KLT_AG, KLT_ANT, NC_AG, NC_ANT, BP, B_AG, B_ANT, JIN,
  TAC_AG, TAC_ANT, TDE_AG, TDE_ANT, NC_FIX, NSAC_AG, NSAC_ANT, PW
};

/* Table 1 defaults (Sec. 2.2.1).  The pulse width default is "saccade
 * duration - 6 ms" and is filled in by or_nominal_table1. */
static const double TABLE1[NP] = {
  2.5, 2.5, 1.2, 1.2, 0.8, 0.5, 0.06, 0.046, 0.022, 0.000043,
  11.7, 2.4, 2.0, 1.9, 14.0, 55.0, 0.5, 0.0
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).                                                 */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24 high bits of a 32-bit word as a uniform number in [0, 1). */
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Plant model                                                               */
/* ------------------------------------------------------------------------ */

#define OR_MAX_REFINE 6   /* at most 2^6 times the base substeps per sample */

/* Substeps per sample so that the RK4 step is close to 0.1 ms. */
int or_nsub(double fs) {
  int n = (int)floor(1.0e4 / fs + 0.5);
  return n < 1 ? 1 : n;
}

/* Tension each muscle holds at fixation angle th: the paper defines tension
 * slope and intercept as the muscle force at the plant's equilibrium points
 * (Sec. 2.1 item 4).  Agonist pulls toward positive angles. */
static double ta_eq(const double* p, double th) { return p[NC_FIX] + p[NC_AG] * th; }
static double tn_eq(const double* p, double th) { return p[NC_FIX] - p[NC_ANT] * th; }

/* Active-state tension that keeps the plant at rest at angle th: the step
 * level of the pulse-step signal, i.e. the control signal's size while the eye
 * holds a fixation (Sec. 2.1). */
double or_step_ag(const double* p, double th) {
  return ta_eq(p, th) * (1.0 + p[KLT_AG] / p[KSE_AG]) + p[KLT_AG] * th;
}
double or_step_ant(const double* p, double th) {
  return tn_eq(p, th) * (1.0 + p[KLT_ANT] / p[KSE_ANT]) - p[KLT_ANT] * th;
}

/* Rest state at angle th: (theta, omega, x, y, Fa, Fn). */
void or_rest_state(const double* p, double th, double* s) {
  s[0] = th;
  s[1] = 0.0;
  s[2] = th + ta_eq(p, th) / p[KSE_AG];
  s[3] = tn_eq(p, th) / p[KSE_ANT] - th;
  s[4] = or_step_ag(p, th);
  s[5] = or_step_ant(p, th);
}

typedef struct { double na, nn, ta, tn; } drive_t;

/* Right-hand side of the plant ODE.
 *   Ta = KSE_AG (x - theta)            agonist series-elastic tension
 *   Tn = KSE_ANT (y + theta)           antagonist series-elastic tension
 *   KP = NC_AG + NC_ANT                passive globe elasticity (the value that
 *                                      makes every fixation an equilibrium)
 *   theta' = omega
 *   J omega' = Ta - Tn - BP omega - KP theta
 *   B_AG x'  = Fa - Ta - KLT_AG x
 *   B_ANT y' = Fn - Tn - KLT_ANT y
 *   tau_a Fa' = Na - Fa,  tau_n Fn' = Nn - Fn                               */
static void deriv(const double* p, const double* s, const drive_t* d, double* ds) {
  double Ta = p[KSE_AG] * (s[2] - s[0]);
  double Tn = p[KSE_ANT] * (s[3] + s[0]);
  double KP = p[NC_AG] + p[NC_ANT];
  ds[0] = s[1];
  ds[1] = (Ta - Tn - p[BP] * s[1] - KP * s[0]) / p[JIN];
  ds[2] = (s[4] - Ta - p[KLT_AG] * s[2]) / p[B_AG];
  ds[3] = (s[5] - Tn - p[KLT_ANT] * s[3]) / p[B_ANT];
  ds[4] = (d->na - s[4]) / d->ta;
  ds[5] = (d->nn - s[5]) / d->tn;
}

/* Neural drive of each phase (Sec. 2.1, pulse-step signal): 0 = fixation
 * before onset, 1 = pulse, 2 = step at the new fixation.  Activation and
 * deactivation "times" are read as first-order time constants in ms. */
static drive_t phase_drive(const double* p, int phase, double th0, double thf) {
  drive_t d;
  if (phase == 1) {
    d.na = p[NSAC_AG];  d.nn = p[NSAC_ANT];
    d.ta = p[TAC_AG] * 1e-3;  d.tn = p[TDE_ANT] * 1e-3;
  } else {
    double th = phase == 0 ? th0 : thf;
    d.na = or_step_ag(p, th);  d.nn = or_step_ant(p, th);
    d.ta = p[TDE_AG] * 1e-3;  d.tn = p[TAC_ANT] * 1e-3;
  }
  return d;
}

static void rk4_step(const double* p, double* s, const drive_t* d, double h) {
  double k1[6], k2[6], k3[6], k4[6], t[6];
  deriv(p, s, d, k1);
  for (int i = 0; i < 6; ++i) t[i] = s[i] + 0.5 * h * k1[i];
  deriv(p, t, d, k2);
  for (int i = 0; i < 6; ++i) t[i] = s[i] + 0.5 * h * k2[i];
  deriv(p, t, d, k3);
  for (int i = 0; i < 6; ++i) t[i] = s[i] + h * k3[i];
  deriv(p, t, d, k4);
  for (int i = 0; i < 6; ++i)
    s[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

int or_substeps(const double* p, double fs);

/* Position of the pulse end in RK4 substeps after onset: index J of the
 * substep that contains it and the fraction of that substep before it. */
static void pulse_end(const double* p, double fs, int nsub, long* J, double* frac) {
  double tau = p[PW] * fs * (double)nsub / 1000.0;
  if (!(tau >= 0.0)) tau = 0.0;
  if (tau > 1.0e9) tau = 1.0e9;
  double fl = floor(tau);
  *J = (long)fl;
  *frac = tau - fl;
}

/* RK4 trajectory sampled at t_k = k / fs, k = 0..L-1.  The onset is on the
 * sample grid (t_on = onset / fs).  Saccades toward negative angles are run
 * mirrored and negated (Fig. 1 shows the plant for positive saccades).
 * theta: [L] (may be NULL); state: [L][6] or NULL (mirrored frame). */
int or_simulate_rk4(const double* p, int L, double fs, int onset, double th0,
                    double thf, double* theta, double* state) {
  if (L <= 0 || !(fs > 0.0)) return -1;
  int mirror = thf < th0;
  if (mirror) { th0 = -th0; thf = -thf; }
  int nsub = or_substeps(p, fs);
  double h = 1.0 / (fs * nsub);
  long J; double frac;
  pulse_end(p, fs, nsub, &J, &frac);
  drive_t d0 = phase_drive(p, 0, th0, thf);
  drive_t d1 = phase_drive(p, 1, th0, thf);
  drive_t d2 = phase_drive(p, 2, th0, thf);
  double s[6];
  or_rest_state(p, th0, s);
  if (theta) theta[0] = mirror ? -s[0] : s[0];
  if (state) memcpy(state, s, sizeof s);
  long g_on = (long)onset * nsub;
  for (int k = 0; k + 1 < L; ++k) {
    for (int j = 0; j < nsub; ++j) {
      long rel = (long)k * nsub + j - g_on;
      if (rel < 0) rk4_step(p, s, &d0, h);
      else if (rel < J) rk4_step(p, s, &d1, h);
      else if (rel == J) { rk4_step(p, s, &d1, frac * h); rk4_step(p, s, &d2, h - frac * h); }
      else rk4_step(p, s, &d2, h);
    }
    if (theta) theta[k + 1] = mirror ? -s[0] : s[0];
    if (state) memcpy(state + 6 * (k + 1), s, sizeof s);
  }
  return 0;
}

/* Integrate with a constant drive (na, nn, ta, tn in s) from state s for
 * nsteps RK4 steps of size h; used to pin the steady-state closed form. */
void or_integrate_const(const double* p, double* s, double na, double nn,
                        double ta, double tn, double h, long nsteps) {
  drive_t d = {na, nn, ta, tn};
  for (long i = 0; i < nsteps; ++i) rk4_step(p, s, &d, h);
}

/* Derivative at a state (exposed so tests can check invariants). */
void or_deriv(const double* p, const double* s, double na, double nn, double ta,
              double tn, double* ds) {
  drive_t d = {na, nn, ta, tn};
  deriv(p, s, &d, ds);
}

/* ------------------------------------------------------------------------ */
/* Exact piecewise solution: the plant is linear with piecewise-constant     */
/* input, so each segment is z(t) = expm(t M) z(0), z = [state; 1], with M   */
/* the 7x7 augmented system matrix written out entry by entry.               */
/* ------------------------------------------------------------------------ */
static void mat7_mul(const double* a, const double* b, double* c) {
  double t[49];
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 7; ++k) acc += a[i * 7 + k] * b[k * 7 + j];
      t[i * 7 + j] = acc;
    }
  memcpy(c, t, sizeof t);
}

/* expm by scaling and squaring with a 24-term Taylor series. */
void or_expm7(const double* m, double* e) {
  double norm = 0.0;
  for (int j = 0; j < 7; ++j) {
    double col = 0.0;
    for (int i = 0; i < 7; ++i) col += fabs(m[i * 7 + j]);
    if (col > norm) norm = col;
  }
  int sq = 0;
  while (norm > 0.25 && sq < 60) { norm *= 0.5; ++sq; }
  double a[49], term[49], sum[49];
  double scale = ldexp(1.0, -sq);
  for (int i = 0; i < 49; ++i) a[i] = m[i] * scale;
  memset(sum, 0, sizeof sum);
  memset(term, 0, sizeof term);
  for (int i = 0; i < 7; ++i) { sum[i * 8] = 1.0; term[i * 8] = 1.0; }
  for (int k = 1; k <= 24; ++k) {
    mat7_mul(term, a, term);
    for (int i = 0; i < 49; ++i) { term[i] /= (double)k; sum[i] += term[i]; }
  }
  for (int s = 0; s < sq; ++s) mat7_mul(sum, sum, sum);
  memcpy(e, sum, sizeof sum);
}

static void system_matrix(const double* p, const drive_t* d, double* m) {
  double KP = p[NC_AG] + p[NC_ANT];
  memset(m, 0, 49 * sizeof(double));
  /* theta row */
  m[0 * 7 + 1] = 1.0;
  /* omega row */
  m[1 * 7 + 0] = -(p[KSE_AG] + p[KSE_ANT] + KP) / p[JIN];
  m[1 * 7 + 1] = -p[BP] / p[JIN];
  m[1 * 7 + 2] = p[KSE_AG] / p[JIN];
  m[1 * 7 + 3] = -p[KSE_ANT] / p[JIN];
  /* x row */
  m[2 * 7 + 0] = p[KSE_AG] / p[B_AG];
  m[2 * 7 + 2] = -(p[KSE_AG] + p[KLT_AG]) / p[B_AG];
  m[2 * 7 + 4] = 1.0 / p[B_AG];
  /* y row */
  m[3 * 7 + 0] = -p[KSE_ANT] / p[B_ANT];
  m[3 * 7 + 3] = -(p[KSE_ANT] + p[KLT_ANT]) / p[B_ANT];
  m[3 * 7 + 5] = 1.0 / p[B_ANT];
  /* active-state rows */
  m[4 * 7 + 4] = -1.0 / d->ta;
  m[4 * 7 + 6] = d->na / d->ta;
  m[5 * 7 + 5] = -1.0 / d->tn;
  m[5 * 7 + 6] = d->nn / d->tn;
}

static void advance_exact(const double* p, const drive_t* d, double dt, double* z) {
  if (dt <= 0.0) return;
  double m[49], e[49], t[7];
  system_matrix(p, d, m);
  for (int i = 0; i < 49; ++i) m[i] *= dt;
  or_expm7(m, e);
  for (int i = 0; i < 7; ++i) {
    double acc = 0.0;
    for (int k = 0; k < 7; ++k) acc += e[i * 7 + k] * z[k];
    t[i] = acc;
  }
  memcpy(z, t, sizeof t);
}

/* Exact trajectory with the same pulse-end instant as the RK4 path
 * (t_sw = t_on + (J + frac) h). */
int or_simulate_exact(const double* p, int L, double fs, int onset, double th0,
                      double thf, double* theta) {
  if (L <= 0 || !(fs > 0.0)) return -1;
  int mirror = thf < th0;
  if (mirror) { th0 = -th0; thf = -thf; }
  int nsub = or_substeps(p, fs);
  double h = 1.0 / (fs * nsub);
  long J; double frac;
  pulse_end(p, fs, nsub, &J, &frac);
  double t_on = onset / fs;
  double t_sw = t_on + ((double)J + frac) * h;
  drive_t d[3] = {phase_drive(p, 0, th0, thf), phase_drive(p, 1, th0, thf),
                  phase_drive(p, 2, th0, thf)};
  double z[7];
  or_rest_state(p, th0, z);
  z[6] = 1.0;
  theta[0] = mirror ? -z[0] : z[0];
  for (int k = 0; k + 1 < L; ++k) {
    double ta = k / fs, tb = (k + 1) / fs;
    double cuts[4] = {ta, 0, 0, tb};
    int nc = 1;
    if (t_on > ta && t_on < tb) cuts[nc++] = t_on;
    if (t_sw > ta && t_sw < tb) cuts[nc++] = t_sw;
    cuts[nc++] = tb;
    for (int c = 0; c + 1 < nc; ++c) {
      double a = cuts[c], b = cuts[c + 1];
      double mid = 0.5 * (a + b);
      int ph = mid < t_on ? 0 : (mid < t_sw ? 1 : 2);
      advance_exact(p, &d[ph], b - a, z);
    }
    theta[k + 1] = mirror ? -z[0] : z[0];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Objective                                                                 */
/* ------------------------------------------------------------------------ */

/* Size estimate of the plant's fastest mode (s^-1): the negated trace of the
 * mechanical block plus the fastest activation rate. */
static double stiff_est(const double* p) {
  double tmin = p[TAC_AG];
  if (p[TAC_ANT] < tmin) tmin = p[TAC_ANT];
  if (p[TDE_AG] < tmin) tmin = p[TDE_AG];
  if (p[TDE_ANT] < tmin) tmin = p[TDE_ANT];
  return p[BP] / p[JIN] + (p[KSE_AG] + p[KLT_AG]) / p[B_AG] + (p[KSE_ANT] + p[KLT_ANT]) / p[B_ANT] + 1000.0 / tmin;
}

/* RK4 is stable on the negative real axis up to |h lambda| ~ 2.78.  Substeps
 * per sample for candidate p: the base count (h ~ 0.1 ms) doubled until h
 * times the estimate is at most 2.5, at most OR_MAX_REFINE times (stiff
 * corners of a wide search box, Fig. 4's 10x and 0.1x values). */
int or_substeps(const double* p, double fs) {
  int n = or_nsub(fs);
  double h = 1.0 / (fs * n);
  const double est = stiff_est(p);
  for (int k = 0; k < OR_MAX_REFINE && !(h * est <= 2.5); ++k) {
    h *= 0.5;
    n *= 2;
  }
  return n;
}

/* Stiffness guard: a candidate whose fastest mode is too fast even for the
 * finest substep scores +inf.  Same rule on both sides. */
int or_stiff(const double* p, double fs) {
  double h = 1.0 / (fs * or_substeps(p, fs));
  return !(h * stiff_est(p) <= 2.5);
}

/* Mean squared error and mean absolute error of the RK4 trajectory against
 * the recorded trace y[L].  Non-finite results become +inf. */
int or_errors(const double* p, int L, double fs, int onset, double th0,
              double thf, const double* y, double* mse, double* mae) {
  if (or_stiff(p, fs)) { *mse = INFINITY; if (mae) *mae = INFINITY; return 0; }
  double* th = (double*)malloc(sizeof(double) * (size_t)L);
  if (!th) return -2;
  or_simulate_rk4(p, L, fs, onset, th0, thf, th, NULL);
  double s2 = 0.0, s1 = 0.0;
  for (int k = 0; k < L; ++k) {
    double e = th[k] - y[k];
    s2 += e * e;
    s1 += fabs(e);
  }
  free(th);
  double m2 = s2 / L, m1 = s1 / L;
  *mse = isfinite(m2) ? m2 : INFINITY;
  if (mae) *mae = isfinite(m1) ? m1 : INFINITY;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Nominal OPC vector                                                        */
/* ------------------------------------------------------------------------ */

/* Table 1 with W = duration - 6 ms. */
void or_nominal_table1(double dur_ms, double* p) {
  memcpy(p, TABLE1, sizeof TABLE1);
  p[PW] = dur_ms - 6.0;
}

/* Largest sampled position of the nominal saccade from 0 to amplitude A with
 * agonist pulse height nsac (1 kHz grid, 250 ms after onset). */
static double nominal_peak(double A, double dur_ms, double nsac) {
  double p[NP];
  or_nominal_table1(dur_ms, p);
  p[NSAC_AG] = nsac;
  enum { LC = 251 };
  double th[LC];
  or_simulate_rk4(p, LC, 1000.0, 0, 0.0, A, th, NULL);
  double pk = th[0];
  for (int k = 1; k < LC; ++k) if (th[k] > pk) pk = th[k];
  return pk;
}

/* Agonist pulse height that makes the nominal saccade's peak equal its
 * amplitude A > 0 (bisection).  Table 1's single value cannot produce the
 * range of amplitudes the workloads use; if even the step level of the new
 * fixation overshoots, the step level is returned. */
double or_calibrate_pulse(double A, double dur_ms) {
  double p[NP];
  or_nominal_table1(dur_ms, p);
  double lo = or_step_ag(p, A);
  if (nominal_peak(A, dur_ms, lo) >= A) return lo;
  double hi = lo > 1.0 ? 2.0 * lo : 2.0;
  int guard = 0;
  while (nominal_peak(A, dur_ms, hi) < A && guard++ < 40) { lo = hi; hi *= 2.0; }
  for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (nominal_peak(A, dur_ms, mid) < A) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Nelder-Mead (Lagarias, Reeds, Wright, Wright 1998), parallel wave form    */
/* ------------------------------------------------------------------------ */

#define NMAX NP
typedef double (*objective_fn)(const double* u, void* ctx);

typedef struct {
  int n;
  double x[NMAX + 1][NMAX];   /* vertices in sorted order */
  double f[NMAX + 1];
} simplex_t;

/* Stable sort of the vertices by f (insertion sort). */
static void simplex_sort(simplex_t* s) {
  int m = s->n + 1;
  for (int i = 1; i < m; ++i) {
    double fi = s->f[i];
    double xi[NMAX];
    memcpy(xi, s->x[i], sizeof(double) * s->n);
    int j = i - 1;
    while (j >= 0 && s->f[j] > fi) {
      s->f[j + 1] = s->f[j];
      memcpy(s->x[j + 1], s->x[j], sizeof(double) * s->n);
      --j;
    }
    s->f[j + 1] = fi;
    memcpy(s->x[j + 1], xi, sizeof(double) * s->n);
  }
}

/* Replace the worst vertex by (xn, fn) and move it in front of the first
 * vertex with a strictly larger value (a new point goes after ties). */
static void simplex_insert(simplex_t* s, const double* xn, double fn) {
  int i = s->n;
  while (i > 0 && s->f[i - 1] > fn) {
    s->f[i] = s->f[i - 1];
    memcpy(s->x[i], s->x[i - 1], sizeof(double) * s->n);
    --i;
  }
  s->f[i] = fn;
  memcpy(s->x[i], xn, sizeof(double) * s->n);
}

/* Exit test (Sec. 3.3): every vertex within tolx of the best in max-norm and
 * every value within tolf of the best value. */
int or_nm_converged(const simplex_t* s, double tolx, double tolf) {
  double dx = 0.0, df = 0.0;
  for (int i = 1; i <= s->n; ++i) {
    double a = fabs(s->f[i] - s->f[0]);
    if (!(a <= df)) df = a;          /* NaN/inf propagate as "not converged" */
    for (int j = 0; j < s->n; ++j) {
      double b = fabs(s->x[i][j] - s->x[0][j]);
      if (b > dx) dx = b;
    }
  }
  return dx <= tolx && df <= tolf;
}

/* Branch codes returned by one iteration (for branch-coverage tests). */
enum { NM_REFLECT = 1, NM_EXPAND = 2, NM_CONTRACT_OUT = 3, NM_CONTRACT_IN = 4, NM_SHRINK = 5 };

/* One iteration: build the n + 4 trial points (reflection, expansion, outside
 * and inside contraction, n shrink points), evaluate them all, then decide.
 * Coefficients rho = 1, chi = 2, gamma = sigma = 1/2. */
static int nm_iteration(simplex_t* s, objective_fn fn, void* ctx) {
  int n = s->n;
  double xbar[NMAX], xr[NMAX], xe[NMAX], xco[NMAX], xci[NMAX];
  double xs[NMAX + 1][NMAX], fs[NMAX + 1];
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += s->x[i][j];
    xbar[j] = acc / n;
  }
  for (int j = 0; j < n; ++j) {
    double w = s->x[n][j];
    xr[j] = xbar[j] + 1.0 * (xbar[j] - w);
    xe[j] = xbar[j] + 2.0 * (xr[j] - xbar[j]);
    xco[j] = xbar[j] + 0.5 * (xr[j] - xbar[j]);
    xci[j] = xbar[j] - 0.5 * (xbar[j] - w);
  }
  for (int i = 1; i <= n; ++i)
    for (int j = 0; j < n; ++j)
      xs[i][j] = s->x[0][j] + 0.5 * (s->x[i][j] - s->x[0][j]);
  double fr = fn(xr, ctx), fe = fn(xe, ctx), fco = fn(xco, ctx), fci = fn(xci, ctx);
  for (int i = 1; i <= n; ++i) fs[i] = fn(xs[i], ctx);

  double f1 = s->f[0], fn_ = s->f[n - 1], fw = s->f[n];
  int shrink = 0, branch;
  if (fr < f1) {
    if (fe < fr) { simplex_insert(s, xe, fe); branch = NM_EXPAND; }
    else { simplex_insert(s, xr, fr); branch = NM_REFLECT; }
  } else if (fr < fn_) {
    simplex_insert(s, xr, fr); branch = NM_REFLECT;
  } else if (fr < fw) {
    if (fco <= fr) { simplex_insert(s, xco, fco); branch = NM_CONTRACT_OUT; }
    else shrink = 1;
  } else {
    if (fci < fw) { simplex_insert(s, xci, fci); branch = NM_CONTRACT_IN; }
    else shrink = 1;
  }
  if (shrink) {
    for (int i = 1; i <= n; ++i) {
      memcpy(s->x[i], xs[i], sizeof(double) * n);
      s->f[i] = fs[i];
    }
    simplex_sort(s);
    branch = NM_SHRINK;
  }
  return branch;
}

/* ------------------------------------------------------------------------ */
/* Generic NM driver for textbook test functions                            */
/* ------------------------------------------------------------------------ */
typedef struct { int id; int n; } testfn_ctx;

static double testfn(const double* u, void* vctx) {
  testfn_ctx* c = (testfn_ctx*)vctx;
  if (c->id == 0) {                     /* sum_i (i+1) (u_i - 1)^2 */
    double acc = 0.0;
    for (int i = 0; i < c->n; ++i) acc += (i + 1) * (u[i] - 1.0) * (u[i] - 1.0);
    return acc;
  }
  if (c->id == 1) {                     /* Rosenbrock, 2-D */
    double a = u[1] - u[0] * u[0], b = 1.0 - u[0];
    return 100.0 * a * a + b * b;
  }
  /* double well per coordinate: sum_i (u_i^2 - 1)^2 (non-convex, can shrink) */
  double acc = 0.0;
  for (int i = 0; i < c->n; ++i) acc += (u[i] * u[i] - 1.0) * (u[i] * u[i] - 1.0);
  return acc;
}

/* Minimise test function `id` from the given initial simplex (n+1 rows of n);
 * writes the final simplex (sorted) back and returns the iteration count.
 * branches[it] receives the branch code of each iteration if non-NULL. */
int or_nm_testfn(int id, int n, double* verts, int max_iter, double tolx,
                 double tolf, double* fvals, int* branches) {
  if (n < 1 || n > NMAX) return -1;
  testfn_ctx c = {id, n};
  simplex_t s;
  s.n = n;
  for (int i = 0; i <= n; ++i) {
    memcpy(s.x[i], verts + i * n, sizeof(double) * n);
    s.f[i] = testfn(s.x[i], &c);
  }
  simplex_sort(&s);
  int it = 0;
  for (; it < max_iter; ++it) {
    if (or_nm_converged(&s, tolx, tolf)) break;
    int b = nm_iteration(&s, testfn, &c);
    if (branches) branches[it] = b;
  }
  for (int i = 0; i <= n; ++i) {
    memcpy(verts + i * n, s.x[i], sizeof(double) * n);
    fvals[i] = s.f[i];
  }
  return it;
}

/* One iteration from a given (unsorted) simplex: returns the branch taken;
 * verts/fvals receive the sorted result. */
int or_nm_one_step_testfn(int id, int n, double* verts, double* fvals) {
  testfn_ctx c = {id, n};
  simplex_t s;
  s.n = n;
  for (int i = 0; i <= n; ++i) {
    memcpy(s.x[i], verts + i * n, sizeof(double) * n);
    s.f[i] = testfn(s.x[i], &c);
  }
  simplex_sort(&s);
  int b = nm_iteration(&s, testfn, &c);
  for (int i = 0; i <= n; ++i) {
    memcpy(verts + i * n, s.x[i], sizeof(double) * n);
    fvals[i] = s.f[i];
  }
  return b;
}

/* ------------------------------------------------------------------------ */
/* OPMM objective in log-parameter coordinates                               */
/* ------------------------------------------------------------------------ */
/* Search coordinates of the 9-parameter model (Sec. 2.2.2, Table 2), in the
 * table's order: K_SE (both muscles), K_LT (both), B_AG, B_ANT, B_P, N_C_AG,
 * N_C_ANT, J, N_C_FIX.  The model shares one series elasticity and one
 * length-tension coefficient between the muscles and does not estimate the
 * neural control signal.  For each OPC entry (Fig. 4 order) the model
 * coordinate that scales it, or -1 for the entries held at the box centre
 * (activation and deactivation times, pulse heights, pulse width). */
static const int kModel9Coord[NP] = {0, 0, 1, 1, 5, 6, 4, 2, 3, 7, -1, -1, -1, -1, 8, -1, -1, -1};

/* Coordinate map of a model: coord[j] = the search coordinate that scales OPC
 * entry j, or -1 (held at the centre).  free_mask selects, among the model's
 * own parameters (18: the OPC entries; 9: the Table 2 entries in order), those
 * estimated.  A 9-parameter centre must give both muscles the same series
 * elasticity and the same length-tension coefficient.  Returns the search
 * dimension n, or -1 for an unknown model or an untied centre. */
static int model_map(int model, uint32_t free_mask, const double* pc, int* coord) {
  int n = 0;
  if (model == 18) {
    for (int j = 0; j < NP; ++j) coord[j] = (free_mask >> j & 1u) ? n++ : -1;
    return n;
  }
  if (model == 9) {
    if (pc && (pc[0] != pc[1] || pc[2] != pc[3])) return -1;
    int idx[9];
    for (int i = 0; i < 9; ++i) idx[i] = (free_mask >> i & 1u) ? n++ : -1;
    for (int j = 0; j < NP; ++j) coord[j] = kModel9Coord[j] < 0 ? -1 : idx[kModel9Coord[j]];
    return n;
  }
  return -1;
}

typedef struct {
  const double* pc;        /* box centre (nominal OPC) [18] */
  const int* coord;        /* search coordinate of each OPC entry, or -1 [18] */
  int n;
  double lnlo, lnhi;
  int L, onset;
  double fs, th0, thf;
  const double* y;
} opmm_ctx_t;

/* p_j = pc_j exp(clamp(u_coord(j))) for estimated entries; the others stay
 * at pc_j. */
static void u_to_p(const opmm_ctx_t* c, const double* u, double* p) {
  memcpy(p, c->pc, sizeof(double) * NP);
  for (int j = 0; j < NP; ++j) {
    if (c->coord[j] < 0) continue;
    double v = u[c->coord[j]];
    if (v < c->lnlo) v = c->lnlo;
    if (v > c->lnhi) v = c->lnhi;
    p[j] = c->pc[j] * exp(v);
  }
}

static double opmm_objective(const double* u, void* vctx) {
  const opmm_ctx_t* c = (const opmm_ctx_t*)vctx;
  double p[NP], mse;
  u_to_p(c, u, p);
  if (or_errors(p, c->L, c->fs, c->onset, c->th0, c->thf, c->y, &mse, NULL) != 0)
    return INFINITY;
  return mse;
}

/* Initial simplex centre of start s (Philox counter (saccade, s, block, 0),
 * key = 64-bit seed): start 0 is the box centre, the others are uniform in
 * the box.  Vertex i > 0 is the centre moved by `step` along coordinate i-1. */
void or_start_centre(int n, int s, uint32_t sac_index, uint64_t seed,
                     double lnlo, double lnhi, double* c) {
  if (s == 0) { for (int j = 0; j < n; ++j) c[j] = 0.0; return; }
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int blk = 0; 4 * blk < n; ++blk) {
    uint32_t ctr[4] = {sac_index, (uint32_t)s, (uint32_t)blk, 0u}, r[4];
    or_philox4x32_10(ctr, key, r);
    for (int q = 0; q < 4 && 4 * blk + q < n; ++q)
      c[4 * blk + q] = lnlo + (lnhi - lnlo) * u01(r[q]);
  }
}

typedef struct {
  const opmm_ctx_t* ctx;
  int S, T, nthreads, tid;
  uint32_t sac_index;
  uint64_t seed;
  double step, tolx, tolf;
  double* best_u;    /* [S][n] */
  double* best_f;    /* [S] */
  int* iters;        /* [S] */
} fit_job_t;

static void run_simplex(const fit_job_t* jb, int si) {
  const opmm_ctx_t* c = jb->ctx;
  int n = c->n;
  simplex_t s;
  s.n = n;
  double centre[NMAX];
  or_start_centre(n, si, jb->sac_index, jb->seed, c->lnlo, c->lnhi, centre);
  for (int i = 0; i <= n; ++i) {
    memcpy(s.x[i], centre, sizeof(double) * n);
    if (i > 0) s.x[i][i - 1] += jb->step;
    s.f[i] = opmm_objective(s.x[i], (void*)c);
  }
  simplex_sort(&s);
  int it = 0;
  for (; it < jb->T; ++it) {
    if (or_nm_converged(&s, jb->tolx, jb->tolf)) break;
    nm_iteration(&s, opmm_objective, (void*)c);
  }
  memcpy(jb->best_u + (size_t)si * n, s.x[0], sizeof(double) * n);
  jb->best_f[si] = s.f[0];
  jb->iters[si] = it;
}

static void* fit_worker(void* arg) {
  fit_job_t* jb = (fit_job_t*)arg;
  for (int si = jb->tid; si < jb->S; si += jb->nthreads) run_simplex(jb, si);
  return NULL;
}

/* Multi-start parallel NM fit of one recorded saccade.
 *   pc[18]      box centre (nominal OPC)
 *   model       18 or 9 (the search coordinates, model_map)
 *   free_mask   bit j set = the model's parameter j is estimated
 *   y[L]        recorded trace
 *   S, T        simplices, iteration cap
 * Outputs: per-simplex best value and vertex, iterations, and the index of
 * the winning simplex (lowest value, ties to the lowest index). */
int or_fit(const double* pc, int model, uint32_t free_mask, int L, double fs, int onset,
           double th0, double thf, const double* y, int S, int T, double box_lo,
           double box_hi, double step, double tolx, double tolf, uint64_t seed,
           uint32_t sac_index, int nthreads, double* best_u_all,
           double* best_f_all, int* iters_all, int* winner) {
  int coord[NP];
  const int n = model_map(model, free_mask, pc, coord);
  if (n < 1 || S < 1 || T < 0 || L < 1 || !(box_lo > 0.0) || !(box_hi >= box_lo))
    return -1;
  opmm_ctx_t c = {pc, coord, n, log(box_lo), log(box_hi), L, onset, fs, th0, thf, y};
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  fit_job_t jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    fit_job_t jb = {&c, S, T, nthreads, t, sac_index, seed, step, tolx, tolf,
                    best_u_all, best_f_all, iters_all};
    jobs[t] = jb;
  }
  if (nthreads == 1) fit_worker(&jobs[0]);
  else {
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, fit_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  }
  int w = 0;
  for (int si = 1; si < S; ++si) if (best_f_all[si] < best_f_all[w]) w = si;
  *winner = w;
  return 0;
}

/* Objective values at a list of points u[m][n] (grid search and scoring). */
int or_score(const double* pc, int model, uint32_t free_mask, int L, double fs, int onset,
             double th0, double thf, const double* y, double box_lo,
             double box_hi, const double* u, int m, double* f) {
  int coord[NP];
  const int n = model_map(model, free_mask, pc, coord);
  if (n < 1) return -1;
  opmm_ctx_t c = {pc, coord, n, log(box_lo), log(box_hi), L, onset, fs, th0, thf, y};
  for (int i = 0; i < m; ++i) f[i] = opmm_objective(u + (size_t)i * n, &c);
  return 0;
}

/* Full OPC vector at a point u (applies the same clamp as the objective). */
int or_u_to_p(const double* pc, int model, uint32_t free_mask, double box_lo, double box_hi,
              const double* u, double* p) {
  int coord[NP];
  const int n = model_map(model, free_mask, pc, coord);
  if (n < 1) return -1;
  opmm_ctx_t c = {pc, coord, n, log(box_lo), log(box_hi), 0, 0, 0, 0, 0, NULL};
  u_to_p(&c, u, p);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient-based refinement (Sec. 5 names gradient methods as the            */
/* alternative estimator to test): Levenberg-Marquardt on the residual vector */
/* ------------------------------------------------------------------------ */

/* Residual vector r(u) of length m; returns 0, or nonzero when u cannot be
 * simulated (too stiff): that point counts as f = +inf. */
typedef int (*residual_fn)(const double* u, double* r, void* ctx);

/* Levenberg-Marquardt from u (n coordinates, projected onto [lnlo, lnhi]),
 * K iterations, central-difference Jacobian of step delta, initial damping
 * lambda0.  One iteration:
 *   - at a new point, J[k][j] = (r_k(u + delta e_j) - r_k(u - delta e_j)) /
 *     (2 delta) (a column whose two points cannot be simulated is zero),
 *     A = J^T J, g = J^T r(u);
 *   - solve (A + lambda D) du = -g, D = diag(max(A_jj, 1e-9 max_i A_ii))
 *     (Marquardt's scaling with a floor), by Cholesky;
 *   - u' = clamp(u + du); accept when f(u') < f(u) (then lambda / 10, floor
 *     1e-12, and a new Jacobian), else lambda * 10 (ceiling 1e12).
 * f(u) = sum_k r_k^2 / m.  Stops early when max_i A_ii = 0 or the system is not
 * positive definite.  Outputs u, f, the accepted steps and the residual
 * evaluations. */
static int lm_run(residual_fn res, void* ctx, int n, int m, double lnlo, double lnhi, double* u, int K,
                  double delta, double lambda0, double* f_out, int* accepted, long* nres) {
  double* r = (double*)malloc(sizeof(double) * (size_t)m * (2 * (size_t)n + 2));
  if (!r) return -2;
  double* rp = r + m;                 /* r(u + delta e_j) */
  double* rm = rp + m;                /* r(u - delta e_j) */
  double* rt = rm + m;                /* r(u') */
  double* J = rt + m;                 /* [m][n] stored by column: J + j * m */
  double A[NMAX * NMAX], g[NMAX], M[NMAX * NMAX], du[NMAX], ut[NMAX], uj[NMAX];
  for (int j = 0; j < n; ++j) u[j] = u[j] < lnlo ? lnlo : (u[j] > lnhi ? lnhi : u[j]);
  long evals = 0;
  int acc = 0;
  double f = INFINITY;
  if (res(u, r, ctx) == 0) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += r[k] * r[k];
    f = s / m;
  }
  ++evals;
  double lambda = lambda0;
  int need_jac = 1;
  for (int it = 0; it < K && isfinite(f); ++it) {
    if (need_jac) {
      for (int j = 0; j < n; ++j) {
        memcpy(uj, u, sizeof(double) * n);
        uj[j] = u[j] + delta;
        const int bp = res(uj, rp, ctx);
        uj[j] = u[j] - delta;
        const int bm = res(uj, rm, ctx);
        evals += 2;
        double* col = J + (size_t)j * m;
        for (int k = 0; k < m; ++k) col[k] = (bp || bm) ? 0.0 : (rp[k] - rm[k]) / (2.0 * delta);
      }
      for (int a = 0; a < n; ++a) {
        const double* ca = J + (size_t)a * m;
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += ca[k] * r[k];
        g[a] = s;
        for (int b = 0; b <= a; ++b) {
          const double* cb = J + (size_t)b * m;
          double t = 0.0;
          for (int k = 0; k < m; ++k) t += ca[k] * cb[k];
          A[a * n + b] = A[b * n + a] = t;
        }
      }
      need_jac = 0;
    }
    double amax = 0.0;
    for (int j = 0; j < n; ++j) amax = A[j * n + j] > amax ? A[j * n + j] : amax;
    if (!(amax > 0.0)) break;
    memcpy(M, A, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
      const double d = A[j * n + j] > 1e-9 * amax ? A[j * n + j] : 1e-9 * amax;
      M[j * n + j] += lambda * d;
    }
    /* Cholesky M = L L^T in place (lower triangle), then L y = -g, L^T du = y */
    int ok = 1;
    for (int j = 0; j < n && ok; ++j) {
      double s = M[j * n + j];
      for (int k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
      if (!(s > 0.0)) { ok = 0; break; }
      const double ljj = sqrt(s);
      M[j * n + j] = ljj;
      for (int i = j + 1; i < n; ++i) {
        double t = M[i * n + j];
        for (int k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
        M[i * n + j] = t / ljj;
      }
    }
    if (!ok) break;
    for (int i = 0; i < n; ++i) {
      double t = -g[i];
      for (int k = 0; k < i; ++k) t -= M[i * n + k] * du[k];
      du[i] = t / M[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = du[i];
      for (int k = i + 1; k < n; ++k) t -= M[k * n + i] * du[k];
      du[i] = t / M[i * n + i];
    }
    for (int j = 0; j < n; ++j) {
      const double v = u[j] + du[j];
      ut[j] = v < lnlo ? lnlo : (v > lnhi ? lnhi : v);
    }
    double ft = INFINITY;
    if (res(ut, rt, ctx) == 0) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += rt[k] * rt[k];
      ft = s / m;
    }
    ++evals;
    if (ft < f) {
      memcpy(u, ut, sizeof(double) * n);
      memcpy(r, rt, sizeof(double) * m);
      f = ft;
      ++acc;
      lambda = lambda / 10.0 > 1e-12 ? lambda / 10.0 : 1e-12;
      need_jac = 1;
    } else {
      lambda = lambda * 10.0 < 1e12 ? lambda * 10.0 : 1e12;
    }
  }
  free(r);
  *f_out = f;
  if (accepted) *accepted = acc;
  if (nres) *nres = evals;
  return 0;
}

/* OPMM residual: the RK4 trajectory of p(u) minus the recorded trace. */
static int opmm_residual(const double* u, double* r, void* vctx) {
  const opmm_ctx_t* c = (const opmm_ctx_t*)vctx;
  double p[NP];
  u_to_p(c, u, p);
  if (or_stiff(p, c->fs)) return 1;
  or_simulate_rk4(p, c->L, c->fs, c->onset, c->th0, c->thf, r, NULL);
  for (int k = 0; k < c->L; ++k) r[k] -= c->y[k];
  return 0;
}

/* Refine one saccade's OPC vector from search point u (in/out, n
 * coordinates of the model) with lm_run; the box is centre * [box_lo,
 * box_hi] as in the search. */
int or_refine(const double* pc, int model, uint32_t free_mask, int L, double fs, int onset,
              double th0, double thf, const double* y, double box_lo, double box_hi,
              double* u, int K, double delta, double lambda0, double* f, int* accepted,
              long* nres) {
  int coord[NP];
  const int n = model_map(model, free_mask, pc, coord);
  if (n < 1 || L < 1 || K < 0 || !(delta > 0.0) || !(lambda0 > 0.0) || !(box_lo > 0.0) ||
      !(box_hi >= box_lo))
    return -1;
  opmm_ctx_t c = {pc, coord, n, log(box_lo), log(box_hi), L, onset, fs, th0, thf, y};
  return lm_run(opmm_residual, &c, n, L, c.lnlo, c.lnhi, u, K, delta, lambda0, f, accepted, nres);
}

/* Textbook residuals that pin lm_run: id 0, a linear least-squares problem
 * r = A u - b with A = [[1,2,0],[0,1,1],[1,0,3],[2,1,1],[0,0,1],[1,1,1]] and
 * b = [1,2,3,4,5,6] (m = 6, n = 3); id 1, Rosenbrock's function as residuals
 * (10 (u1 - u0^2), 1 - u0) (m = 2, n = 2). */
static int lm_testres(const double* u, double* r, void* vctx) {
  const int id = *(const int*)vctx;
  if (id == 0) {
    static const double Am[6][3] = {{1, 2, 0}, {0, 1, 1}, {1, 0, 3}, {2, 1, 1}, {0, 0, 1}, {1, 1, 1}};
    for (int k = 0; k < 6; ++k) r[k] = Am[k][0] * u[0] + Am[k][1] * u[1] + Am[k][2] * u[2] - (k + 1);
  } else {
    r[0] = 10.0 * (u[1] - u[0] * u[0]);
    r[1] = 1.0 - u[0];
  }
  return 0;
}

int or_lm_testfn(int id, double* u, int K, double lo, double hi, double delta, double lambda0,
                 double* f, int* accepted) {
  if (id != 0 && id != 1) return -1;
  const int n = id == 0 ? 3 : 2, m = id == 0 ? 6 : 2;
  long nres = 0;
  return lm_run(lm_testres, &id, n, m, lo, hi, u, K, delta, lambda0, f, accepted, &nres);
}
