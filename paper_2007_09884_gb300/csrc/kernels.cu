// kernels.cu -- CUDA kernels of the OPMM estimation path (sm_103a).
//
//   k_gather      copy caller traces into the packed, 16-byte aligned buffer
//   k_nominal     box centres: Table 1, W = D - 6 ms, calibrated agonist pulse
//   k_simulate    trajectories of (OPC, saccade) pairs
//   k_score       objective of many OPC vectors against one saccade
//   k_search      persistent multi-start parallel Nelder-Mead (Algorithm 1)
//   k_finalize    per-saccade winner and FP64 re-computation of its error
//   k_refine      Levenberg-Marquardt refinement of search results
//   k_refine_check  FP64 error of the refined vectors
//   k_admit, k_advance  request loop: slot admission and iteration progress
//
// The hot loop is k_search's candidate evaluation: one thread integrates one
// trial OPC vector's plant in registers (plant.cuh), scoring each sample against
// the trace staged once per block in shared memory by a TMA bulk copy, with a
// compensated FP32 sum.  Per block, two groups of G simplices of one saccade
// advance side by side: all 22 trial points of every simplex of a group are
// evaluated in one wave (Sec. 3.3: all simplex transformations are computed at
// once), ordered by pulse-end time and taken in 32-candidate chunks by all of
// the block's warps; the warp that completes a group's wave takes that group's
// Lagarias decisions and publishes its next wave while the other warps
// evaluate the other group's.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/opmm.h"
#include "common.cuh"
#include "launch.h"
#include "plant.cuh"

namespace opmm {

__device__ __forceinline__ SacConst sac_const(const DevSac& d) {
  SacConst s;
  s.L = d.L; s.onset = d.onset; s.nsub = d.nsub;
  s.fs = d.fs; s.h = d.h; s.th0 = d.th0; s.thf = d.thf;
  return s;
}

// ------------------------------------------------------------------ gather
__global__ void k_gather(const float* const* src, const DevSac* sacs, float* dst, int n) {
  const int b = blockIdx.x;
  if (b >= n) return;
  const DevSac d = sacs[b];
  const float* s = src[b];
  float* o = dst + d.off;
  const int Lp = (d.L + 3) & ~3;
  for (int k = threadIdx.x; k < Lp; k += blockDim.x) o[k] = k < d.L ? s[k] : 0.0f;
}

// ------------------------------------------------------------------ sinks
// Blocked compensated summation: the squared errors of each block of samples
// (the sample loops run in blocks of 4) are summed plainly, and each block sum
// is added to the running total with Kahan compensation, so the relative error
// stays O(4 eps) per block instead of growing with the window length.
struct KahanSink {
  const float* z;   // trace minus end fixation, positive frame
  float sum, c;
  float part;
  __device__ __forceinline__ void emit(int k, float dth) {
    const float d = dth - z[k];
    part = fmaf(d, d, part);
  }
  __device__ __forceinline__ void block_end() {
    const float y = part - c;
    const float t = sum + y;
    c = (t - sum) - y;
    sum = t;
    part = 0.0f;
  }
};

struct WriteSink {
  float* out;
  float sign, thf;
  __device__ __forceinline__ void emit(int k, float dth) { out[k] = sign * (thf + dth); }
  __device__ __forceinline__ void block_end() {}
};

struct PeakSink {
  float m;
  __device__ __forceinline__ void emit(int, float dth) { m = fmaxf(m, dth); }
  __device__ __forceinline__ void block_end() {}
};

// Objective of one OPC vector: mean squared error over the window; the
// samples up to onset (the plant at rest) are folded into (sum0, c0).
// pe (optional): set to 1 when the pulse ends inside the window.
template <bool SYNC = false, bool PACK = false>
__device__ __forceinline__ float objective(const float* p, const SacConst& sc, const float* z,
                                           float sum0, float c0, float* qs = nullptr, int qstride = 0,
                                           int* pe = nullptr, unsigned mask = 0xffffffffu) {
  KahanSink s{z, sum0, c0, 0.0f};
  if (walk<KahanSink, SYNC, PACK>(p, sc, s, qs, qstride, true, pe, mask) < 0) return INFINITY;
  s.block_end();
  const float f = (s.sum - s.c) / (float)sc.L;
  return isfinite(f) ? f : INFINITY;
}

// Parameter sources of the register-lean walk: each load() re-derives the
// candidate's OPC vector instead of keeping it live.
struct PtrSrc {
  const float* p;
  __device__ __forceinline__ void load(float (&o)[kNumParams]) const {
#pragma unroll
    for (int j = 0; j < kNumParams; ++j) o[j] = p[j];
  }
};

// Candidate in ln-parameter space, from two rows in shared memory: a vertex
// (u = a), or the search's trial-point form u = a + (b - a) / 2 (a = b for the
// deciding warp's four trial points, best vertex and vertex q - 3 for a shrink
// point).
struct ULinSrc {
  const float* a;   // first row
  const float* b;   // second row
  bool half;        // u = a + (b - a) / 2, else u = a
  const float* pc;  // box centre
  float lnlo, lnhi;
  __device__ __forceinline__ void load(float (&o)[kNumParams]) const;
};


// Stage one saccade for a block: TMA bulk copy of the raw trace, then the
// positive-frame trace minus the end fixation and the compensated sum of the
// rest samples.  All threads call it; returns false on a wait timeout.
struct TraceStage {
  float sum0, c0;
};

__device__ bool stage_trace(const DevSac& d, const float* traces, float* yraw, float* z, uint64_t* bar,
                            uint32_t& phase, TraceStage* st) {
  if (threadIdx.x == 0) {
    fence_proxy_async_smem();
    const uint32_t bytes = (uint32_t)(((d.L + 3) & ~3) * 4);
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_1d(yraw, traces + d.off, bytes, bar);
  }
  const bool ok = mbar_wait(bar, phase, kMaxWaitTries);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  for (int k = threadIdx.x; k < d.L; k += blockDim.x) z[k] = d.sign * yraw[k] - d.thf;
  if (threadIdx.x == 0) {
    float sum = 0.0f, c = 0.0f;
    const int kend = min(d.onset, d.L - 1);
    for (int k = 0; k <= kend; ++k) {
      const float e = d.th0 - d.sign * yraw[k];
      const float y = fmaf(e, e, -c);
      const float t = sum + y;
      c = (t - sum) - y;
      sum = t;
    }
    st->sum0 = sum;
    st->c0 = c;
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------ nominal
// Largest sample of the default plant's saccade from 0 to A with agonist
// pulse nsac, 1 kHz grid, 250 ms after onset.
__device__ float nominal_peak(float* p, float A, float nsac) {
  p[kNsacAg] = nsac;
  SacConst sc;
  sc.L = 251; sc.onset = 0; sc.nsub = 10; sc.fs = 1000.0f; sc.h = 1.0e-4f; sc.th0 = 0.0f; sc.thf = A;
  PeakSink pk{-A};
  walk(p, sc, pk);
  return A + pk.m;
}

// One warp per saccade.  Calibrated mode: the agonist pulse for which the
// default plant's saccade peaks at its amplitude A; round 0 brackets the
// crossing between lo 2^(i-1) and lo 2^i (lo = step level of A), six rounds of
// a 32-point search narrow the bracket; if the step level already reaches A
// it is used as is.
__global__ void k_nominal(const DevSac* sacs, int n, int pulse_mode, const float* init_opc, float* pc) {
  const int lane = threadIdx.x & 31;
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b >= n) return;
  float* out = pc + (size_t)b * kNumParams;
  if (init_opc) {
    if (lane < kNumParams) out[lane] = init_opc[(size_t)b * kNumParams + lane];
    return;
  }
  const DevSac d = sacs[b];
  float p[kNumParams];
#pragma unroll
  for (int j = 0; j < kNumParams; ++j) p[j] = kTable1[j];
  p[kPw] = d.dur_ms - 6.0f;
  float nsac = kTable1[kNsacAg];
  if (pulse_mode == OPMM_PULSE_CALIBRATED) {
    const float A = d.thf - d.th0;
    float s[6];
    rest_state(p, A, s);
    const float lo = s[4];
    float pk = nominal_peak(p, A, lo * ldexpf(1.0f, lane));
    unsigned hit = __ballot_sync(0xffffffffu, pk >= A);
    if (hit & 1u) {
      nsac = lo;
    } else if (hit == 0u) {
      nsac = lo * ldexpf(1.0f, 31);
    } else {
      const int i0 = __ffs(hit) - 1;
      float a = lo * ldexpf(1.0f, i0 - 1);
      float bb = lo * ldexpf(1.0f, i0);
      for (int round = 0; round < 6; ++round) {
        const float x = a + (bb - a) * ((float)(lane + 1) * (1.0f / 33.0f));
        pk = nominal_peak(p, A, x);
        const unsigned h = __ballot_sync(0xffffffffu, pk >= A);
        const int i = h ? __ffs(h) - 1 : 32;
        const float xlo = __shfl_sync(0xffffffffu, x, i > 0 ? i - 1 : 0);
        const float xhi = __shfl_sync(0xffffffffu, x, i < 32 ? i : 31);
        const float na = i == 0 ? a : xlo;
        const float nb = i == 32 ? bb : xhi;
        a = na;
        bb = nb;
      }
      nsac = 0.5f * (a + bb);
    }
  }
  p[kNsacAg] = nsac;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kNumParams; ++j) out[j] = p[j];
  }
}

// ------------------------------------------------------------------ simulate
__global__ void k_simulate(const float* opc, int n, const DevSac* sacs, const int* sac_of,
                           const long long* out_off, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float p[kNumParams];
#pragma unroll
  for (int j = 0; j < kNumParams; ++j) p[j] = opc[(size_t)i * kNumParams + j];
  const DevSac d = sacs[sac_of ? sac_of[i] : i];
  const SacConst sc = sac_const(d);
  float* o = out + out_off[i];
  const int kend = min(d.onset, d.L - 1);
  for (int k = 0; k <= kend; ++k) o[k] = d.sign * d.th0;
  WriteSink w{o, d.sign, d.thf};
  walk(p, sc, w);
}

// ------------------------------------------------------------------ score
__global__ void k_score(const float* opc, int m, const DevSac* sac, const float* traces, float* f,
                        unsigned* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ TraceStage st;
  const DevSac d = *sac;
  const int lp = (d.L + 3) & ~3;
  float* yraw = reinterpret_cast<float*>(smraw);
  float* z = yraw + lp;
  if (threadIdx.x == 0) { mbar_init(&bar, 1); fence_mbar_init(); }
  __syncthreads();
  uint32_t phase = 0;
  if (!stage_trace(d, traces, yraw, z, &bar, phase, &st)) {
    if (threadIdx.x == 0) raise_error(err, kErrWaitTimeout);
    return;
  }
  const SacConst sc = sac_const(d);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    float p[kNumParams];
#pragma unroll
    for (int j = 0; j < kNumParams; ++j) p[j] = opc[(size_t)i * kNumParams + j];
    f[i] = objective(p, sc, z, st.sum0, st.c0);
  }
}

// ------------------------------------------------------------------ search
// Unit record (kUnitRecFloats words): [0] best f, [1] winning simplex (int),
// [2] its iterations (int), [3] candidate evaluations of the unit (int),
// [4..21] best vertex (ln units), [22] evaluations whose pulse ends inside the
// window (int), [23] unused.  With the 9-parameter model the vertex takes
// [4..12].
constexpr int kUnitRec = kUnitRecFloats;
constexpr int kSortBins = 512;           // pulse-end time bins of the per-wave ordering

// The search runs over N coordinates: N = 18, the OPC entries themselves, or
// N = 9, the 9-parameter model (Sec. 2.2.2, Table 2).  A simplex has N + 1
// vertices and each iteration N + 4 trial points.
template <int N>
__host__ __device__ constexpr int verts() { return N + 1; }
template <int N>
__host__ __device__ constexpr int trials() { return N + 4; }

// Search coordinate that scales OPC entry j (Fig. 4 order): j itself for N =
// 18; for N = 9 the coordinate of the Table 2 quantity the entry carries, in
// the table's order (K_SE, K_LT, B_AG, B_ANT, B_P, N_C_AG, N_C_ANT, J,
// N_C_FIX; the shared series elasticity and length-tension coefficient scale
// both muscles' entries), or -1 for the neural control signal, which that
// model does not estimate (activation and deactivation times, pulse heights
// and width stay at the box centre).
template <int N>
__host__ __device__ constexpr int search_coord(int j) {
  if (N == kNumParams) return j;
  switch (j) {
    case kSeAg: case kSeAnt: return 0;
    case kLtAg: case kLtAnt: return 1;
    case kBAg: return 2;
    case kBAnt: return 3;
    case kBp: return 4;
    case kNcAg: return 5;
    case kNcAnt: return 6;
    case kJ: return 7;
    case kNcFix: return 8;
    default: return -1;
  }
}

// OPC vector of search point u: p_j = pc_j exp(clamp(u_c)) for c =
// search_coord(j) >= 0, else pc_j.
template <int N>
__device__ __forceinline__ void u_to_p(const float* u, const float* pc, float lnlo, float lnhi, float (&p)[kNumParams]) {
#pragma unroll
  for (int j = 0; j < kNumParams; ++j) {
    const int c = search_coord<N>(j);
    p[j] = c < 0 ? pc[j] : pc[j] * __expf(fminf(fmaxf(u[c < 0 ? 0 : c], lnlo), lnhi));
  }
}

// Saved simplex (serving): vertices, values, centroid, order, active, iterations.
template <int N>
__host__ __device__ constexpr int state_floats() { return verts<N>() * N + verts<N>() + N + verts<N>() + 2; }
static_assert(state_floats<kNumParams>() == kSearchStateFloats, "saved simplex layout");
constexpr int kHistPer = kSortBins / 32;              // bins per lane of the scanning warp
constexpr int kHistLen = kSortBins + 32;                // bin b stored at b + b / kHistPer

// One block runs G simplices in each of two groups (a unit of 2G simplices of
// one saccade) with twelve warps, all of which evaluate: a group's wave (its
// 22 trial points per simplex, or its initial vertices) is published in
// chunks of 32 candidates that the warps claim in turn; the warp that
// completes a wave's last chunk takes that group's Nelder-Mead decisions,
// orders and publishes its next wave, while the other warps work on the other
// group's wave.  There is no block barrier between steps.  Twelve warps at 168
// registers per thread fill the SM's register file (3 warps per SM
// sub-partition).
constexpr int kSearchWarps = 12;
// Longest a search warp waits with nothing to claim (SM clock cycles, about
// four seconds): far above one chunk's evaluation plus one group's decisions;
// past it the warp raises kErrWaitTimeout and the block leaves the kernel.
constexpr long long kMaxIdleCycles = 8000000000LL;
template <int G, int N>
__host__ __device__ constexpr int search_threads() { return 32 * kSearchWarps; }
// candidates per lane when one warp orders a wave
template <int G, int N>
__host__ __device__ constexpr int wave_per_lane() { return (G * trials<N>() + 31) / 32; }

// State of one group of G simplices over N coordinates.
template <int G, int N>
struct GroupSmem {
  static constexpr int kNV = verts<N>();
  static constexpr int kNT = trials<N>();
  float U[G][kNV][N];            // vertices, by slot
  float XT[G][4][N];             // reflection, expansion, outside/inside contraction
  float XB[G][N];                // centroid of the best n vertices
  float F[G][kNV];               // vertex values, by slot
  float FT[G][kNT];              // trial values
  int hist[kHistLen];            // counting sort of the pending wave by pulse-end time (padded)
  unsigned short perm[G * kNT];  // candidate ids of the pending wave in key order
  int kr[G * kNT];               // ordering scratch: key << 16 | rank within the key's bin, or -1
  unsigned char ord[G][kNV + 1]; // ord[r] = slot of rank r
  int active[G];
  int iters[G];
  int okf[G];   // decision scratch: value spread within tol_f
  int okx[G];   // decision scratch: vertex spread within tol_x
  int shr[G];   // decision scratch: the simplex shrinks this step
  int nsim;     // simplices of this group (0: empty group)
  int nvalid;   // candidates of the pending wave
  int kind;     // pending wave: 0 initial vertices, 1 trial points
  int state;    // kPending (a wave is ordered) or kDone; written by the deciding warp only
  int it;       // trial waves evaluated in this launch
  int evals;    // candidate evaluations of this group
  int pe;       // of those, candidates whose pulse ends inside the window
  int pub;      // published wave: sequence number << 16 | chunks (0 chunks: nothing to take)
  int claim;    // sequence number << 16 | next chunk of 32 candidates (in key order) to claim
  int done;     // chunks of the published wave evaluated
};

enum : int { kPending = 0, kDone = 2 };

// The staged saccade of a search block.
struct SacStage {
  float pc[kNumParams];          // box centre of the current saccade
  SacConst sc;
  TraceStage st;
};

template <int G, int N, int NG>
struct SearchSmem {
  GroupSmem<G, N> grp[NG];
  SacStage sv;
  int cur_b;
  int unit;
  int abort;                     // a warp's bounded wait gave up: the block leaves
  uint64_t bar;
};

constexpr int kQSlotFloats = (int)(sizeof(Prop2) / sizeof(float));

// Dynamic shared memory: the block state, the raw and shifted traces (lcap
// floats each) and one single-substep propagator slot per thread.
template <int G, int N, int NG>
size_t search_smem_bytes(int lcap) {
  return ((sizeof(SearchSmem<G, N, NG>) + 127) / 128) * 128 + 2 * (size_t)lcap * sizeof(float) +
         (size_t)kQSlotFloats * search_threads<G, N>() * sizeof(float);
}

// Trial point coordinate (Lagarias et al. coefficients rho 1, chi 2, gamma 1/2).
__device__ __forceinline__ float trial_coord(int q, float xb, float w) {
  const float xr = xb + (xb - w);
  switch (q) {
    case 0: return xr;
    case 1: return xb + 2.0f * (xr - xb);
    case 2: return xb + 0.5f * (xr - xb);
    default: return xb - 0.5f * (xb - w);
  }
}

__device__ __forceinline__ float shrink_coord(float x1, float xi) { return x1 + 0.5f * (xi - x1); }

__device__ __forceinline__ void ULinSrc::load(float (&o)[kNumParams]) const {
#pragma unroll
  for (int j = 0; j < kNumParams; ++j) {
    const float u = half ? shrink_coord(a[j], b[j]) : a[j];
    o[j] = pc[j] * __expf(fminf(fmaxf(u, lnlo), lnhi));
  }
}

// Objective through the register-lean walk.
__device__ __forceinline__ float objective_lean(const ULinSrc& src, const SacConst& sc, const float* z,
                                                float sum0, float c0, int* pe = nullptr) {
  {
    float p[kNumParams];
    src.load(p);
    Coef k;
    make_coef(p, k);
    if (refine_shift(k, sc.h) < 0) return INFINITY;
  }
  KahanSink s{z, sum0, c0, 0.0f};
  walk_lean(src, sc, s, pe);
  s.block_end();
  const float f = (s.sum - s.c) / (float)sc.L;
  return isfinite(f) ? f : INFINITY;
}

// Objective of search point u; the lanes in `mask` call it together and
// reconverge inside the walk; PACK picks the packed sample update.
template <int N, bool PACK>
__device__ __forceinline__ float eval_u(const float (&u)[N], const float* pc, float lnlo,
                                        float lnhi, const SacConst& sc, const float* z, float sum0,
                                        float c0, float* qs, int qstride, int* pe, unsigned mask) {
  float p[kNumParams];
  u_to_p<N>(u, pc, lnlo, lnhi, p);
  return objective<true, PACK>(p, sc, z, sum0, c0, qs, qstride, pe, mask);
}

// Sort key of a candidate: its pulse-end time, binned over the window (the
// last bin holds pulses that outlast the window).  Lanes of a warp then run
// nearly the same number of pulse-phase and step-phase samples.
__device__ __forceinline__ int switch_key(float u_pw, float pc_pw, float lnlo, float lnhi, const SacConst& sc) {
  const int ntot = sc.L - 1 - sc.onset;
  if (ntot <= 0) return 0;
  const float w = pc_pw * __expf(fminf(fmaxf(u_pw, lnlo), lnhi));
  const float tau = fmaxf(w * sc.fs * 1e-3f, 0.0f);       // in samples after onset
  const float x = tau * ((float)(kSortBins - 1) / (float)ntot);
  return x >= (float)(kSortBins - 1) ? kSortBins - 1 : (int)x;
}

__device__ __forceinline__ int hist_slot(int b) { return b + b / kHistPer; }

// Rows of trial point q of simplex gi, as u = a + (b - a) / 2 coordinate by
// coordinate: a = b = the deciding warp's XT row for q < 4 (so u = a exactly),
// the best vertex and vertex q - 3 for the shrink points.  One form for every
// lane, so a warp holding both kinds does not diverge.
template <int G, int N>
__device__ __forceinline__ void trial_rows(const GroupSmem<G, N>& g, int gi, int q, const float*& a, const float*& b) {
  const unsigned char* o = g.ord[gi];
  a = q < 4 ? g.XT[gi][q] : g.U[gi][o[0]];
  b = q < 4 ? g.XT[gi][q] : g.U[gi][o[q - 3]];
}

// Centroid of the best n vertices and the vertex-spread half of the exit test
// (Sec. 3.3: every vertex within tol_x of the best in max-norm), spread over
// the deciding warp's lanes by (simplex, coordinate); `sel` picks the
// simplices to process.  g.okx[gi] must be 1 on entry and is cleared by any
// coordinate that fails.
template <int G, int N, class Sel>
__device__ __forceinline__ void centroids(GroupSmem<G, N>& g, int lane, float tolx, Sel sel) {
  for (int p = lane; p < g.nsim * N; p += 32) {
    const int gi = p / N, j = p - gi * N;
    if (!sel(gi)) continue;
    const unsigned char* o = g.ord[gi];
    float x[verts<N>()];
#pragma unroll
    for (int r = 0; r < verts<N>(); ++r) x[r] = g.U[gi][o[r]][j];
    float acc = 0.0f;
    bool ok = true;
#pragma unroll
    for (int r = 0; r < N; ++r) acc += x[r];
#pragma unroll
    for (int r = 1; r < verts<N>(); ++r) ok = ok && (fabsf(x[r] - x[0]) <= tolx);
    g.XB[gi][j] = acc / (float)N;
    if (!ok) g.okx[gi] = 0;
  }
}

// Stable ranking of 19 values by one thread: rank[r] = #{s : v_s < v_r or
// (v_s == v_r and s < r)}; the slots are written to ord in rank order.  The
// outer loop is kept rolled: this runs on the decision path, and its fully
// unrolled form (19 x 19 compares) crowds the instruction cache that the
// evaluating warps share.
template <int G, int N>
__device__ __forceinline__ void rank_simplex(GroupSmem<G, N>& g, int gi, const int (&sl)[verts<N>()], const float (&fv)[verts<N>()]) {
#pragma unroll 1
  for (int r = 0; r < verts<N>(); ++r) {
    int rank = 0;
#pragma unroll
    for (int t = 0; t < verts<N>(); ++t) rank += (fv[t] < fv[r] || (fv[t] == fv[r] && t < r)) ? 1 : 0;
    g.ord[gi][rank] = (unsigned char)sl[r];
  }
}

// Value spread within tol_f (the other half of the exit test) from the ranked
// values in ord.
template <int G, int N>
__device__ __forceinline__ int value_spread_ok(const GroupSmem<G, N>& g, int gi, float tolf) {
  const float f0 = g.F[gi][g.ord[gi][0]];
  bool ok = true;
#pragma unroll
  for (int r = 1; r < verts<N>(); ++r) ok = ok && (fabsf(g.F[gi][g.ord[gi][r]] - f0) <= tolf);
  return ok ? 1 : 0;
}

// Ranking and first centroid of freshly evaluated initial simplices.
template <int G, int N>
__device__ __forceinline__ void init_rank(GroupSmem<G, N>& g, int lane, float tolx, float tolf) {
  for (int gi = lane; gi < g.nsim; gi += 32) {
    int sl[verts<N>()];
    float fv[verts<N>()];
#pragma unroll
    for (int r = 0; r < verts<N>(); ++r) {
      sl[r] = r;
      fv[r] = g.F[gi][r];
    }
    rank_simplex<G, N>(g, gi, sl, fv);
    g.active[gi] = 1;
    g.iters[gi] = 0;
    g.okx[gi] = 1;
    g.okf[gi] = value_spread_ok<G, N>(g, gi, tolf);
  }
  __syncwarp();
  centroids<G, N>(g, lane, tolx, [](int) { return true; });
  __syncwarp();
  for (int gi = lane; gi < g.nsim; gi += 32)
    if (g.okx[gi] && g.okf[gi]) g.active[gi] = 0;
  __syncwarp();
}

// Lagarias decision and re-sort of every active simplex of a group after a
// trial wave.  One lane per simplex takes the decision (the slots and values
// of its 19 vertices in registers, in rank order) and applies a replacement;
// shrinks, centroids and the vertex-spread test are spread over all lanes.
template <int G, int N>
__device__ __forceinline__ void decide_group(GroupSmem<G, N>& g, int lane, float tolx, float tolf) {
  for (int gi = lane; gi < g.nsim; gi += 32) {
    g.shr[gi] = 0;
    g.okx[gi] = 1;
    if (!g.active[gi]) continue;
    unsigned char* o = g.ord[gi];
    int sl[verts<N>()];
    float fv[verts<N>()];
#pragma unroll
    for (int r = 0; r < verts<N>(); ++r) {
      sl[r] = o[r];
      fv[r] = g.F[gi][sl[r]];
    }
    const float f1 = fv[0], fn = fv[N - 1], fw = fv[N];
    const float fr = g.FT[gi][0], fe = g.FT[gi][1], fco = g.FT[gi][2], fci = g.FT[gi][3];
    int kind;
    float fnew = 0.0f;
    if (fr < f1) {
      if (fe < fr) { kind = 1; fnew = fe; } else { kind = 0; fnew = fr; }
    } else if (fr < fn) {
      kind = 0; fnew = fr;
    } else if (fr < fw) {
      if (fco <= fr) { kind = 2; fnew = fco; } else kind = -1;
    } else {
      if (fci < fw) { kind = 3; fnew = fci; } else kind = -1;
    }
    g.iters[gi] += 1;
    if (kind >= 0) {
      // replace the worst vertex; the new point goes after every vertex with
      // a value <= its own (ties stay in front of it)
      const int ws = sl[N];
#pragma unroll
      for (int j = 0; j < N; ++j) g.U[gi][ws][j] = g.XT[gi][kind][j];
      g.F[gi][ws] = fnew;
      int pos = 0;
#pragma unroll
      for (int r = 0; r < N; ++r) pos += fv[r] <= fnew ? 1 : 0;
#pragma unroll
      for (int r = N; r >= 1; --r)
        if (r > pos) {
          sl[r] = sl[r - 1];
          fv[r] = fv[r - 1];
        }
#pragma unroll
      for (int r = 0; r < verts<N>(); ++r)
        if (r == pos) {
          sl[r] = ws;
          fv[r] = fnew;
        }
#pragma unroll
      for (int r = 0; r < verts<N>(); ++r) o[r] = (unsigned char)sl[r];
      bool okf = true;
#pragma unroll
      for (int r = 1; r < verts<N>(); ++r) okf = okf && (fabsf(fv[r] - fv[0]) <= tolf);
      g.okf[gi] = okf ? 1 : 0;
    } else {
      // shrink toward the best vertex: the values now, the coordinates below
#pragma unroll
      for (int r = 1; r < verts<N>(); ++r) g.F[gi][sl[r]] = g.FT[gi][4 + r - 1];
      g.shr[gi] = 1;
    }
  }
  __syncwarp();
  // shrink coordinates: for each shrinking simplex, its 18 x 18 (vertex rank
  // >= 1, coordinate) updates over the lanes (the best vertex's row is only read)
  static_assert(G <= 32, "one ballot bit per simplex");
  const unsigned smask = __ballot_sync(0xffffffffu, lane < g.nsim && g.shr[lane]);
  for (unsigned m = smask; m; m &= m - 1) {
    const int gi = __ffs(m) - 1;
    const unsigned char* o = g.ord[gi];
    for (int e = lane; e < N * N; e += 32) {
      const int r = e / N + 1, j = e - (r - 1) * N;
      g.U[gi][o[r]][j] = shrink_coord(g.U[gi][o[0]][j], g.U[gi][o[r]][j]);
    }
  }
  __syncwarp();
  // stable re-sort of the shrunk simplices
  for (int gi = lane; gi < g.nsim; gi += 32) {
    if (!g.shr[gi]) continue;
    int sl[verts<N>()];
    float fv[verts<N>()];
#pragma unroll
    for (int r = 0; r < verts<N>(); ++r) {
      sl[r] = g.ord[gi][r];
      fv[r] = g.F[gi][sl[r]];
    }
    rank_simplex<G, N>(g, gi, sl, fv);
    g.okf[gi] = value_spread_ok<G, N>(g, gi, tolf);
  }
  __syncwarp();
  centroids<G, N>(g, lane, tolx, [&](int gi) { return g.active[gi] != 0; });
  __syncwarp();
  for (int gi = lane; gi < g.nsim; gi += 32)
    if (g.active[gi] && g.okx[gi] && g.okf[gi]) g.active[gi] = 0;
  __syncwarp();
}

// Set up a group's next wave (one warp): the initial vertices (kind 0) or the
// 22 trial points of every active simplex; a group with nothing left to
// evaluate, or at its iteration cap, is done.  The warp writes the four trial
// points (reflection, expansion, both contractions) to XT; the 18 shrink
// points are formed by the evaluating threads from the vertices.
template <int G, int N>
__device__ __forceinline__ void next_wave(GroupSmem<G, N>& g, int kind, int t_run, int lane) {
  static_assert(G <= 32, "one lane per simplex counts the active ones");
  int nact = 0;
  if (kind == 1) {
    nact = (int)__reduce_add_sync(0xffffffffu, lane < g.nsim ? (unsigned)g.active[lane] : 0u);
    if (g.it >= t_run || nact == 0) {
      if (lane == 0) g.state = kDone;
      if (lane == 0) g.nvalid = 0;
      __syncwarp();
      return;
    }
  }
  for (int i = lane; i < kHistLen; i += 32) g.hist[i] = 0;
  if (kind == 1) {
#pragma unroll 2
    for (int e = lane; e < g.nsim * N; e += 32) {
      const int gi = e / N, j = e - gi * N;
      if (g.active[gi]) {
        const float xb = g.XB[gi][j], w = g.U[gi][g.ord[gi][N]][j];
#pragma unroll
        for (int q = 0; q < 4; ++q) g.XT[gi][q][j] = trial_coord(q, xb, w);
      }
    }
  }
  if (lane == 0) g.kind = kind;
  if (lane == 0) g.state = kPending;
  if (lane == 0 && kind == 1) g.evals += trials<N>() * nact;
  __syncwarp();
}

// Counting sort of a group's freshly set-up wave by pulse-end time, by the
// warp that set it up: lane l keys candidates l, l + 32, ..., the histogram
// (cleared by next_wave) is scanned by the same warp, and afterwards
// g.perm[0 .. g.nvalid) lists the candidates in key order.
template <int G, int N>
__device__ __forceinline__ void order_wave(GroupSmem<G, N>& g, const SacStage& V, const SearchParams& P, int lane) {
  constexpr int R = wave_per_lane<G, N>();
  static_assert(G * trials<N>() <= 32 * R, "every candidate keyed");
  static_assert(G * trials<N>() < (1 << 16), "bin rank in 16 bits");
  constexpr int kPwCoord = search_coord<N>(kPw);   // -1: pulse width held at the centre
  const int ncand = (g.kind == 0 ? verts<N>() : trials<N>()) * g.nsim;
#pragma unroll 4
  for (int r = 0; r < R; ++r) {
    const int c = lane + 32 * r;
    int key = -1;
    if (c < ncand) {
      if (g.kind == 0) {
        const int gi = c / verts<N>(), v = c - gi * verts<N>();
        key = switch_key(kPwCoord < 0 ? 0.0f : g.U[gi][v][kPwCoord < 0 ? 0 : kPwCoord], V.pc[kPw], P.lnlo,
                         P.lnhi, V.sc);
      } else {
        const int gi = c / trials<N>(), q = c - gi * trials<N>();
        if (g.active[gi]) {
          const float* a;
          const float* bb;
          trial_rows(g, gi, q, a, bb);
          const int jp = kPwCoord < 0 ? 0 : kPwCoord;
          key = switch_key(kPwCoord < 0 ? 0.0f : shrink_coord(a[jp], bb[jp]), V.pc[kPw], P.lnlo, P.lnhi, V.sc);
        }
      }
    }
    if (c < G * trials<N>()) g.kr[c] = key >= 0 ? (key << 16) | atomicAdd(&g.hist[hist_slot(key)], 1) : -1;
  }
  __syncwarp();
  {
    // lane l owns bins [per l, per l + per), stored at hist_slot(per l + i) =
    // (per + 1) l + i: one padding word per lane keeps the lanes on distinct
    // banks; the counts are read once into registers
    constexpr int per = kHistPer;
    static_assert(per * 32 == kSortBins && (per + 1) * 31 + per <= kHistLen, "histogram layout");
    int* h = g.hist + lane * (per + 1);
    int v[per];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) {
      v[i] = h[i];
      sum += v[i];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    int run = incl - sum;
#pragma unroll
    for (int i = 0; i < per; ++i) {
      h[i] = run;
      run += v[i];
    }
    if (lane == 31) g.nvalid = incl;
  }
  __syncwarp();
#pragma unroll 4
  for (int c = lane; c < ncand; c += 32) {
    const int kr = g.kr[c];
    if (kr >= 0) g.perm[g.hist[hist_slot(kr >> 16)] + (kr & 0xffff)] = (unsigned short)c;
  }
  __syncwarp();
}

__device__ __forceinline__ int vload(const int& x) { return *reinterpret_cast<const volatile int*>(&x); }

// Make a group's set-up wave (or its end) visible to the block's warps.  The
// wave's data is written before; then the done count and the claim word are
// reset for the next sequence number, then the published word (sequence,
// chunks) is written, with block-scope fences between, so a warp that claims a
// chunk of this sequence sees the wave.  A finished group publishes 0 chunks.
template <int G, int N>
__device__ __forceinline__ void publish_wave(GroupSmem<G, N>& g, int lane) {
  __syncwarp();
  __threadfence_block();
  // every lane computes the words; lane 0 alone stores them (single
  // predicated stores, so the warp never splits around them)
  const int seq = ((vload(g.pub) >> 16) + 1) & 0x7fff;
  const int n = g.state == kDone ? 0 : (g.nvalid + 31) >> 5;
  if (lane == 0) atomicExch(&g.done, 0);
  if (lane == 0) atomicExch(&g.claim, seq << 16);
  __threadfence_block();
  if (lane == 0) atomicExch(&g.pub, (seq << 16) | n);
  __syncwarp();
}

// Claim the next chunk of a group's published wave, by the whole warp with
// uniform control flow: lane 0 alone reads the words and attempts the
// compare-and-swap (single predicated instructions) and every value is
// broadcast, so the warp stays converged.  Returns the chunk index and its
// wave's chunk count, or -1 when the wave has no chunk left, the claim word
// belongs to another sequence (a wave being published), or other warps kept
// winning the race (the caller tries again).
template <int G, int N>
__device__ __forceinline__ int try_claim(GroupSmem<G, N>& g, int lane, int& nchunks) {
  int pub = 0, old = 0;
  if (lane == 0) pub = vload(g.pub);
  pub = __shfl_sync(0xffffffffu, pub, 0);
  const int n = pub & 0xffff;
  if (n == 0) return -1;
  const int want = pub & ~0xffff;
  if (lane == 0) old = vload(g.claim);
  old = __shfl_sync(0xffffffffu, old, 0);
#pragma unroll 1
  for (int t = 0; t < 64; ++t) {
    if ((old & ~0xffff) != want || (old & 0xffff) >= n) return -1;
    int prev = 0;
    if (lane == 0) prev = atomicCAS(&g.claim, old, old + 1);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev == old) {
      __threadfence_block();
      nchunks = n;
      return old & 0xffff;
    }
    old = prev;
  }
  return -1;
}

// The warp that completed a group's wave: Nelder-Mead decisions on the values
// just computed (ranking of the initial simplices, or the Lagarias step of
// every active simplex), then the group's next wave, its ordering and its
// publication.
template <int G, int N>
__device__ __forceinline__ void advance_group(GroupSmem<G, N>& g, const SacStage& V, const SearchParams& P, int lane,
                                              int t_run) {
  if (g.kind == 0) {
    init_rank<G, N>(g, lane, P.tolx, P.tolf);
  } else {
    decide_group<G, N>(g, lane, P.tolx, P.tolf);
    if (lane == 0) g.it += 1;
    __syncwarp();
  }
  next_wave<G, N>(g, 1, t_run, lane);
  if (g.state == kPending) order_wave<G, N>(g, V, P, lane);
  publish_wave<G, N>(g, lane);
}

// Evaluate the candidate at position pos (key order) of a group's pending
// wave; qs is the calling thread's propagator slot.  Returns 1 when that
// candidate's pulse ends inside the window (its pulse-end sample was
// integrated substep by substep), else 0 (also for pos past the wave).
template <int G, int N, bool LEAN, bool PACK>
__device__ __forceinline__ int eval_candidate(GroupSmem<G, N>& g, const SacStage& S, const SearchParams& P,
                                              const float* z, float* qs, int pos) {
  constexpr int NT = search_threads<G, N>();
  const unsigned live = __ballot_sync(0xffffffffu, pos < g.nvalid);   // the lanes that walk
  if (pos >= g.nvalid) return 0;
  int pe = 0;
  const SacConst& sc = S.sc;
  const float sum0 = S.st.sum0, c0 = S.st.c0;
  const int c = g.perm[pos];
  static_assert(!LEAN || N == N, "register-lean walk: 18 coordinates only");
  // both kinds of wave through one walk: a vertex is the row pair (v, v), for
  // which a + (a - a) / 2 = a exactly
  const float* a;
  const float* bb;
  float* out;
  if (g.kind == 0) {
    const int gi = c / verts<N>(), v = c - gi * verts<N>();
    a = bb = g.U[gi][v];
    out = &g.F[gi][v];
  } else {
    const int gi = c / trials<N>(), q = c - gi * trials<N>();
    trial_rows(g, gi, q, a, bb);
    out = &g.FT[gi][q];
  }
  if constexpr (LEAN) {
    const ULinSrc src{a, bb, true, S.pc, P.lnlo, P.lnhi};
    *out = objective_lean(src, sc, z, sum0, c0, &pe);
  } else {
    float u[N];
#pragma unroll
    for (int j = 0; j < N; ++j) u[j] = shrink_coord(a[j], bb[j]);
    *out = eval_u<N, PACK>(u, S.pc, P.lnlo, P.lnhi, sc, z, sum0, c0, qs, NT, &pe, live);
  }
  return pe;
}

// Group of a unit's simplex sg and its index in that group: group h holds the
// unit's simplices [group_start(h), group_start(h + 1)).
template <int G, int NG>
__device__ __forceinline__ int group_start(int h, int nunit, bool balanced) {
  return balanced ? (nunit * h) / NG : min(nunit, h * G);
}
template <int G, int NG>
__device__ __forceinline__ int group_of(int sg, int nunit, bool balanced, int& gi) {
  int h = 0;
#pragma unroll
  for (int t = 1; t < NG; ++t)
    if (sg >= group_start<G, NG>(t, nunit, balanced)) h = t;
  gi = sg - group_start<G, NG>(h, nunit, balanced);
  return h;
}

template <int G, int N, int NG, int MINB, bool LEAN, bool PACK>
__global__ void __launch_bounds__(search_threads<G, N>(), MINB) k_search(SearchParams P) {
  constexpr int NT = search_threads<G, N>();
  static_assert(NG >= 2 && NG <= kSearchWarps, "one warp sets up each group's first wave");
  extern __shared__ __align__(128) unsigned char smraw[];
  SearchSmem<G, N, NG>& S = *reinterpret_cast<SearchSmem<G, N, NG>*>(smraw);
  float* yraw = reinterpret_cast<float*>(smraw + ((sizeof(SearchSmem<G, N, NG>) + 127) / 128) * 128);
  float* z = yraw + P.lcap;
  float* qslot = z + P.lcap;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    mbar_init(&S.bar, 1);
    fence_mbar_init();
    S.cur_b = -1;
    S.abort = 0;
  }
  __syncthreads();
  uint32_t phase = 0;

  for (;;) {
    if (tid == 0) S.unit = atomicAdd(P.counter, 1);
    __syncthreads();
    const int unit = S.unit;
    if (unit >= P.n_units) break;
    const int2 un = P.slot_list ? make_int2(P.slot_list[unit / P.ngroups], unit % P.ngroups) : P.units[unit];
    const int b = un.x, g0 = un.y;
    if (b != S.cur_b) {
      const DevSac d = P.sacs[b];
      if (!stage_trace(d, P.traces, yraw, z, &S.bar, phase, &S.sv.st)) {
        if (tid == 0) raise_error(P.err, kErrWaitTimeout);
        return;
      }
      if (tid < kNumParams) S.sv.pc[tid] = P.pc[(size_t)b * kNumParams + tid];
      if (tid == 0) {
        S.sv.sc = sac_const(d);
        S.cur_b = b;
      }
      __syncthreads();
    }
    // this unit's simplices: units of NG G (the last takes the rest), or, with
    // P.balanced, the saccade's S simplices split evenly over its P.ngroups
    // units; within the unit, groups of G in order, or an even split
    int s0, nunit;
    const bool bal = P.balanced != 0;
    if (bal) {
      s0 = (int)(((long long)g0 * P.S) / P.ngroups);
      nunit = (int)(((long long)(g0 + 1) * P.S) / P.ngroups) - s0;   // <= NG G
    } else {
      s0 = g0 * NG * G;
      nunit = min(NG * G, P.S - s0);
    }
    // resumable mode (serving): iterations already done by this saccade and
    // this launch's share; the simplex state lives in HBM between launches
    const int it0 = P.state ? P.progress[b] : 0;
    const int t_run = P.state ? min(P.round_iters, P.T - it0) : P.T;
    if (tid < NG) {
      GroupSmem<G, N>& g = S.grp[tid];
      g.nsim = group_start<G, NG>(tid + 1, nunit, bal) - group_start<G, NG>(tid, nunit, bal);
      g.it = 0;
      g.evals = 0;
      g.pe = 0;
      g.nvalid = 0;
      g.state = g.nsim > 0 ? kPending : kDone;
      g.pub = 0;
      g.claim = 0;
      g.done = 0;
    }
    if (it0 > 0) {
      // restore the simplices: vertices, values, centroid, order, flags
      const float* gstate = P.state + ((size_t)b * P.S + (size_t)s0) * state_floats<N>();
      for (int idx = tid; idx < nunit * state_floats<N>(); idx += NT) {
        const int sg = idx / state_floats<N>(), r = idx - sg * state_floats<N>();
        int gi;
        GroupSmem<G, N>& g = S.grp[group_of<G, NG>(sg, nunit, bal, gi)];
        const float v = gstate[idx];
        if (r < verts<N>() * N) (&g.U[gi][0][0])[r] = v;
        else if (r < verts<N>() * N + verts<N>()) g.F[gi][r - verts<N>() * N] = v;
        else if (r < verts<N>() * N + verts<N>() + N) g.XB[gi][r - verts<N>() * N - verts<N>()] = v;
        else if (r < verts<N>() * N + 2 * verts<N>() + N) g.ord[gi][r - verts<N>() * N - verts<N>() - N] = (unsigned char)__float_as_int(v);
        else if (r == state_floats<N>() - 2) g.active[gi] = __float_as_int(v);
        else if (r == state_floats<N>() - 1) g.iters[gi] = __float_as_int(v);
      }
    } else {
      // ---- initial simplices: centre (Philox for starts >= 1) + step e_i
      constexpr int kBlk = (N + 3) / 4;   // Philox blocks of 4 coordinates
      for (int t5 = tid; t5 < kBlk * nunit; t5 += NT) {
        const int sg = t5 / kBlk, blk = t5 - sg * kBlk;
        int gi;
        GroupSmem<G, N>& g = S.grp[group_of<G, NG>(sg, nunit, bal, gi)];
        const int s = s0 + sg;
        uint32_t r[4] = {0u, 0u, 0u, 0u};
        if (s != 0) philox4x32_10((uint32_t)P.sac_index[b], (uint32_t)s, (uint32_t)blk, 0u, P.seed_lo, P.seed_hi, r);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * blk + q;
          if (j < N)
            g.U[gi][0][j] = s == 0 ? 0.0f : P.lnlo + (P.lnhi - P.lnlo) * ((float)(r[q] >> 8) * (1.0f / 16777216.0f));
        }
      }
      __syncthreads();
      for (int idx = tid; idx < nunit * N * N; idx += NT) {
        const int sg = idx / (N * N);
        int gi;
        GroupSmem<G, N>& g = S.grp[group_of<G, NG>(sg, nunit, bal, gi)];
        const int rem = idx - sg * N * N;
        const int v = rem / N + 1, j = rem - (v - 1) * N;
        float x = g.U[gi][0][j];
        if (j == v - 1) x += P.step;
        g.U[gi][v][j] = x;
      }
    }
    __syncthreads();
    // warp h < NG sets up, orders and publishes group h's first wave
    if (warp < NG) {
      GroupSmem<G, N>& g = S.grp[warp];
      if (g.nsim > 0) {
        if (it0 == 0 && lane == 0) g.evals = verts<N>() * g.nsim;
        __syncwarp();
        next_wave<G, N>(g, it0 > 0 ? 1 : 0, t_run, lane);
        if (g.state == kPending) order_wave<G, N>(g, S.sv, P, lane);
        publish_wave<G, N>(g, lane);
      }
    }
    __syncthreads();

    // ---- steps, with no block barrier: each warp claims 32-candidate chunks
    // of any group's published wave (the group it worked on last first, then
    // the following ones in turn), evaluates them and counts them done; the
    // warp that completes a wave takes that group's decisions and publishes
    // its next wave while the other warps work on the other groups' waves.
    // All warps start on group 0, so the groups' waves complete one after
    // another and each group's decisions overlap the evaluation of the
    // others'.  Every decision to leave the loop is taken on lane 0 and
    // broadcast; a warp that finds nothing to claim waits, for at most
    // kMaxIdleCycles, until a wave is published or every group is done.
    int pref = 0;
    long long idle_since = -1;
#pragma unroll 1
    for (;;) {
      int gsel = -1, ch = -1, nch = 0;
#pragma unroll 1
      for (int t = 0; t < NG && ch < 0; ++t) {
        const int h = pref + t < NG ? pref + t : pref + t - NG;
        ch = try_claim<G, N>(S.grp[h], lane, nch);
        if (ch >= 0) gsel = h;
      }
      if (ch >= 0) {
        __syncwarp();   // orders lane 0's acquire of the wave before every lane's reads
        GroupSmem<G, N>& g = S.grp[gsel];
        const int npe = __popc(__ballot_sync(0xffffffffu,
                                             eval_candidate<G, N, LEAN, PACK>(g, S.sv, P, z, qslot + tid, ch * 32 + lane)));
        __syncwarp();
        __threadfence_block();   // the chunk's values before its done count
        if (lane == 0 && npe) atomicAdd(&g.pe, npe);
        int done_before = 0;
        if (lane == 0) done_before = atomicAdd(&g.done, 1);
        done_before = __shfl_sync(0xffffffffu, done_before, 0);
        const bool last = done_before == nch - 1;
        if (last) __threadfence_block();
        __syncwarp();
        if (last) {
          advance_group<G, N>(g, S.sv, P, lane, t_run);
          pref = gsel + 1 < NG ? gsel + 1 : 0;
        } else {
          pref = gsel;
        }
        idle_since = -1;
        continue;
      }
      // nothing to claim: 1 = every group done or the block aborts, 2 = waited
      // too long; lane 0's view of the words and the clock decides for the warp
      int fin = 0;
      {
        const long long now = clock64();
        if (idle_since < 0) idle_since = now;
        bool all_done = true;
#pragma unroll
        for (int h = 0; h < NG; ++h) all_done = all_done && vload(S.grp[h].state) == kDone;
        fin = (vload(S.abort) || all_done) ? 1 : (now - idle_since > kMaxIdleCycles ? 2 : 0);
      }
      fin = __shfl_sync(0xffffffffu, fin, 0);
      if (fin == 2) {
        if (lane == 0) raise_error(P.err, kErrWaitTimeout);
        if (lane == 0) atomicExch(&S.abort, 1);
        break;
      }
      if (fin) break;
      __nanosleep(128);
    }
    __syncthreads();
    if (S.abort) return;

    if (P.state) {
      // save the simplices for the next launch
      float* gstate = P.state + ((size_t)b * P.S + (size_t)s0) * state_floats<N>();
      for (int idx = tid; idx < nunit * state_floats<N>(); idx += NT) {
        const int sg = idx / state_floats<N>(), r = idx - sg * state_floats<N>();
        int gi;
        const GroupSmem<G, N>& g = S.grp[group_of<G, NG>(sg, nunit, bal, gi)];
        float v;
        if (r < verts<N>() * N) v = (&g.U[gi][0][0])[r];
        else if (r < verts<N>() * N + verts<N>()) v = g.F[gi][r - verts<N>() * N];
        else if (r < verts<N>() * N + verts<N>() + N) v = g.XB[gi][r - verts<N>() * N - verts<N>()];
        else if (r < verts<N>() * N + 2 * verts<N>() + N) v = __int_as_float((int)g.ord[gi][r - verts<N>() * N - verts<N>() - N]);
        else if (r == state_floats<N>() - 2) v = __int_as_float(g.active[gi]);
        else if (r == state_floats<N>() - 1) v = __int_as_float(g.iters[gi]);
        else v = 0.0f;
        gstate[idx] = v;
      }
    }

    // ---- unit result: lowest value, ties to the lowest simplex index
    if (tid < 32) {
      float* rec = P.unit_best + (size_t)(P.slot_list ? b * P.ngroups + g0 : unit) * kUnitRec;
      float f = INFINITY;
      int best = 0x7fffffff;
      for (int sg = lane; sg < nunit; sg += 32) {
        int gi;
        const GroupSmem<G, N>& g = S.grp[group_of<G, NG>(sg, nunit, bal, gi)];
        const float fv = g.F[gi][g.ord[gi][0]];
        if (fv < f || (fv == f && sg < best)) { f = fv; best = sg; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float f2 = __shfl_xor_sync(0xffffffffu, f, o);
        const int b2 = __shfl_xor_sync(0xffffffffu, best, o);
        if (f2 < f || (f2 == f && b2 < best)) { f = f2; best = b2; }
      }
      const int evals_prev = it0 > 0 ? __float_as_int(rec[3]) : 0;
      const int pe_prev = it0 > 0 ? __float_as_int(rec[22]) : 0;
      int evals = 0, pes = 0;
      for (int h = 0; h < NG; ++h) {
        evals += S.grp[h].evals;
        pes += S.grp[h].pe;
      }
      __syncwarp();
      if (best < nunit) {
        int gi;
        const GroupSmem<G, N>& g = S.grp[group_of<G, NG>(best, nunit, bal, gi)];
        if (lane < N) rec[4 + lane] = g.U[gi][g.ord[gi][0]][lane];
        if (lane == 0) {
          rec[0] = f;
          rec[1] = __int_as_float(s0 + best);
          rec[2] = __int_as_float(g.iters[gi]);
          rec[3] = __int_as_float(evals_prev + evals);
          rec[22] = __int_as_float(pe_prev + pes);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ finalize
// FP64 re-computation of the winner's error (the serial check next to the
// parallel value, as Fig. 4's CPU_check column).  The same RK4 map is applied
// in double precision as dense 6x6 step matrices: within one input phase one
// RK4 step of e' = A e is e <- e + Q e with Q = hA(I + hA/2(I + hA/3(I + hA/4))),
// raised to one sample interval by squaring; the pulse-end substep is split
// into two RK4 steps.  Independent of the FP32 search formulation (dense
// matrices, double precision, its own equilibria).
struct M6 {
  double a[6][6];
};

__device__ void m6_zero(M6& m) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) m.a[i][j] = 0.0;
}

// r = a + b + a b (increment form of (I + a)(I + b)); r may alias neither
__device__ void m6_mul_inc(const M6& a, const M6& b, M6& r) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = a.a[i][j] + b.a[i][j];
      for (int k = 0; k < 6; ++k) acc = fma(a.a[i][k], b.a[k][j], acc);
      r.a[i][j] = acc;
    }
}

// plant matrix of one phase (state theta, omega, x, y, Fa, Fn)
__device__ void plant_matrix64(const double* p, double ita, double itn, M6& A) {
  m6_zero(A);
  const double kp = p[kNcAg] + p[kNcAnt];
  const double iJ = 1.0 / p[kJ], iBa = 1.0 / p[kBAg], iBn = 1.0 / p[kBAnt];
  A.a[0][1] = 1.0;
  A.a[1][0] = -(p[kSeAg] + p[kSeAnt] + kp) * iJ;
  A.a[1][1] = -p[kBp] * iJ;
  A.a[1][2] = p[kSeAg] * iJ;
  A.a[1][3] = -p[kSeAnt] * iJ;
  A.a[2][0] = p[kSeAg] * iBa;
  A.a[2][2] = -(p[kSeAg] + p[kLtAg]) * iBa;
  A.a[2][4] = iBa;
  A.a[3][0] = -p[kSeAnt] * iBn;
  A.a[3][3] = -(p[kSeAnt] + p[kLtAnt]) * iBn;
  A.a[3][5] = iBn;
  A.a[4][4] = -ita;
  A.a[5][5] = -itn;
}

// Q = T4(hA) - I by Horner
__device__ void step_inc64(const M6& A, double h, M6& Q) {
  M6 W, T;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) W.a[i][j] = (i == j ? 1.0 : 0.0) + 0.25 * h * A.a[i][j];
  const double c[2] = {h / 3.0, 0.5 * h};
  for (int lev = 0; lev < 2; ++lev) {
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 6; ++k) acc = fma(A.a[i][k], W.a[k][j], acc);
        T.a[i][j] = (i == j ? 1.0 : 0.0) + c[lev] * acc;
      }
    W = T;
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc = fma(A.a[i][k], W.a[k][j], acc);
      Q.a[i][j] = h * acc;
    }
}

__device__ void pow_inc64(const M6& q, int n, M6& out) {
  M6 base = q, tmp;
  bool have = false;
  while (true) {
    if (n & 1) {
      if (have) { m6_mul_inc(out, base, tmp); out = tmp; }
      else { out = base; have = true; }
    }
    n >>= 1;
    if (!n) break;
    m6_mul_inc(base, base, tmp);
    base = tmp;
  }
}

__device__ void apply_inc64(const M6& q, double* e) {
  double n[6];
  for (int i = 0; i < 6; ++i) {
    double acc = e[i];
    for (int k = 0; k < 6; ++k) acc = fma(q.a[i][k], e[k], acc);
    n[i] = acc;
  }
  for (int i = 0; i < 6; ++i) e[i] = n[i];
}

// one RK4 step of length hs on e' = A e (Horner form of T4(hs A) e)
__device__ void rk4_vec64(const M6& A, double hs, double* e) {
  double w[6], v[6];
  for (int i = 0; i < 6; ++i) w[i] = e[i];
  const double c[4] = {0.25 * hs, hs / 3.0, 0.5 * hs, hs};
  for (int lev = 0; lev < 4; ++lev) {
    for (int i = 0; i < 6; ++i) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc = fma(A.a[i][k], w[k], acc);
      v[i] = acc;
    }
    for (int i = 0; i < 6; ++i) w[i] = fma(c[lev], v[i], e[i]);
  }
  for (int i = 0; i < 6; ++i) e[i] = w[i];
}

// equilibrium under constant active-state tensions (fa, fn), double
__device__ void equilibrium64(const double* p, double fa, double fn, double* s) {
  const double ag = p[kSeAg] / (p[kSeAg] + p[kLtAg]);
  const double an = p[kSeAnt] / (p[kSeAnt] + p[kLtAnt]);
  const double kp = p[kNcAg] + p[kNcAnt];
  const double th = (ag * fa - an * fn) / (kp + ag * p[kLtAg] + an * p[kLtAnt]);
  const double ta = ag * (fa - p[kLtAg] * th), tn = an * (fn + p[kLtAnt] * th);
  s[0] = th; s[1] = 0.0;
  s[2] = th + ta / p[kSeAg];
  s[3] = tn / p[kSeAnt] - th;
  s[4] = fa; s[5] = fn;
}

__device__ void step_levels64(const double* p, double th, double* fa, double* fn) {
  const double ta = p[kNcFix] + p[kNcAg] * th, tn = p[kNcFix] - p[kNcAnt] * th;
  *fa = ta * (1.0 + p[kLtAg] / p[kSeAg]) + p[kLtAg] * th;
  *fn = tn * (1.0 + p[kLtAnt] / p[kSeAnt]) - p[kLtAnt] * th;
}

// Mean squared and mean absolute error of the winner's trajectory, FP64.
__device__ void errors64(const float* pf, const DevSac& d, const float* y, double* mse, double* mae) {
  double p[kNumParams];
  for (int j = 0; j < kNumParams; ++j) p[j] = (double)pf[j];
  const double th0 = d.th0, thf = d.thf, sg = d.sign;
  // substeps refined for stiff candidates, the oracle's rule in double
  const double tmin = fmin(fmin(p[kTacAg], p[kTacAnt]), fmin(p[kTdeAg], p[kTdeAnt]));
  const double est = p[kBp] / p[kJ] + (p[kSeAg] + p[kLtAg]) / p[kBAg] + (p[kSeAnt] + p[kLtAnt]) / p[kBAnt] +
                     1000.0 / tmin;
  int nsub = d.nsub;
  double h = 1.0 / ((double)d.fs * nsub);
  for (int r = 0; r < kMaxRefine && !(h * est <= 2.5); ++r) {
    h *= 0.5;
    nsub *= 2;
  }
  double tau = p[kPw] * (double)d.fs * (double)nsub / 1000.0;
  if (!(tau >= 0.0)) tau = 0.0;
  if (tau > 1.0e9) tau = 1.0e9;
  const double fl = floor(tau);
  const double frac = tau - fl;
  double fa0, fn0, faf, fnf;
  step_levels64(p, th0, &fa0, &fn0);
  step_levels64(p, thf, &faf, &fnf);
  double s0[6], s1[6], s2[6];
  equilibrium64(p, fa0, fn0, s0);          // rest at th0
  equilibrium64(p, p[kNsacAg], p[kNsacAnt], s1);
  equilibrium64(p, faf, fnf, s2);          // rest at thf
  double s2e = 0.0, s1e = 0.0;
  const int kend = d.onset < d.L - 1 ? d.onset : d.L - 1;
  for (int k = 0; k <= kend; ++k) {       // at rest up to onset
    const double e = sg * th0 - (double)y[k];
    s2e += e * e;
    s1e += fabs(e);
  }
  const int ntot = d.L - 1 - d.onset;
  if (ntot > 0) {
    M6 A1, A2, Q1, Q2, P1, P2;
    plant_matrix64(p, 1000.0 / p[kTacAg], 1000.0 / p[kTdeAnt], A1);
    plant_matrix64(p, 1000.0 / p[kTdeAg], 1000.0 / p[kTacAnt], A2);
    step_inc64(A1, h, Q1);
    step_inc64(A2, h, Q2);
    pow_inc64(Q1, nsub, P1);
    pow_inc64(Q2, nsub, P2);
    long long n1;
    int jsw = 0;
    bool sw;
    if (fl >= (double)ntot * nsub) { n1 = ntot; sw = false; }
    else { const long long J = (long long)fl; n1 = J / nsub; jsw = (int)(J - n1 * nsub); sw = true; }
    double e[6];
    for (int i = 0; i < 6; ++i) e[i] = s0[i] - s1[i];
    int k = d.onset + 1;
    for (long long i = 0; i < n1; ++i, ++k) {
      apply_inc64(P1, e);
      const double r = sg * (s1[0] + e[0]) - (double)y[k];
      s2e += r * r;
      s1e += fabs(r);
    }
    if (sw) {
      for (int s = 0; s < jsw; ++s) apply_inc64(Q1, e);
      rk4_vec64(A1, frac * h, e);
      for (int i = 0; i < 6; ++i) e[i] += s1[i] - s2[i];
      rk4_vec64(A2, h - frac * h, e);
      for (int s = jsw + 1; s < nsub; ++s) apply_inc64(Q2, e);
      double r = sg * (s2[0] + e[0]) - (double)y[k];
      s2e += r * r;
      s1e += fabs(r);
      ++k;
      for (; k < d.L; ++k) {
        apply_inc64(P2, e);
        r = sg * (s2[0] + e[0]) - (double)y[k];
        s2e += r * r;
        s1e += fabs(r);
      }
    }
  }
  *mse = s2e / d.L;
  *mae = s1e / d.L;
}

template <int N>
__global__ void k_finalize(const DevSac* sacs, const float* traces, const float* pc, const int* ustart,
                           int ngroups, const float* unit_best, float lnlo, float lnhi, int n,
                           opmm_fit_result* out, const int* list) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = list ? list[i] : i;
  int w = -1, wsimp = 0x7fffffff, evals = 0, pe = 0;
  float wf = INFINITY;
  const int u0 = ustart ? ustart[b] : b * ngroups;   // slot-major records when no start table
  for (int u = u0; u < u0 + ngroups; ++u) {
    const float* rec = unit_best + (size_t)u * kUnitRec;
    const float f = rec[0];
    const int s = __float_as_int(rec[1]);
    evals += __float_as_int(rec[3]);
    pe += __float_as_int(rec[22]);
    if (w < 0 || f < wf || (f == wf && s < wsimp)) { w = u; wf = f; wsimp = s; }
  }
  opmm_fit_result r;
  const DevSac d = sacs[b];
  const float* rec = unit_best + (size_t)w * kUnitRec;
  {
    float p[kNumParams];
    u_to_p<N>(rec + 4, pc + (size_t)b * kNumParams, lnlo, lnhi, p);
    for (int j = 0; j < kNumParams; ++j) r.opc[j] = p[j];
  }
  r.f = wf;
  r.iterations_run = __float_as_int(rec[2]);
  r.winner = wsimp;
  r.evaluations = evals;
  r.pulse_end_evals = pe;
  r.reserved = 0;
  r.source = OPMM_SOURCE_PLAIN;
  if (isfinite(wf)) {
    double mse, mae;
    errors64(r.opc, d, traces + d.off, &mse, &mae);
    r.rms_deg = sqrt(mse);
    r.l1_deg = mae;
    r.status = 0;
  } else {
    r.rms_deg = INFINITY;
    r.l1_deg = INFINITY;
    r.status = 1;
  }
  out[i] = r;
}

// ------------------------------------------------------------------ refinement
// Gradient-based refinement after the search (Sec. 5 proposes gradient
// methods as the alternative to Nelder-Mead): Levenberg-Marquardt on the
// residual vector r_k = theta_k(u) - y_k of one saccade per block, in the
// search's ln coordinates, box and clamp.  One iteration: at a new point the
// Jacobian by central differences of step delta (2N trajectories, one per
// thread; a column whose two points are too stiff is zero), A = J^T J and
// g = J^T r (FP32 products, compensated sums); (A + lambda D) du = -g with
// D = diag(max(A_jj, 1e-9
// max_i A_ii)) solved by Cholesky in FP64; u' = clamp(u + du); accept when
// f(u') < f(u) (lambda / 10, floor 1e-12, new Jacobian), else lambda * 10
// (ceiling 1e12).  f = sum_k r_k^2 / L over every sample.  Stops early when
// A is zero or the system is not positive definite.  Trajectories (2N + 2
// rows of lcap floats) go to shared memory when they fit, else to a per-block
// scratch area in global memory.
constexpr int kRefineThreads = 64;

struct RowSink {
  float* out;
  __device__ __forceinline__ void emit(int k, float dth) { out[k] = dth; }
  __device__ __forceinline__ void block_end() {}
};

// theta_k - thf (positive frame) for every sample of the window into row;
// false (row untouched past onset) when the candidate is too stiff.
// qs: the calling thread's propagator slot in shared memory (stride
// kRefineThreads), so that the powering runs in place as in the search.
__device__ bool refine_row(const float (&p)[kNumParams], const SacConst& sc, float* row, int* pe, float* qs) {
  const int kend = min(sc.onset, sc.L - 1);
  for (int k = 0; k <= kend; ++k) row[k] = sc.th0 - sc.thf;
  RowSink s{row};
  return walk(p, sc, s, qs, kRefineThreads, true, pe) >= 0;
}

template <int N>
struct RefineSmem {
  double A[N * N];
  double M[N * N];   // damped system, factored in place
  double du[N];
  double inv[N];     // reciprocals of the factor's diagonal
  double g[N];
  double red[kRefineThreads];
  float u[N], ut[N];
  float pc[kNumParams];
  double f, ft, lambda;
  int bad[2 * N];
  int need_jac, go, trial_ok, cur, acc, evals, pe;
  SacConst sc;
  TraceStage st;
  uint64_t bar;
};

// Block sum of per-thread FP64 partials (all threads call it).
template <int N>
__device__ double refine_sum(RefineSmem<N>& S, double v) {
  S.red[threadIdx.x] = v;
  __syncthreads();
  for (int o = kRefineThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) S.red[threadIdx.x] += S.red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = S.red[0];
  __syncthreads();
  return r;
}

// f of a stored trajectory row against the staged trace (all threads).
template <int N>
__device__ double refine_f(RefineSmem<N>& S, const float* row, const float* z, int L) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < L; k += kRefineThreads) {
    const double e = (double)row[k] - (double)z[k];
    acc += e * e;
  }
  return refine_sum<N>(S, acc) / (double)L;
}

// rows_in_smem: the 2N + 2 trajectory rows live in dynamic shared memory after
// the staged trace (short windows; the dot products of J^T J then read shared
// memory), else in the per-block global scratch area.
template <int N>
__global__ void __launch_bounds__(kRefineThreads) k_refine(const DevSac* sacs, const float* traces, const float* pcs,
                                                            const float* start, int K, float lnlo, float lnhi,
                                                            float delta, float lambda0, int lcap, float* scratch,
                                                            int rows_in_smem, opmm_fit_result* out, unsigned* err) {
  __shared__ RefineSmem<N> S;
  extern __shared__ __align__(128) unsigned char smraw[];
  float* yraw = reinterpret_cast<float*>(smraw);
  float* z = yraw + lcap;
  float* qslot = z + lcap;                                  // kQSlotFloats x kRefineThreads
  const int b = blockIdx.x, tid = threadIdx.x;
  const DevSac d = sacs[b];
  float* rows = rows_in_smem ? qslot + kQSlotFloats * kRefineThreads
                             : scratch + (size_t)b * (2 * N + 2) * (size_t)lcap;
  if (tid == 0) {
    mbar_init(&S.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  if (!stage_trace(d, traces, yraw, z, &S.bar, phase, &S.st)) {
    if (tid == 0) raise_error(err, kErrWaitTimeout);
    return;
  }
  if (tid < kNumParams) S.pc[tid] = pcs[(size_t)b * kNumParams + tid];
  if (tid == 0) {
    S.sc = sac_const(d);
    S.lambda = lambda0;
    S.need_jac = 1;
    S.cur = 0;
    S.acc = 0;
    S.evals = 1;
    S.pe = 0;
  }
  __syncthreads();
  // start point: the coordinate of the first OPC entry each one scales
  if (tid < N) {
    int j0 = 0;
    for (int j = kNumParams - 1; j >= 0; --j)
      if (search_coord<N>(j) == tid) j0 = j;
    const float u = logf(start[(size_t)b * kNumParams + j0] / S.pc[j0]);
    S.u[tid] = fminf(fmaxf(u, lnlo), lnhi);
  }
  __syncthreads();
  const SacConst sc = S.sc;
  float* rcur[2] = {rows + (size_t)(2 * N) * lcap, rows + (size_t)(2 * N + 1) * lcap};
  if (tid == 0) {
    float p[kNumParams];
    u_to_p<N>(S.u, S.pc, lnlo, lnhi, p);
    int pe = 0;
    S.trial_ok = refine_row(p, sc, rcur[0], &pe, qslot + tid) ? 1 : 0;
    S.pe += pe;
  }
  __syncthreads();
  {
    const double f = refine_f<N>(S, rcur[0], z, sc.L);
    if (tid == 0) S.f = S.trial_ok && isfinite(f) ? f : INFINITY;
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < K; ++it) {
    if (!isfinite(S.f)) break;
    const float* r0 = rcur[S.cur];
    if (S.need_jac) {
      if (tid < 2 * N) {
        const int j = tid >> 1;
        float ut[N];
#pragma unroll
        for (int c = 0; c < N; ++c) ut[c] = S.u[c];
        ut[j] += (tid & 1) ? -delta : delta;
        float p[kNumParams];
        u_to_p<N>(ut, S.pc, lnlo, lnhi, p);
        int pe = 0;
        S.bad[tid] = refine_row(p, sc, rows + (size_t)tid * lcap, &pe, qslot + tid) ? 0 : 1;
        if (pe) atomicAdd(&S.pe, 1);
      }
      __syncthreads();
      // A (lower triangle) and g: one task per entry, FP64
      constexpr int kTasks = N * (N + 1) / 2 + N;
      // J columns in place of the plus rows (FP32); the products below sum
      // with compensation in FP32 (the GPU's FP64 rate is a small fraction of
      // its FP32 rate) and enter the FP64 solve
      const float inv2d = 1.0f / (2.0f * delta);
      for (int e = tid; e < N * sc.L; e += kRefineThreads) {
        const int j = e / sc.L, k = e - j * sc.L;
        float* jp = rows + (size_t)(2 * j) * lcap;
        jp[k] = (jp[k] - rows[(size_t)(2 * j + 1) * lcap + k]) * inv2d;
      }
      __syncthreads();
      for (int t = tid; t < kTasks; t += kRefineThreads) {
        int a, bb;
        const bool is_g = t >= N * (N + 1) / 2;
        if (is_g) {
          a = t - N * (N + 1) / 2;
          bb = -1;
        } else {
          a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
          while ((a + 1) * (a + 2) / 2 <= t) ++a;
          while (a * (a + 1) / 2 > t) --a;
          bb = t - a * (a + 1) / 2;
        }
        const bool za = S.bad[2 * a] || S.bad[2 * a + 1];
        const bool zb = bb >= 0 && (S.bad[2 * bb] || S.bad[2 * bb + 1]);
        double acc = 0.0;
        if (!za && !zb) {
          const float* ja = rows + (size_t)(2 * a) * lcap;
          const float* jb = is_g ? r0 : rows + (size_t)(2 * bb) * lcap;
          float sum = 0.0f, c = 0.0f;
          for (int k = 0; k < sc.L; ++k) {
            const float other = is_g ? jb[k] - z[k] : jb[k];
            const float y = fmaf(ja[k], other, -c);
            const float tt = sum + y;
            c = (tt - sum) - y;
            sum = tt;
          }
          acc = (double)sum - (double)c;
        }
        if (is_g) S.g[a] = acc;
        else S.A[a * N + bb] = S.A[bb * N + a] = acc;
      }
      __syncthreads();
      if (tid == 0) {
        S.need_jac = 0;
        S.evals += 2 * N;
      }
    }
    // damped normal equations in FP64 by warp 0: the Cholesky factor column by
    // column (every lane forms the diagonal, the rows below go over the lanes,
    // multiplied by the diagonal's reciprocal), then lane 0 substitutes and
    // simulates the trial point
    if (tid < 32) {
      double amax = 0.0;
      for (int j = 0; j < N; ++j) amax = S.A[j * N + j] > amax ? S.A[j * N + j] : amax;
      int go = amax > 0.0 ? 1 : 0;
      double* M = S.M;
      double* du = S.du;
      if (go) {
        for (int e = tid; e < N * N; e += 32) M[e] = S.A[e];
        __syncwarp();
        if (tid < N) {
          const double dj = S.A[tid * N + tid] > 1e-9 * amax ? S.A[tid * N + tid] : 1e-9 * amax;
          M[tid * N + tid] += S.lambda * dj;
        }
        __syncwarp();
        for (int j = 0; j < N; ++j) {
          double sjj = M[j * N + j];
          for (int k = 0; k < j; ++k) sjj -= M[j * N + k] * M[j * N + k];
          if (!(sjj > 0.0)) {
            go = 0;
            break;
          }
          const double ljj = sqrt(sjj), il = 1.0 / ljj;
          __syncwarp();
          if (tid == 0) {
            M[j * N + j] = ljj;
            S.inv[j] = il;
          }
          for (int i = j + 1 + tid; i < N; i += 32) {
            double t = M[i * N + j];
            for (int k = 0; k < j; ++k) t -= M[i * N + k] * M[j * N + k];
            M[i * N + j] = t * il;
          }
          __syncwarp();
        }
      }
      if (go && tid == 0) {
        for (int i = 0; i < N; ++i) {
          double t = -S.g[i];
          for (int k = 0; k < i; ++k) t -= M[i * N + k] * du[k];
          du[i] = t * S.inv[i];
        }
        for (int i = N - 1; i >= 0; --i) {
          double t = du[i];
          for (int k = i + 1; k < N; ++k) t -= M[k * N + i] * du[k];
          du[i] = t * S.inv[i];
        }
        for (int j = 0; j < N; ++j) {
          const double v = (double)S.u[j] + du[j];
          S.ut[j] = (float)(v < (double)lnlo ? (double)lnlo : (v > (double)lnhi ? (double)lnhi : v));
        }
        float p[kNumParams];
        u_to_p<N>(S.ut, S.pc, lnlo, lnhi, p);
        int pe = 0;
        S.trial_ok = refine_row(p, sc, rcur[S.cur ^ 1], &pe, qslot + tid) ? 1 : 0;
        S.pe += pe;
        S.evals += 1;
      }
      if (tid == 0) S.go = go;
    }
    __syncthreads();
    if (!S.go) break;
    {
      const double ft = refine_f<N>(S, rcur[S.cur ^ 1], z, sc.L);
      if (tid == 0) {
        const double f2 = S.trial_ok && isfinite(ft) ? ft : INFINITY;
        if (f2 < S.f) {
          for (int j = 0; j < N; ++j) S.u[j] = S.ut[j];
          S.f = f2;
          S.cur ^= 1;
          S.acc += 1;
          S.lambda = S.lambda / 10.0 > 1e-12 ? S.lambda / 10.0 : 1e-12;
          S.need_jac = 1;
        } else {
          S.lambda = S.lambda * 10.0 < 1e12 ? S.lambda * 10.0 : 1e12;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    opmm_fit_result r;
    float p[kNumParams];
    u_to_p<N>(S.u, S.pc, lnlo, lnhi, p);
    for (int j = 0; j < kNumParams; ++j) r.opc[j] = p[j];
    r.f = (float)S.f;
    r.iterations_run = S.acc;
    r.winner = 0;
    r.evaluations = S.evals;
    r.pulse_end_evals = S.pe;
    r.reserved = 0;
    r.source = OPMM_SOURCE_REFINED;
    // the FP64 check of the refined vector runs in k_refine_check
    r.rms_deg = 0.0;
    r.l1_deg = 0.0;
    r.status = isfinite(S.f) ? 0 : 1;
    out[b] = r;
  }
}

// FP64 re-computation of each refined vector's errors (as k_finalize does for
// the search), one thread per saccade spread over the SMs.
__global__ void k_refine_check(const DevSac* sacs, const float* traces, int n, opmm_fit_result* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  opmm_fit_result& r = out[i];
  if (r.status == 0) {
    const DevSac d = sacs[i];
    double mse, mae;
    errors64(r.opc, d, traces + d.off, &mse, &mae);
    r.rms_deg = sqrt(mse);
    r.l1_deg = mae;
  } else {
    r.rms_deg = INFINITY;
    r.l1_deg = INFINITY;
  }
}

// Allow kernel k the largest dynamic shared memory the device gives one of its
// blocks (the opt-in maximum less its static shared memory), after checking
// that `smem` fits.  The attribute belongs to the kernel for the whole process,
// so it is only ever raised to that fixed maximum: a call for a smaller size
// never lowers the limit under a launch that another plan, a request loop or a
// captured graph makes with a larger one.
template <class K>
static cudaError_t allow_dynamic_smem(K k, size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if ((size_t)optin < fa.sharedSizeBytes || smem > (size_t)optin - fa.sharedSizeBytes) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_refine(int dim, const DevSac* sacs, const float* traces, const float* pcs, const float* start,
                          int n, int K, float lnlo, float lnhi, float delta, float lambda0, int lcap, float* scratch,
                          opmm_fit_result* out, unsigned* err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // the trajectory rows go to shared memory when they fit in 96 KB (windows up
  // to about 600 samples with 18 coordinates), leaving room for two blocks
  const size_t rows_bytes = (2 * (size_t)dim + 2) * (size_t)lcap * sizeof(float);
  const int in_smem = rows_bytes <= (size_t)96 * 1024 ? 1 : 0;
  const size_t smem = 2 * (size_t)lcap * sizeof(float) + (size_t)kQSlotFloats * kRefineThreads * sizeof(float) +
                      (in_smem ? rows_bytes : 0);
  if (dim == 9) {
    cudaError_t e = allow_dynamic_smem(k_refine<9>, smem);
    if (e != cudaSuccess) return e;
    k_refine<9><<<n, kRefineThreads, smem, st>>>(sacs, traces, pcs, start, K, lnlo, lnhi, delta, lambda0, lcap,
                                                 scratch, in_smem, out, err);
  } else if (dim == kNumParams) {
    cudaError_t e = allow_dynamic_smem(k_refine<kNumParams>, smem);
    if (e != cudaSuccess) return e;
    k_refine<kNumParams><<<n, kRefineThreads, smem, st>>>(sacs, traces, pcs, start, K, lnlo, lnhi, delta, lambda0,
                                                          lcap, scratch, in_smem, out, err);
  } else {
    return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_refine_check<<<(n + 3) / 4, 4, 0, st>>>(sacs, traces, n, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ serving
// Place newly admitted requests into their slots: descriptor (offset rebased
// to the slot's trace area), trace, box centre; progress reset.
__global__ void k_admit(const DevSac* new_sacs, const float* new_traces, const float* new_pc, const int* slots, int n,
                        DevSac* sacs, float* traces, float* pc, int* progress, int slot_stride) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int s = slots[i];
  DevSac d = new_sacs[i];
  const long long src = d.off;
  d.off = (long long)s * slot_stride;
  const int lp = (d.L + 3) & ~3;
  for (int k = threadIdx.x; k < lp; k += blockDim.x) traces[d.off + k] = k < d.L ? new_traces[src + k] : 0.0f;
  if (threadIdx.x < kNumParams) pc[(size_t)s * kNumParams + threadIdx.x] = new_pc[(size_t)i * kNumParams + threadIdx.x];
  if (threadIdx.x == 0) {
    sacs[s] = d;
    progress[s] = 0;
  }
}

// Iterations done after a scheduling round.
__global__ void k_advance(const int* slots, int n, int* progress, int iters, int T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = slots[i];
  progress[s] = min(T, progress[s] + iters);
}

cudaError_t launch_admit(const DevSac* new_sacs, const float* new_traces, const float* new_pc, const int* slots, int n,
                         DevSac* sacs, float* traces, float* pc, int* progress, int slot_stride, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_admit<<<n, 128, 0, st>>>(new_sacs, new_traces, new_pc, slots, n, sacs, traces, pc, progress, slot_stride);
  return cudaGetLastError();
}

cudaError_t launch_advance(const int* slots, int n, int* progress, int iters, int T, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_advance<<<(n + 127) / 128, 128, 0, st>>>(slots, n, progress, iters, T);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launch wrappers
cudaError_t launch_gather(const float* const* src, const DevSac* sacs, float* dst, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<n, 128, 0, st>>>(src, sacs, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_nominal(const DevSac* sacs, int n, int pulse_mode, const float* init_opc, float* pc,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (n * 32 + threads - 1) / threads;
  k_nominal<<<blocks, threads, 0, st>>>(sacs, n, pulse_mode, init_opc, pc);
  return cudaGetLastError();
}

cudaError_t launch_simulate(const float* opc, int n, const DevSac* sacs, const int* sac_of,
                            const long long* out_off, float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_simulate<<<(n + 127) / 128, 128, 0, st>>>(opc, n, sacs, sac_of, out_off, out);
  return cudaGetLastError();
}

cudaError_t launch_score(const float* opc, int m, const DevSac* sac, int L, const float* traces, float* f,
                         unsigned* err, int num_sms, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int threads = 256;
  int blocks = (m + threads - 1) / threads;
  if (blocks > 4 * num_sms) blocks = 4 * num_sms;
  const size_t smem = 2 * (size_t)((L + 3) & ~3) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dynamic_smem(k_score, smem);
    if (e != cudaSuccess) return e;
  }
  k_score<<<blocks, threads, smem, st>>>(opc, m, sac, traces, f, err);
  return cudaGetLastError();
}

// Launch-shape variants of the search kernel: simplices per group G, groups
// per block NG (a block runs a unit of NG G simplices), the search
// coordinates N (18, or 9 for the 9-parameter model), the minimum resident
// blocks per SM the register allocation is bounded for, and the walk: the
// register-lean walk, or the packed sample update (two row FMAs per packed
// FP32 instruction, the same arithmetic), or neither.  The host sees the unit
// size (simplices per block), N and the walk.  More groups per block keep
// more waves open, so that the warps always find chunks to claim while a
// group's decisions are taken.
struct SearchVariantDesc { int G, N, NG, minb, lean, pack; };
static const SearchVariantDesc kVariants[] = {
    {16, 18, 2, 1, 0, 0}, {16, 18, 2, 1, 1, 0}, {8, 18, 2, 1, 0, 0}, {32, 18, 2, 1, 0, 0}, {27, 9, 2, 1, 0, 0},
    {16, 18, 4, 1, 0, 0}, {27, 9, 4, 1, 0, 0},  {24, 18, 3, 1, 0, 0}, {16, 18, 2, 1, 0, 1}, {32, 18, 2, 1, 0, 1},
    {16, 18, 4, 1, 0, 1}, {24, 18, 3, 1, 0, 1}, {27, 9, 4, 1, 0, 1}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

static bool variant_ok(int v) { return v >= 0 && v < kNumVariants; }
int search_variant_count() { return kNumVariants; }
int search_variant_g(int v) { return variant_ok(v) ? kVariants[v].NG * kVariants[v].G : 0; }
int search_variant_dim(int v) { return variant_ok(v) ? kVariants[v].N : 0; }
int search_variant_minb(int v) { return variant_ok(v) ? kVariants[v].minb : 0; }
int search_variant_lean(int v) { return variant_ok(v) ? kVariants[v].lean : 0; }
int search_variant_pack(int v) { return variant_ok(v) ? kVariants[v].pack : 0; }
int search_variant_for(int unit, int dim) {
  for (int v = 0; v < kNumVariants; ++v)
    if (kVariants[v].NG * kVariants[v].G == unit && kVariants[v].N == dim) return v;
  return -1;
}

template <int G, int N, int NG, int MINB, bool LEAN, bool PACK>
static cudaError_t occ_v(int lcap, int* bps) {
  const size_t smem = search_smem_bytes<G, N, NG>(lcap);
  cudaError_t e = allow_dynamic_smem(k_search<G, N, NG, MINB, LEAN, PACK>, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_search<G, N, NG, MINB, LEAN, PACK>, search_threads<G, N>(),
                                                       smem);
}

// The dynamic shared-memory attribute is raised to its maximum by
// search_occupancy_v(), which the host calls for the same variant before any
// launch or graph capture.
template <int G, int N, int NG, int MINB, bool LEAN, bool PACK>
static cudaError_t launch_v(const SearchParams& P, int blocks_per_sm, int num_sms, cudaStream_t st) {
  const size_t smem = search_smem_bytes<G, N, NG>(P.lcap);
  k_search<G, N, NG, MINB, LEAN, PACK><<<blocks_per_sm * num_sms, search_threads<G, N>(), smem, st>>>(P);
  return cudaGetLastError();
}

template <int G, int N, int NG, int MINB, bool LEAN, bool PACK>
static int threads_v() { return search_threads<G, N>(); }

template <int G, int N, int NG, int MINB, bool LEAN, bool PACK>
static size_t smem_v(int lcap) { return search_smem_bytes<G, N, NG>(lcap); }

#define OPMM_VARIANT_SWITCH(v, CALL, BAD)             \
  switch (v) {                                        \
    case 0: return CALL(16, 18, 2, 1, false, false);  \
    case 1: return CALL(16, 18, 2, 1, true, false);   \
    case 2: return CALL(8, 18, 2, 1, false, false);   \
    case 3: return CALL(32, 18, 2, 1, false, false);  \
    case 4: return CALL(27, 9, 2, 1, false, false);   \
    case 5: return CALL(16, 18, 4, 1, false, false);  \
    case 6: return CALL(27, 9, 4, 1, false, false);   \
    case 7: return CALL(24, 18, 3, 1, false, false);  \
    case 8: return CALL(16, 18, 2, 1, false, true);   \
    case 9: return CALL(32, 18, 2, 1, false, true);   \
    case 10: return CALL(16, 18, 4, 1, false, true);  \
    case 11: return CALL(24, 18, 3, 1, false, true);  \
    case 12: return CALL(27, 9, 4, 1, false, true);   \
    default: return BAD;                              \
  }

cudaError_t search_occupancy_v(int v, int lcap, int* blocks_per_sm) {
#define OCC_CALL(G, N, NG, M, L, K) occ_v<G, N, NG, M, L, K>(lcap, blocks_per_sm)
  OPMM_VARIANT_SWITCH(v, OCC_CALL, cudaErrorInvalidValue)
#undef OCC_CALL
}

cudaError_t launch_search_v(int v, const SearchParams& P, int blocks_per_sm, int num_sms, cudaStream_t st) {
#define LAUNCH_CALL(G, N, NG, M, L, K) launch_v<G, N, NG, M, L, K>(P, blocks_per_sm, num_sms, st)
  OPMM_VARIANT_SWITCH(v, LAUNCH_CALL, cudaErrorInvalidValue)
#undef LAUNCH_CALL
}

// Threads and dynamic shared memory of a block of variant v.
int search_variant_threads(int v) {
#define THREADS_CALL(G, N, NG, M, L, K) threads_v<G, N, NG, M, L, K>()
  OPMM_VARIANT_SWITCH(v, THREADS_CALL, 0)
#undef THREADS_CALL
}

size_t search_variant_smem(int v, int lcap) {
#define SMEM_CALL(G, N, NG, M, L, K) smem_v<G, N, NG, M, L, K>(lcap)
  OPMM_VARIANT_SWITCH(v, SMEM_CALL, (size_t)0)
#undef SMEM_CALL
}

// Entry points for a fixed 18-coordinate unit size (static fit).
cudaError_t search_occupancy(int unit, int lcap, int* blocks_per_sm) {
  return search_occupancy_v(search_variant_for(unit, kNumParams), lcap, blocks_per_sm);
}

cudaError_t launch_search(int unit, const SearchParams& P, int blocks_per_sm, int num_sms, cudaStream_t st) {
  return launch_search_v(search_variant_for(unit, kNumParams), P, blocks_per_sm, num_sms, st);
}

cudaError_t launch_finalize(const DevSac* sacs, const float* traces, const float* pc, const int* ustart,
                            int ngroups, const float* unit_best, float lnlo, float lnhi, int n,
                            opmm_fit_result* out, cudaStream_t st, const int* list, int dim) {
  if (n <= 0) return cudaSuccess;
  // the FP64 recomputation is latency bound per thread and the FP64 pipe is
  // narrow: spread the saccades over all SMs, a few threads per block
  if (dim == 9)
    k_finalize<9><<<(n + 3) / 4, 4, 0, st>>>(sacs, traces, pc, ustart, ngroups, unit_best, lnlo, lnhi, n, out, list);
  else if (dim == kNumParams)
    k_finalize<kNumParams><<<(n + 3) / 4, 4, 0, st>>>(sacs, traces, pc, ustart, ngroups, unit_best, lnlo, lnhi, n,
                                                       out, list);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace opmm
