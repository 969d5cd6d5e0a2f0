// surrogate.cu -- host side of the learned surrogate: parameters and AdamW
// state, on-device training (data generated by the plant itself), inference
// that re-centres a fit's search box, gradient access for checking, and
// save / load.  The network maps a resampled saccade (512 features) through
// four 512-wide GELU layers to 18 outputs y with centre = nominal * exp(0.2 y).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/opmm.h"
#include "launch.h"
#include "mlp.h"
#include "runtime.h"

namespace opmm {

using namespace mlp;

namespace {
constexpr int kCal = 512;               // calibration table points
constexpr float kCalLo = 0.5f, kCalHi = 45.0f;
constexpr int kTrainLcap = 400;         // longest training window
}  // namespace

// Activations and gradients of one batch of M rows (M a multiple of 128).
constexpr int kWgradSplit = 4;          // largest number of K slices of the weight-gradient GEMM
struct MlpBuffers {
  int M = 0;
  DevBuf X, Xt, H[kLayers], Ht[kLayers], Z[kLayers], Y, dY, rowloss, dZ[kLayers], dZt[kLayers], colpart[kLayers],
      wpart, dWpart, dbpart;
  Status ensure(int m) {
    if (m <= M) return Status();
    Status s;
    const size_t act = (size_t)m * kHidden;
    s = X.ensure(act * 2);
    if (s.ok()) s = Xt.ensure(act * 2);
    for (int l = 0; l < kLayers && s.ok(); ++l) {
      s = H[l].ensure(act * 2);
      if (s.ok()) s = Ht[l].ensure(act * 2);
      if (s.ok()) s = Z[l].ensure(act * 4);
      if (s.ok()) s = dZ[l].ensure(act * 2);
      if (s.ok()) s = dZt[l].ensure(act * 2);
      // column sums per 128-row tile (GEMM epilogue) or per 32-row block (head)
      if (s.ok()) s = colpart[l].ensure((size_t)(m / (l == kLayers - 1 ? 32 : kBM)) * kHidden * 4);
    }
    if (s.ok()) s = Y.ensure((size_t)m * kOut * 4);
    if (s.ok()) s = dY.ensure((size_t)m * kOut * 4);
    if (s.ok()) s = rowloss.ensure((size_t)m * 4);
    if (s.ok()) s = wpart.ensure((size_t)kLayers * kWgradSplit * kHidden * kHidden * 4);
    if (s.ok()) s = dWpart.ensure((size_t)(m / 32) * kOut * kHidden * 4);
    if (s.ok()) s = dbpart.ensure((size_t)(m / 32) * kOut * 4);
    if (s.ok()) M = m;
    return s;
  }
};

struct SurrogateState {
  DevBuf w, g, m1, m2, wb, wt;           // FP32 master, gradient, Adam moments; BF16 copies
  DevBuf cal_amp, cal_pulse;             // agonist pulse by amplitude (calibrated nominal)
  MlpBuffers buf;
  MlpBuffers infer;                      // admission-time inference of the request loop
  // training data: two slots, so that one batch is generated (on a side
  // stream) while the network trains on the other
  struct DataSlot {
    DevBuf sacs, traces, hidden, target, X, Xt;
  } slot[2];
  DevBuf outoff, losses;
  DevBuf tstate;                         // device step state: next sample base per slot, step index
  DevBuf bctab;                          // AdamW bias corrections of the steps of a call
  int train_M = 0;
  int step = 0;
  bool ready = false;
};

static __nv_bfloat16* bf(const DevBuf& b, size_t off = 0) { return b.as<__nv_bfloat16>() + off; }
static float* f32(const DevBuf& b, size_t off = 0) { return b.as<float>() + off; }

static Status ensure_state(opmm_ctx* ctx) {
  if (!ctx->surrogate) ctx->surrogate = new SurrogateState();
  SurrogateState& S = *ctx->surrogate;
  Status s = S.w.ensure(sizeof(float) * kNumParams);
  if (s.ok()) s = S.g.ensure(sizeof(float) * kNumParams);
  if (s.ok()) s = S.m1.ensure(sizeof(float) * kNumParams);
  if (s.ok()) s = S.m2.ensure(sizeof(float) * kNumParams);
  if (s.ok()) s = S.wb.ensure(sizeof(__nv_bfloat16) * kWbElems);
  if (s.ok()) s = S.wt.ensure(sizeof(__nv_bfloat16) * kWtElems);
  if (s.ok()) s = S.cal_amp.ensure(sizeof(float) * kCal);
  if (s.ok()) s = S.cal_pulse.ensure(sizeof(float) * kCal);
  if (s.ok()) s = cuda_status(gemm_prepare(), "GEMM attributes");
  return s;
}

// Agonist pulse of the calibrated nominal plant on an amplitude grid, by the
// same device calibration the fits use (k_nominal).
static Status build_calibration(opmm_ctx* ctx) {
  SurrogateState& S = *ctx->surrogate;
  std::vector<DevSac> hs(kCal);
  std::vector<float> amp(kCal);
  for (int i = 0; i < kCal; ++i) {
    const float A = kCalLo + (kCalHi - kCalLo) * (float)i / (float)(kCal - 1);
    amp[(size_t)i] = A;
    DevSac d{};
    d.L = 2; d.onset = 0; d.nsub = 10; d.fs = 1000.0f; d.h = 1e-4f;
    d.th0 = 0.0f; d.thf = A; d.sign = 1.0f; d.dur_ms = 2.2f * A + 21.0f;
    hs[(size_t)i] = d;
  }
  DevBuf dsac, dpc;
  Status s = dsac.ensure(sizeof(DevSac) * kCal);
  if (s.ok()) s = dpc.ensure(sizeof(float) * kCal * OPMM_NPARAM);
  if (!s.ok()) return s;
  cudaStream_t st = ctx->stream;
  s = cuda_status(cudaMemcpyAsync(dsac.ptr, hs.data(), sizeof(DevSac) * kCal, cudaMemcpyHostToDevice, st), "H2D cal");
  if (s.ok()) s = cuda_status(launch_nominal(dsac.as<DevSac>(), kCal, OPMM_PULSE_CALIBRATED, nullptr, f32(dpc), st), "calibrate");
  std::vector<float> pc((size_t)kCal * OPMM_NPARAM), pulse(kCal);
  if (s.ok()) s = cuda_status(cudaMemcpyAsync(pc.data(), dpc.ptr, pc.size() * 4, cudaMemcpyDeviceToHost, st), "D2H cal");
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "calibration");
  if (!s.ok()) return s;
  for (int i = 0; i < kCal; ++i) pulse[(size_t)i] = pc[(size_t)i * OPMM_NPARAM + 15]  /* agonist pulse (H_ag) */;
  s = cuda_status(cudaMemcpy(S.cal_amp.ptr, amp.data(), kCal * 4, cudaMemcpyHostToDevice), "H2D amp");
  if (s.ok()) s = cuda_status(cudaMemcpy(S.cal_pulse.ptr, pulse.data(), kCal * 4, cudaMemcpyHostToDevice), "H2D pulse");
  return s;
}

static Status refresh_copies(opmm_ctx* ctx) {
  SurrogateState& S = *ctx->surrogate;
  return cuda_status(pack_params(f32(S.w), (int)kNumParams, AdamLayout{}, bf(S.wb), bf(S.wt), ctx->stream), "pack");
}

// Hidden layers of M rows from X on the tensor cores: H = GELU(Z) (BF16)
// and, for training, Z (pre-activations, FP32) and H's transpose.
static Status forward_hidden(opmm_ctx* ctx, MlpBuffers& B, int M, const __nv_bfloat16* X, bool keep_transposes,
                             cudaStream_t st) {
  SurrogateState& S = *ctx->surrogate;
  for (int l = 0; l < kLayers; ++l) {
    GemmLaunch L;
    L.M = M;
    L.N = kHidden;
    L.K = kHidden;
    L.epi = kEpiBiasGelu;
    L.ldo = kHidden;
    L.ldt = M;
    L.stages = 6;
    L.err = ctx->d_err.as<unsigned>();
    GemmProblem& p = L.p[0];
    p.A = l == 0 ? X : bf(B.H[l - 1]);
    p.B = bf(S.wb, (size_t)l * kHidden * kHidden);
    p.bias = f32(S.w, (size_t)l * kLayerParams + (size_t)kHidden * kHidden);
    p.out_bf16 = bf(B.H[l]);
    p.out_f32 = keep_transposes ? f32(B.Z[l]) : nullptr;   // Z only for the backward pass
    p.out_t = keep_transposes ? bf(B.Ht[l]) : nullptr;
    Status s = cuda_status(gemm(L, st), "GEMM fwd");
    if (!s.ok()) return s;
  }
  return Status();
}

// Inference: hidden layers, then the output layer on CUDA cores into B.Y.
static Status forward(opmm_ctx* ctx, MlpBuffers& B, int M, cudaStream_t st) {
  SurrogateState& S = *ctx->surrogate;
  Status s = forward_hidden(ctx, B, M, bf(B.X), false, st);
  if (!s.ok()) return s;
  return cuda_status(head_fwd_loss(bf(B.H[kLayers - 1]), bf(S.wb, (size_t)kLayers * kHidden * kHidden),
                                   f32(S.w, kHeadB), nullptr, M, f32(B.Y), f32(B.dY), nullptr, st),
                     "head");
}

// One training pass of M rows against targets T into S.g (and the batch
// loss into *loss when given): hidden layers; the head kernel (output layer,
// loss terms, output-layer gradient partials, the layer-3 error); the error
// of layers 2, 1, 0 by GEMMs whose epilogue applies GELU' and rounds
// (dZ_{l-1} = BF16((dZ_l . W_l) * GELU'(Z_{l-1}))); all four weight gradients
// dW_l = dZ_l^T . H_{l-1} in one grouped launch over K slices; the
// gradient assembly, with the AdamW step of every entry when `adam` is given.
// AdamW settings of a step of a replayable sequence: the step's index t is
// read on the device from *t_idx, its bias corrections from bc_tab[2 t],
// bc_tab[2 t + 1] and its loss goes to loss[t].
struct AdamStep {
  float lr, wd;
  const float* bc_tab;
  int* t_idx;
};
static Status train_pass(opmm_ctx* ctx, MlpBuffers& B, int M, const __nv_bfloat16* X, const __nv_bfloat16* Xt,
                         const float* T, float* loss, const AdamStep* adam, cudaStream_t st) {
  SurrogateState& S = *ctx->surrogate;
  Status s = forward_hidden(ctx, B, M, X, true, st);
  if (!s.ok()) return s;
  s = cuda_status(head_train(bf(B.H[kLayers - 1]), bf(S.wb, (size_t)kLayers * kHidden * kHidden), f32(S.w, kHeadB), T,
                             f32(B.Z[kLayers - 1]), M, f32(B.Y), f32(B.dY), f32(B.rowloss), bf(B.dZ[kLayers - 1]),
                             bf(B.dZt[kLayers - 1]), f32(B.colpart[kLayers - 1]), f32(B.dWpart), f32(B.dbpart), st),
                  "head");
  for (int l = kLayers - 1; l >= 1 && s.ok(); --l) {
    // dZ_{l-1} from dH_{l-1}[m][k] = sum_n dZ_l[m][n] W_l[n][k]
    GemmLaunch L;
    L.M = M;
    L.N = kHidden;
    L.K = kHidden;
    L.epi = kEpiGeluBwd;
    L.ldo = kHidden;
    L.ldt = M;
    L.stages = 6;
    L.err = ctx->d_err.as<unsigned>();
    GemmProblem& p = L.p[0];
    p.A = bf(B.dZ[l]);
    p.B = bf(S.wt, (size_t)l * kHidden * kHidden);
    p.zin = f32(B.Z[l - 1]);
    p.out_bf16 = bf(B.dZ[l - 1]);
    p.out_t = bf(B.dZt[l - 1]);
    p.colpart = f32(B.colpart[l - 1]);
    s = cuda_status(gemm(L, st), "GEMM dgrad");
  }
  if (s.ok()) {
    // dW_l[n][k] = sum_m dZ_l[m][n] H_{l-1}[m][k] in 128 x 256 tiles, K = M
    // split in slices so that the four layers fill the GPU (4 x 8 tiles x 4)
    GemmLaunch L;
    L.np = kLayers;
    L.M = kHidden;
    L.N = kHidden;
    L.K = M;
    L.ksplit = M % (4 * kBK) == 0 && M >= 1024 ? kWgradSplit : M >= 2 * kBM ? 2 : 1;
    L.epi = kEpiF32;
    L.bn = 256;
    L.ldo = kHidden;
    L.zstride = (long long)kHidden * kHidden;
    L.stages = 4;
    L.err = ctx->d_err.as<unsigned>();
    for (int l = 0; l < kLayers; ++l) {
      GemmProblem& p = L.p[l];
      p.A = bf(B.dZt[l]);
      p.B = l == 0 ? Xt : bf(B.Ht[l - 1]);
      p.out_f32 = f32(B.wpart, (size_t)l * L.ksplit * kHidden * kHidden);
    }
    s = cuda_status(gemm(L, st), "GEMM wgrad");
    if (s.ok()) {
      FinishArgs a{};
      a.wpart = f32(B.wpart);
      a.ksplit = L.ksplit;
      for (int l = 0; l < kLayers; ++l) {
        a.colpart[l] = f32(B.colpart[l]);
        a.ntiles[l] = l == kLayers - 1 ? M / 32 : M / kBM;
      }
      a.dWpart = f32(B.dWpart);
      a.dbpart = f32(B.dbpart);
      a.nblk = M / 32;
      a.row_loss = f32(B.rowloss);
      a.M = M;
      a.loss = loss;
      a.g = f32(S.g);
      if (adam) {
        a.adam = 1;
        a.lr = adam->lr;
        a.wd = adam->wd;
        a.b1 = 0.9f;
        a.b2 = 0.999f;
        a.eps = 1e-8f;
        a.bc_tab = adam->bc_tab;
        a.t_idx = adam->t_idx;
        a.w = f32(S.w);
        a.m1 = f32(S.m1);
        a.m2 = f32(S.m2);
        a.wb = bf(S.wb);
        a.wt = bf(S.wt);
      }
      s = cuda_status(grad_finish(a, st), adam ? "gradient assembly and AdamW" : "gradient assembly");
    }
  }
  return s;
}

// Re-centre n freshly staged requests (serving admission) on stream st.
Status surrogate_centres(opmm_ctx* ctx, const DevSac* sacs, const float* traces, int n, float* pc, cudaStream_t st) {
  if (!ctx->surrogate || !ctx->surrogate->ready) return Status(OPMM_EINVAL, "no surrogate");
  MlpBuffers& B = ctx->surrogate->infer;
  const int M = (n + kBM - 1) / kBM * kBM;
  if (B.M < M) {
    Status s = B.ensure(M);
    if (!s.ok()) return s;
    s = cuda_status(cudaMemsetAsync(B.X.ptr, 0, (size_t)M * kIn * 2, st), "clear features");
    if (!s.ok()) return s;
  }
  Status s = cuda_status(featurize(sacs, traces, n, bf(B.X), nullptr, M, st), "featurize");
  if (s.ok()) s = forward(ctx, B, M, st);
  if (s.ok()) s = cuda_status(apply_centres(f32(B.Y), n, pc, st), "centres");
  return s;
}

void surrogate_release(opmm_ctx* ctx) {
  delete ctx->surrogate;
  ctx->surrogate = nullptr;
}

// Box centres of a plan from the network: featurize the staged traces, run the
// forward pass, centre = nominal centre * exp(0.2 y).
Status surrogate_prepare_plan(opmm_ctx* ctx, opmm_plan* p, const opmm_saccade*, int32_t n) {
  if (!ctx->surrogate || !ctx->surrogate->ready)
    return Status(OPMM_EINVAL, "use_surrogate set but no surrogate is initialised or loaded");
  const int M = (n + kBM - 1) / kBM * kBM;
  auto* bufs = new MlpBuffers();
  Status s = bufs->ensure(M);
  if (!s.ok()) {
    delete bufs;
    return s;
  }
  s = cuda_status(cudaMemset(bufs->X.ptr, 0, (size_t)M * kIn * 2), "clear features");
  if (!s.ok()) {
    delete bufs;
    return s;
  }
  std::shared_ptr<MlpBuffers> keep(bufs);
  p->pre_search_kernels = 1 + kLayers + 2;
  p->pre_search = [keep, M](opmm_plan* pl, cudaStream_t st) -> Status {
    opmm_ctx* c = pl->ctx;
    Status r = cuda_status(featurize(pl->d_sacs.as<DevSac>(), pl->d_traces.as<float>(), pl->n, bf(keep->X), nullptr, M, st),
                           "featurize");
    if (r.ok()) r = forward(c, *keep, M, st);
    if (r.ok()) r = cuda_status(apply_centres(f32(keep->Y), pl->n, pl->d_pc.as<float>(), st), "centres");
    return r;
  };
  return Status();
}

}  // namespace opmm

using namespace opmm;

static int sfail(opmm_ctx* ctx, const Status& s) {
  (void)ctx;
  set_last_error(s.msg);
  return s.code;
}

#define STRY(expr)                                 \
  do {                                             \
    Status _s = (expr);                            \
    if (!_s.ok()) return sfail(ctx, _s);           \
  } while (0)

extern "C" int opmm_surrogate_init(opmm_ctx* ctx, uint64_t seed) {
  if (!ctx) return OPMM_EINVAL;
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  STRY(ensure_state(ctx));
  SurrogateState& S = *ctx->surrogate;
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases (splitmix64)
  std::vector<float> w((size_t)kNumParams);
  uint64_t x = seed;
  auto next = [&]() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  const double bound = 1.0 / std::sqrt((double)kHidden);
  for (size_t i = 0; i < w.size(); ++i) w[i] = (float)((2.0 * next() - 1.0) * bound);
  STRY(cuda_status(cudaMemcpy(S.w.ptr, w.data(), w.size() * 4, cudaMemcpyHostToDevice), "H2D params"));
  STRY(cuda_status(cudaMemset(S.m1.ptr, 0, (size_t)kNumParams * 4), "clear m1"));
  STRY(cuda_status(cudaMemset(S.m2.ptr, 0, (size_t)kNumParams * 4), "clear m2"));
  STRY(build_calibration(ctx));
  STRY(refresh_copies(ctx));
  STRY(cuda_status(cudaStreamSynchronize(ctx->stream), "init"));
  S.step = 0;
  S.ready = true;
  return OPMM_OK;
}

extern "C" int opmm_surrogate_num_params(int64_t* n) {
  if (!n) return OPMM_EINVAL;
  *n = kNumParams;
  return OPMM_OK;
}

extern "C" int opmm_surrogate_get_params(opmm_ctx* ctx, float* out) {
  if (!ctx || !out) return OPMM_EINVAL;
  if (!ctx->surrogate || !ctx->surrogate->ready) return sfail(ctx, Status(OPMM_EINVAL, "no surrogate"));
  STRY(cuda_status(cudaMemcpy(out, ctx->surrogate->w.ptr, (size_t)kNumParams * 4, cudaMemcpyDeviceToHost), "D2H params"));
  return OPMM_OK;
}

extern "C" int opmm_surrogate_set_params(opmm_ctx* ctx, const float* in) {
  if (!ctx || !in) return OPMM_EINVAL;
  if (!ctx->surrogate || !ctx->surrogate->ready) return sfail(ctx, Status(OPMM_EINVAL, "no surrogate"));
  STRY(cuda_status(cudaMemcpy(ctx->surrogate->w.ptr, in, (size_t)kNumParams * 4, cudaMemcpyHostToDevice), "H2D params"));
  STRY(refresh_copies(ctx));
  STRY(cuda_status(cudaStreamSynchronize(ctx->stream), "set params"));
  return OPMM_OK;
}

extern "C" int opmm_surrogate_grad(opmm_ctx* ctx, const float* x, const float* t, int32_t m, float* loss, float* grad,
                                   float* y_out) {
  if (!ctx || !x || !t || !loss || !grad || m <= 0 || m % kBM) return ctx ? sfail(ctx, Status(OPMM_EINVAL, "grad: rows must be a positive multiple of 128")) : OPMM_EINVAL;
  if (!ctx->surrogate || !ctx->surrogate->ready) return sfail(ctx, Status(OPMM_EINVAL, "no surrogate"));
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  SurrogateState& S = *ctx->surrogate;
  MlpBuffers& B = S.buf;
  STRY(B.ensure(m));
  cudaStream_t st = ctx->stream;
  // host features -> BF16 (round to nearest even) and the transpose
  std::vector<__nv_bfloat16> xb((size_t)m * kIn), xt((size_t)m * kIn);
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < kIn; ++k) {
      const __nv_bfloat16 v = __float2bfloat16_rn(x[(size_t)i * kIn + k]);
      xb[(size_t)i * kIn + k] = v;
      xt[(size_t)k * m + i] = v;
    }
  DevBuf dt;
  STRY(dt.ensure((size_t)m * kOut * 4));
  STRY(cuda_status(cudaMemcpyAsync(B.X.ptr, xb.data(), xb.size() * 2, cudaMemcpyHostToDevice, st), "H2D X"));
  STRY(cuda_status(cudaMemcpyAsync(B.Xt.ptr, xt.data(), xt.size() * 2, cudaMemcpyHostToDevice, st), "H2D Xt"));
  STRY(cuda_status(cudaMemcpyAsync(dt.ptr, t, (size_t)m * kOut * 4, cudaMemcpyHostToDevice, st), "H2D T"));
  STRY(cuda_status(cudaMemsetAsync(ctx->d_err.ptr, 0, 4, st), "clear error"));
  STRY(train_pass(ctx, B, m, bf(B.X), bf(B.Xt), f32(dt), nullptr, nullptr, st));
  std::vector<float> rl((size_t)m);
  STRY(cuda_status(cudaMemcpyAsync(rl.data(), B.rowloss.ptr, (size_t)m * 4, cudaMemcpyDeviceToHost, st), "D2H loss"));
  STRY(cuda_status(cudaMemcpyAsync(grad, S.g.ptr, (size_t)kNumParams * 4, cudaMemcpyDeviceToHost, st), "D2H grad"));
  if (y_out) STRY(cuda_status(cudaMemcpyAsync(y_out, B.Y.ptr, (size_t)m * kOut * 4, cudaMemcpyDeviceToHost, st), "D2H Y"));
  unsigned e = 0;
  STRY(cuda_status(cudaMemcpyAsync(&e, ctx->d_err.ptr, 4, cudaMemcpyDeviceToHost, st), "D2H error"));
  STRY(cuda_status(cudaStreamSynchronize(st), "grad"));
  if (e) return sfail(ctx, Status(OPMM_ETIMEDOUT, "GEMM pipeline wait expired"));
  double l = 0.0;
  for (float v : rl) l += v;
  *loss = (float)l;
  return OPMM_OK;
}

extern "C" int opmm_surrogate_apply_grad(opmm_ctx* ctx, const float* grad, float lr, float weight_decay) {
  if (!ctx) return OPMM_EINVAL;
  if (!grad || !(lr > 0.0f) || !std::isfinite(lr) || !(weight_decay >= 0.0f) || !std::isfinite(weight_decay))
    return sfail(ctx, Status(OPMM_EINVAL, "apply_grad: gradient required, lr > 0, weight_decay >= 0"));
  if (!ctx->surrogate || !ctx->surrogate->ready) return sfail(ctx, Status(OPMM_EINVAL, "no surrogate"));
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  SurrogateState& S = *ctx->surrogate;
  cudaStream_t st = ctx->stream;
  STRY(cuda_status(cudaMemcpyAsync(S.g.ptr, grad, (size_t)kNumParams * 4, cudaMemcpyHostToDevice, st), "H2D grad"));
  S.step += 1;
  STRY(cuda_status(adamw(f32(S.w), f32(S.g), f32(S.m1), f32(S.m2), (int)kNumParams, lr, 0.9f, 0.999f, 1e-8f,
                         weight_decay, S.step, AdamLayout{}, bf(S.wb), bf(S.wt), st), "AdamW"));
  STRY(cuda_status(cudaStreamSynchronize(st), "apply_grad"));
  return OPMM_OK;
}

extern "C" int opmm_surrogate_train(opmm_ctx* ctx, int32_t steps, int32_t batch, float lr, float weight_decay,
                                    uint64_t data_seed, int64_t sample_base, float* losses) {
  if (!ctx) return OPMM_EINVAL;
  if (steps < 0 || batch <= 0 || batch % kBM || !(lr > 0.0f))
    return sfail(ctx, Status(OPMM_EINVAL, "train: batch must be a positive multiple of 128, lr > 0"));
  if (!ctx->surrogate || !ctx->surrogate->ready) return sfail(ctx, Status(OPMM_EINVAL, "no surrogate"));
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  SurrogateState& S = *ctx->surrogate;
  MlpBuffers& B = S.buf;
  STRY(B.ensure(batch));
  if (S.train_M < batch) {
    for (auto& D : S.slot) {
      STRY(D.sacs.ensure(sizeof(DevSac) * (size_t)batch));
      STRY(D.traces.ensure(sizeof(float) * (size_t)batch * kTrainLcap));
      STRY(D.hidden.ensure(sizeof(float) * (size_t)batch * kOut));
      STRY(D.target.ensure(sizeof(float) * (size_t)batch * kOut));
      STRY(D.X.ensure((size_t)batch * kIn * 2));
      STRY(D.Xt.ensure((size_t)batch * kIn * 2));
    }
    STRY(S.outoff.ensure(sizeof(long long) * (size_t)batch));
    std::vector<long long> off((size_t)batch);
    for (int i = 0; i < batch; ++i) off[(size_t)i] = (long long)i * kTrainLcap;
    STRY(cuda_status(cudaMemcpy(S.outoff.ptr, off.data(), off.size() * 8, cudaMemcpyHostToDevice), "H2D offsets"));
    S.train_M = batch;
  }
  STRY(S.losses.ensure(sizeof(float) * (size_t)(steps > 0 ? steps : 1)));
  cudaStream_t st = ctx->stream;
  STRY(cuda_status(cudaMemsetAsync(ctx->d_err.ptr, 0, 4, st), "clear error"));
  // Device step state: the sample base of the next batch of each data slot
  // and the index of the next step; the AdamW bias corrections of every step
  // of this call (formed in double on the host as for opmm_surrogate_apply_grad).
  STRY(S.tstate.ensure(32));
  STRY(S.bctab.ensure(sizeof(float) * 2 * (size_t)(steps > 0 ? steps : 1)));
  long long* gbase = S.tstate.as<long long>();
  int* t_idx = reinterpret_cast<int*>(gbase + 2);
  {
    std::vector<float> tab(2 * (size_t)(steps > 0 ? steps : 1));
    for (int t = 0; t < steps; ++t) adam_corrections(0.9f, 0.999f, S.step + 1 + t, &tab[2 * (size_t)t], &tab[2 * (size_t)t + 1]);
    const long long init[2] = {(long long)sample_base, (long long)sample_base + batch};
    STRY(cuda_status(cudaMemcpyAsync(gbase, init, sizeof init, cudaMemcpyHostToDevice, st), "H2D step state"));
    STRY(cuda_status(cudaMemsetAsync(t_idx, 0, sizeof(int), st), "clear step index"));
    STRY(cuda_status(cudaMemcpyAsync(S.bctab.ptr, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st), "H2D corrections"));
    STRY(cuda_status(cudaStreamSynchronize(st), "stage step state"));
  }
  // Steps run in pairs replayed from one CUDA graph: while the network
  // trains on slot 0, the side stream generates slot 1; while it trains on
  // slot 1, slot 0 is refilled for the next pair (after the step that read
  // it).  Every per-step quantity comes from the device step state, so the
  // same graph serves every pair.  Before the first pair, slot 0 is filled;
  // an odd last step runs without the graph.
  struct Side {
    cudaStream_t main = nullptr, s = nullptr;
    cudaEvent_t fork = nullptr, data0 = nullptr, data1 = nullptr, used0 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~Side() {
      if (main) cudaStreamSynchronize(main);
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
      for (cudaEvent_t e : {fork, data0, data1, used0})
        if (e) cudaEventDestroy(e);
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    }
  } side;
  side.main = st;
  STRY(cuda_status(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking), "side stream"));
  for (cudaEvent_t* e : {&side.fork, &side.data0, &side.data1, &side.used0})
    STRY(cuda_status(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event"));
  const AdamStep adam{lr, weight_decay, f32(S.bctab), t_idx};
  auto gen = [&](int b, cudaStream_t s2) -> Status {
    SurrogateState::DataSlot& D = S.slot[b];
    Status r = cuda_status(gen_desc(data_seed, gbase + b, batch, f32(S.cal_amp), f32(S.cal_pulse), kCal,
                                    D.sacs.as<DevSac>(), f32(D.hidden), f32(D.target), kTrainLcap, s2), "generate");
    if (r.ok())
      r = cuda_status(launch_simulate(f32(D.hidden), batch, D.sacs.as<DevSac>(), nullptr, S.outoff.as<long long>(),
                                      f32(D.traces), s2), "simulate");
    if (r.ok()) r = cuda_status(add_noise(data_seed, gbase + b, D.sacs.as<DevSac>(), batch, f32(D.traces), 0.05f, s2), "noise");
    if (r.ok())
      r = cuda_status(featurize(D.sacs.as<DevSac>(), f32(D.traces), batch, bf(D.X), bf(D.Xt), batch, s2), "featurize");
    if (r.ok()) r = cuda_status(bump(gbase + b, 2LL * batch, nullptr, s2), "advance sample base");
    return r;
  };
  auto net = [&](int b, cudaStream_t s1) -> Status {
    SurrogateState::DataSlot& D = S.slot[b];
    // the step index advances in the weight transposes that end the step
    return train_pass(ctx, B, batch, bf(D.X), bf(D.Xt), f32(D.target), f32(S.losses), &adam, s1);
  };
  if (steps > 0) STRY(gen(0, st));
  const int pairs = steps / 2;
  if (pairs > 0) {
    STRY(cuda_status(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"));
    Status cs = cuda_status(cudaEventRecord(side.fork, st), "record");
    if (cs.ok()) cs = cuda_status(cudaStreamWaitEvent(side.s, side.fork, 0), "wait");
    if (cs.ok()) cs = gen(1, side.s);
    if (cs.ok()) cs = cuda_status(cudaEventRecord(side.data1, side.s), "record");
    if (cs.ok()) cs = net(0, st);
    if (cs.ok()) cs = cuda_status(cudaEventRecord(side.used0, st), "record");
    if (cs.ok()) cs = cuda_status(cudaStreamWaitEvent(side.s, side.used0, 0), "wait");
    if (cs.ok()) cs = gen(0, side.s);
    if (cs.ok()) cs = cuda_status(cudaEventRecord(side.data0, side.s), "record");
    if (cs.ok()) cs = cuda_status(cudaStreamWaitEvent(st, side.data1, 0), "wait");
    if (cs.ok()) cs = net(1, st);
    if (cs.ok()) cs = cuda_status(cudaStreamWaitEvent(st, side.data0, 0), "wait");
    const cudaError_t ce = cudaStreamEndCapture(st, &side.graph);
    if (!cs.ok()) return sfail(ctx, cs);
    STRY(cuda_status(ce, "end capture"));
    STRY(cuda_status(cudaGraphInstantiate(&side.exec, side.graph, 0), "instantiate"));
    for (int k = 0; k < pairs; ++k) STRY(cuda_status(cudaGraphLaunch(side.exec, st), "graph launch"));
  }
  if (steps & 1) STRY(net(0, st));
  S.step += steps;
  if (losses && steps > 0)
    STRY(cuda_status(cudaMemcpyAsync(losses, S.losses.ptr, (size_t)steps * 4, cudaMemcpyDeviceToHost, st), "D2H losses"));
  unsigned e = 0;
  STRY(cuda_status(cudaMemcpyAsync(&e, ctx->d_err.ptr, 4, cudaMemcpyDeviceToHost, st), "D2H error"));
  STRY(cuda_status(cudaStreamSynchronize(st), "train"));
  if (e) return sfail(ctx, Status(OPMM_ETIMEDOUT, "GEMM pipeline wait expired"));
  return OPMM_OK;
}

extern "C" int opmm_surrogate_predict(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, int32_t pulse_init,
                                      float* out_opc) {
  if (!ctx) return OPMM_EINVAL;
  if (!sacs || !out_opc || n <= 0) return sfail(ctx, Status(OPMM_EINVAL, "predict: bad arguments"));
  opmm_fit_opts o{};
  o.model = OPMM_MODEL_18;
  o.candidates = 22;
  o.iterations = 0;
  o.box_lo = 1.0f;
  o.box_hi = 1.0f;
  o.init_step = 1e-3f;
  o.pulse_init = pulse_init;
  o.use_surrogate = 1;
  opmm_plan p;
  Status s = surrogate_prepare_plan(ctx, &p, sacs, n);
  if (s.ok()) s = plan_stage(ctx, sacs, n, o, &p);   // stages traces and applies the surrogate
  if (s.ok())
    s = cuda_status(cudaMemcpyAsync(out_opc, p.d_pc.ptr, sizeof(float) * OPMM_NPARAM * (size_t)n, cudaMemcpyDeviceToHost,
                                    ctx->stream), "D2H centres");
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(ctx->stream), "predict");
  if (!s.ok()) return sfail(ctx, s);
  return OPMM_OK;
}

extern "C" int opmm_surrogate_save(opmm_ctx* ctx, const char* path) {
  if (!ctx || !path) return OPMM_EINVAL;
  if (!ctx->surrogate || !ctx->surrogate->ready) return sfail(ctx, Status(OPMM_EINVAL, "no surrogate"));
  std::vector<float> w((size_t)kNumParams);
  STRY(cuda_status(cudaMemcpy(w.data(), ctx->surrogate->w.ptr, w.size() * 4, cudaMemcpyDeviceToHost), "D2H params"));
  FILE* f = std::fopen(path, "wb");
  if (!f) return sfail(ctx, Status(OPMM_EINVAL, std::string("cannot open ") + path));
  const char magic[8] = {'O', 'P', 'M', 'M', 'S', 'G', '1', 0};
  const int64_t n = kNumParams;
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&n, 8, 1, f) == 1 &&
            std::fwrite(w.data(), 4, w.size(), f) == w.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return sfail(ctx, Status(OPMM_EINVAL, "write failed"));
  return OPMM_OK;
}

extern "C" int opmm_surrogate_load(opmm_ctx* ctx, const char* path) {
  if (!ctx || !path) return OPMM_EINVAL;
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  FILE* f = std::fopen(path, "rb");
  if (!f) return sfail(ctx, Status(OPMM_EINVAL, std::string("cannot open ") + path));
  char magic[8];
  int64_t n = 0;
  std::vector<float> w((size_t)kNumParams);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "OPMMSG1", 8) == 0 && std::fread(&n, 8, 1, f) == 1 &&
            n == kNumParams && std::fread(w.data(), 4, w.size(), f) == w.size();
  std::fclose(f);
  if (!ok) return sfail(ctx, Status(OPMM_EINVAL, "not a surrogate weights file of this architecture"));
  const bool fresh = !ctx->surrogate || !ctx->surrogate->ready;
  if (fresh) {
    const int rc = opmm_surrogate_init(ctx, 0);
    if (rc != OPMM_OK) return rc;
  }
  return opmm_surrogate_set_params(ctx, w.data());
}

extern "C" int opmm_featurize(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, float* out) {
  if (!ctx) return OPMM_EINVAL;
  if (!sacs || !out || n <= 0) return sfail(ctx, Status(OPMM_EINVAL, "featurize: bad arguments"));
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  opmm_fit_opts o{};
  o.model = OPMM_MODEL_18;
  o.candidates = 22;
  o.box_lo = 1.0f;
  o.box_hi = 1.0f;
  o.init_step = 1e-3f;
  o.pulse_init = OPMM_PULSE_TABLE1;
  std::vector<float> zero_centres((size_t)n * OPMM_NPARAM, 1.0f);
  o.init_opc = zero_centres.data();
  opmm_plan p;
  STRY(plan_stage(ctx, sacs, n, o, &p));
  DevBuf X;
  STRY(X.ensure((size_t)n * kIn * 2));
  STRY(cuda_status(featurize(p.d_sacs.as<DevSac>(), p.d_traces.as<float>(), n, bf(X), nullptr, n, ctx->stream),
                   "featurize"));
  std::vector<__nv_bfloat16> h((size_t)n * kIn);
  STRY(cuda_status(cudaMemcpyAsync(h.data(), X.ptr, h.size() * 2, cudaMemcpyDeviceToHost, ctx->stream), "D2H"));
  STRY(cuda_status(cudaStreamSynchronize(ctx->stream), "featurize"));
  for (size_t i = 0; i < h.size(); ++i) out[i] = __bfloat162float(h[i]);
  return OPMM_OK;
}

extern "C" int opmm_gemm_bf16(opmm_ctx* ctx, const void* A, const void* B, int32_t M, int32_t N, int32_t K, float* D) {
  if (!ctx) return OPMM_EINVAL;
  if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || M % kBM || N % kBN || K % kBK)
    return sfail(ctx, Status(OPMM_EINVAL, "gemm: M, N multiples of 128 and K a multiple of 64 required"));
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(D))
    return sfail(ctx, Status(OPMM_EINVAL, "gemm: device pointers required"));
  STRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  STRY(cuda_status(gemm_prepare(), "GEMM attributes"));
  GemmLaunch L;
  L.M = M;
  L.N = N;
  L.K = K;
  L.epi = kEpiF32;
  L.ldo = N;
  L.stages = 3;
  L.err = ctx->d_err.as<unsigned>();
  L.p[0].A = static_cast<const __nv_bfloat16*>(A);
  L.p[0].B = static_cast<const __nv_bfloat16*>(B);
  L.p[0].out_f32 = D;
  STRY(cuda_status(cudaMemsetAsync(ctx->d_err.ptr, 0, 4, ctx->stream), "clear error"));
  STRY(cuda_status(gemm(L, ctx->stream), "GEMM"));
  unsigned e = 0;
  STRY(cuda_status(cudaMemcpyAsync(&e, ctx->d_err.ptr, 4, cudaMemcpyDeviceToHost, ctx->stream), "D2H error"));
  STRY(cuda_status(cudaStreamSynchronize(ctx->stream), "gemm"));
  if (e) return sfail(ctx, Status(OPMM_ETIMEDOUT, "GEMM pipeline wait expired"));
  return OPMM_OK;
}
