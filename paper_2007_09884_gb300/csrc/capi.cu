// capi.cu -- host runtime behind the C ABI (include/opmm.h): contexts,
// descriptor validation and staging, device buffers, plans captured as CUDA
// graphs, the launch-shape autotuner and the error discipline of the ABI
// (status codes, no exception crosses the boundary).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/opmm.h"
#include "common.cuh"
#include "launch.h"
#include "runtime.h"

using opmm::DevSac;

namespace opmm {

// ------------------------------------------------------------------ helpers
Status::Status(int c, std::string m) : code(c), msg(std::move(m)) {}

Status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return Status();
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return Status(OPMM_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  }
  return Status(OPMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

DevBuf::~DevBuf() { release(); }
void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}
Status DevBuf::ensure(size_t want) {
  if (want <= bytes && ptr) return Status();
  release();
  if (want == 0) want = 16;
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    return Status(OPMM_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
  }
  bytes = want;
  return Status();
}

HostBuf::~HostBuf() { release(); }
void HostBuf::release() {
  if (ptr) cudaFreeHost(ptr);
  ptr = nullptr;
  bytes = 0;
}
Status HostBuf::ensure(size_t want) {
  if (want <= bytes && ptr) return Status();
  release();
  if (want == 0) want = 16;
  cudaError_t e = cudaHostAlloc(&ptr, want, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    return Status(OPMM_ENOMEM, "pinned allocation of " + std::to_string(want) + " bytes failed");
  }
  bytes = want;
  return Status();
}

int nsub_for(float fs) {
  const int n = (int)std::floor(1.0e4 / (double)fs + 0.5);
  return n < 1 ? 1 : n;
}

// Validate one descriptor (the trace pointer is checked by the callers that
// read traces).
Status check_saccade(const opmm_saccade& s, int i, bool need_duration) {
  auto bad = [&](const char* why) { return Status(OPMM_EINVAL, "saccade " + std::to_string(i) + ": " + why); };
  if (s.n_samples < 1) return bad("n_samples must be >= 1");
  if (s.n_samples > kMaxSamples) return bad("n_samples above the supported maximum (16384)");
  if (!(s.sample_rate_hz > 0.0f) || !std::isfinite(s.sample_rate_hz)) return bad("sample_rate_hz must be > 0");
  if (nsub_for(s.sample_rate_hz) > 4096) return bad("sample_rate_hz too low (more than 4096 substeps per sample)");
  if (s.onset_index < 0 || s.onset_index >= s.n_samples) return bad("onset_index outside [0, n_samples)");
  if (!std::isfinite(s.theta_start_deg) || !std::isfinite(s.theta_end_deg)) return bad("non-finite fixation");
  if (need_duration && !(s.duration_ms > 6.0f && std::isfinite(s.duration_ms)))
    return bad("duration_ms must exceed 6 ms (nominal pulse width = duration - 6 ms)");
  return Status();
}

// Host descriptor in the positive frame; `off` is set by the caller.
DevSac make_devsac(const opmm_saccade& s) {
  DevSac d;
  d.off = 0;
  d.L = s.n_samples;
  d.onset = s.onset_index;
  d.nsub = nsub_for(s.sample_rate_hz);
  d.fs = s.sample_rate_hz;
  d.h = (float)(1.0 / ((double)s.sample_rate_hz * d.nsub));
  const bool mirror = s.theta_end_deg < s.theta_start_deg;
  d.sign = mirror ? -1.0f : 1.0f;
  d.th0 = d.sign * s.theta_start_deg;
  d.thf = d.sign * s.theta_end_deg;
  d.dur_ms = s.duration_ms;
  return d;
}

Status check_opc(const float* opc) {
  for (int j = 0; j < OPMM_NPARAM; ++j)
    if (!(opc[j] > 0.0f) || !std::isfinite(opc[j]))
      return Status(OPMM_EINVAL, "OPC entries must be finite and > 0 (entry " + std::to_string(j) + ")");
  return Status();
}

}  // namespace opmm

using namespace opmm;

// ------------------------------------------------------------------ context
opmm_ctx::opmm_ctx() = default;
opmm_ctx::~opmm_ctx() {
  if (own_stream) cudaStreamDestroy(own_stream);
}

namespace opmm {
// Error text of the last failed call, per calling thread: the serving calls
// run concurrently from several threads.
static thread_local std::string tl_last_error;
void set_last_error(const std::string& msg) { tl_last_error = msg; }
}  // namespace opmm

static int fail(opmm_ctx* ctx, const Status& s) {
  (void)ctx;
  set_last_error(s.msg);
  return s.code;
}

#define TRY(expr)                          \
  do {                                     \
    Status _s = (expr);                    \
    if (!_s.ok()) return fail(ctx, _s);    \
  } while (0)

#define CUDA_TRY(expr, what) TRY(cuda_status((expr), (what)))

static Status ctx_bind(opmm_ctx* ctx) { return cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"); }

static Status ctx_check_error_word(opmm_ctx* ctx) {
  unsigned h = 0;
  Status s = cuda_status(cudaMemcpy(&h, ctx->d_err.as<unsigned>(), sizeof h, cudaMemcpyDeviceToHost),
                         "read error word");
  if (!s.ok()) return s;
  if (h & kErrWaitTimeout) return Status(OPMM_ETIMEDOUT, "a kernel's bounded TMA wait expired");
  if (h) return Status(OPMM_ECUDA, "kernel error bits " + std::to_string(h));
  return Status();
}

extern "C" int opmm_create(int device_ordinal, opmm_ctx** out) {
  if (!out) return OPMM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return OPMM_ECUDA;
  }
  if (device_ordinal < 0 || device_ordinal >= ndev) return OPMM_EINVAL;
  opmm_ctx* ctx = new (std::nothrow) opmm_ctx();
  if (!ctx) return OPMM_ENOMEM;
  ctx->device = device_ordinal;
  Status s = ctx_bind(ctx);
  if (s.ok()) s = cuda_status(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device_ordinal),
                              "query SM count");
  if (s.ok()) s = cuda_status(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking), "create stream");
  if (s.ok()) s = ctx->d_err.ensure(sizeof(unsigned));
  if (s.ok()) s = cuda_status(cudaMemset(ctx->d_err.ptr, 0, sizeof(unsigned)), "clear error word");
  if (!s.ok()) {
    int code = s.code;
    delete ctx;
    return code;
  }
  ctx->stream = ctx->own_stream;
  *out = ctx;
  return OPMM_OK;
}

extern "C" void opmm_destroy(opmm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  serve_shutdown(ctx);
  surrogate_release(ctx);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

extern "C" const char* opmm_last_error(const opmm_ctx* ctx) {
  (void)ctx;
  return tl_last_error.c_str();
}

extern "C" int opmm_set_search_variant(opmm_ctx* ctx, int32_t variant) {
  if (!ctx) return OPMM_EINVAL;
  if (variant < -1 || variant >= search_variant_count())
    return fail(ctx, Status(OPMM_EINVAL, "search variant out of range"));
  ctx->forced_variant = variant;
  return OPMM_OK;
}

extern "C" int opmm_search_variants(int32_t* count) {
  if (!count) return OPMM_EINVAL;
  *count = search_variant_count();
  return OPMM_OK;
}

extern "C" int opmm_search_variant_info(int32_t variant, int32_t* simplices_per_block, int32_t* model) {
  if (variant < 0 || variant >= search_variant_count()) return OPMM_EINVAL;
  if (simplices_per_block) *simplices_per_block = search_variant_g(variant);
  if (model) *model = search_variant_dim(variant) == 9 ? OPMM_MODEL_9 : OPMM_MODEL_18;
  return OPMM_OK;
}

extern "C" int opmm_search_variant_walk(int32_t variant, int32_t* walk) {
  if (variant < 0 || variant >= search_variant_count() || !walk) return OPMM_EINVAL;
  *walk = search_variant_lean(variant) ? OPMM_WALK_LEAN
                                       : (search_variant_pack(variant) ? OPMM_WALK_PACKED : OPMM_WALK_SCALAR);
  return OPMM_OK;
}

extern "C" int opmm_set_stream(opmm_ctx* ctx, void* stream) {
  if (!ctx) return OPMM_EINVAL;
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return OPMM_OK;
}

// ------------------------------------------------------------------ simulate
extern "C" int opmm_simulate(opmm_ctx* ctx, const float* opc, int32_t n, const opmm_saccade* sacs,
                             int32_t n_sacs, const int32_t* sac_index, const int64_t* out_offset,
                             float* out_deg) {
  if (!ctx) return OPMM_EINVAL;
  if (n < 0 || (n > 0 && (!opc || !sacs || !out_offset || !out_deg)) || n_sacs < 1)
    return fail(ctx, Status(OPMM_EINVAL, "opmm_simulate: bad arguments"));
  if (n == 0) return OPMM_OK;
  TRY(ctx_bind(ctx));
  std::vector<DevSac> hs((size_t)n_sacs);
  for (int i = 0; i < n_sacs; ++i) {
    TRY(check_saccade(sacs[i], i, false));
    hs[(size_t)i] = make_devsac(sacs[i]);
  }
  int64_t total = 0;
  for (int i = 0; i < n; ++i) {
    const int s = sac_index ? sac_index[i] : i;
    if (s < 0 || s >= n_sacs) return fail(ctx, Status(OPMM_EINVAL, "sac_index out of range"));
    if (out_offset[i] < 0) return fail(ctx, Status(OPMM_EINVAL, "negative out_offset"));
    total = std::max<int64_t>(total, out_offset[i] + hs[(size_t)s].L);
  }
  const bool opc_dev = is_device_ptr(opc), out_dev = is_device_ptr(out_deg);
  if (!opc_dev)
    for (int i = 0; i < n; ++i) TRY(check_opc(opc + (size_t)i * OPMM_NPARAM));
  cudaStream_t st = ctx->stream;
  DevBuf& b_sac = ctx->scratch[0];
  DevBuf& b_opc = ctx->scratch[1];
  DevBuf& b_idx = ctx->scratch[2];
  DevBuf& b_off = ctx->scratch[3];
  DevBuf& b_out = ctx->scratch[4];
  TRY(b_sac.ensure(sizeof(DevSac) * (size_t)n_sacs));
  TRY(b_off.ensure(sizeof(long long) * (size_t)n));
  CUDA_TRY(cudaMemcpyAsync(b_sac.ptr, hs.data(), sizeof(DevSac) * (size_t)n_sacs, cudaMemcpyHostToDevice, st), "H2D descriptors");
  CUDA_TRY(cudaMemcpyAsync(b_off.ptr, out_offset, sizeof(long long) * (size_t)n, cudaMemcpyHostToDevice, st), "H2D offsets");
  const int* d_idx = nullptr;
  if (sac_index) {
    TRY(b_idx.ensure(sizeof(int) * (size_t)n));
    CUDA_TRY(cudaMemcpyAsync(b_idx.ptr, sac_index, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st), "H2D index");
    d_idx = b_idx.as<int>();
  }
  const float* d_opc = opc;
  if (!opc_dev) {
    TRY(b_opc.ensure(sizeof(float) * OPMM_NPARAM * (size_t)n));
    CUDA_TRY(cudaMemcpyAsync(b_opc.ptr, opc, sizeof(float) * OPMM_NPARAM * (size_t)n, cudaMemcpyHostToDevice, st), "H2D opc");
    d_opc = b_opc.as<float>();
  }
  float* d_out = out_deg;
  if (!out_dev) {
    TRY(b_out.ensure(sizeof(float) * (size_t)total));
    d_out = b_out.as<float>();
  }
  CUDA_TRY(launch_simulate(d_opc, n, b_sac.as<DevSac>(), d_idx, b_off.as<long long>(), d_out, st), "launch simulate");
  if (!out_dev)
    CUDA_TRY(cudaMemcpyAsync(out_deg, d_out, sizeof(float) * (size_t)total, cudaMemcpyDeviceToHost, st), "D2H trajectories");
  CUDA_TRY(cudaStreamSynchronize(st), "simulate");
  return OPMM_OK;
}

// Stage one saccade's trace into scratch slot `slot` (16-byte aligned,
// zero-padded to a multiple of 4 samples).
static Status stage_one(opmm_ctx* ctx, const opmm_saccade& s, DevBuf& buf, cudaStream_t st) {
  const size_t lp = (size_t)((s.n_samples + 3) & ~3);
  Status r = buf.ensure(lp * sizeof(float));
  if (!r.ok()) return r;
  r = cuda_status(cudaMemsetAsync(buf.ptr, 0, lp * sizeof(float), st), "clear trace");
  if (!r.ok()) return r;
  const cudaMemcpyKind kind = is_device_ptr(s.trace_deg) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  return cuda_status(cudaMemcpyAsync(buf.ptr, s.trace_deg, sizeof(float) * (size_t)s.n_samples, kind, st),
                     "copy trace");
}

extern "C" int opmm_score(opmm_ctx* ctx, const float* opc, int32_t m, const opmm_saccade* sac, float* out_f) {
  if (!ctx) return OPMM_EINVAL;
  if (m < 0 || !sac || (m > 0 && (!opc || !out_f)) || !sac->trace_deg)
    return fail(ctx, Status(OPMM_EINVAL, "opmm_score: bad arguments"));
  TRY(check_saccade(*sac, 0, false));
  if (m == 0) return OPMM_OK;
  TRY(ctx_bind(ctx));
  cudaStream_t st = ctx->stream;
  DevSac d = make_devsac(*sac);
  d.off = 0;
  DevBuf& b_sac = ctx->scratch[0];
  DevBuf& b_opc = ctx->scratch[1];
  DevBuf& b_tr = ctx->scratch[5];
  DevBuf& b_f = ctx->scratch[6];
  TRY(b_sac.ensure(sizeof(DevSac)));
  CUDA_TRY(cudaMemcpyAsync(b_sac.ptr, &d, sizeof d, cudaMemcpyHostToDevice, st), "H2D descriptor");
  TRY(stage_one(ctx, *sac, b_tr, st));
  const bool opc_dev = is_device_ptr(opc), f_dev = is_device_ptr(out_f);
  if (!opc_dev)
    for (int i = 0; i < m; ++i) TRY(check_opc(opc + (size_t)i * OPMM_NPARAM));
  const float* d_opc = opc;
  if (!opc_dev) {
    TRY(b_opc.ensure(sizeof(float) * OPMM_NPARAM * (size_t)m));
    CUDA_TRY(cudaMemcpyAsync(b_opc.ptr, opc, sizeof(float) * OPMM_NPARAM * (size_t)m, cudaMemcpyHostToDevice, st), "H2D opc");
    d_opc = b_opc.as<float>();
  }
  float* d_f = out_f;
  if (!f_dev) {
    TRY(b_f.ensure(sizeof(float) * (size_t)m));
    d_f = b_f.as<float>();
  }
  CUDA_TRY(cudaMemsetAsync(ctx->d_err.ptr, 0, sizeof(unsigned), st), "clear error word");
  CUDA_TRY(launch_score(d_opc, m, b_sac.as<DevSac>(), d.L, b_tr.as<float>(), d_f, ctx->d_err.as<unsigned>(),
                        ctx->num_sms, st), "launch score");
  if (!f_dev) CUDA_TRY(cudaMemcpyAsync(out_f, d_f, sizeof(float) * (size_t)m, cudaMemcpyDeviceToHost, st), "D2H scores");
  CUDA_TRY(cudaStreamSynchronize(st), "score");
  TRY(ctx_check_error_word(ctx));
  return OPMM_OK;
}

extern "C" int opmm_nominal_opc(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, int32_t pulse_init,
                                float* out_opc) {
  if (!ctx) return OPMM_EINVAL;
  if (n < 0 || (n > 0 && (!sacs || !out_opc))) return fail(ctx, Status(OPMM_EINVAL, "opmm_nominal_opc: bad arguments"));
  if (pulse_init != OPMM_PULSE_TABLE1 && pulse_init != OPMM_PULSE_CALIBRATED)
    return fail(ctx, Status(OPMM_EINVAL, "unknown pulse_init"));
  if (n == 0) return OPMM_OK;
  TRY(ctx_bind(ctx));
  std::vector<DevSac> hs((size_t)n);
  for (int i = 0; i < n; ++i) {
    TRY(check_saccade(sacs[i], i, true));
    hs[(size_t)i] = make_devsac(sacs[i]);
  }
  cudaStream_t st = ctx->stream;
  DevBuf& b_sac = ctx->scratch[0];
  DevBuf& b_pc = ctx->scratch[7];
  TRY(b_sac.ensure(sizeof(DevSac) * (size_t)n));
  TRY(b_pc.ensure(sizeof(float) * OPMM_NPARAM * (size_t)n));
  CUDA_TRY(cudaMemcpyAsync(b_sac.ptr, hs.data(), sizeof(DevSac) * (size_t)n, cudaMemcpyHostToDevice, st), "H2D descriptors");
  CUDA_TRY(launch_nominal(b_sac.as<DevSac>(), n, pulse_init, nullptr, b_pc.as<float>(), st), "launch nominal");
  CUDA_TRY(cudaMemcpyAsync(out_opc, b_pc.ptr, sizeof(float) * OPMM_NPARAM * (size_t)n, cudaMemcpyDeviceToHost, st), "D2H opc");
  CUDA_TRY(cudaStreamSynchronize(st), "nominal");
  return OPMM_OK;
}

// ------------------------------------------------------------------ plans
// Search coordinates of a model: 18 (the OPC entries) or 9 (Table 2).
static int model_dim(int32_t model) { return model == OPMM_MODEL_9 ? 9 : OPMM_NPARAM; }

Status opmm::check_opts(const opmm_fit_opts& o) {
  if (o.model != OPMM_MODEL_18 && o.model != OPMM_MODEL_9)
    return Status(OPMM_EINVAL, "model must be OPMM_MODEL_18 or OPMM_MODEL_9");
  if (o.model == OPMM_MODEL_9 && o.use_surrogate)
    return Status(OPMM_EINVAL, "the surrogate estimates the 18-parameter model only");
  if (o.candidates < model_dim(o.model) + 4)
    return Status(OPMM_EINVAL, "candidates must cover one simplex's n + 4 trial points (22, or 13 for OPMM_MODEL_9)");
  if (o.iterations < 0 || o.iterations > 1000000) return Status(OPMM_EINVAL, "iterations outside [0, 1e6]");
  if (!(o.box_lo > 0.0f) || !(o.box_lo <= 1.0f) || !(o.box_hi >= 1.0f) || !std::isfinite(o.box_hi))
    return Status(OPMM_EINVAL, "box must satisfy 0 < box_lo <= 1 <= box_hi");
  if (!(o.init_step > 0.0f) || !std::isfinite(o.init_step)) return Status(OPMM_EINVAL, "init_step must be > 0");
  if (!(o.tol_x >= 0.0f) || !(o.tol_f >= 0.0f)) return Status(OPMM_EINVAL, "tolerances must be >= 0");
  if (o.pulse_init != OPMM_PULSE_TABLE1 && o.pulse_init != OPMM_PULSE_CALIBRATED)
    return Status(OPMM_EINVAL, "unknown pulse_init");
  return Status();
}

opmm_plan::~opmm_plan() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ev_search[0]) cudaEventDestroy(ev_search[0]);
  if (ev_search[1]) cudaEventDestroy(ev_search[1]);
}

namespace opmm {

// Trace staging and box centres, in stream order: device gather or one H2D
// copy of the packed traces, nominal centres (unless given), then any
// pre-search stage (the surrogate's re-centring).
Status enqueue_centres(opmm_plan* p, cudaStream_t st) {
  Status s;
  if (p->traces_on_device) {
    s = cuda_status(launch_gather(p->d_src.as<const float*>(), p->d_sacs.as<DevSac>(), p->d_traces.as<float>(), p->n, st),
                    "launch gather");
  } else {
    s = cuda_status(cudaMemcpyAsync(p->d_traces.ptr, p->h_traces.ptr, p->trace_floats * sizeof(float),
                                    cudaMemcpyHostToDevice, st), "H2D traces");
  }
  if (!s.ok()) return s;
  if (!p->centres_given) {
    s = cuda_status(launch_nominal(p->d_sacs.as<DevSac>(), p->n, p->opts.pulse_init, nullptr, p->d_pc.as<float>(), st),
                    "launch nominal");
    if (!s.ok()) return s;
  } else if (p->pre_search) {
    // the surrogate scales the caller's centres: restore them first
    s = cuda_status(cudaMemcpyAsync(p->d_pc.ptr, p->d_pc_given.ptr, sizeof(float) * OPMM_NPARAM * (size_t)p->n,
                                    cudaMemcpyDeviceToDevice, st), "restore centres");
    if (!s.ok()) return s;
  }
  if (p->pre_search) {
    s = p->pre_search(p, st);
    if (!s.ok()) return s;
  }
  return Status();
}

// Everything one fit launches, in stream order (graph-captured by plans).
Status enqueue_fit(opmm_plan* p, cudaStream_t st) {
  opmm_ctx* ctx = p->ctx;
  Status s;
  s = cuda_status(cudaMemsetAsync(ctx->d_err.ptr, 0, sizeof(unsigned), st), "clear error word");
  if (!s.ok()) return s;
  s = enqueue_centres(p, st);
  if (!s.ok()) return s;
  s = cuda_status(cudaMemsetAsync(p->d_counter.ptr, 0, sizeof(int), st), "clear work counter");
  if (!s.ok()) return s;
  SearchParams P = p->params;
  // inside stream capture the events become external record nodes of the
  // graph; outside capture they are plain records
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  s = cuda_status(cudaStreamIsCapturing(st, &cap), "query capture");
  if (!s.ok()) return s;
  const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (p->ev_search[0]) {
    s = cuda_status(cudaEventRecordWithFlags(p->ev_search[0], st, ev_flags), "record search start");
    if (!s.ok()) return s;
  }
  s = cuda_status(launch_search_v(p->variant, P, p->blocks_per_sm, ctx->num_sms, st), "launch search");
  if (!s.ok()) return s;
  if (p->ev_search[1]) {
    s = cuda_status(cudaEventRecordWithFlags(p->ev_search[1], st, ev_flags), "record search end");
    if (!s.ok()) return s;
  }
  s = cuda_status(launch_finalize(p->d_sacs.as<DevSac>(), p->d_traces.as<float>(), p->d_pc.as<float>(),
                                  p->d_ustart.as<int>(), p->ngroups, p->d_unit_best.as<float>(), P.lnlo, P.lnhi, p->n,
                                  p->d_results.as<opmm_fit_result>(), st, nullptr, p->dim),
                  "launch finalize");
  if (!s.ok()) return s;
  s = cuda_status(cudaMemcpyAsync(p->h_results.ptr, p->d_results.ptr, sizeof(opmm_fit_result) * (size_t)p->n,
                                  cudaMemcpyDeviceToHost, st), "D2H results");
  if (!s.ok()) return s;
  return cuda_status(cudaMemcpyAsync(p->h_err.ptr, ctx->d_err.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                     "D2H error word");
}

// Candidate launch shapes: the search kernel's variants (simplices per block G,
// threads = 22 G rounded to warps, register bound for MINB resident blocks) at
// the occupancy the device allows for this trace capacity.  Returns (variant,
// blocks per SM) pairs.
static std::vector<std::pair<int, int>> shape_candidates(int lcap, int dim) {
  std::vector<std::pair<int, int>> out;
  for (int v = 0; v < search_variant_count(); ++v) {
    if (search_variant_dim(v) != dim) continue;
    int bps = 0;
    if (search_occupancy_v(v, lcap, &bps) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (bps >= 1) out.push_back({v, bps});
  }
  return out;
}

// Project-written autotuner: time each candidate shape on a sample of this
// plan's own batch and keep the fastest; the choice is cached per (device,
// trace capacity, simplices, saccade count bucket).  The sample is every
// k-th saccade in the unit list's order (longest windows first), about
// kProbeSimplices simplices in all, run for the plan's own iteration count
// (at most kProbeIters): shapes differ in how they overlap a group's
// decisions with the other groups' evaluation, which the steady state of a
// whole search shows and the first iterations do not (a two-iteration probe
// picked 3 x 24 where 2 x 32 runs the 30-iteration batch fit 4% faster).
// Results of probe runs are overwritten by the real run.
static Status autotune(opmm_plan* p) {
  opmm_ctx* ctx = p->ctx;
  // the probes run the plan's own iteration count (at most 32), so it is part
  // of the key, with the model's coordinate count
  const auto key = std::make_tuple(p->lcap, p->S, p->n >= 64 ? 64 : p->n,
                                   std::min(p->opts.iterations, 32) * 64 + (p->dim << 1));
  auto it = ctx->tune_cache.find(key);
  auto cands = shape_candidates(p->lcap, p->dim);
  if (cands.empty()) return Status(OPMM_ECUDA, "no launchable search shape (shared memory)");
  if (ctx->forced_variant >= 0) {
    for (auto& cd : cands)
      if (cd.first == ctx->forced_variant) {
        p->variant = cd.first;
        p->blocks_per_sm = cd.second;
        return Status();
      }
    return Status(OPMM_EINVAL, "forced search variant cannot be launched with this batch or model");
  }
  if (it != ctx->tune_cache.end()) {
    p->variant = it->second.first;
    p->blocks_per_sm = it->second.second;
    p->tune_log = ctx->tune_logs[key];
    return Status();
  }
  if (!p->autotune || cands.size() == 1) {
    p->variant = cands[0].first;        // variant 0 (16 simplices per block) when launchable
    p->blocks_per_sm = cands[0].second;
    return Status();
  }
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  Status s = cuda_status(cudaEventCreate(&e0), "event");
  if (!s.ok()) return s;
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  std::pair<int, int> best = cands[0];
  constexpr long long kProbeSimplices = 160000;
  constexpr int kProbeIters = 32;   // also in the cache key above
  const long long want = std::max(1LL, (kProbeSimplices + p->S - 1) / std::max(1, p->S));
  const int stride = (int)std::max(1LL, (long long)p->n / want);
  for (auto& c : cands) {
    // the unit list depends on G: rebuild it (the probe's sample) for the probe
    s = build_units(p, search_variant_g(c.first), stride);
    if (!s.ok()) break;
    SearchParams P = p->params;
    P.T = std::min(p->opts.iterations, kProbeIters);
    // each shape runs twice and the second run is timed: the first launch of
    // a kernel also pays for loading it
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && s.ok(); ++rep) {
      cudaMemsetAsync(p->d_counter.ptr, 0, sizeof(int), st);
      cudaEventRecord(e0, st);
      cudaError_t le = launch_search_v(c.first, P, c.second, ctx->num_sms, st);
      cudaEventRecord(e1, st);
      cudaError_t se = cudaStreamSynchronize(st);
      if (le != cudaSuccess || se != cudaSuccess) s = cuda_status(le != cudaSuccess ? le : se, "autotune probe");
      else cudaEventElapsedTime(&ms, e0, e1);
    }
    if (!s.ok()) break;
    p->tune_log.push_back({c.first, c.second, ms});
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!s.ok()) return s;
  p->variant = best.first;
  p->blocks_per_sm = best.second;
  ctx->tune_cache[key] = best;
  ctx->tune_logs[key] = p->tune_log;
  return Status();
}

// Unit list for G simplices per block: saccades in decreasing order of work
// (samples after onset), each split into ceil(S / G) groups of simplices.
// With probe_stride k > 1, the autotuner's sample: only the saccades at
// positions k/2, k/2 + k, ... of that order (the unit starts are then not
// meaningful; no result is read from a probe).
Status build_units(opmm_plan* p, int G, int probe_stride) {
  p->ngroups = (p->S + G - 1) / G;
  const size_t nu = (size_t)p->n * (size_t)p->ngroups;
  if (nu > (size_t)0x7fffffff) return Status(OPMM_EINVAL, "too many work units");
  std::vector<int> order((size_t)p->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int wa = p->hsacs[(size_t)a].L - p->hsacs[(size_t)a].onset;
    const int wb = p->hsacs[(size_t)b].L - p->hsacs[(size_t)b].onset;
    return wa > wb;
  });
  std::vector<int2> units(nu);
  std::vector<int> ustart((size_t)p->n);
  size_t u = 0;
  for (size_t k = 0; k < order.size(); ++k) {
    const int b = order[k];
    ustart[(size_t)b] = (int)u;
    if (probe_stride > 1 && (int)(k % (size_t)probe_stride) != probe_stride / 2) continue;
    for (int g = 0; g < p->ngroups; ++g) units[u++] = make_int2(b, g);
  }
  p->n_units = (int)u;
  Status s = p->d_units.ensure(nu * sizeof(int2));
  if (s.ok()) s = p->d_ustart.ensure((size_t)p->n * sizeof(int));
  if (s.ok()) s = p->d_unit_best.ensure(nu * kUnitRecFloats * sizeof(float));
  if (!s.ok()) return s;
  cudaStream_t st = p->ctx->stream;
  s = cuda_status(cudaMemcpyAsync(p->d_units.ptr, units.data(), nu * sizeof(int2), cudaMemcpyHostToDevice, st), "H2D units");
  if (s.ok())
    s = cuda_status(cudaMemcpyAsync(p->d_ustart.ptr, ustart.data(), (size_t)p->n * sizeof(int), cudaMemcpyHostToDevice, st),
                    "H2D unit starts");
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "stage units");
  p->params.units = p->d_units.as<int2>();
  p->params.n_units = p->n_units;
  p->params.ngroups = p->ngroups;
  p->params.balanced = 0;
  p->params.unit_best = p->d_unit_best.as<float>();
  return s;
}

// Validate, stage descriptors and traces, allocate, compute the box centres.
Status plan_stage(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts& o, opmm_plan* p) {
  Status s = check_opts(o);
  if (!s.ok()) return s;
  if (n < 1 || !sacs) return Status(OPMM_EINVAL, "empty batch");
  p->ctx = ctx;
  p->n = n;
  p->opts = o;
  p->opts.init_opc = nullptr;
  p->dim = model_dim(o.model);
  p->S = o.candidates / (p->dim + 4);
  p->centres_given = o.init_opc != nullptr;
  p->hsacs.resize((size_t)n);
  p->src.resize((size_t)n);
  int lmax = 0;
  long long off = 0;
  for (int i = 0; i < n; ++i) {
    s = check_saccade(sacs[i], i, o.init_opc == nullptr);
    if (!s.ok()) return s;
    if (!sacs[i].trace_deg) return Status(OPMM_EINVAL, "saccade " + std::to_string(i) + ": null trace");
    DevSac d = make_devsac(sacs[i]);
    d.off = off;
    off += (d.L + 3) & ~3;
    lmax = std::max(lmax, d.L);
    p->hsacs[(size_t)i] = d;
    p->src[(size_t)i] = sacs[i].trace_deg;
  }
  p->trace_floats = (size_t)off;
  p->lcap = (lmax + 3) & ~3;
  p->traces_on_device = is_device_ptr(sacs[0].trace_deg);
  for (int i = 1; i < n; ++i)
    if (is_device_ptr(sacs[i].trace_deg) != p->traces_on_device)
      return Status(OPMM_EINVAL, "all traces of a batch must be host memory or all device memory");
  if (o.init_opc)
    for (int i = 0; i < n; ++i) {
      const float* c = o.init_opc + (size_t)i * OPMM_NPARAM;
      s = check_opc(c);
      if (!s.ok()) return s;
      // the 9-parameter model scales one shared series elasticity and one
      // shared length-tension coefficient: the centre must give both muscles
      // the same values
      if (p->dim == 9 && (c[0] != c[1] || c[2] != c[3]))
        return Status(OPMM_EINVAL, "saccade " + std::to_string(i) +
                                       ": OPMM_MODEL_9 needs K_SE_AG == K_SE_ANT and K_LT_AG == K_LT_ANT in init_opc");
    }
  cudaStream_t st = ctx->stream;
  s = p->d_sacs.ensure(sizeof(DevSac) * (size_t)n);
  if (s.ok()) s = p->d_traces.ensure(sizeof(float) * p->trace_floats);
  if (s.ok()) s = p->d_pc.ensure(sizeof(float) * OPMM_NPARAM * (size_t)n);
  if (s.ok()) s = p->d_sac_index.ensure(sizeof(int) * (size_t)n);
  if (s.ok()) s = p->d_counter.ensure(sizeof(int));
  if (s.ok()) s = p->d_results.ensure(sizeof(opmm_fit_result) * (size_t)n);
  if (s.ok()) s = p->h_results.ensure(sizeof(opmm_fit_result) * (size_t)n);
  if (s.ok()) s = p->h_err.ensure(sizeof(unsigned));
  if (s.ok() && p->traces_on_device) s = p->d_src.ensure(sizeof(float*) * (size_t)n);
  if (s.ok() && !p->traces_on_device) s = p->h_traces.ensure(sizeof(float) * p->trace_floats);
  if (!s.ok()) return s;
  std::vector<int> sidx((size_t)n);
  for (int i = 0; i < n; ++i) sidx[(size_t)i] = p->sac_index_base + i;
  s = cuda_status(cudaMemcpyAsync(p->d_sacs.ptr, p->hsacs.data(), sizeof(DevSac) * (size_t)n, cudaMemcpyHostToDevice, st),
                  "H2D descriptors");
  if (s.ok())
    s = cuda_status(cudaMemcpyAsync(p->d_sac_index.ptr, sidx.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st),
                    "H2D saccade index");
  if (s.ok() && p->traces_on_device)
    s = cuda_status(cudaMemcpyAsync(p->d_src.ptr, p->src.data(), sizeof(float*) * (size_t)n, cudaMemcpyHostToDevice, st),
                    "H2D trace pointers");
  if (s.ok() && o.init_opc)
    s = cuda_status(cudaMemcpyAsync(p->d_pc.ptr, o.init_opc, sizeof(float) * OPMM_NPARAM * (size_t)n,
                                    cudaMemcpyHostToDevice, st), "H2D box centres");
  if (s.ok() && o.init_opc && o.use_surrogate) {
    s = p->d_pc_given.ensure(sizeof(float) * OPMM_NPARAM * (size_t)n);
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(p->d_pc_given.ptr, o.init_opc, sizeof(float) * OPMM_NPARAM * (size_t)n,
                                      cudaMemcpyHostToDevice, st), "H2D box centres");
  }
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "stage plan");
  if (!s.ok()) return s;

  SearchParams& P = p->params;
  P.sacs = p->d_sacs.as<DevSac>();
  P.traces = p->d_traces.as<float>();
  P.pc = p->d_pc.as<float>();
  P.sac_index = p->d_sac_index.as<int>();
  P.S = p->S;
  P.T = o.iterations;
  P.lcap = p->lcap;
  P.lnlo = (float)std::log((double)o.box_lo);
  P.lnhi = (float)std::log((double)o.box_hi);
  P.step = o.init_step;
  P.tolx = o.tol_x;
  P.tolf = o.tol_f;
  P.seed_lo = (uint32_t)(o.seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(o.seed >> 32);
  P.counter = p->d_counter.as<int>();
  P.err = ctx->d_err.as<unsigned>();

  // stage the traces and centres now (the tuner's probes and direct callers need them)
  if (!p->traces_on_device) pack_host_traces(p);
  s = enqueue_centres(p, st);
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "stage");
  return s;
}

// plan_stage, then the search part: launch shape, work units, graph capture.
Status plan_build(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts& o, bool capture,
                  bool tune, opmm_plan* p) {
  p->autotune = tune;
  Status s = plan_stage(ctx, sacs, n, o, p);
  if (!s.ok()) return s;
  cudaStream_t st = ctx->stream;
  s = autotune(p);
  if (!s.ok()) return s;
  p->G = search_variant_g(p->variant);
  s = build_units(p, p->G);
  if (!s.ok()) return s;
  p->threads = search_variant_threads(p->variant);
  s = cuda_status(cudaEventCreate(&p->ev_search[0]), "event");
  if (s.ok()) s = cuda_status(cudaEventCreate(&p->ev_search[1]), "event");
  if (!s.ok()) return s;
  if (capture) {
    cudaStream_t cs = st;
    s = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!s.ok()) return s;
    Status es = enqueue_fit(p, cs);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (!es.ok()) {
      if (g) cudaGraphDestroy(g);
      return es;
    }
    s = cuda_status(ee, "end capture");
    if (!s.ok()) return s;
    p->graph = g;
    s = cuda_status(cudaGraphInstantiate(&p->exec, g, 0), "instantiate graph");
    if (!s.ok()) return s;
  }
  return Status();
}

void pack_host_traces(opmm_plan* p) {
  float* dst = p->h_traces.as<float>();
  for (int i = 0; i < p->n; ++i) {
    const DevSac& d = p->hsacs[(size_t)i];
    std::memcpy(dst + d.off, p->src[(size_t)i], sizeof(float) * (size_t)d.L);
    for (int k = d.L; k < ((d.L + 3) & ~3); ++k) dst[d.off + k] = 0.0f;
  }
}

Status plan_run(opmm_plan* p, opmm_fit_result* out) {
  opmm_ctx* ctx = p->ctx;
  Status s = cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!s.ok()) return s;
  if (!p->traces_on_device) pack_host_traces(p);
  cudaStream_t st = ctx->stream;
  if (p->exec) s = cuda_status(cudaGraphLaunch(p->exec, st), "graph launch");
  else s = enqueue_fit(p, st);
  if (!s.ok()) return s;
  s = cuda_status(cudaStreamSynchronize(st), "fit");
  if (!s.ok()) return s;
  const unsigned e = *p->h_err.as<unsigned>();
  if (e & kErrWaitTimeout) return Status(OPMM_ETIMEDOUT, "a kernel's bounded TMA wait expired");
  if (e) return Status(OPMM_ECUDA, "kernel error bits " + std::to_string(e));
  if (out) {
    std::memcpy(out, p->h_results.ptr, sizeof(opmm_fit_result) * (size_t)p->n);
    if (p->opts.use_surrogate)
      for (int i = 0; i < p->n; ++i) out[i].source = OPMM_SOURCE_SEEDED;
  }
  return Status();
}

}  // namespace opmm

extern "C" int opmm_plan_create(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts* opts,
                                opmm_plan** out) {
  if (!ctx) return OPMM_EINVAL;
  if (!opts || !out) return fail(ctx, Status(OPMM_EINVAL, "opmm_plan_create: null argument"));
  *out = nullptr;
  TRY(ctx_bind(ctx));
  opmm_plan* p = new (std::nothrow) opmm_plan();
  if (!p) return fail(ctx, Status(OPMM_ENOMEM, "plan allocation"));
  Status s;
  try {
    if (opts->use_surrogate) s = surrogate_prepare_plan(ctx, p, sacs, n);
    if (s.ok()) s = plan_build(ctx, sacs, n, *opts, true, true, p);
  } catch (const std::bad_alloc&) {
    s = Status(OPMM_ENOMEM, "host allocation failed");
  }
  if (!s.ok()) {
    delete p;
    return fail(ctx, s);
  }
  *out = p;
  return OPMM_OK;
}

extern "C" int opmm_plan_execute(opmm_plan* plan, opmm_fit_result* out) {
  if (!plan) return OPMM_EINVAL;
  opmm_ctx* ctx = plan->ctx;
  if (!out) return fail(ctx, Status(OPMM_EINVAL, "null output"));
  TRY(plan_run(plan, out));
  return OPMM_OK;
}

extern "C" int opmm_plan_info(const opmm_plan* plan, int32_t* g, int32_t* threads, int32_t* bps, int32_t* kernels) {
  if (!plan) return OPMM_EINVAL;
  if (g) *g = plan->G;
  if (threads) *threads = plan->threads;
  if (bps) *bps = plan->blocks_per_sm;
  if (kernels) *kernels = (plan->traces_on_device ? 1 : 0) + (plan->centres_given ? 0 : 1) + plan->pre_search_kernels + 2;
  return OPMM_OK;
}

extern "C" int opmm_plan_variant(const opmm_plan* plan, int32_t* variant) {
  if (!plan || !variant) return OPMM_EINVAL;
  *variant = plan->variant;
  return OPMM_OK;
}

extern "C" int opmm_plan_tuning(const opmm_plan* plan, int32_t* variant, int32_t* simplices_per_block,
                                int32_t* min_blocks, int32_t* blocks_per_sm, float* probe_ms, int32_t cap,
                                int32_t* count) {
  if (!plan || !count || cap < 0) return OPMM_EINVAL;
  const int n = (int)plan->tune_log.size();
  *count = n;
  for (int i = 0; i < n && i < cap; ++i) {
    const auto& t = plan->tune_log[(size_t)i];
    if (variant) variant[i] = t.variant;
    if (simplices_per_block) simplices_per_block[i] = search_variant_g(t.variant);
    if (min_blocks) min_blocks[i] = search_variant_minb(t.variant);
    if (blocks_per_sm) blocks_per_sm[i] = t.bps;
    if (probe_ms) probe_ms[i] = t.ms;
  }
  return OPMM_OK;
}

extern "C" int opmm_plan_last_search_ms(const opmm_plan* plan, float* ms) {
  if (!plan || !ms) return OPMM_EINVAL;
  if (!plan->ev_search[0] || !plan->ev_search[1]) return OPMM_EINVAL;
  cudaError_t e = cudaEventElapsedTime(ms, plan->ev_search[0], plan->ev_search[1]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return OPMM_NOT_READY;
  }
  return OPMM_OK;
}

extern "C" void opmm_plan_destroy(opmm_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->ctx->device);
  delete plan;
}

static Status fit_once(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts& o,
                       opmm_fit_result* out) {
  opmm_plan p;
  Status s;
  try {
    if (o.use_surrogate) s = surrogate_prepare_plan(ctx, &p, sacs, n);
    if (s.ok()) s = plan_build(ctx, sacs, n, o, false, false, &p);
    if (s.ok()) s = plan_run(&p, out);
  } catch (const std::bad_alloc&) {
    s = Status(OPMM_ENOMEM, "host allocation failed");
  }
  return s;
}

extern "C" int opmm_fit_batch(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts* opts,
                              opmm_fit_result* out) {
  if (!ctx) return OPMM_EINVAL;
  if (!opts || !out) return fail(ctx, Status(OPMM_EINVAL, "opmm_fit_batch: null argument"));
  TRY(ctx_bind(ctx));
  TRY(fit_once(ctx, sacs, n, *opts, out));
  return OPMM_OK;
}

// Levenberg-Marquardt refinement of given OPC vectors (see kernels.cu,
// k_refine): staging and box centres as a plan of the same model, then one
// block per saccade.
extern "C" int opmm_refine_batch(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const float* start_opc,
                                 const opmm_refine_opts* ro, opmm_fit_result* out) {
  if (!ctx) return OPMM_EINVAL;
  if (!ro || !out || !start_opc) return fail(ctx, Status(OPMM_EINVAL, "opmm_refine_batch: null argument"));
  if (ro->iterations < 0 || ro->iterations > 10000)
    return fail(ctx, Status(OPMM_EINVAL, "opmm_refine_batch: iterations outside [0, 1e4]"));
  if (!(ro->fd_step > 0.0f) || !std::isfinite(ro->fd_step) || !(ro->lambda0 > 0.0f) || !std::isfinite(ro->lambda0))
    return fail(ctx, Status(OPMM_EINVAL, "opmm_refine_batch: fd_step and lambda0 must be finite and > 0"));
  if (n < 1) return fail(ctx, Status(OPMM_EINVAL, "opmm_refine_batch: empty batch"));
  if (is_device_ptr(start_opc)) return fail(ctx, Status(OPMM_EINVAL, "opmm_refine_batch: start_opc must be host memory"));
  for (int i = 0; i < n; ++i) TRY(check_opc(start_opc + (size_t)i * OPMM_NPARAM));
  TRY(ctx_bind(ctx));
  opmm_fit_opts fo{};
  fo.model = ro->model;
  fo.candidates = (ro->model == OPMM_MODEL_9 ? 9 : OPMM_NPARAM) + 4;
  fo.iterations = 0;
  fo.box_lo = ro->box_lo;
  fo.box_hi = ro->box_hi;
  fo.init_step = 0.05f;
  fo.pulse_init = ro->pulse_init;
  fo.init_opc = ro->centre_opc;
  opmm_plan p;
  TRY(plan_stage(ctx, sacs, n, fo, &p));
  cudaStream_t st = ctx->stream;
  DevBuf& b_start = ctx->scratch[8];
  DevBuf& b_rows = ctx->scratch[9];
  DevBuf& b_out = ctx->scratch[10];
  const size_t rows = (size_t)n * (2 * (size_t)p.dim + 2) * (size_t)p.lcap;
  TRY(b_start.ensure(sizeof(float) * OPMM_NPARAM * (size_t)n));
  TRY(b_rows.ensure(sizeof(float) * rows));
  TRY(b_out.ensure(sizeof(opmm_fit_result) * (size_t)n));
  CUDA_TRY(cudaMemcpyAsync(b_start.ptr, start_opc, sizeof(float) * OPMM_NPARAM * (size_t)n, cudaMemcpyHostToDevice, st),
           "H2D start");
  CUDA_TRY(cudaMemsetAsync(ctx->d_err.ptr, 0, sizeof(unsigned), st), "clear error word");
  CUDA_TRY(launch_refine(p.dim, p.d_sacs.as<DevSac>(), p.d_traces.as<float>(), p.d_pc.as<float>(), b_start.as<float>(), n,
                         ro->iterations, p.params.lnlo, p.params.lnhi, ro->fd_step, ro->lambda0, p.lcap,
                         b_rows.as<float>(), b_out.as<opmm_fit_result>(), ctx->d_err.as<unsigned>(), st),
           "launch refine");
  unsigned e = 0;
  CUDA_TRY(cudaMemcpyAsync(out, b_out.ptr, sizeof(opmm_fit_result) * (size_t)n, cudaMemcpyDeviceToHost, st), "D2H results");
  CUDA_TRY(cudaMemcpyAsync(&e, ctx->d_err.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "D2H error word");
  CUDA_TRY(cudaStreamSynchronize(st), "refine");
  if (e & kErrWaitTimeout) return fail(ctx, Status(OPMM_ETIMEDOUT, "a kernel's bounded TMA wait expired"));
  if (e) return fail(ctx, Status(OPMM_ECUDA, "kernel error bits " + std::to_string(e)));
  return OPMM_OK;
}

extern "C" int opmm_fit_batch_seeded(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts* seeded,
                                     const opmm_fit_opts* plain, float fallback_rms_deg, opmm_fit_result* out,
                                     int32_t* n_fallback) {
  if (!ctx) return OPMM_EINVAL;
  if (!seeded || !plain || !out) return fail(ctx, Status(OPMM_EINVAL, "opmm_fit_batch_seeded: null argument"));
  if (!seeded->use_surrogate || plain->use_surrogate)
    return fail(ctx, Status(OPMM_EINVAL, "opmm_fit_batch_seeded: seeded must use the surrogate, plain must not"));
  if (!(fallback_rms_deg >= 0.0f)) return fail(ctx, Status(OPMM_EINVAL, "opmm_fit_batch_seeded: fallback_rms_deg < 0"));
  if (n_fallback) *n_fallback = 0;
  TRY(ctx_bind(ctx));
  TRY(fit_once(ctx, sacs, n, *seeded, out));
  // saccades the seeded search did not fit well enough go to the plain search
  std::vector<int> miss;
  for (int i = 0; i < n; ++i)
    if (out[i].status != 0 || !(out[i].rms_deg <= (double)fallback_rms_deg)) miss.push_back(i);
  if (n_fallback) *n_fallback = (int32_t)miss.size();
  if (miss.empty()) return OPMM_OK;
  const size_t m = miss.size();
  std::vector<opmm_saccade> sub(m);
  std::vector<float> sub_pc;
  for (size_t j = 0; j < m; ++j) sub[j] = sacs[miss[j]];
  opmm_fit_opts po = *plain;
  if (plain->init_opc) {
    sub_pc.resize(m * 18);
    for (size_t j = 0; j < m; ++j)
      std::memcpy(&sub_pc[j * 18], plain->init_opc + (size_t)miss[j] * 18, 18 * sizeof(float));
    po.init_opc = sub_pc.data();
  }
  std::vector<opmm_fit_result> fb(m);
  TRY(fit_once(ctx, sub.data(), (int32_t)m, po, fb.data()));
  for (size_t j = 0; j < m; ++j) {
    opmm_fit_result& r = out[miss[j]];
    const int32_t evals = r.evaluations + fb[j].evaluations;
    const int32_t pe = r.pulse_end_evals + fb[j].pulse_end_evals;
    const bool better = fb[j].status == 0 && (r.status != 0 || fb[j].rms_deg < r.rms_deg);
    if (better) {
      r = fb[j];
      r.source = OPMM_SOURCE_FALLBACK;
    }
    r.evaluations = evals;
    r.pulse_end_evals = pe;
  }
  return OPMM_OK;
}
