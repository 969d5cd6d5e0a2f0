// ivt.cu -- front end: velocity-threshold (I-VT) saccade detection and
// cleaning of raw position streams on the device, producing the windows and
// descriptors the estimator takes (the paper segments its recordings with
// I-VT and drops saccades shorter than 6 ms or smaller than 4 deg, Sec. 4;
// the threshold and the cleaning rule are the caller's, see opmm.h).
//
// Step k (samples k - 1, k) is fast when both samples are valid (finite, in
// [valid_min, valid_max]) and |x_k - x_(k-1)| * fs > threshold, in FP32.  A
// saccade is a maximal run of fast steps [a, b): onset sample s = a - 1, end
// sample e = b - 1.  Pass 1 (HBM bound, grid-stride over the stream) records
// every run start; pass 2 walks each run and its window, one thread per run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/opmm.h"
#include "launch.h"
#include "runtime.h"

namespace opmm {

namespace {

struct IvtDev {
  const float* x;
  long long n;
  float fs, thr, vmin, vmax, min_dur, min_amp;
  int pre, post;
};

__device__ __forceinline__ bool ivt_valid(float v, const IvtDev& P) {
  return isfinite(v) && v >= P.vmin && v <= P.vmax;
}

// |x_k - x_(k-1)| * fs, or -1 when the step is not between two valid samples.
__device__ __forceinline__ float ivt_speed(const IvtDev& P, long long k) {
  if (k < 1 || k >= P.n) return -1.0f;
  const float a = P.x[k - 1], b = P.x[k];
  if (!ivt_valid(a, P) || !ivt_valid(b, P)) return -1.0f;
  return fabsf(b - a) * P.fs;
}

// Pass 1: the first step of every run of fast steps.
__global__ void k_ivt_starts(IvtDev P, long long* starts, int cap, int* count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = 1 + (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P.n; k += stride) {
    const bool f = ivt_speed(P, k) > P.thr;
    if (!f) continue;
    const bool fp = ivt_speed(P, k - 1) > P.thr;
    if (fp) continue;
    const int i = atomicAdd(count, 1);
    if (i < cap) starts[i] = k;
  }
}

// Pass 2: one thread per run: its end, amplitude, duration, peak velocity,
// the window check and the event record; keep[i] = 1 for a kept saccade.
__global__ void k_ivt_events(IvtDev P, const long long* starts, const int* count, int cap, opmm_ivt_event* ev,
                             int* keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = min(*count, cap);
  if (i >= m) return;
  const long long a = starts[i];
  long long b = a;
  float peak = 0.0f;
  for (;;) {
    const float sp = ivt_speed(P, b);
    if (!(sp > P.thr)) break;
    peak = fmaxf(peak, sp);
    ++b;
  }
  const long long s = a - 1, e = b - 1;
  const float xs = P.x[s], xe = P.x[e];
  const float amp = fabsf(xe - xs);
  const float dur = ((float)(e - s) * 1000.0f) / P.fs;
  const long long ws = s - P.pre, we = e + P.post;
  bool ok = dur >= P.min_dur && amp >= P.min_amp && ws >= 0 && we <= P.n - 1;
  for (long long k = ws; ok && k <= we; ++k) ok = ivt_valid(P.x[k], P);
  opmm_ivt_event r;
  r.onset = s;
  r.end = e;
  r.window_start = ws;
  r.n_samples = (int32_t)(we - ws + 1);
  r.onset_index = (int32_t)(s - ws);
  r.theta_start_deg = xs;
  r.theta_end_deg = xe;
  r.amplitude_deg = amp;
  r.duration_ms = dur;
  r.peak_velocity_dps = peak;
  r.reserved = 0;
  ev[i] = r;
  keep[i] = ok ? 1 : 0;
}

int ivt_fail(const Status& s) {
  set_last_error(s.msg);
  return s.code;
}

}  // namespace

}  // namespace opmm

using namespace opmm;

extern "C" int opmm_detect_saccades(opmm_ctx* ctx, const float* stream_deg, int64_t n_samples, float sample_rate_hz,
                                    const opmm_ivt_opts* opts, opmm_ivt_event* out, int32_t max_events,
                                    int32_t* n_events) {
  if (!ctx) return OPMM_EINVAL;
  if (!stream_deg || !opts || !n_events || (max_events > 0 && !out))
    return ivt_fail(Status(OPMM_EINVAL, "opmm_detect_saccades: null argument"));
  if (n_samples < 2 || n_samples > (int64_t)1 << 40)
    return ivt_fail(Status(OPMM_EINVAL, "opmm_detect_saccades: n_samples outside [2, 2^40]"));
  if (!(sample_rate_hz > 0.0f) || !std::isfinite(sample_rate_hz) || !(opts->threshold_dps > 0.0f) ||
      !std::isfinite(opts->threshold_dps) || !(opts->min_duration_ms >= 0.0f) || !(opts->min_amplitude_deg >= 0.0f) ||
      !(opts->valid_min_deg <= opts->valid_max_deg) || opts->pre_samples < 0 || opts->post_samples < 0 ||
      max_events < 0)
    return ivt_fail(Status(OPMM_EINVAL, "opmm_detect_saccades: bad options"));
  Status s = cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!s.ok()) return ivt_fail(s);
  cudaStream_t st = ctx->stream;
  const float* x = stream_deg;
  DevBuf& b_x = ctx->scratch[11];
  DevBuf& b_starts = ctx->scratch[12];
  DevBuf& b_ev = ctx->scratch[13];
  DevBuf& b_keep = ctx->scratch[14];
  DevBuf& b_count = ctx->scratch[15];
  if (!is_device_ptr(stream_deg)) {
    s = b_x.ensure(sizeof(float) * (size_t)n_samples);
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(b_x.ptr, stream_deg, sizeof(float) * (size_t)n_samples, cudaMemcpyHostToDevice, st),
                      "H2D stream");
    if (!s.ok()) return ivt_fail(s);
    x = b_x.as<float>();
  }
  // a run needs a fast step and a slower one before it: at most n / 2 starts,
  // and at most 2^24 are kept track of (a noisier stream is refused)
  const long long cap_ll = std::min<long long>(n_samples / 2 + 1, (long long)1 << 24);
  const int cap = (int)cap_ll;
  s = b_starts.ensure(sizeof(long long) * (size_t)cap);
  if (s.ok()) s = b_count.ensure(sizeof(int));
  if (s.ok()) s = cuda_status(cudaMemsetAsync(b_count.ptr, 0, sizeof(int), st), "clear count");
  if (!s.ok()) return ivt_fail(s);
  IvtDev P{x, (long long)n_samples, sample_rate_hz, opts->threshold_dps, opts->valid_min_deg, opts->valid_max_deg,
           opts->min_duration_ms, opts->min_amplitude_deg, opts->pre_samples, opts->post_samples};
  const int threads = 256;
  const long long want = (n_samples + threads - 1) / threads;
  const int blocks = (int)std::min<long long>(want, (long long)ctx->num_sms * 8);
  k_ivt_starts<<<blocks, threads, 0, st>>>(P, b_starts.as<long long>(), cap, b_count.as<int>());
  s = cuda_status(cudaGetLastError(), "launch I-VT starts");
  int count = 0;
  if (s.ok()) s = cuda_status(cudaMemcpyAsync(&count, b_count.ptr, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H count");
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "I-VT starts");
  if (!s.ok()) return ivt_fail(s);
  if (count > cap)
    return ivt_fail(Status(OPMM_ENOMEM, "opmm_detect_saccades: more than 2^24 velocity runs (raise the threshold)"));
  const int m = std::min(count, cap);
  std::vector<opmm_ivt_event> hev((size_t)m);
  std::vector<int> hkeep((size_t)m);
  if (m > 0) {
    s = b_ev.ensure(sizeof(opmm_ivt_event) * (size_t)m);
    if (s.ok()) s = b_keep.ensure(sizeof(int) * (size_t)m);
    if (!s.ok()) return ivt_fail(s);
    k_ivt_events<<<(m + 127) / 128, 128, 0, st>>>(P, b_starts.as<long long>(), b_count.as<int>(), cap,
                                                  b_ev.as<opmm_ivt_event>(), b_keep.as<int>());
    s = cuda_status(cudaGetLastError(), "launch I-VT events");
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(hev.data(), b_ev.ptr, sizeof(opmm_ivt_event) * (size_t)m, cudaMemcpyDeviceToHost, st),
                      "D2H events");
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(hkeep.data(), b_keep.ptr, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, st),
                      "D2H keep");
    if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "I-VT events");
    if (!s.ok()) return ivt_fail(s);
  }
  // kept events in onset order (pass 1 finds runs in no particular order)
  std::vector<opmm_ivt_event> kept;
  kept.reserve((size_t)m);
  for (int i = 0; i < m; ++i)
    if (hkeep[(size_t)i]) kept.push_back(hev[(size_t)i]);
  std::sort(kept.begin(), kept.end(), [](const opmm_ivt_event& a, const opmm_ivt_event& b) { return a.onset < b.onset; });
  *n_events = (int32_t)std::min<size_t>(kept.size(), (size_t)0x7fffffff);
  const size_t w = std::min<size_t>(kept.size(), (size_t)max_events);
  for (size_t i = 0; i < w; ++i) out[i] = kept[i];
  return OPMM_OK;
}
