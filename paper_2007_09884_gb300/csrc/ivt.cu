// ivt.cu -- front end: velocity-threshold (I-VT) saccade detection and
// cleaning of raw position streams on the device, producing the windows and
// descriptors the estimator takes (the paper segments its recordings with
// I-VT and drops saccades shorter than 6 ms or smaller than 4 deg, Sec. 4;
// the threshold and the cleaning rule are the caller's, see opmm.h).
//
// Step k (samples k - 1, k) is fast when both samples are valid (finite, in
// [valid_min, valid_max]) and |x_k - x_(k-1)| * fs > threshold, in FP32.  A
// saccade is a maximal run of fast steps [a, b): onset sample s = a - 1, end
// sample e = b - 1.  Run starts are compacted in stream order in two HBM
// passes over tiles of kTile steps (count per tile, scan of the counts, write
// at the tile's offset by warp ballots); then one thread per run walks the
// run and its window.
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

constexpr int kIvtThreads = 256;
constexpr int kIvtIters = 16;
constexpr long long kTile = (long long)kIvtThreads * kIvtIters;   // steps per tile (one block)

// step k starts a run of fast steps
__device__ __forceinline__ bool ivt_run_start(const IvtDev& P, long long k) {
  return ivt_speed(P, k) > P.thr && !(ivt_speed(P, k - 1) > P.thr);
}

// Pass 1a: run starts per tile.  Steps of a tile are visited in order
// (iteration, warp, lane), consecutive lanes on consecutive samples.
__global__ void __launch_bounds__(kIvtThreads) k_ivt_count(IvtDev P, int* tile_count) {
  const long long t0 = 1 + (long long)blockIdx.x * kTile;
  int c = 0;
#pragma unroll 4
  for (int it = 0; it < kIvtIters; ++it) {
    const long long k = t0 + (long long)it * kIvtThreads + threadIdx.x;
    c += (k < P.n && ivt_run_start(P, k)) ? 1 : 0;
  }
  __shared__ int warp_sum[kIvtThreads / 32];
  int v = c;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int sum = 0;
    for (int w = 0; w < kIvtThreads / 32; ++w) sum += warp_sum[w];
    tile_count[blockIdx.x] = sum;
  }
}

// Exclusive scan of the tile counts (one block); total written to *total.
__global__ void k_ivt_scan(const int* tile_count, int ntiles, long long* tile_off, long long* total) {
  __shared__ long long part[1024];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += 1024) {
    const int i = base + (int)threadIdx.x;
    const long long v = i < ntiles ? tile_count[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const long long add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < ntiles) tile_off[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Pass 1b: write each tile's run starts at its offset, in stream order.
__global__ void __launch_bounds__(kIvtThreads) k_ivt_write(IvtDev P, const long long* tile_off, long long* starts) {
  __shared__ int warp_cnt[kIvtThreads / 32];
  const long long t0 = 1 + (long long)blockIdx.x * kTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long run = tile_off[blockIdx.x];
  for (int it = 0; it < kIvtIters; ++it) {
    const long long k = t0 + (long long)it * kIvtThreads + threadIdx.x;
    const bool f = k < P.n && ivt_run_start(P, k);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < kIvtThreads / 32; ++w) {
      before += w < warp ? warp_cnt[w] : 0;
      all += warp_cnt[w];
    }
    if (f) starts[run + before + __popc(m & ((1u << lane) - 1u))] = k;
    run += all;
    __syncthreads();
  }
}

// Pass 2: one thread per run: its end, amplitude, duration, peak velocity,
// the window check and the event record; keep[i] = 1 for a kept saccade.
__global__ void k_ivt_events(IvtDev P, const long long* starts, int m, opmm_ivt_event* ev, int* keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
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
  DevBuf& b_off = ctx->scratch[10];
  if (!is_device_ptr(stream_deg)) {
    s = b_x.ensure(sizeof(float) * (size_t)n_samples);
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(b_x.ptr, stream_deg, sizeof(float) * (size_t)n_samples, cudaMemcpyHostToDevice, st),
                      "H2D stream");
    if (!s.ok()) return ivt_fail(s);
    x = b_x.as<float>();
  }
  IvtDev P{x, (long long)n_samples, sample_rate_hz, opts->threshold_dps, opts->valid_min_deg, opts->valid_max_deg,
           opts->min_duration_ms, opts->min_amplitude_deg, opts->pre_samples, opts->post_samples};
  // run starts in stream order: count per tile, scan, write
  const long long ntiles_ll = (n_samples - 1 + kTile - 1) / kTile;
  if (ntiles_ll > 0x7fffffffLL) return ivt_fail(Status(OPMM_EINVAL, "opmm_detect_saccades: stream too long"));
  const int ntiles = (int)ntiles_ll;
  s = b_count.ensure(sizeof(int) * (size_t)ntiles);
  if (s.ok()) s = b_off.ensure(sizeof(long long) * ((size_t)ntiles + 1));
  if (!s.ok()) return ivt_fail(s);
  long long* d_off = b_off.as<long long>();
  k_ivt_count<<<ntiles, kIvtThreads, 0, st>>>(P, b_count.as<int>());
  k_ivt_scan<<<1, 1024, 0, st>>>(b_count.as<int>(), ntiles, d_off, d_off + ntiles);
  s = cuda_status(cudaGetLastError(), "launch I-VT count");
  long long total = 0;
  if (s.ok()) s = cuda_status(cudaMemcpyAsync(&total, d_off + ntiles, sizeof total, cudaMemcpyDeviceToHost, st), "D2H runs");
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "I-VT count");
  if (!s.ok()) return ivt_fail(s);
  if (total > (1LL << 26))
    return ivt_fail(Status(OPMM_ENOMEM, "opmm_detect_saccades: more than 2^26 velocity runs (raise the threshold)"));
  const int m = (int)total;
  // run records come back through pinned staging
  HostBuf& h_ev = ctx->h_scratch[0];
  HostBuf& h_keep = ctx->h_scratch[1];
  if (m > 0) {
    s = b_starts.ensure(sizeof(long long) * (size_t)m);
    if (s.ok()) s = b_ev.ensure(sizeof(opmm_ivt_event) * (size_t)m);
    if (s.ok()) s = b_keep.ensure(sizeof(int) * (size_t)m);
    if (s.ok()) s = h_ev.ensure(sizeof(opmm_ivt_event) * (size_t)m);
    if (s.ok()) s = h_keep.ensure(sizeof(int) * (size_t)m);
    if (!s.ok()) return ivt_fail(s);
    k_ivt_write<<<ntiles, kIvtThreads, 0, st>>>(P, d_off, b_starts.as<long long>());
    k_ivt_events<<<(m + 127) / 128, 128, 0, st>>>(P, b_starts.as<long long>(), m, b_ev.as<opmm_ivt_event>(),
                                                  b_keep.as<int>());
    s = cuda_status(cudaGetLastError(), "launch I-VT events");
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(h_ev.ptr, b_ev.ptr, sizeof(opmm_ivt_event) * (size_t)m, cudaMemcpyDeviceToHost, st),
                      "D2H events");
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(h_keep.ptr, b_keep.ptr, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, st),
                      "D2H keep");
    if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "I-VT events");
    if (!s.ok()) return ivt_fail(s);
  }
  // kept events, already in onset order
  size_t found = 0;
  const opmm_ivt_event* hev = h_ev.as<opmm_ivt_event>();
  const int* hkeep = h_keep.as<int>();
  for (int i = 0; i < m; ++i) {
    if (!hkeep[i]) continue;
    if (found < (size_t)max_events) out[found] = hev[i];
    ++found;
  }
  *n_events = (int32_t)std::min<size_t>(found, (size_t)0x7fffffff);
  return OPMM_OK;
}
