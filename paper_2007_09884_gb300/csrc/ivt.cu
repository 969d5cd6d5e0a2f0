// ivt.cu -- front end: velocity-threshold (I-VT) saccade detection and
// cleaning of raw position streams on the device, producing the windows and
// descriptors the estimator takes (the paper segments its recordings with
// I-VT and drops saccades shorter than 6 ms or smaller than 4 deg, Sec. 4;
// the threshold and the cleaning rule are the caller's, see opmm.h).
//
// Step k (samples k - 1, k) is fast when both samples are valid (finite, in
// [valid_min, valid_max]) and |x_k - x_(k-1)| * fs > threshold, in FP32.  A
// saccade is a maximal run of fast steps [a, b): onset sample s = a - 1, end
// sample e = b - 1.  Run starts are compacted in stream order over tiles of
// kTile steps, four steps per thread from one 16-byte load: one HBM pass
// counts each tile's starts and records up to kIvtRec of them (tile-local, in
// any order), a scan of the counts gives the tile offsets, one warp per
// sparse tile ranks its recorded starts into stream order, and only tiles
// with more starts than that (a threshold near the noise) are read a second
// time, writing in order by warp scans; then one warp per run walks the run
// and checks its window.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cfloat>
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
  float fs, thr;
  float vmin, vmax;   // valid range clamped to [-FLT_MAX, FLT_MAX] on the host
  float min_dur, min_amp;
  int pre, post;
};

// Finite and inside [valid_min, valid_max]: with the bounds clamped to the
// finite range, the two comparisons alone decide it (NaN and +-inf fail one).
__device__ __forceinline__ bool ivt_valid(float v, const IvtDev& P) { return v >= P.vmin && v <= P.vmax; }

// |x_k - x_(k-1)| * fs, or -1 when the step is not between two valid samples.
__device__ __forceinline__ float ivt_speed(const IvtDev& P, long long k) {
  if (k < 1 || k >= P.n) return -1.0f;
  const float a = P.x[k - 1], b = P.x[k];
  if (!ivt_valid(a, P) || !ivt_valid(b, P)) return -1.0f;
  return fabsf(b - a) * P.fs;
}

constexpr int kIvtThreads = 256;
constexpr int kIvtIters = 8;
constexpr int kVec = 4;                                                     // steps per thread and iteration
constexpr long long kTile = (long long)kIvtThreads * kIvtIters * kVec;     // steps per tile (one block)

// Run starts among steps 4m+1 .. 4m+4 (bit i for step 4m+1+i).  Group m's
// samples 4m .. 4m+3 come in one 16-byte load when the stream is aligned;
// sample 4m-1 (for step 4m) and sample 4m+4 from the neighbouring lanes.
// Every lane of the warp calls it, with consecutive m on consecutive lanes.
// FULL: every sample the group touches, 4m-1 .. 4m+4, lies in the stream
// (sample -1 of the first group aside), so no load needs a bounds check.
template <bool VEC, bool FULL>
__device__ __forceinline__ unsigned ivt_group_starts(const IvtDev& P, long long m) {
  const float nan = __int_as_float(0x7fc00000);
  const long long b = 4 * m;
  const float* xb = P.x + b;
  float x0, x1, x2, x3;
  if (VEC && (FULL || b + 3 < P.n)) {
    const float4 v = *reinterpret_cast<const float4*>(xb);
    x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
  } else if (FULL) {
    x0 = xb[0]; x1 = xb[1]; x2 = xb[2]; x3 = xb[3];
  } else {
    x0 = b < P.n ? xb[0] : nan;
    x1 = b + 1 < P.n ? xb[1] : nan;
    x2 = b + 2 < P.n ? xb[2] : nan;
    x3 = b + 3 < P.n ? xb[3] : nan;
  }
  const int lane = threadIdx.x & 31;
  float xm = __shfl_up_sync(0xffffffffu, x3, 1);
  float x4 = __shfl_down_sync(0xffffffffu, x0, 1);
  if (lane == 0) xm = (b >= 1 && (FULL || b - 1 < P.n)) ? xb[-1] : nan;
  if (lane == 31) x4 = (FULL || b + 4 < P.n) ? xb[4] : nan;
  // per sample validity once, then fast steps 4m .. 4m+4 (step 0 does not
  // exist: sample -1 reads as NaN, which is not valid)
  const bool vm = ivt_valid(xm, P), v0 = ivt_valid(x0, P), v1 = ivt_valid(x1, P), v2 = ivt_valid(x2, P);
  const bool v3 = ivt_valid(x3, P), v4 = ivt_valid(x4, P);
  const bool f0 = vm && v0 && fabsf(x0 - xm) * P.fs > P.thr;
  const bool f1 = v0 && v1 && fabsf(x1 - x0) * P.fs > P.thr;
  const bool f2 = v1 && v2 && fabsf(x2 - x1) * P.fs > P.thr;
  const bool f3 = v2 && v3 && fabsf(x3 - x2) * P.fs > P.thr;
  const bool f4 = v3 && v4 && fabsf(x4 - x3) * P.fs > P.thr;
  return (f1 && !f0 ? 1u : 0u) | (f2 && !f1 ? 2u : 0u) | (f3 && !f2 ? 4u : 0u) | (f4 && !f3 ? 8u : 0u);
}

// A tile whose every group touches only samples inside the stream: its last
// group reads sample 4m+4 = (t + 1) kTile.
__device__ __forceinline__ bool ivt_tile_full(const IvtDev& P) { return ((long long)blockIdx.x + 1) * kTile < P.n; }

__device__ __forceinline__ long long ivt_group(int it) {
  return (long long)blockIdx.x * (kIvtThreads * kIvtIters) + (long long)it * kIvtThreads + threadIdx.x;
}

constexpr int kIvtRec = 64;   // run starts a tile records during the count pass

// Pass 1a: run starts per tile; the first kIvtRec found are recorded as
// tile-local step indices (step - first step of the tile, < kTile), in the
// order the warps happen to claim slots.  The loop over the stream only
// loads and tests (each thread's eight 4-bit start masks packed in one
// word); the records collect in shared memory afterwards and go out at the
// end.
template <bool VEC>
__global__ void __launch_bounds__(kIvtThreads) k_ivt_count(IvtDev P, int* tile_count, unsigned short* rec) {
  static_assert(kIvtIters * kVec <= 32, "start masks packed in one word");
  __shared__ int n_found;
  __shared__ unsigned short found[kIvtRec];
  if (threadIdx.x == 0) n_found = 0;
  unsigned packed = 0;
  if (ivt_tile_full(P)) {   // block-uniform
#pragma unroll 4
    for (int it = 0; it < kIvtIters; ++it) packed |= ivt_group_starts<VEC, true>(P, ivt_group(it)) << (kVec * it);
  } else {
#pragma unroll 4
    for (int it = 0; it < kIvtIters; ++it) packed |= ivt_group_starts<VEC, false>(P, ivt_group(it)) << (kVec * it);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (__syncthreads_or(packed != 0u)) {             // block-uniform: most tiles of a fixation start nothing
    for (int it = 0; it < kIvtIters; ++it) {
      const unsigned bits = packed >> (kVec * it) & 15u;
      if (!__ballot_sync(0xffffffffu, bits != 0u)) continue;   // warp-uniform
      const int c = __popc(bits);
      int inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      int base = 0;
      if (lane == 31) base = atomicAdd(&n_found, inc);
      int slot = __shfl_sync(0xffffffffu, base, 31) + inc - c;
      const int local = 4 * (it * kIvtThreads + (int)threadIdx.x);
      for (int i = 0; i < kVec; ++i)
        if (bits >> i & 1u) {
          if (slot < kIvtRec) found[slot] = (unsigned short)(local + i);
          ++slot;
        }
    }
    __syncthreads();
  }
  const int c = n_found;
  if ((int)threadIdx.x < min(c, kIvtRec)) rec[(size_t)blockIdx.x * kIvtRec + threadIdx.x] = found[threadIdx.x];
  if (threadIdx.x == 0) tile_count[blockIdx.x] = c;
}

// Exclusive scan of the tile counts (one block of 1024 threads, each taking
// a contiguous run of tiles); the total goes to *total.
__global__ void __launch_bounds__(1024) k_ivt_scan(const int* tile_count, int ntiles, long long* tile_off,
                                                   long long* total) {
  __shared__ long long warp_tot[32];
  const int per = (ntiles + 1023) / 1024;
  const int t0 = (int)threadIdx.x * per;
  long long mine = 0;
  for (int i = t0; i < t0 + per && i < ntiles; ++i) mine += tile_count[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    long long v = warp_tot[lane], wi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_tot[lane] = wi - v;   // exclusive prefix of the warps
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  long long run = warp_tot[warp] + inc - mine;
  for (int i = t0; i < t0 + per && i < ntiles; ++i) {
    tile_off[i] = run;
    run += tile_count[i];
  }
}

// Pass 1b, sparse tiles (at most kIvtRec starts): one warp per tile ranks
// the recorded starts (distinct indices: the rank is the number smaller) and
// writes them at the tile's offset in stream order.
__global__ void k_ivt_place(const int* tile_count, const unsigned short* rec, const long long* tile_off, int ntiles,
                            long long* starts) {
  const int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;                       // warp-uniform
  const int c = tile_count[t];
  if (c == 0 || c > kIvtRec) return;             // warp-uniform
  const unsigned short* r = rec + (size_t)t * kIvtRec;
  const int v0 = lane < c ? (int)r[lane] : 0x10000;             // padding ranks after every index
  const int v1 = lane + 32 < c ? (int)r[lane + 32] : 0x10000;
  int r0 = 0, r1 = 0;
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    const int a = __shfl_sync(0xffffffffu, v0, j), b = __shfl_sync(0xffffffffu, v1, j);
    r0 += (a < v0) + (b < v0);
    r1 += (a < v1) + (b < v1);
  }
  const long long first = (long long)t * kTile + 1;   // step of local index 0
  const long long off = tile_off[t];
  if (lane < c) starts[off + r0] = first + v0;
  if (lane + 32 < c) starts[off + r1] = first + v1;
}

// Pass 1b, dense tiles (more than kIvtRec starts): read the tile again and
// write its run starts at its offset in stream order (iteration, warp, lane,
// step).  Every other block returns at once.
template <bool VEC>
__global__ void __launch_bounds__(kIvtThreads) k_ivt_write(IvtDev P, const int* tile_count, const long long* tile_off,
                                                           long long* starts) {
  if (tile_count[blockIdx.x] <= kIvtRec) return;   // block-uniform
  __shared__ int warp_cnt[kIvtThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long run = tile_off[blockIdx.x];
  for (int it = 0; it < kIvtIters; ++it) {
    const long long m = ivt_group(it);
    const unsigned bits = ivt_group_starts<VEC, false>(P, m);
    const int c = __popc(bits);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_cnt[warp] = inc;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < kIvtThreads / 32; ++w) {
      before += w < warp ? warp_cnt[w] : 0;
      all += warp_cnt[w];
    }
    long long pos = run + before + inc - c;
    for (int i = 0; i < kVec; ++i)
      if (bits >> i & 1u) starts[pos++] = 4 * m + 1 + i;
    run += all;
    __syncthreads();
  }
}

// Pass 2: one warp per run: the run's end (the first slow step, found 32
// steps at a time), peak velocity, the window check, the event record;
// keep[i] = 1 for a kept saccade.
__global__ void k_ivt_events(IvtDev P, const long long* starts, int m, opmm_ivt_event* ev, int* keep) {
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const long long a = starts[i];
  long long b = a;
  float peak = 0.0f;
  for (long long k0 = a;; k0 += 64) {                  // 64 steps per pass: both loads in flight together
    const float sp0 = ivt_speed(P, k0 + lane), sp1 = ivt_speed(P, k0 + 32 + lane);
    const unsigned slow0 = __ballot_sync(0xffffffffu, !(sp0 > P.thr));
    const unsigned slow1 = __ballot_sync(0xffffffffu, !(sp1 > P.thr));
    const int stop = slow0 ? __ffs(slow0) - 1 : (slow1 ? 32 + __ffs(slow1) - 1 : 64);   // steps before it are the run's
    if (lane < stop) peak = fmaxf(peak, sp0);
    if (32 + lane < stop) peak = fmaxf(peak, sp1);
    if (stop < 64) {
      b = k0 + stop;
      break;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) peak = fmaxf(peak, __shfl_xor_sync(0xffffffffu, peak, o));
  const long long s = a - 1, e = b - 1;
  const float xs = P.x[s], xe = P.x[e];
  const float amp = fabsf(xe - xs);
  const float dur = ((float)(e - s) * 1000.0f) / P.fs;
  const long long ws = s - P.pre, we = e + P.post;
  bool ok = dur >= P.min_dur && amp >= P.min_amp && ws >= 0 && we <= P.n - 1;
  if (ok) {
    bool good = true;
#pragma unroll 4
    for (long long k = ws + lane; k <= we; k += 32) good &= ivt_valid(P.x[k], P);   // loads independent of one another
    ok = __all_sync(0xffffffffu, good);
  }
  if (lane == 0) {
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
  DevBuf& b_rec = ctx->scratch[9];
  if (!is_device_ptr(stream_deg)) {
    s = b_x.ensure(sizeof(float) * (size_t)n_samples);
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(b_x.ptr, stream_deg, sizeof(float) * (size_t)n_samples, cudaMemcpyHostToDevice, st),
                      "H2D stream");
    if (!s.ok()) return ivt_fail(s);
    x = b_x.as<float>();
  }
  IvtDev P{x, (long long)n_samples, sample_rate_hz, opts->threshold_dps, std::max(opts->valid_min_deg, -FLT_MAX),
           std::min(opts->valid_max_deg, FLT_MAX),
           opts->min_duration_ms, opts->min_amplitude_deg, opts->pre_samples, opts->post_samples};
  // run starts in stream order: count per tile, scan, write
  const long long ntiles_ll = (n_samples - 1 + kTile - 1) / kTile;
  if (ntiles_ll > 0x7fffffffLL) return ivt_fail(Status(OPMM_EINVAL, "opmm_detect_saccades: stream too long"));
  const int ntiles = (int)ntiles_ll;
  s = b_count.ensure(sizeof(int) * (size_t)ntiles);
  if (s.ok()) s = b_off.ensure(sizeof(long long) * ((size_t)ntiles + 1));
  if (!s.ok()) return ivt_fail(s);
  long long* d_off = b_off.as<long long>();
  s = b_rec.ensure(sizeof(unsigned short) * kIvtRec * (size_t)ntiles);
  if (!s.ok()) return ivt_fail(s);
  unsigned short* d_rec = b_rec.as<unsigned short>();
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;   // 16-byte loads need an aligned stream
  if (vec) k_ivt_count<true><<<ntiles, kIvtThreads, 0, st>>>(P, b_count.as<int>(), d_rec);
  else k_ivt_count<false><<<ntiles, kIvtThreads, 0, st>>>(P, b_count.as<int>(), d_rec);
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
    const long long warps_per_block = 4;
    k_ivt_place<<<(unsigned)((ntiles + warps_per_block - 1) / warps_per_block), 32 * warps_per_block, 0, st>>>(
        b_count.as<int>(), d_rec, d_off, ntiles, b_starts.as<long long>());
    if (vec) k_ivt_write<true><<<ntiles, kIvtThreads, 0, st>>>(P, b_count.as<int>(), d_off, b_starts.as<long long>());
    else k_ivt_write<false><<<ntiles, kIvtThreads, 0, st>>>(P, b_count.as<int>(), d_off, b_starts.as<long long>());
    k_ivt_events<<<(unsigned)((m + warps_per_block - 1) / warps_per_block), 32 * warps_per_block, 0, st>>>(
        P, b_starts.as<long long>(), m, b_ev.as<opmm_ivt_event>(), b_keep.as<int>());
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
