// static_fit.cu -- single-saccade fit that allocates no memory.
//
// Some callers cannot call cudaMalloc: a real-time eye-tracking loop that must
// not stall on an allocation (cudaMalloc and cudaFree may synchronise the whole
// device), or a host program whose device memory is entirely owned by another
// allocator or fixed budget.  opmm_fit_saccade_static serves them: the caller
// passes the trace and the result slot in device memory, and every buffer the
// fit needs beyond them (staged trace, descriptor, box centre, work list,
// per-group results, work counter, error word) lives in the file-scope array
// g_opmm_static_scratch below.  That array has a fixed size (see
// kStaticScratchBytes) and, like any __device__ variable, is held by every GPU
// that loads the library until the process exits.
//
// Set-up: every call, with the device current, looks up the array's device
// address with cudaGetSymbolAddress (cheap, and never stale after a device
// reset) and makes sure the search kernel may use the shared memory this trace
// needs.  The first call on a device also loads the library's kernels there;
// make it before any stream capture.
//
// All calls share the one array, so calls whose work overlaps on the GPU
// (different streams or threads at the same time) race; the call is
// synchronous, so back-to-back calls from one thread are safe.  The array keeps
// the last call's contents; everything that must start at zero (work counter,
// error word) is cleared by each call.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/opmm.h"
#include "common.cuh"
#include "launch.h"
#include "runtime.h"

namespace opmm {

namespace {

constexpr int kStaticMaxSamples = 4096;        // longest trace accepted
constexpr int kStaticMaxCandidates = 65536;    // largest per-iteration budget accepted
constexpr int kStaticG = 32;                   // simplices per block (one unit)
constexpr int kStaticMaxUnits = (kStaticMaxCandidates / 22 + kStaticG - 1) / kStaticG;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kOffHeader = 0;                                        // int counter, unsigned err
constexpr size_t kOffSac = 256;                                         // DevSac
constexpr size_t kOffCentre = 512;                                      // float[18]
constexpr size_t kOffIndex = 768;                                       // int sac_index, int ustart
constexpr size_t kOffSrc = 1024;                                        // const float* src[1]
constexpr size_t kOffUnits = 1280;                                      // int2[kStaticMaxUnits]
constexpr size_t kOffBest = align256(kOffUnits + sizeof(int2) * kStaticMaxUnits);
constexpr size_t kOffTrace = align256(kOffBest + sizeof(float) * kUnitRecFloats * kStaticMaxUnits);
constexpr size_t kStaticScratchBytes = align256(kOffTrace + sizeof(float) * kStaticMaxSamples);
// 27,648 bytes: the size the header and the design notes state.
static_assert(kStaticScratchBytes == 27648, "update the documented scratch size");

static __device__ __align__(256) unsigned char g_opmm_static_scratch[kStaticScratchBytes];

struct Centre {
  float v[18];
};

// Fill the per-call part of the scratch array from kernel arguments (no host
// to device copy is needed) and clear what must start at zero.
__global__ void k_static_setup(unsigned char* base, DevSac d, Centre c, int has_centre, const float* src,
                               int ngroups) {
  const int t = threadIdx.x;
  if (t == 0) {
    *reinterpret_cast<int*>(base + kOffHeader) = 0;                    // work counter
    *reinterpret_cast<unsigned*>(base + kOffHeader + 4) = 0u;          // error word
    *reinterpret_cast<DevSac*>(base + kOffSac) = d;
    reinterpret_cast<int*>(base + kOffIndex)[0] = 0;                   // Philox counter word
    reinterpret_cast<int*>(base + kOffIndex)[1] = 0;                   // first unit of saccade 0
    *reinterpret_cast<const float**>(base + kOffSrc) = src;
  }
  if (has_centre && t < 18) reinterpret_cast<float*>(base + kOffCentre)[t] = c.v[t];
  for (int g = t; g < ngroups; g += blockDim.x) reinterpret_cast<int2*>(base + kOffUnits)[g] = make_int2(0, g);
}

// Per-call set-up on the current device: the scratch array's device address,
// the SM count and how many search blocks of this trace capacity fit on an SM.
struct DeviceSetup {
  unsigned char* scratch = nullptr;
  int num_sms = 0;
  int blocks_per_sm = 0;
};

Status device_setup(int dev, int lcap, DeviceSetup* s) {
  void* p = nullptr;
  Status r = cuda_status(cudaGetSymbolAddress(&p, g_opmm_static_scratch), "cudaGetSymbolAddress");
  if (!r.ok()) return r;
  r = cuda_status(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (!r.ok()) return r;
  r = cuda_status(search_occupancy(kStaticG, lcap, &s->blocks_per_sm), "search occupancy");
  if (!r.ok()) return r;
  if (s->blocks_per_sm < 1) return Status(OPMM_ECUDA, "search kernel does not fit on this device");
  s->scratch = static_cast<unsigned char*>(p);
  return Status();
}

}  // namespace

}  // namespace opmm

using namespace opmm;

extern "C" int opmm_fit_saccade_static(const opmm_saccade* sac, const opmm_fit_opts* opts,
                                       opmm_fit_result* out_device, void* cuda_stream) {
  if (!sac || !opts || !out_device || !sac->trace_deg) return OPMM_EINVAL;
  // the options every fit accepts, then this entry point's own limits
  if (!check_opts(*opts).ok()) return OPMM_EINVAL;
  if (opts->model != OPMM_MODEL_18 || opts->use_surrogate) return OPMM_EINVAL;
  if (opts->candidates > kStaticMaxCandidates) return OPMM_EINVAL;
  const bool need_duration = opts->init_opc == nullptr;
  if (!check_saccade(*sac, 0, need_duration).ok()) return OPMM_EINVAL;
  if (sac->n_samples > kStaticMaxSamples) return OPMM_EINVAL;
  if (opts->init_opc && !check_opc(opts->init_opc).ok()) return OPMM_EINVAL;
  if (!is_device_ptr(sac->trace_deg) || !is_device_ptr(out_device)) return OPMM_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return OPMM_ECUDA;
  }
  const int lcap = (sac->n_samples + 3) & ~3;
  DeviceSetup setup;
  Status s = device_setup(dev, lcap, &setup);
  if (!s.ok()) {
    cudaGetLastError();
    return s.code;
  }
  DeviceSetup* ds = &setup;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = ds->scratch;
  DevSac d = make_devsac(*sac);
  d.off = 0;
  const int S = opts->candidates / (OPMM_NPARAM + 4);
  const int ngroups = (S + kStaticG - 1) / kStaticG;
  Centre c{};
  if (opts->init_opc)
    for (int j = 0; j < 18; ++j) c.v[j] = opts->init_opc[j];

  k_static_setup<<<1, 256, 0, st>>>(base, d, c, opts->init_opc ? 1 : 0, sac->trace_deg, ngroups);
  cudaError_t e = cudaGetLastError();
  const DevSac* d_sac = reinterpret_cast<const DevSac*>(base + kOffSac);
  float* d_trace = reinterpret_cast<float*>(base + kOffTrace);
  float* d_pc = reinterpret_cast<float*>(base + kOffCentre);
  if (e == cudaSuccess)
    e = launch_gather(reinterpret_cast<const float* const*>(base + kOffSrc), d_sac, d_trace, 1, st);
  if (e == cudaSuccess && !opts->init_opc) e = launch_nominal(d_sac, 1, opts->pulse_init, nullptr, d_pc, st);
  SearchParams P{};
  P.sacs = d_sac;
  P.traces = d_trace;
  P.pc = d_pc;
  P.sac_index = reinterpret_cast<const int*>(base + kOffIndex);
  P.units = reinterpret_cast<const int2*>(base + kOffUnits);
  P.n_units = ngroups;
  P.ngroups = ngroups;
  P.S = S;
  P.T = opts->iterations;
  P.lcap = lcap;
  P.lnlo = (float)std::log((double)opts->box_lo);
  P.lnhi = (float)std::log((double)opts->box_hi);
  P.step = opts->init_step;
  P.tolx = opts->tol_x;
  P.tolf = opts->tol_f;
  P.seed_lo = (uint32_t)(opts->seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(opts->seed >> 32);
  P.counter = reinterpret_cast<int*>(base + kOffHeader);
  P.unit_best = reinterpret_cast<float*>(base + kOffBest);
  P.err = reinterpret_cast<unsigned*>(base + kOffHeader + 4);
  if (e == cudaSuccess) e = launch_search(kStaticG, P, ds->blocks_per_sm, ds->num_sms, st);
  if (e == cudaSuccess)
    e = launch_finalize(d_sac, d_trace, d_pc, reinterpret_cast<const int*>(base + kOffIndex) + 1, ngroups,
                        P.unit_best, P.lnlo, P.lnhi, 1, out_device, st);
  unsigned err_word = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err_word, P.err, sizeof err_word, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return OPMM_ECUDA;
  }
  if (err_word & kErrWaitTimeout) return OPMM_ETIMEDOUT;
  if (err_word) return OPMM_ECUDA;
  return OPMM_OK;
}
