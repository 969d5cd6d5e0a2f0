// runtime.h -- host-side runtime types behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/opmm.h"
#include "common.cuh"
#include "launch.h"

namespace opmm {

constexpr int kMaxSamples = 16384;

struct Status {
  int code = OPMM_OK;
  std::string msg;
  Status() = default;
  Status(int c, std::string m);
  bool ok() const { return code == OPMM_OK; }
};

Status cuda_status(cudaError_t e, const char* what);
void set_last_error(const std::string& msg);   // per-thread text for opmm_last_error
bool is_device_ptr(const void* p);
int nsub_for(float fs);
Status check_saccade(const opmm_saccade& s, int i, bool need_duration);
Status check_opc(const float* opc);
Status check_opts(const opmm_fit_opts& o);   // the fit options every fit entry point accepts
DevSac make_devsac(const opmm_saccade& s);

// Grow-only device buffer.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  Status ensure(size_t want);
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Grow-only pinned host buffer.
struct HostBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf();
  Status ensure(size_t want);
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

struct SurrogateState;
struct ServeState;

struct TuneProbe {
  int variant;
  int bps;
  float ms;
};

}  // namespace opmm

struct opmm_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  int forced_variant = -1;            // -1: autotune; else a search kernel variant
  opmm::DevBuf d_err;                 // device error word of the kernels
  opmm::DevBuf scratch[16];           // per-call scratch of the synchronous entry points
  opmm::HostBuf h_scratch[2];         // pinned host scratch of the synchronous entry points
  std::map<std::tuple<int, int, int, int>, std::pair<int, int>> tune_cache;
  std::map<std::tuple<int, int, int, int>, std::vector<opmm::TuneProbe>> tune_logs;
  opmm::SurrogateState* surrogate = nullptr;   // owned, released by surrogate_release
  opmm::ServeState* serve = nullptr;           // owned, released by serve_shutdown
  opmm_ctx();
  ~opmm_ctx();
};

struct opmm_plan {
  opmm_ctx* ctx = nullptr;
  int n = 0;
  opmm_fit_opts opts{};
  int dim = 18;                       // search coordinates: 18, or 9 (OPMM_MODEL_9)
  int S = 0;                          // simplices per saccade
  int variant = 0;                    // search kernel variant (see kernels.cu)
  int G = 16;                         // simplices per block
  int threads = 0;
  int blocks_per_sm = 1;
  int ngroups = 0;                    // simplex groups per saccade
  int n_units = 0;
  int lcap = 0;
  int sac_index_base = 0;             // Philox counter word of saccade 0
  bool autotune = false;
  bool traces_on_device = false;
  bool centres_given = false;
  int pre_search_kernels = 0;
  std::vector<opmm::TuneProbe> tune_log;  // autotuner probes (variant, blocks/SM, ms)
  std::function<opmm::Status(opmm_plan*, cudaStream_t)> pre_search;   // e.g. surrogate centres
  std::vector<opmm::DevSac> hsacs;
  std::vector<const float*> src;
  size_t trace_floats = 0;
  opmm::SearchParams params{};
  opmm::DevBuf d_sacs, d_traces, d_pc, d_sac_index, d_units, d_ustart, d_unit_best, d_counter, d_results, d_src;
  opmm::DevBuf d_pc_given;            // caller's centres when the surrogate rescales them
  opmm::HostBuf h_traces, h_results, h_err;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_search[2] = {nullptr, nullptr};   // around the search kernel
  ~opmm_plan();
};

namespace opmm {

Status build_units(opmm_plan* p, int G, int probe_stride = 1);
Status plan_stage(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts& o, opmm_plan* p);
Status plan_build(opmm_ctx* ctx, const opmm_saccade* sacs, int32_t n, const opmm_fit_opts& o, bool capture,
                  bool tune, opmm_plan* p);
Status enqueue_centres(opmm_plan* p, cudaStream_t st);
Status plan_run(opmm_plan* p, opmm_fit_result* out);
Status enqueue_fit(opmm_plan* p, cudaStream_t st);
void pack_host_traces(opmm_plan* p);

// surrogate.cu
void surrogate_release(opmm_ctx* ctx);
Status surrogate_prepare_plan(opmm_ctx* ctx, opmm_plan* p, const opmm_saccade* sacs, int32_t n);

// serve.cu
void serve_shutdown(opmm_ctx* ctx);

}  // namespace opmm
