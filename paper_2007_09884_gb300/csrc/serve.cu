// serve.cu -- continuous-batching request loop (opmm_serve_*).
//
// Requests (single saccades) are queued by opmm_serve_submit.  A scheduler
// thread, on its own stream, repeats rounds:
//   1. admit queued requests into free device slots (the slot count is set at
//      start from the free-HBM budget; requests beyond the queue bound are
//      refused with OPMM_EBUSY): one packed H2D copy of descriptors and traces,
//      box centres (calibrated nominal, optionally re-centred by the
//      surrogate), scatter into the slots;
//   2. advance every occupied slot by `round_iters` Nelder-Mead iterations
//      with one launch of the persistent search kernel in resumable mode: the
//      simplices of each slot live in HBM between rounds, so requests that
//      arrived at different times share every launch;
//   3. finalize the slots that reached the iteration cap (winner, FP64 check),
//      copy their results back, free the slots, wake pollers.
// A request's simplices evolve the same way whatever else shares the launch
// (seeded by the request alone, deterministic per simplex), so a result is
// the same alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/opmm.h"
#include "launch.h"
#include "runtime.h"

namespace opmm {

Status surrogate_centres(opmm_ctx* ctx, const DevSac* sacs, const float* traces, int n, float* pc, cudaStream_t st);

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket;
  opmm_saccade desc;
  std::vector<float> trace;
  double t_submit;
};

struct Done {
  opmm_fit_result r;
  double latency_us;
};

}  // namespace

struct ServeState {
  opmm_ctx* ctx = nullptr;
  opmm_fit_opts fit{};
  opmm_serve_opts cfg{};
  int S = 0, G = 16, ngroups = 0, variant = 0, bps = 1, slots = 0, lcap = 0;
  bool seeded = false;
  cudaStream_t st = nullptr;
  SearchParams P{};
  DevBuf sacs, traces, pc, sac_index, state, progress, unit_best, results, slot_list, counter, done_list;
  DevBuf new_sacs, new_traces, new_pc, new_slots, err;
  HostBuf h_new_sacs, h_new_traces, h_results, h_ints, h_err;
  std::vector<int> free_slots, progress_h;
  std::vector<float> centre;                 // caller's box centre (if given)
  std::vector<uint64_t> slot_ticket;
  std::vector<double> slot_t;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_map<uint64_t, int> known;   // ticket -> 1 while queued or running
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  std::atomic<bool> stop{false};
  uint64_t next_ticket = 1;
  opmm_serve_stats stats{};
  Status error;

  Status round();
  void loop();
};

Status ServeState::round() {
  // ---- 1. admissions
  // at most one request per free slot, and never more than the staging holds
  std::vector<Request> admit;
  std::vector<int> taken;
  {
    std::lock_guard<std::mutex> lock(mu);
    const size_t cap = std::min<size_t>((size_t)cfg.max_admit_per_round, free_slots.size());
    while (!pending.empty() && admit.size() < cap) {
      admit.push_back(std::move(pending.front()));
      pending.pop_front();
      taken.push_back(free_slots.back());
      free_slots.pop_back();
    }
  }
  Status s;
  if (!admit.empty()) {
    const int na = (int)admit.size();
    DevSac* hs = h_new_sacs.as<DevSac>();
    float* ht = h_new_traces.as<float>();
    int* hslots = h_ints.as<int>();
    long long off = 0;
    for (int i = 0; i < na; ++i) {
      DevSac d = make_devsac(admit[(size_t)i].desc);
      d.off = off;
      std::memcpy(ht + off, admit[(size_t)i].trace.data(), sizeof(float) * (size_t)d.L);
      off += (d.L + 3) & ~3;
      hs[i] = d;
      hslots[i] = taken[(size_t)i];
    }
    s = cuda_status(cudaMemcpyAsync(new_sacs.ptr, hs, sizeof(DevSac) * (size_t)na, cudaMemcpyHostToDevice, st), "H2D admit");
    if (s.ok()) s = cuda_status(cudaMemcpyAsync(new_traces.ptr, ht, sizeof(float) * (size_t)off, cudaMemcpyHostToDevice, st), "H2D traces");
    if (s.ok()) s = cuda_status(cudaMemcpyAsync(new_slots.ptr, hslots, sizeof(int) * (size_t)na, cudaMemcpyHostToDevice, st), "H2D slots");
    if (s.ok()) {
      if (fit.init_opc) {
        std::vector<float> c((size_t)na * OPMM_NPARAM);
        for (int i = 0; i < na; ++i) std::memcpy(&c[(size_t)i * OPMM_NPARAM], fit.init_opc, sizeof(float) * OPMM_NPARAM);
        s = cuda_status(cudaMemcpyAsync(new_pc.ptr, c.data(), c.size() * 4, cudaMemcpyHostToDevice, st), "H2D centres");
        if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "centres");
      } else {
        s = cuda_status(launch_nominal(new_sacs.as<DevSac>(), na, fit.pulse_init, nullptr, new_pc.as<float>(), st), "nominal");
      }
    }
    if (s.ok() && seeded) s = surrogate_centres(ctx, new_sacs.as<DevSac>(), new_traces.as<float>(), na, new_pc.as<float>(), st);
    if (s.ok())
      s = cuda_status(launch_admit(new_sacs.as<DevSac>(), new_traces.as<float>(), new_pc.as<float>(), new_slots.as<int>(), na,
                                   sacs.as<DevSac>(), traces.as<float>(), pc.as<float>(), progress.as<int>(), lcap, st),
                      "admit");
    if (!s.ok()) return s;
    for (int i = 0; i < na; ++i) {
      const int slot = taken[(size_t)i];
      slot_ticket[(size_t)slot] = admit[(size_t)i].ticket;
      slot_t[(size_t)slot] = admit[(size_t)i].t_submit;
      progress_h[(size_t)slot] = 0;
    }
    stats.admitted += (uint64_t)na;
  }
  // ---- 2. one round of the search over all occupied slots
  std::vector<int> active;
  for (int sl = 0; sl < slots; ++sl)
    if (slot_ticket[(size_t)sl]) active.push_back(sl);
  if (active.empty()) return Status();
  const int nact = (int)active.size();
  int* hl = h_ints.as<int>() + slots;
  std::copy(active.begin(), active.end(), hl);
  s = cuda_status(cudaMemcpyAsync(slot_list.ptr, hl, sizeof(int) * (size_t)nact, cudaMemcpyHostToDevice, st), "H2D list");
  if (s.ok()) s = cuda_status(cudaMemsetAsync(counter.ptr, 0, sizeof(int), st), "clear counter");
  SearchParams p = P;
  p.slot_list = slot_list.as<int>();
  p.n_units = nact * ngroups;
  if (s.ok()) s = cuda_status(launch_search_v(variant, p, bps, ctx->num_sms, st), "search round");
  if (s.ok()) s = cuda_status(launch_advance(slot_list.as<int>(), nact, progress.as<int>(), cfg.round_iters, fit.iterations, st), "advance");
  // ---- 3. completions
  std::vector<int> comp;
  for (int sl : active) {
    progress_h[(size_t)sl] = std::min(fit.iterations, progress_h[(size_t)sl] + cfg.round_iters);
    if (progress_h[(size_t)sl] >= fit.iterations) comp.push_back(sl);
  }
  int* hd = h_ints.as<int>() + 2 * slots;
  std::copy(comp.begin(), comp.end(), hd);
  const int ncomp = (int)comp.size();
  if (s.ok() && ncomp) {
    s = cuda_status(cudaMemcpyAsync(done_list.ptr, hd, sizeof(int) * (size_t)ncomp, cudaMemcpyHostToDevice, st), "H2D done");
    // unit records are slot-major: slot b's groups start at b * ngroups
    if (s.ok())
      s = cuda_status(launch_finalize(sacs.as<DevSac>(), traces.as<float>(), pc.as<float>(), nullptr, ngroups,
                                      unit_best.as<float>(), P.lnlo, P.lnhi, ncomp, results.as<opmm_fit_result>(), st,
                                      done_list.as<int>()),
                      "finalize");
    if (s.ok())
      s = cuda_status(cudaMemcpyAsync(h_results.ptr, results.ptr, sizeof(opmm_fit_result) * (size_t)ncomp,
                                      cudaMemcpyDeviceToHost, st), "D2H results");
  }
  if (s.ok()) s = cuda_status(cudaMemcpyAsync(h_err.ptr, err.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "D2H err");
  if (s.ok()) s = cuda_status(cudaStreamSynchronize(st), "round");
  if (!s.ok()) return s;
  if (*h_err.as<unsigned>()) return Status(OPMM_ETIMEDOUT, "a search kernel's bounded wait expired");
  stats.rounds += 1;
  if (ncomp) {
    const double t = now_us();
    std::lock_guard<std::mutex> lock(mu);
    const opmm_fit_result* r = h_results.as<opmm_fit_result>();
    for (int i = 0; i < ncomp; ++i) {
      const int sl = comp[(size_t)i];
      const uint64_t tk = slot_ticket[(size_t)sl];
      done[tk] = Done{r[i], t - slot_t[(size_t)sl]};
      if (seeded) done[tk].r.source = OPMM_SOURCE_SEEDED;
      slot_ticket[(size_t)sl] = 0;
      free_slots.push_back(sl);
    }
    stats.completed += (uint64_t)ncomp;
  }
  if (ncomp) cv_done.notify_all();
  return Status();
}

void ServeState::loop() {
  cudaSetDevice(ctx->device);
  while (!stop.load()) {
    bool idle;
    {
      std::lock_guard<std::mutex> lock(mu);
      idle = pending.empty() && (int)free_slots.size() == slots;
    }
    if (idle) {
      std::unique_lock<std::mutex> lock(mu);
      cv_work.wait_for(lock, std::chrono::milliseconds(2), [&] { return stop.load() || !pending.empty(); });
      continue;
    }
    Status s = round();
    if (!s.ok()) {
      std::lock_guard<std::mutex> lock(mu);
      error = s;
      stop.store(true);
      cv_done.notify_all();
      break;
    }
  }
}

void serve_shutdown(opmm_ctx* ctx) {
  ServeState* sv = ctx->serve;
  if (!sv) return;
  sv->stop.store(true);
  sv->cv_work.notify_all();
  if (sv->th.joinable()) sv->th.join();
  if (sv->st) {
    cudaStreamSynchronize(sv->st);
    cudaStreamDestroy(sv->st);
  }
  delete sv;
  ctx->serve = nullptr;
}

}  // namespace opmm

using namespace opmm;

static int vfail(opmm_ctx* ctx, const Status& s) {
  (void)ctx;
  set_last_error(s.msg);
  return s.code;
}

#define VTRY(expr)                         \
  do {                                     \
    Status _s = (expr);                    \
    if (!_s.ok()) return vfail(ctx, _s);   \
  } while (0)

extern "C" int opmm_serve_start(opmm_ctx* ctx, const opmm_serve_opts* cfg, const opmm_fit_opts* fit) {
  if (!ctx) return OPMM_EINVAL;
  if (!cfg || !fit) return vfail(ctx, Status(OPMM_EINVAL, "serve: null options"));
  if (ctx->serve) return vfail(ctx, Status(OPMM_EINVAL, "serve: already running"));
  if (cfg->round_iters < 1 || cfg->max_queue < 1 || cfg->max_samples < 1 || cfg->max_samples > kMaxSamples ||
      cfg->max_admit_per_round < 1)
    return vfail(ctx, Status(OPMM_EINVAL, "serve: round_iters, max_queue, max_admit_per_round >= 1; max_samples in [1, 16384]"));
  if (fit->model != OPMM_MODEL_18 || fit->candidates < 22 || fit->iterations < 1 || !(fit->box_lo > 0.0f) ||
      !(fit->box_lo <= 1.0f) || !(fit->box_hi >= 1.0f) || !(fit->init_step > 0.0f))
    return vfail(ctx, Status(OPMM_EINVAL, "serve: bad fit options (iterations >= 1)"));
  if (fit->use_surrogate && (!ctx->surrogate))
    return vfail(ctx, Status(OPMM_EINVAL, "serve: use_surrogate needs an initialised or loaded surrogate"));
  if (fit->init_opc) VTRY(check_opc(fit->init_opc));
  VTRY(cuda_status(cudaSetDevice(ctx->device), "cudaSetDevice"));
  auto* sv = new ServeState();
  sv->ctx = ctx;
  sv->fit = *fit;
  sv->cfg = *cfg;
  sv->seeded = fit->use_surrogate != 0;
  sv->S = fit->candidates / (OPMM_NPARAM + 4);
  sv->variant = ctx->forced_variant >= 0 ? ctx->forced_variant : search_variant_for(32, OPMM_NPARAM);
  sv->G = search_variant_g(sv->variant);
  sv->ngroups = (sv->S + sv->G - 1) / sv->G;
  sv->lcap = (cfg->max_samples + 3) & ~3;
  Status s = cuda_status(search_occupancy_v(sv->variant, sv->lcap, &sv->bps), "occupancy");
  if (s.ok() && sv->bps < 1) s = Status(OPMM_ECUDA, "search kernel does not fit");
  // admission budget: bytes per slot against the device budget
  const size_t slot_bytes = (size_t)sv->S * kSearchStateFloats * 4 + (size_t)sv->ngroups * kUnitRecFloats * 4 +
                            (size_t)sv->lcap * 4 + OPMM_NPARAM * 4 + sizeof(DevSac) + sizeof(opmm_fit_result) + 16;
  size_t free_b = 0, total_b = 0;
  if (s.ok()) s = cuda_status(cudaMemGetInfo(&free_b, &total_b), "memory info");
  size_t budget = cfg->max_device_bytes ? (size_t)cfg->max_device_bytes : free_b / 2;
  if (budget > free_b) budget = free_b;
  const long long fit_slots = (long long)(budget / slot_bytes);
  sv->slots = (int)std::min<long long>(cfg->max_slots, fit_slots);
  if (s.ok() && sv->slots < 1) s = Status(OPMM_EBUSY, "serve: the device memory budget does not hold one request");
  const int n = sv->slots;
  if (s.ok()) s = cuda_status(cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking), "stream");
  if (s.ok()) s = sv->sacs.ensure(sizeof(DevSac) * (size_t)n);
  if (s.ok()) s = sv->traces.ensure(sizeof(float) * (size_t)n * sv->lcap);
  if (s.ok()) s = sv->pc.ensure(sizeof(float) * OPMM_NPARAM * (size_t)n);
  if (s.ok()) s = sv->sac_index.ensure(sizeof(int) * (size_t)n);
  if (s.ok()) s = sv->state.ensure(sizeof(float) * (size_t)n * sv->S * kSearchStateFloats);
  if (s.ok()) s = sv->progress.ensure(sizeof(int) * (size_t)n);
  if (s.ok()) s = sv->unit_best.ensure(sizeof(float) * (size_t)n * sv->ngroups * kUnitRecFloats);
  if (s.ok()) s = sv->results.ensure(sizeof(opmm_fit_result) * (size_t)n);
  if (s.ok()) s = sv->slot_list.ensure(sizeof(int) * (size_t)n);
  if (s.ok()) s = sv->done_list.ensure(sizeof(int) * (size_t)n);
  if (s.ok()) s = sv->counter.ensure(sizeof(int));
  if (s.ok()) s = sv->err.ensure(sizeof(unsigned));
  const int adm = std::min(cfg->max_admit_per_round, n);
  if (s.ok()) s = sv->new_sacs.ensure(sizeof(DevSac) * (size_t)adm);
  if (s.ok()) s = sv->new_traces.ensure(sizeof(float) * (size_t)adm * sv->lcap);
  if (s.ok()) s = sv->new_pc.ensure(sizeof(float) * OPMM_NPARAM * (size_t)adm);
  if (s.ok()) s = sv->new_slots.ensure(sizeof(int) * (size_t)adm);
  if (s.ok()) s = sv->h_new_sacs.ensure(sizeof(DevSac) * (size_t)adm);
  if (s.ok()) s = sv->h_new_traces.ensure(sizeof(float) * (size_t)adm * sv->lcap);
  if (s.ok()) s = sv->h_results.ensure(sizeof(opmm_fit_result) * (size_t)n);
  if (s.ok()) s = sv->h_ints.ensure(sizeof(int) * (size_t)n * 3);
  if (s.ok()) s = sv->h_err.ensure(sizeof(unsigned));
  if (s.ok()) s = cuda_status(cudaMemset(sv->sac_index.ptr, 0, sizeof(int) * (size_t)n), "clear index");
  if (s.ok()) s = cuda_status(cudaMemset(sv->err.ptr, 0, sizeof(unsigned)), "clear err");
  if (!s.ok()) {
    if (sv->st) cudaStreamDestroy(sv->st);
    delete sv;
    return vfail(ctx, s);
  }
  SearchParams& P = sv->P;
  P.sacs = sv->sacs.as<DevSac>();
  P.traces = sv->traces.as<float>();
  P.pc = sv->pc.as<float>();
  P.sac_index = sv->sac_index.as<int>();
  P.S = sv->S;
  P.T = fit->iterations;
  P.lcap = sv->lcap;
  P.lnlo = (float)std::log((double)fit->box_lo);
  P.lnhi = (float)std::log((double)fit->box_hi);
  P.step = fit->init_step;
  P.tolx = fit->tol_x;
  P.tolf = fit->tol_f;
  P.seed_lo = (uint32_t)(fit->seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(fit->seed >> 32);
  P.counter = sv->counter.as<int>();
  P.unit_best = sv->unit_best.as<float>();
  P.err = sv->err.as<unsigned>();
  P.ngroups = sv->ngroups;
  P.balanced = 1;
  P.state = sv->state.as<float>();
  P.progress = sv->progress.as<int>();
  P.round_iters = cfg->round_iters;
  sv->free_slots.resize((size_t)n);
  for (int i = 0; i < n; ++i) sv->free_slots[(size_t)i] = n - 1 - i;
  sv->progress_h.assign((size_t)n, 0);
  sv->slot_ticket.assign((size_t)n, 0);
  sv->slot_t.assign((size_t)n, 0.0);
  sv->stats.slots = n;
  if (fit->init_opc) {
    // keep the caller's centre for the lifetime of the server
    sv->centre.assign(fit->init_opc, fit->init_opc + OPMM_NPARAM);
    sv->fit.init_opc = sv->centre.data();
  }
  ctx->serve = sv;
  sv->th = std::thread([sv] { sv->loop(); });
  return OPMM_OK;
}

extern "C" int opmm_serve_submit(opmm_ctx* ctx, const opmm_saccade* sac, uint64_t* ticket) {
  if (!ctx) return OPMM_EINVAL;
  if (!sac || !ticket || !sac->trace_deg) return vfail(ctx, Status(OPMM_EINVAL, "submit: null argument"));
  ServeState* sv = ctx->serve;
  if (!sv) return vfail(ctx, Status(OPMM_EINVAL, "submit: server not running"));
  VTRY(check_saccade(*sac, 0, sv->fit.init_opc == nullptr));
  if (sac->n_samples > sv->lcap) return vfail(ctx, Status(OPMM_EINVAL, "submit: trace longer than the server's max_samples"));
  Request r;
  r.desc = *sac;
  r.trace.resize((size_t)sac->n_samples);
  if (is_device_ptr(sac->trace_deg)) {
    VTRY(cuda_status(cudaMemcpy(r.trace.data(), sac->trace_deg, sizeof(float) * r.trace.size(), cudaMemcpyDeviceToHost),
                     "copy trace"));
  } else {
    std::memcpy(r.trace.data(), sac->trace_deg, sizeof(float) * r.trace.size());
  }
  r.desc.trace_deg = nullptr;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (!sv->error.ok()) return vfail(ctx, sv->error);
    if ((int)sv->pending.size() >= sv->cfg.max_queue) {
      sv->stats.rejected += 1;
      return vfail(ctx, Status(OPMM_EBUSY, "submit: queue full"));
    }
    r.ticket = sv->next_ticket++;
    r.t_submit = now_us();
    *ticket = r.ticket;
    sv->known[r.ticket] = 1;
    sv->pending.push_back(std::move(r));
    sv->stats.submitted += 1;
  }
  sv->cv_work.notify_one();
  return OPMM_OK;
}

extern "C" int opmm_serve_poll(opmm_ctx* ctx, uint64_t ticket, opmm_fit_result* out, int32_t timeout_us,
                               double* latency_us) {
  if (!ctx) return OPMM_EINVAL;
  ServeState* sv = ctx->serve;
  if (!sv || !out) return vfail(ctx, Status(OPMM_EINVAL, "poll: server not running or null output"));
  std::unique_lock<std::mutex> lock(sv->mu);
  if (!sv->known.count(ticket)) return vfail(ctx, Status(OPMM_EINVAL, "poll: unknown or already collected ticket"));
  auto ready = [&] { return sv->done.count(ticket) > 0 || !sv->error.ok(); };
  if (!ready() && timeout_us > 0) sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready);
  auto it = sv->done.find(ticket);
  if (it == sv->done.end()) {
    if (!sv->error.ok()) return vfail(ctx, sv->error);
    return timeout_us > 0 ? vfail(ctx, Status(OPMM_ETIMEDOUT, "poll: deadline passed")) : OPMM_NOT_READY;
  }
  *out = it->second.r;
  if (latency_us) *latency_us = it->second.latency_us;
  sv->done.erase(it);
  sv->known.erase(ticket);
  return OPMM_OK;
}

extern "C" int opmm_serve_stats_get(opmm_ctx* ctx, opmm_serve_stats* out) {
  if (!ctx || !out) return OPMM_EINVAL;
  ServeState* sv = ctx->serve;
  if (!sv) return vfail(ctx, Status(OPMM_EINVAL, "stats: server not running"));
  std::lock_guard<std::mutex> lock(sv->mu);
  *out = sv->stats;
  out->queued = (int32_t)sv->pending.size();
  out->active = sv->slots - (int32_t)sv->free_slots.size();
  return OPMM_OK;
}

extern "C" int opmm_serve_stop(opmm_ctx* ctx) {
  if (!ctx) return OPMM_EINVAL;
  serve_shutdown(ctx);
  return OPMM_OK;
}
