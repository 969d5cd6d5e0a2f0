// launch.h -- host-side entry points of the CUDA kernels (internal to the
// library; the public interface is include/opmm.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/opmm.h"

namespace opmm {

struct DevSac;

// Arguments of the persistent search kernel.
struct SearchParams {
  const DevSac* sacs;      // [B] staged saccades
  const float* traces;     // packed traces
  const float* pc;         // [B][18] box centres
  const int* sac_index;    // [B] Philox counter word of each saccade
  const int2* units;       // [n_units] (saccade, simplex group), most work first
  int n_units;
  int S;                   // simplices per saccade
  int T;                   // iteration cap
  int lcap;                // trace capacity of the shared-memory stage (floats, multiple of 4)
  float lnlo, lnhi;        // ln of the box bounds
  float step;              // initial simplex edge
  float tolx, tolf;
  uint32_t seed_lo, seed_hi;
  int* counter;            // work-queue head, zeroed before each launch
  float* unit_best;        // [n_units][24] results per unit
  unsigned* err;           // error bits
  // resumable mode (serving); state == nullptr for a one-launch fit
  const int* slot_list;    // if set, unit u is (slot_list[u / ngroups], u % ngroups)
  int ngroups;             // units per saccade
  int balanced;            // 1: unit g holds simplices [g S / ngroups, (g + 1) S / ngroups) (request
                           // loop: short searches); 0: units of 2 G simplices, the last takes the rest
  float* state;            // [slots][S][kStateFloats] saved simplices
  const int* progress;     // [slots] iterations already run
  int round_iters;         // iterations per launch
};

constexpr int kSearchStateFloats = 19 * 18 + 19 + 18 + 19 + 2;   // per saved simplex

cudaError_t launch_gather(const float* const* src, const DevSac* sacs, float* dst, int n, cudaStream_t st);
cudaError_t launch_nominal(const DevSac* sacs, int n, int pulse_mode, const float* init_opc, float* pc,
                           cudaStream_t st);
cudaError_t launch_simulate(const float* opc, int n, const DevSac* sacs, const int* sac_of,
                            const long long* out_off, float* out, cudaStream_t st);
cudaError_t launch_score(const float* opc, int m, const DevSac* sac, int L, const float* traces, float* f,
                         unsigned* err, int num_sms, cudaStream_t st);
// Search kernel variants (see kernels.cu): unit size (simplices per block),
// search coordinates (18, or 9 for the 9-parameter model), threads and
// dynamic shared memory per block.
int search_variant_count();
int search_variant_g(int v);
int search_variant_dim(int v);
int search_variant_minb(int v);
int search_variant_lean(int v);
int search_variant_pack(int v);
int search_variant_for(int unit, int dim);
int search_variant_threads(int v);
size_t search_variant_smem(int v, int lcap);
cudaError_t search_occupancy_v(int v, int lcap, int* blocks_per_sm);
cudaError_t launch_search_v(int v, const SearchParams& P, int blocks_per_sm, int num_sms, cudaStream_t st);
cudaError_t search_occupancy(int unit, int lcap, int* blocks_per_sm);
cudaError_t launch_search(int unit, const SearchParams& P, int blocks_per_sm, int num_sms, cudaStream_t st);
cudaError_t launch_finalize(const DevSac* sacs, const float* traces, const float* pc, const int* ustart,
                            int ngroups, const float* unit_best, float lnlo, float lnhi, int n,
                            opmm_fit_result* out, cudaStream_t st, const int* list = nullptr, int dim = 18);

// Levenberg-Marquardt refinement of n saccades (dim 18 or 9); scratch holds
// n * (2 dim + 2) * lcap floats.
cudaError_t launch_refine(int dim, const DevSac* sacs, const float* traces, const float* pcs, const float* start,
                          int n, int K, float lnlo, float lnhi, float delta, float lambda0, int lcap, float* scratch,
                          opmm_fit_result* out, unsigned* err, cudaStream_t st);

cudaError_t launch_admit(const DevSac* new_sacs, const float* new_traces, const float* new_pc, const int* slots, int n,
                         DevSac* sacs, float* traces, float* pc, int* progress, int slot_stride, cudaStream_t st);
cudaError_t launch_advance(const int* slots, int n, int* progress, int iters, int T, cudaStream_t st);

// Words per (saccade, simplex-unit) result record of the search kernel.
constexpr int kUnitRecFloats = 24;

}  // namespace opmm
