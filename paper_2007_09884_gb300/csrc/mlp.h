// mlp.h -- internal interface of the surrogate's kernels (mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace opmm {
namespace mlp {

constexpr int kFeatPoints = 256;          // resampled points (1 ms apart from onset)
constexpr int kIn = 2 * kFeatPoints;      // position + velocity features
constexpr int kHidden = 512;              // width of the four hidden layers
constexpr int kLayers = 4;                // hidden layers (tensor-core GEMMs)
constexpr int kOut = 18;                  // OPC vector in log units
constexpr float kTargetScale = 0.2f;      // output y = ln(p / centre) / 0.2

// GEMM tiling: 128 x 128 output tile, 64-wide K slices in a ring of
// shared-memory stages: 3 stages (97 KB, two CTAs per SM, so one CTA's
// epilogue overlaps the other's main loop: large GEMMs) or 6 stages (193 KB,
// one CTA per SM, a deeper prefetch: the network's one-wave GEMMs).  The
// epilogue stages its output tile in the ring (free once every MMA has read
// it) and writes it out in whole rows.
constexpr int kBM = 128, kBN = 128, kBK = 64;   // kBN: the usual tile width (256 for the weight gradients)
constexpr int kTileABytes = kBM * kBK * 2;
constexpr int stage_bytes(int bn) { return kTileABytes + bn * kBK * 2; }
// epilogue warps (then one TMA producer warp and one MMA issuer warp)
constexpr int gemm_epi_warps(int stages) { return stages <= 3 ? 8 : 16; }
constexpr int gemm_threads(int stages) { return gemm_epi_warps(stages) * 32 + 64; }
// ring, then 256 bytes of barriers and the tile's bias (512 bytes), plus the
// 1024-byte alignment of the ring
constexpr size_t gemm_smem(int stages, int bn) { return (size_t)stages * stage_bytes(bn) + 1024 + 256 + 512; }
constexpr int kMaxGroup = 4;              // GEMM problems of one launch

// Epilogues: kEpiBiasGelu  z = acc + bias -> out_f32 (z, optional), out_bf16
//                          = GELU(z), out_t = its transpose (optional);
//            kEpiF32       out_f32 = acc (K slice s at out_f32 + s * zstride);
//            kEpiGeluBwd   d = BF16(acc * GELU'(zin)) -> out_bf16, out_t (its
//                          transpose), colpart[row tile][col] = column sums
//                          of d over the tile's 128 rows (FP32, in row order).
// The FP32 epilogue runs with either ring; the others stage 128 KB and take
// the 6-stage ring.
enum : int { kEpiBiasGelu = 0, kEpiF32 = 1, kEpiGeluBwd = 3 };

// Operands and outputs of one problem of a grouped launch: D = A . B^T with
// A [M][K] and B [N][K] row-major BF16.
struct GemmProblem {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  const float* bias;           // [N] (kEpiBiasGelu)
  __nv_bfloat16* out_bf16;     // [M][ldo]
  float* out_f32;              // [M][ldo]
  __nv_bfloat16* out_t;        // [N][ldt] or nullptr
  const float* zin;            // [M][ldo] pre-activations (kEpiGeluBwd)
  float* colpart;              // [M / 128][N] (kEpiGeluBwd)
};

// One launch: np problems of the same shape, each split into ksplit slices
// of K (K / ksplit a multiple of 64), in tiles of 128 x bn.  Launchable
// (stages, epilogue, bn): (3, F32, 128), (6, BiasGelu, 128), (6, GeluBwd,
// 128), (4, F32, 256); the 256-wide tile runs the tensor cores at twice the
// rate of the 128-wide one (M = 128, N = 256 per instruction).
struct GemmLaunch {
  int np = 1, M = 0, N = 0, K = 0, ksplit = 1, epi = kEpiF32, bn = kBN;
  int ldo = 0, ldt = 0;
  long long zstride = 0;       // elements between the outputs of consecutive K slices
  int stages = 3;
  unsigned* err = nullptr;
  GemmProblem p[kMaxGroup] = {};
};

// Flat FP32 parameter vector: for l < 4, W_l [512 out][in] then b_l [512]
// (in = 512); then W_5 [18][512] and b_5 [18].  BF16 working copies: wb holds
// the weight matrices in the same order, wt the transposes of the hidden ones.
constexpr long long kLayerParams = (long long)kHidden * kHidden + kHidden;
constexpr long long kHeadW = (long long)kLayers * kLayerParams;
constexpr long long kHeadB = kHeadW + (long long)kOut * kHidden;
constexpr long long kNumParams = kHeadB + kOut;
constexpr long long kWbElems = (long long)kLayers * kHidden * kHidden + (long long)kOut * kHidden;
constexpr long long kWtElems = (long long)kLayers * kHidden * kHidden;

struct AdamLayout {
  __device__ __forceinline__ bool is_weight(long long i) const {
    if (i >= kHeadB) return false;
    if (i >= kHeadW) return true;
    return (i % kLayerParams) < (long long)kHidden * kHidden;
  }
  // the row-major BF16 working copy of a weight entry (biases have none)
  __device__ __forceinline__ void store_bf16(long long i, float w, __nv_bfloat16* wb) const {
    if (i >= kHeadB) return;
    if (i >= kHeadW) {
      wb[(long long)kLayers * kHidden * kHidden + (i - kHeadW)] = __float2bfloat16_rn(w);
      return;
    }
    const long long l = i / kLayerParams, r = i % kLayerParams;
    if (r >= (long long)kHidden * kHidden) return;
    wb[l * kHidden * kHidden + r] = __float2bfloat16_rn(w);
  }
};

// Gradient assembly, every sum in a fixed order: hidden weight matrices from
// the K-slice partials of the weight-gradient GEMM (slice order), hidden
// biases from the per-row-tile column sums of the rounded errors, the output
// layer from the head kernel's per-block partials (eight interleaved partial
// sums per entry, then their sum in order).  The batch loss (the sum of the
// rows' terms) goes into loss[t] when given.  With adam set, each entry's
// AdamW step follows from its assembled gradient (as k_adamw), and the
// transposed BF16 copies are refreshed after.  t = *t_idx when t_idx is
// given (a step of a replayed sequence; the transposes then advance it by
// one), else 0; the bias corrections are bc_tab[2 t], bc_tab[2 t + 1] when
// bc_tab is given, else bc1, bc2.
struct FinishArgs {
  const float* wpart;          // [4][ksplit][512][512]
  int ksplit;
  const float* colpart[kLayers];
  int ntiles[kLayers];         // partials summed per hidden bias
  const float* dWpart;         // [nblk][18][512]
  const float* dbpart;         // [nblk][18]
  int nblk;
  const float* row_loss;
  int M;
  float* loss;
  int* t_idx;                  // read by every block; advanced after the AdamW step
  const float* bc_tab;
  float* g;
  int adam;
  float lr, b1, b2, eps, wd, bc1, bc2;
  float* w;
  float* m1;
  float* m2;
  __nv_bfloat16* wb;
  __nv_bfloat16* wt;
};


cudaError_t gemm_prepare();
cudaError_t gemm(const GemmLaunch& L, cudaStream_t st);
cudaError_t head_fwd_loss(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, int M,
                          float* Y, float* dY, float* row_loss, cudaStream_t st);
// Training head: output layer, loss terms, dY, the layer-3 error dZ3 (and
// its transpose and per-32-row column sums), output-layer gradient partials
// per 32-row block.  M a multiple of 32.
cudaError_t head_train(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, const float* Z,
                       int M, float* Y, float* dY, float* row_loss, __nv_bfloat16* dZ, __nv_bfloat16* dZt, float* colpart,
                       float* dWpart, float* dbpart, cudaStream_t st);
cudaError_t grad_finish(const FinishArgs& a, cudaStream_t st);
cudaError_t adam_corrections(float b1, float b2, int step, float* bc1, float* bc2);
cudaError_t transpose_layers(const __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st, int* step_idx = nullptr);
cudaError_t adamw(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                  float wd, int step, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st);
cudaError_t pack_params(const float* w, int n, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt,
                        cudaStream_t st);
cudaError_t featurize(const DevSac* sacs, const float* traces, int n, __nv_bfloat16* X, __nv_bfloat16* Xt, int ldt,
                      cudaStream_t st);
cudaError_t apply_centres(const float* Y, int n, float* pc, cudaStream_t st);
cudaError_t bump(long long* p64, long long by64, int* p32, cudaStream_t st);
cudaError_t gen_desc(uint64_t seed, const long long* base, int n, const float* cal_amp, const float* cal_pulse, int ncal,
                     DevSac* sacs, float* hidden, float* target, int lcap, cudaStream_t st);
cudaError_t add_noise(uint64_t seed, const long long* base, const DevSac* sacs, int n, float* traces, float sigma,
                      cudaStream_t st);

}  // namespace mlp
}  // namespace opmm
