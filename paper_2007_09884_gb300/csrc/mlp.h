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

// GEMM tiling: 128 x 128 output tile, 64-wide K slices, 3-stage ring (99 KB of
// shared memory, so two CTAs share an SM and one's epilogue overlaps the
// other's main loop).
constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 3;
constexpr int kTileABytes = kBM * kBK * 2;
constexpr int kTileBBytes = kBN * kBK * 2;
constexpr int kStageBytes = kTileABytes + kTileBBytes;
constexpr int kGemmThreads = 192;         // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer
constexpr size_t kGemmSmem = (size_t)kStages * kStageBytes + 1024 + 256;

enum : int { kEpiBiasGelu = 0, kEpiF32 = 1, kEpiBias = 2 };

struct GemmArgs {
  int M, N, K;
  int epi;                     // kEpi*
  const float* bias;           // [N] or nullptr
  __nv_bfloat16* out_bf16;     // [M][ldo] (kEpiBiasGelu, kEpiBias)
  float* out_f32;              // [M][ldo]: result (kEpiF32) or pre-activation (kEpiBiasGelu, optional)
  __nv_bfloat16* out_t;        // optional transposed BF16 copy [N][ldt]
  int ldo, ldt;
  unsigned* err;
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
  __device__ __forceinline__ void scatter(long long i, float w, __nv_bfloat16* wb, __nv_bfloat16* wt) const {
    if (i >= kHeadB) return;
    if (i >= kHeadW) {
      wb[(long long)kLayers * kHidden * kHidden + (i - kHeadW)] = __float2bfloat16_rn(w);
      return;
    }
    const long long l = i / kLayerParams, r = i % kLayerParams;
    if (r >= (long long)kHidden * kHidden) return;
    const long long o = r / kHidden, c = r % kHidden;
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    wb[l * kHidden * kHidden + r] = b;
    wt[l * kHidden * kHidden + c * kHidden + o] = b;
  }
};

cudaError_t gemm_prepare();
cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, const GemmArgs& args,
                    cudaStream_t st);
cudaError_t transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C, cudaStream_t st);
cudaError_t gelu_bwd(const float* dH, const float* Z, int M, int N, __nv_bfloat16* dZ, __nv_bfloat16* dZt,
                     float* colpart, float* db, cudaStream_t st);
cudaError_t head_fwd_loss(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, int M,
                          float* Y, float* dY, float* row_loss, cudaStream_t st);
cudaError_t head_bwd(const float* dY, const __nv_bfloat16* H, const __nv_bfloat16* W5, int M, float* dH, float* dWpart,
                     float* dbpart, float* dW, float* db, cudaStream_t st);
cudaError_t adamw(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                  float wd, int step, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st);
cudaError_t pack_params(const float* w, int n, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt,
                        cudaStream_t st);
cudaError_t featurize(const DevSac* sacs, const float* traces, int n, __nv_bfloat16* X, __nv_bfloat16* Xt, int ldt,
                      cudaStream_t st);
cudaError_t apply_centres(const float* Y, int n, float* pc, cudaStream_t st);
cudaError_t gen_desc(uint64_t seed, long long base, int n, const float* cal_amp, const float* cal_pulse, int ncal,
                     DevSac* sacs, float* hidden, float* target, int lcap, cudaStream_t st);
cudaError_t add_noise(uint64_t seed, long long base, const DevSac* sacs, int n, float* traces, float sigma,
                      cudaStream_t st);
cudaError_t sum_array(const float* x, int n, float* out, cudaStream_t st);

}  // namespace mlp
}  // namespace opmm
