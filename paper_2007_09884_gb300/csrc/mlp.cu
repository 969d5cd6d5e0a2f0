// mlp.cu -- kernels of the learned surrogate (sm_103a).
//
// The surrogate is a multilayer perceptron 512 -> 512 x 4 (GELU) -> 18 that
// maps a resampled saccade to an OPC estimate.  Its dense layers run on the
// 5th-generation tensor cores:
//
//   k_gemm_tn   D[M,N] = A[M,K] . B[N,K]^T, BF16 operands, FP32 accumulate.
//               Warp 4 streams 128x64 tiles of A and B into a 3-stage shared
//               memory ring with TMA (cp.async.bulk.tensor, 128-byte swizzle);
//               one thread of warp 5 issues tcgen05.mma (M = 128, N = 128,
//               K = 16 per instruction) into an FP32 accumulator in tensor
//               memory and releases each stage with tcgen05.commit; warps 0-3
//               (one warpgroup, one TMEM lane quarter each) read the
//               accumulator with tcgen05.ld and apply the epilogue (bias,
//               GELU, BF16 conversion, optional transposed copy).
//
// Around it: the output layer (18 wide, CUDA cores), the loss, GELU backward
// with deterministic column sums, transposes, AdamW, the on-device training
// data generator and the featurizer.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/opmm.h"
#include "common.cuh"
#include "mlp.h"
#include "plant.cuh"

namespace opmm {
namespace mlp {

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzling:
// rows of 64 BF16 (128 B), 8-row core groups 1024 B apart (stride byte
// offset), leading byte offset unused by this layout, descriptor version 1,
// layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// ------------------------------------------------------------------ GEMM
__global__ void __launch_bounds__(kGemmThreads, 2)
    k_gemm_tn(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, GemmArgs g) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* bail = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = blockIdx.x, tm = blockIdx.y;
  const int nk = g.K / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *bail = 0;
    fence_mbar_init();
  }
  if (warp == 5) tc_alloc(tmem_slot, kBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      // TMA producer
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % kStages;
        const uint32_t use = (uint32_t)(kb / kStages);
        if (kb >= kStages && !mbar_wait(&empty[s], (use & 1u) ^ 1u, kMaxWaitTries)) {
          raise_error(g.err, kErrWaitTimeout);
          atomicExch(bail, 1);
          break;
        }
        unsigned char* st = sm + s * kStageBytes;
        mbar_arrive_expect_tx(&full[s], kStageBytes);
        tma_load_2d(st, &ta, kb * kBK, tm * kBM, &full[s]);
        tma_load_2d(st + kTileABytes, &tb, kb * kBK, tn * kBN, &full[s]);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = f16_idesc(kBM, kBN);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % kStages;
        const uint32_t use = (uint32_t)(kb / kStages);
        if (!mbar_wait(&full[s], use & 1u, kMaxWaitTries)) {
          raise_error(g.err, kErrWaitTimeout);
          atomicExch(bail, 1);
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sm + s * kStageBytes);
        const uint32_t b0 = a0 + kTileABytes;
#pragma unroll
        for (int k = 0; k < kBK / 16; ++k)
          tc_mma(tmem, sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32), idesc, (kb | k) != 0 ? 1u : 0u);
        tc_commit(&empty[s]);
      }
      tc_commit(done);
    }
  } else {
    // epilogue warpgroup: warp w owns TMEM lanes [32 w, 32 w + 32) = rows of the tile
    const bool ok = mbar_wait(done, 0u, kMaxWaitTries);
    if (!ok) raise_error(g.err, kErrWaitTimeout);
    tc_fence_after();
    const int row = tm * kBM + warp * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < kBN && ok; c0 += 16) {
      float v[16];
      tc_ld16(tbase + (uint32_t)c0, v);
      const int col = tn * kBN + c0;
      if (g.epi == kEpiF32) {
        float4* o = reinterpret_cast<float4*>(g.out_f32 + (size_t)row * g.ldo + col);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      } else {
        if (g.bias) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += g.bias[col + i];
        }
        if (g.epi == kEpiBiasGelu) {
          if (g.out_f32) {
            float4* o = reinterpret_cast<float4*>(g.out_f32 + (size_t)row * g.ldo + col);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = gelu(v[i]);
        }
        __nv_bfloat162 h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        uint4* o = reinterpret_cast<uint4*>(g.out_bf16 + (size_t)row * g.ldo + col);
        o[0] = *reinterpret_cast<uint4*>(&h[0]);
        o[1] = *reinterpret_cast<uint4*>(&h[4]);
        if (g.out_t) {
          // transposed copy: for each column the warp writes 32 consecutive rows
#pragma unroll
          for (int i = 0; i < 16; ++i)
            g.out_t[(size_t)(col + i) * g.ldt + row] = __float2bfloat16_rn(v[i]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tc_dealloc(tmem, kBN);
}

// ------------------------------------------------------------------ elementwise / reductions
// 32x32 tiled transpose of a BF16 matrix [R][C] -> [C][R].
__global__ void k_transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C) t[i][threadIdx.x] = in[(size_t)r * C + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < C) out[(size_t)c * R + r] = t[threadIdx.x][i];
  }
}

// dZ = dH * GELU'(Z) for a [M][N] layer: writes dZ (BF16, row-major and
// transposed) and per-32-row partial column sums (bias gradient, reduced
// deterministically by k_colsum).
__global__ void k_gelu_bwd(const float* dH, const float* Z, int M, int N, __nv_bfloat16* dZ, __nv_bfloat16* dZt,
                           float* colpart) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + tx;
    const size_t idx = (size_t)r * N + c;
    const float d = dH[idx] * gelu_grad(Z[idx]);
    const __nv_bfloat16 b = __float2bfloat16_rn(d);
    dZ[idx] = b;
    t[i][tx] = __bfloat162float(b);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + tx;
    dZt[(size_t)c * M + r] = __float2bfloat16_rn(t[tx][i]);
  }
  if (threadIdx.y == 0) {
    float s = 0.0f;
    for (int i = 0; i < 32; ++i) s += t[i][tx];
    colpart[(size_t)blockIdx.y * N + c0 + tx] = s;
  }
}

// out[n] = sum over row blocks of part[rb][n] (fixed order).
__global__ void k_colsum(const float* part, int rblocks, int N, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int rb = 0; rb < rblocks; ++rb) s += part[(size_t)rb * N + n];
  out[n] = s;
}

// Output layer and loss: Y[m][o] = H[m] . W5[o] + b5[o] (o < 18, CUDA cores);
// loss contribution and dY = 2 (Y - T) / (M * 18).  One warp per row.
__global__ void k_head_fwd_loss(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, int M,
                                float* Y, float* dY, float* row_loss) {
  const int lane = threadIdx.x & 31;
  const int m = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (m >= M) return;
  float acc[kOut];
#pragma unroll
  for (int o = 0; o < kOut; ++o) acc[o] = 0.0f;
  for (int k = lane; k < kHidden; k += 32) {
    const float h = __bfloat162float(H[(size_t)m * kHidden + k]);
#pragma unroll
    for (int o = 0; o < kOut; ++o) acc[o] = fmaf(h, __bfloat162float(W5[(size_t)o * kHidden + k]), acc[o]);
  }
  float l = 0.0f;
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    float v = acc[o];
#pragma unroll
    for (int s = 16; s; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    v += b5[o];
    if (lane == 0) {
      Y[(size_t)m * kOut + o] = v;
      if (T) {
        const float d = v - T[(size_t)m * kOut + o];
        l += d * d;
        dY[(size_t)m * kOut + o] = 2.0f * d / (float)(M * kOut);
      }
    }
  }
  if (lane == 0 && row_loss) row_loss[m] = l / (float)(M * kOut);
}

// Backward of the output layer: dH[m][k] = sum_o dY[m][o] W5[o][k] (FP32);
// partial sums over 32-row blocks of dW5[o][k] = sum_m dY[m][o] H[m][k] and
// db5[o] = sum_m dY[m][o].  Block: 32 rows x 512 columns, 256 threads.
__global__ void k_head_bwd(const float* dY, const __nv_bfloat16* H, const __nv_bfloat16* W5, int M, float* dH,
                           float* dWpart, float* dbpart) {
  __shared__ float sdy[32][kOut];
  const int r0 = blockIdx.x * 32;
  for (int i = threadIdx.x; i < 32 * kOut; i += blockDim.x) sdy[i / kOut][i % kOut] = dY[(size_t)(r0 + i / kOut) * kOut + i % kOut];
  __syncthreads();
  for (int k = threadIdx.x; k < kHidden; k += blockDim.x) {
    float w[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) w[o] = __bfloat162float(W5[(size_t)o * kHidden + k]);
    float gw[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) gw[o] = 0.0f;
    for (int i = 0; i < 32; ++i) {
      const int m = r0 + i;
      const float h = __bfloat162float(H[(size_t)m * kHidden + k]);
      float s = 0.0f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) {
        s = fmaf(sdy[i][o], w[o], s);
        gw[o] = fmaf(sdy[i][o], h, gw[o]);
      }
      dH[(size_t)m * kHidden + k] = s;
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) dWpart[((size_t)blockIdx.x * kOut + o) * kHidden + k] = gw[o];
  }
  if (threadIdx.x < kOut) {
    float s = 0.0f;
    for (int i = 0; i < 32; ++i) s += sdy[i][threadIdx.x];
    dbpart[(size_t)blockIdx.x * kOut + threadIdx.x] = s;
  }
}

// AdamW on the flat FP32 parameter vector; refreshes the BF16 working copies
// (weights [out][in] and, for the hidden layers, their transposes [in][out]).
__global__ void k_adamw(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                        float wd, float bc1, float bc2, const AdamLayout L, __nv_bfloat16* wb, __nv_bfloat16* wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  const bool decay = L.is_weight(i);
  float wi = w[i];
  if (decay) wi -= lr * wd * wi;
  wi -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  w[i] = wi;
  L.scatter(i, wi, wb, wt);
}

// Refresh the BF16 working copies from the FP32 master parameters.
__global__ void k_pack_params(const float* w, int n, const AdamLayout L, __nv_bfloat16* wb, __nv_bfloat16* wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  L.scatter(i, w[i], wb, wt);
}

// ------------------------------------------------------------------ data
// Featurizer: resample the trace on a 1 ms grid from onset (256 points, linear
// interpolation, held after the window end) in the positive frame, position
// normalised by the amplitude (start fixation = 0, end fixation = 1) and
// velocity as 10 x the per-millisecond difference.  Output BF16 [n][512]
// and its transpose [512][n_pad].
__global__ void k_featurize(const DevSac* sacs, const float* traces, int n, __nv_bfloat16* X, __nv_bfloat16* Xt,
                            int ldt) {
  const int lane = threadIdx.x & 31;
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b >= n) return;
  const DevSac d = sacs[b];
  const float* y = traces + d.off;
  const float amp = fmaxf(d.thf - d.th0, 0.5f);
  const float inv = 1.0f / amp;
  float pos[kFeatPoints / 32 + 1];
#pragma unroll
  for (int j = 0; j <= kFeatPoints / 32; ++j) {
    const int i = lane + 32 * j;
    float v = 0.0f;
    if (i <= kFeatPoints) {
      float s = (float)d.onset + (float)i * d.fs * 1e-3f;
      s = fminf(s, (float)(d.L - 1));
      const int k0 = (int)floorf(s);
      const int k1 = min(k0 + 1, d.L - 1);
      const float w = s - (float)k0;
      const float yy = (1.0f - w) * y[k0] + w * y[k1];
      v = (d.sign * yy - d.th0) * inv;
    }
    pos[j] = v;
  }
#pragma unroll
  for (int j = 0; j < kFeatPoints / 32; ++j) {
    const int i = lane + 32 * j;
    const float nxt = __shfl_down_sync(0xffffffffu, pos[j], 1);
    const float nxt2 = __shfl_sync(0xffffffffu, pos[j + 1], 0);
    const float p1 = lane == 31 ? nxt2 : nxt;
    const float vel = (i == kFeatPoints - 1) ? 0.0f : 10.0f * (p1 - pos[j]);
    const __nv_bfloat16 bp = __float2bfloat16_rn(pos[j]);
    const __nv_bfloat16 bv = __float2bfloat16_rn(vel);
    X[(size_t)b * kIn + i] = bp;
    X[(size_t)b * kIn + kFeatPoints + i] = bv;
    if (Xt) {
      Xt[(size_t)i * ldt + b] = bp;
      Xt[(size_t)(kFeatPoints + i) * ldt + b] = bv;
    }
  }
}

// Box centres from the network's output: centre = nominal * exp(scale * y).
__global__ void k_apply_centres(const float* Y, int n, float scale, float* pc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kOut) return;
  pc[i] *= __expf(scale * Y[i]);
}

// Training data: per sample g = base + i, Philox4x32-10 (key = seed,
// counter = (g, word, 0, 0)) draws the rate (250/500/1000 Hz), the window
// (40-400 samples, redrawn until a 1 deg saccade fits), the amplitude
// (log-uniform up to 40 deg, capped by the window), the direction, the 18
// hidden multipliers U(0.8, 1.2) and N(0, 0.05^2) noise (Box-Muller).  The
// hidden OPC is the interpolated nominal centre times the multipliers.
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

__global__ void k_gen_desc(uint64_t seed, long long base, int n, const float* cal_amp, const float* cal_pulse,
                           int ncal, DevSac* sacs, float* hidden, float* target, int lcap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long g = base + i;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint32_t r[4];
  philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 0u, 0u, k0, k1, r);
  const float rates[3] = {250.0f, 500.0f, 1000.0f};
  const float fs = rates[min(2, (int)(u01(r[0]) * 3.0f))];
  const int on = (int)ceilf(0.010f * fs - 1e-6f);
  int L = 40 + min(360, (int)(u01(r[1]) * 361.0f));
  float amax = 0.0f;
  for (int t = 0; t < 16; ++t) {
    amax = fminf(40.0f, ((1000.0f * L / fs) - (1000.0f * on / fs) - 20.0f - 21.0f) / 2.2f);
    if (amax >= 1.0f) break;
    uint32_t q[4];
    philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 1u, (uint32_t)t, k0, k1, q);
    L = 40 + min(360, (int)(u01(q[0]) * 361.0f));
  }
  if (amax < 1.0f) { L = 400; amax = fminf(40.0f, ((1000.0f * L / fs) - (1000.0f * on / fs) - 41.0f) / 2.2f); }
  L = min(L, lcap);
  const float A = __expf(u01(r[2]) * __logf(amax));
  const float sign = u01(r[3]) < 0.5f ? 1.0f : -1.0f;
  const float D = 2.2f * A + 21.0f;
  DevSac d;
  d.off = (long long)i * lcap;
  d.L = L;
  d.onset = on;
  d.nsub = max(1, (int)floorf(1.0e4f / fs + 0.5f));
  d.fs = fs;
  d.h = 1.0f / (fs * (float)d.nsub);
  d.th0 = 0.0f;
  d.thf = A;
  d.sign = sign;
  d.dur_ms = D;
  sacs[i] = d;
  // nominal centre: Table 1, W = D - 6, agonist pulse interpolated in amplitude
  float t = (A - cal_amp[0]) / (cal_amp[ncal - 1] - cal_amp[0]) * (float)(ncal - 1);
  t = fminf(fmaxf(t, 0.0f), (float)(ncal - 1));
  const int j0 = min((int)t, ncal - 2);
  const float f = t - (float)j0;
  const float nsac = (1.0f - f) * cal_pulse[j0] + f * cal_pulse[j0 + 1];
  for (int blk = 0; blk < 5; ++blk) {
    uint32_t q[4];
    philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 2u, (uint32_t)blk, k0, k1, q);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * blk + c;
      if (j < kOut) {
        const float mult = 0.8f + 0.4f * u01(q[c]);
        float nom = kTable1[j];
        if (j == kPw) nom = D - 6.0f;
        if (j == kNsacAg) nom = nsac;
        hidden[(size_t)i * kOut + j] = nom * mult;
        target[(size_t)i * kOut + j] = __logf(mult) * (1.0f / kTargetScale);
      }
    }
  }
}

// Noisy trace: simulated trajectory plus N(0, 0.05^2) deg noise, in place.
__global__ void k_add_noise(uint64_t seed, long long base, const DevSac* sacs, int n, float* traces, float sigma) {
  const int b = blockIdx.x;
  if (b >= n) return;
  const DevSac d = sacs[b];
  const long long g = base + b;
  for (int k2 = threadIdx.x * 2; k2 < d.L; k2 += 2 * blockDim.x) {
    uint32_t q[4];
    philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 3u, (uint32_t)k2, (uint32_t)seed, (uint32_t)(seed >> 32), q);
    const float u1 = fmaxf(u01(q[0]), 1e-7f), u2 = u01(q[1]);
    const float rad = sqrtf(-2.0f * __logf(u1));
    traces[d.off + k2] += sigma * rad * __cosf(6.283185307f * u2);
    if (k2 + 1 < d.L) traces[d.off + k2 + 1] += sigma * rad * __sinf(6.283185307f * u2);
  }
}

// Sum of n floats by one block in a fixed order (deterministic).
__global__ void k_sum(const float* x, int n, float* out) {
  __shared__ float s[256];
  float a = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += x[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// ------------------------------------------------------------------ host launchers
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D tensor map of a row-major BF16 matrix [rows][cols], box 64 x 128
// (128-byte rows, 128-byte swizzle).
static bool make_map(CUtensorMap* map, const void* base, int rows, int cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t gemm_prepare() {
  return cudaFuncSetAttribute(k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
}

cudaError_t gemm_tn(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, const GemmArgs& args,
                    cudaStream_t st) {
  if (M % kBM || N % kBN || K % kBK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K) || !make_map(&tb, B, N, K)) return cudaErrorInvalidValue;
  GemmArgs g = args;
  g.M = M;
  g.N = N;
  g.K = K;
  dim3 grid(N / kBN, M / kBM);
  k_gemm_tn<<<grid, kGemmThreads, kGemmSmem, st>>>(ta, tb, g);
  return cudaGetLastError();
}

cudaError_t transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C, cudaStream_t st) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, st>>>(in, out, R, C);
  return cudaGetLastError();
}

cudaError_t gelu_bwd(const float* dH, const float* Z, int M, int N, __nv_bfloat16* dZ, __nv_bfloat16* dZt,
                     float* colpart, float* db, cudaStream_t st) {
  dim3 grid(N / 32, M / 32), block(32, 8);
  k_gelu_bwd<<<grid, block, 0, st>>>(dH, Z, M, N, dZ, dZt, colpart);
  k_colsum<<<(N + 127) / 128, 128, 0, st>>>(colpart, M / 32, N, db);
  return cudaGetLastError();
}

cudaError_t head_fwd_loss(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, int M,
                          float* Y, float* dY, float* row_loss, cudaStream_t st) {
  k_head_fwd_loss<<<(M * 32 + 255) / 256, 256, 0, st>>>(H, W5, b5, T, M, Y, dY, row_loss);
  return cudaGetLastError();
}

cudaError_t head_bwd(const float* dY, const __nv_bfloat16* H, const __nv_bfloat16* W5, int M, float* dH, float* dWpart,
                     float* dbpart, float* dW, float* db, cudaStream_t st) {
  k_head_bwd<<<M / 32, 256, 0, st>>>(dY, H, W5, M, dH, dWpart, dbpart);
  k_colsum<<<(kOut * kHidden + 127) / 128, 128, 0, st>>>(dWpart, M / 32, kOut * kHidden, dW);
  k_colsum<<<1, 32, 0, st>>>(dbpart, M / 32, kOut, db);
  return cudaGetLastError();
}

cudaError_t adamw(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                  float wd, int step, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st) {
  // bias corrections 1 - beta^t of the FP32 betas the kernel uses, formed in
  // double: in FP32 the cancellation in 1 - 0.999^t would cost up to 2^-24 /
  // (1 - 0.999^t) of relative precision (1.5e-5 at t = 2)
  const float bc1 = (float)(1.0 - pow((double)b1, (double)step));
  const float bc2 = (float)(1.0 - pow((double)b2, (double)step));
  k_adamw<<<(n + 255) / 256, 256, 0, st>>>(w, g, m1, m2, n, lr, b1, b2, eps, wd, bc1, bc2, L, wb, wt);
  return cudaGetLastError();
}

cudaError_t pack_params(const float* w, int n, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt,
                        cudaStream_t st) {
  k_pack_params<<<(n + 255) / 256, 256, 0, st>>>(w, n, L, wb, wt);
  return cudaGetLastError();
}

cudaError_t featurize(const DevSac* sacs, const float* traces, int n, __nv_bfloat16* X, __nv_bfloat16* Xt, int ldt,
                      cudaStream_t st) {
  k_featurize<<<(n * 32 + 127) / 128, 128, 0, st>>>(sacs, traces, n, X, Xt, ldt);
  return cudaGetLastError();
}

cudaError_t apply_centres(const float* Y, int n, float* pc, cudaStream_t st) {
  k_apply_centres<<<(n * kOut + 255) / 256, 256, 0, st>>>(Y, n, kTargetScale, pc);
  return cudaGetLastError();
}

cudaError_t gen_desc(uint64_t seed, long long base, int n, const float* cal_amp, const float* cal_pulse, int ncal,
                     DevSac* sacs, float* hidden, float* target, int lcap, cudaStream_t st) {
  k_gen_desc<<<(n + 127) / 128, 128, 0, st>>>(seed, base, n, cal_amp, cal_pulse, ncal, sacs, hidden, target, lcap);
  return cudaGetLastError();
}

cudaError_t add_noise(uint64_t seed, long long base, const DevSac* sacs, int n, float* traces, float sigma,
                      cudaStream_t st) {
  k_add_noise<<<n, 128, 0, st>>>(seed, base, sacs, n, traces, sigma);
  return cudaGetLastError();
}

cudaError_t sum_array(const float* x, int n, float* out, cudaStream_t st) {
  k_sum<<<1, 256, 0, st>>>(x, n, out);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace opmm
