// mlp.cu -- kernels of the learned surrogate (sm_103a).
//
// The surrogate is a multilayer perceptron 512 -> 512 x 4 (GELU) -> 18 that
// maps a resampled saccade to an OPC estimate.  Its dense layers run on the
// 5th-generation tensor cores:
//
//   k_gemm_tn   D = A . B^T for up to four same-shape problems per launch
//               (each optionally split into K slices), BF16 operands, FP32
//               accumulate: a producer warp streams 128 x 64 tiles of A and
//               BN x 64 tiles of B into a shared-memory ring with TMA
//               (cp.async.bulk.tensor, 128-byte swizzle), one thread of the
//               MMA warp issues tcgen05.mma (M = 128, N = BN, K = 16) into a
//               TMEM accumulator and frees each stage with tcgen05.commit,
//               and 8 or 16 epilogue warps read the accumulator with
//               tcgen05.ld, apply the epilogue (bias + GELU with Z and H^T;
//               GELU' with the rounded error, its transpose and bias-gradient
//               column sums; plain FP32) and stage the tile for bulk tensor
//               stores.
//
// Around it: the training head (output layer, loss, the layer-3 error, the
// output layer's gradient partials), the gradient assembly fused with AdamW,
// the transposes of the BF16 weights, the inference head, the on-device
// training data generator and the featurizer.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

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

// Bulk tensor store of a shared-memory box to global memory (tile mode,
// bulk-group completion), and the wait until this thread's bulk groups have
// read their shared-memory sources.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

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

// 64 consecutive FP32 accumulator columns of this thread's TMEM lane, with
// the wait for the load in the same statement (the registers are not valid
// before it).
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane (load
// and wait in one statement).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[32]) { tc_ld32(taddr, v); }
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[64]) { tc_ld64(taddr, v); }

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

// The Gaussian CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2 with erf from
// Abramowitz and Stegun, Handbook of Mathematical Functions, formula 7.1.26:
// for x >= 0, erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) e^(-x^2)
// with t = 1 / (1 + p x), absolute error at most 1.5e-7.  Written as
// Phi = 1 - q (z >= 0) or q (z < 0) with q = poly(t) e^(-z^2 / 2) / 2, so
// the negative side has no cancellation; e = e^(-z^2 / 2) also gives the
// density phi(z) = e / sqrt(2 pi) that GELU' needs.  GELU(z) = z Phi(z),
// GELU'(z) = Phi(z) + z phi(z).
// A&S 7.1.26: p 0.3275911 a1 0.254829592 a2 -0.284496736 a3 1.421413741 a4 -1.453152027 a5 1.061405429
__device__ __forceinline__ float gauss_cdf(float z, float& e) {
  const float x = fabsf(z) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
  e = __expf(-0.5f * z * z);
  const float q = 0.5f * poly * e;
  return z >= 0.0f ? 1.0f - q : q;
}
__device__ __forceinline__ float gelu(float z) {
  float e;
  return z * gauss_cdf(z, e);
}
__device__ __forceinline__ float gelu_grad(float z) {
  float e;
  const float cdf = gauss_cdf(z, e);
  return fmaf(z, 0.39894228040143268f * e, cdf);
}

// ------------------------------------------------------------------ GEMM
// Tensor maps of a grouped launch: A and B of each problem, and its outputs
// (FP32 in 32-column boxes, BF16 row-major and transposed in 64-column
// boxes, all 128 rows high with the 128-byte swizzle).
struct GemmMaps {
  CUtensorMap a[kMaxGroup];
  CUtensorMap b[kMaxGroup];
  CUtensorMap of[kMaxGroup];
  CUtensorMap ob[kMaxGroup];
  CUtensorMap ot[kMaxGroup];
};

// The launch's shape and the problems' outputs, as the kernel sees them.
struct GemmArgs {
  int M, N, nkb, ksplit, ldo, ldt;     // nkb: 64-wide K blocks per slice
  long long zstride;
  unsigned* err;
  GemmProblem p[kMaxGroup];
};

// Barrier of the NT epilogue threads (named barrier 1).
template <int NT>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

// D tile (tm, tn) of problem blockIdx.z / ksplit over K slice blockIdx.z %
// ksplit.  Warp 8 lane 0 streams the A and B tiles of each 64-wide K block
// into the ring (TMA, 128-byte swizzle); warp 9 lane 0 issues four
// tcgen05.mma (K = 16 each) per stage into a 128 x 128 FP32 accumulator in
// tensor memory and frees the stage with tcgen05.commit.  Warps 0 .. EW - 1
// are the epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its tile
// rows) and NC = 512 / EW columns from NC (w / 4), applies the epilogue EPI
// and stages the tile in the ring, which every MMA has finished reading by
// then, in the boxes of the output tensor maps; one thread then writes the
// boxes out with bulk tensor stores.  EW = 16 with the 6-stage
// ring (one CTA per SM; the network's one-wave GEMMs, whose time is the
// latency of one tile: the per-element math of GELU and GELU' is spread over
// as many threads as the registers allow) and 8 with the 3-stage ring (two
// CTAs per SM).  Staging, as the 128-byte swizzle of the tensor maps lays a
// box out (row q of a box at 128 q bytes, its 16-byte chunk c at position
// c ^ (q & 7)): Sf, BN / 32 FP32 boxes of [128 rows][32 columns] at 0; Sbf,
// two BF16 boxes of [128 rows][64 columns] at 64 KB; St, the transpose, two
// BF16 boxes of [128 columns][64 rows] at 96 KB.  The swizzle also puts the
// 32 rows of a warp that write one logical chunk on distinct banks.  Every
// wait is bounded; a wait that expires raises the error word and the tile's
// output is not written.
template <int STAGES, int EPI, int BN>
__global__ void __launch_bounds__(gemm_threads(STAGES), STAGES <= 3 ? 2 : 1)
    k_gemm_tn(const __grid_constant__ GemmMaps maps, const __grid_constant__ GemmArgs g) {
  constexpr int EW = gemm_epi_warps(STAGES), ET = EW * 32, NC = BN * 4 / EW;
  constexpr int kTmaWarp = EW, kMmaWarp = EW + 1;
  constexpr int kStageBytes = stage_bytes(BN);
  static_assert(EPI == kEpiF32 || BN == 128, "the BF16 epilogues take 128-wide tiles");
  static_assert(STAGES * kStageBytes >= (EPI == kEpiF32 ? kBM * BN * 4 : 131072),
                "the epilogue stages its tile in the ring");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + STAGES * kStageBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* bail = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = blockIdx.x, tm = blockIdx.y;
  const int prob = blockIdx.z / g.ksplit, slice = blockIdx.z - prob * g.ksplit;
  const int kb0 = slice * g.nkb;
  const int nk = g.nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *bail = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tc_alloc(tmem_slot, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // TMA producer
      const CUtensorMap* ma = &maps.a[prob];
      const CUtensorMap* mb = &maps.b[prob];
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t use = (uint32_t)(kb / STAGES);
        if (kb >= STAGES && !mbar_wait(&empty[s], (use & 1u) ^ 1u, kMaxWaitTries)) {
          raise_error(g.err, kErrWaitTimeout);
          atomicExch(bail, 1);
          break;
        }
        unsigned char* st = sm + s * kStageBytes;
        mbar_arrive_expect_tx(&full[s], kStageBytes);
        tma_load_2d(st, ma, (kb0 + kb) * kBK, tm * kBM, &full[s]);
        tma_load_2d(st + kTileABytes, mb, (kb0 + kb) * kBK, tn * BN, &full[s]);
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = f16_idesc(kBM, BN);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t use = (uint32_t)(kb / STAGES);
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
    // epilogue.  Before the accumulator is ready (overlapping the main loop):
    // the tile's bias in shared memory (kEpiBiasGelu) or GELU' of this
    // thread's NC pre-activations (kEpiGeluBwd).
    const GemmProblem& P = g.p[prob];
    const int tid = threadIdx.x;                 // 0 .. ET - 1
    const int q = warp & 3;                      // TMEM lane quarter
    const int r = q * 32 + lane;                 // tile row
    const int row = tm * kBM + r;
    const int cb = (warp >> 2) * NC;             // first tile column of this warp
    float* sbias = reinterpret_cast<float*>(sm + STAGES * kStageBytes + 256);   // [128], after the barriers
    float gz[EPI == kEpiGeluBwd ? NC : 1];
    if constexpr (EPI == kEpiBiasGelu) {
      if (tid < kBN) sbias[tid] = P.bias[tn * kBN + tid];
    }
    if constexpr (EPI == kEpiGeluBwd) {
      const float4* zp = reinterpret_cast<const float4*>(P.zin + (size_t)row * g.ldo + tn * BN + cb);
#pragma unroll
      for (int i = 0; i < NC / 4; ++i) {
        const float4 z = zp[i];
        gz[4 * i] = gelu_grad(z.x);
        gz[4 * i + 1] = gelu_grad(z.y);
        gz[4 * i + 2] = gelu_grad(z.z);
        gz[4 * i + 3] = gelu_grad(z.w);
      }
    }
    const bool ok = mbar_wait(done, 0u, kMaxWaitTries);
    if (!ok) {
      raise_error(g.err, kErrWaitTimeout);
      atomicExch(bail, 1);
    }
    tc_fence_after();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    epi_bar<ET>();
    const bool go = *reinterpret_cast<volatile int*>(bail) == 0;
    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
    unsigned char* Sf = sm;                      // BN / 32 boxes [128][32] FP32
    unsigned char* Sbf = sm + 65536;             // 2 boxes [128][64] BF16
    unsigned char* St = sm + 98304;              // 2 boxes [128 columns][64 rows] BF16
    const bool want_f32 = EPI == kEpiF32 || (EPI == kEpiBiasGelu && P.out_f32 != nullptr);
    const bool want_t = EPI != kEpiF32 && P.out_t != nullptr;
    const int sw = r & 7;
    if (go) {
      float v[NC];
      tc_ld(tbase + (uint32_t)cb, v);
#pragma unroll
      for (int c = 0; c < NC; c += 16) {
        const int col0 = cb + c;                 // column within the tile
        if constexpr (EPI == kEpiGeluBwd) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[c + i] *= gz[c + i];
        }
        if constexpr (EPI == kEpiBiasGelu) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[c + i] += sbias[col0 + i];
        }
        if (want_f32) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int cc = col0 + 4 * j;         // box cc / 32, chunk (cc % 32) / 4
            *reinterpret_cast<float4*>(Sf + (cc >> 5) * 16384 + r * 128 + ((((cc & 31) >> 2) ^ sw) << 4)) =
                make_float4(v[c + 4 * j], v[c + 4 * j + 1], v[c + 4 * j + 2], v[c + 4 * j + 3]);
          }
        }
        if constexpr (EPI != kEpiF32) {
          if constexpr (EPI == kEpiBiasGelu) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[c + i] = gelu(v[c + i]);
          }
          __nv_bfloat162 h[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[c + 2 * i], v[c + 2 * i + 1]);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int cc = col0 + 8 * j;         // box cc / 64, chunk (cc % 64) / 8
            *reinterpret_cast<uint4*>(Sbf + (cc >> 6) * 16384 + r * 128 + ((((cc & 63) >> 3) ^ sw) << 4)) =
                *reinterpret_cast<const uint4*>(&h[4 * j]);
          }
          if (want_t) {
            // element (row r, column cc): box r / 64, box row cc, chunk (r % 64) / 8
            unsigned char* tb = St + (r >> 6) * 16384 + (r & 7) * 2;
            const int rc = (r & 63) >> 3;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int c0 = col0 + 2 * i, c1 = c0 + 1;
              *reinterpret_cast<__nv_bfloat16*>(tb + c0 * 128 + ((rc ^ (c0 & 7)) << 4)) = h[i].x;
              *reinterpret_cast<__nv_bfloat16*>(tb + c1 * 128 + ((rc ^ (c1 & 7)) << 4)) = h[i].y;
            }
          }
        }
      }
    }
    // the staged boxes become visible to the bulk copies (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    epi_bar<ET>();
    if (go) {
      const int y0 = tm * kBM;
      const int x0 = tn * BN;
      if (tid == 0) {
        if (want_f32) {
          const int yf = EPI == kEpiF32 ? y0 + slice * g.M : y0;   // K slices stacked by rows
#pragma unroll 1
          for (int bx = 0; bx < BN / 32; ++bx) tma_store_2d(&maps.of[prob], x0 + 32 * bx, yf, Sf + bx * 16384);
        }
        if constexpr (EPI != kEpiF32) {
          for (int bx = 0; bx < 2; ++bx) tma_store_2d(&maps.ob[prob], x0 + 64 * bx, y0, Sbf + bx * 16384);
          if (want_t)
            for (int bx = 0; bx < 2; ++bx) tma_store_2d(&maps.ot[prob], y0 + 64 * bx, x0, St + bx * 16384);
        }
        bulk_commit();
      }
      if constexpr (EPI == kEpiGeluBwd) {
        if (tid < 128) {
          // column sum of the rounded errors over the tile's rows, in row order
          const unsigned char* cbp = Sbf + (tid >> 6) * 16384 + (tid & 7) * 2;
          const int ch = (tid & 63) >> 3;
          float s = 0.0f;
          for (int rr = 0; rr < 128; ++rr)
            s += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(cbp + rr * 128 + ((ch ^ (rr & 7)) << 4)));
          P.colpart[(size_t)tm * g.N + x0 + tid] = s;
        }
      }
      // the copies must have read the staging area before the block exits
      // (their writes are complete when the grid is)
      if (tid == 0) bulk_wait_read();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) tc_dealloc(tmem, BN);
}

// ------------------------------------------------------------------ elementwise / reductions
// Transposes of the hidden weight matrices: wt_l = wb_l^T for the four
// 512 x 512 BF16 matrices (blockIdx.z = layer), through a 32 x 32 tile.
// When step_idx is given (the step index of a replayed training sequence),
// one thread advances it: this kernel follows the step's AdamW, the last
// reader of the index.
__global__ void k_transpose_layers(const __nv_bfloat16* wb, __nv_bfloat16* wt, int* step_idx) {
  if (step_idx && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    *step_idx += 1;
  __shared__ __nv_bfloat16 t[32][34];
  const size_t lo = (size_t)blockIdx.z * kHidden * kHidden;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) t[i][threadIdx.x] = wb[lo + (size_t)(r0 + i) * kHidden + c0 + threadIdx.x];
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) wt[lo + (size_t)(c0 + i) * kHidden + r0 + threadIdx.x] = t[threadIdx.x][i];
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

// Output layer, loss and the first steps of the backward pass for 32 rows
// per block (training; 512 threads): y = H3 . W5^T + b5, the rows' loss terms
// and dY = 2 (y - t) / (M 18); then per column k (one thread each): the
// block's partial sums of dW5[o][k] = sum_m dY[m][o] H3[m][k] (and of db5 =
// sum_m dY), dH3 = dY . W5 and the rounded layer-3 error dZ3 = BF16(dH3 *
// GELU'(Z3)), written row-major and transposed (through shared memory, in
// whole rows) with its column sums over the block's rows.  W5 (as FP32) and
// the block's H3 rows are staged in shared memory; each thread's 32 Z3
// values are loaded at the start, so their latency overlaps the forward
// part.  Every sum runs in a fixed order.
constexpr int kHeadRows = 32;
constexpr int kHeadThreads = 512;
static_assert(kHeadThreads == kHidden && kHeadRows == 2 * (kHeadThreads / 32), "one thread per column, two rows per warp");
constexpr int kSdzPitch = kHidden + 2;     // BF16 elements: rows one bank apart
constexpr int kSdyPitch = 20;              // FP32 elements per row of dY in shared memory (16-byte rows)
static_assert(kOut == 18 && kSdyPitch >= kOut && kSdyPitch % 4 == 0, "dY rows read as four float4 and a float2");
constexpr size_t kHeadSmem = (size_t)kOut * kHidden * 4 + (size_t)kHeadRows * kHidden * 2 +
                             (size_t)kHeadRows * kSdzPitch * 2 + 2 * (size_t)kHeadRows * kSdyPitch * 4;

__global__ void __launch_bounds__(kHeadThreads) k_head_train(const __nv_bfloat16* H, const __nv_bfloat16* W5,
                                                             const float* b5, const float* T, const float* Z, int M,
                                                             float* Y, float* dY, float* row_loss, __nv_bfloat16* dZ,
                                                             __nv_bfloat16* dZt, float* colpart, float* dWpart,
                                                             float* dbpart) {
  extern __shared__ __align__(16) unsigned char hsm[];
  float* sw = reinterpret_cast<float*>(hsm);                                    // [18][512]
  __nv_bfloat16* sh = reinterpret_cast<__nv_bfloat16*>(sw + kOut * kHidden);   // [32][512]
  __nv_bfloat16* sdz = sh + kHeadRows * kHidden;                                // [32][kSdzPitch]
  float* sdy = reinterpret_cast<float*>(sdz + kHeadRows * kSdzPitch);           // [32][kSdyPitch]
  float* stg = sdy + kHeadRows * kSdyPitch;                                     // [32][kSdyPitch] targets
  __shared__ float sb5[kOut];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = blockIdx.x * kHeadRows;
  float z[kHeadRows];
#pragma unroll
  for (int i = 0; i < kHeadRows; ++i) z[i] = Z[(size_t)(r0 + i) * kHidden + tid];
  for (int i = tid; i < kOut * kHidden / 2; i += kHeadThreads) {
    const float2 w = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(W5)[i]);
    reinterpret_cast<float2*>(sw)[i] = w;
  }
  {
    const uint4* hs = reinterpret_cast<const uint4*>(H + (size_t)r0 * kHidden);
    uint4* hd = reinterpret_cast<uint4*>(sh);
    for (int i = tid; i < kHeadRows * kHidden / 8; i += kHeadThreads) hd[i] = hs[i];
    // the block's targets, so that the loss below reads none of them from
    // global memory between its stores
    for (int i = tid; i < kHeadRows * kOut; i += kHeadThreads) stg[(i / kOut) * kSdyPitch + i % kOut] = T[(size_t)r0 * kOut + i];
    if (tid < kOut) sb5[tid] = b5[tid];
  }
  __syncthreads();
  // forward and loss: warp w takes rows 2 w and 2 w + 1 together (each W5
  // pair read from shared memory serves both), lane l the column pairs
  // 2 l + 64 j
  float acc2[2][kOut];
#pragma unroll
  for (int o = 0; o < kOut; ++o) acc2[0][o] = acc2[1][o] = 0.0f;
#pragma unroll 2
  for (int k = 2 * lane; k < kHidden; k += 64) {
    const float2 h0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(sh + (2 * warp) * kHidden + k));
    const float2 h1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(sh + (2 * warp + 1) * kHidden + k));
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      const float2 w = *reinterpret_cast<const float2*>(sw + o * kHidden + k);
      acc2[0][o] = fmaf(h0.y, w.y, fmaf(h0.x, w.x, acc2[0][o]));
      acc2[1][o] = fmaf(h1.y, w.y, fmaf(h1.x, w.x, acc2[1][o]));
    }
  }
  // Sum the 36 lane partials (2 rows x 18 outputs) over the warp by a
  // reduce-scatter: the values as v[2 o + rr] (o < 32, zero past 18); at each
  // of five levels a lane keeps the half its lane bit selects and adds its
  // partner's copy of that half (62 shuffles in all), after which lane o holds
  // output o of both rows.
  {
    float v[64];
#pragma unroll
    for (int o = 0; o < 32; ++o) {
      v[2 * o] = o < kOut ? acc2[0][o] : 0.0f;
      v[2 * o + 1] = o < kOut ? acc2[1][o] : 0.0f;
    }
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
      const int off = 16 >> lev, half = 32 >> lev;
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float send = up ? v[j] : v[j + half];
        const float keep = up ? v[j + half] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    const int o = lane;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int i = 2 * warp + rr;
      const int m = r0 + i;
      float l = 0.0f;
      if (o < kOut) {
        const float y = v[rr] + sb5[o];
        const float d = y - stg[i * kSdyPitch + o];
        l = d * d;
        const float g = 2.0f * d / (float)(M * kOut);
        Y[(size_t)m * kOut + o] = y;
        dY[(size_t)m * kOut + o] = g;
        sdy[i * kSdyPitch + o] = g;
      }
#pragma unroll
      for (int sft = 16; sft; sft >>= 1) l += __shfl_xor_sync(0xffffffffu, l, sft);
      if (lane == 0) row_loss[m] = l / (float)(M * kOut);
    }
  }
  __syncthreads();
  // per column: output-layer gradient partials, dH3, GELU backward
  {
    const int k = tid;
    float w[kOut], gw[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      w[o] = sw[o * kHidden + k];
      gw[o] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < kHeadRows; ++i) {
      const float h = __bfloat162float(sh[i * kHidden + k]);
      float dy[kOut];
#pragma unroll
      for (int o = 0; o < 16; o += 4) {
        const float4 t = *reinterpret_cast<const float4*>(sdy + i * kSdyPitch + o);
        dy[o] = t.x;
        dy[o + 1] = t.y;
        dy[o + 2] = t.z;
        dy[o + 3] = t.w;
      }
      {
        const float2 t = *reinterpret_cast<const float2*>(sdy + i * kSdyPitch + 16);
        dy[16] = t.x;
        dy[17] = t.y;
      }
      float s = 0.0f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) {
        s = fmaf(dy[o], w[o], s);
        gw[o] = fmaf(dy[o], h, gw[o]);
      }
      const float d = s * gelu_grad(z[i]);
      sdz[i * kSdzPitch + k] = __float2bfloat16_rn(d);
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) dWpart[((size_t)blockIdx.x * kOut + o) * kHidden + k] = gw[o];
  }
  if (tid < kOut) {
    float s = 0.0f;
    for (int i = 0; i < kHeadRows; ++i) s += sdy[i * kSdyPitch + tid];
    dbpart[(size_t)blockIdx.x * kOut + tid] = s;
  }
  __syncthreads();
  // dZ3 row-major (pairs of columns per thread), its transpose (8 rows of one
  // column per 16-byte store) and the column sums
  for (int q = tid; q < kHeadRows * kHidden / 2; q += kHeadThreads) {
    const int i = q / (kHidden / 2), c2 = q - i * (kHidden / 2);
    *reinterpret_cast<__nv_bfloat162*>(dZ + (size_t)(r0 + i) * kHidden + 2 * c2) =
        *reinterpret_cast<const __nv_bfloat162*>(sdz + i * kSdzPitch + 2 * c2);
  }
  for (int q = tid; q < kHidden * (kHeadRows / 8); q += kHeadThreads) {
    const int k = q / (kHeadRows / 8), part = q - k * (kHeadRows / 8);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sdz[(part * 8 + e) * kSdzPitch + k];
    *reinterpret_cast<uint4*>(dZt + (size_t)k * M + r0 + part * 8) = *reinterpret_cast<const uint4*>(v);
  }
  {
    const int k = tid;
    float s = 0.0f;
    for (int i = 0; i < kHeadRows; ++i) s += __bfloat162float(sdz[i * kSdzPitch + k]);
    colpart[(size_t)blockIdx.x * kHidden + k] = s;
  }
}

// One AdamW step on one entry with gradient gi: moments m1, m2, then
// decoupled weight decay (weight matrices only) and the bias-corrected step.
__device__ __forceinline__ void adamw_math(float gi, float& m1, float& m2, float& w, bool decay, float lr, float b1,
                                           float b2, float eps, float wd, float bc1, float bc2) {
  const float a = b1 * m1 + (1.0f - b1) * gi;
  const float b = b2 * m2 + (1.0f - b2) * gi * gi;
  m1 = a;
  m2 = b;
  float wi = w;
  if (decay) wi -= lr * wd * wi;
  wi -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  w = wi;
}

// The AdamW step of flat entry i, refreshing its row-major BF16 working copy.
__device__ __forceinline__ void adamw_update(long long i, float gi, float* w, float* m1, float* m2, float lr, float b1,
                                             float b2, float eps, float wd, float bc1, float bc2, const AdamLayout& L,
                                             __nv_bfloat16* wb) {
  float a = m1[i], b = m2[i], wi = w[i];
  adamw_math(gi, a, b, wi, L.is_weight(i), lr, b1, b2, eps, wd, bc1, bc2);
  m1[i] = a;
  m2[i] = b;
  w[i] = wi;
  L.store_bf16(i, wi, wb);
}

// AdamW on the flat FP32 parameter vector with a given gradient; refreshes
// the row-major BF16 working copies (their transposes follow from
// k_transpose_layers).
__global__ void k_adamw(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                        float wd, float bc1, float bc2, const AdamLayout L, __nv_bfloat16* wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  adamw_update(i, g[i], w, m1, m2, lr, b1, b2, eps, wd, bc1, bc2, L, wb);
}

// Refresh the row-major BF16 working copies from the FP32 master parameters.
__global__ void k_pack_params(const float* w, int n, const AdamLayout L, __nv_bfloat16* wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  L.store_bf16(i, w[i], wb);
}

// Gradient assembly and, when a.adam is set, the AdamW step (see FinishArgs).
// Blocks [0, kFinishWBlocks): four consecutive hidden weight entries per
// thread (16-byte loads and stores), each summing its K-slice partials in
// slice order.  The next kFinishRBlocks blocks: 32 bias or output-layer
// entries each, eight partial sums per entry (partials j, j + 8, ...) added
// in order.  The last block: the batch
// loss (strided per thread, then a tree over the block).
constexpr int kFinishW = kLayers * kHidden * kHidden;                     // hidden weight entries
constexpr int kFinishR = kLayers * kHidden + kOut * kHidden + kOut;       // reduced entries
constexpr int kFinishWBlocks = kFinishW / 1024;
constexpr int kFinishBiasGroups = kLayers * kHidden / 32;                // hidden biases, 32 per block
constexpr int kFinishHeadWGroups = kOut * kHidden / 32;                  // output-layer weights, 32 per block
constexpr int kFinishRBlocks = kFinishBiasGroups + kFinishHeadWGroups + 1;   // + the output biases

__global__ void __launch_bounds__(256) k_grad_finish(const __grid_constant__ FinishArgs a) {
  const int tid = threadIdx.x;
  const int t = a.t_idx ? *a.t_idx : 0;            // step within a replayed sequence
  const float bc1 = a.bc_tab ? a.bc_tab[2 * t] : a.bc1;
  const float bc2 = a.bc_tab ? a.bc_tab[2 * t + 1] : a.bc2;
  if (blockIdx.x == kFinishWBlocks + kFinishRBlocks) {
    if (!a.loss) return;
    __shared__ float s[256];
    float acc = 0.0f;
    for (int i = tid; i < a.M; i += blockDim.x) acc += a.row_loss[i];
    s[tid] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (tid < w) s[tid] += s[tid + w];
      __syncthreads();
    }
    if (tid == 0) a.loss[t] = s[0];
    return;
  }
  constexpr long long kW = (long long)kHidden * kHidden;
  if (blockIdx.x < kFinishWBlocks) {
    static_assert(kW % 4 == 0 && kLayerParams % 4 == 0, "16-byte groups stay within a matrix");
    const int e = (blockIdx.x * 256 + tid) * 4;
    const int l = e / (int)kW;
    const long long r = e - (long long)l * kW;
    const float* p = a.wpart + (size_t)l * a.ksplit * kW + r;
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int s = 0; s < a.ksplit; ++s) {
      const float4 x = *reinterpret_cast<const float4*>(p + (size_t)s * kW);
      v[0] += x.x;
      v[1] += x.y;
      v[2] += x.z;
      v[3] += x.w;
    }
    const long long i = (long long)l * kLayerParams + r;
    *reinterpret_cast<float4*>(a.g + i) = make_float4(v[0], v[1], v[2], v[3]);
    if (a.adam) {
      const float4 m1 = *reinterpret_cast<const float4*>(a.m1 + i);
      const float4 m2 = *reinterpret_cast<const float4*>(a.m2 + i);
      const float4 w = *reinterpret_cast<const float4*>(a.w + i);
      float am[4] = {m1.x, m1.y, m1.z, m1.w}, av[4] = {m2.x, m2.y, m2.z, m2.w}, aw[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) adamw_math(v[j], am[j], av[j], aw[j], true, a.lr, a.b1, a.b2, a.eps, a.wd, bc1, bc2);
      *reinterpret_cast<float4*>(a.m1 + i) = make_float4(am[0], am[1], am[2], am[3]);
      *reinterpret_cast<float4*>(a.m2 + i) = make_float4(av[0], av[1], av[2], av[3]);
      *reinterpret_cast<float4*>(a.w + i) = make_float4(aw[0], aw[1], aw[2], aw[3]);
      __nv_bfloat162 b[2] = {__floats2bfloat162_rn(aw[0], aw[1]), __floats2bfloat162_rn(aw[2], aw[3])};
      *reinterpret_cast<uint2*>(a.wb + (size_t)l * kW + r) = *reinterpret_cast<const uint2*>(b);
    }
    return;
  }
  // 32 consecutive entries of one kind per block: thread (j, e) = (tid / 32,
  // tid % 32) sums partials j, j + 8, ... of entry e (a warp reads 32
  // consecutive entries of one partial row), then warp 0 adds the eight
  // group sums in order
  __shared__ float part[8][32];
  const int grp = blockIdx.x - kFinishWBlocks, j = tid >> 5, e = tid & 31;
  const float* p;
  int n, stride, cnt;
  long long i0;
  if (grp < kFinishBiasGroups) {
    const int l = grp / (kHidden / 32), c0 = (grp - l * (kHidden / 32)) * 32;
    p = a.colpart[l] + c0;
    n = a.ntiles[l];
    stride = kHidden;
    i0 = (long long)l * kLayerParams + kW + c0;
    cnt = 32;
  } else if (grp < kFinishBiasGroups + kFinishHeadWGroups) {
    const int c0 = (grp - kFinishBiasGroups) * 32;
    p = a.dWpart + c0;
    n = a.nblk;
    stride = kOut * kHidden;
    i0 = kHeadW + c0;
    cnt = 32;
  } else {
    p = a.dbpart;
    n = a.nblk;
    stride = kOut;
    i0 = kHeadB;
    cnt = kOut;
  }
  float v = 0.0f;
  if (e < cnt)
    for (int t = j; t < n; t += 8) v += p[(size_t)t * stride + e];
  part[j][e] = v;
  __syncthreads();
  if (j == 0 && e < cnt) {
    float sum = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += part[q][e];
    const long long i = i0 + e;
    a.g[i] = sum;
    if (a.adam) adamw_update(i, sum, a.w, a.m1, a.m2, a.lr, a.b1, a.b2, a.eps, a.wd, bc1, bc2, AdamLayout{}, a.wb);
  }
}

// ------------------------------------------------------------------ data
// Featurizer: resample the trace on a 1 ms grid from onset (256 points, linear
// interpolation, held after the window end) in the positive frame, position
// normalised by the amplitude (start fixation = 0, end fixation = 1) and
// velocity as 10 x the per-millisecond difference.  Output BF16 [n][512]
// and, optionally, its transpose [512][ldt].  A block of 4 warps takes 32
// saccades (a warp per saccade at a time) and stages their features in shared
// memory, then writes whole rows of X and, for each feature, the 32
// saccades' values as 64 contiguous bytes of Xt.
constexpr int kFeatRows = 32;
constexpr int kSxPitch = kIn + 2;          // BF16 elements: rows one bank apart

__global__ void __launch_bounds__(128) k_featurize(const DevSac* sacs, const float* traces, int n, __nv_bfloat16* X,
                                                   __nv_bfloat16* Xt, int ldt) {
  __shared__ __align__(16) __nv_bfloat16 sx[kFeatRows * kSxPitch];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b0 = blockIdx.x * kFeatRows;
  for (int rb = warp; rb < kFeatRows; rb += 4) {
    const int b = b0 + rb;
    if (b >= n) break;
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
      sx[rb * kSxPitch + i] = __float2bfloat16_rn(pos[j]);
      sx[rb * kSxPitch + kFeatPoints + i] = __float2bfloat16_rn(vel);
    }
  }
  __syncthreads();
  const int nr = min(kFeatRows, n - b0);
  for (int q = tid; q < nr * (kIn / 2); q += 128) {
    const int i = q / (kIn / 2), c2 = q - i * (kIn / 2);
    *reinterpret_cast<__nv_bfloat162*>(X + (size_t)(b0 + i) * kIn + 2 * c2) =
        *reinterpret_cast<const __nv_bfloat162*>(sx + i * kSxPitch + 2 * c2);
  }
  if (Xt) {
    for (int q = tid; q < kIn * (kFeatRows / 8); q += 128) {
      const int k = q / (kFeatRows / 8), part = q - k * (kFeatRows / 8);
      if (part * 8 + 8 <= nr) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sx[(part * 8 + e) * kSxPitch + k];
        *reinterpret_cast<uint4*>(Xt + (size_t)k * ldt + b0 + part * 8) = *reinterpret_cast<const uint4*>(v);
      } else {
        for (int e = 0; part * 8 + e < nr; ++e) Xt[(size_t)k * ldt + b0 + part * 8 + e] = sx[(part * 8 + e) * kSxPitch + k];
      }
    }
  }
}

// Device-side counters of a replayable training step: *p64 += by64 (the
// sample base of a data slot), *p32 += 1 (the step index).
__global__ void k_bump(long long* p64, long long by64, int* p32) {
  if (threadIdx.x == 0) {
    if (p64) *p64 += by64;
    if (p32) *p32 += 1;
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

__global__ void k_gen_desc(uint64_t seed, const long long* base_ptr, int n, const float* cal_amp, const float* cal_pulse,
                           int ncal, DevSac* sacs, float* hidden, float* target, int lcap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long g = *base_ptr + i;
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
__global__ void k_add_noise(uint64_t seed, const long long* base_ptr, const DevSac* sacs, int n, float* traces,
                            float sigma) {
  const int b = blockIdx.x;
  if (b >= n) return;
  const DevSac d = sacs[b];
  const long long g = *base_ptr + b;
  for (int k2 = threadIdx.x * 2; k2 < d.L; k2 += 2 * blockDim.x) {
    uint32_t q[4];
    philox4x32_10((uint32_t)g, (uint32_t)(g >> 32), 3u, (uint32_t)k2, (uint32_t)seed, (uint32_t)(seed >> 32), q);
    const float u1 = fmaxf(u01(q[0]), 1e-7f), u2 = u01(q[1]);
    const float rad = sqrtf(-2.0f * __logf(u1));
    traces[d.off + k2] += sigma * rad * __cosf(6.283185307f * u2);
    if (k2 + 1 < d.L) traces[d.off + k2 + 1] += sigma * rad * __sinf(6.283185307f * u2);
  }
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

// 2-D tensor map of a row-major matrix [rows][cols] (row stride in bytes),
// box box_cols x box_rows with 128-byte box rows and the 128-byte swizzle.
static bool make_map_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dt, int rows, int cols, size_t stride,
                        int box_cols, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D tensor map of a row-major BF16 matrix [rows][cols], box 64 x box_rows
// (128-byte rows, 128-byte swizzle).
static bool make_map(CUtensorMap* map, const void* base, int rows, int cols, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S, int E, int BN>
static cudaError_t gemm_attr() {
  return cudaFuncSetAttribute(k_gemm_tn<S, E, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(S, BN));
}

cudaError_t gemm_prepare() {
  cudaError_t e = gemm_attr<3, kEpiF32, 128>();
  if (e == cudaSuccess) e = gemm_attr<6, kEpiBiasGelu, 128>();
  if (e == cudaSuccess) e = gemm_attr<6, kEpiGeluBwd, 128>();
  if (e == cudaSuccess) e = gemm_attr<4, kEpiF32, 256>();
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_head_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeadSmem);
  return e;
}

cudaError_t gemm(const GemmLaunch& L, cudaStream_t st) {
  if (L.np < 1 || L.np > kMaxGroup || L.ksplit < 1 || L.M <= 0 || L.N <= 0 || L.K <= 0) return cudaErrorInvalidValue;
  if (L.M % kBM || L.N % L.bn || L.K % (L.ksplit * kBK)) return cudaErrorInvalidValue;
  // launchable (stages, epilogue, width): the epilogue's staging must fit the ring
  const int kind = (L.stages == 3 && L.epi == kEpiF32 && L.bn == 128)        ? 0
                   : (L.stages == 6 && L.epi == kEpiBiasGelu && L.bn == 128) ? 1
                   : (L.stages == 6 && L.epi == kEpiGeluBwd && L.bn == 128)  ? 2
                   : (L.stages == 4 && L.epi == kEpiF32 && L.bn == 256)      ? 3
                                                                              : -1;
  if (kind < 0) return cudaErrorInvalidValue;
  if (L.ldo % 8 || (L.epi != kEpiF32 && L.ldt % 8)) return cudaErrorInvalidValue;
  if (L.ksplit > 1 && (L.epi != kEpiF32 || L.zstride != (long long)L.M * L.ldo)) return cudaErrorInvalidValue;
  GemmMaps maps;
  memset(&maps, 0, sizeof maps);
  GemmArgs g{};
  for (int i = 0; i < L.np; ++i) {
    const GemmProblem& p = L.p[i];
    auto mis = [](const void* x) { return (reinterpret_cast<uintptr_t>(x) & 15u) != 0; };
    if (mis(p.A) || mis(p.B)) return cudaErrorInvalidValue;
    const bool f32 = L.epi == kEpiF32 || (L.epi == kEpiBiasGelu && p.out_f32);
    if (f32 && (!p.out_f32 || mis(p.out_f32))) return cudaErrorInvalidValue;
    if (L.epi != kEpiF32 && (!p.out_bf16 || mis(p.out_bf16))) return cudaErrorInvalidValue;
    if (p.out_t && mis(p.out_t)) return cudaErrorInvalidValue;
    if (L.epi == kEpiBiasGelu && !p.bias) return cudaErrorInvalidValue;
    if (L.epi == kEpiGeluBwd && (!p.zin || !p.colpart || mis(p.zin))) return cudaErrorInvalidValue;
    if (!make_map(&maps.a[i], p.A, L.M, L.K, kBM) || !make_map(&maps.b[i], p.B, L.N, L.K, L.bn)) return cudaErrorInvalidValue;
    // outputs: FP32 (K slices stacked by rows), BF16 row-major, BF16 transposed
    if (f32 && !make_map_2d(&maps.of[i], p.out_f32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, L.M * L.ksplit, L.N,
                            (size_t)L.ldo * 4, 32, kBM))
      return cudaErrorInvalidValue;
    if (L.epi != kEpiF32 && !make_map_2d(&maps.ob[i], p.out_bf16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.M, L.N,
                                         (size_t)L.ldo * 2, 64, kBM))
      return cudaErrorInvalidValue;
    if (p.out_t && !make_map_2d(&maps.ot[i], p.out_t, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.N, L.M, (size_t)L.ldt * 2, 64,
                                kBM))
      return cudaErrorInvalidValue;
    g.p[i] = p;
  }
  g.M = L.M;
  g.N = L.N;
  g.nkb = L.K / L.ksplit / kBK;
  g.ksplit = L.ksplit;
  g.ldo = L.ldo;
  g.ldt = L.ldt;
  g.zstride = L.zstride;
  g.err = L.err;
  dim3 grid(L.N / L.bn, L.M / kBM, L.np * L.ksplit);
  if (kind == 0) k_gemm_tn<3, kEpiF32, 128><<<grid, gemm_threads(3), gemm_smem(3, 128), st>>>(maps, g);
  else if (kind == 1) k_gemm_tn<6, kEpiBiasGelu, 128><<<grid, gemm_threads(6), gemm_smem(6, 128), st>>>(maps, g);
  else if (kind == 2) k_gemm_tn<6, kEpiGeluBwd, 128><<<grid, gemm_threads(6), gemm_smem(6, 128), st>>>(maps, g);
  else k_gemm_tn<4, kEpiF32, 256><<<grid, gemm_threads(4), gemm_smem(4, 256), st>>>(maps, g);
  return cudaGetLastError();
}

cudaError_t head_fwd_loss(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, int M,
                          float* Y, float* dY, float* row_loss, cudaStream_t st) {
  k_head_fwd_loss<<<(M * 32 + 255) / 256, 256, 0, st>>>(H, W5, b5, T, M, Y, dY, row_loss);
  return cudaGetLastError();
}

cudaError_t head_train(const __nv_bfloat16* H, const __nv_bfloat16* W5, const float* b5, const float* T, const float* Z,
                       int M, float* Y, float* dY, float* row_loss, __nv_bfloat16* dZ, __nv_bfloat16* dZt, float* colpart,
                       float* dWpart, float* dbpart, cudaStream_t st) {
  if (M % kHeadRows) return cudaErrorInvalidValue;
  k_head_train<<<M / kHeadRows, kHeadThreads, kHeadSmem, st>>>(H, W5, b5, T, Z, M, Y, dY, row_loss, dZ, dZt, colpart, dWpart,
                                                     dbpart);
  return cudaGetLastError();
}

cudaError_t grad_finish(const FinishArgs& a, cudaStream_t st) {
  static_assert(kFinishW % 1024 == 0 && (long long)kFinishW + kFinishR == kNumParams, "every entry once");
  static_assert(kFinishBiasGroups * 32 + kFinishHeadWGroups * 32 + kOut == kFinishR, "every reduced entry once");
  k_grad_finish<<<kFinishWBlocks + kFinishRBlocks + 1, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && a.adam) e = transpose_layers(a.wb, a.wt, st, a.t_idx);
  return e;
}

cudaError_t adam_corrections(float b1, float b2, int step, float* bc1, float* bc2) {
  // bias corrections 1 - beta^t of the FP32 betas the kernels use, formed in
  // double: in FP32 the cancellation in 1 - 0.999^t would cost up to 2^-24 /
  // (1 - 0.999^t) of relative precision (1.5e-5 at t = 2)
  *bc1 = (float)(1.0 - pow((double)b1, (double)step));
  *bc2 = (float)(1.0 - pow((double)b2, (double)step));
  return cudaSuccess;
}

cudaError_t transpose_layers(const __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st, int* step_idx) {
  k_transpose_layers<<<dim3(kHidden / 32, kHidden / 32, kLayers), dim3(32, 8), 0, st>>>(wb, wt, step_idx);
  return cudaGetLastError();
}

cudaError_t adamw(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                  float wd, int step, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t st) {
  float bc1, bc2;
  adam_corrections(b1, b2, step, &bc1, &bc2);
  k_adamw<<<(n + 255) / 256, 256, 0, st>>>(w, g, m1, m2, n, lr, b1, b2, eps, wd, bc1, bc2, L, wb);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? transpose_layers(wb, wt, st) : e;
}

cudaError_t pack_params(const float* w, int n, const AdamLayout& L, __nv_bfloat16* wb, __nv_bfloat16* wt,
                        cudaStream_t st) {
  k_pack_params<<<(n + 255) / 256, 256, 0, st>>>(w, n, L, wb);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? transpose_layers(wb, wt, st) : e;
}

cudaError_t featurize(const DevSac* sacs, const float* traces, int n, __nv_bfloat16* X, __nv_bfloat16* Xt, int ldt,
                      cudaStream_t st) {
  if (Xt && ldt % 8) return cudaErrorInvalidValue;
  k_featurize<<<(n + kFeatRows - 1) / kFeatRows, 128, 0, st>>>(sacs, traces, n, X, Xt, ldt);
  return cudaGetLastError();
}

cudaError_t bump(long long* p64, long long by64, int* p32, cudaStream_t st) {
  k_bump<<<1, 32, 0, st>>>(p64, by64, p32);
  return cudaGetLastError();
}

cudaError_t apply_centres(const float* Y, int n, float* pc, cudaStream_t st) {
  k_apply_centres<<<(n * kOut + 255) / 256, 256, 0, st>>>(Y, n, kTargetScale, pc);
  return cudaGetLastError();
}

cudaError_t gen_desc(uint64_t seed, const long long* base, int n, const float* cal_amp, const float* cal_pulse, int ncal,
                     DevSac* sacs, float* hidden, float* target, int lcap, cudaStream_t st) {
  k_gen_desc<<<(n + 127) / 128, 128, 0, st>>>(seed, base, n, cal_amp, cal_pulse, ncal, sacs, hidden, target, lcap);
  return cudaGetLastError();
}

cudaError_t add_noise(uint64_t seed, const long long* base, const DevSac* sacs, int n, float* traces, float sigma,
                      cudaStream_t st) {
  k_add_noise<<<n, 128, 0, st>>>(seed, base, sacs, n, traces, sigma);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace opmm
