// common.cuh -- device helpers shared by the OPMM kernels: batch descriptors,
// Philox4x32-10, TMA bulk copies with bounded mbarrier waits, error flags.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace opmm {

// Error bits a kernel may raise in the context's device error word.
enum : unsigned {
  kErrWaitTimeout = 1u << 0,   // a bounded mbarrier wait gave up
  kErrBadShape = 1u << 1,      // a trace longer than the staged buffer
};

// Device copy of one staged saccade (positive frame: th0 <= thf).
struct DevSac {
  long long off;     // first sample in the packed trace buffer (multiple of 4)
  int L;             // samples
  int onset;         // onset sample
  int nsub;          // RK4 substeps per sample
  float fs;          // Hz
  float h;           // RK4 step, s
  float th0, thf;    // fixations in the positive frame
  float sign;        // +1, or -1 for a mirrored (negative-going) saccade
  float dur_ms;      // detected saccade duration (sets the nominal pulse width)
};

// Table 1 (Sec. 2.2.1): 18-parameter defaults in the OPC order of Fig. 4.
// The pulse width entry is filled from the saccade duration (W = D - 6 ms).
static __constant__ const float kTable1[18] = {
    2.5f, 2.5f, 1.2f, 1.2f, 0.8f, 0.5f, 0.06f, 0.046f, 0.022f, 0.000043f,
    11.7f, 2.4f, 2.0f, 1.9f, 14.0f, 55.0f, 0.5f, 0.0f};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32 multiplies,
// Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ---------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk (non-tensor) TMA copy global -> shared, completion on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for the phase with the given parity to complete; gives up after
// max_tries polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_tries) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < max_tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

constexpr uint32_t kMaxWaitTries = 1u << 22;

__device__ __forceinline__ void raise_error(unsigned* err, unsigned bits) {
  if (err) atomicOr(err, bits);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace opmm
