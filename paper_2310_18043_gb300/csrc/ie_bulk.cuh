// Device helpers shared by the band-solve kernels: shared-memory addresses, mbarriers,
// bulk (TMA 1D) global-to-shared copies with bounded completion waits, and complex64
// arithmetic (the complex128 versions live in ie_internal.cuh).
#pragma once

#include "ie_internal.cuh"

namespace iebulk {
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the warp is suspended (it issues nothing) until the phase
// completes or about hint_ns nanoseconds have passed, instead of returning at once and
// spinning, which takes issue slots from the warps that do the work
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity,
                                                    uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
constexpr uint32_t IE_SUSPEND_NS = 20000;   // one suspended try_wait lasts at most ~20 us
// bounded wait: false after IE_WAIT_NS (the clock is read only once the first suspended wait
// has run out)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait_sleep(bar, parity, IE_SUSPEND_NS)) return true;
  const unsigned long long t0 = ie_globaltimer();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, IE_SUSPEND_NS)) return true;
    if (ie_globaltimer() - t0 > IE_WAIT_NS) return false;
  }
}

// complex64: c - a*b, c + a*b, c - conj(a)*b, c + conj(a)*b
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfms_conj(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
// complex128: c - conj(a)*b
__device__ __forceinline__ double2 cfms_conj(double2 a, double2 b, double2 c) {
  return make_double2(fma(-a.x, b.x, fma(-a.y, b.y, c.x)), fma(-a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }

// The short dense products of a panel -- H <- T H over the 16 members (forward) and
// x_head = inv(U_block) h_head over the NB head rows (backward) -- are summed in four fixed
// partial ranges (members 4g..4g+3, head rows 2g..2g+1), then the partials are added in a
// fixed order. The synchronised kernels compute the four partials on four different warps in FP64
// (one per SM sub-partition), one thread computes all four otherwise; the order of every
// floating-point operation is the same either way, so every launch shape gives identical
// results. (The conjugate-transpose solve uses the same split for its U^H head block.)
constexpr int NPART = 4;
template <typename CT>
__device__ __forceinline__ CT sum_parts(const CT* part, int stride, int o) {
  CT s = part[o];
#pragma unroll
  for (int g = 1; g < NPART; ++g) {
    const CT x = part[g * stride + o];
    s.x += x.x;
    s.y += x.y;
  }
  return s;
}

}  // namespace iebulk
