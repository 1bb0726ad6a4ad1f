// tcgen05 building blocks (sm_100 family, inline PTX) shared by the tensor-core kernels: FP32 values
// split into two TF32 parts, shared-memory matrix descriptors of K-major operands without swizzle,
// the kind::tf32 instruction descriptor, bounded mbarrier waits, TMEM allocation, MMA issue, commit
// and the 32x32b accumulator loads with TwoSum accumulation into registers.
//
// Operand layout (K-major, no swizzle): core matrices of 8 rows x 16 bytes (4 TF32 values along K),
// rows 16 B apart inside a core matrix; K-adjacent core matrices LBO = 128 B apart, 8-row groups
// SBO = (K per stage / 4) x 128 B apart. One MMA k-step (K = 8) covers two K-adjacent core matrices.
#pragma once

#include <stdint.h>

namespace pk {
namespace tc {

// x = big + small: big is x rounded to TF32 (ties away from zero), small = x - big is exact in FP32.
// Three products big.big + big.small + small.big then err by about 3 x 2^-22 of |a b|.
__device__ __forceinline__ void split(float x, float& big, float& small) {
  big = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  small = x - big;
}

// Byte offset of element (row, k) in a K-major operand holding kk values of K per row.
__device__ __forceinline__ uint32_t off(int row, int k, int kk) {
  return uint32_t(((row >> 3) * (kk / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shared-memory descriptor: start address, LBO = 128 B, SBO, version 1 (sm_100 family), no swizzle.
// A k-step advances the start address by 256 B, i.e. adds 16 to the descriptor.
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFF) | (uint64_t((128u >> 4) & 0x3FFF) << 16) | (uint64_t((sbo >> 4) & 0x3FFF) << 32) |
         (uint64_t(1) << 46);
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, N and M.
__host__ __device__ constexpr uint32_t idesc_tf32(int n, int m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of the given parity of the mbarrier at shared address bar, at most limit_ns.
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp-wide: allocates ncols TMEM columns, the address written to shared memory at slot.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A B (+ D when accumulate), single issuing thread.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d), "l"(a),
      "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier at bar completes a phase when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes, added to TwoSum pairs (hi, lo).
__device__ __forceinline__ void read_acc16(uint32_t taddr, float (&hi)[16], float (&lo)[16]) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float x = __uint_as_float(v[j]);
    const float sum = __fadd_rn(hi[j], x);
    const float bb = __fsub_rn(sum, hi[j]);
    lo[j] = __fadd_rn(lo[j], __fadd_rn(__fsub_rn(hi[j], __fsub_rn(sum, bb)), __fsub_rn(x, bb)));
    hi[j] = sum;
  }
}

}  // namespace tc
}  // namespace pk
