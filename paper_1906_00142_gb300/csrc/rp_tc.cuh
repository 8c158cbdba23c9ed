// Fifth-generation tensor-core building blocks (sm_100-family tcgen05, inline
// PTX): tensor-memory allocation, shared-memory matrix descriptors for the
// 128-byte-swizzled K-major layout, the instruction descriptor, MMA issue and
// commit, bounded mbarrier waits and tensor-memory loads.
//
// Operand layout used throughout (SWIZZLE_128B, K-major): an R x 32 tile of
// 4-byte elements (or R x 64 of 2-byte elements) is stored as R/8 atoms of
// 8 rows x 128 bytes (1024 B, 1024-byte aligned); row r of an atom starts at
// byte 128 (r % 8), and its 16-byte chunk c is stored at chunk position
// c ^ (r % 8).  Consecutive atoms along M/N are 1024 bytes apart (the stride
// byte offset); an MMA's K slice s (32 bytes) starts 32 s bytes into the
// rows.
#pragma once
#include <stdint.h>

namespace rpk {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row r, k) of a swizzled K-major tile whose rows
// are 128 bytes (k counted in elements of `esize` bytes).
__host__ __device__ __forceinline__ uint32_t sw128_offset(int r, int k, int esize) {
  const int byte = k * esize;
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((byte >> 4) ^ (r & 7)) & 7) << 4) +
                    (byte & 15));
}

// Shared-memory matrix descriptor: start address, leading byte offset 16
// (unused by the swizzled K-major layout), stride byte offset 1024, the
// descriptor version bits of sm_100, SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator, A and B of the same format
// (kind::tf32: 2 = TF32; kind::f16: 0 = F16, 1 = BF16), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
constexpr int kFmtTF32 = 2;
constexpr int kFmtBF16 = 1;

// Tensor memory: allocation by one full warp; the address is written to
// shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor core.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] (+)= A . B^T, M x N x K with K = 8 (tf32) or 16 (bf16).
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

// Arrive on the mbarrier once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the phase with the given parity to complete; gives up after
// `limit` polls and returns false (the caller records an error and skips the
// dependent work).
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(mbar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Warp-wide load of 16 consecutive 32-bit columns of the warp's 32 lanes
// (lane field of taddr = 32 (warp % 4)); thread l receives lane l's values.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Round-to-nearest split of an FP32 value into a TF32 head and an FP32 tail
// (the tail is rounded to TF32 by the tensor core): x = hi + lo with
// |lo| <= 2^-11 |x|, so hi.hi + hi.lo + lo.hi carries ~FP32 precision.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xFFFFE000u;   // round the 13 dropped mantissa bits to nearest
  hi = __uint_as_float(u);
  lo = x - hi;
}

}  // namespace tc
}  // namespace rpk
