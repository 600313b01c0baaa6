// Blackwell (sm_103a) tensor-core building blocks, written as inline PTX:
// tensor-memory allocation, shared-memory operand descriptors, the tf32 MMA
// with FP32 accumulation in tensor memory, its completion through an
// mbarrier, and the load of the accumulator back into registers.
//
// Operands are staged by the CTA's threads in shared memory in the
// no-swizzle K-major canonical layout: "core matrices" of 8 rows x 16 bytes
// (4 tf32 values per row), element (row m, k) of a tile at byte
//   (m / 8) * SBO + (k / 4) * LBO + (m % 8) * 16 + (k % 4) * 4,
// LBO = 128 (next core matrix along K), SBO = 128 * K / 4 (next 8 rows).
// One MMA consumes K = 8 (two core matrices along K); the k-th step of a
// tile starts 2 * LBO * k bytes further.
//
// Every wait is bounded: a wait that gives up records where in a device
// error word and the kernel finishes without touching the result.
#pragma once
#include <cstdint>

namespace hz {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tf32 value of x rounded to nearest (ties away), as an fp32 bit pattern
// whose 13 low mantissa bits are zero: what the tensor core reads exactly
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (m, k) in a K-major no-swizzle tile with K columns
template <int K>
__device__ __forceinline__ int kmajor_offset(int m, int k) {
  return (m >> 3) * (128 * K / 4) + (k >> 2) * 128 + (m & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor (K-major, no swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);            // bits 0-13: start address
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;       // bits 16-29: leading byte offset
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;       // bits 32-45: stride byte offset
  d |= (uint64_t)1 << 46;                            // bits 46-47: descriptor version
  return d;                                          // base offset 0, no swizzle
}

// instruction descriptor of kind::tf32, FP32 accumulator, A and B K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                     // D format: F32
         | (2u << 7)                   // A format: TF32
         | (2u << 10)                  // B format: TF32
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24); // M / 16
}

// tensor-memory allocation of `cols` columns by one whole warp; the address
// is written to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// D (+)= A * B, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// the MMAs this thread issued so far arrive on the mbarrier when complete
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// wait until the phase of the given parity completes; false after `limit`
// polls (the caller records the failure)
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(mbar);
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// one arrival on the mbarrier that also announces `bytes` of asynchronous
// copies the phase must wait for
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}

// bulk copy (the TMA's non-tensor form) of `bytes` from global to shared
// memory, counted against the mbarrier's transaction bytes; both addresses
// 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// generic-proxy writes to shared memory made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's lane (warp w of a
// 4-warp group reads lanes 32w .. 32w + 31; taddr carries lane and column)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace hz
