// dm_tc.cuh -- 5th-generation tensor core (tcgen05) building blocks for
// sm_103a: tensor-memory allocation, shared-memory matrix descriptors, the
// kind::f16 MMA with BF16 operands and FP32 accumulation, completion through
// mbarriers (bounded waits), and TMEM -> register loads.
//
// Operand tiles live in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices (8 x 8 BF16), the two core matrices of
// a 16-wide K step side by side (leading byte offset 128 B), consecutive 8-row
// groups 256 B apart (stride byte offset).  Element (row i, k) of a tile with
// K = 16 sits at byte (i / 8) * 256 + (k / 8) * 128 + (i % 8) * 16 + (k % 8) * 2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmwf {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) inside a [rows x 16] K-major tile
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor (K-major, no swizzle, version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;     // leading byte offset: next K core matrix
  d |= (uint64_t)((256u >> 4) & 0x3FFF) << 32;     // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                          // descriptor version (tcgen05)
  return d;                                        // base offset 0, no swizzle
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, dense
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                       // D format F32
         | (1u << 7)                     // A format BF16
         | (1u << 10)                    // B format BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A wait gives up after this much wall time; a normal one lasts microseconds.
constexpr uint64_t MBAR_TIMEOUT_NS = 1000000000ull;

// Bounded wait on an mbarrier phase. It gives up after MBAR_TIMEOUT_NS of wall
// time (%globaltimer, read every 16 tries), or after 1 ms once *err shows that
// another wait has already given up, so that a failure ends every CTA quickly.
// Each try suspends the thread until the phase completes or MBAR_SUSPEND_NS
// pass (the try_wait time hint), so that a waiting warp does not take issue
// slots from the warps it waits for.  2^22 tries bound it should the timer not
// advance (at least tens of milliseconds, at most about 17 s).  Returns false
// (and sets *err, when given) when it gives up.
constexpr uint32_t MBAR_SUSPEND_NS = 4000;
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase, int *err) {
  const uint32_t a = smem_u32(mbar);
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(phase), "r"(MBAR_SUSPEND_NS)
        : "memory");
    if (ok) return true;
    if ((it & 15u) == 15u) {
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) t0 = now;
      const uint64_t dt = now - t0;
      if (dt > MBAR_TIMEOUT_NS) break;
      if (err && dt > 1000000ull && *(volatile int *)err) break;
    }
  }
  if (err) atomicExch(err, 1);
  return false;
}

// Plain arrival of this thread on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Arrive on an mbarrier (count 1) and add bytes to the transaction count of its current phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completion reported to the mbarrier as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// TMEM allocation of ncols columns by one whole warp; address stored at *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread t of warp w gets row
// 32 (w % 4) + t, columns col .. col + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// split 8 FP32 values into 8 BF16 hi and 8 BF16 lo packed as 16-byte rows
// (packed conversions: two values per cvt.rn.bf16x2.f32; the widening back to
// FP32 is exact)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &h, uint32_t &l) {
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h2);
  const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  h = *reinterpret_cast<const uint32_t *>(&h2);
  l = *reinterpret_cast<const uint32_t *>(&l2);
}

__device__ __forceinline__ void split8(const float x[8], uint4 &hi, uint4 &lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split2(x[2 * i], x[2 * i + 1], h[i], l[i]);
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// split an FP32 value into BF16 hi + lo bit patterns (x ~ hi + lo to ~16 bits)
__device__ __forceinline__ void split1(float x, uint16_t &hi, uint16_t &lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = *reinterpret_cast<const uint16_t *>(&h);
  lo = *reinterpret_cast<const uint16_t *>(&l);
}

}  // namespace tc
}  // namespace dmwf
