// tcgen05 / TMA / mbarrier building blocks shared by the tensor-core kernels
// (inline PTX for sm_103a).
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace dsrg {

constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // bound of every device-side wait

// The first TAIL_Q auxiliary functions (with decaying factors the largest
// terms) are contracted on CUDA cores in FP32 with round-to-nearest; the
// tensor cores, whose FP32 accumulator truncates toward zero at every
// instruction, take Q >= TAIL_Q.
constexpr int TAIL_Q = 32;
constexpr int TAIL_PAD = 256;  // zero rows after the last plane row of the FP32 tail rows

// ------------------------------- PTX helpers -------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on phase `parity`; false if it ran out or another role aborted.
static __device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                       int* status) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > TC_WAIT_NS) {
      *abort_flag = 1;
      atomicExch(status, 1);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(su32(dst)),
      "l"((unsigned long long)map), "r"(su32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
// Bring a box of the tensor into L2 ahead of its load (no shared-memory write).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int c0, int c1) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   (unsigned long long)map),
               "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
// One MMA D (+)= A·B. COL selects the A-operand collector buffer: 0 reads A from
// shared memory and keeps nothing, 1 reads it and keeps it (fill), 2 takes the
// A kept by the previous MMA of this thread, which must have had the same
// descriptor, and releases it (lastuse). Reusing A saves one shared-memory
// read of the A tile.
template <bool BF16, int COL = 0>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
#define DSRG_MMA(KIND, CU)                                                                   \
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"                               \
               " tcgen05.mma.cta_group::1.kind::" KIND CU " [%0], %1, %2, %3, p;\n}\n" ::"r"(d), \
               "l"(a), "l"(b), "r"(idesc), "r"(acc)                                          \
               : "memory")
  if (BF16) {
    if (COL == 1) DSRG_MMA("f16", ".collector::a::fill");
    else if (COL == 2) DSRG_MMA("f16", ".collector::a::lastuse");
    else DSRG_MMA("f16", "");
  } else {
    if (COL == 1) DSRG_MMA("tf32", ".collector::a::fill");
    else if (COL == 2) DSRG_MMA("tf32", ".collector::a::lastuse");
    else DSRG_MMA("tf32", "");
  }
#undef DSRG_MMA
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void named_bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Eight consecutive floats from global memory, read-only path (32-byte aligned).
__device__ __forceinline__ void ldg8(const float* p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "l"(p));
}

// x_ab += sum_{q < TAIL_Q} T_a[q] T_b[q] for the 16 columns b of one chunk, in
// FP32 with round-to-nearest, q from the last to the first. T holds fl32(B) of
// the first TAIL_Q auxiliary functions, one 128-byte row per plane row; `ra` is
// this thread's row, `rb` the first of the chunk's 16 rows (the same for every
// lane of the warp, so each load is a broadcast; 32-byte loads halve their count).
__device__ __forceinline__ void tail_add16(const float* __restrict__ ra,
                                           const float* __restrict__ rb, uint32_t (&r)[16]) {
  float t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = 0.f;
#pragma unroll 1
  for (int q8 = TAIL_Q / 8 - 1; q8 >= 0; --q8) {
    float a[8];
    ldg8(ra + 8 * q8, a);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float b[8];
      ldg8(rb + k * TAIL_Q + 8 * q8, b);
#pragma unroll
      for (int i = 7; i >= 0; --i) t[k] = fmaf(a[i], b[i], t[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) r[k] = __float_as_uint(__uint_as_float(r[k]) + t[k]);
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows at a
// 64-byte pitch (8-row groups 512 bytes apart).
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;           // descriptor version of tcgen05
  d |= (uint64_t)4 << 61;           // 64-byte swizzle
  return d;
}
// Shared-memory matrix descriptor: K-major operand, 32-byte swizzle, rows at a
// 32-byte pitch (8-row groups 256 bytes apart); one MMA K step per row.
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(256 >> 4) << 32;  // stride byte offset: 8 rows x 32 B
  d |= (uint64_t)1 << 46;           // descriptor version of tcgen05
  d |= (uint64_t)6 << 61;           // 32-byte swizzle
  return d;
}
// Instruction descriptor: D = F32, A/B = TF32 (2) or BF16 (1), both K-major, M = 128, N given
// (a multiple of 16, 16..256).
template <bool BF16>
__host__ __device__ constexpr uint32_t idesc_128xn(uint32_t n) {
  return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) | ((n >> 3) << 17) |
         ((128u >> 4) << 24);
}
// Instruction descriptor: D = F32, A/B = TF32 (2) or BF16 (1), both K-major, M = N = 128.
template <bool BF16>
__host__ __device__ constexpr uint32_t idesc_128x128() {
  return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) | ((128u >> 3) << 17) |
         ((128u >> 4) << 24);
}

}  // namespace dsrg
