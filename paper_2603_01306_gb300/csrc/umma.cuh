// Inline-PTX wrappers for the 5th-generation tensor cores of sm_100-class
// GPUs (sm_103a): tensor-memory allocation, tcgen05.mma with BF16 operands
// from shared memory and an FP32 accumulator in tensor memory, completion
// through mbarriers, and tensor-memory loads for the epilogue; plus the
// shared-memory matrix descriptors of K-major swizzled tiles and the 3-D
// tensor TMA copy that fills them.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace relax {

// ------------------------------------------------------------ tensor memory
// Allocate `ncols` columns (a power of two >= 32) of the SM's tensor memory
// for this CTA; the base address is written to `dst` in shared memory.  One
// whole warp executes it.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// ordering of tcgen05 operations around thread synchronisation
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---------------------------------------------------------------------- MMA
// D[tmem] = (accumulate ? D : 0) + A * B^T, A (M x 16) and B (N x 16) BF16
// tiles in shared memory given by descriptors, D FP32 (M lanes x N columns).
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same with a collector-buffer hint for A: consecutive MMAs that read the
// same A tile keep it in the tensor core's collector instead of reading
// shared memory again.  COL 1: read A and keep it (fill); 2: use the kept A
// (use); 3: use it for the last time (lastuse); 0: no hint.  An MMA with hint
// 2 or 3 must follow, in issue order, an MMA of the same A with hint 1 or 2.
template <int COL>
__device__ __forceinline__ void umma_bf16_col(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  static_assert(COL >= 0 && COL <= 3, "collector hint");
  if constexpr (COL == 0) {
    umma_bf16(d_tmem, adesc, bdesc, idesc, accumulate);
  } else if constexpr (COL == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else if constexpr (COL == 2) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
// the mbarrier gets one arrival once every tcgen05 operation this thread has
// issued so far has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Instruction descriptor of kind::f16: BF16 A and B, both K-major, FP32 D,
// M rows (64 or 128) by N columns (a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4)                            // D format: FP32
         | (1u << 7)                          // A format: BF16
         | (1u << 10)                         // B format: BF16
         | ((uint32_t)(N >> 3) << 17)         // N / 8
         | ((uint32_t)(M >> 4) << 24);        // M / 16
}

// Shared-memory descriptor of a K-major tile whose rows are SW bytes (64 or
// 128) apart, written with the matching TMA swizzle: 8-row groups of 8*SW
// bytes follow each other (stride byte offset), the leading byte offset is
// unused for swizzled K-major tiles.  The tile must start on an 8*SW byte
// boundary; a K offset inside a row is added to the start address (16-byte
// units), the swizzle being applied by the hardware to the full address.
template <int SW>
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t saddr) {
  static_assert(SW == 64 || SW == 128, "64- or 128-byte swizzle");
  constexpr uint64_t layout = SW == 128 ? 2 : 4;   // SWIZZLE_128B / SWIZZLE_64B
  return (uint64_t)((saddr >> 4) & 0x3FFFu)         // start address
         | ((uint64_t)1 << 16)                       // leading byte offset (unused)
         | ((uint64_t)((8 * SW) >> 4) << 32)         // stride byte offset
         | ((uint64_t)1 << 46)                       // descriptor version of sm_100
         | (layout << 61);
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes (lane i of
// the warp reads TMEM lane base + i): r[j] = column col0 + j.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// the same for 16 consecutive columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 16 consecutive 32-bit columns of this warp's 32 lanes <- r
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------- TMA
// 3-D tensor box (x = K, y = row, z = plane) -> shared memory, completion on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace relax
