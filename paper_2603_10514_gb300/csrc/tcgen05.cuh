// tcgen05.cuh -- device helpers shared by the tensor-core kernels (gemm_oz.cu, gemm_tc.cu):
// mbarrier waits (all bounded), cluster / CTA-pair addressing, TMA tile loads whose
// completion counts on a barrier of either CTA of a pair, shared-memory matrix descriptors,
// the CTA-pair tcgen05 MMA and commit, and the TMEM load.  Inline PTX for sm_103a.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace chase {
namespace tc {

constexpr long long kTcWait = 4000000000LL;  // ~2 s of clock64 per bounded wait

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(b)), "r"(c));
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t ph) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s32(b)), "r"(ph)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t ph) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s32(b)), "r"(ph)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t ph) {
  if (bar_try(b, ph)) return true;
  const long long t0 = clock64();
  while (true) {
    if (bar_try(b, ph)) return true;
    if (clock64() - t0 > kTcWait) return false;
  }
}
// bounded wait that never suspends the thread (the MMA issuer: data is usually there)
__device__ __forceinline__ bool bar_poll(uint64_t* b, uint32_t ph) {
  if (bar_test(b, ph)) return true;
  const long long t0 = clock64();
  while (true) {
    if (bar_test(b, ph)) return true;
    if (clock64() - t0 > kTcWait) return false;
  }
}
// The same shared-memory offset in CTA `rank` of the cluster, as a shared::cluster address.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(s32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void arrive_remote(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster_addr)
               : "memory");
}
// TMA tile load into this CTA's shared memory whose completion is counted on a barrier of
// either CTA of the pair (given as a shared::cluster address).
__device__ __forceinline__ void tma3_pair(void* dst, const CUtensorMap* m, uint32_t bar_cluster_addr,
                                          int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(s32(dst)),
      "l"((uint64_t)m), "r"(bar_cluster_addr), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// 2-D form of tma3_pair (maps {K, rows}).
__device__ __forceinline__ void tma2_pair(void* dst, const CUtensorMap* m, uint32_t bar_cluster_addr,
                                          int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(s32(dst)),
      "l"((uint64_t)m), "r"(bar_cluster_addr), "r"(x), "r"(y)
      : "memory");
}
// Shared-memory matrix descriptor, K-major, 128-byte swizzle: rows of 128 bytes (64 BF16
// of K), 8-row groups 1024 bytes apart.  The K16 step k of a block starts 32 k bytes in.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t a) {
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Arrive on the barrier at this offset in both CTAs of the pair once the pair's MMAs issued
// so far have completed.
__device__ __forceinline__ void commit_pair(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(s32(b)),
      "h"((uint16_t)3)
      : "memory");
}
// D[256 x N] (+)= A[256 x 16] B[16 x N] over a CTA pair: rows 0-127 of A and D in the
// even CTA (the issuer), rows 128-255 in the odd one; B's first N/2 rows (K-major) in the
// even CTA, the rest in the odd one, at the same shared-memory offsets.
__device__ __forceinline__ void mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}


}  // namespace tc
}  // namespace chase
