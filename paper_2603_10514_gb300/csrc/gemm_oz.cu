// gemm_oz.cu -- FP64-accurate dense products on the BF16 tensor cores by the
// Ozaki scheme (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 2012): the filter's A*V, the Rayleigh-Ritz
// product A*Q and the block products of the QR and Rayleigh-Ritz steps.
//
// Slicing.  Every row m of the (stacked real) left operand is scaled by 2^-e_m
// so that its entries lie in (-1, 1), every column c of the right operand by
// 2^-f_c, and each scaled entry is cut into S = 7 signed 8-bit digits by
// rounding to nearest: x = sum_i d_i 2^{-8i} + O(2^-57), |d_1| <= 256,
// |d_i| <= 128 (i > 1).  Then
//   (A V)[m, c] = 2^{e_m + f_c} sum_{t=2}^{8} 2^{-8t} L_t[m, c],
//   L_t = sum_{i + j = t} A_i V_j        (pairs with i + j > 8 are dropped:
//                                         their weight is below 2^-56),
// 28 BF16 products per output.  Digit i is stored pre-scaled as
// d_i 2^{-8(i-3)} (exact in BF16: an integer of at most 8 significant bits
// times a power of two), so that every pair of level t contributes
// d_i d_j 2^{-8(t-6)}: one scale per level on both operands.
//   * Levels 2..5 carry the leading bits and are summed exactly: the integer
//     L_t over a K chunk of 128 is below 128 (2^16 + 2^15) < 2^24 (level 5, the
//     largest), so the tensor core's FP32 accumulation of the scaled integers is
//     exact; after every chunk the epilogue converts them (32-bit conversions),
//     shifts them into place and adds them into one int64 per output, which
//     stays exact over the whole K.
//   * Levels 6..8 weigh at most 2^-32 of level 2; each has its own FP32
//     accumulator over the whole K, read once at the end.  One shared
//     accumulator for all three does not work: measured on GB300, adding the
//     small levels into the larger running sum loses their low bits with a
//     bias (the accumulation truncates), and the error grew linearly in K to
//     ~1e-11 relative at K = 8192; with one accumulator per level it is 5e-15.
// The result is A*V to within ~2^-53 K max|A_m.| max|V_.c| per entry, the
// accuracy class of an FP64 GEMM.
//
// Two kernels per product (oz_part_kernel), 320 threads each: a TMA producer warp,
// an MMA warp that allocates TMEM and issues tcgen05.mma.kind::f16 (M 128, K 16)
// from one thread, and 8 epilogue warps reading TMEM with tcgen05.ld.
//   * tail (levels 6..8): 128 x 128 tiles, 3 accumulators x 128 TMEM columns,
//     two 112 KB stages of all 7 A and 7 V digit tiles per 32-wide K block, 36
//     MMAs per block; K may be split freely; writes 2^{e-48} sum_t acc_t per
//     output (one FP64 slab per split).
//   * exact (levels 2..5): 128 x 64 tiles, digit planes 1..4 only (no pair of
//     these levels uses a higher digit), four 48 KB stages, 20 MMAs per block;
//     two sets of the 4 level accumulators (2 x 4 x 64 columns) so that the
//     epilogue converts one 128-wide K chunk (32-bit conversions, shifted into an
//     int64 per output) while the next accumulates; adds the tail values and
//     applies the Chebyshev three-term update (or writes split-K partials).
// Measured on GB300 (probes with the digit-pair patterns fed from shared memory):
// 48 cycles per M128 N64 K16 MMA for 7 interleaved accumulators, 32 per N64
// equivalent at N = 128 with 3 accumulators; the split runs the 18 tail pairs at
// the wider tile.
// Digit slicing is integer arithmetic on the FP64 bit patterns (FP64 issues at
// 2 per clock per SM on this part; the integer pipes at 64).
// All mbarrier waits are bounded; on expiry the kernel records the failure in
// the device status word, waits (bounded) for its copies and MMAs in flight,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

constexpr int OZ_S = 7;          // digits per entry
constexpr int OZ_B = 8;          // bits per digit
constexpr int OZ_T0 = 6;         // first tail level; digit i is stored as d_i 2^{-8(i - 3)}
constexpr int OBM = 128, OBK = 32;
constexpr int OZ_CHUNK_KB = 4;   // 4 K blocks = 128 K per exact chunk
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr long long kOzWait = 4000000000LL;
static_assert(kOzPlaneBytes == 2 * OZ_S, "workspace plane size");

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(b)), "r"(c));
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(b)) : "memory");
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
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t ph) {
  if (bar_try(b, ph)) return true;
  const long long t0 = clock64();
  while (true) {
    if (bar_try(b, ph)) return true;
    if (clock64() - t0 > kOzWait) return false;
  }
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* m, uint64_t* b, int x, int y,
                                     int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(s32(dst)),
      "l"((uint64_t)m), "r"(s32(b)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// Shared-memory matrix descriptor, K-major, 64-byte swizzle: rows of 64 bytes (32 BF16
// of K), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t a) {
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ __forceinline__ void commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   s32(b))
               : "memory");
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Level-split product: the exact levels 2..5 and the tail levels 6..8 as two
// kernels.  The tail kernel needs no per-chunk readout, so with three
// accumulators it runs 128-wide N tiles (3 x 128 TMEM columns), which the tensor
// core feeds ~1.5x faster per flop than 64-wide ones; it may split K freely and
// writes its FP64 values (one slab per split) for the exact kernel.  The exact
// kernel reads only digit planes 1..4 of each operand (no pair of levels 2..5 uses
// a higher digit), keeps two sets of its four level accumulators (2 x 4 x 64 TMEM
// columns) so that the epilogue reads one chunk while the next accumulates, and
// adds the tail values before the three-term update.
// ---------------------------------------------------------------------------
template <bool kTail>
struct PartCfg {
  static constexpr int BN = kTail ? 128 : 64;
  static constexpr int PLANES = kTail ? OZ_S : 4;          // digit planes read
  static constexpr int NST = kTail ? 2 : 4;                // stages
  static constexpr int A_T = OBM * OBK * 2;                // 8 KB
  static constexpr int V_T = BN * OBK * 2;                 // 4 or 8 KB
  static constexpr int STG = PLANES * (A_T + V_T);         // 48 or 112 KB
  static constexpr int SMEM = NST * STG + 1024 + 256;
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(OBM >> 4) << 24);
};
static_assert(PartCfg<true>::SMEM <= 232448 && PartCfg<false>::SMEM <= 232448, "shared memory");
static_assert(3 * PartCfg<true>::BN <= 512 && 2 * 4 * PartCfg<false>::BN <= 512, "TMEM");
static_assert(PartCfg<true>::STG % 1024 == 0 && PartCfg<false>::STG % 1024 == 0, "stage alignment");

__device__ __forceinline__ void mma_n(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                      uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// MMAs of one K block of the part's levels.  Accumulator of level t: tail t - 6 at
// column (t - 6) BN; exact t - 2 at column buf 4 BN + (t - 2) BN.  restart: the first
// MMA into each accumulator (pair i = 1, K-step 0) overwrites it.
template <bool kTail>
__device__ __forceinline__ void issue_part(uint32_t tmem, uint32_t buf, uint64_t da0, uint64_t dv0,
                                           bool restart) {
  using C = PartCfg<kTail>;
#pragma unroll
  for (int t = kTail ? OZ_T0 : 2; t <= (kTail ? OZ_S + 1 : OZ_T0 - 1); ++t) {
#pragma unroll
    for (int i = 1; i <= OZ_S; ++i) {
      const int j = t - i;
      if (j < 1 || j > OZ_S) continue;
      const uint32_t col = kTail ? (uint32_t)((t - OZ_T0) * C::BN)
                                 : (uint32_t)(buf * 4 * C::BN + (t - 2) * C::BN);
      const uint64_t da = da0 + (uint64_t)(((i - 1) * C::A_T) >> 4);
      const uint64_t dv = dv0 + (uint64_t)(((j - 1) * C::V_T) >> 4);
#pragma unroll
      for (int kk = 0; kk < OBK / 16; ++kk) {
        const uint64_t off = (uint64_t)((kk * 32) >> 4);
        mma_n(tmem + col, da + off, dv + off, C::IDESC, (i == 1 && kk == 0 && restart) ? 0u : 1u);
      }
    }
  }
}

// kTail: tail[z][r + c M] = 2^{e - 48} sum_{t >= 6} acc_t over this CTA's K range (z = split).
// !kTail: v = 2^{e - 40} G1 (+ sum_z tail[z] when this is split 0), then partial[z] or the
// three-term update into out64.
template <bool kTail>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_part_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                   int M, int N, int nkb_total, int kbs, int col0, const int* __restrict__ rowexp,
                   const int* __restrict__ colexp, double alpha, double beta, const double* X64,
                   double gamma, const double* Z64, double* out64, int ldo,
                   double* __restrict__ partial, double* tail, int tail_splits,
                   DevStatus* status) {
  using C = PartCfg<kTail>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + C::NST * C::STG);
  uint64_t* full = bars;                 // [NST]
  uint64_t* empty = bars + C::NST;       // [NST]
  uint64_t* cfull = bars + 2 * C::NST;   // [2] exact chunk accumulated in buffer b
  uint64_t* cfree = cfull + 2;           // [2] buffer b read out
  uint64_t* tdone = cfree + 2;           // every MMA finished
  uint32_t* tslot = (uint32_t*)(tdone + 1);
  int* s_err = (int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * C::BN, m0 = blockIdx.y * OBM;
  const int kbeg = blockIdx.z * kbs;
  const int nkb = max(0, min(kbs, nkb_total - kbeg));
  const int nchunks = (nkb + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NST; ++i) { bar_init(&full[i], 1); bar_init(&empty[i], 1); }
    for (int b = 0; b < 2; ++b) { bar_init(&cfull[b], 1); bar_init(&cfree[b], OZ_EPI_WARPS); }
    bar_init(tdone, 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(tslot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer ----------------
    int issued = 0;
    for (int kb = 0; kb < nkb && !*(volatile int*)s_err; ++kb) {
      const int s = kb % C::NST;
      if (!bar_wait(&empty[s], (uint32_t)(((kb / C::NST) & 1) ^ 1))) { atomicOr(s_err, 1); break; }
      bar_expect(&full[s], C::STG);
      unsigned char* st = smem + s * C::STG;
      const int x = (kbeg + kb) * OBK;
      for (int i = 0; i < C::PLANES; ++i) tma3(st + i * C::A_T, &mapA, &full[s], x, m0, i);
      for (int j = 0; j < C::PLANES; ++j)
        tma3(st + C::PLANES * C::A_T + j * C::V_T, &mapV, &full[s], x, col0 + n0, j);
      issued = kb + 1;
    }
    for (int b = max(0, issued - C::NST); b < issued; ++b)
      if (!bar_wait(&full[b % C::NST], (uint32_t)((b / C::NST) & 1))) atomicOr(s_err, 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool bad = false;
    for (int kb = 0; kb < nkb && !bad; ++kb) {
      const int chunk = kb / OZ_CHUNK_KB;
      const bool chunk_start = (kb % OZ_CHUNK_KB) == 0;
      const bool chunk_last = (kb % OZ_CHUNK_KB) == OZ_CHUNK_KB - 1 || kb == nkb - 1;
      const uint32_t buf = (uint32_t)(chunk & 1);
      if (!kTail && chunk_start && chunk >= 2) {
        // the epilogue has read this buffer's previous chunk (chunk - 2)
        if (!bar_wait(&cfree[buf], (uint32_t)(((chunk - 2) >> 1) & 1))) { bad = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      const int s = kb % C::NST;
      if (!bar_wait(&full[s], (uint32_t)((kb / C::NST) & 1))) { bad = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = s32(smem + s * C::STG);
      const uint64_t da0 = desc_sw64(sa), dv0 = desc_sw64(sa + C::PLANES * C::A_T);
      issue_part<kTail>(tmem, buf, da0, dv0, kTail ? (kb == 0) : chunk_start);
      if (!kTail && chunk_last) commit(&cfull[buf]);
      commit(&empty[s]);
    }
    if (bad) atomicOr(s_err, 2);
    commit(tdone);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int cg = (warp - 2) >> 2;  // column half of the tile
    const int r = m0 + 32 * q + lane;
    const int er = (r < M) ? rowexp[r] : 0;
    bool ok = true;
    if constexpr (kTail) {
      if (nkb > 0 && !__all_sync(0xffffffffu, bar_wait(tdone, 0u))) {
        ok = false;
        if (lane == 0) atomicOr(s_err, 4);
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (__shfl_sync(0xffffffffu, (int)(ok && !*(volatile int*)s_err), 0)) {
        double* tz = tail + (size_t)blockIdx.z * M * N;
#pragma unroll 1
        for (int h = 0; h < C::BN / 2 / 16; ++h) {  // 4 groups of 16 columns of this half
          const int cbase = cg * (C::BN / 2) + 16 * h;
          double y[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) y[j] = 0.0;
          if (nkb > 0) {
#pragma unroll 1
            for (int t = OZ_S + 1; t >= OZ_T0; --t) {
              uint32_t tl[16];
              ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((t - OZ_T0) * C::BN + cbase), tl);
#pragma unroll
              for (int j = 0; j < 16; ++j) y[j] += (double)__uint_as_float(tl[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = n0 + cbase + j;
            if (r < M && c < N) {
              const int e = er + colexp[col0 + c];
              tz[(size_t)r + (size_t)c * M] = ldexp(y[j], e - OZ_B * 6);  // 2^{e-40} 2^-8 sum
            }
          }
        }
      }
    } else {
      long long g1[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) g1[j] = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        const uint32_t buf = (uint32_t)(c & 1);
        if (!__all_sync(0xffffffffu, bar_wait(&cfull[buf], (uint32_t)((c >> 1) & 1)))) {
          ok = false;
          if (lane == 0) atomicOr(s_err, 4);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + buf * 4 * C::BN + (uint32_t)(cg * 32);
#pragma unroll 1
        for (int t = 2; t < OZ_T0; ++t) {
          uint32_t rr[32];
          ld32(tb + (uint32_t)((t - 2) * C::BN), rr);
          const float unscale = __int_as_float((127 - OZ_B * (OZ_T0 - t)) << 23);
#pragma unroll
          for (int j = 0; j < 32; ++j)
            g1[j] += (long long)__float2int_rz(__uint_as_float(rr[j]) * unscale) << (OZ_B * (OZ_T0 - 1 - t));
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0 && c + 2 < nchunks) bar_arrive(&cfree[buf]);
      }
      if (ok && nkb > 0 && !__all_sync(0xffffffffu, bar_wait(tdone, 0u))) {
        ok = false;
        if (lane == 0) atomicOr(s_err, 4);
      }
      if (nkb == 0) ok = true;
      if (__shfl_sync(0xffffffffu, (int)(ok && !*(volatile int*)s_err), 0) && r < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = n0 + cg * 32 + j;
          if (c < N) {
            const int e = er + colexp[col0 + c];
            double v0 = (nkb == 0) ? 0.0 : ldexp((double)g1[j], e - OZ_B * 5);
            if (blockIdx.z == 0)
              for (int z = 0; z < tail_splits; ++z) v0 += tail[(size_t)z * M * N + (size_t)r + (size_t)c * M];
            if (partial) {
              partial[(size_t)blockIdx.z * M * N + (size_t)r + (size_t)c * M] = v0;
            } else {
              const size_t idx = (size_t)r + (size_t)(col0 + c) * ldo;
              double v = alpha * v0;
              if (beta != 0.0) v = fma(beta, X64[idx], v);
              if (gamma != 0.0) v = fma(gamma, Z64[idx], v);
              out64[idx] = v;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    if (nkb > 0 && !bar_wait(tdone, 0u) && lane == 0) atomicOr(s_err, 8);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
  if (threadIdx.x == 32 && *s_err) atomicOr(&status->timeout, *s_err);
}

// Sum of the split-K partial results in a fixed order, then the three-term epilogue.
__global__ void oz_reduce_kernel(int M, int N, int S, const double* __restrict__ P, int col0,
                                 double alpha, double beta, const double* X64, double gamma,
                                 const double* Z64, double* out64, int ldo) {
  const size_t total = (size_t)M * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % M), c = (int)(t / M);
    double y = 0.0;
    for (int z = 0; z < S; ++z) y += P[(size_t)z * total + t];
    const size_t idx = (size_t)r + (size_t)(col0 + c) * ldo;
    double v = alpha * y;
    if (beta != 0.0) v = fma(beta, X64[idx], v);
    if (gamma != 0.0) v = fma(gamma, Z64[idx], v);
    out64[idx] = v;
  }
}

// ---------------- slicing ----------------

// |x| as its IEEE bit pattern: for non-negative doubles the integer order is the numeric
// order, so row / column maxima need no FP64 instructions (FP64 issues at 2 per clock per
// SM here, integer work at 64).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ int exp_bound(unsigned long long amax_bits) {
  // smallest e with amax < 2^e (0 for an all-zero row/column)
  if (amax_bits == 0) return 0;
  int e;
  frexp(__longlong_as_double((long long)amax_bits), &e);  // amax = f 2^e, f in [0.5, 1)
  return e;
}

// Digits by rounding to nearest: d_1 in [-256, 256], d_i in [-128, 128] for i > 1 (the
// remainder after a nearest rounding is at most half a unit), stored as d_i 2^{-8(i-3)},
// all exact in BF16.  The slicing error is at most 2^-57 of the row / column scale and
// unbiased, so it accumulates like a random walk over K instead of growing linearly as
// truncation's one-signed error does.
// Integer form: R = round(x 2^{56 - e}) (|R| < 2^56, from the significand and exponent
// fields), then balanced base-256 digits from the top, d = floor((R + 2^{s-1}) / 2^s),
// R -= d 2^s for s = 48, 40, ..., 8, and the last digit the remainder.
__device__ __forceinline__ void write_digits(double x, int e, __nv_bfloat16* base, size_t idx,
                                             size_t plane) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long m = bits & ((1LL << 52) - 1);
  long long R = 0;
  if (ex != 0x7FF) {
    int sh;
    if (ex == 0) {
      sh = 1 - 1075 + 56 - e;  // subnormal: x = m 2^-1074
    } else {
      m |= 1LL << 52;
      sh = ex - 1075 + 56 - e;  // x = m 2^{ex - 1075}; |x| < 2^e gives m 2^sh < 2^56
    }
    if (sh >= 0) R = m << sh;
    else if (sh > -64) R = (m + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) R = -R;
  }
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const int s = OZ_B * (OZ_S - 1 - i);
    long long d = R;
    if (s > 0) {
      d = (R + (1LL << (s - 1))) >> s;
      R -= d << s;
    }
    const float v = __int2float_rn((int)d) * __int_as_float((127 + OZ_B * (2 - i)) << 23);
    base[idx + (size_t)i * plane] = __float2bfloat16_rz(v);  // exact: 8 significant bits
  }
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wi] = v;
  __syncthreads();
  unsigned long long m = 0;
  for (int i = 0; i < nw; ++i) m = red[i] > m ? red[i] : m;
  return m;
}

// Stacked real A (M = n or 2n): digits of row m into planes (row-major, ld kp), row
// exponent into rowexp[m].  Row m of Ahat = column m of Ahat (symmetric), read from A.
template <class T>
__global__ void __launch_bounds__(256) oz_slice_A_kernel(int n, const T* __restrict__ A, int lda,
                                                         int kp, __nv_bfloat16* planes,
                                                         size_t plane, int* rowexp) {
  __shared__ unsigned long long red[8];
  const int M = Sc<T>::cplx ? 2 * n : n;
  const int m = blockIdx.x;
  const int mm = m % n;
  const bool mre = m < n;
  auto elem = [&](int k) -> double {
    if constexpr (Sc<T>::cplx) {
      const z64 a = A[(size_t)(k % n) + (size_t)mm * lda];  // A[k mod n, mm]
      const bool kre = k < n;
      return (kre == mre) ? a.x : (kre ? -a.y : a.y);
    } else {
      return A[(size_t)k + (size_t)m * lda];
    }
  };
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < M; k += 256) {
    const unsigned long long b = abs_bits(elem(k));
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) rowexp[m] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < M) ? elem(k) : 0.0;
    write_digits(x, e, planes, (size_t)m * kp + k, plane);
  }
}

// FP64 stacked block V64 (M x ncols, ld ldi): digits of column c into planes
// (column-major, ld kp; rows >= M zero), column exponent into colexp[c].
__global__ void __launch_bounds__(256) oz_slice_V_kernel(int M, int c0, const double* __restrict__ V64,
                                                         int ldi, int kp, __nv_bfloat16* planes,
                                                         size_t plane, int* colexp) {
  __shared__ unsigned long long red[8];
  const int c = c0 + blockIdx.x;
  const double* col = V64 + (size_t)c * ldi;
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < M; k += 256) {
    const unsigned long long b = abs_bits(col[k]);
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) colexp[c] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < M) ? col[k] : 0.0;
    write_digits(x, e, planes, (size_t)c * kp + k, plane);
  }
}

// Caller's block V (n x ncols, ld ldv) -> stacked FP64 (M x ncols, ld ldo).
template <class T>
__global__ void stack_V_kernel(int n, int ncols, const T* __restrict__ V, int ldv, double* V64,
                               int ldo) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t total = (size_t)M * ncols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), a = (int)(t / M);
    double x;
    if constexpr (Sc<T>::cplx) {
      const z64 v = V[(size_t)(i % n) + (size_t)a * ldv];
      x = (i < n) ? v.x : v.y;
    } else {
      x = V[(size_t)i + (size_t)a * ldv];
    }
    V64[(size_t)i + (size_t)a * ldo] = x;
  }
}

// Xt (l x n, ld ldt) is the transpose of a column-major X (n x l): row m of X is column m
// of Xt.  Digits of the rows of the stacked operator [[Xr, -Xi], [Xi, Xr]] (2n x 2l; real:
// X itself, n x l) into planes (row-major, ld kp), row exponents into rowexp.
template <class T>
__global__ void __launch_bounds__(256) oz_slice_rows_kernel(int n, int l, const T* __restrict__ Xt,
                                                            int ldt, int kp, __nv_bfloat16* planes,
                                                            size_t plane, int* rowexp) {
  __shared__ unsigned long long red[8];
  const int m = blockIdx.x;
  const int mm = Sc<T>::cplx ? (m % n) : m;
  const bool mre = !Sc<T>::cplx || m < n;
  const int K = Sc<T>::cplx ? 2 * l : l;
  const T* row = Xt + (size_t)mm * ldt;  // X[mm, 0..l)
  auto elem = [&](int k) -> double {
    if constexpr (Sc<T>::cplx) {
      const z64 x = row[k % l];
      const bool kre = k < l;
      // [[Xr, -Xi], [Xi, Xr]]
      return mre ? (kre ? x.x : -x.y) : (kre ? x.y : x.x);
    } else {
      return row[k];
    }
  };
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < K; k += 256) {
    const unsigned long long b = abs_bits(elem(k));
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) rowexp[m] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < K) ? elem(k) : 0.0;
    write_digits(x, e, planes, (size_t)m * kp + k, plane);
  }
}

// Digits of the columns of a block Y (n x q, ld ldy) in stacked form: plane column j < q
// holds [Re Y; Im Y][:, j]; with `pair` (complex only) plane column q + j holds the stacked
// -i Y[:, j] = [Im Y; -Re Y][:, j].  Then, with X's columns as the left operand's rows,
// Xhat^T [Yhat | stack(-i Y)] = [Re(X^H Y) | Im(X^H Y)].  Both columns of a pair share the
// exponent of Y[:, j].  Planes column-major (ld kp; rows >= M are zero).
template <class T>
__global__ void __launch_bounds__(512) oz_slice_cols_kernel(int n, int q, const T* __restrict__ Y,
                                                            int ldy, int kp, bool pair,
                                                            __nv_bfloat16* planes, size_t plane,
                                                            int* colexp) {
  __shared__ unsigned long long red[16];
  const int j = blockIdx.x;
  const int M = Sc<T>::cplx ? 2 * n : n;
  const T* col = Y + (size_t)j * ldy;
  unsigned long long amax = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    unsigned long long b;
    if constexpr (Sc<T>::cplx) {
      const unsigned long long b0 = abs_bits(col[i].x), b1 = abs_bits(col[i].y);
      b = b0 > b1 ? b0 : b1;
    } else {
      b = abs_bits(col[i]);
    }
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) {
    colexp[j] = e;
    if (pair) colexp[q + j] = e;
  }
  for (int k = threadIdx.x; k < kp; k += blockDim.x) {
    double x = 0.0, y = 0.0;
    if (k < M) {
      if constexpr (Sc<T>::cplx) {
        const z64 v = col[k % n];
        x = (k < n) ? v.x : v.y;
        y = (k < n) ? v.y : -v.x;
      } else {
        x = col[k];
      }
    }
    write_digits(x, e, planes, (size_t)j * kp + k, plane);
    if (pair) write_digits(y, e, planes, (size_t)(q + j) * kp + k, plane);
  }
}

// out (l x 2l FP64, ld ldo) -> G (l x l, ld ldg) with G = out[:, :l] + i out[:, l:] (real: copy)
template <class T>
__global__ void gram_assemble_kernel(int l, const double* __restrict__ out, int ldo, T* G, int ldg) {
  const size_t total = (size_t)l * l;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(t % l), q = (int)(t / l);
    if constexpr (Sc<T>::cplx) {
      G[(size_t)p + (size_t)q * ldg] = z64{out[(size_t)p + (size_t)q * ldo], out[(size_t)p + (size_t)(q + l) * ldo]};
    } else {
      G[(size_t)p + (size_t)q * ldg] = out[(size_t)p + (size_t)q * ldo];
    }
  }
}

// Xt = X^T (plain transpose, no conjugation): X n x l (ld ldx) -> Xt l x n (ld ldt).
template <class T>
__global__ void transpose_kernel(int n, int l, const T* __restrict__ X, int ldx, T* Xt, int ldt) {
  __shared__ T tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + threadIdx.x, j = j0 + r;
    if (i < n && j < l) tile[r][threadIdx.x] = X[(size_t)i + (size_t)j * ldx];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + threadIdx.x, i = i0 + r;
    if (i < n && j < l) Xt[(size_t)j + (size_t)i * ldt] = tile[threadIdx.x][r];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 3-D BF16 map over S digit planes: {kp (contiguous), rows, S}, box {32, box_rows, 1};
// consecutive planes are plane_rows * kp elements apart (plane_rows >= rows).
int make_map3(CUtensorMap* map, const void* base, int kp, int rows, int plane_rows, int box_rows) {
  auto enc = encoder();
  if (!enc) return CHASE_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)OZ_S};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)plane_rows};
  cuuint32_t box[3] = {OBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : CHASE_ERR_CUDA;
}

}  // namespace

size_t oz_plane_elems(int rows, int kp) { return (size_t)rows * kp; }

template <class T>
int oz_slice_A(cudaStream_t st, int n, const T* A, int lda, int kp, void* planes, int* rowexp,
               int* launches) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  oz_slice_A_kernel<T><<<M, 256, 0, st>>>(n, A, lda, kp, (__nv_bfloat16*)planes,
                                          (size_t)M * kp, rowexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

int oz_slice_V(cudaStream_t st, int M, int c0, int c1, const double* V64, int ldi, int kp,
               int ncols_total, void* planes, int* colexp, int* launches) {
  if (c1 <= c0) return 0;
  oz_slice_V_kernel<<<c1 - c0, 256, 0, st>>>(M, c0, V64, ldi, kp, (__nv_bfloat16*)planes,
                                             (size_t)ncols_total * kp, colexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

int oz_gemm(cudaStream_t st, int M, int kp, const void* Aplanes, const int* rowexp,
            int a_plane_rows, const void* Vplanes, const int* colexp, int ncols_total, int col0, int N, double alpha,
            double beta, const double* X64, double gamma, const double* Z64, double* out64, int ldo,
            DevStatus* dst, Scratch scr, Scratch tailbuf, int* launches) {
  if (N <= 0) return 0;
  CUtensorMap mA, mV64, mV128;
  if (a_plane_rows < M) a_plane_rows = M;
  if (make_map3(&mA, Aplanes, kp, M, a_plane_rows, OBM) ||
      make_map3(&mV64, Vplanes, kp, ncols_total, ncols_total, PartCfg<false>::BN) ||
      make_map3(&mV128, Vplanes, kp, ncols_total, ncols_total, PartCfg<true>::BN))
    return CHASE_ERR_CUDA;
  CHASE_CUDA_TRY(cudaFuncSetAttribute(oz_part_kernel<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PartCfg<true>::SMEM));
  CHASE_CUDA_TRY(cudaFuncSetAttribute(oz_part_kernel<false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PartCfg<false>::SMEM));
  const int nkb = kp / OBK;
  const size_t slab = (size_t)M * N * sizeof(double);
  if (slab > tailbuf.bytes) return CHASE_ERR_OOM;
  // tail levels: split K freely (no exact chunks) up to about four waves of CTAs, one
  // slab of FP64 values per split
  const int tiles_t = ceil_div(N, PartCfg<true>::BN) * ceil_div(M, OBM);
  int St = std::max(1, std::min(nkb, ceil_div(4 * kNumSMs, tiles_t)));
  while (St > 1 && (size_t)St * slab > tailbuf.bytes) --St;
  const int kbs_t = ceil_div(nkb, St);
  St = ceil_div(nkb, kbs_t);
  double* tail = (double*)tailbuf.ptr;
  dim3 grid_t(ceil_div(N, PartCfg<true>::BN), ceil_div(M, OBM), St);
  oz_part_kernel<true><<<grid_t, OZ_THREADS, PartCfg<true>::SMEM, st>>>(
      mA, mV128, M, N, nkb, kbs_t, col0, rowexp, colexp, 0.0, 0.0, nullptr, 0.0, nullptr, nullptr, 0,
      nullptr, tail, 0, dst);
  if (launches) ++*launches;
  // exact levels: split K in whole chunks until there are about four waves of CTAs
  const int tiles = ceil_div(N, PartCfg<false>::BN) * ceil_div(M, OBM);
  const int nchunks = ceil_div(nkb, OZ_CHUNK_KB);
  int S = std::max(1, std::min(nchunks, ceil_div(4 * kNumSMs, tiles)));
  while (S > 1 && (size_t)S * slab > scr.bytes) --S;
  const int kbs = ceil_div(nchunks, S) * OZ_CHUNK_KB;
  S = ceil_div(nkb, kbs);
  double* partial = (S > 1) ? (double*)scr.ptr : nullptr;
  dim3 grid(ceil_div(N, PartCfg<false>::BN), ceil_div(M, OBM), S);
  oz_part_kernel<false><<<grid, OZ_THREADS, PartCfg<false>::SMEM, st>>>(
      mA, mV64, M, N, nkb, kbs, col0, rowexp, colexp, alpha, beta, X64, gamma, Z64, out64, ldo,
      partial, tail, St, dst);
  if (launches) ++*launches;
  if (S > 1) {
    const size_t total = (size_t)M * N;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)kNumSMs * 16);
    oz_reduce_kernel<<<blocks, 256, 0, st>>>(M, N, S, partial, col0, alpha, beta, X64, gamma, Z64,
                                             out64, ldo);
    if (launches) ++*launches;
  }
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_stack_V(cudaStream_t st, int n, int ncols, const T* V, int ldv, double* V64, int ldo,
               int* launches) {
  if (ncols <= 0) return 0;
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t work = (size_t)M * ncols;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((work + 255) / 256, (size_t)kNumSMs * 16));
  stack_V_kernel<T><<<blocks, 256, 0, st>>>(n, ncols, V, ldv, V64, ldo);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_slice_rows(cudaStream_t st, int n, int l, const T* Xt, int ldt, int kp, void* planes,
                  int* rowexp, int* launches) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  oz_slice_rows_kernel<T><<<M, 256, 0, st>>>(n, l, Xt, ldt, kp, (__nv_bfloat16*)planes,
                                             (size_t)M * kp, rowexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_slice_cols(cudaStream_t st, int n, int q, const T* Y, int ldy, int kp, bool pair,
                  void* planes, int* colexp, int* launches) {
  if (q <= 0) return 0;
  pair = pair && Sc<T>::cplx;
  const size_t ncols_total = pair ? 2 * (size_t)q : (size_t)q;
  oz_slice_cols_kernel<T><<<q, 512, 0, st>>>(n, q, Y, ldy, kp, pair, (__nv_bfloat16*)planes,
                                             ncols_total * kp, colexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_gram_assemble(cudaStream_t st, int l, const double* out, int ldo, T* G, int ldg, int* launches) {
  const size_t work = (size_t)l * l;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((work + 255) / 256, (size_t)kNumSMs * 16));
  gram_assemble_kernel<T><<<blocks, 256, 0, st>>>(l, out, ldo, G, ldg);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int transpose(cudaStream_t st, int n, int l, const T* X, int ldx, T* Xt, int ldt, int* launches) {
  dim3 grid(ceil_div(n, 32), ceil_div(l, 32)), block(32, 8);
  transpose_kernel<T><<<grid, block, 0, st>>>(n, l, X, ldx, Xt, ldt);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

#define OZ_INST(T)                                                                                \
  template int oz_slice_rows<T>(cudaStream_t, int, int, const T*, int, int, void*, int*, int*);   \
  template int oz_slice_cols<T>(cudaStream_t, int, int, const T*, int, int, bool, void*, int*,   \
                                int*);                                                            \
  template int oz_gram_assemble<T>(cudaStream_t, int, const double*, int, T*, int, int*);         \
  template int transpose<T>(cudaStream_t, int, int, const T*, int, T*, int, int*);
OZ_INST(double)
OZ_INST(z64)
#undef OZ_INST

template int oz_stack_V<double>(cudaStream_t, int, int, const double*, int, double*, int, int*);
template int oz_stack_V<z64>(cudaStream_t, int, int, const z64*, int, double*, int, int*);
template int oz_slice_A<double>(cudaStream_t, int, const double*, int, int, void*, int*, int*);
template int oz_slice_A<z64>(cudaStream_t, int, const z64*, int, int, void*, int*, int*);

}  // namespace chase
