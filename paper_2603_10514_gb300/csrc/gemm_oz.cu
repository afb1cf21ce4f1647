// gemm_oz.cu -- FP64-accurate dense products on the BF16 tensor cores by the
// Ozaki scheme (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 2012), for the filter's A*V and the
// Rayleigh-Ritz product A*Q.
//
// Slicing.  Every row m of the (stacked real) A is scaled by 2^-e_m so that its
// entries lie in (-1, 1), every column c of V by 2^-f_c, and each scaled entry
// is cut into S = 8 signed digits by rounding to nearest: x = sum_i d_i 2^{-7i}
// + O(2^-57), |d_1| <= 128, |d_i| <= 64 (i > 1).  Digits are exact in BF16.  Then
//   (A V)[m, c] = 2^{e_m + f_c} sum_{t=2}^{9} 2^{-7t} L_t[m, c],
//   L_t = sum_{i + j = t} A_i V_j        (pairs with i + j > 9 are dropped:
//                                         their weight is below 2^-63),
// 36 BF16 products per output.  Levels 2..5 carry the leading bits and must
// be summed exactly: each is an integer whose partial sum over a K chunk of
// 256 is bounded by 256 * (2 * 128 * 64 + 2 * 64 * 64) < 2^23 (level 5, the
// largest), so every partial sum is an integer FP32 represents and the tensor
// core's FP32 accumulation is exact; after every chunk the epilogue adds them, shifted
// into place, into one int64 per output, which stays exact over the whole K.
// Levels 6..9 weigh at most 2^-28 of level 2, so FP32 accumulation over the
// whole K (relative rounding 2^-24) keeps their error below 2^-52 of the
// result; they are read once at the end.  The result is A*V to within
// ~2^-53 K max|A_m.| max|V_.c| per entry, the accuracy class of an FP64 GEMM.
//
// Kernel: one CTA per 128 x 64 output tile, 320 threads:
//   warp 0     TMA producer: per 64-wide K block, the 8 V digit tiles
//              (64 x 64 BF16, one "V stage", 2 stages) and the 8 A digit
//              tiles (128 x 64 BF16) streamed through a 4-deep ring;
//   warp 1     allocates all 512 TMEM columns (8 levels x 64) and issues the
//              tcgen05.mma.kind::f16 (M 128, N 64, K 16): 144 per K block;
//   warps 2-9  epilogue: per 256-wide chunk, tcgen05.ld of levels 2..5 for 32
//              rows x 32 columns and exact int64 accumulation; at the end
//              levels 6..9, the FP64 recombination and the Chebyshev
//              three-term update.
// All mbarrier waits are bounded; on expiry the kernel records the failure in
// the device status word, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

constexpr int OZ_S = 8;          // digits per entry
constexpr int OZ_B = 7;          // bits per digit
constexpr int OZ_LEVELS = 8;     // t = 2 .. 9
constexpr int OBM = 128, OBN = 64, OBK = 64;
constexpr int OZ_CHUNK_KB = 4;   // 4 K blocks = 256 K per exact chunk (levels 2..5)
constexpr int OA_RING = 4;
constexpr int A_TILE = OBM * OBK * 2;          // 16 KB
constexpr int V_TILE = OBN * OBK * 2;          // 8 KB
constexpr int V_STAGE = OZ_S * V_TILE;         // 64 KB
constexpr int OZ_THREADS = 320;
constexpr int OZ_SMEM = 2 * V_STAGE + OA_RING * A_TILE + 1024 + 512;
constexpr long long kOzWait = 4000000000LL;

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
__device__ __forceinline__ uint64_t desc_sw128(uint32_t a) {
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OBN >> 3) << 17) |
                            ((uint32_t)(OBM >> 4) << 24);
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
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

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
                   int M, int N, int nkb_total, int kbs, int col0, const int* __restrict__ rowexp,
                   const int* __restrict__ colexp, double alpha, double beta, const double* X64,
                   double gamma, const double* Z64, double* out64, int ldo,
                   double* __restrict__ partial, DevStatus* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* vst = smem;                          // 2 V stages
  unsigned char* ast = smem + 2 * V_STAGE;            // A ring
  uint64_t* bars = (uint64_t*)(ast + OA_RING * A_TILE);
  uint64_t* vfull = bars;                             // [2]
  uint64_t* vempty = bars + 2;                        // [2]
  uint64_t* afull = bars + 4;                         // [4]
  uint64_t* aempty = bars + 8;                        // [4]
  uint64_t* cfull = bars + 12;                        // chunk accumulated in TMEM
  uint64_t* cfree = bars + 13;                        // chunk read out of TMEM
  uint32_t* tslot = (uint32_t*)(bars + 14);
  int* s_err = (int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * OBN, m0 = blockIdx.y * OBM;
  // split-K: this CTA's K blocks are [kbeg, kbeg + nkb), a whole number of exact chunks
  const int kbeg = blockIdx.z * kbs;
  const int nkb = max(0, min(kbs, nkb_total - kbeg));
  const int nchunks = (nkb + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) { bar_init(&vfull[i], 1); bar_init(&vempty[i], 1); }
    for (int i = 0; i < OA_RING; ++i) { bar_init(&afull[i], 1); bar_init(&aempty[i], 1); }
    bar_init(cfull, 1);
    bar_init(cfree, 8);  // one arrival per epilogue warp
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
    int ai = 0;
    for (int kb = 0; kb < nkb && !*(volatile int*)s_err; ++kb) {
      const int vs = kb & 1;
      const uint32_t vph = (uint32_t)((kb >> 1) & 1);
      if (!bar_wait(&vempty[vs], vph ^ 1)) { atomicOr(s_err, 1); break; }
      bar_expect(&vfull[vs], V_STAGE);
      for (int j = 0; j < OZ_S; ++j)
        tma3(vst + vs * V_STAGE + j * V_TILE, &mapV, &vfull[vs], (kbeg + kb) * OBK, col0 + n0, j);
      for (int i = 0; i < OZ_S; ++i, ++ai) {
        const int as = ai % OA_RING;
        const uint32_t aph = (uint32_t)((ai / OA_RING) & 1);
        if (!bar_wait(&aempty[as], aph ^ 1)) { atomicOr(s_err, 1); break; }
        bar_expect(&afull[as], A_TILE);
        tma3(ast + as * A_TILE, &mapA, &afull[as], (kbeg + kb) * OBK, m0, i);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // Fully unrolled: pair (i, j), level t = i + j, 4 K-steps of 16 per pair; the only
    // runtime inputs per MMA are the chunk-start / first-block flags.
    int ai = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int chunk = kb / OZ_CHUNK_KB;
      const bool chunk_start = (kb % OZ_CHUNK_KB) == 0;
      const bool first_kb = kb == 0;
      if (chunk_start && chunk > 0) {
        if (!bar_wait(cfree, (uint32_t)((chunk - 1) & 1))) { atomicOr(s_err, 2); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      const int vs = kb & 1;
      if (!bar_wait(&vfull[vs], (uint32_t)((kb >> 1) & 1))) { atomicOr(s_err, 2); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dv0 = desc_sw128(s32(vst + vs * V_STAGE));
      bool bad = false;
#pragma unroll
      for (int i = 1; i <= OZ_S; ++i) {
        const int as = ai % OA_RING;
        if (!bar_wait(&afull[as], (uint32_t)((ai / OA_RING) & 1))) { bad = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t da = desc_sw128(s32(ast + as * A_TILE));
#pragma unroll
        for (int j = 1; j <= OZ_S + 1 - i; ++j) {
          const int t = i + j;
          const uint32_t dcol = tmem + (uint32_t)((t - 2) * OBN);
          const uint64_t dv = dv0 + (uint64_t)(((j - 1) * V_TILE) >> 4);
          const bool restart_flag = (t <= 5) ? chunk_start : first_kb;
#pragma unroll
          for (int kk = 0; kk < OBK / 16; ++kk) {
            const uint64_t off = (uint64_t)((kk * 32) >> 4);
            const uint32_t acc = (i == 1 && kk == 0 && restart_flag) ? 0u : 1u;
            mma(dcol, da + off, dv + off, acc);
          }
        }
        commit(&aempty[as]);
        ++ai;
      }
      if (bad) { atomicOr(s_err, 2); break; }
      commit(&vempty[vs]);
      if ((kb % OZ_CHUNK_KB) == OZ_CHUNK_KB - 1 || kb == nkb - 1) commit(cfull);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int hc = (warp - 2) >> 2;    // column half of the 64-wide tile
    const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(hc * 32);
    long long g1[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) g1[j] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      if (!bar_wait(cfull, (uint32_t)(c & 1))) { ok = false; atomicOr(s_err, 4); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int t = 2; t <= 5; ++t) {
        uint32_t r[32];
        ld32(tbase + (uint32_t)((t - 2) * OBN), r);
        const long long sh = 1LL << (OZ_B * (5 - t));
#pragma unroll
        for (int j = 0; j < 32; ++j) g1[j] += (long long)__float2int_rz(__uint_as_float(r[j])) * sh;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0 && c + 1 < nchunks) bar_arrive(cfree);
    }
    const int r = m0 + 32 * q + lane;
    if (nkb == 0) ok = true;  // empty split: contributes zeros
    if (ok && !*(volatile int*)s_err) {
      // levels 6..9 (FP32 over the whole K), combined with level sum 2..5 in FP64
      double y[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) y[j] = 0.0;
#pragma unroll 1
      for (int t = 9; t >= 6 && nkb > 0; --t) {
        uint32_t rr[32];
        ld32(tbase + (uint32_t)((t - 2) * OBN), rr);
        const double w = ldexp(1.0, -OZ_B * (t - 5));  // relative to the 2..5 sum's unit
#pragma unroll
        for (int j = 0; j < 32; ++j) y[j] = fma((double)__uint_as_float(rr[j]), w, y[j]);
      }
      if (r < M) {
        const int er = rowexp[r];
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
          const int c = n0 + hc * 32 + j;
          if (c >= N) break;
          const int e = er + colexp[col0 + c];
          // value = 2^{e} 2^{-35} (G1 + sum_{t>=6} 2^{-7(t-5)} L_t)
          const double v0 = (nkb == 0) ? 0.0 : ldexp((double)g1[j] + y[j], e - OZ_B * 5);
          if (partial) {
            partial[(size_t)blockIdx.z * M * N + (size_t)r + (size_t)c * M] = v0;
            continue;
          }
          const size_t idx = (size_t)r + (size_t)(col0 + c) * ldo;
          double v = alpha * v0;
          if (beta != 0.0) v = fma(beta, X64[idx], v);
          if (gamma != 0.0) v = fma(gamma, Z64[idx], v);
          out64[idx] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
  if (threadIdx.x == 0 && *s_err) atomicOr(&status->timeout, *s_err);
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

__device__ __forceinline__ int exp_bound(double amax) {
  // smallest e with amax < 2^e (0 for an all-zero row/column)
  if (!(amax > 0.0)) return 0;
  int e;
  frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
  return e;
}

// Digits by rounding to nearest: d_1 in [-128, 128], d_i in [-64, 64] for i > 1 (the
// remainder after a nearest rounding is at most half a unit), all exact in BF16.  The
// slicing error is then at most 2^-57 of the row / column scale and unbiased, so it
// accumulates like a random walk over K instead of growing linearly as truncation's
// one-signed error does.
__device__ __forceinline__ void write_digits(double x, int e, __nv_bfloat16* base, size_t idx,
                                             size_t plane) {
  double r = ldexp(x, -e);  // |r| < 1, exact
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const double s = r * 128.0;
    const double d = rint(s);
    r = s - d;
    base[idx + (size_t)i * plane] = __double2bfloat16(d);
  }
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int i = 0; i < nw; ++i) m = fmax(m, red[i]);
  return m;
}

// Stacked real A (M = n or 2n): digits of row m into planes (row-major, ld kp), row
// exponent into rowexp[m].  Row m of Ahat = column m of Ahat (symmetric), read from A.
template <class T>
__global__ void __launch_bounds__(256) oz_slice_A_kernel(int n, const T* __restrict__ A, int lda,
                                                         int kp, __nv_bfloat16* planes,
                                                         size_t plane, int* rowexp) {
  __shared__ double red[8];
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
  double amax = 0.0;
  for (int k = threadIdx.x; k < M; k += 256) amax = fmax(amax, fabs(elem(k)));
  amax = block_max(amax, red);
  const int e = exp_bound(amax);
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
  __shared__ double red[8];
  const int c = c0 + blockIdx.x;
  const double* col = V64 + (size_t)c * ldi;
  double amax = 0.0;
  for (int k = threadIdx.x; k < M; k += 256) amax = fmax(amax, fabs(col[k]));
  amax = block_max(amax, red);
  const int e = exp_bound(amax);
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
  __shared__ double red[8];
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
  double amax = 0.0;
  for (int k = threadIdx.x; k < K; k += 256) amax = fmax(amax, fabs(elem(k)));
  amax = block_max(amax, red);
  const int e = exp_bound(amax);
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
  __shared__ double red[16];
  const int j = blockIdx.x;
  const int M = Sc<T>::cplx ? 2 * n : n;
  const T* col = Y + (size_t)j * ldy;
  double amax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if constexpr (Sc<T>::cplx) amax = fmax(amax, fmax(fabs(col[i].x), fabs(col[i].y)));
    else amax = fmax(amax, fabs(col[i]));
  }
  amax = block_max(amax, red);
  const int e = exp_bound(amax);
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

// 3-D BF16 map over S digit planes: {kp (contiguous), rows, S}, box {64, box_rows, 1};
// consecutive planes are plane_rows * kp elements apart (plane_rows >= rows).
int make_map3(CUtensorMap* map, const void* base, int kp, int rows, int plane_rows, int box_rows) {
  auto enc = encoder();
  if (!enc) return CHASE_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)OZ_S};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)plane_rows};
  cuuint32_t box[3] = {OBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
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
            DevStatus* dst, Scratch scr, int* launches) {
  if (N <= 0) return 0;
  CUtensorMap mA, mV;
  if (a_plane_rows < M) a_plane_rows = M;
  if (make_map3(&mA, Aplanes, kp, M, a_plane_rows, OBM) ||
      make_map3(&mV, Vplanes, kp, ncols_total, ncols_total, OBN))
    return CHASE_ERR_CUDA;
  CHASE_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      OZ_SMEM));
  const int nkb = kp / OBK;
  const int tiles = ceil_div(N, OBN) * ceil_div(M, OBM);
  // split K (in whole exact chunks) until there are about four waves of CTAs
  const int nchunks = ceil_div(nkb, OZ_CHUNK_KB);
  int S = std::max(1, std::min(nchunks, ceil_div(4 * kNumSMs, tiles)));
  while (S > 1 && (size_t)S * M * N * sizeof(double) > scr.bytes) --S;
  const int kbs = ceil_div(nchunks, S) * OZ_CHUNK_KB;
  S = ceil_div(nkb, kbs);
  double* partial = (S > 1) ? (double*)scr.ptr : nullptr;
  dim3 grid(ceil_div(N, OBN), ceil_div(M, OBM), S);
  oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, st>>>(mA, mV, M, N, nkb, kbs, col0, rowexp, colexp,
                                                    alpha, beta, X64, gamma, Z64, out64, ldo,
                                                    partial, dst);
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
