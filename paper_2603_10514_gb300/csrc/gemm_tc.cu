// gemm_tc.cu -- the filter's A*V product on the 5th-generation tensor cores
// (tcgen05 + TMEM + TMA) in split BF16 precision, for the mixed-precision
// filter (BF16x3: three BF16 products with FP32 accumulation).
//
//   Y = Ah*Vh + Ah*Vl + Al*Vh        (hi/lo BF16 splits of A and V, FP32 in TMEM)
//   out64 = alpha*Y + beta*X64 + gamma*Z64          (FP64 epilogue, in place allowed)
//   next_h/next_l = BF16 hi/lo split of out64       (B operand of the next step)
//
// Operands are "stacked real": a complex Hermitian A of order n becomes the
// real symmetric 2n x 2n matrix [[Re A, -Im A], [Im A, Re A]] and a complex
// block V becomes [Re V; Im V], so one real product gives [Re AV; Im AV].
// Storage: A planes row-major with K contiguous (leading dimension kp, a
// multiple of 64 elements, zero padded); V planes column-major with K
// contiguous (same kp); FP64 blocks column-major with leading dimension ldv.
//
// One CTA computes one 128 x 128 output tile; 256 threads in four roles:
//   warp 0      TMA producer: 4 tiles (Ah, Al, Vh, Vl; 64 x 128 BF16 each,
//               128-byte swizzle) per 64-wide K block into a 3-stage ring;
//   warp 1      allocates 128 TMEM columns; one thread issues
//               tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 128, K = 16),
//               12 per K block, and commits each stage back to the producer;
//   warps 4..7  epilogue: tcgen05.ld of its 32 TMEM lanes (tile rows), FP64
//               three-term update, BF16 split of the result.
// Every mbarrier wait is bounded (~2 s of clock64); on expiry the kernel sets
// a flag in the device status word, drains, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

constexpr int TBM = 128;
constexpr int TBN = 128;
constexpr int TBK = 64;  // 64 BF16 = one 128-byte swizzle row
constexpr int TSTAGES = 3;
constexpr int TILE_BYTES = TBM * TBK * 2;            // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;          // Ah, Al, Vh, Vl
constexpr int TC_THREADS = 256;
constexpr int TC_SMEM = TSTAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false if the phase did not complete within kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile whose rows are 128 bytes,
// 128-byte swizzle, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;               // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // SBO
  d |= (uint64_t)1 << 46;               // version
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
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
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_filter_bf16x3_kernel(const __grid_constant__ CUtensorMap mapAh,
                            const __grid_constant__ CUtensorMap mapAl,
                            const __grid_constant__ CUtensorMap mapVh,
                            const __grid_constant__ CUtensorMap mapVl, int M, int N, int nkb,
                            int col0, double alpha, double beta, const double* X64, double gamma,
                            const double* Z64, double* out64, int ldv, __nv_bfloat16* next_h,
                            __nv_bfloat16* next_l, int kp, DevStatus* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TSTAGES * STAGE_BYTES);
  uint64_t* empty = full + TSTAGES;
  uint64_t* tmem_full = empty + TSTAGES;
  uint32_t* tmem_slot = (uint32_t*)(tmem_full + 1);
  int* s_err = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * TBN, m0 = blockIdx.y * TBM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tmem_full, 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TSTAGES;
      const uint32_t ph = (uint32_t)((kb / TSTAGES) & 1);
      if (!mbar_wait(&empty[s], ph ^ 1)) { atomicOr(s_err, 1); break; }
      if (*(volatile int*)s_err) break;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int k = kb * TBK;
      tma_load_2d(st + 0 * TILE_BYTES, &mapAh, &full[s], k, m0);
      tma_load_2d(st + 1 * TILE_BYTES, &mapAl, &full[s], k, m0);
      tma_load_2d(st + 2 * TILE_BYTES, &mapVh, &full[s], k, col0 + n0);
      tma_load_2d(st + 3 * TILE_BYTES, &mapVl, &full[s], k, col0 + n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = idesc_bf16(TBM, TBN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TSTAGES;
      const uint32_t ph = (uint32_t)((kb / TSTAGES) & 1);
      if (!mbar_wait(&full[s], ph)) { atomicOr(s_err, 2); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
      const uint64_t dAh = smem_desc_sw128(base + 0 * TILE_BYTES);
      const uint64_t dAl = smem_desc_sw128(base + 1 * TILE_BYTES);
      const uint64_t dVh = smem_desc_sw128(base + 2 * TILE_BYTES);
      const uint64_t dVl = smem_desc_sw128(base + 3 * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk) {
        const uint64_t off = (uint64_t)((kk * 16 * 2) >> 4);  // 32 bytes per K=16 step
        mma_bf16(tmem, dAh + off, dVh + off, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, dAh + off, dVl + off, idesc, 1u);
        mma_bf16(tmem, dAl + off, dVh + off, idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(tmem_full);
  } else if (warp >= 4) {
    // ---------------- epilogue ----------------
    const int q = warp - 4;  // TMEM lanes 32q .. 32q+31 = tile rows
    bool ok = mbar_wait(tmem_full, 0);
    if (!ok) atomicOr(s_err, 4);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = m0 + 32 * q + lane;
    if (ok && !*(volatile int*)s_err) {
      for (int cb = 0; cb < TBN / 32; ++cb) {
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cb * 32), acc);
        if (r < M) {
#pragma unroll 4
          for (int j = 0; j < 32; ++j) {
            const int c = n0 + cb * 32 + j;
            if (c >= N) break;
            const size_t idx = (size_t)r + (size_t)(col0 + c) * ldv;
            double v = alpha * (double)acc[j];
            if (beta != 0.0) v = fma(beta, X64[idx], v);
            if (gamma != 0.0) v = fma(gamma, Z64[idx], v);
            out64[idx] = v;
            const __nv_bfloat16 hi = __double2bfloat16(v);
            const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
            const size_t bidx = (size_t)r + (size_t)(col0 + c) * kp;
            next_h[bidx] = hi;
            next_l[bidx] = lo;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN));
  }
  if (threadIdx.x == 0 && *s_err) atomicOr(&status->timeout, *s_err);
}

// ---------------- operand preparation ----------------

// Stacked real A (row-major, K contiguous, ld kp) split into BF16 hi / lo.
// Complex: Ahat = [[Ar, -Ai], [Ai, Ar]] (symmetric because A is Hermitian).
template <class T>
__global__ void split_A_kernel(int n, const T* __restrict__ A, int lda, int kp,
                               __nv_bfloat16* Ah, __nv_bfloat16* Al) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t total = (size_t)M * kp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % kp), m = (int)(t / kp);
    double x = 0.0;
    if (k < M) {
      // Ahat[m, k] = Ahat[k, m] (symmetric): read column m of Ahat, contiguous in k
      if constexpr (Sc<T>::cplx) {
        const int kk = k % n, mm = m % n;
        const bool kre = k < n, mre = m < n;
        const z64 a = A[(size_t)kk + (size_t)mm * lda];  // A[kk, mm]
        // Ahat[k, m]: block (k-half, m-half): (re,re) Ar, (re,im) -Ai, (im,re) Ai, (im,im) Ar
        x = (kre == mre) ? a.x : (kre ? -a.y : a.y);
      } else {
        x = A[(size_t)k + (size_t)m * lda];
      }
    }
    const __nv_bfloat16 hi = __double2bfloat16(x);
    Ah[t] = hi;
    Al[t] = __double2bfloat16(x - (double)__bfloat162float(hi));
  }
}

// Complex/real block V (n x ncols, ld ldv) -> stacked FP64 (M x ncols, ld ldo) and its
// BF16 hi/lo split (ld kp, rows >= M zero).
template <class T>
__global__ void split_V_kernel(int n, int ncols, const T* __restrict__ V, int ldv, double* V64,
                               int ldo, int kp, __nv_bfloat16* Vh, __nv_bfloat16* Vl) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t total = (size_t)kp * ncols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % kp), a = (int)(t / kp);
    double x = 0.0;
    if (i < M) {
      if constexpr (Sc<T>::cplx) {
        const z64 v = V[(size_t)(i % n) + (size_t)a * ldv];
        x = (i < n) ? v.x : v.y;
      } else {
        x = V[(size_t)i + (size_t)a * ldv];
      }
      V64[(size_t)i + (size_t)a * ldo] = x;
    }
    const __nv_bfloat16 hi = __double2bfloat16(x);
    Vh[t] = hi;
    Vl[t] = __double2bfloat16(x - (double)__bfloat162float(hi));
  }
}

// Stacked FP64 columns [c0, c1) back into the caller's layout.
template <class T>
__global__ void unstack_V_kernel(int n, int c0, int c1, const double* __restrict__ V64, int ldi,
                                 T* V, int ldv, bool subtract) {
  const size_t total = (size_t)n * (c1 - c0);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), a = c0 + (int)(t / n);
    T u;
    if constexpr (Sc<T>::cplx) {
      u = z64{V64[(size_t)i + (size_t)a * ldi], V64[(size_t)(i + n) + (size_t)a * ldi]};
    } else {
      u = V64[(size_t)i + (size_t)a * ldi];
    }
    T* d = V + (size_t)i + (size_t)a * ldv;
    *d = subtract ? Sc<T>::sub(*d, u) : u;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  // looked up once (thread-safe static initialisation: batch sessions call from several threads)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return nullptr;
  }();
  return fn;
}

// 2-D BF16 tensor map: inner dimension `inner` (contiguous, row length kp elements),
// `outer` rows; box 64 x 128 with 128-byte swizzle.
int make_map(CUtensorMap* map, const void* base, int kp, int outer) {
  auto enc = get_encode();
  if (!enc) return CHASE_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {TBK, 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : CHASE_ERR_CUDA;
}

inline int grid_for(size_t work) {
  return (int)std::max<size_t>(1, std::min<size_t>((work + 255) / 256, (size_t)kNumSMs * 16));
}

}  // namespace

int tc_kpad(int M) { return ((M + TBK - 1) / TBK) * TBK; }

template <class T>
int tc_split_A(cudaStream_t st, int n, const T* A, int lda, int kp, void* Ah, void* Al,
               int* launches) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  split_A_kernel<T><<<grid_for((size_t)M * kp), 256, 0, st>>>(n, A, lda, kp, (__nv_bfloat16*)Ah,
                                                              (__nv_bfloat16*)Al);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int tc_split_V(cudaStream_t st, int n, int ncols, const T* V, int ldv, double* V64, int ldo, int kp,
               void* Vh, void* Vl, int* launches) {
  split_V_kernel<T><<<grid_for((size_t)kp * ncols), 256, 0, st>>>(
      n, ncols, V, ldv, V64, ldo, kp, (__nv_bfloat16*)Vh, (__nv_bfloat16*)Vl);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int tc_unstack_V(cudaStream_t st, int n, int c0, int c1, const double* V64, int ldi, T* V, int ldv,
                 int* launches, bool subtract) {
  if (c1 <= c0) return 0;
  unstack_V_kernel<T><<<grid_for((size_t)n * (c1 - c0)), 256, 0, st>>>(n, c0, c1, V64, ldi, V, ldv,
                                                                      subtract);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

int tc_filter_step(cudaStream_t st, int M, int kp, const void* Ah, const void* Al,
                   const void* Vh_in, const void* Vl_in, int ncols_total, int col0, int N,
                   double alpha, double beta, const double* X64, double gamma, const double* Z64,
                   double* out64, int ldv, void* Vh_out, void* Vl_out, DevStatus* dst,
                   int* launches) {
  if (N <= 0) return 0;
  CUtensorMap mAh, mAl, mVh, mVl;
  if (make_map(&mAh, Ah, kp, M) || make_map(&mAl, Al, kp, M) ||
      make_map(&mVh, Vh_in, kp, ncols_total) || make_map(&mVl, Vl_in, kp, ncols_total))
    return CHASE_ERR_CUDA;
  CHASE_CUDA_TRY(cudaFuncSetAttribute(tc_filter_bf16x3_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  dim3 grid(ceil_div(N, TBN), ceil_div(M, TBM));
  tc_filter_bf16x3_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(
      mAh, mAl, mVh, mVl, M, N, kp / TBK, col0, alpha, beta, X64, gamma, Z64, out64, ldv,
      (__nv_bfloat16*)Vh_out, (__nv_bfloat16*)Vl_out, kp, dst);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template int tc_split_A<double>(cudaStream_t, int, const double*, int, int, void*, void*, int*);
template int tc_split_A<z64>(cudaStream_t, int, const z64*, int, int, void*, void*, int*);
template int tc_split_V<double>(cudaStream_t, int, int, const double*, int, double*, int, int,
                                void*, void*, int*);
template int tc_split_V<z64>(cudaStream_t, int, int, const z64*, int, double*, int, int, void*,
                             void*, int*);
template int tc_unstack_V<double>(cudaStream_t, int, int, int, const double*, int, double*, int,
                                  int*, bool);
template int tc_unstack_V<z64>(cudaStream_t, int, int, int, const double*, int, z64*, int, int*, bool);

}  // namespace chase
