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
// CTA pairs (clusters of two along grid x), one pair per 256-row block and column tile of
// BN <= 256: the even CTA issues tcgen05.mma.cta_group::2.kind::f16 (M 256, N BN, K 16),
// three per K step (Ah Vh, Ah Vl, Al Vh) into one FP32 accumulator in TMEM (its 128 rows in
// each CTA); each CTA loads its own 128 rows of Ah and Al and half of the tile's rows of Vh
// and Vl (TMA, 128-byte swizzle, 64-wide K blocks, three 64 KB stages: 12 MMAs per barrier
// round trip); 16 epilogue warps per CTA read TMEM (tcgen05.ld), apply the FP64 three-term
// update and write the BF16 split of the result.  Same structure as the modular-product
// kernel of gemm_oz.cu (and its measured reasons).
// Every mbarrier wait is bounded (~2 s of clock64); on expiry the kernel sets a flag in the
// device status word, drains, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace chase {

namespace {

using namespace tc;

constexpr int TBM = 128;   // rows of A per CTA (a pair covers 256)
constexpr int TBK = 64;    // 64 BF16 = one 128-byte swizzle row
constexpr int TBN_MAX = 256;
constexpr int TSTAGES = 3;
constexpr int T_A1 = TBM * TBK * 2;                 // 16 KB: 128 rows of Ah (or Al)
constexpr int T_B1 = (TBN_MAX / 2) * TBK * 2;       // 16 KB: up to 128 rows of Vh (or Vl)
constexpr int STAGE_BYTES = 2 * T_A1 + 2 * T_B1;    // Ah, Al, Vh half, Vl half
constexpr int TC_EPI_WARPS = 16;
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_SMEM = TSTAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t TC_TMEM_COLS = TBN_MAX;
static_assert(TC_SMEM <= 232448, "shared memory");

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_filter_bf16x3_kernel(const __grid_constant__ CUtensorMap mapAh,
                            const __grid_constant__ CUtensorMap mapAl,
                            const __grid_constant__ CUtensorMap mapVh,
                            const __grid_constant__ CUtensorMap mapVl, int M, int N, int BN,
                            int ntile, int nkb, int col0, double alpha, double beta,
                            const double* X64, double gamma, const double* Z64, double* out64,
                            int ldv, __nv_bfloat16* next_h, __nv_bfloat16* next_l, int kp,
                            DevStatus* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TSTAGES * STAGE_BYTES);  // [TSTAGES] (the even CTA's)
  uint64_t* empty = full + TSTAGES;                            // [TSTAGES]
  uint64_t* tfull = empty + TSTAGES;                           // accumulator complete
  uint32_t* tslot = (uint32_t*)(tfull + 1);
  int* s_err = (int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  // pair index p = blockIdx.x / 2 over (row pair, column tile), column tiles fastest
  const int pr = (int)(blockIdx.x >> 1);
  const int n0 = (pr % ntile) * BN, m0 = (2 * (pr / ntile) + (int)(blockIdx.x & 1)) * TBM;
  const int half = BN >> 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < TSTAGES; ++i) { bar_init(&full[i], 1); bar_init(&empty[i], 1); }
    bar_init(tfull, 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // one warp of each CTA of the pair allocates the pair's accumulator
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    const uint32_t bytes = (uint32_t)(2 * (2 * T_A1) + 2 * BN * TBK * 2);  // the pair's copies
    const uint32_t full0 = peer_addr(full, 0);
    int issued = 0;
    for (int kb = 0; kb < nkb && !*(volatile int*)s_err; ++kb) {
      const int s = kb % TSTAGES;
      if (!bar_wait(&empty[s], (uint32_t)(((kb / TSTAGES) & 1) ^ 1))) { atomicOr(s_err, 1); break; }
      if (rank == 0) bar_expect(&full[s], bytes);
      unsigned char* st = smem + s * STAGE_BYTES;
      const uint32_t fb = full0 + 8u * (uint32_t)s;
      const int k = kb * TBK, vrow = col0 + n0 + (int)rank * half;
      tma2_pair(st, &mapAh, fb, k, m0);
      tma2_pair(st + T_A1, &mapAl, fb, k, m0);
      tma2_pair(st + 2 * T_A1, &mapVh, fb, k, vrow);
      tma2_pair(st + 2 * T_A1 + T_B1, &mapVl, fb, k, vrow);
      issued = kb + 1;
    }
    for (int kb = issued; kb < issued + TSTAGES; ++kb)
      if (!bar_wait(&empty[kb % TSTAGES], (uint32_t)(((kb / TSTAGES) & 1) ^ 1))) { atomicOr(s_err, 1); break; }
    if (rank == 0)
      for (int b = max(0, issued - TSTAGES); b < issued; ++b)
        if (!bar_wait(&full[b % TSTAGES], (uint32_t)((b / TSTAGES) & 1))) { atomicOr(s_err, 1); break; }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer (even CTA): M 256 x N BN x K 16, three per K step ----------------
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)((2 * TBM) >> 4) << 24);
    bool bad = false;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TSTAGES;
      if (!bar_poll(&full[s], (uint32_t)((kb / TSTAGES) & 1))) { bad = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = s32(smem + s * STAGE_BYTES);
      const uint64_t dAh = desc_sw128(sa), dAl = desc_sw128(sa + T_A1);
      const uint64_t dVh = desc_sw128(sa + 2 * T_A1), dVl = desc_sw128(sa + 2 * T_A1 + T_B1);
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk) {
        const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes per K = 16 step
        mma_pair(tmem, dAh + off, dVh + off, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_pair(tmem, dAh + off, dVl + off, idesc, 1u);
        mma_pair(tmem, dAl + off, dVh + off, idesc, 1u);
      }
      commit_pair(&empty[s]);
    }
    if (bad) atomicOr(s_err, 2);
    commit_pair(tfull);
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs: own TMEM lanes = own 128 rows) ----------------
    const int q = warp & 3, cq = (warp - 2) >> 2;  // lane quarter, column quarter
    const int r = m0 + 32 * q + lane;
    const int cw = BN >> 2;
    const bool ok = __all_sync(0xffffffffu, bar_wait(tfull, 0u));
    if (!ok && lane == 0) atomicOr(s_err, 4);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !*(volatile int*)s_err) {
      for (int cb = 0; cb * 32 < cw; ++cb) {
        uint32_t v[32];
        ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cq * cw + cb * 32), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (r < M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int jj = cb * 32 + j;
            const int c = n0 + cq * cw + jj;
            if (jj >= cw || c >= N) continue;
            const size_t idx = (size_t)r + (size_t)(col0 + c) * ldv;
            double y = alpha * (double)__uint_as_float(v[j]);
            if (beta != 0.0) y = fma(beta, X64[idx], y);
            if (gamma != 0.0) y = fma(gamma, Z64[idx], y);
            out64[idx] = y;
            const __nv_bfloat16 hi = __double2bfloat16(y);
            const __nv_bfloat16 lo = __double2bfloat16(y - (double)__bfloat162float(hi));
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
  if (warp == 1 && !bar_wait(tfull, 0u) && lane == 0) atomicOr(s_err, 8);
  cluster_sync();  // neither CTA frees the pair's TMEM or exits while the other may signal it
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
  if (threadIdx.x == 32 && *s_err) atomicOr(&status->timeout, *s_err);
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
// `outer` rows; box 64 x box_rows with 128-byte swizzle.
int make_map(CUtensorMap* map, const void* base, int kp, int outer, int box_rows) {
  auto enc = get_encode();
  if (!enc) return CHASE_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {TBK, (cuuint32_t)box_rows};
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
  // column tiles of at most 256 (a multiple of 16), as even as possible; CTA pairs over
  // 256-row blocks
  const int ntile = ceil_div(N, TBN_MAX);
  const int BN = ceil_div(ceil_div(N, ntile), 16) * 16;
  CUtensorMap mAh, mAl, mVh, mVl;
  if (make_map(&mAh, Ah, kp, M, TBM) || make_map(&mAl, Al, kp, M, TBM) ||
      make_map(&mVh, Vh_in, kp, ncols_total, BN / 2) || make_map(&mVl, Vl_in, kp, ncols_total, BN / 2))
    return CHASE_ERR_CUDA;
  CHASE_CUDA_TRY(cudaFuncSetAttribute(tc_filter_bf16x3_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  const int mblk = ceil_div(M, 2 * TBM) * 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntile * mblk);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = TC_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CHASE_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_filter_bf16x3_kernel, mAh, mAl, mVh, mVl, M, N, BN, ntile,
                                    kp / TBK, col0, alpha, beta, X64, gamma, Z64, out64, ldv,
                                    (__nv_bfloat16*)Vh_out, (__nv_bfloat16*)Vl_out, kp, dst));
  if (launches) ++*launches;
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
