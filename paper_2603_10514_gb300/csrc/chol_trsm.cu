// chol_trsm.cu -- the small ell x ell factorisations of CholeskyQR
// (Algorithm 2: R = chol(X^H X); Algorithm 3: chol(R + sI)) and the inverse of
// the triangular factor used for X <- X R^{-1}.
//
// Cholesky: right-looking, one CTA of 1024 threads, upper triangle in global
// memory (an ell x ell FP64 matrix, <= 23 MB, stays in the 129 MB L2).  A
// non-positive or non-finite pivot j is reported as info = j + 1 in the device
// status word (LAPACK convention) and the kernel returns -- no trap.
//
// For ell > 128 the factorisation is blocked (block 64, right-looking): the
// diagonal block is factored by one CTA in shared memory, the block row is
// R_kk^{-H} G_k. (inverse of the diagonal block, then a product), and the
// trailing update G -= R_k.^H R_k. is a K = 64 product over all SMs; the FP64
// pipe of the whole GPU does the O(ell^3) work instead of one SM's.
//
// Triangular inverse: one CTA per column j of R^{-1}; column j solves
// R x = e_j by back substitution in column-oriented (axpy) form held in
// shared memory.
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

template <class T>
__global__ void __launch_bounds__(1024) potrf_upper_kernel(int n, T* G, int ldg,
                                                           double shift_factor, DevStatus* dst) {
  __shared__ double s_piv;
  __shared__ int s_fail;
  __shared__ double s_red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  if (shift_factor > 0.0) {
    // shift s = shift_factor * ||X||_F^2 with ||X||_F^2 = trace(X^H X)
    double tr = 0.0;
    for (int j = tid; j < n; j += nt) tr += Sc<T>::re(G[(size_t)j + (size_t)j * ldg]);
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) s_red[warp] = tr;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += s_red[w];
      s_piv = shift_factor * t;
    }
    __syncthreads();
    const double s = s_piv;
    for (int j = tid; j < n; j += nt) {
      T& g = G[(size_t)j + (size_t)j * ldg];
      g = Sc<T>::add(g, Sc<T>::from_re(s));
    }
    __syncthreads();
  }
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      double d = Sc<T>::re(G[(size_t)j + (size_t)j * ldg]);
      int fail = !(d > 0.0) || !isfinite(d);
      s_fail = fail;
      if (fail) dst->chol_info = j + 1;
      s_piv = fail ? 1.0 : sqrt(d);
    }
    __syncthreads();
    if (s_fail) return;
    const double r = s_piv, inv = 1.0 / r;
    // row j of R: G[j, k] / r for k > j, diagonal r
    for (int k = j + tid; k < n; k += nt) {
      T& g = G[(size_t)j + (size_t)k * ldg];
      g = (k == j) ? Sc<T>::from_re(r) : Sc<T>::scale(g, inv);
    }
    __syncthreads();
    // trailing update of the upper triangle: G[p, q] -= conj(R[j, p]) R[j, q], j < p <= q;
    // one warp per column q, lanes along p (contiguous in column-major storage)
    for (int q = j + 1 + warp; q < n; q += nwarps) {
      const T rq = G[(size_t)j + (size_t)q * ldg];
      T* col = G + (size_t)q * ldg;
      for (int p = j + 1 + lane; p <= q; p += 32) {
        T rp = G[(size_t)j + (size_t)p * ldg];
        col[p] = Sc<T>::sub(col[p], Sc<T>::mul(Sc<T>::conj(rp), rq));
      }
    }
    __syncthreads();
  }
  // zero the strict lower triangle so that G is exactly R
  for (int k = warp; k < n; k += nwarps)
    for (int i = k + 1 + lane; i < n; i += 32) G[(size_t)i + (size_t)k * ldg] = Sc<T>::zero();
}

template <class T>
__global__ void __launch_bounds__(256) trtri_upper_kernel(int n, const T* __restrict__ R, int ldr,
                                                          T* Rinv, int ldri) {
  extern __shared__ unsigned char smem_raw[];
  T* x = reinterpret_cast<T*>(smem_raw);
  const int j = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i <= j; i += nt) x[i] = Sc<T>::zero();
  __syncthreads();
  if (tid == 0) {
    T rjj = R[(size_t)j + (size_t)j * ldr];
    // 1 / rjj (the diagonal of a Cholesky factor is real and positive)
    x[j] = Sc<T>::from_re(1.0 / Sc<T>::re(rjj));
  }
  __syncthreads();
  for (int p = j; p >= 1; --p) {
    const T xp = x[p];
    for (int i = tid; i < p; i += nt) {
      T r = R[(size_t)i + (size_t)p * ldr];
      x[i] = Sc<T>::sub(x[i], Sc<T>::mul(r, xp));
    }
    __syncthreads();
    if (tid == 0) {
      double d = Sc<T>::re(R[(size_t)(p - 1) + (size_t)(p - 1) * ldr]);
      x[p - 1] = Sc<T>::scale(x[p - 1], 1.0 / d);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt)
    Rinv[(size_t)i + (size_t)j * ldri] = (i <= j) ? x[i] : Sc<T>::zero();
}

constexpr int CNB = 64;

// G[j, j] += shift_factor * trace(G)   (one CTA)
template <class T>
__global__ void __launch_bounds__(1024) add_shift_kernel(int n, T* G, int ldg, double factor) {
  __shared__ double red[32];
  __shared__ double s_shift;
  double tr = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) tr += Sc<T>::re(G[(size_t)j + (size_t)j * ldg]);
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    s_shift = factor * t;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    T& g = G[(size_t)j + (size_t)j * ldg];
    g = Sc<T>::add(g, Sc<T>::from_re(s_shift));
  }
}

// Factors the b x b diagonal block at (off, off) in shared memory (upper, in place): one CTA
// of 1024 threads (the rank-1 updates of a 64 x 64 block take 2 entries per thread).
template <class T>
__global__ void __launch_bounds__(1024) chol_diag_kernel(int b, T* G, int ldg, int off,
                                                         DevStatus* dst) {
  extern __shared__ unsigned char diag_smem[];
  T(*B)[CNB + 1] = reinterpret_cast<T(*)[CNB + 1]>(diag_smem);  // CNB x (CNB + 1)
  __shared__ double s_piv;
  __shared__ int s_fail;
  if (*(volatile int*)&dst->chol_info) return;
  const int tid = threadIdx.x;
  for (int t = tid; t < b * b; t += blockDim.x) {
    const int i = t % b, j = t / b;
    B[i][j] = (i <= j) ? G[(size_t)(off + i) + (size_t)(off + j) * ldg] : Sc<T>::zero();
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      const double d = Sc<T>::re(B[j][j]);
      const int fail = !(d > 0.0) || !isfinite(d);
      s_fail = fail;
      if (fail) atomicCAS(&dst->chol_info, 0, off + j + 1);
      s_piv = fail ? 1.0 : sqrt(d);
    }
    __syncthreads();
    if (s_fail) return;
    const double r = s_piv, inv = 1.0 / r;
    for (int k = j + tid; k < b; k += blockDim.x) B[j][k] = (k == j) ? Sc<T>::from_re(r) : Sc<T>::scale(B[j][k], inv);
    __syncthreads();
    const int m = b - j - 1;
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int p = j + 1 + t % m, q = j + 1 + t / m;
      if (p <= q) B[p][q] = Sc<T>::sub(B[p][q], Sc<T>::mul(Sc<T>::conj(B[j][p]), B[j][q]));
    }
    __syncthreads();
  }
  for (int t = tid; t < b * b; t += blockDim.x) {
    const int i = t % b, j = t / b;
    if (i <= j) G[(size_t)(off + i) + (size_t)(off + j) * ldg] = B[i][j];
  }
}

}  // namespace

template <class T>
int potrf_upper_blocked(cudaStream_t st, int n, T* G, int ldg, double shift_factor, DevStatus* dst,
                        T* scratch, Scratch gscr, int* launches) {
  if (shift_factor > 0.0) {
    add_shift_kernel<T><<<1, 1024, 0, st>>>(n, G, ldg, shift_factor);
    if (launches) ++*launches;
  }
  T* Rkk_inv = scratch;                 // CNB x CNB
  T* tmp = scratch + CNB * CNB;         // CNB x n
  const int dsmem = (int)(sizeof(T) * CNB * (CNB + 1));
  CHASE_CUDA_TRY(cudaFuncSetAttribute(chol_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      dsmem));
  for (int off = 0; off < n; off += CNB) {
    const int b = std::min(CNB, n - off);
    chol_diag_kernel<T><<<1, 1024, dsmem, st>>>(b, G, ldg, off, dst);
    if (launches) ++*launches;
    const int rest = n - off - b;
    if (rest <= 0) break;
    T* Gkk = G + (size_t)off + (size_t)off * ldg;
    T* Gpanel = G + (size_t)off + (size_t)(off + b) * ldg;        // b x rest
    T* Gtrail = G + (size_t)(off + b) + (size_t)(off + b) * ldg;  // rest x rest
    // the inverse of the diagonal block: one CTA per column (its FP64 work over b SMs)
    int rc = trtri_upper<T>(st, b, Gkk, ldg, Rkk_inv, b, launches);
    if (rc) return rc;
    // block row: R_k. = R_kk^{-H} G_k.
    rc = gemm<T>(st, true, b, rest, b, Rkk_inv, b, Gpanel, ldg, tmp, b, 1.0, 0.0, nullptr, 0, 0.0,
                 nullptr, 0, gscr, false, false, launches);
    if (rc) return rc;
    CHASE_CUDA_TRY(cudaMemcpy2DAsync(Gpanel, sizeof(T) * (size_t)ldg, tmp, sizeof(T) * (size_t)b,
                                     sizeof(T) * (size_t)b, rest, cudaMemcpyDeviceToDevice, st));
    // trailing update of the upper triangle: G -= R_k.^H R_k.
    rc = gemm<T>(st, true, rest, rest, b, Gpanel, ldg, Gpanel, ldg, Gtrail, ldg, -1.0, 1.0, Gtrail,
                 ldg, 0.0, nullptr, 0, gscr, true, false, launches);
    if (rc) return rc;
  }
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int potrf_upper(cudaStream_t st, int n, T* G, int ldg, double shift_factor, DevStatus* dst,
                int* launches) {
  if (n <= 0) return 0;
  potrf_upper_kernel<T><<<1, 1024, 0, st>>>(n, G, ldg, shift_factor, dst);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int trtri_upper(cudaStream_t st, int n, const T* R, int ldr, T* Rinv, int ldri, int* launches) {
  if (n <= 0) return 0;
  size_t smem = sizeof(T) * (size_t)n;
  if (smem > 48 * 1024) {
    CHASE_CUDA_TRY(cudaFuncSetAttribute(trtri_upper_kernel<T>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  trtri_upper_kernel<T><<<n, 256, smem, st>>>(n, R, ldr, Rinv, ldri);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template int potrf_upper<double>(cudaStream_t, int, double*, int, double, DevStatus*, int*);
template int potrf_upper<z64>(cudaStream_t, int, z64*, int, double, DevStatus*, int*);
template int potrf_upper_blocked<double>(cudaStream_t, int, double*, int, double, DevStatus*,
                                         double*, Scratch, int*);
template int potrf_upper_blocked<z64>(cudaStream_t, int, z64*, int, double, DevStatus*, z64*,
                                      Scratch, int*);
template int trtri_upper<double>(cudaStream_t, int, const double*, int, double*, int, int*);
template int trtri_upper<z64>(cudaStream_t, int, const z64*, int, z64*, int, int*);

}  // namespace chase
