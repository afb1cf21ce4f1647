// lanczos.cu -- spectral bounds for the filter by a few Lanczos runs
// (Algorithm 1: "estimate lambda_1, lambda_ell and lambda_n").
//
// nruns runs advance together: one product A * [q_1 ... q_nruns] per step
// (the FP64 product kernel), column-wise alpha / beta, full
// re-orthogonalisation of each run's new vector against its own basis, then
// the m x m tridiagonal of every run is diagonalised by the device Jacobi
// solver.  The host only reduces the m * nruns Ritz values and weights to the
// three bounds:
//   b_sup      = max_r (theta_max^r + |beta_m^r|)   -- an upper bound of lambda_n
//   lambda1    = min_r theta_min^r
//   lambda_ell = smallest pooled Ritz value where the spectral-density estimate
//                (n / nruns) sum_r sum_{theta_i^r <= x} tau_i^r reaches ell
// (tau_i^r: squared first component of the i-th eigenvector of run r's T).
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

#define TRY_LZ(x)            \
  do {                       \
    int _rc = (x);           \
    if (_rc) return _rc;     \
  } while (0)

namespace chase {

namespace {

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
__device__ inline T block_sum_t(T v, double* red);

template <>
__device__ inline double block_sum_t<double>(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

template <>
__device__ inline z64 block_sum_t<z64>(z64 v, double* red) {
  const double a = block_sum_t<double>(v.x, red);
  const double b = block_sum_t<double>(v.y, red);
  return z64{a, b};
}

// coef[r * ldc + p] = q_p^r^H w_r for p = 0..np-1 (one CTA per (r, p)); the basis of run r's
// step p is Qb + p * pstride + r * n.
template <class T>
__global__ void __launch_bounds__(256) lz_dots_kernel(int n, const T* __restrict__ Qb,
                                                      size_t pstride, const T* __restrict__ W,
                                                      T* coef, int ldc) {
  __shared__ double red[8];
  const int r = blockIdx.x, p = blockIdx.y;
  const T* q = Qb + (size_t)p * pstride + (size_t)r * n;
  const T* w = W + (size_t)r * n;
  T s = Sc<T>::zero();
  for (int i = threadIdx.x; i < n; i += 256) Sc<T>::fmac(s, q[i], w[i]);
  s = block_sum_t<T>(s, red);
  if (threadIdx.x == 0) coef[(size_t)r * ldc + p] = s;
}

// w_r -= sum_{p < np} coef[r, p] q_p^r   (elementwise, one thread per (i, r))
template <class T>
__global__ void lz_sub_kernel(int n, int nruns, const T* __restrict__ Qb, size_t pstride, T* W,
                              const T* __restrict__ coef, int ldc, int np) {
  const size_t total = (size_t)n * nruns;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), r = (int)(t / n);
    T w = W[t];
    for (int p = 0; p < np; ++p)
      w = Sc<T>::sub(w, Sc<T>::mul(coef[(size_t)r * ldc + p], Qb[(size_t)p * pstride + (size_t)r * n + i]));
    W[t] = w;
  }
}

// alpha_r = Re(coef[r, j]) (the Rayleigh quotient of step j), stored for the tridiagonal.
template <class T>
__global__ void lz_store_alpha_kernel(int nruns, const T* coef, int ldc, int j, double* alpha,
                                      int m) {
  const int r = threadIdx.x;
  if (r < nruns) alpha[r * m + j] = Sc<T>::re(coef[(size_t)r * ldc + j]);
}

// beta_r = ||w_r||; q_{j+1}^r = w_r / beta_r (one CTA per run).
template <class T>
__global__ void __launch_bounds__(256) lz_normalize_kernel(int n, const T* __restrict__ W, T* qn,
                                                           double* beta, int m, int j) {
  __shared__ double red[8];
  const int r = blockIdx.x;
  const T* w = W + (size_t)r * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += Sc<T>::abs2(w[i]);
  s = block_sum_t<double>(s, red);
  const double b = sqrt(s);
  if (threadIdx.x == 0) beta[r * m + j] = b;
  const double inv = (b > 0.0) ? 1.0 / b : 0.0;
  for (int i = threadIdx.x; i < n; i += 256) qn[(size_t)r * n + i] = Sc<T>::scale(w[i], inv);
}

// Tridiagonal of run r as a dense m x m real matrix (column-major, ld m).
__global__ void lz_tridiag_kernel(int m, const double* alpha, const double* beta, int r, double* T) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m; t += gridDim.x * blockDim.x) {
    const int i = t % m, k = t / m;
    double v = 0.0;
    if (i == k) v = alpha[r * m + i];
    else if (i == k + 1) v = beta[r * m + k];
    else if (k == i + 1) v = beta[r * m + i];
    T[t] = v;
  }
}

}  // namespace

template <class T>
int lanczos_bounds(cudaStream_t st, int n, const T* A, int lda, int nruns, const T* V0, int ldv,
                   int m, int ell, double* out, void* work, size_t work_bytes, Scratch scr,
                   int* launches) {
  // workspace: basis (m + 1) x n x nruns | W n x nruns | coef nruns x (m + 1) | alpha, beta |
  //            T m x m | S m x m | theta m | jacobi work
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t pstride = (size_t)n * nruns;
  size_t off = 0;
  char* base = (char*)work;
  T* Qb = (T*)(base + off); off += al(sizeof(T) * pstride * (m + 1));
  T* W = (T*)(base + off); off += al(sizeof(T) * pstride);
  T* coef = (T*)(base + off); off += al(sizeof(T) * (size_t)nruns * (m + 1));
  double* alpha = (double*)(base + off); off += al(sizeof(double) * (size_t)nruns * m);
  double* beta = (double*)(base + off); off += al(sizeof(double) * (size_t)nruns * m);
  double* Tm = (double*)(base + off); off += al(sizeof(double) * (size_t)m * m);
  double* Sm = (double*)(base + off); off += al(sizeof(double) * (size_t)m * m);
  double* th = (double*)(base + off); off += al(sizeof(double) * (size_t)m);
  void* jw = base + off;
  if (off > work_bytes) return CHASE_ERR_OOM;
  const size_t jw_bytes = work_bytes - off;
  int nl = 0;
  // q_0 = v / ||v|| for every run
  TRY_LZ(copy_cols<T>(st, n, nruns, V0, ldv, W, n, &nl));
  lz_normalize_kernel<T><<<nruns, 256, 0, st>>>(n, W, Qb, beta, m, 0);  // beta[.,0] rewritten below
  ++nl;
  const int blocks = (int)std::min<size_t>((pstride + 255) / 256, (size_t)kNumSMs * 16);
  for (int j = 0; j < m; ++j) {
    T* qj = Qb + (size_t)j * pstride;
    // W = A q_j (all runs at once)
    TRY_LZ(gemm<T>(st, false, n, nruns, n, A, lda, qj, n, W, n, 1.0, 0.0, nullptr, 0, 0.0, nullptr,
                   0, scr, false, false, &nl));
    // coefficients against q_0..q_j: coef[., j] is alpha_j; subtracting all of them is the
    // three-term step plus full re-orthogonalisation (classical Gram-Schmidt, twice)
    for (int pass = 0; pass < 2; ++pass) {
      lz_dots_kernel<T><<<dim3(nruns, j + 1), 256, 0, st>>>(n, Qb, pstride, W, coef, m + 1);
      if (pass == 0) lz_store_alpha_kernel<T><<<1, 32, 0, st>>>(nruns, coef, m + 1, j, alpha, m);
      lz_sub_kernel<T><<<blocks, 256, 0, st>>>(n, nruns, Qb, pstride, W, coef, m + 1, j + 1);
      nl += (pass == 0) ? 3 : 2;
    }
    lz_normalize_kernel<T><<<nruns, 256, 0, st>>>(n, W, Qb + (size_t)(j + 1) * pstride, beta, m, j);
    ++nl;
  }
  // Ritz values and weights of each run
  std::vector<double> hth((size_t)nruns * m), htau((size_t)nruns * m), hbeta((size_t)nruns * m);
  std::vector<double> S1((size_t)m);
  for (int r = 0; r < nruns; ++r) {
    lz_tridiag_kernel<<<std::max(1, (m * m + 255) / 256), 256, 0, st>>>(m, alpha, beta, r, Tm);
    ++nl;
    int sweeps = 0;
    int rc = jacobi_eig<double>(st, m, Tm, m, Sm, m, th, jw, jw_bytes, 60, &sweeps, &nl);
    if (rc) return rc;
    CHASE_CUDA_TRY(cudaMemcpyAsync(hth.data() + (size_t)r * m, th, sizeof(double) * m,
                                   cudaMemcpyDeviceToHost, st));
    // first row of the eigenvector matrix: S[0, i] at stride m
    CHASE_CUDA_TRY(cudaMemcpy2DAsync(S1.data(), sizeof(double), Sm, sizeof(double) * m,
                                     sizeof(double), m, cudaMemcpyDeviceToHost, st));
    CHASE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < m; ++i) htau[(size_t)r * m + i] = S1[i] * S1[i];
  }
  CHASE_CUDA_TRY(cudaMemcpyAsync(hbeta.data(), beta, sizeof(double) * (size_t)nruns * m,
                                 cudaMemcpyDeviceToHost, st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  double bsup = -1e300, l1 = 1e300;
  for (int r = 0; r < nruns; ++r) {
    const double* t = hth.data() + (size_t)r * m;
    bsup = std::max(bsup, t[m - 1] + std::fabs(hbeta[(size_t)r * m + m - 1]));
    l1 = std::min(l1, t[0]);
  }
  std::vector<int> ord((size_t)nruns * m);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hth[a] < hth[b]; });
  double cum = 0.0, lell = hth[ord.back()];
  for (int idx : ord) {
    cum += htau[idx] * (double)n / (double)nruns;
    if (cum >= (double)ell * (1.0 - 1e-10)) { lell = hth[idx]; break; }  // up to rounding
  }
  out[0] = l1;
  out[1] = std::max(lell, l1);
  out[2] = bsup;
  if (launches) *launches += nl;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

size_t lanczos_work_bytes(size_t elem, int n, int nruns, int m) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t ps = (size_t)n * nruns;
  return al(elem * ps * (m + 1)) + al(elem * ps) + al(elem * (size_t)nruns * (m + 1)) +
         2 * al(8 * (size_t)nruns * m) + 2 * al(8 * (size_t)m * m) + al(8 * (size_t)m) +
         /* jacobi */ al(jacobi_work_bytes(m, sizeof(double))) + 256;
}

template int lanczos_bounds<double>(cudaStream_t, int, const double*, int, int, const double*, int,
                                    int, int, double*, void*, size_t, Scratch, int*);
template int lanczos_bounds<z64>(cudaStream_t, int, const z64*, int, int, const z64*, int, int, int,
                                 double*, void*, size_t, Scratch, int*);

}  // namespace chase
