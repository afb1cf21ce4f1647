// vec.cu -- streaming kernels around the dense products: Hermitian fill of a
// Gram matrix, residual norms of eq. res, column copies and permutations used
// by locking and by the per-column degrees of the filter, and a NaN/Inf scan.
// All are HBM-bound; grids are sized in multiples of the 152 SMs.
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

inline int grid_for(size_t work, int threads) {
  return (int)std::max<size_t>(1, std::min<size_t>((work + threads - 1) / threads, (size_t)kNumSMs * 16));
}

template <class T>
__global__ void herm_fill_lower_kernel(int n, T* G, int ldg) {
  size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    if (i > j) G[(size_t)i + (size_t)j * ldg] = Sc<T>::conj(G[(size_t)j + (size_t)i * ldg]);
    else if (i == j) G[(size_t)i + (size_t)i * ldg] = Sc<T>::from_re(Sc<T>::re(G[(size_t)i + (size_t)i * ldg]));
  }
}

// One CTA per column: r_a = ||AV[:,a] - theta_a V[:,a]|| / ||V[:,a]||.
template <class T>
__global__ void __launch_bounds__(256) resid_norms_kernel(int n, const T* __restrict__ AV, int ldav,
                                                          const T* __restrict__ V, int ldv,
                                                          const double* __restrict__ theta,
                                                          double* res) {
  __shared__ double r0[8], r1[8];
  const int a = blockIdx.x;
  const double th = theta[a];
  const T* av = AV + (size_t)a * ldav;
  const T* v = V + (size_t)a * ldv;
  double s = 0.0, sv = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    T x = v[i];
    T d = Sc<T>::sub(av[i], Sc<T>::scale(x, th));
    s += Sc<T>::abs2(d);
    sv += Sc<T>::abs2(x);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = s; r1[threadIdx.x >> 5] = sv; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < 8; ++w) { a0 += r0[w]; a1 += r1[w]; }
    res[a] = (a1 > 0.0) ? sqrt(a0) / sqrt(a1) : sqrt(a0);
  }
}

template <class T>
__global__ void gather_cols_kernel(int n, int ncols, const T* src, int lds, const int* perm, T* dst,
                                   int ldd) {
  size_t total = (size_t)n * ncols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), a = (int)(t / n);
    dst[(size_t)i + (size_t)a * ldd] = src[(size_t)i + (size_t)perm[a] * lds];
  }
}

template <class T>
__global__ void select_cols_kernel(int n, int ncols, const T* s0, const T* s1, int lds,
                                   const int* sel, T* dst, int ldd) {
  size_t total = (size_t)n * ncols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), a = (int)(t / n);
    const T* s = sel[a] ? s1 : s0;
    dst[(size_t)i + (size_t)a * ldd] = s[(size_t)i + (size_t)a * lds];
  }
}

template <class T>
__global__ void nonfinite_kernel(int n, int ncols, const T* X, int ldx, DevStatus* st) {
  size_t total = (size_t)n * ncols;
  int bad = 0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), a = (int)(t / n);
    bad |= !Sc<T>::finite(X[(size_t)i + (size_t)a * ldx]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->nonfinite, 1);
}

}  // namespace

template <class T>
int herm_fill_lower(cudaStream_t st, int n, T* G, int ldg, int* launches) {
  if (n <= 0) return 0;
  herm_fill_lower_kernel<T><<<grid_for((size_t)n * n, 256), 256, 0, st>>>(n, G, ldg);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int resid_norms(cudaStream_t st, int n, int ncols, const T* AV, int ldav, const T* V, int ldv,
                const double* dtheta, double* dres, int* launches) {
  if (n <= 0 || ncols <= 0) return 0;
  resid_norms_kernel<T><<<ncols, 256, 0, st>>>(n, AV, ldav, V, ldv, dtheta, dres);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int copy_cols(cudaStream_t st, int n, int ncols, const T* src, int lds, T* dst, int ldd,
              int* launches) {
  if (n <= 0 || ncols <= 0) return 0;
  CHASE_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(T) * (size_t)ldd, src, sizeof(T) * (size_t)lds,
                                   sizeof(T) * (size_t)n, ncols, cudaMemcpyDeviceToDevice, st));
  (void)launches;
  return 0;
}

template <class T>
int gather_cols(cudaStream_t st, int n, int ncols, const T* src, int lds, const int* dperm, T* dst,
                int ldd, int* launches) {
  if (n <= 0 || ncols <= 0) return 0;
  gather_cols_kernel<T><<<grid_for((size_t)n * ncols, 256), 256, 0, st>>>(n, ncols, src, lds, dperm,
                                                                          dst, ldd);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int select_cols(cudaStream_t st, int n, int ncols, const T* src0, const T* src1, int lds,
                const int* dsel, T* dst, int ldd, int* launches) {
  if (n <= 0 || ncols <= 0) return 0;
  select_cols_kernel<T><<<grid_for((size_t)n * ncols, 256), 256, 0, st>>>(n, ncols, src0, src1, lds,
                                                                          dsel, dst, ldd);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int nonfinite_check(cudaStream_t st, int n, int ncols, const T* X, int ldx, DevStatus* dst,
                    int* launches) {
  if (n <= 0 || ncols <= 0) return 0;
  nonfinite_kernel<T><<<grid_for((size_t)n * ncols, 256), 256, 0, st>>>(n, ncols, X, ldx, dst);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

#define CHASE_INST(T)                                                                           \
  template int herm_fill_lower<T>(cudaStream_t, int, T*, int, int*);                            \
  template int resid_norms<T>(cudaStream_t, int, int, const T*, int, const T*, int,             \
                              const double*, double*, int*);                                    \
  template int copy_cols<T>(cudaStream_t, int, int, const T*, int, T*, int, int*);              \
  template int gather_cols<T>(cudaStream_t, int, int, const T*, int, const int*, T*, int, int*); \
  template int select_cols<T>(cudaStream_t, int, int, const T*, const T*, int, const int*, T*,  \
                              int, int*);                                                       \
  template int nonfinite_check<T>(cudaStream_t, int, int, const T*, int, DevStatus*, int*);
CHASE_INST(double)
CHASE_INST(z64)
#undef CHASE_INST

}  // namespace chase
