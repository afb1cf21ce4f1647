// householder.cu -- Householder QR with explicit thin Q: the fallback of
// Algorithm 3 when even the shifted Cholesky factorisation fails.
//
// Column j: reflector v = x - alpha e_1 (x = X[j:, j], alpha = -e^{i arg x_0}
// ||x||), normalised, stored in Vh[:, j]; H_j = I - 2 v v^H is applied to the
// trailing columns (one CTA per column: block-reduced dot product, then axpy).
// Q = H_0 ... H_{l-1} [I; 0] is then accumulated backwards in place of X.
// It runs rarely (the estimate picks a Cholesky variant in the common case), so
// it favours simplicity: 3 l launches, each streaming the trailing block.
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

constexpr int HT = 256;

__device__ inline double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

template <class T>
__device__ inline T block_sum_t(T v, double* red);

template <>
__device__ inline double block_sum_t<double>(double v, double* red) { return block_sum(v, red); }

template <>
__device__ inline z64 block_sum_t<z64>(z64 v, double* red) {
  double a = block_sum(v.x, red);
  double b = block_sum(v.y, red);
  return z64{a, b};
}

// Builds reflector j from X[j:, j] into Vh[:, j] (zeros above row j).
template <class T>
__global__ void __launch_bounds__(HT) hh_reflector_kernel(int n, int j, const T* X, int ldx, T* Vh,
                                                          int ldv) {
  __shared__ double red[32];
  const T* x = X + (size_t)j * ldx;
  T* v = Vh + (size_t)j * ldv;
  double s = 0.0;
  for (int i = j + threadIdx.x; i < n; i += HT) s += Sc<T>::abs2(x[i]);
  const double nx2 = block_sum(s, red);
  const T x0 = x[j];
  const double ax0 = sqrt(Sc<T>::abs2(x0));
  const double nx = sqrt(nx2);
  T ph = (ax0 == 0.0) ? Sc<T>::one() : Sc<T>::scale(x0, 1.0 / ax0);
  T alpha = Sc<T>::scale(ph, -nx);
  T v0 = Sc<T>::sub(x0, alpha);
  // ||v||^2 = ||x||^2 - |x0|^2 + |x0 - alpha|^2
  double nv2 = nx2 - ax0 * ax0 + Sc<T>::abs2(v0);
  double inv = (nx == 0.0 || nv2 <= 0.0) ? 0.0 : 1.0 / sqrt(nv2);
  for (int i = threadIdx.x; i < n; i += HT) {
    T val;
    if (i < j) val = Sc<T>::zero();
    else if (i == j) val = Sc<T>::scale(v0, inv);
    else val = Sc<T>::scale(x[i], inv);
    v[i] = val;
  }
}

// X[j:, q] -= 2 v (v^H X[j:, q]) for the columns q = q0 + blockIdx.x.
template <class T>
__global__ void __launch_bounds__(HT) hh_apply_kernel(int n, int j, int q0, T* X, int ldx,
                                                      const T* Vh, int ldv) {
  __shared__ double red[32];
  const int q = q0 + blockIdx.x;
  const T* v = Vh + (size_t)j * ldv;
  T* col = X + (size_t)q * ldx;
  T d = Sc<T>::zero();
  for (int i = j + threadIdx.x; i < n; i += HT) Sc<T>::fmac(d, v[i], col[i]);
  d = block_sum_t<T>(d, red);
  const T d2 = Sc<T>::scale(d, 2.0);
  for (int i = j + threadIdx.x; i < n; i += HT) col[i] = Sc<T>::sub(col[i], Sc<T>::mul(v[i], d2));
}

template <class T>
__global__ void set_thin_identity_kernel(int n, int l, T* X, int ldx) {
  size_t total = (size_t)n * l;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), q = (int)(t / n);
    X[(size_t)i + (size_t)q * ldx] = (i == q) ? Sc<T>::one() : Sc<T>::zero();
  }
}

}  // namespace

template <class T>
int householder_qr(cudaStream_t st, int n, int l, T* X, int ldx, T* Vh, int ldv, double* dnorm,
                   int* launches) {
  (void)dnorm;
  if (n <= 0 || l <= 0) return 0;
  int nl = 0;
  for (int j = 0; j < l; ++j) {
    hh_reflector_kernel<T><<<1, HT, 0, st>>>(n, j, X, ldx, Vh, ldv);
    ++nl;
    if (j + 1 < l) {
      hh_apply_kernel<T><<<l - j - 1, HT, 0, st>>>(n, j, j + 1, X, ldx, Vh, ldv);
      ++nl;
    }
  }
  int blocks = std::min(ceil_div((long long)n * l, 256), kNumSMs * 8);
  set_thin_identity_kernel<T><<<blocks, 256, 0, st>>>(n, l, X, ldx);
  ++nl;
  for (int j = l - 1; j >= 0; --j) {
    hh_apply_kernel<T><<<l - j, HT, 0, st>>>(n, j, j, X, ldx, Vh, ldv);
    ++nl;
  }
  if (launches) *launches += nl;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template int householder_qr<double>(cudaStream_t, int, int, double*, int, double*, int, double*, int*);
template int householder_qr<z64>(cudaStream_t, int, int, z64*, int, z64*, int, double*, int*);

}  // namespace chase
