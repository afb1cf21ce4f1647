// gemm_fp64.cu -- FP64 (real and complex) dense products with a fused
// three-term epilogue, for the Chebyshev filter (Algorithm 4), the Gram
// matrices of CholeskyQR (Algorithm 2), the triangular step X R^{-1} and the
// Rayleigh-Ritz products (Algorithm 1).
//
//   C[i,j] = alpha * sum_k op(A)[i,k] B[k,j] + beta * X[i,j] + gamma * Y[i,j]
//
// op(A) = A or A^H.  X and Y may alias C: each element of X / Y is read by the
// thread that then writes the same element of C, which is what lets the filter
// write V_i over V_{i-2} in place.
//
// GB300 has 2 FP64 FMA lanes per SM per clock (~1.2 TFLOP/s for the whole GPU,
// measured), so these products are bound by the FP64 pipe, not by HBM: a
// 64 x (16|32) register-tiled SIMT kernel keeps that pipe busy, and the design
// work goes into load balance across the 152 SMs.  Work is cut into
// (row tile, column tile, K chunk) units, with enough K chunks (split-K) that
// every SM receives ~8 units; partial sums go to scratch memory and a second
// kernel reduces them in a fixed order (deterministic results) and applies the
// epilogue.
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

constexpr int BM = 64;
constexpr int BK = 16;
constexpr int TM = 4;
constexpr int NT = 256;

template <class T, bool TRANS_A, int TN>
__global__ void __launch_bounds__(NT) gemm_kernel(int M, int N, int K, const T* __restrict__ A,
                                                  int lda, const T* __restrict__ B, int ldb, T* C,
                                                  int ldc, double alpha, double beta, const T* X,
                                                  int ldx, double gamma, const T* Y, int ldy,
                                                  int kchunk, T* __restrict__ partial,
                                                  int upper_only, int tri_b) {
  constexpr int BN = 16 * TN;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // column tiles vary fastest so that the CTAs in flight share A's row panels in L2
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  if (upper_only && m0 > n0 + BN - 1) return;
  const int kb = blockIdx.z * kchunk;
  int ke = min(K, kb + kchunk);
  if (tri_b) ke = min(ke, n0 + BN);  // B[k, j] = 0 for k > j

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Sc<T>::zero();

  // register prefetch of the next tile
  T ra[4], rb[TN];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i, kk;
      if (!TRANS_A) { i = tid & 63; kk = (tid >> 6) + 4 * r; }
      else          { kk = tid & 15; i = (tid >> 4) + 16 * r; }
      int gi = m0 + i, gk = k0 + kk;
      T v = Sc<T>::zero();
      if (gi < M && gk < ke) {
        v = TRANS_A ? Sc<T>::conj(A[(size_t)gk + (size_t)gi * lda]) : A[(size_t)gi + (size_t)gk * lda];
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < TN; ++r) {
      int kk = tid & 15, j = (tid >> 4) + 16 * r;
      int gj = n0 + j, gk = k0 + kk;
      T v = Sc<T>::zero();
      if (gj < N && gk < ke) v = B[(size_t)gk + (size_t)gj * ldb];
      rb[r] = v;
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i, kk;
      if (!TRANS_A) { i = tid & 63; kk = (tid >> 6) + 4 * r; }
      else          { kk = tid & 15; i = (tid >> 4) + 16 * r; }
      As[kk][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < TN; ++r) {
      int kk = tid & 15, j = (tid >> 4) + 16 * r;
      Bs[kk][j] = rb[r];
    }
  };

  if (kb < ke) load_tiles(kb);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    __syncthreads();
    store_tiles();
    __syncthreads();
    if (k0 + BK < ke) load_tiles(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) Sc<T>::fma(acc[i][j], a[i], b[j]);
    }
  }

  if (partial) {
    T* P = partial + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
        if (gi < M && gj < N) P[(size_t)gi + (size_t)gj * M] = acc[i][j];
      }
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N) {
        T v = Sc<T>::scale(acc[i][j], alpha);
        if (beta != 0.0) v = Sc<T>::add(v, Sc<T>::scale(X[(size_t)gi + (size_t)gj * ldx], beta));
        if (gamma != 0.0) v = Sc<T>::add(v, Sc<T>::scale(Y[(size_t)gi + (size_t)gj * ldy], gamma));
        C[(size_t)gi + (size_t)gj * ldc] = v;
      }
    }
}

// Sums the split-K partials in a fixed order and applies the epilogue.
template <class T>
__global__ void splitk_reduce_kernel(int M, int N, int S, const T* __restrict__ partial, T* C,
                                     int ldc, double alpha, double beta, const T* X, int ldx,
                                     double gamma, const T* Y, int ldy, int upper_only) {
  size_t total = (size_t)M * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % M), j = (int)(idx / M);
    if (upper_only && i > j) continue;
    T s = partial[idx];
    for (int z = 1; z < S; ++z) s = Sc<T>::add(s, partial[idx + (size_t)z * total]);
    T v = Sc<T>::scale(s, alpha);
    if (beta != 0.0) v = Sc<T>::add(v, Sc<T>::scale(X[(size_t)i + (size_t)j * ldx], beta));
    if (gamma != 0.0) v = Sc<T>::add(v, Sc<T>::scale(Y[(size_t)i + (size_t)j * ldy], gamma));
    C[(size_t)i + (size_t)j * ldc] = v;
  }
}

template <class T, bool TRANS_A, int TN>
void launch_gemm(cudaStream_t st, dim3 grid, int M, int N, int K, const T* A, int lda, const T* B,
                 int ldb, T* C, int ldc, double alpha, double beta, const T* X, int ldx,
                 double gamma, const T* Y, int ldy, int kchunk, T* partial, int upper_only,
                 int tri_b) {
  gemm_kernel<T, TRANS_A, TN><<<grid, NT, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, X,
                                                  ldx, gamma, Y, ldy, kchunk, partial, upper_only,
                                                  tri_b);
}

}  // namespace

template <class T>
int gemm(cudaStream_t st, bool transA, int M, int N, int K, const T* A, int lda, const T* B,
         int ldb, T* C, int ldc, double alpha, double beta, const T* X, int ldx, double gamma,
         const T* Y, int ldy, Scratch scratch, bool upper_only, bool tri_b, int* launches) {
  if (M <= 0 || N <= 0) return 0;
  // 64 x 32 tiles; 64 x 16 when N <= 16, or when a short product (K <= 256, no room for
  // split-K) would otherwise leave SMs idle: twice the CTAs, each with half the FP64 work
  int TN = (N > 16) ? 2 : 1;
  if (TN == 2 && K <= 256) {
    long long t2 = (long long)ceil_div(M, BM) * ceil_div(N, 32);
    if (upper_only) t2 = (t2 + ceil_div(M, BM)) / 2;
    if (t2 < 2LL * kNumSMs) TN = 1;
  }
  const int BN = 16 * TN;
  const int tm = ceil_div(M, BM), tn = ceil_div(N, BN);
  long long tiles = (long long)tm * tn;
  if (upper_only) tiles = (tiles + tm) / 2;
  // split-K so that every SM gets about 8 work units
  int S = 1;
  if (K > 0) {
    long long target = 8LL * kNumSMs;
    S = (int)std::max(1LL, (target + tiles - 1) / tiles);
    S = std::min(S, std::max(1, K / 64));
    size_t need = (size_t)S * M * N * sizeof(T);
    while (S > 1 && need > scratch.bytes) { --S; need = (size_t)S * M * N * sizeof(T); }
  }
  int kchunk = K;
  if (S > 1) {
    kchunk = ceil_div(ceil_div(K, S), BK) * BK;
    S = ceil_div(K, kchunk);
  }
  if (K <= 0) { S = 1; kchunk = 0; }
  T* partial = (S > 1) ? (T*)scratch.ptr : nullptr;
  dim3 grid(tn, tm, S);
  if (transA) {
    if (TN == 2) launch_gemm<T, true, 2>(st, grid, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, X, ldx, gamma, Y, ldy, kchunk, partial, upper_only, tri_b);
    else         launch_gemm<T, true, 1>(st, grid, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, X, ldx, gamma, Y, ldy, kchunk, partial, upper_only, tri_b);
  } else {
    if (TN == 2) launch_gemm<T, false, 2>(st, grid, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, X, ldx, gamma, Y, ldy, kchunk, partial, upper_only, tri_b);
    else         launch_gemm<T, false, 1>(st, grid, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, X, ldx, gamma, Y, ldy, kchunk, partial, upper_only, tri_b);
  }
  if (launches) ++*launches;
  if (S > 1) {
    size_t total = (size_t)M * N;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)kNumSMs * 16);
    splitk_reduce_kernel<T><<<blocks, 256, 0, st>>>(M, N, S, partial, C, ldc, alpha, beta, X, ldx,
                                                    gamma, Y, ldy, upper_only);
    if (launches) ++*launches;
  }
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template int gemm<double>(cudaStream_t, bool, int, int, int, const double*, int, const double*,
                          int, double*, int, double, double, const double*, int, double,
                          const double*, int, Scratch, bool, bool, int*);
template int gemm<z64>(cudaStream_t, bool, int, int, int, const z64*, int, const z64*, int, z64*,
                       int, double, double, const z64*, int, double, const z64*, int, Scratch, bool,
                       bool, int*);

}  // namespace chase
