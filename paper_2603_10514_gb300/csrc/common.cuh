// common.cuh -- scalar types, error handling and small device helpers shared by
// the GB300 kernels of the Chebyshev-filtered subspace iteration library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

namespace chase {

// Interleaved complex double (same bytes as double _Complex / cuDoubleComplex).
struct __align__(16) z64 {
  double x, y;
};

__host__ __device__ inline z64 mkz(double a, double b) { return z64{a, b}; }

// ---- scalar traits ---------------------------------------------------------
template <class T> struct Sc;

template <> struct Sc<double> {
  static constexpr bool cplx = false;
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double one() { return 1.0; }
  __host__ __device__ static double conj(double a) { return a; }
  __host__ __device__ static double re(double a) { return a; }
  __host__ __device__ static double abs2(double a) { return a * a; }
  __host__ __device__ static double from_re(double a) { return a; }
  // acc += a * b
  __device__ static void fma(double& acc, double a, double b) { acc = ::fma(a, b, acc); }
  // acc += conj(a) * b
  __device__ static void fmac(double& acc, double a, double b) { acc = ::fma(a, b, acc); }
  __host__ __device__ static double mul(double a, double b) { return a * b; }
  __host__ __device__ static double add(double a, double b) { return a + b; }
  __host__ __device__ static double sub(double a, double b) { return a - b; }
  __host__ __device__ static double scale(double a, double s) { return a * s; }
  __device__ static bool finite(double a) { return isfinite(a); }
};

template <> struct Sc<z64> {
  static constexpr bool cplx = true;
  __host__ __device__ static z64 zero() { return z64{0.0, 0.0}; }
  __host__ __device__ static z64 one() { return z64{1.0, 0.0}; }
  __host__ __device__ static z64 conj(z64 a) { return z64{a.x, -a.y}; }
  __host__ __device__ static double re(z64 a) { return a.x; }
  __host__ __device__ static double abs2(z64 a) { return a.x * a.x + a.y * a.y; }
  __host__ __device__ static z64 from_re(double a) { return z64{a, 0.0}; }
  __device__ static void fma(z64& acc, z64 a, z64 b) {
    acc.x = ::fma(a.x, b.x, acc.x);
    acc.x = ::fma(-a.y, b.y, acc.x);
    acc.y = ::fma(a.x, b.y, acc.y);
    acc.y = ::fma(a.y, b.x, acc.y);
  }
  __device__ static void fmac(z64& acc, z64 a, z64 b) {  // conj(a) * b
    acc.x = ::fma(a.x, b.x, acc.x);
    acc.x = ::fma(a.y, b.y, acc.x);
    acc.y = ::fma(a.x, b.y, acc.y);
    acc.y = ::fma(-a.y, b.x, acc.y);
  }
  __host__ __device__ static z64 mul(z64 a, z64 b) {
    return z64{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
  }
  __host__ __device__ static z64 add(z64 a, z64 b) { return z64{a.x + b.x, a.y + b.y}; }
  __host__ __device__ static z64 sub(z64 a, z64 b) { return z64{a.x - b.x, a.y - b.y}; }
  __host__ __device__ static z64 scale(z64 a, double s) { return z64{a.x * s, a.y * s}; }
  __device__ static bool finite(z64 a) { return isfinite(a.x) && isfinite(a.y); }
};

// ---- launch helpers --------------------------------------------------------
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Byte range [lo, hi) a column-major n x ncols block with leading dimension ld occupies.
inline bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + bbytes && b0 < a0 + abytes;
}
inline size_t block_bytes(int n, int ncols, int ld, size_t elem) {
  return ncols > 0 ? elem * ((size_t)ld * (size_t)(ncols - 1) + (size_t)n) : 0;
}
// The filters write their result block `out` while they still read `in` and A: `out` must
// be `in` itself (same leading dimension: the in-place filter) or lie clear of both.
inline bool output_placement_ok(const void* out, int ldo, const void* in, int ldi, const void* A,
                                int lda, int n, int ncols, size_t elem) {
  const size_t ob = block_bytes(n, ncols, ldo, elem);
  if (ranges_overlap(out, ob, A, block_bytes(n, n, lda, elem))) return false;
  if (out == in) return ldo == ldi;
  return !ranges_overlap(out, ob, in, block_bytes(n, ncols, ldi, elem));
}

// Device status word written by kernels that can fail without trapping.
struct DevStatus {
  int chol_info;    // first non-positive pivot + 1 (0 = success)
  int nonfinite;    // a NaN/Inf was met
  int timeout;      // a bounded wait gave up
  int pad;
};

#ifdef __CUDACC__
// Grid-wide barrier of a cooperative launch on a counter that only grows: barrier k ends
// once all G CTAs have added their arrival (count >= (k + 1) G).  One release-add per CTA
// and acquire polls with a short back-off.  Bounded: returns false (the caller leaves the
// kernel) when the wait ran out or another CTA gave up.
struct GridBar {
  unsigned count;
  int abort;
  int sweeps;
  int pad;
};
constexpr long long kBarWait = 2000000000LL;  // ~1 s of clock64

__device__ inline bool grid_barrier(GridBar* gb, unsigned nblocks, unsigned& k) {
  __shared__ int s_ok;
  __syncthreads();
  if (nblocks == 1) return true;  // one CTA: the block barrier orders its global writes
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (++k) * nblocks;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gb->count) : "memory");
    const long long t0 = clock64();
    while (true) {
      unsigned c;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(&gb->count) : "memory");
      if ((int)(c - target) >= 0) break;
      if (*(volatile int*)&gb->abort) { ok = 0; break; }
      if (clock64() - t0 > kBarWait) { atomicExch(&gb->abort, 1); ok = 0; break; }
      __nanosleep(20);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

#endif

}  // namespace chase

#define CHASE_CUDA_TRY(expr)                         \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return ::chase::fail_cuda(_e, #expr, __FILE__, __LINE__); \
  } while (0)

namespace chase {
int fail_cuda(cudaError_t e, const char* what, const char* file, int line);
}
