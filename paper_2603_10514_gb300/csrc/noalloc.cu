// noalloc.cu -- chase_filter_noalloc: the Chebyshev filter for callers that
// cannot allocate device memory.
//
// chase_filter (like every handle-based entry point) grows a device workspace
// with cudaMalloc on demand.  Some callers cannot let a library do that: code
// that runs while a CUDA graph is being captured (cudaMalloc is not a stream
// operation and is not allowed during capture), serving processes that reserve
// all of HBM in their own pool up front and must not see a library allocate
// behind their back, and latency-critical loops where cudaMalloc / cudaFree
// would synchronise the device and stall the other streams.  This entry point
// runs the same filter kernels with its scratch in one fixed, file-scope device
// array instead, and calls no allocating routine at all.
//
// The array (CHASE_FILTER_NOALLOC_MAX_BYTES = 32 MiB) is part of the library image: every
// GPU that loads the library holds it until the process exits.  All calls on a
// device share it and it keeps the previous call's contents; nothing in it has
// to start at zero (every element the filter reads was written earlier in the
// same call).  Calls that overlap on the GPU (concurrent streams, or host
// threads calling at the same time on one device) race on the array: order
// them on one stream.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kNoAllocScratchBytes = CHASE_FILTER_NOALLOC_MAX_BYTES;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// The host-side name g_noalloc_scratch is only a stand-in for the array, not a
// device address; the device address is looked up once per device (with that
// device current) and cached.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return CHASE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return CHASE_ERR_CUDA;
    }
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return CHASE_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Algorithm 4 in place on V (n x ncols, ld ldv) with partner buffer P (ld n) and
// split-K scratch `scr`; columns with odd final degree are copied back from P.
template <class T>
int filter_fixed_scratch(cudaStream_t st, int n, const T* A, int lda, int ncols, T* V, int ldv,
                         T* P, const int* deg, double c, double e, double lambda1,
                         chase::Scratch scr) {
  const int mmax = deg[ncols - 1];
  const double sigma1 = e / (lambda1 - c);
  double sigma = sigma1;
  int first = 0;
  for (int step = 1; step <= mmax; ++step) {
    while (first < ncols && deg[first] < step) ++first;
    const int act = ncols - first;
    T* in = (step % 2 == 1) ? V : P;
    T* out = (step % 2 == 1) ? P : V;
    const int ldi = (step % 2 == 1) ? ldv : n;
    const int ldo = (step % 2 == 1) ? n : ldv;
    double alpha, beta, gamma;
    if (step == 1) {
      alpha = sigma1 / e;
      beta = -alpha * c;
      gamma = 0.0;
    } else {
      const double sn = 1.0 / (2.0 / sigma1 - sigma);
      alpha = 2.0 * sn / e;
      beta = -alpha * c;
      gamma = -sigma * sn;
      sigma = sn;
    }
    int rc = chase::gemm<T>(st, false, n, act, n, A, lda, in + (size_t)first * ldi, ldi,
                            out + (size_t)first * ldo, ldo, alpha, beta, in + (size_t)first * ldi,
                            ldi, gamma, out + (size_t)first * ldo, ldo, scr, false, false, nullptr);
    if (rc) return rc;
  }
  int a = 0;
  while (a < ncols) {
    int b = a;
    while (b < ncols && deg[b] == deg[a]) ++b;
    if (deg[a] % 2 == 1) {
      int rc = chase::copy_cols<T>(st, n, b - a, P + (size_t)a * n, n, V + (size_t)a * ldv, ldv,
                                   nullptr);
      if (rc) return rc;
    }
    a = b;
  }
  return 0;
}

template <class T>
int run(cudaStream_t st, void* base, int n, const T* A, int lda, int ncols, const T* V, int ldv,
        const int* deg, double c, double e, double lambda1, T* out, int ldo) {
  const size_t pbytes = align256(sizeof(T) * (size_t)n * ncols);
  T* P = (T*)base;
  chase::Scratch scr{(char*)base + pbytes, kNoAllocScratchBytes - pbytes};
  if (out != V) {
    int rc = chase::copy_cols<T>(st, n, ncols, V, ldv, out, ldo, nullptr);
    if (rc) return rc;
  }
  int rc = filter_fixed_scratch<T>(st, n, A, lda, ncols, out, ldo, P, deg, c, e, lambda1, scr);
  if (rc) return rc;
  // while the stream is captured into a graph the work is only recorded: return at once.
  // A capture that has been invalidated recorded nothing and runs nothing: report it.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return CHASE_ERR_CUDA;
  if (cs == cudaStreamCaptureStatusActive) return CHASE_OK;
  if (cs != cudaStreamCaptureStatusNone) return CHASE_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CHASE_ERR_CUDA;
  return CHASE_OK;
}

}  // namespace

extern "C" int chase_filter_noalloc(chase_dtype dtype, int n, const void* dA, int lda, int ncols,
                                    const void* dV, int ldv, const int* degrees, double c,
                                    double e, double lambda1, void* dVout, int ldvout,
                                    void* cuda_stream) {
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -1;
  if (n < 1) return -2;
  if (!dA) return -3;
  if (lda < n) return -4;
  if (ncols < 0) return -5;
  if (ncols > 0 && !dV) return -6;
  if (ldv < n) return -7;
  if (ncols > 0 && !degrees) return -8;
  for (int a = 0; a < ncols; ++a)
    if (degrees[a] < 0 || (a > 0 && degrees[a] < degrees[a - 1])) return -8;
  if (!(e > 0.0) || !std::isfinite(c)) return -10;
  if (!(lambda1 < c - e)) return -11;
  if (ncols > 0 && !dVout) return -12;
  if (ldvout < n) return -13;
  if (ncols == 0) return CHASE_OK;
  const size_t elem = (dtype == CHASE_R64) ? sizeof(double) : 2 * sizeof(double);
  if (!chase::output_placement_ok(dVout, ldvout, dV, ldv, dA, lda, n, ncols, elem)) return -12;
  if (elem * (size_t)n * (size_t)ncols > kNoAllocScratchBytes) return CHASE_ERR_TOO_LARGE;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return CHASE_ERR_CUDA;
  void* base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (dtype == CHASE_R64)
    return run<double>(st, base, n, (const double*)dA, lda, ncols, (const double*)dV, ldv, degrees,
                       c, e, lambda1, (double*)dVout, ldvout);
  return run<chase::z64>(st, base, n, (const chase::z64*)dA, lda, ncols, (const chase::z64*)dV, ldv,
                         degrees, c, e, lambda1, (chase::z64*)dVout, ldvout);
}
