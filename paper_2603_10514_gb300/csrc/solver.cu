// solver.cu -- host driver of Algorithm 1 (ChASE) on one GB300 and the C ABI
// declared in include/chase_gb300.h.
//
// All device work of a call is ordered on the handle's stream.  Host <-> device
// traffic per outer iteration is small and explicit: the Cholesky info word
// after each factorisation (Algorithm 2's "if info != 0"), and the Ritz values
// and residuals after Rayleigh-Ritz (needed for locking and for the next
// degrees).  A stays resident; the search block lives in handle workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace chase {

int fail_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("CHASE_DEBUG")) fprintf(stderr, "chase: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
  (void)what; (void)file; (void)line; (void)e;
  return CHASE_ERR_CUDA;
}

}  // namespace chase

using namespace chase;

// CUDA-event time of selected launches on one stream (the filter's product kernels):
// event pairs around each launch, summed once the stream has been synchronised.
struct LaunchTimer {
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  bool enabled = true;  // off while a stream is being captured into a graph
  void begin(cudaStream_t st) {
    if (!enabled) return;
    while (ev.size() < used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ev.push_back(e);
    }
    cudaEventRecord(ev[used], st);
  }
  void end(cudaStream_t st) {
    if (!enabled || ev.size() < used + 2) return;
    cudaEventRecord(ev[used + 1], st);
    used += 2;
  }
  double collect() {  // seconds; call after the stream has been synchronised
    double s = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) s += ms;
    }
    used = 0;
    return s * 1e-3;
  }
  ~LaunchTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

struct chase_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* ws = nullptr;  // workspace
  size_t ws_bytes = 0;
  DevStatus* dstat = nullptr;  // device status word
  DevStatus* hstat = nullptr;  // pinned host mirror
  double* hbuf = nullptr;      // pinned host staging (small vectors)
  size_t hbuf_bytes = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int launches = 0;
  LaunchTimer product_timer;  // filter product launches of the current solve / call
  int autotune = 0;           // 1: emulated products tune their launch plans (autotune.cu)
  int tune_trials = 0;        // candidate plans run by the tuner during the current solve
};

namespace {

constexpr size_t kScratchBytes = size_t(128) << 20;  // split-K partial sums
constexpr double kU = 1.1102230246251565e-16;        // 2^-53

#define TRY(x)                    \
  do {                            \
    int _rc = (x);                \
    if (_rc) return _rc;          \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ensure_ws(chase_ctx* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return 0;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CHASE_ERR_OOM;
  }
  h->ws_bytes = bytes;
  return 0;
}

int ensure_hbuf(chase_ctx* h, size_t bytes) {
  if (bytes <= h->hbuf_bytes) return 0;
  if (h->hbuf) cudaFreeHost(h->hbuf);
  h->hbuf = nullptr;
  h->hbuf_bytes = 0;
  if (cudaMallocHost((void**)&h->hbuf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CHASE_ERR_OOM;
  }
  h->hbuf_bytes = bytes;
  return 0;
}

// Workspace carve-up for a problem of order n with block width l.
struct Layout {
  size_t V, P, AQ, T2, Xs, G, Ri, H, Wm, jac, dw, dres, scratch, total;
};

template <class T>
Layout layout_for(int n, int l) {
  Layout L{};
  size_t off = 0;
  const size_t blk = align256(sizeof(T) * (size_t)n * l);
  const size_t sq = align256(sizeof(T) * (size_t)l * l);
  L.V = off; off += blk;
  L.P = off; off += blk;
  L.AQ = off; off += blk;
  L.T2 = off; off += blk;
  L.Xs = off; off += blk;
  L.G = off; off += sq;
  L.Ri = off; off += sq;
  L.H = off; off += sq;
  L.Wm = off; off += sq;
  L.jac = off; off += align256(jacobi_work_bytes(l, sizeof(T)));
  L.dw = off; off += align256(sizeof(double) * (size_t)l);
  L.dres = off; off += align256(sizeof(double) * (size_t)l);
  L.scratch = off; off += kScratchBytes;
  L.total = off;
  return L;
}

double elapsed_s(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms * 1e-3;
}

// ---------------------------------------------------------------------------
// Algorithm 4 on columns [0, ncols) of V (in place), partner buffer P (ld ldp).
// degrees ascending.  Column a ends at step m_a; columns with odd m_a finish in
// P and are copied back at the end (runs of equal degree are contiguous).
// ---------------------------------------------------------------------------
template <class T>
int filter_inplace(chase_ctx* h, int n, const T* A, int lda, int ncols, T* V, int ldv, T* P,
                   int ldp, const int* deg, double c, double e, double lambda1, Scratch scr,
                   double* flops, int* steps = nullptr) {
  cudaStream_t st = h->stream;
  if (ncols <= 0) return 0;
  const int mmax = deg[ncols - 1];
  const double sigma1 = e / (lambda1 - c);
  double sigma = sigma1;
  int first = 0;
  const double per_col = (Sc<T>::cplx ? 8.0 : 2.0) * (double)n * (double)n;
  for (int step = 1; step <= mmax; ++step) {
    while (first < ncols && deg[first] < step) ++first;
    const int act = ncols - first;
    T* in = (step % 2 == 1) ? V : P;   // holds V_{step-1}
    T* out = (step % 2 == 1) ? P : V;  // holds V_{step-2}, receives V_step
    const int ldi = (step % 2 == 1) ? ldv : ldp;
    const int ldo = (step % 2 == 1) ? ldp : ldv;
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
    h->product_timer.begin(st);
    TRY(gemm<T>(st, false, n, act, n, A, lda, in + (size_t)first * ldi, ldi,
                out + (size_t)first * ldo, ldo, alpha, beta, in + (size_t)first * ldi, ldi, gamma,
                out + (size_t)first * ldo, ldo, scr, false, false, &h->launches));
    h->product_timer.end(st);
    if (flops) *flops += per_col * act;
    if (steps) ++*steps;
  }
  // copy back the columns whose final result sits in P (odd degree)
  int a = 0;
  while (a < ncols) {
    int b = a;
    while (b < ncols && deg[b] == deg[a]) ++b;
    if (deg[a] % 2 == 1)
      TRY(copy_cols<T>(st, n, b - a, P + (size_t)a * ldp, ldp, V + (size_t)a * ldv, ldv, &h->launches));
    a = b;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Mixed-precision (BF16x3 on tcgen05) Algorithm 4.  The block is kept in FP64
// ("stacked real": [Re; Im] for complex) in two ping-pong buffers, and its BF16
// hi/lo split in two more; A's split planes are prepared once per call site.
// ---------------------------------------------------------------------------
struct TcBufs {
  int M = 0, kp = 0, ncols = 0;
  void* Ah = nullptr;
  void* Al = nullptr;
  double* V64[2] = {nullptr, nullptr};
  void* Vh[2] = {nullptr, nullptr};
  void* Vl[2] = {nullptr, nullptr};
};

template <class T>
size_t tc_bytes(int n, int ncols) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t kp = (size_t)tc_kpad(M);
  return 2 * align256(2 * (size_t)M * kp) + 2 * align256(8 * kp * ncols) +
         4 * align256(2 * kp * ncols);
}

template <class T>
TcBufs tc_carve(char* base, int n, int ncols) {
  TcBufs B;
  B.M = Sc<T>::cplx ? 2 * n : n;
  B.kp = tc_kpad(B.M);
  B.ncols = ncols;
  size_t off = 0;
  const size_t ab = align256(2 * (size_t)B.M * B.kp);
  const size_t vb64 = align256(8 * (size_t)B.kp * ncols);
  const size_t vb16 = align256(2 * (size_t)B.kp * ncols);
  B.Ah = base + off; off += ab;
  B.Al = base + off; off += ab;
  for (int i = 0; i < 2; ++i) { B.V64[i] = (double*)(base + off); off += vb64; }
  for (int i = 0; i < 2; ++i) { B.Vh[i] = base + off; off += vb16; B.Vl[i] = base + off; off += vb16; }
  return B;
}

template <class T>
int filter_mixed(chase_ctx* h, int n, const T* A, int lda, bool split_A, int ncols, T* V, int ldv,
                 const int* deg, double c, double e, double lambda1, TcBufs& B, double* flops,
                 int* steps) {
  cudaStream_t st = h->stream;
  if (ncols <= 0) return 0;
  const int M = B.M, kp = B.kp;
  if (split_A) TRY(tc_split_A<T>(st, n, A, lda, kp, B.Ah, B.Al, &h->launches));
  TRY(tc_split_V<T>(st, n, ncols, V, ldv, B.V64[0], kp, kp, B.Vh[0], B.Vl[0], &h->launches));
  // padding rows [M, kp) of the partner BF16 planes must read as zero
  CHASE_CUDA_TRY(cudaMemsetAsync(B.Vh[1], 0, 2 * (size_t)kp * ncols, st));
  CHASE_CUDA_TRY(cudaMemsetAsync(B.Vl[1], 0, 2 * (size_t)kp * ncols, st));
  CHASE_CUDA_TRY(cudaMemsetAsync(&h->dstat->timeout, 0, sizeof(int), st));
  const int mmax = deg[ncols - 1];
  const double sigma1 = e / (lambda1 - c);
  double sigma = sigma1;
  int first = 0;
  const double per_col = (Sc<T>::cplx ? 8.0 : 2.0) * (double)n * (double)n;
  for (int step = 1; step <= mmax; ++step) {
    while (first < ncols && deg[first] < step) ++first;
    const int act = ncols - first;
    const int in = (step % 2 == 1) ? 0 : 1, out = 1 - in;
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
    h->product_timer.begin(st);
    TRY(tc_filter_step(st, M, kp, B.Ah, B.Al, B.Vh[in], B.Vl[in], ncols, first, act, alpha, beta,
                       B.V64[in], gamma, B.V64[out], B.V64[out], kp, B.Vh[out], B.Vl[out],
                       h->dstat, &h->launches));
    h->product_timer.end(st);
    if (flops) *flops += per_col * act;
    if (steps) ++*steps;
  }
  // columns ending at an odd step sit in buffer 1, the others in buffer 0
  int a = 0;
  while (a < ncols) {
    int b = a;
    while (b < ncols && deg[b] == deg[a]) ++b;
    TRY(tc_unstack_V<T>(st, n, a, b, B.V64[deg[a] % 2], kp, V, ldv, &h->launches));
    a = b;
  }
  CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h->hstat->timeout) return CHASE_ERR_TIMEOUT;
  return 0;
}

// ---------------------------------------------------------------------------
// FP64-accurate A*V products by the Ozaki scheme II (gemm_oz.cu): residue planes of
// A (prepared once per call site) and of the current block.
// ---------------------------------------------------------------------------
struct OzBufs {
  int M = 0, kp = 0, ncols = 0;  // stacked FP64 blocks: M rows, ld kp
  // complex problems: the three-product layout (Gauss): A and V planes as Re | Im | Re + Im
  // sets of n rows (K padded to kpn); the FP64 blocks stay stacked
  int c3 = 0, n = 0, kpn = 0;
  void* Ap = nullptr;
  int* rowexp = nullptr;
  void* Vp = nullptr;
  int* colexp = nullptr;
  double* V64[2] = {nullptr, nullptr};
  Scratch res{nullptr, 0};  // residues of the modular products (oz_residue_bytes(kp, ncols))
};

template <class T>
size_t oz_bytes(int n, int ncols) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t kp = (size_t)tc_kpad(M);
  // plane rows x K of A and K x columns of V: stacked (real) or three sets of order n (complex)
  const size_t arows = Sc<T>::cplx ? 3 * (size_t)n : (size_t)M;
  const size_t ak = Sc<T>::cplx ? (size_t)tc_kpad(n) : kp;
  const size_t vk = Sc<T>::cplx ? 3 * (size_t)tc_kpad(n) : kp;
  return align256(kOzPlaneBytes * arows * ak) + align256(4 * (size_t)M) + align256(kOzPlaneBytes * vk * ncols) +
         align256(4 * (size_t)ncols) + 2 * align256(8 * kp * ncols) + align256(oz_residue_bytes((int)kp, ncols));
}

template <class T>
OzBufs oz_carve(char* base, int n, int ncols) {
  OzBufs B;
  B.M = Sc<T>::cplx ? 2 * n : n;
  B.kp = tc_kpad(B.M);
  B.ncols = ncols;
  B.c3 = Sc<T>::cplx ? 1 : 0;
  B.n = n;
  B.kpn = tc_kpad(n);
  const size_t arows = B.c3 ? 3 * (size_t)n : (size_t)B.M;
  const size_t ak = B.c3 ? (size_t)B.kpn : (size_t)B.kp;
  const size_t vk = B.c3 ? 3 * (size_t)B.kpn : (size_t)B.kp;
  size_t off = 0;
  B.Ap = base + off; off += align256(kOzPlaneBytes * arows * ak);
  B.rowexp = (int*)(base + off); off += align256(4 * (size_t)B.M);
  B.Vp = base + off; off += align256(kOzPlaneBytes * vk * ncols);
  B.colexp = (int*)(base + off); off += align256(4 * (size_t)ncols);
  for (int i = 0; i < 2; ++i) { B.V64[i] = (double*)(base + off); off += align256(8 * (size_t)B.kp * ncols); }
  B.res = Scratch{base + off, oz_residue_bytes(B.kp, ncols)};
  off += align256(oz_residue_bytes(B.kp, ncols));
  return B;
}

// A's planes in the layout of B (three-product sets for complex problems, stacked otherwise).
template <class T>
int oz_slice_A_bufs(chase_ctx* h, int n, const T* A, int lda, OzBufs& B) {
  if constexpr (Sc<T>::cplx) {
    if (B.c3) return oz_slice_A3(h->stream, n, A, lda, B.kpn, B.Ap, B.rowexp, &h->launches);
  }
  return oz_slice_A<T>(h->stream, n, A, lda, B.kp, B.Ap, B.rowexp, &h->launches);
}

// A grouped-product item of B's operands: out64 = alpha A V64_in[:, col0 .. col0 + N) +
// beta X64 + gamma Z64 (stacked blocks, ld B.kp).
inline OzGroupItem oz_item(const OzBufs& B, int ncols_total, int col0, int N, double alpha, double beta,
                           const double* X64, double gamma, const double* Z64, double* out64,
                           const double* V64_in) {
  OzGroupItem it;
  it.c3 = B.c3;
  it.M = B.c3 ? B.n : B.M;
  it.kp = B.c3 ? B.kpn : B.kp;
  it.a_plane_rows = it.M;
  it.Aplanes = B.Ap;
  it.rowexp = B.rowexp;
  it.Vplanes = B.Vp;
  it.colexp = B.colexp;
  it.ncols_total = ncols_total;
  it.col0 = col0;
  it.N = N;
  it.alpha = alpha;
  it.beta = beta;
  it.gamma = gamma;
  it.X64 = X64;
  it.Z64 = Z64;
  it.out64 = out64;
  it.ldo = B.kp;
  it.resbuf = B.res;
  it.V64_in = V64_in;
  it.ldi = B.kp;
  return it;
}

// Enqueues the whole filter (no host synchronisation: it can be captured into a graph).
template <class T>
int filter_oz_enqueue(chase_ctx* h, int n, const T* A, int lda, bool split_A, int ncols, T* V,
                      int ldv, const int* deg, double c, double e, double lambda1, OzBufs& B,
                      Scratch scr, double* flops, int* steps) {
  cudaStream_t st = h->stream;
  if (ncols <= 0) return 0;
  const int M = B.M, kp = B.kp;
  if (split_A) TRY(oz_slice_A_bufs<T>(h, n, A, lda, B));
  TRY(oz_stack_V<T>(st, n, ncols, V, ldv, B.V64[0], kp, &h->launches));
  CHASE_CUDA_TRY(cudaMemsetAsync(&h->dstat->timeout, 0, sizeof(int), st));
  const int mmax = deg[ncols - 1];
  const double sigma1 = e / (lambda1 - c);
  double sigma = sigma1;
  int first = 0;
  const double per_col = (Sc<T>::cplx ? 8.0 : 2.0) * (double)n * (double)n;
  for (int step = 1; step <= mmax; ++step) {
    while (first < ncols && deg[first] < step) ++first;
    const int act = ncols - first;
    const int in = (step % 2 == 1) ? 0 : 1, out = 1 - in;
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
    if (B.c3) {
      const OzGroupItem it = oz_item(B, ncols, first, act, alpha, beta, B.V64[in], gamma, B.V64[out],
                                     B.V64[out], B.V64[in]);
      TRY(oz_slice_V_group(st, 1, &it, &h->launches));
      h->product_timer.begin(st);
      TRY(oz_gemm_group(st, 1, &it, h->dstat, &h->launches));
      h->product_timer.end(st);
    } else {
      TRY(oz_slice_V(st, M, first, ncols, B.V64[in], kp, kp, ncols, B.Vp, B.colexp, &h->launches));
      h->product_timer.begin(st);
      TRY(oz_gemm(st, M, kp, B.Ap, B.rowexp, 0, B.Vp, B.colexp, ncols, first, act, alpha, beta,
                  B.V64[in], gamma, B.V64[out], B.V64[out], kp, h->dstat, B.res, &h->launches,
                  h->autotune, &h->tune_trials));
      h->product_timer.end(st);
    }
    if (flops) *flops += per_col * act;
    if (steps) ++*steps;
  }
  int a = 0;
  while (a < ncols) {
    int b = a;
    while (b < ncols && deg[b] == deg[a]) ++b;
    TRY(tc_unstack_V<T>(st, n, a, b, B.V64[deg[a] % 2], kp, V, ldv, &h->launches));
    a = b;
  }
  return 0;
}

// Reads the device status word after the filter's work.
inline int filter_finish(chase_ctx* h) {
  CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                                 h->stream));
  CHASE_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (h->hstat->timeout) return CHASE_ERR_TIMEOUT;
  return 0;
}

template <class T>
int filter_oz(chase_ctx* h, int n, const T* A, int lda, bool split_A, int ncols, T* V, int ldv,
              const int* deg, double c, double e, double lambda1, OzBufs& B, Scratch scr,
              double* flops, int* steps) {
  if (ncols <= 0) return 0;
  TRY(filter_oz_enqueue<T>(h, n, A, lda, split_A, ncols, V, ldv, deg, c, e, lambda1, B, scr, flops,
                           steps));
  return filter_finish(h);
}

// The same filter recorded into a CUDA graph and launched as one unit (the launch sequence of
// a filter call is fixed by its degrees).  Needs a stream that can be captured (not one of
// the default streams); otherwise the launches are issued directly.  Product launch times
// are not taken per launch inside a graph.
// *t_build receives the host time spent recording and instantiating the graph (seconds);
// *launched is set when the filter ran as a graph.
template <class T>
int filter_oz_graph(chase_ctx* h, int n, const T* A, int lda, bool split_A, int ncols, T* V,
                    int ldv, const int* deg, double c, double e, double lambda1, OzBufs& B,
                    Scratch scr, double* flops, int* steps, double* t_build, bool* launched) {
  cudaStream_t st = h->stream;
  *launched = false;
  if (ncols <= 0) return 0;
  if ((uintptr_t)st <= 2)  // NULL, cudaStreamLegacy, cudaStreamPerThread: not capturable
    return filter_oz<T>(h, n, A, lda, split_A, ncols, V, ldv, deg, c, e, lambda1, B, scr, flops,
                        steps);
  const auto tb0 = std::chrono::steady_clock::now();
  CHASE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  h->product_timer.enabled = false;
  const int rc = filter_oz_enqueue<T>(h, n, A, lda, split_A, ncols, V, ldv, deg, c, e, lambda1, B,
                                      scr, flops, steps);
  h->product_timer.enabled = true;
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  if (rc || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : CHASE_ERR_CUDA;
  }
  cudaGraphExec_t ge = nullptr;
  if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return CHASE_ERR_CUDA;
  }
  *t_build += std::chrono::duration<double>(std::chrono::steady_clock::now() - tb0).count();
  *launched = true;
  const cudaError_t le = cudaGraphLaunch(ge, st);
  const int frc = (le == cudaSuccess) ? filter_finish(h) : CHASE_ERR_CUDA;
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  return frc;
}

// AQ = A Q (n x nu, both ld n) by the Ozaki-scheme product; A's planes must be ready.
template <class T>
int aq_oz(chase_ctx* h, int n, const T* Q, int nu, T* AQ, OzBufs& B, Scratch scr) {
  cudaStream_t st = h->stream;
  if (nu <= 0) return 0;
  TRY(oz_stack_V<T>(st, n, nu, Q, n, B.V64[0], B.kp, &h->launches));
  if (B.c3) {
    const OzGroupItem it = oz_item(B, B.ncols, 0, nu, 1.0, 0.0, nullptr, 0.0, nullptr, B.V64[1], B.V64[0]);
    TRY(oz_slice_V_group(st, 1, &it, &h->launches));
    TRY(oz_gemm_group(st, 1, &it, h->dstat, &h->launches));
  } else {
    TRY(oz_slice_V(st, B.M, 0, nu, B.V64[0], B.kp, B.kp, B.ncols, B.Vp, B.colexp, &h->launches));
    TRY(oz_gemm(st, B.M, B.kp, B.Ap, B.rowexp, 0, B.Vp, B.colexp, B.ncols, 0, nu, 1.0, 0.0, nullptr,
                0.0, nullptr, B.V64[1], B.kp, h->dstat, B.res, &h->launches, h->autotune,
                &h->tune_trials));
  }
  TRY(tc_unstack_V<T>(st, n, 0, nu, B.V64[1], B.kp, AQ, n, &h->launches));
  return 0;
}

// ---------------------------------------------------------------------------
// FP64-accurate products of the QR and Rayleigh-Ritz steps by the Ozaki scheme:
//   Gram    G = X^H Y (l x l; X's columns are the left operand's rows, Y and
//           -i Y the right operand's columns, K = n or 2n);
//   tall    Y = X B  (X n x kl sliced by rows of its stacked operator
//           [[Xr, -Xi], [Xi, Xr]], B kl x N stacked as [Br; Bi]).
// ---------------------------------------------------------------------------
struct OzProd {
  int n = 0, l = 0, M = 0, kp = 0, kpl = 0;
  void* Gp = nullptr;  int* gexp = nullptr;   // kp x 2l column planes (Y | -iY)
  void* Lp = nullptr;  int* lexp = nullptr;   // kp x l column planes (X, when X != Y)
  void* Rp = nullptr;  int* rexp = nullptr;   // M x kpl row planes of a tall X
  void* Bp = nullptr;  int* bexp = nullptr;   // kpl x l column planes of a small factor
  double* B64 = nullptr;                      // kpl x l stacked small factor
  double* out = nullptr;                      // FP64 result staging, max(M, 2l) x l
  void* Xt = nullptr;                         // X^T (l x n)
  Scratch res{nullptr, 0};                    // residues of the modular products
};

template <class T>
size_t ozp_bytes(int n, int l) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t kp = (size_t)tc_kpad(M);
  const size_t kpl = (size_t)tc_kpad(Sc<T>::cplx ? 2 * l : l);
  const size_t wl = Sc<T>::cplx ? 2 * (size_t)l : (size_t)l;
  return align256(kOzPlaneBytes * kp * wl) + align256(4 * wl) + align256(kOzPlaneBytes * kp * l) + align256(4 * (size_t)l) +
         align256(kOzPlaneBytes * (size_t)M * kpl) + align256(4 * (size_t)M) + align256(kOzPlaneBytes * kpl * l) +
         align256(4 * (size_t)l) + align256(8 * kpl * l) +
         align256(8 * std::max<size_t>(M, wl) * l) + align256(sizeof(T) * (size_t)n * l) +
         align256(oz_residue_bytes((int)std::max<size_t>(M, wl), l));
}

template <class T>
OzProd ozp_carve(char* base, int n, int l) {
  OzProd P;
  P.n = n; P.l = l;
  P.M = Sc<T>::cplx ? 2 * n : n;
  P.kp = tc_kpad(P.M);
  P.kpl = tc_kpad(Sc<T>::cplx ? 2 * l : l);
  const size_t wl = Sc<T>::cplx ? 2 * (size_t)l : (size_t)l;
  size_t off = 0;
  auto take = [&](size_t b) { char* p = base + off; off += align256(b); return p; };
  P.Gp = take(kOzPlaneBytes * (size_t)P.kp * wl);
  P.gexp = (int*)take(4 * wl);
  P.Lp = take(kOzPlaneBytes * (size_t)P.kp * l);
  P.lexp = (int*)take(4 * (size_t)l);
  P.Rp = take(kOzPlaneBytes * (size_t)P.M * P.kpl);
  P.rexp = (int*)take(4 * (size_t)P.M);
  P.Bp = take(kOzPlaneBytes * (size_t)P.kpl * l);
  P.bexp = (int*)take(4 * (size_t)l);
  P.B64 = (double*)take(8 * (size_t)P.kpl * l);
  P.out = (double*)take(8 * std::max<size_t>(P.M, wl) * l);
  P.Xt = take(sizeof(T) * (size_t)n * l);
  const size_t rb = oz_residue_bytes((int)std::max<size_t>(P.M, wl), l);
  P.res = Scratch{take(rb), rb};
  return P;
}

// G = X^H Y (q x q, ld ldg) for X, Y n x q; X == Y uses one slicing for both sides.
template <class T>
int oz_gram(chase_ctx* h, OzProd& P, int q, const T* X, int ldx, const T* Y, int ldy, T* G, int ldg,
            Scratch scr) {
  cudaStream_t st = h->stream;
  if (q <= 0) return 0;
  const bool cplx = Sc<T>::cplx;
  const int wq = cplx ? 2 * q : q;
  TRY(oz_slice_cols<T>(st, P.n, q, Y, ldy, P.kp, true, P.Gp, P.gexp, &h->launches));
  const void* left = P.Gp;
  const int* lexp = P.gexp;
  int plane_rows = wq;
  if (X != Y) {
    TRY(oz_slice_cols<T>(st, P.n, q, X, ldx, P.kp, false, P.Lp, P.lexp, &h->launches));
    left = P.Lp;
    lexp = P.lexp;
    plane_rows = q;
  }
  TRY(oz_gemm(st, q, P.kp, left, lexp, plane_rows, P.Gp, P.gexp, wq, 0, wq, 1.0, 0.0, nullptr, 0.0,
              nullptr, P.out, q, h->dstat, P.res, &h->launches, h->autotune, &h->tune_trials));
  TRY(oz_gram_assemble<T>(st, q, q, P.out, q, G, ldg, &h->launches));
  return 0;
}

// Residue planes of the small right factor B (kl x N, ld ldb) for oz_tall.  kpk: padded K of
// the product (0: the whole block's, P.kpl; a narrower factor passes tc_kpad of its own K so
// that the modular products do not run over zero padding).
template <class T>
int oz_prep_factor(chase_ctx* h, OzProd& P, int kl, int N, const T* B, int ldb, int kpk = 0) {
  cudaStream_t st = h->stream;
  const int K = Sc<T>::cplx ? 2 * kl : kl;
  if (kpk <= 0) kpk = P.kpl;
  TRY(oz_stack_V<T>(st, kl, N, B, ldb, P.B64, kpk, &h->launches));
  TRY(oz_slice_V(st, K, 0, N, P.B64, kpk, kpk, N, P.Bp, P.bexp, &h->launches));
  return 0;
}

// Y = X B (n x N, ld ldy), or Y -= X B with subtract, with X n x kl (ld ldx) and B prepared
// by oz_prep_factor with the same kpk.  Y may alias X: X is fully sliced before Y is written.
template <class T>
int oz_tall(chase_ctx* h, OzProd& P, int kl, const T* X, int ldx, int N, T* Y, int ldy, Scratch scr,
            int kpk = 0, bool subtract = false) {
  cudaStream_t st = h->stream;
  if (N <= 0) return 0;
  if (kpk <= 0) kpk = P.kpl;
  T* Xt = (T*)P.Xt;
  TRY(transpose<T>(st, P.n, kl, X, ldx, Xt, kl, &h->launches));
  TRY(oz_slice_rows<T>(st, P.n, kl, Xt, kl, kpk, P.Rp, P.rexp, &h->launches));
  TRY(oz_gemm(st, P.M, kpk, P.Rp, P.rexp, 0, P.Bp, P.bexp, N, 0, N, 1.0, 0.0, nullptr, 0.0,
              nullptr, P.out, P.M, h->dstat, P.res, &h->launches, h->autotune, &h->tune_trials));
  TRY(tc_unstack_V<T>(st, P.n, 0, N, P.out, P.M, Y, ldy, &h->launches, subtract));
  return 0;
}

// W = X^H Y (qx x qy, ld ldw) for X n x qx and Y n x qy (the rectangular form of oz_gram).
template <class T>
int oz_xhy(chase_ctx* h, OzProd& P, int qx, const T* X, int ldx, int qy, const T* Y, int ldy, T* W,
           int ldw) {
  cudaStream_t st = h->stream;
  if (qx <= 0 || qy <= 0) return 0;
  const int wqy = Sc<T>::cplx ? 2 * qy : qy;
  TRY(oz_slice_cols<T>(st, P.n, qy, Y, ldy, P.kp, true, P.Gp, P.gexp, &h->launches));
  TRY(oz_slice_cols<T>(st, P.n, qx, X, ldx, P.kp, false, P.Lp, P.lexp, &h->launches));
  TRY(oz_gemm(st, qx, P.kp, P.Lp, P.lexp, qx, P.Gp, P.gexp, wqy, 0, wqy, 1.0, 0.0, nullptr, 0.0,
              nullptr, P.out, qx, h->dstat, P.res, &h->launches, h->autotune, &h->tune_trials));
  TRY(oz_gram_assemble<T>(st, qx, qy, P.out, qx, W, ldw, &h->launches));
  return 0;
}

// One CholeskyQR pass (Algorithm 2 body): X <- X R^{-1} with R = chol(X^H X [+ sI]).
// Result lands in X (via Xtmp).  Returns 0, CHASE_CHOL_FAILED (info in *info) or an error.
// With oz the two products run as Ozaki-scheme products.
template <class T>
int cholqr_pass(chase_ctx* h, int n, int l, T* X, int ldx, T* Xtmp, T* G, T* Ri, double shift_factor,
                Scratch scr, int* info, OzProd* oz) {
  cudaStream_t st = h->stream;
  if (oz)
    TRY(oz_gram<T>(h, *oz, l, X, ldx, X, ldx, G, l, scr));
  else
    TRY(gemm<T>(st, true, l, l, n, X, ldx, X, ldx, G, l, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, scr,
                true, false, &h->launches));
  CHASE_CUDA_TRY(cudaMemsetAsync(&h->dstat->chol_info, 0, sizeof(int), st));
  if (l > 128)
    TRY(potrf_upper_blocked<T>(st, l, G, l, shift_factor, h->dstat, Ri, scr, &h->launches));
  else
    TRY(potrf_upper<T>(st, l, G, l, shift_factor, h->dstat, &h->launches));
  CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h->hstat->timeout) return CHASE_ERR_TIMEOUT;
  *info = h->hstat->chol_info;
  if (*info) return CHASE_CHOL_FAILED;
  TRY(trtri_upper<T>(st, l, G, l, Ri, l, &h->launches));
  if (oz) {
    TRY(oz_prep_factor<T>(h, *oz, l, l, Ri, l));
    TRY(oz_tall<T>(h, *oz, l, X, ldx, l, X, ldx, scr));
    return 0;
  }
  TRY(gemm<T>(st, false, n, l, l, X, ldx, Ri, l, Xtmp, n, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0,
              scr, false, true, &h->launches));
  TRY(copy_cols<T>(st, n, l, Xtmp, n, X, ldx, &h->launches));
  return 0;
}

// C <- (I - V op(T) V^H) C, op(T) = T^H (trans) or T, for the panel's reflectors V (n x b,
// ld n; zero above row j0) and a block C (n x nc, ld ldc; rows above j0 are left as they
// are, since V vanishes there).  W, W2: b x nc (ld b).
template <class T>
int wy_apply(chase_ctx* h, int n, int j0, int b, const T* V, const T* Tm, int ldt, bool trans, T* C,
             int ldc, int nc, T* W, T* W2, Scratch scr, OzProd* oz) {
  cudaStream_t st = h->stream;
  if (nc <= 0) return 0;
  if (oz)
    TRY(oz_xhy<T>(h, *oz, b, V, n, nc, C, ldc, W, b));
  else
    TRY(gemm<T>(st, true, b, nc, n - j0, V + j0, n, C + j0, ldc, W, b, 1.0, 0.0, nullptr, 0, 0.0,
                nullptr, 0, scr, false, false, &h->launches));
  TRY(gemm<T>(st, trans, b, nc, b, Tm, ldt, W, b, W2, b, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, scr,
              false, false, &h->launches));
  if (oz) {
    const int kpk = tc_kpad(Sc<T>::cplx ? 2 * b : b);
    TRY(oz_prep_factor<T>(h, *oz, b, nc, W2, b, kpk));
    TRY(oz_tall<T>(h, *oz, b, V, n, nc, C, ldc, scr, kpk, true));
  } else {
    TRY(gemm<T>(st, false, n - j0, nc, b, V + j0, n, W2, b, C + j0, ldc, -1.0, 1.0, C + j0, ldc, 0.0,
                nullptr, 0, scr, false, false, &h->launches));
  }
  return 0;
}

// Householder QR with explicit thin Q in the compact WY form (the fallback of Algorithm 3):
// panels of b columns are factored with the level-2 kernels restricted to the panel, and
// the trailing columns, then the explicit Q (accumulated backwards from [I; 0]), are updated
// by the panel's I - V T V^H as block products, on the emulated-FP64 tensor-core engine when
// oz is given.  Vh: n x l (ld n) for the reflectors; Wb: >= b*l elements; Rb: >= 2*b*l +
// 2*b*b elements (W2, the panels' T factors, the panel Gram).  Narrow blocks (l < 96) take
// the unblocked form.
template <class T>
int householder_blocked(chase_ctx* h, int n, int l, T* X, int ldx, T* Vh, T* Wb, T* Rb, Scratch scr,
                        OzProd* oz) {
  cudaStream_t st = h->stream;
  if (l < 96) return householder_qr<T>(st, n, l, X, ldx, Vh, n, nullptr, &h->launches);
  const int nb = l >= 192 ? 64 : 32;
  const int np = ceil_div(l, nb);
  T* W = Wb;
  T* W2 = Rb;
  T* Ts = Rb + (size_t)nb * l;
  T* Gp = Ts + (size_t)np * nb * nb;
  for (int k = 0; k < np; ++k) {
    const int j0 = k * nb, b = std::min(nb, l - j0);
    T* V = Vh + (size_t)j0 * n;
    T* Tk = Ts + (size_t)k * nb * nb;
    const int pc = hh_panel_coop<T>(st, n, j0, b, X, ldx, Vh, n, Gp, nb, scr, h->dstat, &h->launches);
    if (pc == CHASE_ERR_UNSUPPORTED) {
      TRY(hh_panel<T>(st, n, j0, b, X, ldx, Vh, n, &h->launches));
      TRY(gemm<T>(st, true, b, b, n - j0, V + j0, n, V + j0, n, Gp, nb, 1.0, 0.0, nullptr, 0, 0.0,
                  nullptr, 0, scr, true, false, &h->launches));
    } else {
      TRY(pc);
    }
    TRY(hh_build_T<T>(st, b, Gp, nb, Tk, nb, &h->launches));
    TRY(wy_apply<T>(h, n, j0, b, V, Tk, nb, true, X + (size_t)(j0 + b) * ldx, ldx, l - j0 - b, W, W2,
                    scr, oz));
  }
  TRY(hh_thin_identity<T>(st, n, l, X, ldx, &h->launches));
  for (int k = np - 1; k >= 0; --k) {
    const int j0 = k * nb, b = std::min(nb, l - j0);
    TRY(wy_apply<T>(h, n, j0, b, Vh + (size_t)j0 * n, Ts + (size_t)k * nb * nb, nb, false,
                    X + (size_t)j0 * ldx, ldx, l - j0, W, W2, scr, oz));
  }
  // a bounded wait of a panel kernel that ran out is reported, not left in the result
  CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h->hstat->timeout) return CHASE_ERR_TIMEOUT;
  return 0;
}

// Algorithm 3 with escalation.  X (n x l, ld ldx) in place.  Workspace: Xtmp, Xsave (n x l, ld n),
// G, Ri (l x l).  variant in/out: requested (0 = by log_est) -> used.
template <class T>
int qr_dynamic(chase_ctx* h, int n, int l, T* X, int ldx, double log_est, double cond_hi,
               double cond_lo, int force, T* Xtmp, T* Xsave, T* G, T* Ri, Scratch scr,
               int* variant_used, int* first_fail_info, OzProd* oz = nullptr) {
  cudaStream_t st = h->stream;
  int variant = force;
  if (force == 0) {
    if (log_est > std::log(cond_hi)) variant = 3;
    else if (log_est < std::log(cond_lo)) variant = 1;
    else variant = 2;
  }
  if (first_fail_info) *first_fail_info = 0;
  const bool need_save = (variant != 4);
  if (need_save) TRY(copy_cols<T>(st, n, l, X, ldx, Xsave, n, &h->launches));
  const double shift_factor = 11.0 * ((double)n * l + (double)l * (l + 1)) * kU;
  for (;;) {
    int info = 0, rc = 0;
    if (variant == 1 || variant == 2) {
      for (int p = 0; p < variant && rc == 0; ++p)
        rc = cholqr_pass<T>(h, n, l, X, ldx, Xtmp, G, Ri, 0.0, scr, &info, oz);
    } else if (variant == 3) {
      rc = cholqr_pass<T>(h, n, l, X, ldx, Xtmp, G, Ri, shift_factor, scr, &info, oz);
      for (int p = 0; p < 2 && rc == 0; ++p)
        rc = cholqr_pass<T>(h, n, l, X, ldx, Xtmp, G, Ri, 0.0, scr, &info, oz);
    } else {
      TRY(householder_blocked<T>(h, n, l, X, ldx, Xtmp, G, Ri, scr, oz));
      break;
    }
    if (rc == 0) break;
    if (rc != CHASE_CHOL_FAILED) return rc;
    if (first_fail_info && !*first_fail_info) *first_fail_info = info;
    if (force != 0) {  // forced variant: report, restore the input
      TRY(copy_cols<T>(st, n, l, Xsave, n, X, ldx, &h->launches));
      CHASE_CUDA_TRY(cudaStreamSynchronize(st));
      if (variant_used) *variant_used = variant;
      return CHASE_CHOL_FAILED;
    }
    TRY(copy_cols<T>(st, n, l, Xsave, n, X, ldx, &h->launches));
    variant = (variant < 3) ? 3 : 4;
  }
  if (variant_used) *variant_used = variant;
  return 0;
}

double abs_rho(double x, double c, double e) {
  double t = std::fabs((x - c) / e);
  if (t <= 1.0) return 1.0;
  return t + std::sqrt(t * t - 1.0);
}

double log_cond_est(double theta_k1, int m_k1, int m_ell, double lambda1, double c, double e,
                    double eta) {
  return std::log(eta) + (double)m_k1 * std::log(abs_rho(theta_k1, c, e)) +
         (double)(m_ell - m_k1) * std::log(abs_rho(lambda1, c, e));
}

// ---------------------------------------------------------------------------
// Algorithm 1 as a per-problem state advanced one outer iteration at a time:
// begin (V0 copied, checks, step-0 QR), then per iteration filter() and
// after_filter() (condition estimate + QR, Rayleigh-Ritz, residuals, locking,
// next degrees), then finish() (results to the caller).  chase_solve runs one
// problem through it; a batch session (chase_batch_*) runs many, with the
// emulated-FP64 filters of all its problems grouped into shared launches.
// ---------------------------------------------------------------------------

// One problem's part of a grouped emulated-FP64 filter call.
struct GroupFilterItem {
  OzBufs* B = nullptr;
  int ncols = 0;              // unlocked columns filtered
  const int* deg = nullptr;   // their degrees, ascending
  double c = 0.0, e = 1.0, lambda1 = 0.0;
};

struct SolveBase {
  virtual ~SolveBase() {}
  virtual int begin() = 0;
  virtual int filter() = 0;
  virtual int after_filter() = 0;
  virtual int finish() = 0;
  // the iteration's filter may join a grouped launch (emulated FP64, no graph capture)
  virtual bool group_filter_ok() const = 0;
  virtual int group_filter_prepare(GroupFilterItem* g) = 0;  // A's residues (once), stacked V
  virtual int group_filter_done(double seconds, int launches) = 0;  // V back, stats
  virtual cudaStream_t stream() const = 0;  // where the problem's own work is ordered
  bool done = false;
  int status = CHASE_NOT_CONVERGED;  // result once done
};

template <class T>
size_t solve_bytes(int n, int l, chase_precision prec) {
  const bool mixed = (prec == CHASE_BF16X3);
  const bool emu = (prec == CHASE_BF16X3 || prec == CHASE_FP64_EMU);
  return layout_for<T>(n, l).total + (mixed ? tc_bytes<T>(n, l) : 0) +
         (emu ? align256(oz_bytes<T>(n, l)) + ozp_bytes<T>(n, l) : 0);
}

template <class T>
struct Solve final : SolveBase {
  chase_ctx* h;
  cudaStream_t st;
  int n, lda, nev, nex, l;
  const T* A;
  T* dV;
  int ldv;
  chase_config cfg;
  chase_bounds bd;
  double* evals;
  double* resid;
  chase_stats* stats_out;
  chase_iter_log* logs;
  int log_cap;
  // workspace (solve_bytes) and pinned host staging (4 l doubles)
  char* base;
  double* hstage;
  Layout L;
  T *V = nullptr, *P = nullptr, *AQ = nullptr, *T2 = nullptr, *Xs = nullptr, *G = nullptr,
    *Ri = nullptr, *H = nullptr, *Wm = nullptr;
  void* jac = nullptr;
  size_t jac_bytes = 0;
  double *dw = nullptr, *dres = nullptr;
  Scratch scr{nullptr, 0};
  TcBufs tcb;
  OzBufs ozb;
  OzProd ozp;
  OzProd* ozq = nullptr;
  bool mixed = false, emu = false, lowprec = false, A_split = false, A_oz = false;
  double normA_est = 0.0;
  chase_stats S{};
  std::vector<int> deg;
  std::vector<double> ritz, res;
  double mu1 = 0.0, mu_ell = 0.0, bsup = 0.0;
  int k = 0, it = 0;
  long long matvecs = 0;
  int launches0 = 0;
  double c = 0.0, e = 1.0;  // the current iteration's damped interval
  cudaEvent_t e0 = nullptr, e1 = nullptr, t0 = nullptr, t1 = nullptr;

  Solve(chase_ctx* h_, int n_, const T* A_, int lda_, int nev_, int nex_, const chase_config& cfg_,
        const chase_bounds& bd_, T* dV_, int ldv_, double* evals_, double* resid_,
        chase_stats* stats_, chase_iter_log* logs_, int log_cap_, char* base_, double* hstage_)
      : h(h_), st(h_->stream), n(n_), lda(lda_), nev(nev_), nex(nex_), l(nev_ + nex_), A(A_),
        dV(dV_), ldv(ldv_), cfg(cfg_), bd(bd_), evals(evals_), resid(resid_), stats_out(stats_),
        logs(logs_), log_cap(log_cap_), base(base_), hstage(hstage_) {}

  ~Solve() override {
    for (cudaEvent_t ev : {e0, e1, t0, t1})
      if (ev) cudaEventDestroy(ev);
  }

  void phase_begin() { cudaEventRecord(e0, st); }
  void phase_end(double& acc) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    acc += elapsed_s(e0, e1);
  }

  int begin() override {
    L = layout_for<T>(n, l);
    mixed = (cfg.prec == CHASE_BF16X3);
    emu = (cfg.prec == CHASE_BF16X3 || cfg.prec == CHASE_FP64_EMU);
    const size_t tcb_bytes = mixed ? tc_bytes<T>(n, l) : 0;
    const size_t ozb_bytes = emu ? align256(oz_bytes<T>(n, l)) : 0;
    V = (T*)(base + L.V);
    P = (T*)(base + L.P);
    AQ = (T*)(base + L.AQ);
    T2 = (T*)(base + L.T2);
    Xs = (T*)(base + L.Xs);
    G = (T*)(base + L.G);
    Ri = (T*)(base + L.Ri);
    H = (T*)(base + L.H);
    Wm = (T*)(base + L.Wm);
    jac = base + L.jac;
    jac_bytes = L.dw - L.jac;
    dw = (double*)(base + L.dw);
    dres = (double*)(base + L.dres);
    scr = Scratch{base + L.scratch, kScratchBytes};
    if (mixed) tcb = tc_carve<T>(base + L.total, n, l);
    if (emu) {
      ozb = oz_carve<T>(base + L.total + tcb_bytes, n, l);
      ozp = ozp_carve<T>(base + L.total + tcb_bytes + ozb_bytes, n, l);
      ozq = &ozp;
    }
    lowprec = mixed;
    normA_est = std::max(std::fabs(bd.lambda1), std::fabs(bd.b_sup));
    h->autotune = cfg.autotune;
    h->tune_trials = 0;
    for (cudaEvent_t* ev : {&e0, &e1, &t0, &t1})
      CHASE_CUDA_TRY(cudaEventCreate(ev));
    cudaEventRecord(t0, st);
    launches0 = h->launches;
    deg.assign(l, cfg.deg_init);
    ritz.assign(l, bd.lambda1);
    res.assign(l, 1.0);
    mu1 = bd.lambda1;
    mu_ell = bd.lambda_ell;
    bsup = bd.b_sup;
    CHASE_CUDA_TRY(cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), st));
    TRY(copy_cols<T>(st, n, l, dV, ldv, V, n, &h->launches));
    TRY(nonfinite_check<T>(st, n, n, A, lda, h->dstat, &h->launches));
    TRY(nonfinite_check<T>(st, n, l, V, n, h->dstat, &h->launches));
    CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    CHASE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h->hstat->nonfinite) return CHASE_ERR_NONFINITE;
    // step 0: orthonormalise V0 (CholeskyQR2; Householder if forced or on failure)
    phase_begin();
    int v0 = 0, fi = 0;
    const int rc = qr_dynamic<T>(h, n, l, V, n, std::log(100.0), cfg.cond_hi, cfg.cond_lo,
                                 cfg.qr_force == 4 ? 4 : 0, P, Xs, G, Ri, scr, &v0, &fi, ozq);
    phase_end(S.t_qr);
    if (rc) return rc;
    if (cfg.max_iter <= 0) done = true;
    return 0;
  }

  void interval() {
    c = 0.5 * (bsup + mu_ell);
    e = 0.5 * (bsup - mu_ell);
  }

  int filter() override {
    interval();
    const int nu = l - k;
    int rc = 0;
    phase_begin();
    if (lowprec) {
      double fl = 0.0, tf = 0.0;
      rc = filter_mixed<T>(h, n, A, lda, !A_split, nu, V + (size_t)k * n, n, deg.data() + k, c, e,
                           mu1, tcb, &fl, &S.filter_launches);
      A_split = true;
      phase_end(tf);
      S.t_filter += tf;
      S.t_filter_lowprec += tf;
      S.filter_flops += fl;
      S.filter_flops_lowprec += fl;
      ++S.n_lowprec_iters;
    } else if (emu) {
      if (cfg.graph_filter) {
        // t_filter covers recording, instantiation, launch and completion; the recording
        // and instantiation alone go to t_graph_build.  The product launches inside a graph
        // are not timed one by one, so t_filter_product gets nothing from such a filter.
        bool launched = false;
        rc = filter_oz_graph<T>(h, n, A, lda, !A_oz, nu, V + (size_t)k * n, n, deg.data() + k, c,
                                e, mu1, ozb, scr, &S.filter_flops, &S.filter_launches,
                                &S.t_graph_build, &launched);
        phase_end(S.t_filter);
        if (launched) ++S.graph_launches;
      } else {
        rc = filter_oz<T>(h, n, A, lda, !A_oz, nu, V + (size_t)k * n, n, deg.data() + k, c, e, mu1,
                          ozb, scr, &S.filter_flops, &S.filter_launches);
        phase_end(S.t_filter);
      }
      A_oz = true;
    } else {
      rc = filter_inplace<T>(h, n, A, lda, nu, V + (size_t)k * n, n, P, n, deg.data() + k, c, e,
                             mu1, scr, &S.filter_flops, &S.filter_launches);
      phase_end(S.t_filter);
    }
    S.t_filter_product += h->product_timer.collect();  // the phase end synchronised the stream
    return rc;
  }

  // the grouped launch runs each product's K unsplit (K = n), so longer ones filter alone
  bool group_filter_ok() const override {
    return emu && !lowprec && !cfg.graph_filter && n <= kOzSplitMaxK;
  }
  cudaStream_t stream() const override { return st; }

  int group_filter_prepare(GroupFilterItem* g) override {
    interval();
    const int nu = l - k;
    if (!A_oz) TRY(oz_slice_A_bufs<T>(h, n, A, lda, ozb));
    A_oz = true;
    TRY(oz_stack_V<T>(st, n, nu, V + (size_t)k * n, n, ozb.V64[0], ozb.kp, &h->launches));
    g->B = &ozb;
    g->ncols = nu;
    g->deg = deg.data() + k;
    g->c = c;
    g->e = e;
    g->lambda1 = mu1;
    return 0;
  }

  int group_filter_done(double seconds, int launches) override {
    const int nu = l - k;
    const int* d = deg.data() + k;
    int a = 0;
    while (a < nu) {  // columns ending at an odd step sit in buffer 1, the others in buffer 0
      int b = a;
      while (b < nu && d[b] == d[a]) ++b;
      TRY(tc_unstack_V<T>(st, n, a, b, ozb.V64[d[a] % 2], ozb.kp, V + (size_t)k * n, n,
                          &h->launches));
      a = b;
    }
    const double per_col = (Sc<T>::cplx ? 8.0 : 2.0) * (double)n * (double)n;
    for (int j = 0; j < nu; ++j) S.filter_flops += per_col * d[j];
    S.t_filter += seconds;
    S.filter_launches += launches;
    return 0;
  }

  int after_filter() override {
    const int nu = l - k;
    int rc = 0;
    for (int a = k; a < l; ++a) matvecs += deg[a];
    if (cfg.filtered_hook) {
      CHASE_CUDA_TRY(cudaStreamSynchronize(st));
      cfg.filtered_hook(cfg.filtered_hook_ctx, V, n, l, n, it + 1);
    }
    // --- condition estimate (Eq. full-est) and QR (Algorithm 3) ---
    const double theta_k1 = (it == 0) ? mu1 : ritz[k];
    const double lest_paper = log_cond_est(theta_k1, deg[k], deg[l - 1], mu1, c, e, cfg.eta);
    const double lest_locked = std::max(
        lest_paper, std::log(cfg.eta) + (double)deg[l - 1] * std::log(abs_rho(mu1, c, e)));
    const double lest = (cfg.cond_est_mode == 1) ? lest_locked : lest_paper;
    phase_begin();
    if (k > 0) rc = copy_cols<T>(st, n, k, V, n, T2, n, &h->launches);
    int variant = 0, fi = 0;
    if (!rc) rc = qr_dynamic<T>(h, n, l, V, n, lest, cfg.cond_hi, cfg.cond_lo, cfg.qr_force, P, Xs,
                                G, Ri, scr, &variant, &fi, ozq);
    if (!rc && k > 0) rc = copy_cols<T>(st, n, k, T2, n, V, n, &h->launches);
    phase_end(S.t_qr);
    if (rc) return rc;
    if (variant == 1) ++S.n_chol1;
    else if (variant == 2) ++S.n_chol2;
    else if (variant == 3) ++S.n_shifted;
    else ++S.n_hhqr;
    if (fi) ++S.n_chol_failures;
    // --- Rayleigh-Ritz on the unlocked columns ---
    phase_begin();
    T* Q2 = V + (size_t)k * n;
    if (emu) {
      if (!A_oz) rc = oz_slice_A_bufs<T>(h, n, A, lda, ozb);
      A_oz = true;
      if (!rc) rc = aq_oz<T>(h, n, Q2, nu, AQ, ozb, scr);
    } else {
      rc = gemm<T>(st, false, n, nu, n, A, lda, Q2, n, AQ, n, 1.0, 0.0, nullptr, 0, 0.0, nullptr,
                   0, scr, false, false, &h->launches);
    }
    if (rc) {
    } else if (ozq) {
      rc = oz_gram<T>(h, ozp, nu, Q2, n, AQ, n, H, nu, scr);
    } else {
      rc = gemm<T>(st, true, nu, nu, n, Q2, n, AQ, n, H, nu, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0,
                   scr, true, false, &h->launches);
    }
    if (!rc) rc = herm_fill_lower<T>(st, nu, H, nu, &h->launches);
    int sweeps = 0;
    cudaEvent_t j0 = nullptr, j1 = nullptr;
    cudaEventCreate(&j0);
    cudaEventCreate(&j1);
    cudaEventRecord(j0, st);
    if (!rc) rc = jacobi_eig<T>(st, nu, H, nu, Wm, nu, dw, jac, jac_bytes, 40, &sweeps, &h->launches);
    cudaEventRecord(j1, st);
    cudaEventSynchronize(j1);
    S.t_rr_eig += elapsed_s(j0, j1);
    S.jacobi_sweeps += sweeps;
    cudaEventDestroy(j0);
    cudaEventDestroy(j1);
    // V <- Q2 W, AV = AQ W (into P)
    if (rc) {
    } else if (ozq) {
      rc = oz_prep_factor<T>(h, ozp, nu, nu, Wm, nu);
      if (!rc) rc = oz_tall<T>(h, ozp, nu, AQ, n, nu, P, n, scr);
      if (!rc) rc = oz_tall<T>(h, ozp, nu, Q2, n, nu, Q2, n, scr);
    } else {
      rc = gemm<T>(st, false, n, nu, nu, Q2, n, Wm, nu, T2, n, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0,
                   scr, false, false, &h->launches);
      if (!rc) rc = gemm<T>(st, false, n, nu, nu, AQ, n, Wm, nu, P, n, 1.0, 0.0, nullptr, 0, 0.0,
                            nullptr, 0, scr, false, false, &h->launches);
      if (!rc) rc = copy_cols<T>(st, n, nu, T2, n, Q2, n, &h->launches);
    }
    phase_end(S.t_rr);
    if (rc) return rc;
    // --- residuals (eq. res) ---
    double* hw = hstage;      // l Ritz values
    double* hr = hstage + l;  // l residuals
    phase_begin();
    rc = resid_norms<T>(st, n, nu, P, n, Q2, n, dw, dres, &h->launches);
    if (!rc) rc = (cudaMemcpyAsync(hw, dw, sizeof(double) * nu, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                   cudaMemcpyAsync(hr, dres, sizeof(double) * nu, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                   cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st) == cudaSuccess)
                      ? 0 : CHASE_ERR_CUDA;
    phase_end(S.t_resid);
    if (!rc && h->hstat->timeout) rc = CHASE_ERR_TIMEOUT;
    if (rc) return rc;
    for (int a = 0; a < nu; ++a) {
      ritz[k + a] = hw[a];
      res[k + a] = hr[a];
    }
    // --- locking: contiguous converged prefix among the first nev ---
    int knew = k;
    while (knew < nev && res[knew] < cfg.tol) ++knew;
    if (logs && it < log_cap) {
      chase_iter_log& g = logs[it];
      g.iteration = it + 1; g.locked_before = k; g.locked_after = knew; g.variant = variant;
      g.chol_fail_info = fi; g.deg_min = deg[k]; g.deg_max = deg[l - 1]; g.matvecs = matvecs;
      g.log_cond_est = lest; g.c = c; g.e = e; g.mu1 = mu1; g.mu_ell = mu_ell;
      g.log_cond_est_paper = lest_paper; g.log_cond_est_locked = lest_locked;
    }
    for (int a = k; a < l; ++a) mu1 = std::min(mu1, ritz[a]);
    mu_ell = ritz[l - 1];
    for (int a = k; a < l; ++a) mu_ell = std::max(mu_ell, ritz[a]);
    k = knew;
    ++it;
    if (k >= nev) {
      status = CHASE_OK;
      done = true;
      return 0;
    }
    if (it >= cfg.max_iter) done = true;  // the next degrees are still formed, as before a filter
    // mixed mode: FP64 filters once the wanted residuals reach the BF16x3 regime
    if (lowprec) {
      double rmax = 0.0;
      for (int a = k; a < nev; ++a) rmax = std::max(rmax, res[a]);
      if (rmax <= cfg.mp_switch * normA_est) lowprec = false;
    }
    // --- degrees of the unlocked columns, ascending order ---
    if (cfg.opt_degree) {
      const double c2 = 0.5 * (bsup + mu_ell), e2 = 0.5 * (bsup - mu_ell);
      for (int a = k; a < l; ++a) {
        const double lr = std::log(abs_rho(ritz[a], c2, e2));
        int m;
        if (lr <= 0.0) m = cfg.deg_max;
        else if (!(res[a] > cfg.tol)) m = cfg.deg_min;
        else {
          const double mm = std::ceil(std::log(res[a] / cfg.tol) / lr);
          m = (mm > cfg.deg_max) ? cfg.deg_max : (int)mm;
        }
        m = std::max(cfg.deg_min, std::min(cfg.deg_max, m));
        deg[a] = m;
      }
      // stable sort of [k, l) by degree; apply the permutation to V's columns
      std::vector<int> idx(l - k);
      std::iota(idx.begin(), idx.end(), k);
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return deg[x] < deg[y]; });
      bool moved = false;
      for (int a = 0; a < l - k; ++a) moved |= (idx[a] != k + a);
      if (moved) {
        std::vector<int> d2(l - k);
        std::vector<double> r2(l - k), s2(l - k);
        int* hperm = (int*)(hstage + 2 * (size_t)l);
        for (int a = 0; a < l - k; ++a) {
          d2[a] = deg[idx[a]]; r2[a] = ritz[idx[a]]; s2[a] = res[idx[a]];
          hperm[a] = idx[a] - k;
        }
        for (int a = 0; a < l - k; ++a) { deg[k + a] = d2[a]; ritz[k + a] = r2[a]; res[k + a] = s2[a]; }
        int* dperm = (int*)jac;  // Jacobi workspace is free here
        CHASE_CUDA_TRY(cudaMemcpyAsync(dperm, hperm, sizeof(int) * (l - k), cudaMemcpyHostToDevice, st));
        TRY(copy_cols<T>(st, n, l - k, V + (size_t)k * n, n, T2, n, &h->launches));
        TRY(gather_cols<T>(st, n, l - k, T2, n, dperm, V + (size_t)k * n, n, &h->launches));
        CHASE_CUDA_TRY(cudaStreamSynchronize(st));  // hperm lives in the staging buffer
      }
    } else {
      for (int a = k; a < l; ++a) deg[a] = cfg.deg_init;
    }
    return 0;
  }

  int finish() override {
    // locked pairs ascending (selection order over the locked prefix)
    const int kout = std::min(k, nev);
    std::vector<int> ord(l);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.begin() + kout, [&](int x, int y) { return ritz[x] < ritz[y]; });
    bool moved = false;
    for (int a = 0; a < kout; ++a) moved |= (ord[a] != a);
    if (moved) {
      int* hperm = (int*)(hstage + 2 * (size_t)l);
      for (int a = 0; a < l; ++a) hperm[a] = ord[a];
      int* dperm = (int*)jac;
      CHASE_CUDA_TRY(cudaMemcpyAsync(dperm, hperm, sizeof(int) * l, cudaMemcpyHostToDevice, st));
      TRY(copy_cols<T>(st, n, l, V, n, T2, n, &h->launches));
      TRY(gather_cols<T>(st, n, l, T2, n, dperm, V, n, &h->launches));
    }
    TRY(copy_cols<T>(st, n, l, V, n, dV, ldv, &h->launches));
    cudaEventRecord(t1, st);
    CHASE_CUDA_TRY(cudaStreamSynchronize(st));
    S.t_total = elapsed_s(t0, t1);
    for (int a = 0; a < nev; ++a) {
      evals[a] = ritz[ord[a]];
      resid[a] = res[ord[a]];
    }
    S.iterations = it;
    S.locked = k;
    S.matvecs = matvecs;
    S.kernel_launches = h->launches - launches0;
    S.autotune_trials = h->tune_trials;
    if (stats_out) *stats_out = S;
    return status;
  }
};

template <class T>
int solve_impl(chase_ctx* h, int n, const T* A, int lda, int nev, int nex, const chase_config& cfg,
               const chase_bounds& bd, T* dV, int ldv, double* evals, double* resid,
               chase_stats* stats, chase_iter_log* logs, int log_cap) {
  const int l = nev + nex;
  TRY(ensure_ws(h, solve_bytes<T>(n, l, cfg.prec)));
  TRY(ensure_hbuf(h, sizeof(double) * 4 * (size_t)l + 4096));
  h->product_timer.collect();  // drop events of an earlier call
  Solve<T> s(h, n, A, lda, nev, nex, cfg, bd, dV, ldv, evals, resid, stats, logs, log_cap,
             (char*)h->ws, h->hbuf);
  TRY(s.begin());
  while (!s.done) {
    TRY(s.filter());
    TRY(s.after_filter());
  }
  return s.finish();
}


// The emulated-FP64 filters of several problems (Algorithm 4 for each, with its own damped
// interval, degrees and block) as shared launches: per step of the three-term recurrence one
// grouped slicing, one grouped modular product and one grouped reconstruction over every
// problem whose highest degree has not been reached.  Per problem the arithmetic is that of
// filter_oz (the modular products are exact, so tiling and grouping change no bit).
int group_filter_oz(chase_ctx* h, const std::vector<SolveBase*>& probs) {
  cudaStream_t st = h->stream;
  const int np = (int)probs.size();
  if (np == 0) return 0;
  std::vector<GroupFilterItem> g(np);
  cudaEvent_t a = nullptr, b = nullptr;
  CHASE_CUDA_TRY(cudaEventCreate(&a));
  CHASE_CUDA_TRY(cudaEventCreate(&b));
  // each problem stacks its block (and cuts A's residues once) on its own stream; the shared
  // launches on this stream wait for all of them
  for (int p = 0; p < np; ++p) {
    TRY(probs[p]->group_filter_prepare(&g[p]));
    if (probs[p]->stream() != st) {
      cudaEvent_t r = nullptr;
      CHASE_CUDA_TRY(cudaEventCreateWithFlags(&r, cudaEventDisableTiming));
      cudaEventRecord(r, probs[p]->stream());
      cudaStreamWaitEvent(st, r, 0);
      cudaEventDestroy(r);
    }
  }
  CHASE_CUDA_TRY(cudaMemsetAsync(&h->dstat->timeout, 0, sizeof(int), st));
  cudaEventRecord(a, st);
  int launches = 0, rc = 0;
  std::vector<double> sigma1(np), sigma(np);
  std::vector<int> first(np, 0);
  int mmax = 0;
  for (int p = 0; p < np; ++p) {
    sigma1[p] = g[p].e / (g[p].lambda1 - g[p].c);
    sigma[p] = sigma1[p];
    if (g[p].ncols > 0) mmax = std::max(mmax, g[p].deg[g[p].ncols - 1]);
  }
  std::vector<OzGroupItem> items;
  items.reserve(np);
  for (int step = 1; step <= mmax && !rc; ++step) {
    items.clear();
    for (int p = 0; p < np; ++p) {
      const GroupFilterItem& q = g[p];
      if (q.ncols <= 0 || q.deg[q.ncols - 1] < step) continue;
      while (first[p] < q.ncols && q.deg[first[p]] < step) ++first[p];
      const int in = (step % 2 == 1) ? 0 : 1, out = 1 - in;
      double alpha, beta, gamma;
      if (step == 1) {
        alpha = sigma1[p] / q.e;
        beta = -alpha * q.c;
        gamma = 0.0;
      } else {
        const double sn = 1.0 / (2.0 / sigma1[p] - sigma[p]);
        alpha = 2.0 * sn / q.e;
        beta = -alpha * q.c;
        gamma = -sigma[p] * sn;
        sigma[p] = sn;
      }
      const OzBufs& B = *q.B;
      items.push_back(oz_item(B, q.ncols, first[p], q.ncols - first[p], alpha, beta, B.V64[in], gamma,
                              B.V64[out], B.V64[out], B.V64[in]));
    }
    rc = oz_slice_V_group(st, (int)items.size(), items.data(), &launches);
    if (!rc) rc = oz_gemm_group(st, (int)items.size(), items.data(), h->dstat, &launches);
  }
  cudaEventRecord(b, st);
  const cudaError_t se = cudaEventSynchronize(b);
  const double t = elapsed_s(a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->launches += launches;
  if (rc) return rc;
  if (se != cudaSuccess) return CHASE_ERR_CUDA;
  for (int p = 0; p < np; ++p) TRY(probs[p]->group_filter_done(t, launches));
  CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h->hstat->timeout) return CHASE_ERR_TIMEOUT;
  return 0;
}

// Caching allocator of a batch session: freed blocks stay cached and serve later requests of
// up to twice their size, so that a service admitting problems of similar shapes allocates
// (and synchronises the device for cudaFree) rarely.  Device or pinned host memory.
struct BlockPool {
  bool host;
  std::multimap<size_t, void*> cached;
  size_t cached_bytes = 0;
  explicit BlockPool(bool host_) : host(host_) {}
  static size_t round(size_t b) { return (b + ((size_t)2 << 20) - 1) & ~(((size_t)2 << 20) - 1); }
  void* raw_alloc(size_t b) {
    void* p = nullptr;
    const cudaError_t e = host ? cudaMallocHost(&p, b) : cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void raw_free(void* p) {
    if (host) cudaFreeHost(p);
    else cudaFree(p);
  }
  // returns the block and its (rounded) size in *got; nullptr when the device is full
  void* get(size_t bytes, size_t* got) {
    const size_t want = round(bytes);
    auto it = cached.lower_bound(want);
    if (it != cached.end() && it->first <= 2 * want) {
      void* p = it->second;
      *got = it->first;
      cached_bytes -= it->first;
      cached.erase(it);
      return p;
    }
    void* p = raw_alloc(want);
    if (!p && !cached.empty()) {  // give the cached blocks back and try once more
      release();
      p = raw_alloc(want);
    }
    *got = want;
    return p;
  }
  void put(void* p, size_t bytes) {
    if (!p) return;
    cached.emplace(bytes, p);
    cached_bytes += bytes;
  }
  void release() {
    for (auto& kv : cached) raw_free(kv.second);
    cached.clear();
    cached_bytes = 0;
  }
  ~BlockPool() { release(); }
};

}  // namespace

struct chase_batch_ctx {
  chase_ctx* h = nullptr;
  struct Item {
    int id;
    SolveBase* s;
    chase_ctx* sub;  // the problem's own stream and status word
    void* ws;
    size_t ws_bytes;
    double* hst;
    size_t hst_bytes;
  };
  std::vector<Item> items;                       // in flight
  std::vector<std::pair<int, int>> finished;     // (id, status) not yet reported
  std::vector<chase_ctx*> subs;                  // idle per-problem contexts
  int next_id = 0;
  BlockPool dev{false}, host{true};
  // A context for one problem: a non-blocking stream and a device status word of its own,
  // so that the problems' QR and Rayleigh-Ritz phases run concurrently.
  chase_ctx* get_sub() {
    if (!subs.empty()) {
      chase_ctx* c = subs.back();
      subs.pop_back();
      return c;
    }
    chase_ctx* c = new chase_ctx();
    c->device = h->device;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void**)&c->dstat, sizeof(DevStatus)) != cudaSuccess ||
        cudaMallocHost((void**)&c->hstat, sizeof(DevStatus)) != cudaSuccess) {
      cudaGetLastError();
      free_sub(c);
      return nullptr;
    }
    c->own_stream = true;
    return c;
  }
  static void free_sub(chase_ctx* c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->dstat) cudaFree(c->dstat);
    if (c->hstat) cudaFreeHost(c->hstat);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
  }
  void release(Item& it) {
    if (it.sub) cudaStreamSynchronize(it.sub->stream);
    delete it.s;
    dev.put(it.ws, it.ws_bytes);
    host.put(it.hst, it.hst_bytes);
    if (it.sub) subs.push_back(it.sub);
    it.s = nullptr;
    it.sub = nullptr;
  }
  ~chase_batch_ctx() {
    if (h) cudaStreamSynchronize(h->stream);
    for (Item& it : items) release(it);
    for (chase_ctx* c : subs) free_sub(c);
  }
};

namespace {

// One outer iteration of every problem in flight: the grouped emulated-FP64 filters, the
// other filters one by one, then each problem's QR, Rayleigh-Ritz, residuals and locking.
// Problems that end (converged, out of iterations, or failed) are finalised and queued as
// finished.
// One chase_batch_step: the problems in flight advance asynchronously.  Worker threads run
// each problem's phase after its filter (QR, Rayleigh-Ritz, residuals, locking -- or, for a
// problem that does not group, its own filter first) on the problem's stream; as soon as a
// problem's phase ends it is ready for its next filter, and the calling thread launches one
// grouped emulated-FP64 filter for every problem ready at that moment.  Fast problems thus
// do not wait for slow ones, and the grouped launches take whoever is ready.  The call
// returns once every problem in flight has advanced at least one outer iteration (or ended),
// with no phase running: problems can then be added before the next call.
void batch_advance(chase_batch_ctx* b) {
  const int m = (int)b->items.size();
  if (m == 0) return;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> tasks;
  std::vector<int> done_idx;  // indices whose phase finished, not yet collected
  std::vector<int> rc(m, 0), ended(m, 0), adv(m, 0), solo(m, 0);
  int running = 0;
  bool quit = false;
  const int nw = std::min(m, 16);
  std::vector<std::thread> workers;
  workers.reserve(nw);
  for (int w = 0; w < nw; ++w)
    workers.emplace_back([&]() {
      cudaSetDevice(b->h->device);
      for (;;) {
        int i;
        {
          std::unique_lock<std::mutex> lk(mu);
          cv.wait(lk, [&] { return quit || !tasks.empty(); });
          if (tasks.empty()) return;
          i = tasks.front();
          tasks.pop_front();
        }
        SolveBase* s = b->items[i].s;
        int r = 0;
        if (solo[i]) r = s->filter();
        if (!r) r = s->after_filter();
        if (!r && s->done) r = s->finish();
        {
          std::lock_guard<std::mutex> lk(mu);
          rc[i] = r;
          ended[i] = (r != 0) || s->done;
          done_idx.push_back(i);
          --running;
        }
        cv.notify_all();
      }
    });
  std::vector<int> ready(m);
  std::iota(ready.begin(), ready.end(), 0);
  bool stopping = false;
  for (;;) {
    if (!stopping && !ready.empty()) {
      std::vector<SolveBase*> grp;
      std::vector<int> gi;
      for (int i : ready) {
        solo[i] = !b->items[i].s->group_filter_ok();
        if (!solo[i]) {
          grp.push_back(b->items[i].s);
          gi.push_back(i);
        }
      }
      const int grc = group_filter_oz(b->h, grp);  // phases of other problems run meanwhile
      {
        std::lock_guard<std::mutex> lk(mu);
        for (int i : ready) {
          if (!solo[i] && grc) {  // the shared filter failed: the problem ends with that error
            rc[i] = grc;
            ended[i] = 1;
            done_idx.push_back(i);
            continue;
          }
          tasks.push_back(i);
          ++running;
        }
      }
      cv.notify_all();
      ready.clear();
    }
    std::vector<int> got;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return !done_idx.empty() || (running == 0 && tasks.empty()); });
      got.swap(done_idx);
    }
    for (int i : got) {
      if (ended[i]) continue;
      ++adv[i];
      if (!stopping) ready.push_back(i);
    }
    if (!stopping) {
      bool all = true;
      for (int i = 0; i < m; ++i) all = all && (ended[i] || adv[i] >= 1);
      stopping = all;
    }
    if (stopping) {
      std::unique_lock<std::mutex> lk(mu);
      if (running == 0 && tasks.empty() && done_idx.empty()) break;
    }
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    quit = true;
  }
  cv.notify_all();
  for (std::thread& t : workers) t.join();
  std::vector<chase_batch_ctx::Item> keep;
  for (int i = 0; i < m; ++i) {
    chase_batch_ctx::Item& it = b->items[i];
    if (!ended[i]) {
      keep.push_back(it);
      continue;
    }
    b->finished.emplace_back(it.id, rc[i]);
    b->release(it);
  }
  b->items.swap(keep);
}

}  // namespace

namespace {

template <class T>
int filter_impl(chase_ctx* h, int n, const T* A, int lda, int ncols, const T* dV, int ldv,
                const int* degrees, double c, double e, double lambda1, chase_precision prec,
                T* dVout, int ldo) {
  cudaStream_t st = h->stream;
  if (prec == CHASE_FP64_EMU) {
    const size_t ob = align256(oz_bytes<T>(n, ncols));
    TRY(ensure_ws(h, ob + kScratchBytes));
    OzBufs B = oz_carve<T>((char*)h->ws, n, ncols);
    Scratch scr{(char*)h->ws + ob, kScratchBytes};
    if (dVout != dV) TRY(copy_cols<T>(st, n, ncols, dV, ldv, dVout, ldo, &h->launches));
    double fl = 0.0;
    return filter_oz<T>(h, n, A, lda, true, ncols, dVout, ldo, degrees, c, e, lambda1, B, scr, &fl,
                        nullptr);
  }
  if (prec == CHASE_BF16X3) {
    TRY(ensure_ws(h, tc_bytes<T>(n, ncols)));
    TcBufs B = tc_carve<T>((char*)h->ws, n, ncols);
    if (dVout != dV) TRY(copy_cols<T>(st, n, ncols, dV, ldv, dVout, ldo, &h->launches));
    double fl = 0.0;
    return filter_mixed<T>(h, n, A, lda, true, ncols, dVout, ldo, degrees, c, e, lambda1, B, &fl,
                           nullptr);
  }
  const size_t blk = align256(sizeof(T) * (size_t)n * ncols);
  TRY(ensure_ws(h, blk + kScratchBytes));
  T* P = (T*)h->ws;
  Scratch scr{(char*)h->ws + blk, kScratchBytes};
  if (dVout != dV) TRY(copy_cols<T>(st, n, ncols, dV, ldv, dVout, ldo, &h->launches));
  double fl = 0.0;
  TRY(filter_inplace<T>(h, n, A, lda, ncols, dVout, ldo, P, n, degrees, c, e, lambda1, scr, &fl));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  return 0;
}

template <class T>
int qr_impl(chase_ctx* h, int n, int l, T* X, int ldx, double est, int force, chase_precision prec,
            int* variant_used, int* chol_info) {
  cudaStream_t st = h->stream;
  const size_t blk = align256(sizeof(T) * (size_t)n * l);
  const size_t sq = align256(sizeof(T) * (size_t)l * l);
  const bool emu = (prec == CHASE_FP64_EMU || prec == CHASE_BF16X3);
  const size_t fixed = 2 * blk + 2 * sq + kScratchBytes;
  TRY(ensure_ws(h, fixed + (emu ? ozp_bytes<T>(n, l) : 0)));
  char* base = (char*)h->ws;
  T* Xtmp = (T*)base;
  T* Xsave = (T*)(base + blk);
  T* G = (T*)(base + 2 * blk);
  T* Ri = (T*)(base + 2 * blk + sq);
  Scratch scr{base + 2 * blk + 2 * sq, kScratchBytes};
  double lest = (est > 0.0) ? std::log(est) : -1e300;
  if (!std::isfinite(est) && est > 0) lest = 1e300;
  int v = 0, fi = 0;
  OzProd ozp;
  if (emu) ozp = ozp_carve<T>(base + fixed, n, l);
  int rc = qr_dynamic<T>(h, n, l, X, ldx, lest, 1e8, 20.0, force, Xtmp, Xsave, G, Ri, scr, &v, &fi,
                         emu ? &ozp : nullptr);
  if (variant_used) *variant_used = v;
  if (chol_info) *chol_info = fi;
  if (rc && rc != CHASE_CHOL_FAILED) return rc;
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  return rc;
}

int lanczos_entry(chase_ctx* h, chase_dtype dtype, int n, const void* dA, int lda, int nruns,
                  const void* dV0, int ldv, int steps, int ell, chase_bounds* out) {
  const size_t elem = (dtype == CHASE_R64) ? sizeof(double) : sizeof(z64);
  const size_t wb = lanczos_work_bytes(elem, n, nruns, steps);
  TRY(ensure_ws(h, wb + kScratchBytes));
  Scratch scr{(char*)h->ws + wb, kScratchBytes};
  double b[3];
  int rc;
  if (dtype == CHASE_R64)
    rc = lanczos_bounds<double>(h->stream, n, (const double*)dA, lda, nruns, (const double*)dV0, ldv,
                                steps, ell, b, h->ws, wb, scr, &h->launches);
  else
    rc = lanczos_bounds<z64>(h->stream, n, (const z64*)dA, lda, nruns, (const z64*)dV0, ldv, steps,
                             ell, b, h->ws, wb, scr, &h->launches);
  if (rc) return rc;
  out->lambda1 = b[0];
  out->lambda_ell = b[1];
  out->b_sup = b[2];
  return CHASE_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int chase_config_default(chase_config* cfg) {
  if (!cfg) return -1;
  memset(cfg, 0, sizeof(*cfg));
  cfg->tol = 1e-10;
  cfg->max_iter = 25;
  cfg->deg_init = 20;
  cfg->deg_min = 10;
  cfg->deg_max = 36;
  cfg->opt_degree = 1;
  cfg->eta = 1.0;
  cfg->cond_hi = 1e8;
  cfg->cond_lo = 20.0;
  cfg->qr_force = CHASE_QR_AUTO;
  cfg->prec = CHASE_FP64;
  cfg->mp_switch = 1e-3;
  return CHASE_OK;
}

int chase_create(chase_handle* hp, int device, void* cuda_stream) {
  if (!hp) return -1;
  *hp = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? -2 : CHASE_ERR_CUDA;
  }
  chase_ctx* h = new chase_ctx();
  h->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete h; return CHASE_ERR_CUDA; }
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    // a blocking stream: ordered with work on the legacy default stream, so data the
    // caller prepared there is complete before the handle's work reads it
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamDefault) != cudaSuccess) { delete h; return CHASE_ERR_CUDA; }
    h->own_stream = true;
  }
  if (cudaMalloc((void**)&h->dstat, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost((void**)&h->hstat, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    chase_destroy(h);
    return CHASE_ERR_OOM;
  }
  *hp = h;
  return CHASE_OK;
}

int chase_destroy(chase_handle h) {
  if (!h) return -1;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->ws) cudaFree(h->ws);
  if (h->dstat) cudaFree(h->dstat);
  if (h->hstat) cudaFreeHost(h->hstat);
  if (h->hbuf) cudaFreeHost(h->hbuf);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return CHASE_OK;
}

int chase_workspace_bytes(chase_dtype dtype, int n, int nev, int nex, chase_precision prec,
                          size_t* bytes) {
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -1;
  if (n < 1) return -2;
  if (nev < 1) return -3;
  if (nex < 0 || nev + nex > n) return -4;
  if (!bytes) return -6;
  const int l = nev + nex;
  size_t b = (dtype == CHASE_R64) ? layout_for<double>(n, l).total : layout_for<z64>(n, l).total;
  if (prec == CHASE_BF16X3) b += (dtype == CHASE_R64) ? tc_bytes<double>(n, l) : tc_bytes<z64>(n, l);
  if (prec == CHASE_BF16X3 || prec == CHASE_FP64_EMU)
    b += (dtype == CHASE_R64)
             ? align256(oz_bytes<double>(n, l)) + ozp_bytes<double>(n, l)
             : align256(oz_bytes<z64>(n, l)) + ozp_bytes<z64>(n, l);
  *bytes = b;
  return CHASE_OK;
}

int chase_reserve_workspace(chase_handle h, size_t bytes) {
  if (!h) return -1;
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  return ensure_ws(h, bytes);
}

int chase_solve(chase_handle h, chase_dtype dtype, int n, const void* dA, int lda, int nev, int nex,
                const chase_config* cfg, const chase_bounds* bounds, void* dV, int ldv,
                double* evals, double* resid, chase_stats* stats, chase_iter_log* log,
                int log_cap) {
  if (!h) return -1;
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < n) return -5;
  if (nev < 1) return -6;
  if (nex < 0 || nev + nex > n) return -7;
  chase_config c;
  if (cfg) c = *cfg; else chase_config_default(&c);
  if (!(c.tol > 0.0) || c.max_iter < 0 || c.deg_init < 1 || c.deg_min < 1 || c.deg_max < c.deg_min ||
      !(c.eta > 0.0) || c.qr_force < 0 || c.qr_force > 4 || c.cond_est_mode < 0 ||
      c.cond_est_mode > 1 || c.graph_filter < 0 || c.graph_filter > 1 || c.autotune < 0 ||
      c.autotune > 1)
    return -8;
  if (c.prec != CHASE_FP64 && c.prec != CHASE_BF16X3 && c.prec != CHASE_FP64_EMU)
    return CHASE_ERR_UNSUPPORTED;
  if (c.prec == CHASE_BF16X3 && !(c.mp_switch >= 0.0)) return -8;
  if (bounds && (!(bounds->b_sup > bounds->lambda_ell) || !(bounds->lambda_ell >= bounds->lambda1)))
    return -9;
  if (!dV) return -10;
  if (ldv < n) return -11;
  if (!evals) return -12;
  if (!resid) return -13;
  if (log_cap < 0) return -16;
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  chase_bounds bd;
  if (bounds) {
    bd = *bounds;
  } else {
    if (n < 3) return -9;
    const int l = nev + nex;
    const int nruns = std::min(4, l), steps = std::min(25, n - 1);
    int rc = lanczos_entry(h, dtype, n, dA, lda, nruns, dV, ldv, steps, l, &bd);
    if (rc) return rc;
    if (!(bd.b_sup > bd.lambda_ell)) bd.lambda_ell = 0.5 * (bd.lambda1 + bd.b_sup);
  }
  if (dtype == CHASE_R64)
    return solve_impl<double>(h, n, (const double*)dA, lda, nev, nex, c, bd, (double*)dV, ldv,
                              evals, resid, stats, log, log_cap);
  return solve_impl<z64>(h, n, (const z64*)dA, lda, nev, nex, c, bd, (z64*)dV, ldv, evals,
                         resid, stats, log, log_cap);
}

int chase_filter(chase_handle h, chase_dtype dtype, int n, const void* dA, int lda, int ncols,
                 const void* dV, int ldv, const int* degrees, double c, double e, double lambda1,
                 chase_precision prec, void* dVout, int ldvout) {
  if (!h) return -1;
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < n) return -5;
  if (ncols < 0) return -6;
  if (ncols > 0 && !dV) return -7;
  if (ldv < n) return -8;
  if (ncols > 0 && !degrees) return -9;
  for (int a = 0; a < ncols; ++a)
    if (degrees[a] < 0 || (a > 0 && degrees[a] < degrees[a - 1])) return -9;
  if (!(e > 0.0) || !std::isfinite(c)) return -11;
  if (!(lambda1 < c - e)) return -12;
  if (prec != CHASE_FP64 && prec != CHASE_BF16X3 && prec != CHASE_FP64_EMU)
    return CHASE_ERR_UNSUPPORTED;
  if (ncols > 0 && !dVout) return -14;
  if (ldvout < n) return -15;
  if (ncols == 0) return CHASE_OK;
  {
    const size_t elem = (dtype == CHASE_R64) ? sizeof(double) : sizeof(z64);
    if (!output_placement_ok(dVout, ldvout, dV, ldv, dA, lda, n, ncols, elem)) return -14;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  if (dtype == CHASE_R64)
    return filter_impl<double>(h, n, (const double*)dA, lda, ncols, (const double*)dV, ldv, degrees,
                               c, e, lambda1, prec, (double*)dVout, ldvout);
  return filter_impl<z64>(h, n, (const z64*)dA, lda, ncols, (const z64*)dV, ldv, degrees, c, e,
                          lambda1, prec, (z64*)dVout, ldvout);
}

int chase_qr_prec(chase_handle h, chase_dtype dtype, int n, int ncols, void* dX, int ldx,
                  double est_cond, int qr_force, chase_precision prec, int* variant_used,
                  int* chol_info) {
  if (!h) return -1;
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -2;
  if (n < 1) return -3;
  if (ncols < 1 || ncols > n) return -4;
  if (!dX) return -5;
  if (ldx < n) return -6;
  if (std::isnan(est_cond)) return -7;
  if (qr_force < 0 || qr_force > 4) return -8;
  if (prec != CHASE_FP64 && prec != CHASE_FP64_EMU) return -9;
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  if (dtype == CHASE_R64)
    return qr_impl<double>(h, n, ncols, (double*)dX, ldx, est_cond, qr_force, prec, variant_used,
                           chol_info);
  return qr_impl<z64>(h, n, ncols, (z64*)dX, ldx, est_cond, qr_force, prec, variant_used, chol_info);
}

int chase_qr(chase_handle h, chase_dtype dtype, int n, int ncols, void* dX, int ldx,
             double est_cond, int qr_force, int* variant_used, int* chol_info) {
  return chase_qr_prec(h, dtype, n, ncols, dX, ldx, est_cond, qr_force, CHASE_FP64, variant_used,
                       chol_info);
}

int chase_lanczos_bounds(chase_handle h, chase_dtype dtype, int n, const void* dA, int lda,
                         int nruns, const void* dV0, int ldv, int steps, int ell,
                         chase_bounds* out) {
  if (!h) return -1;
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -2;
  if (n < 2) return -3;
  if (!dA) return -4;
  if (lda < n) return -5;
  if (nruns < 1 || nruns > 32) return -6;
  if (!dV0) return -7;
  if (ldv < n) return -8;
  if (steps < 1 || steps >= n || steps > 256) return -9;
  if (ell < 1 || ell > n) return -10;
  if (!out) return -11;
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  return lanczos_entry(h, dtype, n, dA, lda, nruns, dV0, ldv, steps, ell, out);
}

int chase_cond_est(int ell, int nlocked, const double* ritz, const int* degrees, double lambda1,
                   double c, double e, double eta, double* est, double* log_est) {
  if (ell < 1) return -1;
  if (nlocked < 0 || nlocked >= ell) return -2;
  if (!ritz) return -3;
  if (!degrees) return -4;
  if (!(e > 0.0)) return -7;
  if (!(eta > 0.0)) return -8;
  if (!est) return -9;
  const double l = log_cond_est(ritz[nlocked], degrees[nlocked], degrees[ell - 1], lambda1, c, e, eta);
  *est = std::exp(l);
  if (log_est) *log_est = l;
  return CHASE_OK;
}

int chase_batch_create(chase_batch* bp, chase_handle h) {
  if (!bp) return -1;
  *bp = nullptr;
  if (!h) return -2;
  chase_batch_ctx* b = new chase_batch_ctx();
  b->h = h;
  *bp = b;
  return CHASE_OK;
}

int chase_batch_destroy(chase_batch b) {
  if (!b) return -1;
  if (cudaSetDevice(b->h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  delete b;
  return CHASE_OK;
}

int chase_batch_pending(chase_batch b) {
  if (!b) return -1;
  return (int)(b->items.size() + b->finished.size());
}

int chase_batch_add(chase_batch b, chase_dtype dtype, int n, const void* dA, int lda, int nev,
                    int nex, const chase_config* cfg, const chase_bounds* bounds, void* dV, int ldv,
                    double* evals, double* resid, chase_stats* stats, chase_iter_log* log,
                    int log_cap, int* id) {
  if (!b) return -1;
  if (dtype != CHASE_R64 && dtype != CHASE_C128) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < n) return -5;
  if (nev < 1) return -6;
  if (nex < 0 || nev + nex > n) return -7;
  chase_config c;
  if (cfg) c = *cfg; else chase_config_default(&c);
  if (!(c.tol > 0.0) || c.max_iter < 0 || c.deg_init < 1 || c.deg_min < 1 || c.deg_max < c.deg_min ||
      !(c.eta > 0.0) || c.qr_force < 0 || c.qr_force > 4 || c.cond_est_mode < 0 ||
      c.cond_est_mode > 1 || c.graph_filter < 0 || c.graph_filter > 1 || c.autotune < 0 ||
      c.autotune > 1)
    return -8;
  if (c.prec != CHASE_FP64 && c.prec != CHASE_BF16X3 && c.prec != CHASE_FP64_EMU)
    return CHASE_ERR_UNSUPPORTED;
  if (c.prec == CHASE_BF16X3 && !(c.mp_switch >= 0.0)) return -8;
  if (bounds && (!(bounds->b_sup > bounds->lambda_ell) || !(bounds->lambda_ell >= bounds->lambda1)))
    return -9;
  if (!dV) return -10;
  if (ldv < n) return -11;
  if (!evals) return -12;
  if (!resid) return -13;
  if (log_cap < 0) return -16;
  if (!id) return -17;
  chase_ctx* h = b->h;
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  const int l = nev + nex;
  chase_bounds bd;
  if (bounds) {
    bd = *bounds;
  } else {
    if (n < 3) return -9;
    const int nruns = std::min(4, l), steps = std::min(25, n - 1);
    const int rc = lanczos_entry(h, dtype, n, dA, lda, nruns, dV, ldv, steps, l, &bd);
    if (rc) return rc;
    if (!(bd.b_sup > bd.lambda_ell)) bd.lambda_ell = 0.5 * (bd.lambda1 + bd.b_sup);
  }
  chase_batch_ctx::Item it{};
  const size_t wsb = (dtype == CHASE_R64) ? solve_bytes<double>(n, l, c.prec) : solve_bytes<z64>(n, l, c.prec);
  it.sub = b->get_sub();
  if (!it.sub) return CHASE_ERR_CUDA;
  it.ws = b->dev.get(wsb, &it.ws_bytes);
  it.hst = (double*)b->host.get(sizeof(double) * 4 * (size_t)l + 4096, &it.hst_bytes);
  if (!it.ws || !it.hst) {
    b->release(it);
    return CHASE_ERR_OOM;
  }
  {  // the problem's stream starts after what the caller ordered on the handle's stream
    cudaEvent_t r = nullptr;
    if (cudaEventCreateWithFlags(&r, cudaEventDisableTiming) != cudaSuccess) {
      b->release(it);
      return CHASE_ERR_CUDA;
    }
    cudaEventRecord(r, h->stream);
    cudaStreamWaitEvent(it.sub->stream, r, 0);
    cudaEventDestroy(r);
  }
  if (dtype == CHASE_R64)
    it.s = new Solve<double>(it.sub, n, (const double*)dA, lda, nev, nex, c, bd, (double*)dV, ldv,
                             evals, resid, stats, log, log_cap, (char*)it.ws, it.hst);
  else
    it.s = new Solve<z64>(it.sub, n, (const z64*)dA, lda, nev, nex, c, bd, (z64*)dV, ldv, evals,
                          resid, stats, log, log_cap, (char*)it.ws, it.hst);
  const int rc = it.s->begin();
  if (rc) {
    b->release(it);
    return rc;
  }
  it.id = b->next_id++;
  *id = it.id;
  if (it.s->done) {  // max_iter = 0: nothing to iterate
    b->finished.emplace_back(it.id, it.s->finish());
    b->release(it);
    return CHASE_OK;
  }
  b->items.push_back(it);
  return CHASE_OK;
}

int chase_batch_step(chase_batch b, int* done_ids, int* done_status, int cap, int* ndone) {
  if (!b) return -1;
  if (cap < 0 || (cap > 0 && (!done_ids || !done_status))) return -4;
  if (!ndone) return -5;
  *ndone = 0;
  if (cudaSetDevice(b->h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  if (b->finished.empty() && !b->items.empty()) batch_advance(b);
  int m = 0;
  while (m < cap && !b->finished.empty()) {
    done_ids[m] = b->finished.front().first;
    done_status[m] = b->finished.front().second;
    b->finished.erase(b->finished.begin());
    ++m;
  }
  *ndone = m;
  return CHASE_OK;
}

int chase_solve_batch(chase_handle h, int count, const chase_problem* problems,
                      const chase_config* cfg, int* status) {
  if (!h) return -1;
  if (count < 0) return -2;
  if (count > 0 && !problems) return -3;
  if (count > 0 && !status) return -5;
  chase_batch b = nullptr;
  TRY(chase_batch_create(&b, h));
  std::vector<int> idx_of(count, -1);
  std::map<int, int> slot;  // batch id -> problem index
  for (int i = 0; i < count; ++i) {
    const chase_problem& p = problems[i];
    int id = -1;
    status[i] = chase_batch_add(b, p.dtype, p.n, p.dA, p.lda, p.nev, p.nex, cfg, p.bounds, p.dV,
                                p.ldv, p.evals, p.resid, p.stats, nullptr, 0, &id);
    if (status[i] == CHASE_OK) slot[id] = i;
  }
  std::vector<int> ids(count + 1), sts(count + 1);
  while (chase_batch_pending(b) > 0) {
    int nd = 0;
    const int rc = chase_batch_step(b, ids.data(), sts.data(), count + 1, &nd);
    if (rc) {
      chase_batch_destroy(b);
      return rc;
    }
    for (int j = 0; j < nd; ++j) status[slot[ids[j]]] = sts[j];
  }
  chase_batch_destroy(b);
  return CHASE_OK;
}

int chase_selftest_wait_timeout(chase_handle h, double seconds) {
  if (!h) return -1;
  if (!(seconds > 0.0) || seconds > 10.0) return -2;
  if (cudaSetDevice(h->device) != cudaSuccess) return CHASE_ERR_CUDA;
  cudaStream_t st = h->stream;
  CHASE_CUDA_TRY(cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), st));
  TRY(selftest_wait_timeout(st, seconds, h->dstat, &h->launches));
  CHASE_CUDA_TRY(cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  const int timed_out = h->hstat->timeout;
  CHASE_CUDA_TRY(cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), st));
  CHASE_CUDA_TRY(cudaStreamSynchronize(st));
  return timed_out ? CHASE_ERR_TIMEOUT : CHASE_OK;
}

const char* chase_status_string(int status) {
  if (status < 0) return "invalid argument";
  switch (status) {
    case CHASE_OK: return "ok";
    case CHASE_NOT_CONVERGED: return "not converged within max_iter";
    case CHASE_CHOL_FAILED: return "Cholesky factorisation failed";
    case CHASE_ERR_CUDA: return "CUDA error";
    case CHASE_ERR_OOM: return "out of device memory";
    case CHASE_ERR_TIMEOUT: return "device wait timed out";
    case CHASE_ERR_NONFINITE: return "non-finite value in the input";
    case CHASE_ERR_UNSUPPORTED: return "option not supported by this build";
    case CHASE_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of chase_filter_noalloc";
    default: return "unknown status";
  }
}

}  // extern "C"
