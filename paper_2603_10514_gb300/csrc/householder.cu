// householder.cu -- Householder QR with explicit thin Q: the fallback of
// Algorithm 3 when even the shifted Cholesky factorisation fails.
//
// Column j: reflector v = x - alpha e_1 (x = X[j:, j], alpha = -e^{i arg x_0}
// ||x||), normalised, stored in Vh[:, j]; H_j = I - 2 v v^H.
//
// Two forms.  Unblocked (householder_qr, small l): each reflector is applied to
// the whole trailing block (one CTA per column: block-reduced dot product, then
// axpy) and Q = H_0 ... H_{l-1} [I; 0] is accumulated backwards the same way.
// Blocked (the compact WY form, driven from solver.cu): a panel of b columns is
// factored with the same kernels restricted to the panel (hh_panel), its
// reflectors are gathered as H_{j0} ... H_{j0+b-1} = I - V T V^H with T upper
// triangular (hh_build_T, from the panel's Gram V^H V), and the trailing
// columns and later the explicit Q are updated by matrix products
// (C <- C - V T^H (V^H C), Q <- Q - V T (V^H Q)), which run on the block-product
// engines (FP64 or the emulated-FP64 tensor-core products).
#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

constexpr int HT = 256;
constexpr int kHhSliceMax = 512;  // rows of a CTA's slice in the cooperative panel kernel

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

// One panel factored by a cooperative grid (the blocked form's panel step in one launch).
// The panel's rows [j0, n) are split into G contiguous slices, one per CTA; element (r, q)
// of the panel is always read and written by the same thread (warp q mod 8, the lane of
// row r), so the CTA needs no synchronisation on X.  Per column j = j0 + jj:
//   1. the warp of column j sums |X[r, j]|^2 over its slice's rows r >= j; grid barrier;
//   2. every CTA sums the G partial norms in the same fixed order, forms the reflector
//      v = (x - alpha e_j) / ||x - alpha e_j|| for its rows, writes it to Vh and to shared
//      memory; each warp forms the slice's partial dots v^H X[:, q] of its columns q > j;
//      grid barrier;
//   3. the dots are summed in the same fixed order everywhere and X[:, q] -= 2 v (v^H X[:, q]).
// Then every CTA adds its slice's part of the panel Gram V^H V (upper triangle); after a
// last barrier CTA 0 sums the G parts into G (b x b, ld ldg).  Vh rows < j0 of the panel
// are zeroed.  Scratch (ws): G (1 + b + b(b+1)/2) values of T plus one T for x_j.  Every
// wait is bounded (grid_barrier): on expiry the kernel raises gb->abort and returns.
template <class T>
__global__ void __launch_bounds__(256) hh_panel_coop_kernel(int n, int j0, int b, T* X, int ldx,
                                                            T* Vh, int ldv, T* Gp, int ldg, T* ws,
                                                            GridBar* gb, DevStatus* status) {
  __shared__ T vsl[kHhSliceMax];
  const unsigned G = gridDim.x;
  const int c = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = n - j0, R = (m + (int)G - 1) / (int)G;
  const int g0 = j0 + c * R, g1 = min(n, g0 + R);
  const int nent = b * (b + 1) / 2;
  double* pnorm = (double*)ws;                  // [G]
  T* x0slot = (T*)(pnorm + ((G + 1) & ~1u));    // [1]
  T* pdot = x0slot + 2;                         // [G][b]
  T* pgram = pdot + (size_t)G * b;              // [G][nent]
  unsigned k = 0;

  // the panel's reflectors vanish above row j0
  for (size_t t = (size_t)c * blockDim.x + threadIdx.x; t < (size_t)j0 * b; t += (size_t)G * blockDim.x)
    Vh[(t % j0) + (t / j0 + j0) * (size_t)ldv] = Sc<T>::zero();

  for (int jj = 0; jj < b; ++jj) {
    const int j = j0 + jj;
    T* xj = X + (size_t)j * ldx;
    if (warp == (jj & 7)) {
      double sq = 0.0;
      for (int r = max(g0, j) + lane; r < g1; r += 32) sq += Sc<T>::abs2(xj[r]);
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) pnorm[c] = sq;
      if (j >= g0 && j < g1 && lane == ((j - g0) & 31)) *x0slot = xj[j];
    }
    if (!grid_barrier(gb, G, k)) { if (threadIdx.x == 0) atomicOr(&status->timeout, 16); return; }
    if (warp == (jj & 7)) {
      double sq = 0.0;
      for (int i = lane; i < (int)G; i += 32) sq += __ldcg(pnorm + i);
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      const double nx2 = __shfl_sync(0xffffffffu, sq, 0);
      T x0;
      if constexpr (Sc<T>::cplx) x0 = z64{__ldcg(&x0slot->x), __ldcg(&x0slot->y)};
      else x0 = __ldcg((const double*)x0slot);
      const double ax0 = sqrt(Sc<T>::abs2(x0));
      const double nx = sqrt(nx2);
      const T ph = (ax0 == 0.0) ? Sc<T>::one() : Sc<T>::scale(x0, 1.0 / ax0);
      const T alpha = Sc<T>::scale(ph, -nx);
      const T v0 = Sc<T>::sub(x0, alpha);
      const double nv2 = nx2 - ax0 * ax0 + Sc<T>::abs2(v0);
      const double inv = (nx == 0.0 || nv2 <= 0.0) ? 0.0 : 1.0 / sqrt(nv2);
      T* vj = Vh + (size_t)j * ldv;
      for (int r = g0 + lane; r < g1; r += 32) {
        T val;
        if (r < j) val = Sc<T>::zero();
        else if (r == j) val = Sc<T>::scale(v0, inv);
        else val = Sc<T>::scale(xj[r], inv);
        vsl[r - g0] = val;
        vj[r] = val;
      }
    }
    __syncthreads();
    if (jj + 1 == b) break;
    for (int q = jj + 1; q < b; ++q) {
      if ((q & 7) != warp) continue;
      const T* xq = X + (size_t)(j0 + q) * ldx;
      T d = Sc<T>::zero();
      for (int r = max(g0, j) + lane; r < g1; r += 32) Sc<T>::fmac(d, vsl[r - g0], xq[r]);
      if constexpr (Sc<T>::cplx) {
        for (int o = 16; o > 0; o >>= 1) {
          d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
          d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
        }
      } else {
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      }
      if (lane == 0) pdot[(size_t)c * b + q] = d;
    }
    if (!grid_barrier(gb, G, k)) { if (threadIdx.x == 0) atomicOr(&status->timeout, 16); return; }
    for (int q = jj + 1; q < b; ++q) {
      if ((q & 7) != warp) continue;
      T d = Sc<T>::zero();
      for (int i = lane; i < (int)G; i += 32) {
        const T* pi = pdot + (size_t)i * b + q;
        if constexpr (Sc<T>::cplx) d = Sc<T>::add(d, z64{__ldcg(&pi->x), __ldcg(&pi->y)});
        else d += __ldcg((const double*)pi);
      }
      if constexpr (Sc<T>::cplx) {
        for (int o = 16; o > 0; o >>= 1) {
          d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
          d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
        }
        d.x = __shfl_sync(0xffffffffu, d.x, 0);
        d.y = __shfl_sync(0xffffffffu, d.y, 0);
      } else {
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d = __shfl_sync(0xffffffffu, d, 0);
      }
      const T d2 = Sc<T>::scale(d, 2.0);
      T* xq = X + (size_t)(j0 + q) * ldx;
      for (int r = max(g0, j) + lane; r < g1; r += 32)
        xq[r] = Sc<T>::sub(xq[r], Sc<T>::mul(vsl[r - g0], d2));
    }
  }
  // the slice's part of V^H V (upper triangle, packed by columns)
  __syncthreads();
  for (int e = threadIdx.x; e < nent; e += blockDim.x) {
    int q = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((q + 1) * (q + 2) / 2 <= e) ++q;
    while (q * (q + 1) / 2 > e) --q;
    const int p = e - q * (q + 1) / 2;
    const T* vp = Vh + (size_t)(j0 + p) * ldv;
    const T* vq = Vh + (size_t)(j0 + q) * ldv;
    T acc = Sc<T>::zero();
    for (int r = g0; r < g1; ++r) Sc<T>::fmac(acc, vp[r], vq[r]);
    pgram[(size_t)c * nent + e] = acc;
  }
  if (!grid_barrier(gb, G, k)) { if (threadIdx.x == 0) atomicOr(&status->timeout, 16); return; }
  if (c != 0) return;
  for (int e = threadIdx.x; e < nent; e += blockDim.x) {
    int q = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((q + 1) * (q + 2) / 2 <= e) ++q;
    while (q * (q + 1) / 2 > e) --q;
    const int p = e - q * (q + 1) / 2;
    T acc = Sc<T>::zero();
    for (unsigned i = 0; i < G; ++i) {
      const T* pi = pgram + (size_t)i * nent + e;
      if constexpr (Sc<T>::cplx) acc = Sc<T>::add(acc, z64{__ldcg(&pi->x), __ldcg(&pi->y)});
      else acc += __ldcg((const double*)pi);
    }
    Gp[(size_t)p + (size_t)q * ldg] = acc;
  }
}

// Compact WY factor of one panel: T (b x b, upper) with H_0 ... H_{b-1} = I - V T V^H for
// unit reflectors (tau = 2), from G = V^H V (upper triangle read):
//   T[j, j] = 2,  T[0:j, j] = -2 T[0:j, 0:j] G[0:j, j].
// Row i of T depends only on row i (T is upper triangular), so thread i computes it alone.
template <class T>
__global__ void hh_build_T_kernel(int b, const T* __restrict__ G, int ldg, T* Tm, int ldt) {
  extern __shared__ unsigned char hh_smem[];
  T* sG = (T*)hh_smem;          // b x b (ld b), upper triangle
  T* sT = sG + (size_t)b * b;   // b x b (ld b): row i belongs to thread i
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
    const int p = t % b, q = t / b;
    sG[t] = (p < q) ? G[(size_t)p + (size_t)q * ldg] : Sc<T>::zero();
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i < b) {
    for (int j = 0; j < i; ++j) sT[i + j * b] = Sc<T>::zero();
    sT[i + i * b] = Sc<T>::scale(Sc<T>::one(), 2.0);
    for (int j = i + 1; j < b; ++j) {
      T acc = Sc<T>::zero();
      for (int k = i; k < j; ++k) acc = Sc<T>::add(acc, Sc<T>::mul(sT[i + k * b], sG[k + j * b]));
      sT[i + j * b] = Sc<T>::scale(acc, -2.0);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) Tm[(size_t)(t % b) + (size_t)(t / b) * ldt] = sT[t];
}

}  // namespace

template <class T>
int hh_panel(cudaStream_t st, int n, int j0, int b, T* X, int ldx, T* Vh, int ldv, int* launches) {
  int nl = 0;
  for (int jj = 0; jj < b; ++jj) {
    const int j = j0 + jj;
    hh_reflector_kernel<T><<<1, HT, 0, st>>>(n, j, X, ldx, Vh, ldv);
    ++nl;
    if (jj + 1 < b) {
      hh_apply_kernel<T><<<b - jj - 1, HT, 0, st>>>(n, j, j + 1, X, ldx, Vh, ldv);
      ++nl;
    }
  }
  if (launches) *launches += nl;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
size_t hh_panel_coop_bytes(int b) {
  const size_t nent = (size_t)b * (b + 1) / 2;
  return 256 + 8 * (size_t)(kJacobiMaxCtas + 2) + 2 * sizeof(T) +
         (size_t)kJacobiMaxCtas * ((size_t)b + nent) * sizeof(T);
}

template <class T>
int hh_panel_coop(cudaStream_t st, int n, int j0, int b, T* X, int ldx, T* Vh, int ldv, T* Gp, int ldg,
                  Scratch ws, DevStatus* dst, int* launches) {
  static const int per_sm = [] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, hh_panel_coop_kernel<T>, 256, 0) != cudaSuccess) {
      cudaGetLastError();  // the caller falls back to the per-column panel; no stale error left
      v = 0;
    }
    return v;
  }();
  const int m = n - j0;
  const int Gmax = per_sm * kNumSMs;
  const int G = std::min(kNumSMs, std::max(ceil_div(m, kHhSliceMax), ceil_div(m, 64)));
  if (b > 64 || per_sm <= 0 || G > Gmax || G > kJacobiMaxCtas || ceil_div(m, G) > kHhSliceMax ||
      ws.bytes < hh_panel_coop_bytes<T>(b))
    return CHASE_ERR_UNSUPPORTED;
  GridBar* gb = (GridBar*)ws.ptr;
  T* w = (T*)((char*)ws.ptr + 256);
  CHASE_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), st));
  void* args[] = {&n, &j0, &b, &X, &ldx, &Vh, &ldv, &Gp, &ldg, &w, &gb, &dst};
  CHASE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)hh_panel_coop_kernel<T>, dim3(G), dim3(256),
                                             args, 0, st));
  if (launches) ++*launches;
  return 0;
}

template <class T>
int hh_build_T(cudaStream_t st, int b, const T* G, int ldg, T* Tm, int ldt, int* launches) {
  if (b <= 0) return 0;
  if (b > 64) return CHASE_ERR_UNSUPPORTED;
  const int smem = 2 * b * b * (int)sizeof(T);
  static const bool attr = cudaFuncSetAttribute(hh_build_T_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                2 * 64 * 64 * (int)sizeof(T)) == cudaSuccess;
  if (!attr) return CHASE_ERR_CUDA;
  hh_build_T_kernel<T><<<1, 64, smem, st>>>(b, G, ldg, Tm, ldt);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int hh_thin_identity(cudaStream_t st, int n, int l, T* X, int ldx, int* launches) {
  const int blocks = std::min(ceil_div((long long)n * l, 256), kNumSMs * 8);
  set_thin_identity_kernel<T><<<blocks, 256, 0, st>>>(n, l, X, ldx);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

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
#define HH_INST(T)                                                                          \
  template int hh_panel<T>(cudaStream_t, int, int, int, T*, int, T*, int, int*);           \
  template int hh_panel_coop<T>(cudaStream_t, int, int, int, T*, int, T*, int, T*, int,    \
                                Scratch, DevStatus*, int*);                                \
  template int hh_build_T<T>(cudaStream_t, int, const T*, int, T*, int, int*);             \
  template int hh_thin_identity<T>(cudaStream_t, int, int, T*, int, int*);
HH_INST(double)
HH_INST(z64)
#undef HH_INST

}  // namespace chase
