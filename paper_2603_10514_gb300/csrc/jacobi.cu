// jacobi.cu -- parallel cyclic Jacobi eigensolver for the reduced problem of the
// Rayleigh-Ritz step (Algorithm 1: solve A~ W = W Lambda~).
//
// Round-robin ordering: in each round the indices 0..L-1 (L = l rounded up to
// even; index l is a dummy when l is odd) form L/2 disjoint pairs, so all L/2
// rotations of a round commute and are applied together.  L - 1 rounds make a
// sweep that visits every pair once.  Per round:
//   1. rotations: for pair (p, q) with g = H_pq = |g| e^{i phi},
//        tau = (H_qq - H_pp) / (2|g|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//        c = 1/sqrt(1 + t^2), s = t c,  J = [[c, s e^{i phi}], [-s e^{-i phi}, c]];
//   2. apply: H <- J^H H J, one thread per 2x2 block (pair_a, pair_b) with a <= b,
//      which also writes block (b, a) as the conjugate transpose (H stays exactly
//      Hermitian, and half the FP64 arithmetic of a full update is spent: the
//      rounds are FP64-bound on GB300, 2 FP64 FMAs per clock per SM), and
//      W <- W J, one thread per (row, pair).
// The whole eigensolve is ONE cooperative kernel: every sweep and round runs inside
// it, the two phases of a round separated by grid-wide barriers (a counter and a
// generation word in global memory).  A launch per phase would cost more than the
// phase itself (~7 us of FP64 work per round at l = 600, complex).  Every barrier
// wait is bounded: a CTA that waits too long raises an abort flag that every other
// CTA sees at its next barrier or while it waits, so the kernel always ends, and
// the host reports CHASE_ERR_TIMEOUT.  Data that other CTAs wrote in an earlier
// phase are read with ld.global.cg (L2, not a possibly stale L1 line).
// Sweeps stop when the off-diagonal Frobenius norm is <= l 2^-53 ||H||_F (the
// rounding level a parallel sweep leaves behind; eigenvalues are then accurate
// to that level by Weyl's inequality) or after max_sweeps; the norms are summed
// over the CTAs' partial sums in a fixed order, so every CTA takes the same
// decision and the result is reproducible.
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

struct Rot {
  int p, q;
  double c;
  double sx, sy;  // s e^{i phi}
};

__device__ inline void pair_of(int L, int round, int i, int& p, int& q) {
  // circle of L-1 players (0..L-2) rotating around a fixed player L-1
  const int m = L - 1;
  if (i == 0) {
    p = m;
    q = round % m;
  } else {
    p = (round + i) % m;
    q = (round - i + m) % m;
  }
  if (p > q) { int t = p; p = q; q = t; }
}

template <class T> __device__ inline T ldcg(const T* p);
template <> __device__ inline double ldcg<double>(const double* p) { return __ldcg(p); }
template <> __device__ inline z64 ldcg<z64>(const z64* p) {
  const double2 v = __ldcg((const double2*)p);
  return z64{v.x, v.y};
}

// Rotation i of round `round` from the current H.
template <class T>
__device__ inline Rot make_rot(int l, int L, int round, int i, const T* H, int ldh) {
  int p, q;
  pair_of(L, round, i, p, q);
  Rot r;
  r.p = p; r.q = q; r.c = 1.0; r.sx = 0.0; r.sy = 0.0;
  if (q < l) {
    T g = ldcg(H + (size_t)p + (size_t)q * ldh);
    double ag = sqrt(Sc<T>::abs2(g));
    if (ag > 0.0) {
      double hpp = Sc<T>::re(ldcg(H + (size_t)p + (size_t)p * ldh));
      double hqq = Sc<T>::re(ldcg(H + (size_t)q + (size_t)q * ldh));
      double tau = (hqq - hpp) / (2.0 * ag);
      double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      r.c = c;
      if constexpr (Sc<T>::cplx) {
        r.sx = s * g.x / ag;
        r.sy = s * g.y / ag;
      } else {
        r.sx = s * (g > 0.0 ? 1.0 : -1.0);
        r.sy = 0.0;
      }
    }
  }
  return r;
}

template <class T> __device__ inline T rot_s(const Rot& r);
template <> __device__ inline double rot_s<double>(const Rot& r) { return r.sx; }
template <> __device__ inline z64 rot_s<z64>(const Rot& r) { return z64{r.sx, r.sy}; }

__device__ inline Rot load_rot(const Rot* r) {
  Rot o;
  o.p = __ldcg(&r->p); o.q = __ldcg(&r->q);
  o.c = __ldcg(&r->c); o.sx = __ldcg(&r->sx); o.sy = __ldcg(&r->sy);
  return o;
}

// Work item t of a round's update: t < np^2 is the 2x2 block (pair a rows, pair b columns)
// of H <- J^H H J (a <= b; block (b, a) is written as its conjugate transpose), the
// others (row i, pair b) of W <- W J.
template <class T>
__device__ inline void apply_item(long long t, int l, int np, const Rot* __restrict__ rots, T* H,
                                  int ldh, T* W, int ldw) {
  const long long nblk = (long long)np * np;
  if (t < nblk) {
    const int a = (int)(t % np), b = (int)(t / np);
    if (a > b) return;  // written by block (b, a) as its conjugate transpose
    const Rot ra = load_rot(rots + a), rb = load_rot(rots + b);
    const int pa = ra.p, qa = ra.q, pb = rb.p, qb = rb.q;
    const bool va = qa < l, vb = qb < l;
    // load the 2x2 block (dummy index -> zero row/column, never stored)
    T h_pp = ldcg(H + (size_t)pa + (size_t)pb * ldh);
    T h_qp = va ? ldcg(H + (size_t)qa + (size_t)pb * ldh) : Sc<T>::zero();
    T h_pq = vb ? ldcg(H + (size_t)pa + (size_t)qb * ldh) : Sc<T>::zero();
    T h_qq = (va && vb) ? ldcg(H + (size_t)qa + (size_t)qb * ldh) : Sc<T>::zero();
    // right: [col p, col q] J_b = [c col_p - conj(s) col_q, s col_p + c col_q]
    const double cb = rb.c;
    const T sb = rot_s<T>(rb), sbc = Sc<T>::conj(sb);
    T r_pp = Sc<T>::sub(Sc<T>::scale(h_pp, cb), Sc<T>::mul(h_pq, sbc));
    T r_qp = Sc<T>::sub(Sc<T>::scale(h_qp, cb), Sc<T>::mul(h_qq, sbc));
    T r_pq = Sc<T>::add(Sc<T>::mul(h_pp, sb), Sc<T>::scale(h_pq, cb));
    T r_qq = Sc<T>::add(Sc<T>::mul(h_qp, sb), Sc<T>::scale(h_qq, cb));
    // left: J_a^H [row p; row q] = [c row_p - s row_q; conj(s) row_p + c row_q]
    const double ca = ra.c;
    const T sa = rot_s<T>(ra), sac = Sc<T>::conj(sa);
    T o_pp = Sc<T>::sub(Sc<T>::scale(r_pp, ca), Sc<T>::mul(sa, r_qp));
    T o_pq = Sc<T>::sub(Sc<T>::scale(r_pq, ca), Sc<T>::mul(sa, r_qq));
    T o_qp = Sc<T>::add(Sc<T>::mul(sac, r_pp), Sc<T>::scale(r_qp, ca));
    T o_qq = Sc<T>::add(Sc<T>::mul(sac, r_pq), Sc<T>::scale(r_qq, ca));
    if (a == b) {  // the rotated pair itself: exact zero off-diagonal, real diagonal
      o_pq = Sc<T>::zero();
      o_qp = Sc<T>::zero();
      o_pp = Sc<T>::from_re(Sc<T>::re(o_pp));
      o_qq = Sc<T>::from_re(Sc<T>::re(o_qq));
    }
    H[(size_t)pa + (size_t)pb * ldh] = o_pp;
    if (va) H[(size_t)qa + (size_t)pb * ldh] = o_qp;
    if (vb) H[(size_t)pa + (size_t)qb * ldh] = o_pq;
    if (va && vb) H[(size_t)qa + (size_t)qb * ldh] = o_qq;
    if (a != b) {  // mirror: rows of pair b, columns of pair a
      H[(size_t)pb + (size_t)pa * ldh] = Sc<T>::conj(o_pp);
      if (va) H[(size_t)pb + (size_t)qa * ldh] = Sc<T>::conj(o_qp);
      if (vb) H[(size_t)qb + (size_t)pa * ldh] = Sc<T>::conj(o_pq);
      if (va && vb) H[(size_t)qb + (size_t)qa * ldh] = Sc<T>::conj(o_qq);
    }
  } else {
    const long long u = t - nblk;
    const int i = (int)(u % l), b = (int)(u / l);
    const Rot rb = load_rot(rots + b);
    if (rb.q >= l) return;
    const double cb = rb.c;
    const T sb = rot_s<T>(rb), sbc = Sc<T>::conj(sb);
    T* wp = W + (size_t)i + (size_t)rb.p * ldw;
    T* wq = W + (size_t)i + (size_t)rb.q * ldw;
    T xp = ldcg(wp), xq = ldcg(wq);
    *wp = Sc<T>::sub(Sc<T>::scale(xp, cb), Sc<T>::mul(xq, sbc));
    *wq = Sc<T>::add(Sc<T>::mul(xp, sb), Sc<T>::scale(xq, cb));
  }
}

// Grid-wide barrier of a cooperative launch, bounded: returns false (and the caller leaves
// the kernel) when the wait ran out or another CTA gave up.
struct GridBar {
  unsigned count;
  unsigned gen;
  int abort;
  int sweeps;
};
constexpr long long kBarWait = 2000000000LL;  // ~1 s of clock64

__device__ bool grid_barrier(GridBar* gb, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (nblocks == 1) return true;  // one CTA: the block barrier orders its global writes
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gb->gen;
    volatile int* vab = &gb->abort;
    int ok = 1;
    const unsigned g = *vgen;
    __threadfence();
    if (*vab) {
      ok = 0;
    } else if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*vab) { ok = 0; break; }
        if (clock64() - t0 > kBarWait) { atomicExch(&gb->abort, 1); ok = 0; break; }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The whole cyclic Jacobi iteration: sweeps until ||off(H)||_F <= l u ||H||_F or
// max_sweeps.  partial: 2 doubles per CTA.  gb->sweeps receives the sweep count.
template <class T>
__global__ void __launch_bounds__(256) jacobi_sweeps_kernel(int l, int L, T* H, int ldh, T* W,
                                                            int ldw, Rot* rots, double* partial,
                                                            GridBar* gb, int max_sweeps) {
  const unsigned G = gridDim.x;
  const int np = L / 2;
  const long long items = (long long)np * np + (long long)l * np;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)G * blockDim.x;
  __shared__ double r0[8], r1[8];
  const double tolr = 1.1102230246251565e-16 * (double)l;
  int sw = 0;
  for (; sw <= max_sweeps; ++sw) {
    // ||off(H)||_F^2 and ||H||_F^2: partial sums per CTA, then the same fixed-order total
    // in every CTA
    double off = 0.0, all = 0.0;
    const size_t total = (size_t)l * l;
    for (size_t t = gtid; t < total; t += (size_t)gstride) {
      const int i = (int)(t % l), j = (int)(t / l);
      const double a = Sc<T>::abs2(ldcg(H + (size_t)i + (size_t)j * ldh));
      all += a;
      if (i != j) off += a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { r0[warp] = off; r1[warp] = all; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r0[w]; b += r1[w]; }
      partial[2 * blockIdx.x] = a;
      partial[2 * blockIdx.x + 1] = b;
    }
    if (!grid_barrier(gb, G)) return;
    double so = 0.0, sa = 0.0;
    for (unsigned b = 0; b < G; ++b) { so += __ldcg(partial + 2 * b); sa += __ldcg(partial + 2 * b + 1); }
    if (so <= tolr * tolr * sa || so == 0.0 || sw == max_sweeps) break;
    for (int r = 0; r < L - 1; ++r) {
      // rotations, spread over the CTAs (their FP64 square roots and divisions)
      for (int i = blockIdx.x + G * threadIdx.x; i < np; i += G * blockDim.x)
        rots[i] = make_rot<T>(l, L, r, i, H, ldh);
      if (!grid_barrier(gb, G)) return;
      for (long long t = gtid; t < items; t += gstride) apply_item<T>(t, l, np, rots, H, ldh, W, ldw);
      if (!grid_barrier(gb, G)) return;
    }
    // the partial sums of the next check are written after two more barriers: no CTA
    // still reads this sweep's values by then
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) gb->sweeps = sw;
}

template <class T>
__global__ void jacobi_init_kernel(int l, T* W, int ldw) {
  size_t total = (size_t)l * l;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % l), j = (int)(t / l);
    W[(size_t)i + (size_t)j * ldw] = (i == j) ? Sc<T>::one() : Sc<T>::zero();
  }
}

// Sort eigenvalues ascending (single CTA, rank by counting: ties broken by index)
// and permute W's columns accordingly into Wout.
template <class T>
__global__ void __launch_bounds__(1024) jacobi_sort_kernel(int l, const T* H, int ldh,
                                                           const T* W, int ldw, double* dw,
                                                           int* perm) {
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    double di = Sc<T>::re(H[(size_t)i + (size_t)i * ldh]);
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      double dj = Sc<T>::re(H[(size_t)j + (size_t)j * ldh]);
      rank += (dj < di) || (dj == di && j < i);
    }
    dw[rank] = di;
    perm[rank] = i;
  }
}

template <class T>
__global__ void permute_cols_kernel(int l, const T* W, int ldw, const int* perm, T* Wout,
                                    int ldo) {
  size_t total = (size_t)l * l;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(t % l), j = (int)(t / l);
    Wout[(size_t)i + (size_t)j * ldo] = W[(size_t)i + (size_t)perm[j] * ldw];
  }
}

}  // namespace

size_t jacobi_work_bytes(int l, size_t elem) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int L = (l % 2) ? l + 1 : l;
  return al(sizeof(Rot) * (size_t)(L / 2 + 1)) + al(sizeof(GridBar)) + al(16 * (size_t)kJacobiMaxCtas) +
         al(sizeof(int) * (size_t)l) + al(elem * (size_t)l * l);
}

template <class T>
int jacobi_eig(cudaStream_t st, int l, T* H, int ldh, T* W, int ldw, double* dw, void* work,
               size_t work_bytes, int max_sweeps, int* sweeps, int* launches) {
  if (l <= 0) return 0;
  const int L = (l % 2) ? l + 1 : l;
  if (jacobi_work_bytes(l, sizeof(T)) > work_bytes) return 4;  // CHASE_ERR_OOM
  // workspace: rotations | barrier | per-CTA norm partials | permutation | W copy
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* base = (char*)work;
  Rot* rots = (Rot*)base;
  base += al(sizeof(Rot) * (size_t)(L / 2 + 1));
  GridBar* gb = (GridBar*)base;
  base += al(sizeof(GridBar));
  double* partial = (double*)base;
  base += al(16 * (size_t)kJacobiMaxCtas);
  int* dperm = (int*)base;
  base += al(sizeof(int) * (size_t)l);
  T* Wtmp = (T*)base;
  int nl = 0;
  int blocks = std::min(ceil_div((long long)l * l, 256), kNumSMs * 8);
  jacobi_init_kernel<T><<<blocks, 256, 0, st>>>(l, W, ldw);
  ++nl;
  int sw = 0;
  if (l > 1) {
    // CTAs: about 4 work items of a round per thread, at most one wave of co-resident CTAs
    static int max_coresident[2] = {0, 0};
    int& mc = max_coresident[Sc<T>::cplx ? 1 : 0];
    if (mc == 0) {
      int per_sm = 0;
      CHASE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_sweeps_kernel<T>, 256, 0));
      mc = std::max(1, std::min(per_sm * kNumSMs, kJacobiMaxCtas));
    }
    const long long items = (long long)(L / 2) * (L / 2) + (long long)l * (L / 2);
    const int G = std::max(1, std::min(mc, ceil_div(items, 256 * 4)));
    CHASE_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), st));
    int ms = max_sweeps;
    void* args[] = {(void*)&l, (void*)&L, (void*)&H, (void*)&ldh, (void*)&W, (void*)&ldw, (void*)&rots,
                    (void*)&partial, (void*)&gb, (void*)&ms};
    CHASE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_sweeps_kernel<T>, dim3(G), dim3(256),
                                               args, 0, st));
    ++nl;
    GridBar hb{};
    CHASE_CUDA_TRY(cudaMemcpyAsync(&hb, gb, sizeof(GridBar), cudaMemcpyDeviceToHost, st));
    CHASE_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb.abort) {
      if (launches) *launches += nl;
      return 5;  // CHASE_ERR_TIMEOUT
    }
    sw = hb.sweeps;
  }
  jacobi_sort_kernel<T><<<1, 1024, 0, st>>>(l, H, ldh, W, ldw, dw, dperm);
  ++nl;
  CHASE_CUDA_TRY(cudaMemcpy2DAsync(Wtmp, sizeof(T) * (size_t)l, W, sizeof(T) * (size_t)ldw,
                                   sizeof(T) * (size_t)l, l, cudaMemcpyDeviceToDevice, st));
  permute_cols_kernel<T><<<blocks, 256, 0, st>>>(l, Wtmp, l, dperm, W, ldw);
  ++nl;
  if (sweeps) *sweeps = sw;
  if (launches) *launches += nl;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template int jacobi_eig<double>(cudaStream_t, int, double*, int, double*, int, double*, void*,
                                size_t, int, int*, int*);
template int jacobi_eig<z64>(cudaStream_t, int, z64*, int, z64*, int, double*, void*, size_t, int,
                             int*, int*);

}  // namespace chase
