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

struct __align__(16) Rot {
  int p, q;
  double c;
  double sx, sy;  // s e^{i phi}
};
static_assert(sizeof(Rot) == 32, "two 16-byte loads");

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

template <class T> __device__ inline T rot_s(const Rot& r);
template <> __device__ inline double rot_s<double>(const Rot& r) { return r.sx; }
template <> __device__ inline z64 rot_s<z64>(const Rot& r) { return z64{r.sx, r.sy}; }

// Rotation annihilating g = H_pq from the entries H_pp, H_qq, H_pq of the current H; the
// identity (c = 1, s = 0 exactly) when |g|^2 <= thr2 (threshold Jacobi: an entry of at most
// u ||H||_F left in place keeps the off-diagonal norm within the stopping level l u ||H||_F).
template <class T>
__device__ inline Rot rot_from(int p, int q, double hpp, double hqq, T g, double thr2) {
  Rot r;
  r.p = p; r.q = q; r.c = 1.0; r.sx = 0.0; r.sy = 0.0;
  const double ag2 = Sc<T>::abs2(g);
  double ag = sqrt(ag2);
  if (ag > 0.0 && ag2 > thr2) {
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
  return r;
}

__device__ inline bool rot_identity(const Rot& r) { return r.c == 1.0 && r.sx == 0.0 && r.sy == 0.0; }

__device__ inline Rot load_rot(const Rot* r) {  // two 16-byte loads through L2
  const int4 a = __ldcg((const int4*)r);
  const double2 b = __ldcg((const double2*)r + 1);
  Rot o;
  o.p = a.x;
  o.q = a.y;
  o.c = __hiloint2double(a.w, a.z);
  o.sx = b.x;
  o.sy = b.y;
  return o;
}

// The 2x2 block (rows of pair a, columns of pair b) of J^H H J: loads the block of the
// current H (Hc, ld ldc; a dummy index gives a zero row / column) and returns
// o = {o_pp, o_qp, o_pq, o_qq}.  Used by the owner of the block and, for three entries,
// by the threads that form the next round's rotations: the same arithmetic, so the same
// values.
template <class T>
__device__ inline void block_update(int l, const Rot& ra, const Rot& rb, const T* Hc, int ldc, T* o) {
  const int pa = ra.p, qa = ra.q, pb = rb.p, qb = rb.q;
  const bool va = qa < l, vb = qb < l;
  T h_pp = ldcg(Hc + (size_t)pa + (size_t)pb * ldc);
  T h_qp = va ? ldcg(Hc + (size_t)qa + (size_t)pb * ldc) : Sc<T>::zero();
  T h_pq = vb ? ldcg(Hc + (size_t)pa + (size_t)qb * ldc) : Sc<T>::zero();
  T h_qq = (va && vb) ? ldcg(Hc + (size_t)qa + (size_t)qb * ldc) : Sc<T>::zero();
  if (rot_identity(ra) && rot_identity(rb)) {  // both rotations skipped: the block is unchanged
    o[0] = h_pp; o[1] = h_qp; o[2] = h_pq; o[3] = h_qq;
    return;
  }
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
  o[0] = Sc<T>::sub(Sc<T>::scale(r_pp, ca), Sc<T>::mul(sa, r_qp));
  o[2] = Sc<T>::sub(Sc<T>::scale(r_pq, ca), Sc<T>::mul(sa, r_qq));
  o[1] = Sc<T>::add(Sc<T>::mul(sac, r_pp), Sc<T>::scale(r_qp, ca));
  o[3] = Sc<T>::add(Sc<T>::mul(sac, r_pq), Sc<T>::scale(r_qq, ca));
  if (ra.p == rb.p) {  // the rotated pair itself: exact zero off-diagonal, real diagonal
    o[2] = Sc<T>::zero();
    o[1] = Sc<T>::zero();
    o[0] = Sc<T>::from_re(Sc<T>::re(o[0]));
    o[3] = Sc<T>::from_re(Sc<T>::re(o[3]));
  }
}

// Index of the pair that holds x in round `round` (inverse of pair_of).
__device__ inline int pair_index(int L, int round, int x) {
  const int m = L - 1;
  if (x == m || x == round % m) return 0;
  const int d = ((x - round) % m + m) % m;  // 1 .. m - 1
  return d <= (m - 1) / 2 ? d : m - d;
}

// The next round's rotation for pair (p, q), from the entries (p, p), (q, q), (p, q) of the
// next H formed exactly as their blocks' owners form them: both rotations are loaded once,
// then the three 2x2 blocks' loads are independent of one another (two dependent L2 round
// trips in all, not six).
template <class T>
__device__ inline Rot next_rotation(int l, int L, int round, const Rot* rots, const T* Hc, int ldc,
                                    int p, int q, double thr2) {
  const int ap = pair_index(L, round, p), aq = pair_index(L, round, q);
  const Rot rp = load_rot(rots + ap), rq = load_rot(rots + aq);
  T opp[4], oqq[4], opq[4];
  block_update<T>(l, rp, rp, Hc, ldc, opp);
  block_update<T>(l, rq, rq, Hc, ldc, oqq);
  if (ap <= aq) block_update<T>(l, rp, rq, Hc, ldc, opq);
  else block_update<T>(l, rq, rp, Hc, ldc, opq);
  const double hpp = Sc<T>::re(p == rp.p ? opp[0] : opp[3]);
  const double hqq = Sc<T>::re(q == rq.p ? oqq[0] : oqq[3]);
  // block (a, b) holds rows {ra.p, ra.q} x columns {rb.p, rb.q}; (p, q) or its mirror
  T g;
  if (ap <= aq) {
    g = (p == rp.p) ? (q == rq.p ? opq[0] : opq[2]) : (q == rq.p ? opq[1] : opq[3]);
  } else {
    const T v = (q == rq.p) ? (p == rp.p ? opq[0] : opq[2]) : (p == rp.p ? opq[1] : opq[3]);
    g = Sc<T>::conj(v);
  }
  return rot_from<T>(p, q, hpp, hqq, g, thr2);
}

// Work item t of a round's update, from the current H (Hc) into the next (Hn): t < np^2
// is the 2x2 block (pair a rows, pair b columns) of J^H H J (a <= b; block (b, a) is
// written as its conjugate transpose); the others (row i, pair b) of W <- W J in place.
template <class T>
__device__ inline void apply_item(long long t, int l, int np, const Rot* __restrict__ rots,
                                  const T* Hc, int ldc, T* Hn, int ldn, T* W, int ldw) {
  const long long nblk = (long long)np * np;
  if (t < nblk) {
    const int a = (int)(t % np), b = (int)(t / np);
    if (a > b) return;  // written by block (b, a) as its conjugate transpose
    const Rot ra = load_rot(rots + a), rb = load_rot(rots + b);
    T o[4];
    block_update<T>(l, ra, rb, Hc, ldc, o);
    const int pa = ra.p, qa = ra.q, pb = rb.p, qb = rb.q;
    const bool va = qa < l, vb = qb < l;
    Hn[(size_t)pa + (size_t)pb * ldn] = o[0];
    if (va) Hn[(size_t)qa + (size_t)pb * ldn] = o[1];
    if (vb) Hn[(size_t)pa + (size_t)qb * ldn] = o[2];
    if (va && vb) Hn[(size_t)qa + (size_t)qb * ldn] = o[3];
    if (a != b) {  // mirror: rows of pair b, columns of pair a
      Hn[(size_t)pb + (size_t)pa * ldn] = Sc<T>::conj(o[0]);
      if (va) Hn[(size_t)pb + (size_t)qa * ldn] = Sc<T>::conj(o[1]);
      if (vb) Hn[(size_t)qb + (size_t)pa * ldn] = Sc<T>::conj(o[2]);
      if (va && vb) Hn[(size_t)qb + (size_t)qa * ldn] = Sc<T>::conj(o[3]);
    }
  } else {
    const long long u = t - nblk;
    const int i = (int)(u % l), b = (int)(u / l);
    const Rot rb = load_rot(rots + b);
    if (rb.q >= l || rot_identity(rb)) return;
    const double cb = rb.c;
    const T sb = rot_s<T>(rb), sbc = Sc<T>::conj(sb);
    T* wp = W + (size_t)i + (size_t)rb.p * ldw;
    T* wq = W + (size_t)i + (size_t)rb.q * ldw;
    T xp = ldcg(wp), xq = ldcg(wq);
    *wp = Sc<T>::sub(Sc<T>::scale(xp, cb), Sc<T>::mul(xq, sbc));
    *wq = Sc<T>::add(Sc<T>::mul(xp, sb), Sc<T>::scale(xq, cb));
  }
}

// The whole cyclic Jacobi iteration: sweeps until ||off(H)||_F <= l u ||H||_F or
// max_sweeps.  H alternates between H0 (ld ld0) and H1 (ld ld1) every round (the next
// round's rotations are formed from the previous H while the round writes the next one,
// so a round needs one grid barrier); after an odd number of rounds the result is in H1.
// rots: two sets of L/2 rotations; partial: 2 doubles per CTA; gb->sweeps: sweeps done.
template <class T>
__global__ void __launch_bounds__(256) jacobi_sweeps_kernel(int l, int L, T* H0, int ld0, T* H1,
                                                            int ld1, T* W, int ldw, Rot* rots,
                                                            double* partial, GridBar* gb,
                                                            int max_sweeps) {
  const unsigned G = gridDim.x;
  const int np = L / 2;
  const long long items = (long long)np * np + (long long)l * np;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)G * blockDim.x;
  __shared__ double r0[8], r1[8];
  const double tolr = 1.1102230246251565e-16 * (double)l;
  unsigned k = 0;   // barriers passed
  int cur = 0;      // buffer holding the current H
  int sw = 0;
  double thr2 = 0.0;  // rotation threshold^2 (none before ||H||_F is known)
  for (; sw <= max_sweeps; ++sw) {
    T* Hc = cur ? H1 : H0;
    const int ldc = cur ? ld1 : ld0;
    // ||off(H)||_F^2 and ||H||_F^2: partial sums per CTA, then the same fixed-order total
    // in every CTA
    double off = 0.0, all = 0.0;
    const size_t total = (size_t)l * l;
    for (size_t t = gtid; t < total; t += (size_t)gstride) {
      const int i = (int)(t % l), j = (int)(t / l);
      const double a = Sc<T>::abs2(ldcg(Hc + (size_t)i + (size_t)j * ldc));
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
    // rotations of the sweep's first round, from the current H
    for (int i = blockIdx.x + G * threadIdx.x; i < np; i += G * blockDim.x) {
      int p, q;
      pair_of(L, 0, i, p, q);
      Rot rr;
      rr.p = p; rr.q = q; rr.c = 1.0; rr.sx = 0.0; rr.sy = 0.0;
      if (q < l)
        rr = rot_from<T>(p, q, Sc<T>::re(ldcg(Hc + (size_t)p + (size_t)p * ldc)),
                         Sc<T>::re(ldcg(Hc + (size_t)q + (size_t)q * ldc)),
                         ldcg(Hc + (size_t)p + (size_t)q * ldc), thr2);
      rots[i] = rr;
    }
    if (!grid_barrier(gb, G, k)) return;
    double so = 0.0, sa = 0.0;
    for (unsigned b = 0; b < G; ++b) { so += __ldcg(partial + 2 * b); sa += __ldcg(partial + 2 * b + 1); }
    if (so <= tolr * tolr * sa || so == 0.0 || sw == max_sweeps) break;
    // the next sweep's threshold: |g| <= u ||H||_F (||H||_F does not change under rotations)
    thr2 = 1.2325951644078309e-32 * sa;
    for (int r = 0; r < L - 1; ++r) {
      const T* Hcr = cur ? H1 : H0;
      T* Hn = cur ? H0 : H1;
      const int ldcr = cur ? ld1 : ld0, ldn = cur ? ld0 : ld1;
      const Rot* rc = rots + (size_t)(r & 1) * np;
      Rot* rn = rots + (size_t)((r + 1) & 1) * np;
      // the next round's rotations (spread over the CTAs: their FP64 square roots and
      // divisions), from the entries this round writes, formed here from the current H
      if (r + 1 < L - 1) {
        for (int i = blockIdx.x + G * threadIdx.x; i < np; i += G * blockDim.x) {
          int p, q;
          pair_of(L, r + 1, i, p, q);
          Rot rr;
          rr.p = p; rr.q = q; rr.c = 1.0; rr.sx = 0.0; rr.sy = 0.0;
          if (q < l) rr = next_rotation<T>(l, L, r, rc, Hcr, ldcr, p, q, thr2);
          rn[i] = rr;
        }
      }
      for (long long t = gtid; t < items; t += gstride)
        apply_item<T>(t, l, np, rc, Hcr, ldcr, Hn, ldn, W, ldw);
      cur ^= 1;
      if (!grid_barrier(gb, G, k)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    gb->sweeps = sw;
    gb->pad = cur;
  }
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
  return al(sizeof(Rot) * (size_t)L) + al(sizeof(GridBar)) + al(16 * (size_t)kJacobiMaxCtas) +
         al(sizeof(int) * (size_t)l) + al(elem * (size_t)l * l);
}

template <class T>
int jacobi_eig(cudaStream_t st, int l, T* H, int ldh, T* W, int ldw, double* dw, void* work,
               size_t work_bytes, int max_sweeps, int* sweeps, int* launches, int ctas) {
  if (l <= 0) return 0;
  const int L = (l % 2) ? l + 1 : l;
  if (jacobi_work_bytes(l, sizeof(T)) > work_bytes) return 4;  // CHASE_ERR_OOM
  // workspace: two sets of rotations | barrier | per-CTA norm partials | permutation |
  // l x l buffer (the second H of the sweeps, then a copy of W)
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* base = (char*)work;
  Rot* rots = (Rot*)base;
  base += al(sizeof(Rot) * (size_t)L);
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
  const T* Hfin = H;
  int ldfin = ldh;
  if (l > 1) {
    // CTAs: about 2 work items of a round per thread (measured: fewer CTAs leave the FP64
    // work latency-bound, more make the grid barrier dearer), at most one co-resident wave
    // co-resident CTAs of the kernel, looked up once (thread-safe static initialisation)
    static const int mc = []() {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_sweeps_kernel<T>, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
      }
      return std::max(1, std::min(per_sm * kNumSMs, kJacobiMaxCtas));
    }();
    const long long items = (long long)(L / 2) * (L / 2) + (long long)l * (L / 2);
    int G = std::max(1, std::min(mc, ceil_div(items, 256 * 2)));
    if (ctas > 0) G = std::min(mc, ctas);
    CHASE_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), st));
    int ms = max_sweeps, ld1 = l;
    T* H1 = Wtmp;
    void* args[] = {(void*)&l,   (void*)&L,   (void*)&H,    (void*)&ldh,     (void*)&H1, (void*)&ld1,
                    (void*)&W,   (void*)&ldw, (void*)&rots, (void*)&partial, (void*)&gb, (void*)&ms};
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
    if (hb.pad) {  // the last round wrote the second buffer
      Hfin = Wtmp;
      ldfin = l;
    }
  }
  jacobi_sort_kernel<T><<<1, 1024, 0, st>>>(l, Hfin, ldfin, W, ldw, dw, dperm);
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
                                size_t, int, int*, int*, int);
template int jacobi_eig<z64>(cudaStream_t, int, z64*, int, z64*, int, double*, void*, size_t, int,
                             int*, int*, int);

}  // namespace chase
