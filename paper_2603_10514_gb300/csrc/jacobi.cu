// jacobi.cu -- parallel cyclic Jacobi eigensolver for the reduced problem of the
// Rayleigh-Ritz step (Algorithm 1: solve A~ W = W Lambda~).
//
// Round-robin ordering: in each round the indices 0..L-1 (L = l rounded up to
// even; index l is a dummy when l is odd) form L/2 disjoint pairs, so all L/2
// rotations of a round commute and are applied together.  L - 1 rounds make a
// sweep that visits every pair once.  Per round:
//   1. rot kernel: for pair (p, q) with g = H_pq = |g| e^{i phi},
//        tau = (H_qq - H_pp) / (2|g|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//        c = 1/sqrt(1 + t^2), s = t c,  J = [[c, s e^{i phi}], [-s e^{-i phi}, c]];
//   2. apply kernel: H <- J^H H J, one thread per 2x2 block (pair_a, pair_b) with
//      a <= b, which also writes block (b, a) as the conjugate transpose (H stays
//      exactly Hermitian, and half the FP64 arithmetic of a full update is spent:
//      the rounds are FP64-bound on GB300, 2 FP64 FMAs per clock per SM), and
//      W <- W J, one thread per (row, pair).
// The rotation kernel runs one warp per CTA so that the FP64 square roots and
// divisions of the l/2 rotations spread over many SMs.
// Sweeps stop when the off-diagonal Frobenius norm is <= l 2^-53 ||H||_F (the
// rounding level a parallel sweep leaves behind; eigenvalues are then accurate
// to that level by Weyl's inequality) or after max_sweeps.
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

template <class T>
__global__ void jacobi_rot_kernel(int l, int L, int round, const T* H, int ldh, Rot* rots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L / 2) return;
  int p, q;
  pair_of(L, round, i, p, q);
  Rot r;
  r.p = p; r.q = q; r.c = 1.0; r.sx = 0.0; r.sy = 0.0;
  if (q < l) {
    T g = H[(size_t)p + (size_t)q * ldh];
    double ag = sqrt(Sc<T>::abs2(g));
    if (ag > 0.0) {
      double hpp = Sc<T>::re(H[(size_t)p + (size_t)p * ldh]);
      double hqq = Sc<T>::re(H[(size_t)q + (size_t)q * ldh]);
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
  rots[i] = r;
}

template <class T> __device__ inline T rot_s(const Rot& r);
template <> __device__ inline double rot_s<double>(const Rot& r) { return r.sx; }
template <> __device__ inline z64 rot_s<z64>(const Rot& r) { return z64{r.sx, r.sy}; }

// H <- J^H H J on the 2x2 block (rows of pair a, columns of pair b), and W <- W J.
template <class T>
__global__ void jacobi_apply_kernel(int l, int L, const Rot* __restrict__ rots, T* H, int ldh, T* W,
                                    int ldw) {
  const int np = L / 2;
  const long long nblk = (long long)np * np;
  const long long nw = (long long)l * np;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nblk + nw;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < nblk) {
      const int a = (int)(t % np), b = (int)(t / np);
      if (a > b) continue;  // written by block (b, a) as its conjugate transpose
      const Rot ra = rots[a], rb = rots[b];
      const int pa = ra.p, qa = ra.q, pb = rb.p, qb = rb.q;
      const bool va = qa < l, vb = qb < l;
      // load the 2x2 block (dummy index -> zero row/column, never stored)
      T h_pp = H[(size_t)pa + (size_t)pb * ldh];
      T h_qp = va ? H[(size_t)qa + (size_t)pb * ldh] : Sc<T>::zero();
      T h_pq = vb ? H[(size_t)pa + (size_t)qb * ldh] : Sc<T>::zero();
      T h_qq = (va && vb) ? H[(size_t)qa + (size_t)qb * ldh] : Sc<T>::zero();
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
      const Rot rb = rots[b];
      if (rb.q >= l) continue;
      const double cb = rb.c;
      const T sb = rot_s<T>(rb), sbc = Sc<T>::conj(sb);
      T* wp = W + (size_t)i + (size_t)rb.p * ldw;
      T* wq = W + (size_t)i + (size_t)rb.q * ldw;
      T xp = *wp, xq = *wq;
      *wp = Sc<T>::sub(Sc<T>::scale(xp, cb), Sc<T>::mul(xq, sbc));
      *wq = Sc<T>::add(Sc<T>::mul(xp, sb), Sc<T>::scale(xq, cb));
    }
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

// out[0] = sum_{i != j} |H_ij|^2, out[1] = sum |H_ij|^2  (single CTA, fixed order)
template <class T>
__global__ void __launch_bounds__(1024) jacobi_offnorm_kernel(int l, const T* H, int ldh,
                                                              double* out) {
  __shared__ double r0[32], r1[32];
  double off = 0.0, all = 0.0;
  const size_t total = (size_t)l * l;
  for (size_t t = threadIdx.x; t < total; t += blockDim.x) {
    int i = (int)(t % l), j = (int)(t / l);
    double a = Sc<T>::abs2(H[(size_t)i + (size_t)j * ldh]);
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
    out[0] = a;
    out[1] = b;
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

template <class T>
int jacobi_eig(cudaStream_t st, int l, T* H, int ldh, T* W, int ldw, double* dw, void* work,
               size_t work_bytes, int max_sweeps, int* sweeps, int* launches) {
  if (l <= 0) return 0;
  const int L = (l % 2) ? l + 1 : l;
  // workspace: rotations | off-norm pair | permutation | W copy
  size_t off_rot = 0;
  size_t off_nrm = off_rot + sizeof(Rot) * (size_t)(L / 2 + 1);
  off_nrm = (off_nrm + 255) & ~(size_t)255;
  size_t off_perm = off_nrm + 256;
  size_t off_w = (off_perm + sizeof(int) * (size_t)l + 255) & ~(size_t)255;
  size_t need = off_w + sizeof(T) * (size_t)l * l;
  if (need > work_bytes) return 4;  // CHASE_ERR_OOM
  char* base = (char*)work;
  Rot* rots = (Rot*)(base + off_rot);
  double* dnrm = (double*)(base + off_nrm);
  int* dperm = (int*)(base + off_perm);
  T* Wtmp = (T*)(base + off_w);
  int nl = 0;
  int blocks = std::min(ceil_div((long long)l * l, 256), kNumSMs * 8);
  jacobi_init_kernel<T><<<blocks, 256, 0, st>>>(l, W, ldw);
  ++nl;
  int sw = 0;
  double host_nrm[2] = {0.0, 0.0};
  if (l > 1) {
    const long long work_items = (long long)(L / 2) * (L / 2) + (long long)l * (L / 2);
    const int ablocks = std::min(ceil_div(work_items, 256), kNumSMs * 8);
    const int rblocks = ceil_div(L / 2, 32);
    for (sw = 0; sw < max_sweeps; ++sw) {
      jacobi_offnorm_kernel<T><<<1, 1024, 0, st>>>(l, H, ldh, dnrm);
      ++nl;
      CHASE_CUDA_TRY(cudaMemcpyAsync(host_nrm, dnrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CHASE_CUDA_TRY(cudaStreamSynchronize(st));
      // stop once ||off(H)||_F <= l u ||H||_F: the rounding level of a parallel sweep
      const double tolr = 1.1102230246251565e-16 * (double)l;
      if (host_nrm[0] <= tolr * tolr * host_nrm[1] || host_nrm[0] == 0.0) break;
      for (int r = 0; r < L - 1; ++r) {
        jacobi_rot_kernel<T><<<rblocks, 32, 0, st>>>(l, L, r, H, ldh, rots);
        jacobi_apply_kernel<T><<<ablocks, 256, 0, st>>>(l, L, rots, H, ldh, W, ldw);
        nl += 2;
      }
    }
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
