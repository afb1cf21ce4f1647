// gemm_oz.cu -- FP64-accurate dense products on the BF16 tensor cores by the
// Ozaki scheme II (Ozaki, Uchino & Imamura, "Ozaki Scheme II: A GEMM-oriented
// emulation of floating-point matrix multiplication using an integer modular
// technique", 2025): the filter's A*V, the Rayleigh-Ritz product A*Q and the
// block products of the QR and Rayleigh-Ritz steps.
//
// Integer operands.  Every row m of the (stacked real) left operand is scaled by
// 2^{57 - e_m} (max_k |L[m,k]| < 2^{e_m}) and every column c of the right
// operand by 2^{57 - f_c}; each scaled entry is rounded to the nearest integer,
// so |L_int|, |V_int| <= 2^57 and the rounding error is at most 2^-58 of the
// row (column) scale.  The product of the integer matrices
//   X[m, c] = sum_k L_int[m, k] V_int[k, c],   |X| <= K 2^114,
// is computed EXACTLY, and (A V)[m, c] = 2^{e_m + f_c - 114} X[m, c] is then
// within K 2^-57 max_k|L[m,k]| max_k|V[k,c]| of the exact product: the accuracy
// class of an FP64 GEMM.
//
// Exact integer product by the Chinese remainder theorem.  With S = 17 pairwise
// coprime moduli p_j <= 256 (product P ~ 2^132.95 > 2 K 2^114 for K <= 2^17),
// X is recovered from its residues X mod p_j.  Each residue needs one product
// of residue matrices: L_int mod p_j and V_int mod p_j are stored in symmetric
// range (|r| <= 128, exact in BF16), so one BF16 tensor-core product per
// modulus forms sum_k (L mod p)(V mod p), whose partial sums over a K chunk of
// 1024 stay within 1024 * 128^2 = 2^24 and are therefore exact in the tensor
// core's FP32 accumulator; the epilogue adds the chunks as 32-bit integers and
// reduces mod p_j at the end.  17 BF16 products replace the FP64 product.
// Reconstruction (crt_kernel): X = sum_j r_j C_j mod P with C_j = (P/p_j) *
// ((P/p_j)^{-1} mod p_j), in 160-bit integer arithmetic (32-bit limbs), mapped
// to the symmetric range (-P/2, P/2] and rounded once to FP64.
//
// Modular product kernel (ozm_kernel): CTA pairs (clusters of two along grid x), one pair
// per (256-row block, column tile of BN <= 256 columns, modulus[, K split]).  The even CTA
// issues tcgen05.mma.cta_group::2.kind::f16 (M 256, N BN, K 16) over the pair: each CTA
// holds its own 128 rows of A and half of the BN rows of V in shared memory, and its 128
// rows of the accumulator in its own TMEM (two buffers of 256 columns: the epilogue reads
// one K chunk while the next accumulates).  Per CTA: a TMA producer thread (its copies
// count on the even CTA's stage barrier), 16 epilogue warps reading TMEM with tcgen05.ld.
// Stages: two 64-wide K blocks (128-byte swizzle), 3 stages of 64 KB.
// Measured on GB300: the tensor pipe loses ~100-150 cycles per barrier round trip between
// the producer and the issuer, hidden only when a stage holds >= 8 MMAs (K 128); a pair
// moves 31 % fewer operand bytes per SM than a 128 x BN tile on one SM.  The product of
// the default workload (K 20032, 600 columns) runs 12 % faster than with single-CTA tiles.
// All mbarrier waits are bounded; on expiry the kernel records the failure in
// the device status word, waits (bounded) for its copies and MMAs in flight,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace chase {

#define TRY_OZ(x)          \
  do {                     \
    int _rc = (x);         \
    if (_rc) return _rc;   \
  } while (0)

namespace {

// ---------------------------------------------------------------------------
// Moduli and CRT constants (computed at compile time)
// ---------------------------------------------------------------------------
constexpr int OZ_KBITS = 57;  // integer operands: |x_int| <= 2^57
// 17 pairwise coprime moduli <= 256 (256 = 2^8; 255 = 3 5 17; 253 = 11 23; 247 = 13 19;
// 217 = 7 31; the others prime): P = prod p_j ~ 2^132.95 > 2 * 2^17 * 2^114.
__host__ __device__ constexpr int oz_modulus(int j) {
  constexpr int t[kOzModuli] = {256, 255, 253, 251, 247, 241, 239, 233, 229,
                                227, 223, 217, 211, 199, 197, 193, 191};
  return t[j];
}
static_assert(kOzPlaneBytes == 2 * kOzModuli, "workspace plane size");
static_assert(kOzMaxK <= (1 << 17), "K bound of the modulus product");

struct Big {  // unsigned 160-bit integer, little-endian 32-bit limbs
  uint32_t w[5];
};

constexpr Big big_small(uint32_t x) { return Big{{x, 0, 0, 0, 0}}; }
constexpr Big big_mul_small(Big a, uint32_t k) {
  uint64_t c = 0;
  for (int i = 0; i < 5; ++i) {
    const uint64_t t = (uint64_t)a.w[i] * k + c;
    a.w[i] = (uint32_t)t;
    c = t >> 32;
  }
  return a;
}
constexpr uint32_t big_mod_small(Big a, uint32_t p) {
  uint64_t r = 0;
  for (int i = 4; i >= 0; --i) r = ((r << 32) | a.w[i]) % p;
  return (uint32_t)r;
}
constexpr Big big_shr1(Big a) {
  for (int i = 0; i < 5; ++i) a.w[i] = (a.w[i] >> 1) | (i < 4 ? (a.w[i + 1] << 31) : 0u);
  return a;
}
constexpr uint32_t inv_mod(uint32_t a, uint32_t p) {  // a^{-1} mod p, gcd(a, p) = 1
  long long t = 0, nt = 1, r = p, nr = a % p;
  while (nr != 0) {
    const long long q = r / nr;
    long long tmp = t - q * nt; t = nt; nt = tmp;
    tmp = r - q * nr; r = nr; nr = tmp;
  }
  return (uint32_t)(t < 0 ? t + p : t);
}

struct CrtTable {
  int p[kOzModuli];          // the moduli
  uint32_t C[kOzModuli][5];  // C_j = (P / p_j) ((P / p_j)^{-1} mod p_j) < P
  uint32_t P[5];
  uint32_t Ph[5];            // P / 2
  float p96_over_P;          // 2^96 / P (rounded)
};

constexpr CrtTable make_crt_table() {
  CrtTable t{};
  Big P = big_small(1);
  for (int j = 0; j < kOzModuli; ++j) {
    t.p[j] = oz_modulus(j);
    P = big_mul_small(P, (uint32_t)oz_modulus(j));
  }
  for (int j = 0; j < kOzModuli; ++j) {
    Big Mj = big_small(1);
    for (int i = 0; i < kOzModuli; ++i)
      if (i != j) Mj = big_mul_small(Mj, (uint32_t)oz_modulus(i));
    const uint32_t inv = inv_mod(big_mod_small(Mj, (uint32_t)oz_modulus(j)), (uint32_t)oz_modulus(j));
    const Big Cj = big_mul_small(Mj, inv);
    for (int l = 0; l < 5; ++l) t.C[j][l] = Cj.w[l];
  }
  const Big Ph = big_shr1(P);
  double pd = 0.0;
  for (int l = 4; l >= 0; --l) {
    t.P[l] = P.w[l];
    t.Ph[l] = Ph.w[l];
    pd = pd * 4294967296.0 + (double)P.w[l];
  }
  t.p96_over_P = (float)(79228162514264337593543950336.0 / pd);  // 2^96 / P
  return t;
}

__constant__ CrtTable c_crt = make_crt_table();

// Compile-time checks of the number theory the reconstruction relies on: the moduli are
// pairwise coprime, C_j is 1 mod p_j and 0 mod every other modulus, and P exceeds twice the
// largest integer product, 2 * 2^17 * 2^114 = 2^132 (limb 4 holds P / 2^128).
constexpr int oz_gcd(int a, int b) { return b == 0 ? a : oz_gcd(b, a % b); }
constexpr bool oz_moduli_coprime() {
  for (int i = 0; i < kOzModuli; ++i)
    for (int j = i + 1; j < kOzModuli; ++j)
      if (oz_gcd(oz_modulus(i), oz_modulus(j)) != 1) return false;
  return true;
}
constexpr bool oz_crt_basis_ok() {
  const CrtTable t = make_crt_table();
  for (int j = 0; j < kOzModuli; ++j) {
    const Big Cj{{t.C[j][0], t.C[j][1], t.C[j][2], t.C[j][3], t.C[j][4]}};
    for (int i = 0; i < kOzModuli; ++i)
      if (big_mod_small(Cj, (uint32_t)oz_modulus(i)) != (i == j ? 1u : 0u)) return false;
  }
  return true;
}
static_assert(oz_moduli_coprime(), "moduli must be pairwise coprime");
static_assert(oz_crt_basis_ok(), "CRT basis: C_j = 1 mod p_j, 0 mod p_i");
static_assert(make_crt_table().P[4] >= (1u << (2 * OZ_KBITS + 17 + 1 - 128)), "P > 2 K 2^114");
// The modular epilogue reduces a split's sum |s| <= kOzSplitMaxK * 128^2 = 2^30 with the
// float quotient q = floor(fl(fl(s) * fl(1/p))): fl(s) is within 32 of s and the two roundings
// add a relative 2^-23, so q is within 32/p + 2^30 2^-23 / p < 1 of s/p for p > 160 and one
// correction step lands in [0, p).
constexpr bool oz_moduli_above(int lo) {
  for (int j = 0; j < kOzModuli; ++j)
    if (oz_modulus(j) <= lo) return false;
  return true;
}
static_assert(oz_moduli_above(160), "epilogue reduction: p > 160");
static_assert((long long)kOzSplitMaxK * 128 * 128 <= (1ll << 30), "epilogue reduction: |sum| <= 2^30");
static_assert(kOzMaxK <= kOzMaxSplits * kOzSplitMaxK, "every admissible K fits the splits");

constexpr int MBM = 128, MBK = 64;
constexpr int MKS = 2;             // 64-wide K blocks per stage: 8 MMAs per barrier round trip
constexpr int MNST = 3;            // stages
constexpr int MBN_MAX = 256;
constexpr int M_EPI_WARPS = 16;
constexpr int M_THREADS = 64 + 32 * M_EPI_WARPS;
constexpr int M_CHUNK_ST = 1024 / (MKS * MBK);  // stages per exact 1024-wide K chunk
constexpr int M_A1 = MBM * MBK * 2;              // 16 KB: 128 rows of A, one K block
constexpr int M_B1 = (MBN_MAX / 2) * MBK * 2;    // 16 KB: up to 128 rows of V (half a tile)
constexpr int M_STG = MKS * (M_A1 + M_B1);       // 64 KB
constexpr int M_SMEM = MNST * M_STG + 1024 + 256;
constexpr uint32_t M_TMEM_COLS = 2 * MBN_MAX;    // two accumulators of 256 columns
static_assert(M_SMEM <= 232448, "shared memory");
static_assert(M_STG % 1024 == 0 && M_A1 % 1024 == 0, "stage alignment (128-byte swizzle atoms)");
static_assert(M_CHUNK_ST * MKS * MBK == 1024, "exact chunk");
using namespace tc;

// ---------------------------------------------------------------------------
// Modular products: R[z][c][r] = (sum_{k in split} Lres_j[r, k] Vres_j[k, c]) mod p_j,
// z = split * S + j (grid z).  Lres planes row-major (rows x kp), Vres planes column-major
// (kp x ncols); both K-padded with zeros to kp (a multiple of 64).
// ---------------------------------------------------------------------------
// One CTA of a pair (clusters of two CTAs along grid x): this CTA's rows [m0, m0 + 128)
// and the pair's columns [n0, n0 + BN) of modulus jm over the K blocks [kbeg, kbeg + nkb);
// residues into Rz (column-major M x N).  kbeg is even; an odd nkb reads one zero-filled
// block past kp (the K-padded operands end there), or the first block of the next split
// only when nkb is odd, which the launch never makes for a split other than the last.
__device__ __forceinline__ void ozm_pair_tile(const CUtensorMap* mapA, const CUtensorMap* mapV,
                                              int M, int N, int BN, int col0, int m0, int n0,
                                              int jm, int kbeg, int nkb, uint8_t* __restrict__ Rz,
                                              DevStatus* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + MNST * M_STG);
  uint64_t* full = bars;                // [MNST] stage loaded (both CTAs' copies; the even CTA's)
  uint64_t* empty = bars + MNST;        // [MNST] stage read by the pair's MMAs
  uint64_t* cfull = bars + 2 * MNST;    // [2] chunk accumulated in buffer b
  uint64_t* cfree = cfull + 2;          // [2] buffer b read out by both CTAs (the even CTA's)
  uint64_t* tdone = cfree + 2;          // every MMA finished
  uint32_t* tslot = (uint32_t*)(tdone + 1);
  int* s_err = (int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int half = BN >> 1;
  const int nst = (nkb + MKS - 1) / MKS;
  const int nchunks = (nst + M_CHUNK_ST - 1) / M_CHUNK_ST;

  if (threadIdx.x == 0) {
    for (int i = 0; i < MNST; ++i) { bar_init(&full[i], 1); bar_init(&empty[i], 1); }
    for (int b = 0; b < 2; ++b) { bar_init(&cfull[b], 1); bar_init(&cfree[b], 2 * M_EPI_WARPS); }
    bar_init(tdone, 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // one warp of each CTA of the pair allocates the pair's accumulators
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(tslot)),
                 "r"(M_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before any copy or arrival crosses over
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer (both CTAs): own A rows, own half of the V tile ----------------
    const uint32_t bytes = (uint32_t)(MKS * (2 * M_A1 + BN * MBK * 2));  // the pair's copies of a stage
    const uint32_t full0 = peer_addr(full, 0);
    int issued = 0;
    for (int kb = 0; kb < nst && !*(volatile int*)s_err; ++kb) {
      const int s = kb % MNST;
      if (!bar_wait(&empty[s], (uint32_t)(((kb / MNST) & 1) ^ 1))) { atomicOr(s_err, 1); break; }
      if (rank == 0) bar_expect(&full[s], bytes);
      unsigned char* st = smem + s * M_STG;
      const uint32_t fb = full0 + 8u * (uint32_t)s;
#pragma unroll
      for (int u = 0; u < MKS; ++u) {
        const int x = (kbeg + kb * MKS + u) * MBK;
        tma3_pair(st + u * M_A1, mapA, fb, x, m0, jm);
        tma3_pair(st + MKS * M_A1 + u * M_B1, mapV, fb, x, col0 + n0 + (int)rank * half, jm);
      }
      issued = kb + 1;
    }
    // every release of this CTA's stages has arrived (no arrival may reach it after exit) ...
    for (int kb = issued; kb < issued + MNST; ++kb)
      if (!bar_wait(&empty[kb % MNST], (uint32_t)(((kb / MNST) & 1) ^ 1))) { atomicOr(s_err, 1); break; }
    // ... and, in the even CTA, every copy of both CTAs has landed
    if (rank == 0)
      for (int b = max(0, issued - MNST); b < issued; ++b)
        if (!bar_wait(&full[b % MNST], (uint32_t)((b / MNST) & 1))) { atomicOr(s_err, 1); break; }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer (even CTA): M 256 x N BN x K 16 over the pair ----------------
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)((2 * MBM) >> 4) << 24);
    bool bad = false;
    for (int kb = 0; kb < nst && !bad; ++kb) {
      const int chunk = kb / M_CHUNK_ST;
      const bool cstart = (kb % M_CHUNK_ST) == 0;
      const bool clast = (kb % M_CHUNK_ST) == M_CHUNK_ST - 1 || kb == nst - 1;
      const uint32_t buf = (uint32_t)(chunk & 1);
      if (cstart && chunk >= 2) {
        // both CTAs' epilogues have read this buffer's previous chunk (chunk - 2)
        if (!bar_wait(&cfree[buf], (uint32_t)(((chunk - 2) >> 1) & 1))) { bad = true; break; }
      }
      const int s = kb % MNST;
      if (!bar_poll(&full[s], (uint32_t)((kb / MNST) & 1))) { bad = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = s32(smem + s * M_STG);
#pragma unroll
      for (int kk = 0; kk < MKS * (MBK / 16); ++kk) {
        const uint64_t da = desc_sw128(sa + (kk >> 2) * M_A1);
        const uint64_t dv = desc_sw128(sa + MKS * M_A1 + (kk >> 2) * M_B1);
        mma_pair(tmem + buf * MBN_MAX, da + (uint64_t)((kk & 3) * 2), dv + (uint64_t)((kk & 3) * 2),
                 idesc, (cstart && kk == 0) ? 0u : 1u);
      }
      commit_pair(&empty[s]);
      if (clast) commit_pair(&cfull[buf]);
    }
    if (bad) atomicOr(s_err, 2);
    commit_pair(tdone);
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs, own TMEM lanes = own 128 rows) ----------------
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (the hardware's lane quarter of the warp)
    // and the column quarter (w - 2) / 4 of the tile (BN / 4 <= 64 columns).
    const int q = warp & 3, cq = (warp - 2) >> 2;
    const int r = m0 + 32 * q + lane;
    const int cw = BN >> 2;
    const uint32_t cfree0 = peer_addr(cfree, 0);
    int sum[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) sum[j] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const uint32_t buf = (uint32_t)(c & 1);
      if (!__all_sync(0xffffffffu, bar_wait(&cfull[buf], (uint32_t)((c >> 1) & 1)))) {
        ok = false;
        if (lane == 0) atomicOr(s_err, 4);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + buf * MBN_MAX + (uint32_t)(cq * cw);
      uint32_t v[32];
      ld32(ta, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) sum[j] += __float2int_rn(__uint_as_float(v[j]));
      if (cw > 32) {
        ld32(ta + 32, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0 && c + 2 < nchunks) arrive_remote(cfree0 + 8u * buf);
      if (cw > 32) {
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[32 + j] += __float2int_rn(__uint_as_float(v[j]));
      }
    }
    if (__shfl_sync(0xffffffffu, (int)(ok && !*(volatile int*)s_err), 0) && r < M) {
      // sum mod p in [0, p): |sum| <= 2^30 (K <= kOzSplitMaxK per split), so the float quotient is
      // off by at most one
      const int pm = c_crt.p[jm];
      const float ip = 1.0f / (float)pm;
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        const int col = n0 + cq * cw + j;
        if (j < cw && col - n0 < BN && col < N) {
          const int sv = sum[j];
          const int qq = (int)floorf((float)sv * ip);
          int rr = sv - qq * pm;
          if (rr < 0) rr += pm;
          if (rr >= pm) rr -= pm;
          Rz[(size_t)col * M + r] = (uint8_t)rr;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1 && !bar_wait(tdone, 0u) && lane == 0) atomicOr(s_err, 8);
  cluster_sync();  // neither CTA frees the pair's TMEM or exits while the other may signal it
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(M_TMEM_COLS));
  }
  if (threadIdx.x == 32 && *s_err) atomicOr(&status->timeout, *s_err);
}

// Pair index p = blockIdx.x / 2 runs over (row pair, column tile) with the column tiles
// fastest, so the tiles of one row pair read its A rows from L2 at about the same time.
__device__ __forceinline__ void pair_tile_coords(int x, int ntile, int BN, int* m0, int* n0) {
  const int pr = x >> 1;
  *n0 = (pr % ntile) * BN;
  *m0 = (2 * (pr / ntile) + (x & 1)) * MBM;
}

__global__ void __launch_bounds__(M_THREADS, 1)
    ozm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapV,
               int M, int N, int BN, int ntile, int col0, int nkb_total, int kbs,
               uint8_t* __restrict__ R, DevStatus* status) {
  const int jm = blockIdx.z % kOzModuli, split = blockIdx.z / kOzModuli;
  const int kbeg = split * kbs;
  const int nkb = max(0, min(kbs, nkb_total - kbeg));
  int m0, n0;
  pair_tile_coords(blockIdx.x, ntile, BN, &m0, &n0);
  ozm_pair_tile(&mapA, &mapV, M, N, BN, col0, m0, n0, jm, kbeg, nkb,
                R + (size_t)blockIdx.z * N * M, status);
}

// Grouped products: the tiles of up to kOzGroupMax independent problems in one launch
// (grid x runs over every problem's CTA pairs, z over the moduli); each problem has its own
// operands (tensor maps), sizes and residue buffer.  Used to batch the filter steps of many
// problems.
struct OzmGroupParams {
  CUtensorMap mapA[kOzGroupMax];
  CUtensorMap mapV[kOzGroupMax];
  uint8_t* R[kOzGroupMax];
  int tile0[kOzGroupMax + 1];  // first grid-x CTA of each problem (even: pairs never straddle)
  int M[kOzGroupMax], N[kOzGroupMax], BN[kOzGroupMax], col0[kOzGroupMax], ntile[kOzGroupMax],
      nkb[kOzGroupMax];
  int count;
};
static_assert(sizeof(OzmGroupParams) <= 32000, "kernel parameter space");

__global__ void __launch_bounds__(M_THREADS, 1)
    ozm_group_kernel(const __grid_constant__ OzmGroupParams P, DevStatus* status) {
  int p = 0;
  while (p + 1 < P.count && (int)blockIdx.x >= P.tile0[p + 1]) ++p;
  const int jm = blockIdx.z;
  int m0, n0;
  pair_tile_coords((int)blockIdx.x - P.tile0[p], P.ntile[p], P.BN[p], &m0, &n0);
  ozm_pair_tile(&P.mapA[p], &P.mapV[p], P.M[p], P.N[p], P.BN[p], P.col0[p], m0, n0, jm, 0,
                P.nkb[p], P.R[p] + (size_t)jm * P.N[p] * P.M[p], status);
}

// ---------------------------------------------------------------------------
// CRT reconstruction and epilogue:
//   v = 2^{e_r + f_c - 114} X,  X = CRT(residues) in (-P/2, P/2],
//   out64[r + (col0 + c) ldo] = alpha v + beta X64[.] + gamma Z64[.]  (same index).
// R holds `splits` partial residues per modulus; they are summed mod p_j first.
// ---------------------------------------------------------------------------
// Returns the FP64 rounding m of |X| and the sign, with X = m 2^{*shift}.
// X = sum_j r_j C_j mod P from the residues r_j < p_j, rounded once to FP64: returns the
// signed magnitude and *shift_out with |X| = |value| 2^shift.
__device__ __forceinline__ double crt_finish(const unsigned long long* acc, int* shift_out);
__device__ __forceinline__ double crt_combine(const uint32_t* rj, int* shift_out) {
  unsigned long long acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < kOzModuli; ++j) {
#pragma unroll
    for (int l = 0; l < 5; ++l) acc[l] += (unsigned long long)rj[j] * c_crt.C[j][l];
  }
  return crt_finish(acc, shift_out);
}

// X = (sum_j r_j C_j, accumulated in 32-bit limbs with 64-bit headroom) mod P, rounded once to
// FP64.
__device__ __forceinline__ double crt_finish(const unsigned long long* acc, int* shift_out) {
  uint32_t x[5];
  unsigned long long carry = 0;
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    const unsigned long long t = acc[l] + carry;
    x[l] = (uint32_t)t;
    carry = t >> 32;
  }
  // X < 17 * 256 * P < 2^146: reduce mod P with q = floor(X / P) from the top limbs.  q is
  // below 2^13, so the FP32 estimate (relative error ~2^-22) is off by at most one; both
  // corrections follow.
  const float xf = (float)x[4] * 4294967296.0f + (float)x[3];  // X / 2^96, rounded
  const unsigned int qv = (unsigned int)floorf(xf * c_crt.p96_over_P);
  {
    unsigned long long borrow = 0, cq = 0;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      const unsigned long long prod = (unsigned long long)c_crt.P[l] * qv + cq;
      cq = prod >> 32;
      const unsigned long long sub = (unsigned long long)(uint32_t)prod + borrow;
      const long long d = (long long)x[l] - (long long)sub;
      x[l] = (uint32_t)d;
      borrow = d < 0 ? 1ull : 0ull;
    }
    if (borrow) {  // q was one too large: add P back
      unsigned long long c = 0;
#pragma unroll
      for (int l = 0; l < 5; ++l) {
        const unsigned long long t = (unsigned long long)x[l] + c_crt.P[l] + c;
        x[l] = (uint32_t)t;
        c = t >> 32;
      }
    }
  }
  auto cmp_ge = [&](const uint32_t* b) {
    for (int l = 4; l >= 0; --l) {
      if (x[l] != b[l]) return x[l] > b[l];
    }
    return true;
  };
  if (cmp_ge(c_crt.P)) {  // q was one too small
    long long br = 0;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      const long long d = (long long)x[l] - (long long)c_crt.P[l] - br;
      x[l] = (uint32_t)d;
      br = d < 0 ? 1 : 0;
    }
  }
  // symmetric range: X > P/2 stands for X - P
  bool neg = false;
  bool gt_half = false;
  for (int l = 4; l >= 0; --l) {
    if (x[l] != c_crt.Ph[l]) { gt_half = x[l] > c_crt.Ph[l]; break; }
  }
  if (gt_half) {
    neg = true;
    long long br = 0;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      const long long d = (long long)c_crt.P[l] - (long long)x[l] - br;
      x[l] = (uint32_t)d;
      br = d < 0 ? 1 : 0;
    }
  }
  // round the 160-bit magnitude once to FP64: the leading 64 bits (normalised) and a
  // sticky bit for everything below them
  int top = 4;
  while (top > 0 && x[top] == 0) --top;
  *shift_out = 0;
  if (x[top] == 0) return 0.0;
  const int lz = __clz(x[top]);
  const uint32_t x1 = top >= 1 ? x[top - 1] : 0u, x2 = top >= 2 ? x[top - 2] : 0u;
  unsigned long long hi = ((unsigned long long)x[top] << 32) | x1;
  uint32_t rest = x2;
  if (lz > 0) {
    hi = (hi << lz) | (x2 >> (32 - lz));
    rest = x2 << lz;
  }
  bool sticky = rest != 0;
  for (int l = top - 3; l >= 0; --l) sticky |= x[l] != 0;
  if (sticky) hi |= 1ull;
  const double mag = __ull2double_rn(hi);
  *shift_out = 32 * (top - 1) - lz;  // |X| = hi 2^shift
  return neg ? -mag : mag;
}

__device__ __forceinline__ double crt_value(const uint8_t* __restrict__ R, size_t stride_z,
                                            size_t idx, int splits, int* shift_out) {
  uint32_t rj[kOzModuli];
#pragma unroll
  for (int j = 0; j < kOzModuli; ++j) {
    uint32_t r = R[(size_t)j * stride_z + idx];
    for (int s = 1; s < splits; ++s) r += R[(size_t)(s * kOzModuli + j) * stride_z + idx];
    rj[j] = r % (uint32_t)oz_modulus(j);
  }
  return crt_combine(rj, shift_out);
}

// The epilogue of one reconstructed entry: v = alpha 2^E x + beta X64 + gamma Z64.
__device__ __forceinline__ void crt_store(double x, int sh, int r, int c, const int* __restrict__ rowexp,
                                          const int* __restrict__ colexp, int col0, double alpha,
                                          double beta, const double* X64, double gamma,
                                          const double* Z64, double* out64, int ldo, int er = -1) {
  // x 2^E with |x| in [2^63, 2^64]: one exact multiply by the power of two 2^E built from
  // its exponent field when that is a normal number (ldexp otherwise); er: the row whose
  // exponent scales the entry (r by default)
  const int E = sh + rowexp[er < 0 ? r : er] + colexp[col0 + c] - 2 * OZ_KBITS;
  const double v0 = (E > -1022 && E < 1024) ? x * __longlong_as_double((long long)(E + 1023) << 52)
                                            : ldexp(x, E);
  const size_t idx = (size_t)r + (size_t)(col0 + c) * ldo;
  double v = alpha * v0;
  if (beta != 0.0) v = fma(beta, X64[idx], v);
  if (gamma != 0.0) v = fma(gamma, Z64[idx], v);
  out64[idx] = v;
}

__global__ void __launch_bounds__(256) crt_kernel(int M, int N, int splits, const uint8_t* __restrict__ R,
                                                  const int* __restrict__ rowexp,
                                                  const int* __restrict__ colexp, int col0,
                                                  double alpha, double beta, const double* X64,
                                                  double gamma, const double* Z64, double* out64,
                                                  int ldo) {
  const size_t total = (size_t)M * N;
  const size_t stride_z = total;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % M), c = (int)(t / M);
    int sh;
    const double x = crt_value(R, stride_z, t, splits, &sh);
    crt_store(x, sh, r, c, rowexp, colexp, col0, alpha, beta, X64, gamma, Z64, out64, ldo);
  }
}

// crt_kernel for M N divisible by 4: four consecutive entries per thread, each residue plane
// read as one 4-byte word (a warp reads 128 contiguous bytes per plane instead of 32).
__global__ void __launch_bounds__(256) crt4_kernel(int M, int N, int splits, const uint8_t* __restrict__ R,
                                                   const int* __restrict__ rowexp,
                                                   const int* __restrict__ colexp, int col0,
                                                   double alpha, double beta, const double* X64,
                                                   double gamma, const double* Z64, double* out64,
                                                   int ldo) {
  const size_t total = (size_t)M * N, quads = total / 4;
  const uint32_t* R4 = (const uint32_t*)R;
  const size_t stride4 = total / 4;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < quads;
       q += (size_t)gridDim.x * blockDim.x) {
    uint32_t w[kOzModuli], w2[kOzModuli];
#pragma unroll
    for (int j = 0; j < kOzModuli; ++j) {
      w[j] = __ldg(R4 + (size_t)j * stride4 + q);
      w2[j] = splits > 1 ? __ldg(R4 + (size_t)(kOzModuli + j) * stride4 + q) : 0u;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t rj[kOzModuli];
#pragma unroll
      for (int j = 0; j < kOzModuli; ++j)
        rj[j] = (((w[j] >> (8 * e)) & 0xFFu) + ((w2[j] >> (8 * e)) & 0xFFu)) % (uint32_t)oz_modulus(j);
      int sh;
      const double x = crt_combine(rj, &sh);
      const size_t t = 4 * q + e;
      crt_store(x, sh, (int)(t % M), (int)(t / M), rowexp, colexp, col0, alpha, beta, X64, gamma, Z64,
                out64, ldo);
    }
  }
}

// Reconstruction of one problem in the three-product layout (residues of P1 | P2 | P3, n x N
// each): four consecutive entries per thread, every residue plane read as 4-byte words;
// Re = P1 - P2 to stacked row r, Im = P3 - P1 - P2 to row n + r (both scaled by row r).
__global__ void __launch_bounds__(256) crt3_kernel(int n, int N, const uint8_t* __restrict__ R,
                                                   const int* __restrict__ rowexp,
                                                   const int* __restrict__ colexp, int col0,
                                                   double alpha, double beta, const double* X64,
                                                   double gamma, const double* Z64, double* out64,
                                                   int ldo) {
  const size_t total = (size_t)n * N, quads = total / 4;
  const uint32_t* R4 = (const uint32_t*)R;
  const size_t stride4 = total / 4, set4 = (size_t)kOzModuli * stride4;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < quads;
       q += (size_t)gridDim.x * blockDim.x) {
    uint32_t w1[kOzModuli], w2[kOzModuli], w3[kOzModuli];
#pragma unroll
    for (int j = 0; j < kOzModuli; ++j) {
      w1[j] = __ldg(R4 + (size_t)j * stride4 + q);
      w2[j] = __ldg(R4 + set4 + (size_t)j * stride4 + q);
      w3[j] = __ldg(R4 + 2 * set4 + (size_t)j * stride4 + q);
    }
#pragma unroll 1
    for (int e = 0; e < 4; ++e) {
      unsigned long long are[5] = {0, 0, 0, 0, 0}, aim[5] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int j = 0; j < kOzModuli; ++j) {
        const uint32_t pj = (uint32_t)oz_modulus(j);
        const uint32_t r1 = (w1[j] >> (8 * e)) & 0xFFu, r2 = (w2[j] >> (8 * e)) & 0xFFu,
                       r3 = (w3[j] >> (8 * e)) & 0xFFu;
        const uint32_t re = (r1 + pj - r2) % pj, im = (r3 + 2 * pj - r1 - r2) % pj;
#pragma unroll
        for (int l = 0; l < 5; ++l) {
          are[l] += (unsigned long long)re * c_crt.C[j][l];
          aim[l] += (unsigned long long)im * c_crt.C[j][l];
        }
      }
      const size_t t = 4 * q + e;
      const int r = (int)(t % n), c = (int)(t / n);
      int sh;
      double x = crt_finish(are, &sh);
      crt_store(x, sh, r, c, rowexp, colexp, col0, alpha, beta, X64, gamma, Z64, out64, ldo);
      x = crt_finish(aim, &sh);
      crt_store(x, sh, n + r, c, rowexp, colexp, col0, alpha, beta, X64, gamma, Z64, out64, ldo, r);
    }
  }
}

struct CrtGroupParams {
  const uint8_t* R[kOzGroupMax];
  const int* rowexp[kOzGroupMax];
  const int* colexp[kOzGroupMax];
  const double* X64[kOzGroupMax];
  const double* Z64[kOzGroupMax];
  double* out64[kOzGroupMax];
  double alpha[kOzGroupMax], beta[kOzGroupMax], gamma[kOzGroupMax];
  long long out0[kOzGroupMax + 1];  // first output index of each problem
  int M[kOzGroupMax], N[kOzGroupMax], col0[kOzGroupMax], ldo[kOzGroupMax];
  int c3[kOzGroupMax];  // three-product layout: M = n, residues of P1 | P2 | P3, stacked output
  int count;
};
static_assert(sizeof(CrtGroupParams) <= 32000, "kernel parameter space");

__global__ void __launch_bounds__(256) crt_group_kernel(const __grid_constant__ CrtGroupParams P) {
  const long long total = P.out0[P.count];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = P.count - 1;  // the problem whose range holds t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.out0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int p = lo;
    const long long u = t - P.out0[p];
    const int M = P.M[p];
    const int r = (int)(u % M), c = (int)(u / M);
    if (P.c3[p]) {
      // Re = P1 - P2 (output row r), Im = P3 - P1 - P2 (row n + r), both scaled by row r
      const size_t stride_z = (size_t)M * P.N[p], set = (size_t)kOzModuli * stride_z;
      const uint8_t* R = P.R[p];
      uint32_t re[kOzModuli], im[kOzModuli];
#pragma unroll
      for (int j = 0; j < kOzModuli; ++j) {
        const uint32_t pj = (uint32_t)oz_modulus(j);
        const size_t at = (size_t)j * stride_z + (size_t)u;
        const uint32_t r1 = R[at], r2 = R[set + at], r3 = R[2 * set + at];
        re[j] = (r1 + pj - r2) % pj;
        im[j] = (r3 + 2 * pj - r1 - r2) % pj;
      }
      int sh;
      double x = crt_combine(re, &sh);
      crt_store(x, sh, r, c, P.rowexp[p], P.colexp[p], P.col0[p], P.alpha[p], P.beta[p], P.X64[p],
                P.gamma[p], P.Z64[p], P.out64[p], P.ldo[p]);
      x = crt_combine(im, &sh);
      crt_store(x, sh, M + r, c, P.rowexp[p], P.colexp[p], P.col0[p], P.alpha[p], P.beta[p], P.X64[p],
                P.gamma[p], P.Z64[p], P.out64[p], P.ldo[p], r);
      continue;
    }
    int sh;
    const double x = crt_value(P.R[p], (size_t)M * P.N[p], (size_t)u, 1, &sh);
    const int E = sh + P.rowexp[p][r] + P.colexp[p][P.col0[p] + c] - 2 * OZ_KBITS;
    const double v0 = (E > -1022 && E < 1024) ? x * __longlong_as_double((long long)(E + 1023) << 52)
                                              : ldexp(x, E);
    const size_t idx = (size_t)r + (size_t)(P.col0[p] + c) * P.ldo[p];
    double v = P.alpha[p] * v0;
    if (P.beta[p] != 0.0) v = fma(P.beta[p], P.X64[p][idx], v);
    if (P.gamma[p] != 0.0) v = fma(P.gamma[p], P.Z64[p][idx], v);
    P.out64[p][idx] = v;
  }
}

// ---------------- residues of the integer operands ----------------

// |x| as its IEEE bit pattern: for non-negative doubles the integer order is the numeric
// order, so row / column maxima need no FP64 instructions (FP64 issues at 2 per clock per
// SM here, integer work at 64).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ int exp_bound(unsigned long long amax_bits) {
  // smallest e with amax < 2^e (0 for an all-zero row/column)
  if (amax_bits == 0) return 0;
  int e;
  frexp(__longlong_as_double((long long)amax_bits), &e);  // amax = f 2^e, f in [0.5, 1)
  return e;
}

// x_int = round(x 2^{57 - e}) (|x| < 2^e, so |x_int| <= 2^57), from the significand and
// exponent fields (round half away from zero: the integer of -x is minus that of x).
__device__ __forceinline__ long long oz_int(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long m = bits & ((1LL << 52) - 1);
  long long X = 0;
  if (ex != 0x7FF) {
    int sh;
    if (ex == 0) {
      sh = 1 - 1075 + OZ_KBITS - e;  // subnormal: x = m 2^-1074
    } else {
      m |= 1LL << 52;
      sh = ex - 1075 + OZ_KBITS - e;  // x = m 2^{ex - 1075}; |x| < 2^e gives m 2^sh < 2^57
    }
    if (sh >= 0) X = m << sh;
    else if (sh > -64) X = (m + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) X = -X;
  }
  return X;
}

// Residues of an integer X (|X| < 2^59) mod p_j in symmetric range, stored as BF16 (exact:
// integers of magnitude <= 128) in plane j.
__device__ __forceinline__ void write_residues_int(long long X, __nv_bfloat16* base, size_t idx,
                                                   size_t plane) {
  // |X| = U1 2^29 + U0 with U0 < 2^29 and U1 < 2^30: |X| mod p = ((U1 mod p) (2^29 mod p) +
  // U0 mod p) mod p in 32-bit arithmetic (remainders by compile-time constants; the product
  // stays below 2^16)
  const unsigned long long U = (unsigned long long)(X < 0 ? -X : X);
  const uint32_t U1 = (uint32_t)(U >> 29), U0 = (uint32_t)(U & ((1u << 29) - 1));
#pragma unroll
  for (int j = 0; j < kOzModuli; ++j) {
    const uint32_t p = (uint32_t)oz_modulus(j);
    const uint32_t k29 = (uint32_t)((1ull << 29) % p);
    const uint32_t u = ((U1 % p) * k29 + U0 % p) % p;   // |X| mod p in [0, p)
    int rr = X < 0 ? -(int)u : (int)u;                   // X mod p in (-p, p), sign of X
    if (rr > (int)p / 2) rr -= (int)p;
    else if (rr < -((int)p / 2)) rr += (int)p;
    base[idx + (size_t)j * plane] = __int2bfloat16_rn(rr);  // exact: |rr| <= 128
  }
}

// The symmetric residues of X (|X| < 2^59) mod p_j as small integers (|r| <= 128).
__device__ __forceinline__ void residues_of(long long X, int* r) {
  const unsigned long long U = (unsigned long long)(X < 0 ? -X : X);
  const uint32_t U1 = (uint32_t)(U >> 29), U0 = (uint32_t)(U & ((1u << 29) - 1));
#pragma unroll
  for (int j = 0; j < kOzModuli; ++j) {
    const uint32_t p = (uint32_t)oz_modulus(j);
    const uint32_t k29 = (uint32_t)((1ull << 29) % p);
    const uint32_t u = ((U1 % p) * k29 + U0 % p) % p;
    int rr = X < 0 ? -(int)u : (int)u;
    if (rr > (int)p / 2) rr -= (int)p;
    else if (rr < -((int)p / 2)) rr += (int)p;
    r[j] = rr;
  }
}

// Residues of two adjacent K entries (idx, idx + 1) of three plane sets: the parts' integers
// Xr, Xi and their sum, whose residue is the sum of the parts' residues brought back into the
// symmetric range (a representative of the same class: the modular products use only the
// class, and |r| <= 128 keeps their K chunks exact).  Stored as BF16 pairs.
__device__ __forceinline__ void write_residues3_pair(long long xr0, long long xi0, long long xr1,
                                                     long long xi1, __nv_bfloat16* base, size_t idx,
                                                     size_t plane, size_t set) {
  int a0[kOzModuli], b0[kOzModuli], a1[kOzModuli], b1[kOzModuli];
  residues_of(xr0, a0);
  residues_of(xi0, b0);
  residues_of(xr1, a1);
  residues_of(xi1, b1);
#pragma unroll
  for (int j = 0; j < kOzModuli; ++j) {
    const int p = oz_modulus(j);
    int s0 = a0[j] + b0[j], s1 = a1[j] + b1[j];
    if (s0 > p / 2) s0 -= p; else if (s0 < -(p / 2)) s0 += p;
    if (s1 > p / 2) s1 -= p; else if (s1 < -(p / 2)) s1 += p;
    const size_t at = idx + (size_t)j * plane;
    *(__nv_bfloat162*)(base + at) = __nv_bfloat162(__int2bfloat16_rn(a0[j]), __int2bfloat16_rn(a1[j]));
    *(__nv_bfloat162*)(base + set + at) = __nv_bfloat162(__int2bfloat16_rn(b0[j]), __int2bfloat16_rn(b1[j]));
    *(__nv_bfloat162*)(base + 2 * set + at) = __nv_bfloat162(__int2bfloat16_rn(s0), __int2bfloat16_rn(s1));
  }
}

__device__ __forceinline__ void write_residues(double x, int e, __nv_bfloat16* base, size_t idx,
                                               size_t plane) {
  write_residues_int(oz_int(x, e), base, idx, plane);
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wi] = v;
  __syncthreads();
  unsigned long long mx = 0;
  for (int i = 0; i < nw; ++i) mx = red[i] > mx ? red[i] : mx;
  return mx;
}

// Stacked real A (M = n or 2n): residues of row m into planes (row-major, ld kp), row
// exponent into rowexp[m].  Row m of Ahat = column m of Ahat (symmetric), read from A.
template <class T>
__global__ void __launch_bounds__(256) oz_slice_A_kernel(int n, const T* __restrict__ A, int lda,
                                                         int kp, __nv_bfloat16* planes,
                                                         size_t plane, int* rowexp) {
  __shared__ unsigned long long red[8];
  const int m = blockIdx.x;
  const int mm = m % n;
  const bool mre = m < n;
  const int M = Sc<T>::cplx ? 2 * n : n;
  auto elem = [&](int k) -> double {
    if constexpr (Sc<T>::cplx) {
      const z64 a = A[(size_t)(k % n) + (size_t)mm * lda];  // A[k mod n, mm]
      const bool kre = k < n;
      return (kre == mre) ? a.x : (kre ? -a.y : a.y);
    } else {
      return A[(size_t)k + (size_t)m * lda];
    }
  };
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < M; k += 256) {
    const unsigned long long b = abs_bits(elem(k));
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) rowexp[m] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < M) ? elem(k) : 0.0;
    write_residues(x, e, planes, (size_t)m * kp + k, plane);
  }
}

// FP64 stacked block V64 (M x ncols, ld ldi): residues of column c into planes
// (column-major, ld kp; rows >= M zero), column exponent into colexp[c].
__global__ void __launch_bounds__(256) oz_slice_V_kernel(int M, int c0, const double* __restrict__ V64,
                                                         int ldi, int kp, __nv_bfloat16* planes,
                                                         size_t plane, int* colexp) {
  __shared__ unsigned long long red[8];
  const int c = c0 + blockIdx.x;
  const double* col = V64 + (size_t)c * ldi;
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < M; k += 256) {
    const unsigned long long b = abs_bits(col[k]);
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) colexp[c] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < M) ? col[k] : 0.0;
    write_residues(x, e, planes, (size_t)c * kp + k, plane);
  }
}

// ---- Gauss's three products for complex operands ----
// A = Ar + i Ai, V = Vr + i Vi: with the row exponents of A (over Re and Im together) and the
// column exponents of V as in the stacked form, the integers of Ar, Ai, Vr, Vi are those of
// the stacked operands, and
//   P1 = Ar Vr,  P2 = Ai Vi,  P3 = (Ar + Ai)(Vr + Vi)   (exact integer products mod p_j)
//   Re(A V) = P1 - P2,  Im(A V) = P3 - P1 - P2
// are the stacked product's two halves as the same integers: three real products of order n
// instead of one of order 2n (3/4 of the MMA work and of A's residue planes), the same
// results bit for bit.  The residues of Ar + Ai (|.| <= 2^58) come from the integer sums.
// Layout: three plane sets (Ar | Ai | Ar + Ai, or Vr | Vi | Vr + Vi), each kOzModuli planes,
// one after another.

// Row m of A (complex Hermitian, column-major): its three integer rows from column m of A
// (A[m, k] = conj(A[k, m])): Ar[m, k] = Re A[k, m], Ai[m, k] = -Im A[k, m].
__global__ void __launch_bounds__(256) oz_slice_A3_kernel(int n, const z64* __restrict__ A, int lda,
                                                          int kpn, __nv_bfloat16* planes, size_t plane,
                                                          size_t set, int* rowexp) {
  __shared__ unsigned long long red[8];
  const int m = blockIdx.x;
  const z64* col = A + (size_t)m * lda;
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < n; k += 256) {
    const unsigned long long b = max(abs_bits(col[k].x), abs_bits(col[k].y));
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) rowexp[m] = e;
  for (int k = 2 * threadIdx.x; k < kpn; k += 512) {  // kpn is even: pairs (k, k + 1)
    long long xr[2] = {0, 0}, xi[2] = {0, 0};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (k + d < n) {
        const z64 a = col[k + d];
        xr[d] = oz_int(a.x, e);
        xi[d] = -oz_int(a.y, e);
      }
    }
    write_residues3_pair(xr[0], xi[0], xr[1], xi[1], planes, (size_t)m * kpn + k, plane, set);
  }
}

// Column c of the stacked FP64 block V64 ([Re V; Im V], 2n rows, ld ldi): its exponent over
// both halves, then the three integer columns (Vr | Vi | Vr + Vi), ld kpn.
__device__ __forceinline__ void slice_V3_column(int n, int c, const double* __restrict__ V64, int ldi,
                                                int kpn, __nv_bfloat16* planes, size_t plane, size_t set,
                                                int* colexp, unsigned long long* red) {
  const double* col = V64 + (size_t)c * ldi;
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < 2 * n; k += 256) {
    const unsigned long long b = abs_bits(col[k]);
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) colexp[c] = e;
  for (int k = 2 * threadIdx.x; k < kpn; k += 512) {  // kpn is even: pairs (k, k + 1)
    long long xr[2] = {0, 0}, xi[2] = {0, 0};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (k + d < n) {
        xr[d] = oz_int(col[k + d], e);
        xi[d] = oz_int(col[n + k + d], e);
      }
    }
    write_residues3_pair(xr[0], xi[0], xr[1], xi[1], planes, (size_t)c * kpn + k, plane, set);
  }
}

// Grouped form of oz_slice_V_kernel: one block per sliced column of every problem.
struct SliceGroupParams {
  const double* V64[kOzGroupMax];
  __nv_bfloat16* planes[kOzGroupMax];
  int* colexp[kOzGroupMax];
  long long plane[kOzGroupMax];
  int blk0[kOzGroupMax + 1];  // first block of each problem
  int M[kOzGroupMax], c0[kOzGroupMax], ldi[kOzGroupMax], kp[kOzGroupMax];
  int c3[kOzGroupMax];  // complex problem in the three-product layout (M = n)
  int count;
};
static_assert(sizeof(SliceGroupParams) <= 32000, "kernel parameter space");

__global__ void __launch_bounds__(256) oz_slice_V_group_kernel(const __grid_constant__ SliceGroupParams P) {
  __shared__ unsigned long long red[8];
  int p = 0;
  while (p + 1 < P.count && (int)blockIdx.x >= P.blk0[p + 1]) ++p;
  const int c = P.c0[p] + (blockIdx.x - P.blk0[p]);
  const int M = P.M[p], kp = P.kp[p];
  if (P.c3[p]) {
    slice_V3_column(M, c, P.V64[p], P.ldi[p], kp, P.planes[p], (size_t)P.plane[p],
                    (size_t)kOzModuli * P.plane[p], P.colexp[p], red);
    return;
  }
  const double* col = P.V64[p] + (size_t)c * P.ldi[p];
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < M; k += 256) {
    const unsigned long long b = abs_bits(col[k]);
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) P.colexp[p][c] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < M) ? col[k] : 0.0;
    write_residues(x, e, P.planes[p], (size_t)c * kp + k, (size_t)P.plane[p]);
  }
}

// Caller's block V (n x ncols, ld ldv) -> stacked FP64 (M x ncols, ld ldo).
template <class T>
__global__ void stack_V_kernel(int n, int ncols, const T* __restrict__ V, int ldv, double* V64,
                               int ldo) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t total = (size_t)M * ncols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), a = (int)(t / M);
    double x;
    if constexpr (Sc<T>::cplx) {
      const z64 v = V[(size_t)(i % n) + (size_t)a * ldv];
      x = (i < n) ? v.x : v.y;
    } else {
      x = V[(size_t)i + (size_t)a * ldv];
    }
    V64[(size_t)i + (size_t)a * ldo] = x;
  }
}

// Xt (l x n, ld ldt) is the transpose of a column-major X (n x l): row m of X is column m
// of Xt.  Residues of the rows of the stacked operator [[Xr, -Xi], [Xi, Xr]] (2n x 2l;
// real: X itself, n x l) into planes (row-major, ld kp), row exponents into rowexp.
template <class T>
__global__ void __launch_bounds__(256) oz_slice_rows_kernel(int n, int l, const T* __restrict__ Xt,
                                                            int ldt, int kp, __nv_bfloat16* planes,
                                                            size_t plane, int* rowexp) {
  __shared__ unsigned long long red[8];
  const int m = blockIdx.x;
  const int mm = Sc<T>::cplx ? (m % n) : m;
  const bool mre = !Sc<T>::cplx || m < n;
  const int K = Sc<T>::cplx ? 2 * l : l;
  const T* row = Xt + (size_t)mm * ldt;  // X[mm, 0..l)
  auto elem = [&](int k) -> double {
    if constexpr (Sc<T>::cplx) {
      const z64 x = row[k % l];
      const bool kre = k < l;
      // [[Xr, -Xi], [Xi, Xr]]
      return mre ? (kre ? x.x : -x.y) : (kre ? x.y : x.x);
    } else {
      return row[k];
    }
  };
  unsigned long long amax = 0;
  for (int k = threadIdx.x; k < K; k += 256) {
    const unsigned long long b = abs_bits(elem(k));
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) rowexp[m] = e;
  for (int k = threadIdx.x; k < kp; k += 256) {
    const double x = (k < K) ? elem(k) : 0.0;
    write_residues(x, e, planes, (size_t)m * kp + k, plane);
  }
}

// Residues of the columns of a block Y (n x q, ld ldy) in stacked form: plane column j < q
// holds [Re Y; Im Y][:, j]; with `pair` (complex only) plane column q + j holds the stacked
// -i Y[:, j] = [Im Y; -Re Y][:, j].  Then, with X's columns as the left operand's rows,
// Xhat^T [Yhat | stack(-i Y)] = [Re(X^H Y) | Im(X^H Y)].  Both columns of a pair share the
// exponent of Y[:, j].  Planes column-major (ld kp; rows >= M are zero).
template <class T>
__global__ void __launch_bounds__(512) oz_slice_cols_kernel(int n, int q, const T* __restrict__ Y,
                                                            int ldy, int kp, bool pair,
                                                            __nv_bfloat16* planes, size_t plane,
                                                            int* colexp) {
  __shared__ unsigned long long red[16];
  const int j = blockIdx.x;
  const int M = Sc<T>::cplx ? 2 * n : n;
  const T* col = Y + (size_t)j * ldy;
  unsigned long long amax = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    unsigned long long b;
    if constexpr (Sc<T>::cplx) {
      const unsigned long long b0 = abs_bits(col[i].x), b1 = abs_bits(col[i].y);
      b = b0 > b1 ? b0 : b1;
    } else {
      b = abs_bits(col[i]);
    }
    amax = b > amax ? b : amax;
  }
  const int e = exp_bound(block_max(amax, red));
  if (threadIdx.x == 0) {
    colexp[j] = e;
    if (pair) colexp[q + j] = e;
  }
  for (int k = threadIdx.x; k < kp; k += blockDim.x) {
    double x = 0.0, y = 0.0;
    if (k < M) {
      if constexpr (Sc<T>::cplx) {
        const z64 v = col[k % n];
        x = (k < n) ? v.x : v.y;
        y = (k < n) ? v.y : -v.x;
      } else {
        x = col[k];
      }
    }
    write_residues(x, e, planes, (size_t)j * kp + k, plane);
    if (pair) write_residues(y, e, planes, (size_t)(q + j) * kp + k, plane);
  }
}

// out (l x 2l FP64, ld ldo) -> G (l x l, ld ldg) with G = out[:, :l] + i out[:, l:] (real: copy)
template <class T>
__global__ void gram_assemble_kernel(int qx, int qy, const double* __restrict__ out, int ldo, T* G,
                                     int ldg) {
  const size_t total = (size_t)qx * qy;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(t % qx), q = (int)(t / qx);
    if constexpr (Sc<T>::cplx) {
      G[(size_t)p + (size_t)q * ldg] = z64{out[(size_t)p + (size_t)q * ldo], out[(size_t)p + (size_t)(q + qy) * ldo]};
    } else {
      G[(size_t)p + (size_t)q * ldg] = out[(size_t)p + (size_t)q * ldo];
    }
  }
}

// Xt = X^T (plain transpose, no conjugation): X n x l (ld ldx) -> Xt l x n (ld ldt).
template <class T>
__global__ void transpose_kernel(int n, int l, const T* __restrict__ X, int ldx, T* Xt, int ldt) {
  __shared__ T tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + threadIdx.x, j = j0 + r;
    if (i < n && j < l) tile[r][threadIdx.x] = X[(size_t)i + (size_t)j * ldx];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + threadIdx.x, i = i0 + r;
    if (i < n && j < l) Xt[(size_t)j + (size_t)i * ldt] = tile[threadIdx.x][r];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  // looked up once (thread-safe static initialisation: batch sessions call from several threads)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return nullptr;
  }();
  return fn;
}

// 3-D BF16 map over the residue planes: {kp (contiguous), rows, S}, box {64, box_rows, 1},
// 128-byte swizzle; consecutive planes are plane_rows * kp elements apart.
int make_map3(CUtensorMap* map, const void* base, int kp, int rows, int plane_rows, int box_rows) {
  auto enc = encoder();
  if (!enc) return CHASE_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)kOzModuli};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)plane_rows};
  cuuint32_t box[3] = {MBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : CHASE_ERR_CUDA;
}

}  // namespace

size_t oz_residue_bytes(int M, int N) {
  return (size_t)kOzMaxSplits * kOzModuli * (size_t)M * (size_t)N;
}

template <class T>
int oz_slice_A(cudaStream_t st, int n, const T* A, int lda, int kp, void* planes, int* rowexp,
               int* launches) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  oz_slice_A_kernel<T><<<M, 256, 0, st>>>(n, A, lda, kp, (__nv_bfloat16*)planes,
                                          (size_t)M * kp, rowexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

int oz_slice_A3(cudaStream_t st, int n, const z64* A, int lda, int kpn, void* planes, int* rowexp,
                int* launches) {
  const size_t plane = (size_t)n * kpn;
  oz_slice_A3_kernel<<<n, 256, 0, st>>>(n, A, lda, kpn, (__nv_bfloat16*)planes, plane,
                                        (size_t)kOzModuli * plane, rowexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

int oz_slice_V(cudaStream_t st, int M, int c0, int c1, const double* V64, int ldi, int kp,
               int ncols_total, void* planes, int* colexp, int* launches) {
  if (c1 <= c0) return 0;
  oz_slice_V_kernel<<<c1 - c0, 256, 0, st>>>(M, c0, V64, ldi, kp, (__nv_bfloat16*)planes,
                                             (size_t)ncols_total * kp, colexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

namespace {

// Launch with clusters of two CTAs along x (the CTA pairs of the modular products).
template <class... Params, class... Args>
int launch_pairs(void (*kernel)(Params...), dim3 grid, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(M_THREADS);
  cfg.dynamicSmemBytes = M_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CHASE_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, args...));
  return 0;
}

// The modular products of one plan; returns the number of K splits their residues hold in
// *splits.
int ozm_launch(cudaStream_t st, int M, int kp, const void* Aplanes, int a_plane_rows,
               const void* Vplanes, int ncols_total, int col0, int N, DevStatus* dst,
               Scratch resbuf, int* launches, const OzPlan& plan, int* splits) {
  if (a_plane_rows < M) a_plane_rows = M;
  // column tiles of at most plan.bn_max (a multiple of 16), as even as possible
  const int ntile = ceil_div(N, std::min(plan.bn_max, MBN_MAX));
  const int BN = ceil_div(ceil_div(N, ntile), 16) * 16;
  CUtensorMap mA, mV;
  if (make_map3(&mA, Aplanes, kp, M, a_plane_rows, MBM) ||
      make_map3(&mV, Vplanes, kp, ncols_total, ncols_total, BN / 2))
    return CHASE_ERR_CUDA;
  CHASE_CUDA_TRY(cudaFuncSetAttribute(ozm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, M_SMEM));
  const int nkb = kp / MBK;
  const int mblk = ceil_div(M, 2 * MBM) * 2;  // 128-row blocks, an even number (CTA pairs)
  const size_t slab = (size_t)kOzModuli * (size_t)M * N;  // residue bytes of one split
  // split K (whole 1024-wide chunks) until there are about four waves of CTAs
  constexpr int kChunkKB = 1024 / MBK;  // K blocks of one exact chunk
  const int nchunks = ceil_div(nkb, kChunkKB);
  int S = std::max(1, std::min(nchunks, ceil_div(4 * kNumSMs, ntile * mblk * kOzModuli)));
  if (plan.splits > 0) S = std::min(plan.splits, nchunks);
  // no split longer than kOzSplitMaxK (the range of the epilogue's exact reduction)
  const int min_S = ceil_div(nchunks, kOzSplitMaxK / 1024);
  S = std::max(std::min(S, kOzMaxSplits), min_S);
  while (S > min_S && (size_t)S * slab > resbuf.bytes) --S;
  if ((size_t)S * slab > resbuf.bytes) return CHASE_ERR_OOM;
  const int kbs = ceil_div(nchunks, S) * kChunkKB;  // whole chunks: every split starts on an even block
  S = ceil_div(nkb, kbs);
  TRY_OZ(launch_pairs(ozm_kernel, dim3(ntile * mblk, 1, kOzModuli * S), st, mA, mV, M, N, BN, ntile,
                      col0, nkb, kbs, (uint8_t*)resbuf.ptr, dst));
  if (launches) ++*launches;
  *splits = S;
  return 0;
}

int crt_launch(cudaStream_t st, int M, int N, int S, Scratch resbuf, const int* rowexp,
               const int* colexp, int col0, double alpha, double beta, const double* X64,
               double gamma, const double* Z64, double* out64, int ldo, int* launches) {
  const size_t total = (size_t)M * N;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)kNumSMs * 16));
  if (total % 4 == 0) {
    const int b4 = (int)std::max<size_t>(1, std::min<size_t>((total / 4 + 255) / 256, (size_t)kNumSMs * 16));
    crt4_kernel<<<b4, 256, 0, st>>>(M, N, S, (const uint8_t*)resbuf.ptr, rowexp, colexp, col0, alpha, beta,
                                    X64, gamma, Z64, out64, ldo);
  } else {
    crt_kernel<<<blocks, 256, 0, st>>>(M, N, S, (const uint8_t*)resbuf.ptr, rowexp, colexp, col0, alpha,
                                       beta, X64, gamma, Z64, out64, ldo);
  }
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace

int oz_gemm(cudaStream_t st, int M, int kp, const void* Aplanes, const int* rowexp,
            int a_plane_rows, const void* Vplanes, const int* colexp, int ncols_total, int col0,
            int N, double alpha, double beta, const double* X64, double gamma, const double* Z64,
            double* out64, int ldo, DevStatus* dst, Scratch resbuf, int* launches, int tune,
            int* trials) {
  if (N <= 0 || M <= 0) return 0;
  if (kp % MBK != 0 || kp > kOzMaxK) return CHASE_ERR_UNSUPPORTED;
  OzPlan plan;
  const bool known = oz_plan_lookup(M, N, kp, &plan);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (tune && !known && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
      cs == cudaStreamCaptureStatusNone) {
    // time the modular products of every candidate plan (they read only the residue planes
    // and all yield the same exact residues), keep the fastest, then run it once more and
    // reconstruct: the three-term update, which may read its own output, runs once
    OzPlan cand[6];
    const int nc = oz_plan_candidates(N, cand, 6);
    cudaEvent_t ev[7];
    for (int i = 0; i <= nc; ++i) CHASE_CUDA_TRY(cudaEventCreate(&ev[i]));
    int rc = 0, S = 1;
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < nc && !rc; ++i) {
      rc = ozm_launch(st, M, kp, Aplanes, a_plane_rows, Vplanes, ncols_total, col0, N, dst, resbuf,
                      launches, cand[i], &S);
      cudaEventRecord(ev[i + 1], st);
    }
    if (!rc && cudaEventSynchronize(ev[nc]) == cudaSuccess) {
      int best = 0;
      float tbest = 1e30f;
      for (int i = 0; i < nc; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        if (ms < tbest) { tbest = ms; best = i; }
      }
      oz_plan_store(M, N, kp, cand[best], tbest * 1e-3);
      if (trials) *trials += nc;
      plan = cand[best];
    }
    for (int i = 0; i <= nc; ++i) cudaEventDestroy(ev[i]);
    if (rc) return rc;
  }
  int S = 1;
  TRY_OZ(ozm_launch(st, M, kp, Aplanes, a_plane_rows, Vplanes, ncols_total, col0, N, dst, resbuf,
                    launches, plan, &S));
  return crt_launch(st, M, N, S, resbuf, rowexp, colexp, col0, alpha, beta, X64, gamma, Z64, out64,
                    ldo, launches);
}

int oz_slice_V_group(cudaStream_t st, int count, const OzGroupItem* items, int* launches) {
  for (int g0 = 0; g0 < count; g0 += kOzGroupMax) {
    const int cnt = std::min(kOzGroupMax, count - g0);
    SliceGroupParams P{};
    int blocks = 0;
    P.count = 0;
    for (int i = 0; i < cnt; ++i) {
      const OzGroupItem& it = items[g0 + i];
      if (it.N <= 0) continue;
      const int p = P.count++;
      P.V64[p] = it.V64_in;
      P.planes[p] = (__nv_bfloat16*)const_cast<void*>(it.Vplanes);
      P.colexp[p] = const_cast<int*>(it.colexp);
      P.plane[p] = (long long)it.ncols_total * it.kp;
      P.blk0[p] = blocks;
      P.M[p] = it.M;
      P.c0[p] = it.col0;
      P.ldi[p] = it.ldi;
      P.kp[p] = it.kp;
      P.c3[p] = it.c3;
      blocks += it.N;
    }
    if (P.count == 0) continue;
    P.blk0[P.count] = blocks;
    oz_slice_V_group_kernel<<<blocks, 256, 0, st>>>(P);
    if (launches) ++*launches;
    CHASE_CUDA_TRY(cudaGetLastError());
  }
  return 0;
}

int oz_gemm_group(cudaStream_t st, int count, const OzGroupItem* items, DevStatus* dst, int* launches) {
  CHASE_CUDA_TRY(cudaFuncSetAttribute(ozm_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, M_SMEM));
  OzmGroupParams P{};
  CrtGroupParams C{};
  int tiles = 0;
  long long outs = 0;
  // one launch of the modular products and one of the reconstructions for what is gathered
  auto flush = [&]() -> int {
    if (P.count == 0) return 0;
    P.tile0[P.count] = tiles;
    C.out0[C.count] = outs;
    TRY_OZ(launch_pairs(ozm_group_kernel, dim3(tiles, 1, kOzModuli), st, P, dst));
    if (launches) ++*launches;
    if (C.count == 1 && C.c3[0] && outs % 4 == 0) {  // one complex problem: the vector form
      const int b4 = (int)std::max<long long>(1, std::min<long long>((outs / 4 + 255) / 256, (long long)kNumSMs * 16));
      crt3_kernel<<<b4, 256, 0, st>>>(C.M[0], C.N[0], C.R[0], C.rowexp[0], C.colexp[0], C.col0[0],
                                      C.alpha[0], C.beta[0], C.X64[0], C.gamma[0], C.Z64[0],
                                      C.out64[0], C.ldo[0]);
    } else {
      const int blocks = (int)std::max<long long>(1, std::min<long long>((outs + 255) / 256, (long long)kNumSMs * 16));
      crt_group_kernel<<<blocks, 256, 0, st>>>(C);
    }
    if (launches) ++*launches;
    CHASE_CUDA_TRY(cudaGetLastError());
    P = OzmGroupParams{};
    C = CrtGroupParams{};
    tiles = 0;
    outs = 0;
    return 0;
  };
  for (int i = 0; i < count; ++i) {
    const OzGroupItem& it = items[i];
    if (it.N <= 0 || it.M <= 0) continue;
    if (it.kp % MBK != 0 || it.kp > kOzSplitMaxK) return CHASE_ERR_UNSUPPORTED;  // K is not split here
    const int sets = it.c3 ? 3 : 1;  // three-product layout: P1, P2, P3
    if ((size_t)sets * kOzModuli * it.M * it.N > it.resbuf.bytes) return CHASE_ERR_OOM;
    if (P.count + sets > kOzGroupMax || C.count + 1 > kOzGroupMax) TRY_OZ(flush());
    OzPlan plan;  // the autotuner's tile width for this shape, if it measured one
    oz_plan_lookup(it.M, it.N, it.kp, &plan);
    const int ntile = ceil_div(it.N, std::min(plan.bn_max, MBN_MAX));
    const int BN = ceil_div(ceil_div(it.N, ntile), 16) * 16;
    const int rows = std::max(it.a_plane_rows, it.M);
    const size_t aset = (size_t)kOzModuli * rows * it.kp * 2;             // bytes of one A plane set
    const size_t vset = (size_t)kOzModuli * it.ncols_total * it.kp * 2;   // of one V plane set
    for (int sidx = 0; sidx < sets; ++sidx) {
      const int p = P.count++;
      if (make_map3(&P.mapA[p], (const char*)it.Aplanes + sidx * aset, it.kp, it.M, rows, MBM) ||
          make_map3(&P.mapV[p], (const char*)it.Vplanes + sidx * vset, it.kp, it.ncols_total,
                    it.ncols_total, BN / 2))
        return CHASE_ERR_CUDA;
      P.R[p] = (uint8_t*)it.resbuf.ptr + (size_t)sidx * kOzModuli * it.M * it.N;
      P.tile0[p] = tiles;
      P.M[p] = it.M;
      P.N[p] = it.N;
      P.BN[p] = BN;
      P.col0[p] = it.col0;
      P.ntile[p] = ntile;
      P.nkb[p] = it.kp / MBK;
      tiles += ntile * ceil_div(it.M, 2 * MBM) * 2;  // CTA pairs over 256-row blocks
    }
    const int c = C.count++;
    C.R[c] = (const uint8_t*)it.resbuf.ptr;
    C.rowexp[c] = it.rowexp;
    C.colexp[c] = it.colexp;
    C.X64[c] = it.X64;
    C.Z64[c] = it.Z64;
    C.out64[c] = it.out64;
    C.alpha[c] = it.alpha;
    C.beta[c] = it.beta;
    C.gamma[c] = it.gamma;
    C.out0[c] = outs;
    C.M[c] = it.M;
    C.N[c] = it.N;
    C.col0[c] = it.col0;
    C.ldo[c] = it.ldo;
    C.c3[c] = it.c3;
    outs += (long long)it.M * it.N;
  }
  return flush();
}

template <class T>
int oz_stack_V(cudaStream_t st, int n, int ncols, const T* V, int ldv, double* V64, int ldo,
               int* launches) {
  if (ncols <= 0) return 0;
  const int M = Sc<T>::cplx ? 2 * n : n;
  const size_t work = (size_t)M * ncols;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((work + 255) / 256, (size_t)kNumSMs * 16));
  stack_V_kernel<T><<<blocks, 256, 0, st>>>(n, ncols, V, ldv, V64, ldo);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_slice_rows(cudaStream_t st, int n, int l, const T* Xt, int ldt, int kp, void* planes,
                  int* rowexp, int* launches) {
  const int M = Sc<T>::cplx ? 2 * n : n;
  oz_slice_rows_kernel<T><<<M, 256, 0, st>>>(n, l, Xt, ldt, kp, (__nv_bfloat16*)planes,
                                             (size_t)M * kp, rowexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_slice_cols(cudaStream_t st, int n, int q, const T* Y, int ldy, int kp, bool pair,
                  void* planes, int* colexp, int* launches) {
  if (q <= 0) return 0;
  pair = pair && Sc<T>::cplx;
  const size_t ncols_total = pair ? 2 * (size_t)q : (size_t)q;
  oz_slice_cols_kernel<T><<<q, 512, 0, st>>>(n, q, Y, ldy, kp, pair, (__nv_bfloat16*)planes,
                                             ncols_total * kp, colexp);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int oz_gram_assemble(cudaStream_t st, int qx, int qy, const double* out, int ldo, T* G, int ldg,
                     int* launches) {
  const size_t work = (size_t)qx * qy;
  if (work == 0) return 0;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((work + 255) / 256, (size_t)kNumSMs * 16));
  gram_assemble_kernel<T><<<blocks, 256, 0, st>>>(qx, qy, out, ldo, G, ldg);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <class T>
int transpose(cudaStream_t st, int n, int l, const T* X, int ldx, T* Xt, int ldt, int* launches) {
  dim3 grid(ceil_div(n, 32), ceil_div(l, 32)), block(32, 8);
  transpose_kernel<T><<<grid, block, 0, st>>>(n, l, X, ldx, Xt, ldt);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

#define OZ_INST(T)                                                                                \
  template int oz_slice_rows<T>(cudaStream_t, int, int, const T*, int, int, void*, int*, int*);   \
  template int oz_slice_cols<T>(cudaStream_t, int, int, const T*, int, int, bool, void*, int*,   \
                                int*);                                                            \
  template int oz_gram_assemble<T>(cudaStream_t, int, int, const double*, int, T*, int, int*);    \
  template int transpose<T>(cudaStream_t, int, int, const T*, int, T*, int, int*);
OZ_INST(double)
OZ_INST(z64)
#undef OZ_INST

template int oz_stack_V<double>(cudaStream_t, int, int, const double*, int, double*, int, int*);
template int oz_stack_V<z64>(cudaStream_t, int, int, const z64*, int, double*, int, int*);
template int oz_slice_A<double>(cudaStream_t, int, const double*, int, int, void*, int*, int*);
template int oz_slice_A<z64>(cudaStream_t, int, const z64*, int, int, void*, int*, int*);

}  // namespace chase
