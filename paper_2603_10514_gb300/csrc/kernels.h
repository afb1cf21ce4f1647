// kernels.h -- internal launchers of the GB300 kernels (not part of the C ABI).
// Every launcher enqueues work on `st` and returns 0 or a chase_status code.
#pragma once

#include "common.cuh"

namespace chase {

// Device scratch memory handed to a launcher (split-K partial sums etc.).
struct Scratch {
  void* ptr;
  size_t bytes;
};

// C = alpha * op(A) B + beta * X + gamma * Y  (op = identity or ^H); see gemm_fp64.cu.
// upper_only: only C[i, j] with i <= j is needed (Hermitian results).
// tri_b: B is upper triangular (entries below its diagonal are zero and skipped).
template <class T>
int gemm(cudaStream_t st, bool transA, int M, int N, int K, const T* A, int lda, const T* B,
         int ldb, T* C, int ldc, double alpha, double beta, const T* X, int ldx, double gamma,
         const T* Y, int ldy, Scratch scratch, bool upper_only, bool tri_b, int* launches);

// ---- dense small-matrix kernels (chol_trsm.cu) ----------------------------
// Upper Cholesky of G in place; info (first failing pivot + 1) goes to dst->chol_info.
// shift_factor > 0 first adds s = shift_factor * trace(G) to the diagonal (the shifted
// CholeskyQR step: trace(X^H X) = ||X||_F^2).
template <class T>
int potrf_upper(cudaStream_t st, int n, T* G, int ldg, double shift_factor, DevStatus* dst,
                int* launches);
// Blocked (64) variant for larger n: diagonal blocks on one CTA, block rows and
// trailing updates as products.  scratch: 64*64 + 64*n elements; the strict lower
// triangle of G is left as it was.
template <class T>
int potrf_upper_blocked(cudaStream_t st, int n, T* G, int ldg, double shift_factor, DevStatus* dst,
                        T* scratch, Scratch gscr, int* launches);
// Rinv = R^{-1} for upper-triangular R (zero strict lower part written).
template <class T>
int trtri_upper(cudaStream_t st, int n, const T* R, int ldr, T* Rinv, int ldri, int* launches);

// ---- Householder QR with explicit thin Q (householder.cu) -----------------
template <class T>
int householder_qr(cudaStream_t st, int n, int l, T* X, int ldx, T* Vh, int ldv, double* dnorm,
                   int* launches);
// Blocked form's pieces: reflectors j0 .. j0+b-1 into Vh[:, j0..] applied within the panel
// only; the compact WY factor T (b x b, ld ldt) from G = V^H V; X <- [I; 0] (n x l).
template <class T>
int hh_panel(cudaStream_t st, int n, int j0, int b, T* X, int ldx, T* Vh, int ldv, int* launches);
// The panel step as one cooperative launch (rows split over up to 152 CTAs, two bounded
// grid barriers per column), which also writes the panel Gram V^H V (upper, ld ldg).
// CHASE_ERR_UNSUPPORTED when the grid cannot be co-resident or a slice is too tall (the
// caller then takes hh_panel and a product for the Gram); a wait that ran out sets
// dst->timeout.  Scratch: at least 256 + (b + b(b+1)/2) * 1216 elements.
template <class T>
int hh_panel_coop(cudaStream_t st, int n, int j0, int b, T* X, int ldx, T* Vh, int ldv, T* Gp, int ldg,
                  Scratch ws, DevStatus* dst, int* launches);
template <class T>
int hh_build_T(cudaStream_t st, int b, const T* G, int ldg, T* Tm, int ldt, int* launches);
template <class T>
int hh_thin_identity(cudaStream_t st, int n, int l, T* X, int ldx, int* launches);

// ---- parallel cyclic Jacobi eigensolver (jacobi.cu) ------------------------
// Diagonalises the Hermitian H (l x l, overwritten).  Eigenvalues (ascending)
// go to dw (device) and eigenvectors to W.  Returns sweeps used through *sweeps.
// One cooperative launch runs every sweep; work: jacobi_work_bytes(l, sizeof(T)) bytes.
// Returns 5 (CHASE_ERR_TIMEOUT) if a bounded grid-barrier wait ran out.
constexpr int kJacobiMaxCtas = 1216;  // 8 CTAs of 256 threads on each of the 152 SMs
size_t jacobi_work_bytes(int l, size_t elem);
// ctas > 0 fixes the grid size (at most one wave of co-resident CTAs); 0 picks it from l.
template <class T>
int jacobi_eig(cudaStream_t st, int l, T* H, int ldh, T* W, int ldw, double* dw, void* work,
               size_t work_bytes, int max_sweeps, int* sweeps, int* launches, int ctas = 0);

// ---- streaming kernels (vec.cu) --------------------------------------------
template <class T>
int herm_fill_lower(cudaStream_t st, int n, T* G, int ldg, int* launches);
// r_a = || AV[:,a] - theta_a V[:,a] || / || V[:,a] ||
template <class T>
int resid_norms(cudaStream_t st, int n, int ncols, const T* AV, int ldav, const T* V, int ldv,
                const double* dtheta, double* dres, int* launches);
template <class T>
int copy_cols(cudaStream_t st, int n, int ncols, const T* src, int lds, T* dst, int ldd,
              int* launches);
// dst[:, a] = src[:, perm[a]]  (dperm on device)
template <class T>
int gather_cols(cudaStream_t st, int n, int ncols, const T* src, int lds, const int* dperm, T* dst,
                int ldd, int* launches);
// dst[:, a] = src_{sel[a]}[:, a] with sel[a] in {0,1}: picks each column from one of two buffers
template <class T>
int select_cols(cudaStream_t st, int n, int ncols, const T* src0, const T* src1, int lds,
                const int* dsel, T* dst, int ldd, int* launches);
template <class T>
int nonfinite_check(cudaStream_t st, int n, int ncols, const T* X, int ldx, DevStatus* dst,
                    int* launches);

// ---- tensor-core (tcgen05) split-BF16 filter product (gemm_tc.cu) ---------
// Stacked-real operands: M = n (real) or 2n (complex) rows; kp = M rounded up to 64.
int tc_kpad(int M);
template <class T>
int tc_split_A(cudaStream_t st, int n, const T* A, int lda, int kp, void* Ah, void* Al,
               int* launches);
template <class T>
int tc_split_V(cudaStream_t st, int n, int ncols, const T* V, int ldv, double* V64, int ldo, int kp,
               void* Vh, void* Vl, int* launches);
// V[:, c0:c1] = unstack(V64) (complex: rows i and n + i of V64 are the real and imaginary
// parts); with subtract, V[:, c0:c1] -= unstack(V64).
template <class T>
int tc_unstack_V(cudaStream_t st, int n, int c0, int c1, const double* V64, int ldi, T* V, int ldv,
                 int* launches, bool subtract = false);
// One filter step on columns [col0, col0 + N) of the stacked block (ld kp everywhere).
int tc_filter_step(cudaStream_t st, int M, int kp, const void* Ah, const void* Al,
                   const void* Vh_in, const void* Vl_in, int ncols_total, int col0, int N,
                   double alpha, double beta, const double* X64, double gamma, const double* Z64,
                   double* out64, int ldv, void* Vh_out, void* Vl_out, DevStatus* dst,
                   int* launches);

// ---- FP64-accurate products on BF16 tensor cores (gemm_oz.cu, Ozaki scheme II) -
// Operands become 57-bit integers (one power-of-two scale per row / column); their
// residues mod 17 pairwise coprime moduli <= 256 are BF16 planes.  A planes: row-major
// (M x kp), V planes: column-major (kp x ncols); kp = K rounded up to 64 (zero padded).
constexpr int kOzModuli = 17;                   // residue planes per operand
constexpr size_t kOzPlaneBytes = 2 * kOzModuli; // bytes of residue planes per operand element
constexpr int kOzMaxSplits = 2;                 // K splits of one product (residue slabs)
constexpr int kOzMaxK = 1 << 17;                // longest K the moduli's product covers
constexpr int kOzSplitMaxK = 1 << 16;           // longest K of one split: |sum| <= 2^16 * 128^2 = 2^30,
                                                // the range of the modular epilogue's reduction
// Device bytes of the residue buffer oz_gemm needs for an M x N product.
size_t oz_residue_bytes(int M, int N);
template <class T>
int oz_slice_A(cudaStream_t st, int n, const T* A, int lda, int kp, void* planes, int* rowexp,
               int* launches);
// Complex A (n x n, Hermitian, column-major) into the three-product layout: plane sets
// Re A | Im A | Re A + Im A, each kOzModuli planes of n x kpn (row-major, K contiguous),
// row exponents over Re and Im together (those of the stacked form).
int oz_slice_A3(cudaStream_t st, int n, const z64* A, int lda, int kpn, void* planes, int* rowexp,
                int* launches);
int oz_slice_V(cudaStream_t st, int M, int c0, int c1, const double* V64, int ldi, int kp,
               int ncols_total, void* planes, int* colexp, int* launches);
template <class T>
int oz_stack_V(cudaStream_t st, int n, int ncols, const T* V, int ldv, double* V64, int ldo,
               int* launches);
// Row residues of the stacked operator of a general X given as Xt = X^T (l x n, ld ldt).
template <class T>
int oz_slice_rows(cudaStream_t st, int n, int l, const T* Xt, int ldt, int kp, void* planes,
                  int* rowexp, int* launches);
// Column residues of a block Y (n x q): plane column j = stacked Y[:, j] and, with pair
// (complex only), plane column q + j = stacked (-i Y[:, j]); plane stride (q or 2q) * kp.
template <class T>
int oz_slice_cols(cudaStream_t st, int n, int q, const T* Y, int ldy, int kp, bool pair,
                  void* planes, int* colexp, int* launches);
// G = out[:, :qy] + i out[:, qy:] (complex) or out (real); out qx x 2qy (or qx x qy), ld ldo;
// G qx x qy.
template <class T>
int oz_gram_assemble(cudaStream_t st, int qx, int qy, const double* out, int ldo, T* G, int ldg,
                     int* launches);
template <class T>
int transpose(cudaStream_t st, int n, int l, const T* X, int ldx, T* Xt, int ldt, int* launches);
// Launch plan of an emulated product: cap on the column-tile width (tiles as even as
// possible below it) and K splits (0: about four waves of CTAs, at most kOzMaxSplits).
struct OzPlan {
  int bn_max = 256;
  int splits = 0;
};
// The autotuner's table (autotune.cu): plans measured per shape bucket.
bool oz_plan_lookup(int M, int N, int kp, OzPlan* plan);
void oz_plan_store(int M, int N, int kp, const OzPlan& plan, double seconds);
int oz_plan_candidates(int N, OzPlan* out, int cap);
// out64[:, col0 + c] = alpha * (A V)[:, col0 + c] + beta * X64 + gamma * Z64 for c < N.
// A's planes are a_plane_rows * kp elements apart (0: M * kp).  resbuf: residues of the
// modular products, at least oz_residue_bytes(M, N) / kOzMaxSplits bytes (twice that lets
// the product split K).  kp must be a multiple of 64 and at most kOzMaxK.  The plan is the
// autotuner's pick for the shape's bucket if it has one, else the heuristic; tune = 1 first
// measures every candidate plan on this product (unless the stream is being captured) and
// records the fastest; *trials counts the candidate runs.
int oz_gemm(cudaStream_t st, int M, int kp, const void* Aplanes, const int* rowexp,
            int a_plane_rows, const void* Vplanes, const int* colexp, int ncols_total, int col0, int N, double alpha,
            double beta, const double* X64, double gamma, const double* Z64, double* out64, int ldo,
            DevStatus* dst, Scratch resbuf, int* launches, int tune = 0, int* trials = nullptr);

// One problem's product in a grouped launch (oz_slice_V_group + oz_gemm_group): the same
// operands and epilogue as oz_gemm, without K splits; V64_in / ldi: the FP64 stacked block
// whose columns [col0, col0 + N) oz_slice_V_group cuts into Vplanes first.
constexpr int kOzGroupMax = 64;  // problems per grouped launch (kernel parameter space)
struct OzGroupItem {
  int M = 0, kp = 0, a_plane_rows = 0;
  const void* Aplanes = nullptr;
  const int* rowexp = nullptr;
  const void* Vplanes = nullptr;
  const int* colexp = nullptr;
  int ncols_total = 0, col0 = 0, N = 0;
  double alpha = 1.0, beta = 0.0, gamma = 0.0;
  const double* X64 = nullptr;
  const double* Z64 = nullptr;
  double* out64 = nullptr;
  int ldo = 0;
  Scratch resbuf{nullptr, 0};
  const double* V64_in = nullptr;
  int ldi = 0;
  // complex problem in the three-product layout: M = n, Aplanes / Vplanes hold three plane
  // sets (Re | Im | Re + Im), V64_in / X64 / Z64 / out64 are the stacked [Re; Im] blocks
  int c3 = 0;
};
int oz_slice_V_group(cudaStream_t st, int count, const OzGroupItem* items, int* launches);
int oz_gemm_group(cudaStream_t st, int count, const OzGroupItem* items, DevStatus* dst, int* launches);

// ---- failure path of the bounded device waits (selftest.cu) ----------------
// One thread waits (at most `seconds`) on an mbarrier nothing arrives on and sets
// dst->timeout, as the kernels do when a wait runs out.
int selftest_wait_timeout(cudaStream_t st, double seconds, DevStatus* dst, int* launches);

// ---- Lanczos spectral bounds (lanczos.cu) ----------------------------------
// out = {lambda1, lambda_ell, b_sup} from nruns runs of m steps started at V0's columns.
template <class T>
int lanczos_bounds(cudaStream_t st, int n, const T* A, int lda, int nruns, const T* V0, int ldv,
                   int m, int ell, double* out, void* work, size_t work_bytes, Scratch scr,
                   int* launches);
size_t lanczos_work_bytes(size_t elem, int n, int nruns, int m);

}  // namespace chase
