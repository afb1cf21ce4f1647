/*
 * chase_oracle.c -- plain, slow, FP64 CPU restatement of Chebyshev-filtered
 * subspace iteration (the ChASE method) and of the condition-number estimate
 * that drives its QR choice.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: it exists so that the GPU library can be checked against
 * an independent implementation written directly from the paper
 * (Di Napoli & Wu, "Estimating the condition number of Chebyshev filtered
 * vectors with application to the ChASE library").  It shares no code,
 * header or constant with the CUDA path.
 *
 * Every quantity is FP64.  Real symmetric problems are handled by the same
 * complex routines with zero imaginary parts: every operation below maps real
 * data to real data (Householder phases and Jacobi phases reduce to +-1), so
 * a real problem is solved exactly as a real code would, only slower.
 *
 * Storage: column-major, leading dimensions as in LAPACK.  Index (i, j) of a
 * matrix X with leading dimension ldx is X[i + j*ldx].
 *
 * No blocking, fusion or reordering beyond what the definitions state.  The
 * only concession to speed is an OpenMP loop over output rows in the dense
 * block product, which leaves each output element's arithmetic unchanged.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "chase_oracle.h"

typedef double complex cplx;

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Unit round-off of IEEE binary64, u = 2^-53 (Section 1.3, Table 1). */
static const double ORC_U = 1.1102230246251565e-16;

/* ------------------------------------------------------------------------ */
/* Dense helpers (definitions only)                                         */
/* ------------------------------------------------------------------------ */

/* Y(:, 0:nc) = A * X(:, 0:nc), A is n x n.  Plain definition of the product
 * y_ia = sum_k A_ik x_ka. */
static void orc_matmul_block(int n, const cplx* A, int lda, int nc, const cplx* X, int ldx,
                             cplx* Y, int ldy) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    for (int a = 0; a < nc; ++a) {
      cplx s = 0;
      for (int k = 0; k < n; ++k) s += A[IDX(i, k, lda)] * X[IDX(k, a, ldx)];
      Y[IDX(i, a, ldy)] = s;
    }
  }
}

/* 2-norm of a vector. */
static double orc_nrm2(int n, const cplx* x) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
  return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Chebyshev polynomial filter (Algorithm 4, Section 2.3)                    */
/* ------------------------------------------------------------------------ */

/*
 * Applies p_{m_a}(A) to each column v_a of V (in place), where
 *   p_m(x) = C_m((x - c)/e) / C_m((lambda1 - c)/e)
 * is evaluated through the scaled three-term recurrence with
 *   sigma_1 = e / (lambda1 - c),   sigma_i = 1 / (2/sigma_1 - sigma_{i-1}),
 *   V_1 = (sigma_1/e)(A - cI) V_0,
 *   V_i = (2 sigma_i / e)(A - cI) V_{i-1} - sigma_{i-1} sigma_i V_{i-2}.
 * Column a stops after m_a steps (the per-column degrees of Section 2.3);
 * deg must be ascending and >= 0.  The interval [c-e, c+e] is the one that is
 * damped; lambda1 lies below it.
 */
int orc_filter(int n, const cplx* A, int lda, int ncols, cplx* V, int ldv, const int* deg,
               double c, double e, double lambda1) {
  if (n <= 0 || ncols <= 0) return 0;
  for (int a = 0; a + 1 < ncols; ++a)
    if (deg[a] > deg[a + 1] || deg[a] < 0) return -7;
  int mmax = deg[ncols - 1];
  if (mmax == 0) return 0;
  cplx* prev = calloc((size_t)n * ncols, sizeof(cplx)); /* V_{i-2} */
  cplx* cur = calloc((size_t)n * ncols, sizeof(cplx));  /* V_{i-1} */
  cplx* nxt = calloc((size_t)n * ncols, sizeof(cplx));  /* V_i     */
  cplx* AV = calloc((size_t)n * ncols, sizeof(cplx));
  if (!prev || !cur || !nxt || !AV) { free(prev); free(cur); free(nxt); free(AV); return -100; }
  for (int a = 0; a < ncols; ++a)
    for (int i = 0; i < n; ++i) cur[IDX(i, a, n)] = V[IDX(i, a, ldv)];

  const double sigma1 = e / (lambda1 - c);
  double sigma = sigma1;
  /* first active column index: columns with deg < i are finished */
  int first = 0;
  while (first < ncols && deg[first] < 1) ++first;
  /* step 1 */
  orc_matmul_block(n, A, lda, ncols - first, cur + IDX(0, first, n), n, AV + IDX(0, first, n), n);
  for (int a = first; a < ncols; ++a)
    for (int i = 0; i < n; ++i)
      nxt[IDX(i, a, n)] = (sigma1 / e) * (AV[IDX(i, a, n)] - c * cur[IDX(i, a, n)]);
  for (int a = first; a < ncols; ++a)
    if (deg[a] == 1)
      for (int i = 0; i < n; ++i) V[IDX(i, a, ldv)] = nxt[IDX(i, a, n)];
  { cplx* t = prev; prev = cur; cur = nxt; nxt = t; }
  for (int step = 2; step <= mmax; ++step) {
    while (first < ncols && deg[first] < step) ++first;
    const double sigma_new = 1.0 / (2.0 / sigma1 - sigma);
    orc_matmul_block(n, A, lda, ncols - first, cur + IDX(0, first, n), n, AV + IDX(0, first, n), n);
    for (int a = first; a < ncols; ++a)
      for (int i = 0; i < n; ++i)
        nxt[IDX(i, a, n)] = (2.0 * sigma_new / e) * (AV[IDX(i, a, n)] - c * cur[IDX(i, a, n)]) -
                            (sigma * sigma_new) * prev[IDX(i, a, n)];
    for (int a = first; a < ncols; ++a)
      if (deg[a] == step)
        for (int i = 0; i < n; ++i) V[IDX(i, a, ldv)] = nxt[IDX(i, a, n)];
    sigma = sigma_new;
    { cplx* t = prev; prev = cur; cur = nxt; nxt = t; }
  }
  free(prev); free(cur); free(nxt); free(AV);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Condition-number estimate (Eq. simple-est, Eq. full-est, Definition of    */
/* the convergence ratio, Section 2.2)                                       */
/* ------------------------------------------------------------------------ */

/* |rho| = max over +- of |t +- sqrt(t^2 - 1)| with t = (x - c)/e, for x
 * outside [c-e, c+e]; inside the interval |rho| = 1 (Eq. rho). */
double orc_abs_rho(double x, double c, double e) {
  double t = fabs((x - c) / e);
  if (t <= 1.0) return 1.0;
  return t + sqrt(t * t - 1.0);
}

/*
 * Returns log(kappa_est) where
 *   kappa_est = eta |rho_{k+1}|^{m_{k+1}} |rho_1|^{m_ell - m_{k+1}}   (Eq. full-est)
 * which for k = 0 and one degree m reduces to eta |rho_1|^m (Eq. simple-est).
 * theta_k1 is the Ritz value attached to the first unlocked column, lambda1
 * the lowest eigenvalue estimate, m_k1 and m_ell the degrees of the first
 * unlocked and of the last column.  Computed in log space so that estimates
 * beyond the double range stay finite.
 */
double orc_log_cond_est(double theta_k1, int m_k1, int m_ell, double lambda1, double c, double e,
                        double eta) {
  double lr1 = log(orc_abs_rho(lambda1, c, e));
  double lrk = log(orc_abs_rho(theta_k1, c, e));
  return log(eta) + (double)m_k1 * lrk + (double)(m_ell - m_k1) * lr1;
}

/* ------------------------------------------------------------------------ */
/* QR variants (Algorithms 2 and 3)                                          */
/* ------------------------------------------------------------------------ */

/* G = X^H X (ell x ell), then G <- (G + G^H)/2 so that it is exactly Hermitian. */
static void orc_gram(int n, int l, const cplx* X, int ldx, cplx* G) {
  for (int p = 0; p < l; ++p)
    for (int q = 0; q < l; ++q) {
      cplx s = 0;
      for (int i = 0; i < n; ++i) s += conj(X[IDX(i, p, ldx)]) * X[IDX(i, q, ldx)];
      G[IDX(p, q, l)] = s;
    }
  for (int p = 0; p < l; ++p)
    for (int q = p; q < l; ++q) {
      cplx h = 0.5 * (G[IDX(p, q, l)] + conj(G[IDX(q, p, l)]));
      G[IDX(p, q, l)] = h;
      G[IDX(q, p, l)] = conj(h);
    }
}

/*
 * Cholesky factorisation G = R^H R with R upper triangular and positive
 * diagonal, written into the upper triangle of G (the strict lower triangle
 * is zeroed).  Returns 0, or j+1 if the j-th pivot is not positive/finite
 * (LAPACK's info convention).
 */
int orc_cholesky_upper(int l, cplx* G, int ldg) {
  for (int j = 0; j < l; ++j) {
    double d = creal(G[IDX(j, j, ldg)]);
    for (int i = 0; i < j; ++i) {
      cplx r = G[IDX(i, j, ldg)];
      d -= creal(r) * creal(r) + cimag(r) * cimag(r);
    }
    if (!(d > 0.0) || !isfinite(d)) return j + 1;
    double rjj = sqrt(d);
    G[IDX(j, j, ldg)] = rjj;
    for (int k = j + 1; k < l; ++k) {
      cplx s = G[IDX(j, k, ldg)];
      for (int i = 0; i < j; ++i) s -= conj(G[IDX(i, j, ldg)]) * G[IDX(i, k, ldg)];
      G[IDX(j, k, ldg)] = s / rjj;
    }
  }
  for (int j = 0; j < l; ++j)
    for (int i = j + 1; i < l; ++i) G[IDX(i, j, ldg)] = 0;
  return 0;
}

/* X <- X R^{-1} for R upper triangular: each row x of X is replaced by q with
 * q R = x, solved by forward substitution over the columns. */
void orc_right_solve_upper(int n, int l, cplx* X, int ldx, const cplx* R, int ldr) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < l; ++j) {
      cplx s = X[IDX(i, j, ldx)];
      for (int p = 0; p < j; ++p) s -= X[IDX(i, p, ldx)] * R[IDX(p, j, ldr)];
      X[IDX(i, j, ldx)] = s / R[IDX(j, j, ldr)];
    }
  }
}

/* CholeskyQR(X, cholDeg) of Algorithm 2.  Returns 0 or the Cholesky info of
 * the failing pass (X is then partially transformed). */
int orc_cholqr(int n, int l, cplx* X, int ldx, int passes) {
  cplx* G = malloc(sizeof(cplx) * (size_t)l * l);
  if (!G) return -100;
  for (int it = 0; it < passes; ++it) {
    orc_gram(n, l, X, ldx, G);
    int info = orc_cholesky_upper(l, G, l);
    if (info) { free(G); return info; }
    orc_right_solve_upper(n, l, X, ldx, G, l);
  }
  free(G);
  return 0;
}

/*
 * Shifted Cholesky step of Algorithm 3's high-condition branch:
 *   R = X^H X,  s = 11 (m n + n (n+1)) u ||X||_F^2,  R <- chol(R + sI),  X <- X R^{-1}
 * with m = rows, n = columns of X (reading: the shift scales with the Gram
 * matrix, hence the squared Frobenius norm, as in shifted CholeskyQR).
 * Returns the Cholesky info.
 */
int orc_shifted_chol_step(int n, int l, cplx* X, int ldx) {
  cplx* G = malloc(sizeof(cplx) * (size_t)l * l);
  if (!G) return -100;
  orc_gram(n, l, X, ldx, G);
  double fro2 = 0.0;
  for (int j = 0; j < l; ++j) fro2 += creal(G[IDX(j, j, l)]);
  double s = 11.0 * ((double)n * l + (double)l * (l + 1)) * ORC_U * fro2;
  for (int j = 0; j < l; ++j) G[IDX(j, j, l)] += s;
  int info = orc_cholesky_upper(l, G, l);
  if (!info) orc_right_solve_upper(n, l, X, ldx, G, l);
  free(G);
  return info;
}

/*
 * Householder QR with explicit thin Q (Golub & Van Loan, Householder QR and
 * backward accumulation).  Overwrites X (n x l, n >= l) with Q.
 * Reflector j: v = x - alpha e_1 with alpha = -exp(i arg x_0) ||x||.
 */
void orc_householder_qr(int n, int l, cplx* X, int ldx) {
  cplx* Vh = calloc((size_t)n * l, sizeof(cplx)); /* reflector vectors, unit norm */
  for (int j = 0; j < l; ++j) {
    int m = n - j;
    cplx* x = X + IDX(j, j, ldx);
    double nx = orc_nrm2(m, x);
    cplx* v = Vh + IDX(j, j, n);
    if (nx == 0.0) continue; /* zero column: identity reflector */
    cplx ph = (cabs(x[0]) == 0.0) ? 1.0 : x[0] / cabs(x[0]);
    cplx alpha = -ph * nx;
    for (int i = 0; i < m; ++i) v[i] = x[i];
    v[0] -= alpha;
    double nv = orc_nrm2(m, v);
    if (nv == 0.0) continue;
    for (int i = 0; i < m; ++i) v[i] /= nv;
    /* apply H = I - 2 v v^H to X(j:n, j:l) */
    for (int q = j; q < l; ++q) {
      cplx* col = X + IDX(j, q, ldx);
      cplx d = 0;
      for (int i = 0; i < m; ++i) d += conj(v[i]) * col[i];
      for (int i = 0; i < m; ++i) col[i] -= 2.0 * v[i] * d;
    }
  }
  /* Q = H_0 H_1 ... H_{l-1} [I; 0], accumulated backwards */
  for (int q = 0; q < l; ++q)
    for (int i = 0; i < n; ++i) X[IDX(i, q, ldx)] = (i == q) ? 1.0 : 0.0;
  for (int j = l - 1; j >= 0; --j) {
    int m = n - j;
    cplx* v = Vh + IDX(j, j, n);
    for (int q = j; q < l; ++q) {
      cplx* col = X + IDX(j, q, ldx);
      cplx d = 0;
      for (int i = 0; i < m; ++i) d += conj(v[i]) * col[i];
      for (int i = 0; i < m; ++i) col[i] -= 2.0 * v[i] * d;
    }
  }
  free(Vh);
}

/*
 * Dynamic CAQR selection of Algorithm 3.
 *   est > cond_hi (1e8): shifted Cholesky step, then CholeskyQR2; a failing
 *                        Cholesky falls back to Householder QR;
 *   est < cond_lo (20) : CholeskyQR1;
 *   otherwise          : CholeskyQR2.
 * force: 0 = choose by est, 1 = CholQR1, 2 = CholQR2, 3 = shifted, 4 = HHQR.
 * Reading where the paper is silent: a failing CholeskyQR1/2 escalates to the
 * shifted branch, whose failure falls back to Householder QR.  The input X is
 * kept so that each escalation restarts from the unfactorised block.
 * Returns the variant that produced the result (1..4).
 */
int orc_qr_dynamic(int n, int l, cplx* X, int ldx, double log_est, double cond_hi, double cond_lo,
                   int force, int* chol_fail_info) {
  int variant = force;
  if (force == 0) {
    if (log_est > log(cond_hi)) variant = 3;
    else if (log_est < log(cond_lo)) variant = 1;
    else variant = 2;
  }
  if (chol_fail_info) *chol_fail_info = 0;
  cplx* X0 = malloc(sizeof(cplx) * (size_t)n * l);
  for (int q = 0; q < l; ++q)
    for (int i = 0; i < n; ++i) X0[IDX(i, q, n)] = X[IDX(i, q, ldx)];
  for (;;) {
    int info = 0;
    if (variant == 1 || variant == 2) {
      info = orc_cholqr(n, l, X, ldx, variant);
    } else if (variant == 3) {
      info = orc_shifted_chol_step(n, l, X, ldx);
      if (!info) info = orc_cholqr(n, l, X, ldx, 2);
    } else {
      orc_householder_qr(n, l, X, ldx);
      break;
    }
    if (!info) break;
    if (chol_fail_info && !*chol_fail_info) *chol_fail_info = info;
    if (force != 0) break; /* a forced Cholesky variant reports its failure */
    for (int q = 0; q < l; ++q)
      for (int i = 0; i < n; ++i) X[IDX(i, q, ldx)] = X0[IDX(i, q, n)];
    variant = (variant < 3) ? 3 : 4;
  }
  free(X0);
  return variant;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigensolver for the Rayleigh-Ritz problem (Algorithm 1's    */
/* reduced problem).                                                         */
/* ------------------------------------------------------------------------ */

/*
 * Diagonalises the Hermitian H (l x l, overwritten) by cyclic Jacobi
 * rotations: for the pair (p, q) with g = H_pq = |g| e^{i phi}, the unitary
 *   J = [[c, s e^{i phi}], [-s e^{-i phi}, c]],  t = tan(theta),
 *   tau = (H_qq - H_pp) / (2|g|),  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
 *   c = 1/sqrt(1 + t^2),  s = t c
 * zeroes H_pq in J^H H J.  Sweeps stop when the off-diagonal Frobenius norm
 * is <= u ||H||_F.  Outputs eigenvalues ascending in w and the matching
 * eigenvectors in the columns of W.  Returns the number of sweeps, or -1 if
 * it did not converge in 100 sweeps.
 */
int orc_jacobi_eig(int l, cplx* H, int ldh, double* w, cplx* W, int ldw) {
  for (int p = 0; p < l; ++p)
    for (int q = 0; q < l; ++q) W[IDX(p, q, ldw)] = (p == q) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int q = 0; q < l; ++q)
    for (int p = 0; p < l; ++p) { double a = cabs(H[IDX(p, q, ldh)]); fro += a * a; }
  fro = sqrt(fro);
  int sweep = 0, converged = 0;
  for (sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int q = 0; q < l; ++q)
      for (int p = 0; p < l; ++p)
        if (p != q) { double a = cabs(H[IDX(p, q, ldh)]); off += a * a; }
    off = sqrt(off);
    if (off <= ORC_U * fro || off == 0.0) { converged = 1; break; }
    for (int p = 0; p < l - 1; ++p) {
      for (int q = p + 1; q < l; ++q) {
        cplx g = H[IDX(p, q, ldh)];
        double ag = cabs(g);
        if (ag == 0.0) continue;
        cplx ph = g / ag;
        double hpp = creal(H[IDX(p, p, ldh)]), hqq = creal(H[IDX(q, q, ldh)]);
        double tau = (hqq - hpp) / (2.0 * ag);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        cplx jpq = sn * ph, jqp = -sn * conj(ph);
        /* H <- H J (columns p, q) */
        for (int i = 0; i < l; ++i) {
          cplx hip = H[IDX(i, p, ldh)], hiq = H[IDX(i, q, ldh)];
          H[IDX(i, p, ldh)] = hip * cs + hiq * jqp;
          H[IDX(i, q, ldh)] = hip * jpq + hiq * cs;
        }
        /* H <- J^H H (rows p, q) */
        for (int j = 0; j < l; ++j) {
          cplx hpj = H[IDX(p, j, ldh)], hqj = H[IDX(q, j, ldh)];
          H[IDX(p, j, ldh)] = cs * hpj + conj(jqp) * hqj;
          H[IDX(q, j, ldh)] = conj(jpq) * hpj + cs * hqj;
        }
        H[IDX(p, q, ldh)] = 0;
        H[IDX(q, p, ldh)] = 0;
        H[IDX(p, p, ldh)] = creal(H[IDX(p, p, ldh)]);
        H[IDX(q, q, ldh)] = creal(H[IDX(q, q, ldh)]);
        /* W <- W J */
        for (int i = 0; i < l; ++i) {
          cplx wip = W[IDX(i, p, ldw)], wiq = W[IDX(i, q, ldw)];
          W[IDX(i, p, ldw)] = wip * cs + wiq * jqp;
          W[IDX(i, q, ldw)] = wip * jpq + wiq * cs;
        }
      }
    }
  }
  /* sort ascending (selection sort keeps it obvious) */
  for (int p = 0; p < l; ++p) w[p] = creal(H[IDX(p, p, ldh)]);
  for (int p = 0; p < l; ++p) {
    int m = p;
    for (int q = p + 1; q < l; ++q) if (w[q] < w[m]) m = q;
    if (m != p) {
      double tw = w[p]; w[p] = w[m]; w[m] = tw;
      for (int i = 0; i < l; ++i) {
        cplx tv = W[IDX(i, p, ldw)]; W[IDX(i, p, ldw)] = W[IDX(i, m, ldw)]; W[IDX(i, m, ldw)] = tv;
      }
    }
  }
  return converged ? sweep : -1;
}

/*
 * One-sided (Hestenes) Jacobi SVD: singular values of X (n x l, n >= l),
 * descending, in sv.  Used only to obtain the exact kappa_2 of a filtered
 * block (the quantity the paper computes with a parallel SVD, Section 4.3).
 * Column pairs are rotated until |x_p^H x_q| <= u sqrt(|x_p|^2 |x_q|^2).
 */
int orc_jacobi_svd(int n, int l, const cplx* X, int ldx, double* sv) {
  cplx* Y = malloc(sizeof(cplx) * (size_t)n * l);
  for (int q = 0; q < l; ++q)
    for (int i = 0; i < n; ++i) Y[IDX(i, q, n)] = X[IDX(i, q, ldx)];
  int sweep, converged = 0;
  for (sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < l - 1; ++p) {
      for (int q = p + 1; q < l; ++q) {
        double alpha = 0.0, beta = 0.0;
        cplx gamma = 0;
        for (int i = 0; i < n; ++i) {
          cplx yp = Y[IDX(i, p, n)], yq = Y[IDX(i, q, n)];
          alpha += creal(yp) * creal(yp) + cimag(yp) * cimag(yp);
          beta += creal(yq) * creal(yq) + cimag(yq) * cimag(yq);
          gamma += conj(yp) * yq;
        }
        double ag = cabs(gamma);
        if (ag == 0.0 || ag <= ORC_U * sqrt(alpha * beta)) continue;
        rotated = 1;
        /* diagonalise the 2x2 Gram [[alpha, gamma], [conj(gamma), beta]] */
        cplx ph = gamma / ag;
        double tau = (beta - alpha) / (2.0 * ag);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        cplx jpq = sn * ph, jqp = -sn * conj(ph);
        for (int i = 0; i < n; ++i) {
          cplx yp = Y[IDX(i, p, n)], yq = Y[IDX(i, q, n)];
          Y[IDX(i, p, n)] = yp * cs + yq * jqp;
          Y[IDX(i, q, n)] = yp * jpq + yq * cs;
        }
      }
    }
    if (!rotated) { converged = 1; break; }
  }
  for (int q = 0; q < l; ++q) sv[q] = orc_nrm2(n, Y + IDX(0, q, n));
  for (int p = 0; p < l; ++p) { /* descending */
    int m = p;
    for (int q = p + 1; q < l; ++q) if (sv[q] > sv[m]) m = q;
    double t = sv[p]; sv[p] = sv[m]; sv[m] = t;
  }
  free(Y);
  return converged ? sweep : -1;
}

/* ------------------------------------------------------------------------ */
/* Spectral bounds by a few Lanczos runs (Algorithm 1, "estimate lambda_1,   */
/* lambda_ell and lambda_n")                                                 */
/* ------------------------------------------------------------------------ */

/*
 * nruns Lanczos runs of m steps from the columns of V0 (n x nruns), with full
 * re-orthogonalisation against the run's basis.  Each run yields the tridiagonal
 * T = tridiag(beta, alpha, beta), its eigenvalues theta_i (Ritz values) and the
 * squared first components tau_i of its eigenvectors.  Reading of the paper's
 * one-line description:
 *   b_sup       = max over runs of (theta_max + |beta_m|)     (an upper bound of lambda_n)
 *   lambda1     = min over runs of theta_min
 *   lambda_ell  = the smallest pooled Ritz value at which the spectral-density
 *                 estimate  (n / nruns) sum_runs sum_{theta_i <= x} tau_i  reaches ell
 *                 (to within a relative 1e-10, the rounding of the sum).
 * Outputs the three numbers in out[0..2] and every run's Ritz values in ritz
 * (nruns x m, may be NULL).
 */
int orc_lanczos_bounds(int n, const cplx* A, int lda, int nruns, const cplx* V0, int ldv, int m,
                       int ell, double* out, double* ritz_out) {
  cplx* Q = malloc(sizeof(cplx) * (size_t)n * (m + 1));
  cplx* w = malloc(sizeof(cplx) * (size_t)n);
  double* alpha = malloc(sizeof(double) * m);
  double* beta = malloc(sizeof(double) * m);
  cplx* T = malloc(sizeof(cplx) * (size_t)m * m);
  cplx* S = malloc(sizeof(cplx) * (size_t)m * m);
  double* th = malloc(sizeof(double) * (size_t)nruns * m);
  double* tau = malloc(sizeof(double) * (size_t)nruns * m);
  double bsup = -1e300, l1 = 1e300;
  for (int r = 0; r < nruns; ++r) {
    const cplx* v = V0 + IDX(0, r, ldv);
    double nv = orc_nrm2(n, v);
    for (int i = 0; i < n; ++i) Q[i] = v[i] / nv;
    for (int j = 0; j < m; ++j) {
      cplx* q = Q + IDX(0, j, n);
      orc_matmul_block(n, A, lda, 1, q, n, w, n);
      cplx a = 0;
      for (int i = 0; i < n; ++i) a += conj(q[i]) * w[i];
      alpha[j] = creal(a);
      for (int i = 0; i < n; ++i) w[i] -= alpha[j] * q[i];
      if (j > 0)
        for (int i = 0; i < n; ++i) w[i] -= beta[j - 1] * Q[IDX(i, j - 1, n)];
      /* full re-orthogonalisation (classical Gram-Schmidt, once) */
      for (int p = 0; p <= j; ++p) {
        cplx d = 0;
        for (int i = 0; i < n; ++i) d += conj(Q[IDX(i, p, n)]) * w[i];
        for (int i = 0; i < n; ++i) w[i] -= d * Q[IDX(i, p, n)];
      }
      beta[j] = orc_nrm2(n, w);
      cplx* qn = Q + IDX(0, j + 1, n);
      for (int i = 0; i < n; ++i) qn[i] = (beta[j] > 0.0) ? w[i] / beta[j] : 0.0;
    }
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) T[IDX(p, q, m)] = 0;
    for (int p = 0; p < m; ++p) {
      T[IDX(p, p, m)] = alpha[p];
      if (p + 1 < m) { T[IDX(p, p + 1, m)] = beta[p]; T[IDX(p + 1, p, m)] = beta[p]; }
    }
    double* thr = th + (size_t)r * m;
    orc_jacobi_eig(m, T, m, thr, S, m);
    for (int i = 0; i < m; ++i) {
      double s0 = cabs(S[IDX(0, i, m)]);
      tau[(size_t)r * m + i] = s0 * s0;
    }
    if (thr[m - 1] + fabs(beta[m - 1]) > bsup) bsup = thr[m - 1] + fabs(beta[m - 1]);
    if (thr[0] < l1) l1 = thr[0];
    if (ritz_out)
      for (int i = 0; i < m; ++i) ritz_out[(size_t)r * m + i] = thr[i];
  }
  /* spectral-density estimate: pooled Ritz values in ascending order */
  const int tot = nruns * m;
  int* ord = malloc(sizeof(int) * tot);
  for (int i = 0; i < tot; ++i) ord[i] = i;
  for (int i = 1; i < tot; ++i) { /* insertion sort by theta, ties by index */
    int k = ord[i], j = i - 1;
    while (j >= 0 && th[ord[j]] > th[k]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = k;
  }
  /* "reaches ell" up to the rounding of the weights and of their sum: when the start
   * vectors are orthonormal and the runs span the space, every eigenvalue's weights sum
   * to exactly 1 and the estimate hits the integer ell at the last copy of lambda_ell */
  double cum = 0.0, lell = th[ord[tot - 1]];
  for (int i = 0; i < tot; ++i) {
    cum += tau[ord[i]] * (double)n / (double)nruns;
    if (cum >= (double)ell * (1.0 - 1e-10)) { lell = th[ord[i]]; break; }
  }
  if (lell < l1) lell = l1;
  out[0] = l1;
  out[1] = lell;
  out[2] = bsup;
  free(ord); free(Q); free(w); free(alpha); free(beta); free(T); free(S); free(th); free(tau);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The ChASE outer loop (Algorithm 1)                                        */
/* ------------------------------------------------------------------------ */

static void orc_swap_cols(int n, cplx* V, int ldv, int a, int b) {
  if (a == b) return;
  for (int i = 0; i < n; ++i) {
    cplx t = V[IDX(i, a, ldv)]; V[IDX(i, a, ldv)] = V[IDX(i, b, ldv)]; V[IDX(i, b, ldv)] = t;
  }
}

/*
 * Solves for the nev lowest eigenpairs of the Hermitian A (n x n).
 *
 * V (n x ell, ell = nev + nex) holds V0 on entry (the random or warm start of
 * Algorithm 1) and, on exit, the final block: columns 0..k-1 are the locked
 * eigenvectors Y in ascending eigenvalue order.  evals/resid (nev each)
 * receive Lambda and the residuals of eq. res.  A per-iteration log is written
 * to logs[0..max_iter-1] when logs != NULL.
 *
 * Steps (one outer iteration):
 *   c = (b_sup + mu_ell)/2, e = (b_sup - mu_ell)/2
 *   filter the unlocked columns with their degrees (Algorithm 4)
 *   kappa_est from Eq. full-est; QR of [Y V] by Algorithm 3; restore Y
 *   Rayleigh-Ritz on the unlocked columns: H = Q2^H A Q2, Jacobi, V = Q2 W
 *   residuals r_a = ||A v_a - theta_a v_a|| / ||v_a|| (eq. res)
 *   lock the contiguous prefix of converged pairs among the first nev
 *   mu_1 <- min(mu_1, theta_min), mu_ell <- largest Ritz value of the block
 *   with degree optimisation: m_a = clamp(ceil(ln(r_a/tol)/ln|rho_a|)),
 *   columns re-sorted by ascending degree.
 * Returns 0 on convergence, 1 if max_iter was reached.
 */
int orc_solve(int n, const cplx* A, int lda, int nev, int nex, cplx* V, int ldv,
              const orc_params* prm, double* evals, double* resid, orc_iter_log* logs,
              orc_summary* sum) {
  const int l = nev + nex;
  int k = 0; /* locked columns */
  double mu1 = prm->lambda1, mu_ell = prm->lambda_ell, bsup = prm->b_sup;
  int* deg = malloc(sizeof(int) * l);
  double* ritz = malloc(sizeof(double) * l);
  double* res = malloc(sizeof(double) * l);
  cplx* Yk = malloc(sizeof(cplx) * (size_t)n * l);
  cplx* AQ = malloc(sizeof(cplx) * (size_t)n * l);
  cplx* H = malloc(sizeof(cplx) * (size_t)l * l);
  cplx* W = malloc(sizeof(cplx) * (size_t)l * l);
  cplx* T = malloc(sizeof(cplx) * (size_t)n * l);
  double* w = malloc(sizeof(double) * l);
  long long matvecs = 0;
  int status = 1, it;
  int counts[5] = {0, 0, 0, 0, 0};

  for (int a = 0; a < l; ++a) { deg[a] = prm->deg_init; ritz[a] = mu1; res[a] = 1.0; }

  /* step 0: orthonormalise V0 (CholeskyQR2, Householder on failure) */
  {
    int fi = 0;
    int v0 = orc_qr_dynamic(n, l, V, ldv, log(100.0), prm->cond_hi, prm->cond_lo,
                            prm->qr_force == 4 ? 4 : 0, &fi);
    (void)v0;
  }

  for (it = 0; it < prm->max_iter; ++it) {
    const double c = 0.5 * (bsup + mu_ell), e = 0.5 * (bsup - mu_ell);
    const int nu = l - k;
    /* filter the unlocked columns */
    orc_filter(n, A, lda, nu, V + IDX(0, k, ldv), ldv, deg + k, c, e, mu1);
    for (int a = k; a < l; ++a) matvecs += deg[a];
    /* condition estimate (Eq. full-est); at the first iteration every column
     * still carries mu1 as its Ritz value, which gives Eq. simple-est */
    double theta_k1 = (it == 0) ? mu1 : ritz[k];
    double lest_paper = orc_log_cond_est(theta_k1, deg[k], deg[l - 1], mu1, c, e, prm->eta);
    /* the locked block Y contributes unit singular values: with filter gains <= 1 the
     * largest singular value of [Y V] is 1, and the smallest is bounded below by the gain
     * |rho_1|^{-m_ell} of the last column; the locked-aware form takes that bound too */
    double lest_locked = log(prm->eta) + (double)deg[l - 1] * log(orc_abs_rho(mu1, c, e));
    if (lest_locked < lest_paper) lest_locked = lest_paper;
    double lest = (prm->cond_est_mode == 1) ? lest_locked : lest_paper;
    double lkap = 0.0;
    if (prm->log_exact_kappa) {
      double* sv = malloc(sizeof(double) * l);
      orc_jacobi_svd(n, l, V, ldv, sv);
      lkap = log(sv[0] / sv[l - 1]);
      free(sv);
    }
    /* QR of [Y V] */
    for (int q = 0; q < k; ++q)
      for (int i = 0; i < n; ++i) Yk[IDX(i, q, n)] = V[IDX(i, q, ldv)];
    int fi = 0;
    int variant = orc_qr_dynamic(n, l, V, ldv, lest, prm->cond_hi, prm->cond_lo, prm->qr_force, &fi);
    counts[variant] += 1;
    for (int q = 0; q < k; ++q)
      for (int i = 0; i < n; ++i) V[IDX(i, q, ldv)] = Yk[IDX(i, q, n)];
    /* Rayleigh-Ritz on the unlocked columns */
    cplx* Q2 = V + IDX(0, k, ldv);
    orc_matmul_block(n, A, lda, nu, Q2, ldv, AQ, n);
    for (int p = 0; p < nu; ++p)
      for (int q = 0; q < nu; ++q) {
        cplx s = 0;
        for (int i = 0; i < n; ++i) s += conj(Q2[IDX(i, p, ldv)]) * AQ[IDX(i, q, n)];
        H[IDX(p, q, nu)] = s;
      }
    for (int p = 0; p < nu; ++p)
      for (int q = p; q < nu; ++q) {
        cplx h = 0.5 * (H[IDX(p, q, nu)] + conj(H[IDX(q, p, nu)]));
        H[IDX(p, q, nu)] = h;
        H[IDX(q, p, nu)] = conj(h);
      }
    orc_jacobi_eig(nu, H, nu, w, W, nu);
    /* V <- Q2 W */
    for (int q = 0; q < nu; ++q)
      for (int i = 0; i < n; ++i) {
        cplx s = 0;
        for (int p = 0; p < nu; ++p) s += Q2[IDX(i, p, ldv)] * W[IDX(p, q, nu)];
        T[IDX(i, q, n)] = s;
      }
    for (int q = 0; q < nu; ++q)
      for (int i = 0; i < n; ++i) Q2[IDX(i, q, ldv)] = T[IDX(i, q, n)];
    for (int a = 0; a < nu; ++a) ritz[k + a] = w[a];
    /* residuals (eq. res) with an explicit product A v_a */
    orc_matmul_block(n, A, lda, nu, Q2, ldv, AQ, n);
    for (int a = 0; a < nu; ++a) {
      for (int i = 0; i < n; ++i) T[i] = AQ[IDX(i, a, n)] - w[a] * Q2[IDX(i, a, ldv)];
      res[k + a] = orc_nrm2(n, T) / orc_nrm2(n, Q2 + IDX(0, a, ldv));
    }
    /* lock the contiguous converged prefix among the first nev */
    int knew = k;
    while (knew < nev && res[knew] < prm->tol) ++knew;
    if (logs) {
      orc_iter_log* g = &logs[it];
      g->iteration = it + 1; g->locked_before = k; g->locked_after = knew;
      g->log_cond_est = lest; g->variant = variant; g->chol_fail_info = fi;
      g->matvecs = matvecs; g->c = c; g->e = e; g->mu1 = mu1; g->mu_ell = mu_ell;
      g->log_cond_est_paper = lest_paper; g->log_cond_est_locked = lest_locked;
      g->log_kappa_exact = lkap;
      g->deg_min = deg[k]; g->deg_max = deg[l - 1];
    }
    /* spectral bounds for the next filter */
    for (int a = k; a < l; ++a) if (ritz[a] < mu1) mu1 = ritz[a];
    mu_ell = ritz[l - 1];
    for (int a = k; a < l; ++a) if (ritz[a] > mu_ell) mu_ell = ritz[a];
    k = knew;
    if (k >= nev) { status = 0; ++it; break; }
    /* degrees for the unlocked columns */
    if (prm->opt_degree) {
      const double c2 = 0.5 * (bsup + mu_ell), e2 = 0.5 * (bsup - mu_ell);
      for (int a = k; a < l; ++a) {
        double lr = log(orc_abs_rho(ritz[a], c2, e2));
        int m;
        if (lr <= 0.0 || !(res[a] > prm->tol)) m = (lr <= 0.0) ? prm->deg_max : prm->deg_min;
        else {
          double mm = ceil(log(res[a] / prm->tol) / lr);
          m = (mm > prm->deg_max) ? prm->deg_max : (int)mm;
        }
        if (m < prm->deg_min) m = prm->deg_min;
        if (m > prm->deg_max) m = prm->deg_max;
        deg[a] = m;
      }
      /* stable sort of the unlocked columns by ascending degree */
      for (int a = k + 1; a < l; ++a) {
        int b = a;
        while (b > k && deg[b - 1] > deg[b]) {
          int td = deg[b]; deg[b] = deg[b - 1]; deg[b - 1] = td;
          double tr = ritz[b]; ritz[b] = ritz[b - 1]; ritz[b - 1] = tr;
          double ts = res[b]; res[b] = res[b - 1]; res[b - 1] = ts;
          orc_swap_cols(n, V, ldv, b, b - 1);
          --b;
        }
      }
    } else {
      for (int a = k; a < l; ++a) deg[a] = prm->deg_init;
    }
  }
  /* locked pairs in ascending order of eigenvalue */
  int kout = k < nev ? k : nev;
  for (int p = 0; p < kout; ++p) {
    int m = p;
    for (int q = p + 1; q < kout; ++q) if (ritz[q] < ritz[m]) m = q;
    if (m != p) {
      double t = ritz[p]; ritz[p] = ritz[m]; ritz[m] = t;
      t = res[p]; res[p] = res[m]; res[m] = t;
      orc_swap_cols(n, V, ldv, p, m);
    }
  }
  for (int a = 0; a < nev; ++a) {
    evals[a] = ritz[a];
    resid[a] = res[a];
  }
  if (sum) {
    sum->iterations = it; sum->locked = k; sum->matvecs = matvecs;
    sum->n_chol1 = counts[1]; sum->n_chol2 = counts[2]; sum->n_shifted = counts[3];
    sum->n_hhqr = counts[4];
  }
  free(deg); free(ritz); free(res); free(Yk); free(AQ); free(H); free(W); free(T); free(w);
  return status;
}
