/*
 * chase_oracle.h -- declarations of the plain FP64 CPU oracle.
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of the benchmark, never by the GPU library.
 */
#ifndef CHASE_ORACLE_H
#define CHASE_ORACLE_H

#include <complex.h>

typedef struct {
  double tol;          /* residual threshold of eq. res */
  int max_iter;        /* outer iterations of Algorithm 1 */
  int deg_init;        /* degree of every column in the first filter */
  int deg_min, deg_max;
  int opt_degree;      /* 0: every column keeps deg_init */
  double eta;          /* constant of Proposition th:2-2 (1 by the paper's remark) */
  double cond_hi;      /* Algorithm 3 threshold for shifted CholeskyQR2 (1e8) */
  double cond_lo;      /* Algorithm 3 threshold for CholeskyQR1 (20) */
  int qr_force;        /* 0 auto, 1 CholQR1, 2 CholQR2, 3 shifted, 4 Householder */
  double lambda1;      /* estimate of the lowest eigenvalue */
  double lambda_ell;   /* estimate of the ell-th eigenvalue (lower edge of the damped interval) */
  double b_sup;        /* upper bound of the spectrum (must be >= lambda_n) */
  int cond_est_mode;   /* 0: Eq. full-est as printed; 1: max(Eq. full-est, eta |rho_1|^{m_ell}) */
  int log_exact_kappa; /* 1: log kappa_2 of [Y V] before each QR (one-sided Jacobi SVD) */
} orc_params;

typedef struct {
  int iteration, locked_before, locked_after, variant, chol_fail_info, deg_min, deg_max;
  long long matvecs;
  double log_cond_est, c, e, mu1, mu_ell;
  double log_cond_est_paper, log_cond_est_locked; /* both forms, whichever drove the choice */
  double log_kappa_exact;  /* ln kappa_2([Y V]) when requested, else 0 */
} orc_iter_log;

typedef struct {
  int iterations, locked, n_chol1, n_chol2, n_shifted, n_hhqr;
  long long matvecs;
} orc_summary;

int orc_filter(int n, const double complex* A, int lda, int ncols, double complex* V, int ldv,
               const int* deg, double c, double e, double lambda1);
double orc_abs_rho(double x, double c, double e);
double orc_log_cond_est(double theta_k1, int m_k1, int m_ell, double lambda1, double c, double e,
                        double eta);
int orc_cholesky_upper(int l, double complex* G, int ldg);
void orc_right_solve_upper(int n, int l, double complex* X, int ldx, const double complex* R,
                           int ldr);
int orc_cholqr(int n, int l, double complex* X, int ldx, int passes);
int orc_shifted_chol_step(int n, int l, double complex* X, int ldx);
void orc_householder_qr(int n, int l, double complex* X, int ldx);
int orc_qr_dynamic(int n, int l, double complex* X, int ldx, double log_est, double cond_hi,
                   double cond_lo, int force, int* chol_fail_info);
int orc_jacobi_eig(int l, double complex* H, int ldh, double* w, double complex* W, int ldw);
int orc_jacobi_svd(int n, int l, const double complex* X, int ldx, double* sv);
int orc_lanczos_bounds(int n, const double complex* A, int lda, int nruns, const double complex* V0,
                       int ldv, int m, int ell, double* out, double* ritz_out);
int orc_solve(int n, const double complex* A, int lda, int nev, int nex, double complex* V, int ldv,
              const orc_params* prm, double* evals, double* resid, orc_iter_log* logs,
              orc_summary* sum);

#endif
