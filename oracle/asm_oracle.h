/*
 * asm_oracle.h -- plain, slow FP64 CPU oracle of the average spectrum method
 * with blocked modes sampling (Ghanem & Koch, arXiv:1912.01379).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call this code.
 * It shares no source, header, table or helper with the CUDA library under
 * paper_1912_01379_gb300/csrc, and it does not include or link that library.
 *
 * Every function states the passage of the paper it follows.  Where the paper
 * is silent the reading is stated next to the code.
 */
#ifndef ASM_ORACLE_H
#define ASM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): out = bijection(ctr; key). */
void ora_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Standard normal helpers (FP64).  Phi = CDF, Q = 1 - Phi. */
double ora_norm_cdf(double z);
double ora_norm_quantile(double p);            /* Phi^{-1}(p), 0 < p < 1 */
double ora_erfcx(double x);                    /* exp(x^2) erfc(x) */
double ora_log_q(double x);                    /* log Q(x) for x >= 0 */

/* One draw of N(mu, sigma^2) truncated to [lo, hi] by the inverse CDF at u. */
double ora_truncnorm(double mu, double sigma, double lo, double hi, double u);

/* n draws of N(0,1) restricted to [a, b] by Robert's rejection sampler
 * (Statistics and Computing 5 (1995) 121), with uniforms from Philox4x64-10
 * keyed by (seed, stream).  Independent of ora_truncnorm: a distributional
 * cross-check.  Returns the number of proposals made. */
long ora_truncnorm_robert(double a, double b, uint64_t seed, uint64_t stream, int n, double *out);

/* Cholesky C = L L^T of an n x n SPD matrix (row-major). 0 on success. */
int ora_cholesky(int n, const double *C, double *L);

/* One-sided Jacobi SVD of the m x n row-major matrix A: A V = U diag(s),
 * V n x n orthogonal, s sorted descending, sign convention applied.
 * U is m x n row-major (column j = U_j, zero where s_j = 0).
 * Returns the number of sweeps (> 0) or a negative value on failure. */
int ora_jacobi_svd(int m, int n, const double *A, double *s, double *U, double *V);

typedef struct ora_problem ora_problem;

/* Whitening and per-block SVDs (Sec. IV, Eq. chi2 and its whitened form;
 * Sec. IV.B modes; Sec. IV.C blocks).  Levels are lists of contiguous blocks:
 * level l has level_nblocks[l] blocks whose starts are the next entries of
 * block_start (each level starts at 0; a block ends where the next begins,
 * the last one at N).  *err receives 0 or a negative code:
 *  -1 shape, -2 covariance not SPD, -3 non-finite input, -4 improper zero mode
 *  (a flat direction along which f >= 0 does not bound the move). */
ora_problem *ora_setup(int M, int N, const double *K, const double *G, const double *C,
                       int n_levels, const int *level_nblocks, const int *block_start,
                       int *err);
/* Same with the exponent of reading R2 (zero modes) given: sign-changing modes
 * with d <= d_1 max(M, n) 2^-flat_exp are sampled flat (ora_setup: 40; 52
 * leaves only the numerically zero modes flat).  1 <= flat_exp <= 52. */
ora_problem *ora_setup_ex(int M, int N, const double *K, const double *G, const double *C,
                          int n_levels, const int *level_nblocks, const int *block_start, int flat_exp,
                          int *err);
void ora_free(ora_problem *p);

/* Rounding-sensitivity probe (tests only): with unit_exp = e in 1..60 (0: off),
 * every move's inputs are moved by one rounding at unit roundoff 2^-e (e = 52:
 * FP64 rounding, e = 24: FP32 rounding), each up or down by bits 3k+1..3k+3
 * of the move's Philox word (k = pattern, 0..15), before the draw: the conditional mean mu = h_j/d_j - e_j
 * of a Gaussian move (Sec. IV.B) by 2^-e (sum_m |U_jm| (|g~_m| + sum_n |K~_mn
 * f_n|) / d_j + sum_i |V_ji f_i|), the size of the terms it is summed from, and
 * each finite end of the interval [lo, hi] by 2^-e of its size.  Two correct
 * implementations of the sampler at that precision (e.g. one tracking the
 * residual incrementally, one recomputing the block's data from scratch)
 * differ at least by such roundings, so the probe's divergence from the plain
 * run measures how far a step-by-step comparison can be held. */
void ora_set_jitter(ora_problem *p, int unit_exp, int pattern);

/* Sizes of the exported factors: total entries of d, V and U over all blocks. */
void ora_sizes(const ora_problem *p, long *n_d, long *n_V, long *n_U);

/* Export K~ (M x N row-major), g~ (M) and, block after block in level order:
 * d (n_b), V mode-major (n_b x n_b, V[j*n_b + i] = component i of mode j),
 * U mode-major (min(M, n_b) x M, U[j*M + m]). */
void ora_export(const ora_problem *p, double *Kt, double *gt, double *d, double *V, double *U);

/* Starting vector f0_n = s* with s* the best non-negative scale of the flat
 * model (Sec. IV.E, a one-parameter stand-in for the NNLS start). */
void ora_initial_f(const ora_problem *p, double *f0);

/* Conditional of mode j of block b of level l at state f (N values):
 * delta = e_j' - e_j ~ N(mu, sigma^2) restricted to [lo, hi];
 * sigma = 0 marks a zero mode (flat on [lo, hi]). */
int ora_conditional(const ora_problem *p, int level, int block, int j, const double *f,
                    double *mu, double *sigma, double *lo, double *hi);

/* chi^2(f) = || g~ - K~ f ||^2. */
double ora_chi2(const ora_problem *p, const double *f);

/* Run `chains` independent chains for burn_in + sweeps sweeps from f0.
 * Outputs (may be NULL): f_final (chains x N), S1 and S2 (chains x N, sums of
 * f and f^2 over the kept sweeps), chi2_final (chains), trace (first
 * n_traced chains, f after every sweep: n_traced x (burn_in+sweeps) x N),
 * stats[4] = {positivity violations, degenerate intervals, zero-mode moves,
 * tail solver iterations at the cap}.  n_threads <= 0 uses the default. */
int ora_run(const ora_problem *p, int chains, long burn_in, long sweeps, uint64_t seed,
            uint64_t problem_id, int n_threads, double *f_final, double *S1, double *S2,
            double *chi2_final, double *trace, int n_traced, long *stats);

/* Same, starting from the given per-chain states f_start (chains x N) at sweep
 * index sweep0 (used to split a run into pieces). */
int ora_run_from(const ora_problem *p, int chains, const double *f_start, long sweep0,
                 long burn_in, long sweeps, uint64_t seed, uint64_t problem_id, int n_threads,
                 double *f_final, double *S1, double *S2, double *chi2_final,
                 double *trace, int n_traced, long *stats);

/* Same, with the global id of local chain 0 (chain q uses id chain0 + q in
 * its random-number counters): shards of a run reproduce the whole run. */
int ora_run_ids(const ora_problem *p, int chains, const double *f_start, long sweep0,
                long burn_in, long sweeps, uint64_t seed, uint64_t problem_id, uint64_t chain0,
                int n_threads, double *f_final, double *S1, double *S2, double *chi2_final,
                double *trace, int n_traced, long *stats);

#ifdef __cplusplus
}
#endif
#endif
