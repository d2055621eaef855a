/*
 * lisa_sampler.h -- C ABI of the sampler's proposal and accept steps for the
 * batched likelihood of lisa_td.h (arXiv:2501.08261, Sec. II.C, Fisher
 * initialization: starting points drawn from a Gaussian with mean at the
 * injection and covariance equal to the inverse Fisher matrix, the Fisher
 * matrix built from finite differences of the likelihood; the sampler accepts
 * or rejects every proposal by the exact likelihood).
 *
 * Conventions are those of lisa_td.h: extern "C", int status (LISA_TD_OK or a
 * negative LISA_TD_E* code, message in lisa_td_last_error()), *_dev device
 * pointers, *_host host pointers read during the call only, stream = a
 * cudaStream_t as void* on which the work is enqueued (no host sync).
 * Parameter vectors are FP64 [15] in the order of lisa_td.h.  The D sampled
 * parameters (1 <= D <= 15, distinct, each in 0..14) are given by idx_host[D];
 * the other entries stay at their mean.
 */
#ifndef LISA_SAMPLER_H
#define LISA_SAMPLER_H

#include <stdint.h>

#include "lisa_td.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LISA_NPARAM 15

/* Number of finite-difference stencil points for D sampled parameters:
 * 1 + 2 D + 2 D (D - 1)  (451 for D = 15). */
int lisa_fisher_npoints(int32_t D);

/* Stencil of the Fisher matrix F = -d^2 logL / dtheta_a dtheta_b at theta0
 * (Sec. II.C; central second differences): points_dev [P][15] in the order
 * theta0; for each a: theta0 + eps_a e_a, theta0 - eps_a e_a; for each pair
 * a < b (lexicographic): (+a +b), (+a -b), (-a +b), (-a -b).  theta0_dev
 * [15]; eps_host [D] > 0 step sizes in the units of each parameter.  The
 * caller evaluates logL at the points (lisa_td_loglike_batch). */
int lisa_fisher_points(const double* theta0_dev, const int32_t* idx_host,
                       const double* eps_host, int32_t D, double* points_dev, void* stream);

/* F [D][D] (row-major, symmetric) from logl_dev [P] at the stencil points:
 *   F_aa = -(L(+a) - 2 L(0) + L(-a)) / eps_a^2,
 *   F_ab = -(L(++) - L(+-) - L(-+) + L(--)) / (4 eps_a eps_b). */
int lisa_fisher_assemble(const double* logl_dev, const double* eps_host, int32_t D,
                         double* fisher_dev, void* stream);

/* Cholesky factor: lower-triangular l_dev [D][D] with
 * L L^T = a_dev [D][D] + diag(diag_host) (FP64, upper triangle of l set to 0).
 * diag_host [D] >= 0 or NULL; the sampler passes the precision 12 / w^2 of
 * each uniform prior of width w, so that directions the data leave
 * unconstrained take the prior's width.  info_dev [1]: 0, or j + 1 if the
 * leading (j+1) x (j+1) block is not positive definite (L then partial). */
int lisa_cholesky(const double* a_dev, const double* diag_host, int32_t D, double* l_dev,
                  int32_t* info_dev, void* stream);

/* Gaussian proposal q = N(mu, F^-1) with F = L L^T: for each of W walkers,
 * x = mu + L^-T z on the sampled parameters (others = mu), and
 * log q(x) = -|z|^2/2 + sum_i log L_ii - (D/2) log 2 pi.
 * mu_dev [15], l_dev [D][D] lower, z_dev [W][D] standard normal draws (the
 * caller's random numbers), x_dev [W][15], logq_dev [W]. */
int lisa_gauss_draw(const double* mu_dev, const double* l_dev, const int32_t* idx_host,
                    int32_t D, const double* z_dev, int32_t W, double* x_dev, double* logq_dev,
                    void* stream);

/* Random-walk proposal with the Fisher covariance: x' = x + step L^-T z for
 * each walker (x_dev, x_prop_dev [W][15], z_dev [W][D]); symmetric, so the
 * accept step takes log q = 0 for both positions. */
int lisa_gauss_walk(const double* x_dev, const double* l_dev, const int32_t* idx_host, int32_t D,
                    const double* z_dev, int32_t W, double step, double* x_prop_dev, void* stream);

/* log q(x) of the same Gaussian at given positions x_dev [W][15]. */
int lisa_gauss_logq(const double* mu_dev, const double* l_dev, const int32_t* idx_host,
                    int32_t D, const double* x_dev, int32_t W, double* logq_dev, void* stream);

/* One Metropolis-Hastings decision per walker for an independence proposal
 * with target pi^beta (tempered chains; beta = 1 is the posterior): accept x'
 * when log u < [beta logL(x') - log q(x')] - [beta logL(x) - log q(x)] and
 * lo <= x' <= hi componentwise (uniform prior box; Table I's prior ranges) and
 * logL(x') > -inf.  On acceptance x, logL, log q of the walker are replaced
 * in place.  x_prop_dev [W][15], logl_prop_dev [W], logq_prop_dev [W],
 * u_dev [W] uniform in (0, 1] (the caller's random numbers), beta_dev [W]
 * inverse temperatures or NULL (all 1), lo_host / hi_host [15]; x_dev
 * [W][15], logl_dev [W], logq_dev [W] in/out; accepted_dev [W] int32 0/1
 * (may be NULL).  For a symmetric proposal pass log q = 0 for both. */
int lisa_mh_accept(int32_t W, const double* x_prop_dev, const double* logl_prop_dev,
                   const double* logq_prop_dev, const double* u_dev, const double* beta_dev,
                   const double* lo_host, const double* hi_host, double* x_dev, double* logl_dev,
                   double* logq_dev, int32_t* accepted_dev, void* stream);

/* Parallel tempering (the sampler of Sec. II.C is ptemcee): replica exchange
 * between adjacent temperatures for walkers stored temperature-major,
 * x_dev [T][W][15], logl_dev / logq_dev [T][W].  betas_host [T] in (0, 1],
 * decreasing with the index (betas[0] = 1, the posterior).  For k = T-2 down
 * to 0 the states (x, logL, log q) of (k, w) and (k+1, w) are exchanged when
 * log u[k][w] < (beta_k - beta_{k+1}) (logL_{k+1,w} - logL_{k,w});
 * u_dev [T-1][W] uniform in (0, 1]; swapped_dev [T-1][W] int32 0/1 (may be
 * NULL).  2 <= T <= 15. */
int lisa_pt_swap(int32_t T, int32_t W, const double* betas_host, const double* u_dev,
                 double* x_dev, double* logl_dev, double* logq_dev, int32_t* swapped_dev,
                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LISA_SAMPLER_H */
