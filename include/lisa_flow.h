/*
 * lisa_flow.h -- C ABI of the learned proposal: an affine-coupling
 * normalising flow (RealNVP form) over the D sampled parameters, whose matrix
 * products run on the tensor cores (bf16 operands, fp32 accumulation).
 *
 * Role in the method (arXiv:2501.08261, Sec. II.C): the sampler is started
 * from, and its proposals are judged against, the Fisher-Gaussian
 * N(theta_inj, F^-1); the flow is trained on chain samples of that sampler
 * and then used as the independence proposal of lisa_mh_accept, every
 * proposal still accepted or rejected by the exact likelihood.
 *
 * Model.  Frame u = (x[idx] - mu[idx]) / scale.  Layer l (l = 0..L-1) splits
 * its input by perm_l: a = perm_l[0 .. d_a), b = perm_l[d_a .. D), with
 * d_a = ceil(D/2) for even l and floor(D/2) for odd l;
 *   h1 = tanh(W1 u_a + b1), h2 = tanh(W2 h1 + b2), (s_raw, t) = W3 h2 + b3,
 *   s = tanh(s_raw),  y_a = u_a,  y_b = u_b * exp(s) + t.
 * log q(x) = sum_i (-z_i^2 / 2 - log(2 pi) / 2) + sum_l sum s_l - sum log scale.
 * Parameters (FP32, packed per layer in the order W1 [H][d_a], b1 [H],
 * W2 [H][H], b2 [H], W3 [2 d_b][H] (s rows, then t rows), b3 [2 d_b]).
 * H = 128, 1 <= D <= 15, 1 <= L <= 16.
 *
 * Conventions as in lisa_td.h (int status, lisa_td_last_error(), *_dev
 * device pointers, *_host host pointers read during the call, stream-ordered
 * work, no host synchronisation after flow_create).  A wait of a flow kernel
 * on its tensor-core work is bounded; if it gives up, the next call on the
 * context returns LISA_TD_ETIMEOUT.
 */
#ifndef LISA_FLOW_H
#define LISA_FLOW_H

#include <stdint.h>

#include "lisa_td.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flow_ctx flow_ctx;   /* opaque */

/* idx_host [dim]: parameter indices (0..14, distinct) of the flow's
 * coordinates; perm_host [layers][dim]: permutation of 0..dim-1 per layer;
 * max_batch: largest W / batch of later calls.  Parameters start at zero
 * (the identity map); frame mu = 0, scale = 1. */
int flow_create(flow_ctx** out, int32_t dim, int32_t layers, int32_t hidden, int32_t max_batch,
                const int32_t* idx_host, const int32_t* perm_host, void* stream);

int flow_nparams(const flow_ctx* f, int64_t* n);

/* Limit of every wait of the flow kernels on their tensor-core work, in
 * polls of the mbarrier (failure-path testing; no paper counterpart).
 * polls < 0 restores the default (2^22 polls, far beyond any product's
 * duration); 0 makes the first wait of each CTA give up at once.  A wait that
 * gives up marks the context, the CTA stops issuing products, waits (with the
 * default limit) for the product already in flight, frees its tensor memory
 * and ends; the next call on the context returns LISA_TD_ETIMEOUT and clears
 * the mark.  LISA_TD_ERANGE above the default. */
int flow_set_wait_limit(flow_ctx* f, int64_t polls);

/* Copy packed FP32 parameters in / out (device pointers, [nparams]).
 * flow_set_params also resets the Adam moments and step count. */
int flow_set_params(flow_ctx* f, const float* params_dev, void* stream);
int flow_get_params(const flow_ctx* f, float* params_dev, void* stream);

/* Frame: mu_dev [15] (FP64), scale_dev [dim] (FP64, > 0). */
int flow_set_frame(flow_ctx* f, const double* mu_dev, const double* scale_dev, void* stream);

/* log q(x) for W positions x_dev [W][15] -> logq_dev [W] (FP64 out). */
int flow_logprob(flow_ctx* f, const double* x_dev, int32_t W, double* logq_dev, void* stream);

/* Proposals from standard-normal draws z_dev [W][dim] (the caller's random
 * numbers): x_dev [W][15] (entries outside idx = mu) and log q(x) [W]. */
int flow_propose(flow_ctx* f, const double* z_dev, int32_t W, double* x_dev, double* logq_dev,
                 void* stream);

/* Loss -mean_w log q(x_w) over a batch x_dev [B][15] and its gradient with
 * respect to the packed parameters: loss_dev [1] (FP32), grad_dev [nparams]
 * (FP32).  Either output may be NULL.  B <= min(max_batch, 8192). */
int flow_grad(flow_ctx* f, const double* x_dev, int32_t B, float* loss_dev, float* grad_dev,
              void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step
 * count kept by the context) with the gradient grad_dev [nparams]. */
int flow_adam(flow_ctx* f, const float* grad_dev, float lr, void* stream);

/* Training: `epochs` passes over samples_dev [S][15] in batches of `batch`
 * (a batch that does not divide S drops the remainder), each batch one
 * flow_grad + flow_adam.  Epoch e visits sample (a_e i + c_e) mod S at
 * position i, a_e coprime to S (a fixed, stateless shuffle).
 * loss_dev [epochs]: mean batch loss of each epoch (may be NULL). */
int flow_train(flow_ctx* f, const double* samples_dev, int64_t S, int32_t epochs, int32_t batch,
               float lr, float* loss_dev, void* stream);

void flow_destroy(flow_ctx* f);

#ifdef __cplusplus
}
#endif
#endif /* LISA_FLOW_H */
