/*
 * qrs_proposal.h -- learned frequency-sampling proposal of libqrs.
 *
 * The paper samples frequencies by a fixed heuristic and notes (Sec. 5) that
 * a mapping that takes the properties of the PSD into account may be
 * possible.  This is such a mapping: a small MLP maps a differential-piston
 * geometry g = (r0, L0, D, Bx, By) -- Fried parameter, outer scale, aperture
 * diameter, baseline vector -- to a density over the n_rho x n_theta
 * log-polar cells of [fmin, fmax]; mixed with the uniform cell density and
 * quantised to a two-level integer CDF it drives the IMPORTANCE sampler of
 * qrs.h, whose weights w = W J / N_f with J = 2 pi ln(fmax/fmin) rho^2 /
 * (C p_c) keep Eq. 3 unbiased.  It is trained
 * on what the plain method itself produces: per-cell contributions of plain
 * log-polar R2 draws to the differential-piston structure function of the
 * geometry (Sec. 4.4 with the Eq. 7 filter),
 *     V_c = sum_{draws} sum_{k in c} w_k A(|f_k|)^2 2 (1 - cos 2 pi f_k . B),
 * normalised to a target distribution t_c = V_c / sum V.
 *
 * Network (FP32): features x = ((ln r0 - ln 0.12)/0.6, (ln L0 - ln 30)/0.8,
 * (ln D - ln 3)/0.6, (ln|B| - ln 15)/1.5, Bx/|B|, By/|B|); h1 = relu(x W1 + b1),
 * h2 = relu(h1 W2 + b2), z = h2 W3 + b3 + prior (logits; the prior of
 * qrs_proposal_prior, or none); widths 6 -> 128 -> 128 -> C,
 * C = n_rho n_theta (2048 for 64 x 32).  Loss: mean over samples of the cross
 * entropy -sum_c t_c log softmax(z)_c.  Optimiser: Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected).
 * Parameter vector (FP32, this order, row-major, "in x out"):
 *     W1[6][128] b1[128] W2[128][128] b2[128] W3[128][C] b3[C]
 * qrs_mlp_param_count(C) gives its length (281,600 for C = 2048).
 *
 * Conventions as in qrs.h: device pointers, caller-owned, enqueued on `stream`.
 * Cell counts: 1 <= C = n_rho n_theta <= 32768 in every call (formed in 64
 * bits; QRS_ERR_ARG otherwise, nothing launched).
 */
#ifndef QRS_PROPOSAL_H
#define QRS_PROPOSAL_H

#include <stdint.h>

#include "qrs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of FP32 parameters of the network with C output cells. */
int64_t qrs_mlp_param_count(int32_t n_cells);

/* He-normal initialisation (weights N(0, 2/fan_in) from Philox4x32-10 of `seed`
 * by Box-Muller, biases 0) of params [qrs_mlp_param_count(n_cells)]; the
 * output layer's weights W3 are multiplied by out_scale (1: He; small values
 * start the logits at the prior when one is used).  out_scale >= 0. */
qrs_status qrs_mlp_init(qrs_handle* h, int32_t n_cells, uint64_t seed, float out_scale, float* params, void* stream);

/* Training targets from plain draws: for each geometry geom[i] = (r0, L0, D,
 * Bx, By) (device FP64 [n][5]), the per-cell structure-function contributions
 * v_k = w_k A(|f_k|)^2 2 (1 - cos 2 pi f_k . B) of n_draws plain realisations
 * (LOGPOLAR [dom.fmin, dom.fmax], R2, n_f terms, stream seed `seed`, cells
 * n_rho x n_theta; the PSD kind of `psd`, its r0/L0 replaced by the
 * geometry's), reduced per cell and normalised to sum 1:
 *   QRS_TARGET_MEAN  t_c ~ sum_{k in c} v_k         (the cell's share of D(B))
 *   QRS_TARGET_RMS   t_c ~ sqrt(sum_{k in c} v_k^2) (the variance-optimal cell
 *                    probability of the importance estimator when v varies
 *                    inside cells: minimises sum_c (1/p_c) int_c g^2 rho^2)
 *   targets [n][n_rho n_theta] FP32.   workspace: n_draws n_f draw records. */
/* fold selects the cells the contributions are binned into:
 *   0        the draw's own cells (angles from the x axis, the whole turn);
 *   1, 2, 4  cells in the frame of the geometry's baseline, over one of `fold`
 *            mirrored sectors of 1/fold turn -- the cells of an IMPORTANCE
 *            sampler with this fold and frame = atan2(By, Bx) / 2 pi (qrs.h).
 *            Term k (stream point k) has R2 coordinate Y (0.64 turns); with
 *            the frame as a 0.64 turn (x = atan2(By, Bx) / 2 pi in FP64,
 *            trunc(x 2^63) as a signed integer, doubled mod 2^64),
 *            W = Y - frame mod 2^64, the sector q is the top log2(fold) bits
 *            of W, the rest W' (complemented when q is odd) gives the angular
 *            cell ((W' >> 32) n_theta) >> 32; the radial band is the draw's. */
#define QRS_TARGET_MEAN 0
#define QRS_TARGET_RMS 1

qrs_status qrs_proposal_targets(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, int32_t n_rho,
                                int32_t n_theta, uint64_t seed, int64_t n_f, int32_t n_draws, int32_t kind,
                                int32_t fold, const double* geom, int64_t n, float* targets, void* stream);

/* Prior of the logits: for each geometry and importance cell c (the cells of
 * an IMPORTANCE sampler with this fold and frame = atan2(By, Bx) / 2 pi), the
 * mean over 64 points placed in the cell -- (u, t) = ((i_rho + s_x) / n_rho,
 * (i_theta + s_y) / n_theta), (s_x, s_y) the first 64 points of the R2
 * sequence of Eq. 6 from (1/2, 1/2) -- of
 *     g = W(rho) A(pi D rho)^2 (1 - cos(2 pi rho |B| cos phi)) rho^2,
 * rho = fmin (fmax/fmin)^u, phi the angle from the baseline (2 pi t / fold in
 * the folded frame, 2 pi t - atan2(By, Bx) for fold 0): the cell's share of
 * the differential-piston structure function at B (Sec. 4.4 with the Eq. 7
 * filter) up to a constant, a PSD-aware mapping in the sense of Sec. 5.
 * prior [n][n_rho n_theta] (device FP32) = log(v_c / max v), floored at -60.
 * The PSD kind from psd (r0, L0 from the geometries; psd's own filter off). */
qrs_status qrs_proposal_prior(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, int32_t n_rho,
                              int32_t n_theta, int32_t fold, const double* geom, int64_t n, float* prior, void* stream);

/* Forward pass: logits [n][C] = MLP(features of geom [n][5], device FP64)
 * + prior [n][C] (device FP32, e.g. from qrs_proposal_prior), or the MLP
 * alone when prior is NULL. */
qrs_status qrs_mlp_forward(qrs_handle* h, int32_t n_cells, const float* params, const double* geom,
                           const float* prior, int64_t n, float* logits, void* stream);

/* Loss and gradient at params: grad [param_count] (overwritten), loss [1]
 * (device FP32, the mean cross entropy of softmax(logits) against targets,
 * logits as in qrs_mlp_forward with the same prior or NULL; the prior is a
 * constant of the loss).  targets [n][C] rows sum to 1. */
qrs_status qrs_mlp_loss_grad(qrs_handle* h, int32_t n_cells, const float* params, const double* geom,
                             const float* prior, const float* targets, int64_t n, float* grad, float* loss,
                             void* stream);

/* One Adam step (step >= 1: bias correction t = step) with learning rate lr:
 * params, m, v [param_count] updated in place from grad. */
qrs_status qrs_mlp_adam(qrs_handle* h, int32_t n_cells, float* params, float* m, float* v, const float* grad,
                        float lr, int64_t step, void* stream);

/* ------------------------------------------------------------ training ---
 * Training state of the network: the parameters and Adam's two moment
 * vectors (device FP32 [qrs_mlp_param_count(n_cells)] each, caller-owned)
 * and the number of Adam steps taken (host).  A fresh run: params from
 * qrs_mlp_init, m = v = 0, step = 0. */
typedef struct qrs_mlp_state {
    int32_t n_cells;
    int32_t reserved;
    int64_t step;
    float* params;
    float* m;
    float* v;
} qrs_mlp_state;

#define QRS_LR_CONSTANT 0
#define QRS_LR_COSINE 1

/* Full-batch Adam on the mean cross entropy of qrs_mlp_loss_grad (with the
 * prior [n][C] or NULL): `steps`
 * steps t = state->step + 1 .. state->step + steps, each the loss and
 * gradient at the current parameters followed by qrs_mlp_adam's update with
 * bias correction t; state->params, m, v are updated in place and
 * state->step advances by `steps` (on success).  The learning rate of step t
 * is formed in FP64 and rounded once to FP32:
 *   QRS_LR_CONSTANT  lr
 *   QRS_LR_COSINE    lr (1 + cos(pi (t - 1) / total_steps)) / 2, the cosine
 *                    schedule of a run of total_steps steps (total_steps >=
 *                    state->step + steps), so a run split into several calls
 *                    follows the same schedule as one call.
 * The result equals, bit for bit, the same steps taken one call at a time
 * through qrs_mlp_loss_grad and qrs_mlp_adam, and a run resumed from a
 * checkpoint (qrs_mlp_save / qrs_mlp_load) equals an uninterrupted one.
 *   geom [n][5] device FP64, targets [n][n_cells] device FP32 (rows sum to 1),
 *   loss_trace: device FP32 [steps] receiving each step's loss (before its
 *   update), or NULL.
 * Workspace: the handle's (the backward pass's buffers and the gradient).
 * Errors: QRS_ERR_ARG for invalid sizes, pointers, lr <= 0, an unknown
 * schedule, total_steps too small; nothing is launched then. */
qrs_status qrs_proposal_train(qrs_handle* h, qrs_mlp_state* state, const double* geom, const float* prior,
                              const float* targets, int64_t n, int64_t steps, double lr, int32_t schedule,
                              int64_t total_steps, float* loss_trace, void* stream);

/* Checkpoint of a training state: qrs_mlp_save writes n_cells, step, params,
 * m and v to the file `path` (host path; the file holds the 8 bytes
 * "QRSMLP01", int32 n_cells, int32 0, int64 step, int64 parameter count, then
 * the three FP32 vectors), after synchronising `stream`.  qrs_mlp_load reads
 * one into a state whose n_cells and device vectors the caller has set up,
 * and sets state->step; a file of another size or network returns
 * QRS_ERR_ARG with the state untouched.  Both return when the copies are
 * complete. */
qrs_status qrs_mlp_save(qrs_handle* h, const qrs_mlp_state* state, const char* path, void* stream);
qrs_status qrs_mlp_load(qrs_handle* h, qrs_mlp_state* state, const char* path, void* stream);

/* Two-level sampling CDF from one row of logits (device [n_rho n_theta]):
 * p = (1 - eps) softmax(beta z) + eps / C over the cells; the marginal over
 * radial bands and, per band, the conditional over its angular cells, each
 * quantised to integer widths >= 1 summing to 2^32 (floor of p (2^32 - n) plus
 * one, the remainder to the largest entry); cdf [n_rho + n_rho n_theta]
 * (device uint32) holds their start points in the format of
 * qrs_sampler.cell_cdf.  0 < eps <= 1 (the mixture with the uniform density
 * bounds every weight); 0 < beta <= 16 (beta < 1 flattens the network's
 * density: the targets are variance-optimal for independent draws, and the
 * stratified R2 draws gain from a flatter one). */
qrs_status qrs_proposal_cdf(qrs_handle* h, int32_t n_rho, int32_t n_theta, const float* logits, float eps,
                            float beta, uint32_t* cdf, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QRS_PROPOSAL_H */
