/*
 * sgtp_mlp.h -- C ABI of the learned proposal of the B300 SGTP engine.
 *
 * Not part of the SGTP paper: a small network maps Frenet-relative ego and
 * opponent features to a Gaussian over the control sequence of a best
 * response.  In a learned plan, K_prop of the K samples of every best
 * response are drawn from that Gaussian and the rest from the paper's plain
 * sampler N(U-bar, diag(sigma_a^2, sigma_delta^2)) (Sec. II); selection is
 * unchanged (Eq. selection, least-violation fallback, Sec. III-B), so the
 * plain sampler remains the fallback.  The network is trained on best
 * responses the plain planner selects.
 *
 * Network: x (64 features) -> 256 -> 256 -> 256 -> 4T, ReLU hidden layers,
 * BF16 weights and activations, FP32 accumulation on the tensor cores, FP32
 * master weights for Adam.  Output row: [mu_a(T), mu_delta(T), logsig_a(T),
 * logsig_delta(T)] in units of the plain sampler's sigma per channel;
 * logsig is clamped to [-5, 2].  The proposal is a residual around the
 * plain sampler's centre: per step, mean = U-bar + sigma_plain mu and
 * sigma = sigma_plain exp(logsig), so mu = 0, logsig = 0 is the plain
 * sampler.  Parameters are laid out per layer l as W_l [out][in]
 * (row-major) followed by b_l [out].
 *
 * Features of vehicle i (all float32, computed on the device by the plan
 * kernel; sgtp_ibr_plan_learned can write them out):
 *   0   d_i / 5                    lateral offset
 *   1,2 sin e_psi, cos e_psi       heading error against the raceline
 *   3   v_i / 60
 *   4-7 100 kappa(s_i + {0, 20, 40, 80} m)   raceline curvature ahead
 *   8 + 6q .. 13 + 6q, q = 0..8: the q-th nearest opponent by |Delta s|:
 *       [1, Delta s / 40, d_j / 5, (v_j - v_i) / 10, wrap(psi_j - psi_i),
 *        (prog_j - v_i T dt) / 40]   (zeros for absent slots)
 *       with Delta s = wrap(s_j - s_i) and prog_j the opponent prediction's
 *       progress gain over the horizon
 *   62  n_opp / 9
 *   63  1 if the response uses the game term (rounds >= 1), else 0
 */
#ifndef SGTP_MLP_H
#define SGTP_MLP_H

#include "sgtp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SGTP_MLP_IN 64
#define SGTP_MLP_HIDDEN 256

typedef struct sgtp_mlp sgtp_mlp;   /* opaque, device resident, library owned */

/* Number of parameters of the network for horizon T (4T outputs). */
size_t sgtp_mlp_param_count(int32_t T);

/* Create a network for horizon T with Kaiming-uniform weights drawn from
 * Philox with `seed` and zero biases; Adam moments zero.  Blocks. */
sgtp_status sgtp_mlp_create(int32_t T, uint64_t seed, void *stream, sgtp_mlp **out);
void sgtp_mlp_destroy(sgtp_mlp *m);

/* Grow the network's batch scratch to `batch` rows (setup-time allocation;
 * forward / train_step call it themselves when needed, so call it before
 * capturing them in a graph). */
sgtp_status sgtp_mlp_reserve(sgtp_mlp *m, int32_t batch);

/* Forward pass on a DEVICE batch x [batch x 64] -> out [batch x 4T] (FP32,
 * before the logsig clamp). */
sgtp_status sgtp_mlp_forward(sgtp_mlp *m, const float *x, int32_t batch, float *out, void *stream);

/* Forward pass followed by the proposal transform: prop [batch x T x 4]
 * DEVICE floats, per step (a_nom + sigma_a mu_a, delta_nom + sigma_delta
 * mu_delta, sigma_a exp(logsig_a), sigma_delta exp(logsig_delta)), logsig
 * clamped to [-5, 2] -- the input of sgtp_best_response_mixed.  u_nom
 * [batch x T x 2] DEVICE: each row's nominal controls U-bar (NULL: zero). */
sgtp_status sgtp_mlp_proposal(sgtp_mlp *m, const float *x, const float *u_nom, int32_t batch, float sigma_a,
                              float sigma_delta, float *prop, void *stream);

/* One training step on a DEVICE batch: forward, Gaussian NLL of target
 * [batch x 2T] per step, mean over
 * batch x 2T elements (the learned proposal trains on the residuals
 * ((U*_a - a_nom) / sigma_a, (U*_delta - delta_nom) / sigma_delta) of the
 * selected controls U* around the nominal); backward; and, when apply != 0,
 * one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the FP32 master
 * weights with a refreshed BF16 copy.  Optional DEVICE outputs: loss_out [1]
 * and grad_out [param_count] (the gradient before the update). */
sgtp_status sgtp_mlp_train_step(sgtp_mlp *m, const float *x, const float *target, int32_t batch, float lr,
                                float *loss_out, float *grad_out, int32_t apply, void *stream);

/* Copy the FP32 master parameters to / from HOST memory (param_count
 * floats); set also refreshes the BF16 copy.  Both block. */
sgtp_status sgtp_mlp_get_params(const sgtp_mlp *m, float *host_out);
sgtp_status sgtp_mlp_set_params(sgtp_mlp *m, const float *host_in);

/* T, parameter count, Adam steps taken, and the device BF16 parameter copy. */
sgtp_status sgtp_mlp_info(const sgtp_mlp *m, int32_t *T, int64_t *n_params, int64_t *step, const void **bf16_params);

/* The best response of sgtp_best_response with K_prop of its K samples drawn
 * from a per-step proposal: prop [T x 4] DEVICE floats (mean a, mean delta,
 * sigma a, sigma delta); samples k < K_prop use u = Pi_U(mean + sigma z) with
 * the noise stream bit set (counter word 1 bit 31), the others the plain
 * sampler.  cost_star [1] (DEVICE, optional) receives the selected sample's
 * cost (its violation when no sample is feasible). */
sgtp_status sgtp_best_response_mixed(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, const float *x0,
                                     const float *u_nom, float vref_scale, const float *opp, int32_t n_opp,
                                     int32_t T, int32_t K, uint64_t seed, uint32_t race, uint32_t agent,
                                     uint32_t round, int32_t game_on, const float *prop, int32_t K_prop,
                                     int32_t *k_star, float *u_star, float *xi_star, int32_t *any_feasible,
                                     float *cost_star, void *workspace, size_t workspace_bytes, void *stream);

/* The planning call of sgtp_ibr_plan with the learned proposal: before each
 * best response (every round and the extra ego response) the kernel
 * computes the vehicle's features and runs the network on the tensor cores;
 * K_prop of the K samples come from the resulting Gaussian, the rest from
 * the plain sampler.  mlp may be NULL (plain sampler only).  feat_out
 * (optional, DEVICE, (L+2) x n_v x 64 floats) receives the features of every
 * best response (slot r = round r; in slot L+1 only the ego's row is
 * written), with or without a network -- the training inputs.  prop_out
 * (optional, DEVICE, (L+2) x n_v x T x 4 floats, same slots; ignored when
 * mlp is NULL) receives each proposal (mean a, mean delta, sigma a, sigma
 * delta per step).  With K_prop = 0 the result equals sgtp_ibr_plan's. */
sgtp_status sgtp_ibr_plan_learned(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                  const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                                  int32_t L, int32_t ego, uint64_t seed, uint32_t race, const sgtp_mlp *mlp,
                                  int32_t K_prop, float *xi_out, int32_t *k_star_out, float *xi_hist, float *u_hist,
                                  float *feat_out, float *prop_out, int32_t *status_dev,
                                  const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* sgtp_batch_plan with the learned proposal (every race's horizon must be
 * the network's T).  feat_out / prop_out (optional) have (L+2) slots of
 * agents x 64 features / agents x T x 4 proposal values, agents in the
 * batch's order (race by race), with the semantics of
 * sgtp_ibr_plan_learned. */
sgtp_status sgtp_batch_plan_learned(const sgtp_batch *b, const sgtp_params *p, const sgtp_mlp *mlp, int32_t K_prop,
                                   const float *X0, float *U_io, const float *vref_scale, uint64_t seed,
                                   float *xi_out, int32_t *k_star_out, float *xi_hist, float *u_hist,
                                   float *feat_out, float *prop_out, int32_t *status_dev,
                                   const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                   void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SGTP_MLP_H */
