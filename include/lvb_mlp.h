/*
 * lvb_mlp.h -- the learned skin: a small network proposes each flagged
 * particle's skin from its local kinematics (an extension of the paper's
 * rule skin_p = K |v_p| dt, Eq. skin_formulus1; the paper itself has no
 * network).  The displacement check (Eq. update) still guards every list,
 * so a wrong proposal costs time, never a missed contact.
 *
 * Network (8 -> 32 -> 32 -> 1, ReLU), evaluated exactly as written, in
 * binary32 with bfloat16 weights and activations (round to nearest even):
 *   z_k  = bf16((f_k - mu_k) * isd_k)
 *   h1_o = bf16(relu(b1_o + sum_{k=0..7}  W1[o][k] z_k))     sums in k order
 *   h2_o = bf16(relu(b2_o + sum_{k=0..31} W2[o][k] h1_k))
 *   y    = b3 + sum_{k=0..31} w3[k] h2_k
 *   yc   = fminf(fmaxf(y, y_lo), y_hi)
 *   skin = (2 r) * yc                       (diameter form, y_steps = 0)
 *   skin = (2 r) * (f0 * (yc * y_steps))    (travel form, y_steps > 0)
 * then the cap of lvb.h; each product is rounded once, in the order
 * written.  relu(x) = x if x > 0 else 0; fmaxf / fminf return the other
 * operand when one is NaN.  Products of bfloat16 values are exact in
 * binary32, so the result does not depend on fused multiply-add use.  The
 * output range [y_lo, y_hi] keeps every proposal positive and bounded: the
 * network is used on states its training data may not cover.  In the
 * diameter form y is the skin in diameters; in the travel form it is the
 * skin in units of the particle's travel over y_steps steps at its present
 * speed (f0 d = |v| dt), a per-particle factor K / y_steps of the paper's
 * rule K |v| dt.
 *
 * Features f (binary32, at the step that flags the particle, from the state
 * before its update; d = 2 r, dt the policy's time step):
 *   f0 = (|v| dt) / d           f1 = ((|a| dt) dt) / d
 *   f2 = r / H                  (H: the scene's cap on r + skin)
 *   f3 = partners of the particle in the list
 *   f4 = steps since the particle's last update (0 at init)
 *   f5 = |x - xref| / skin_old  (0 if skin_old = 0)
 *   f6 = particles whose reference position lies in the cell of x
 *   f7 = (min over the box planes of the gap x - lo - r, hi - x - r) / d
 * |.| is sqrt((x*x + y*y) + z*z) with the correctly rounded square root;
 * at lvb_init all of f3..f6 are 0.
 *
 * Label used for training (rebuild logs): the largest displacement of the
 * particle over the `horizon` steps after its update, divided by d -- the
 * skin that would have kept it valid for exactly that many steps.
 */
#ifndef LVB_MLP_H
#define LVB_MLP_H

#include <stdint.h>

#include "lvb.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LVB_MLP_IN 8
#define LVB_MLP_HIDDEN 32
#define LVB_MLP_PARAMS 1377   /* 32*8 + 32 + 32*32 + 32 + 32 + 1 */

/* Device layout of the weights given to LVB_SKIN_LEARNED (lvb_skin_policy.mlp).
 * W1, W2, w3 hold bfloat16 values stored as binary32 (lvb_mlp_pack rounds
 * them).  W1 and W2 are stored input-major, [in][out] (W1[k * 32 + o] is
 * the weight from input k to hidden unit o), so that the 32 units' weights
 * of one input lie together; the master parameters of lvb_mlp_pack and of
 * training are [out][in]. */
typedef struct {
    float W1[LVB_MLP_HIDDEN * LVB_MLP_IN];
    float b1[LVB_MLP_HIDDEN];
    float W2[LVB_MLP_HIDDEN * LVB_MLP_HIDDEN];
    float b2[LVB_MLP_HIDDEN];
    float w3[LVB_MLP_HIDDEN];
    float b3;
    float mu[LVB_MLP_IN];
    float isd[LVB_MLP_IN];
    float y_lo, y_hi;    /* output range (in the output's unit) */
    float y_steps;       /* 0: diameter form; > 0: travel form over y_steps steps */
} lvb_mlp_weights;

/*
 * lvb_mlp_pack -- write an lvb_mlp_weights record from master parameters.
 *   params : host, LVB_MLP_PARAMS binary32 in the order W1, b1, W2, b2, w3, b3.
 *   mu, isd: host, LVB_MLP_IN each (feature offset and inverse scale).
 *   y_range: host, {y_lo, y_hi} with y_lo <= y_hi, or NULL for {0, +inf}
 *            (then yc = max(y, 0)).
 *   y_steps: 0 for the diameter form, else the travel form's step count
 *            (finite, > 0).
 *   out    : host or device lvb_mlp_weights (weights rounded to bfloat16).
 * Errors: EINVAL (NULL pointer, y_lo > y_hi or NaN, y_steps negative, NaN
 * or infinite), EDEVICE.
 */
int lvb_mlp_pack(const float *params, const float *mu, const float *isd, const float *y_range,
                 float y_steps, lvb_mlp_weights *out);

/*
 * lvb_mlp_infer -- the network on n feature rows: skin[i] by the weights'
 * output form with d = diam[i] and f0 = feats[i][0] (no cap), and y[i].
 * feats: device n x 8; diam, skin, y: device n (y may be NULL); w: device
 * weights.  Enqueues on `stream`.
 */
int lvb_mlp_infer(const float *feats, const float *diam, int64_t n, const lvb_mlp_weights *w,
                  float *skin, float *y, void *stream);

/* Training losses (the paper has no learned part: an extension). */
#define LVB_MLP_LOSS_SQUARED  0  /* mean of (y - t)^2 */
#define LVB_MLP_LOSS_RELATIVE 1  /* mean of ((y - t) / max(t, floor))^2: every
                                    label counts by its relative error, so
                                    slow particles are fitted as closely as
                                    fast ones (floor: the output range's
                                    lower end y_lo) */

/*
 * lvb_mlp_grad -- mean squared error of y against labels over n samples and
 * its gradient with respect to the master parameters (straight-through
 * through the bfloat16 roundings).  samples: device n x 9 (8 features,
 * label); params, mu, isd: host; rel_floor: 0 for the squared error, > 0
 * for the relative error with that floor; grad: host LVB_MLP_PARAMS; loss:
 * host.  Synchronises.  Errors: EINVAL (rel_floor < 0 or NaN).
 */
int lvb_mlp_grad(const float *samples, int64_t n, const float *params, const float *mu,
                 const float *isd, float rel_floor, float *grad, double *loss, void *stream);

/*
 * lvb_mlp_train -- train the network on the GPU with Adam.
 *   samples     : device n x 9 (features, label).
 *   loss_kind   : LVB_MLP_LOSS_SQUARED or LVB_MLP_LOSS_RELATIVE.
 *   params      : host in/out, LVB_MLP_PARAMS master parameters.
 *   mu, isd     : host out, the feature normalisation computed from the
 *                 samples (mean and 1/std per feature).
 *   y_range     : host out, {y_lo, y_hi} from the labels' mean m and
 *                 standard deviation sd: y_lo = m / 16, y_hi = m + 4 sd.
 *   losses      : host out, mean loss of every epoch (epochs entries).
 * Synchronises.  Errors: EINVAL, ENOMEM, EDEVICE.
 */
int lvb_mlp_train(const float *samples, int64_t n, int32_t epochs, int32_t batch, float lr,
                  uint64_t seed, int32_t loss_kind, float *params, float *mu, float *isd,
                  float *y_range, float *losses, void *stream);

/*
 * lvb_mlp_travel_labels -- rebuild-log samples turned into training samples
 * for the travel form of the output over `horizon` steps (y_steps =
 * horizon): the label becomes the largest displacement in units of the
 * particle's travel over the horizon at its speed when updated, times a
 * margin, clipped at a quantile.
 *   samples : device n x 9 (8 features, label), e.g. from lvb_log_read.
 *   out     : device, room for n x 9; must not overlap samples.  Receives,
 *             in their input order, the samples with f0 > 0 (a particle at
 *             rest has no travel and is left out), features unchanged and
 *             label
 *               y = (label * margin) / (f0 * horizon)     (binary32, each
 *                                                          operation rounded)
 *             then y = fminf(y, c), c the order statistic k = floor(clip_q
 *             (m - 1)) (0-based, ascending, binary64 product) of the m
 *             values y.
 *   horizon : >= 1 (the log's horizon); margin > 0, finite; 0 < clip_q <= 1.
 *   n_out   : host out, m.
 * Synchronises.  Errors: EINVAL, ENOMEM, EDEVICE.
 */
int lvb_mlp_travel_labels(const float *samples, int64_t n, int32_t horizon, float margin,
                          float clip_q, float *out, int64_t *n_out, void *stream);

/*
 * lvb_log_enable -- start recording training samples from a broad-phase
 * context (PARTIAL trigger): each particle's update opens a record with its
 * features; `horizon` steps later the record closes with its label and is
 * appended to a device buffer of `capacity` samples (later ones are
 * dropped).  A particle with an open record opens no other.  horizon >= 1.
 */
int lvb_log_enable(lvb_ctx *ctx, int32_t horizon, int64_t capacity);

/* lvb_log_read -- copy the recorded samples (n x 9 binary32, host or device)
 * and their count; cap limits the copy (LVB_ECAPACITY if more exist, with
 * *n_samples set).  Synchronises. */
int lvb_log_read(lvb_ctx *ctx, float *samples, int64_t cap, int64_t *n_samples);

#ifdef __cplusplus
}
#endif

#endif /* LVB_MLP_H */
