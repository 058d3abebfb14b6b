/*
 * libtpcf emulator ABI: a small multilayer perceptron that maps model parameters
 * theta = (f, b1, b2, sigma8, alpha, eps) to the tree-level anisotropic 3PCF
 * multipoles zeta_{l1 l2 L}(r1, r2) (the model of Sec. 2.3-2.5 of
 * arXiv:2408.03036, whose evaluation dominates parameter inference, Sec. 5).
 * The paper itself has no emulator; this is an accelerator for its model.
 *
 * Network: widths[0] inputs, hidden layers widths[1..n-1] with SiLU, widths[n]
 * linear outputs.  Weights are kept in FP32 (master copy, Adam state) and used
 * as BF16 in every product, with FP32 accumulation.  Inputs are scaled to
 * [-1, 1] with the box given to tpcf_emu_set_input_box; outputs are learned
 * standardised by the per-output mean and standard deviation that
 * tpcf_emu_fit_output_scaling measures on the training targets.  The loss is
 * the mean squared error of the standardised outputs.
 *
 * Parameters are one FP32 vector: for every layer l, W_l [in_l][out_l]
 * (row-major) followed by b_l [out_l].
 *
 * All device pointers are caller-owned and all calls are asynchronous on the
 * given stream (NULL: the legacy default stream); the handle owns its weights,
 * optimiser state and scratch.  Batches run in passes of up to 32768 rows; the
 * per-pass scratch is allocated on first use and grows with the batch (a call
 * that grows it synchronises its stream first).  Status codes are those of tpcf.h.
 */
#ifndef TPCF_EMU_H
#define TPCF_EMU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpcf_emu_s *tpcf_emu;

/* Creates a network with n_layers linear layers (widths[0..n_layers], host;
 * 1 <= n_layers <= 8, widths 1..4096) and Glorot-uniform weights drawn from a
 * counter-based hash of (seed, parameter index); biases start at zero. */
int tpcf_emu_create(const int32_t *widths, int32_t n_layers, uint64_t seed, tpcf_emu *out);

/* Releases the handle (synchronises the device first).  NULL is accepted. */
int tpcf_emu_destroy(tpcf_emu emu);

/* Number of parameters (host out). */
int tpcf_emu_param_count(tpcf_emu emu, int64_t *n_params);

/* Input box: x_scaled = 2 (x - lo) / (hi - lo) - 1 per input (host lo, hi [widths[0]]). */
int tpcf_emu_set_input_box(tpcf_emu emu, const float *lo, const float *hi);

/* Measures the per-output mean and standard deviation of n rows of targets
 * (dev y [n][widths[n_layers]]) and keeps them as the output scaling. */
int tpcf_emu_fit_output_scaling(tpcf_emu emu, const float *y, int64_t n, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch: dev x [batch][in],
 * dev y [batch][out] in physical units; dev loss (one double, may be NULL)
 * receives the batch loss before the update. */
int tpcf_emu_train_step(tpcf_emu emu, const float *x, const float *y, int64_t batch, float lr, double *loss,
                        void *stream);

/* Loss and its gradient with respect to every parameter (dev grad [n_params])
 * on a batch, without updating anything. */
int tpcf_emu_gradients(tpcf_emu emu, const float *x, const float *y, int64_t batch, float *grad, double *loss,
                       void *stream);

/* Predictions in physical units: dev x [n][in] -> dev y [n][out]; any n >= 0. */
int tpcf_emu_predict(tpcf_emu emu, const float *x, int64_t n, float *y, void *stream);

/* Copies the FP32 parameters out of / into the handle (dev params [n_params]).
 * Setting them also resets the optimiser state. */
int tpcf_emu_get_params(tpcf_emu emu, float *params, void *stream);
int tpcf_emu_set_params(tpcf_emu emu, const float *params, void *stream);

/* Host copies of the output scaling (host mean, std [out]). */
int tpcf_emu_get_output_scaling(tpcf_emu emu, float *mean, float *std_dev);

/* Sets the output scaling from host arrays (mean, std [out]; every std > 0), as
 * a checkpoint restores it. */
int tpcf_emu_set_output_scaling(tpcf_emu emu, const float *mean, const float *std_dev);

/* Host copies of the input box (host lo, hi [in]). */
int tpcf_emu_get_input_box(tpcf_emu emu, float *lo, float *hi);

/* The Adam state, for checkpoints: first and second moments (dev m, v
 * [n_params]) and the step count (host).  Setting it after tpcf_emu_set_params
 * (which resets the state) resumes training exactly where it was saved. */
int tpcf_emu_get_optimizer(tpcf_emu emu, float *m, float *v, int64_t *step, void *stream);
int tpcf_emu_set_optimizer(tpcf_emu emu, const float *m, const float *v, int64_t step, void *stream);

#ifdef __cplusplus
}
#endif

#endif
