/*
 * dtwgb_encoder.h -- the proposal encoder: a small convolutional network whose
 * embedding distances are trained to follow DTW distances, used to propose
 * initial medoids and medoid-swap candidates for k-medoids.  The paper has no
 * learned part; this is the project's addition on top of its k-medoids
 * (Mathematical background, last paragraph), and every cost it proposes is
 * re-evaluated with exact DTW.
 *
 * Network (one series of length T, T a multiple of 64, 64 <= T <= 832):
 *   z1 = conv1(x) + b1, h1 = GELU(z1)      1 -> 64 channels, kernel 7, zero padding 3
 *   z2 = conv2(h1) + b2, h2 = GELU(z2)    64 -> 64 channels, kernel 7
 *   z3 = conv3(h2) + b3, h3 = GELU(z3)    64 -> 64 channels, kernel 7
 *   g = mean over time of h3; e = Wl g + bl  (64-dim embedding)
 * GELU(z) = z * Phi(z).  Weights and activations are bfloat16, accumulation is
 * float32; the 64-channel convolutions run on the tensor cores (tcgen05 with
 * TMEM accumulators).  Master weights and Adam state are float32.
 *
 * Parameters are one float32 vector of dtw_encoder_num_params() values:
 * W1 [64][7], b1 [64], W2 [7][64][64] (tap, out, in), b2 [64], W3 [7][64][64],
 * b3 [64], Wl [64][64] (out, in), bl [64].
 *
 * Training step (full batch): series x [S][T], targets s [S][S] (symmetric;
 * the diagonal is ignored):
 *   L = (1 / P) * sum_{a < b} (||e_a - e_b|| - s_ab)^2,   P = S (S - 1) / 2,
 * then one Adam update (beta1 0.9, beta2 0.999, eps 1e-8) with rate lr.
 *
 * All array arguments are device pointers unless marked host.  Calls enqueue
 * on `stream` and do not synchronise unless they return host values.
 */
#ifndef DTWGB_ENCODER_H
#define DTWGB_ENCODER_H

#include <stdint.h>

#include "dtwgb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtw_encoder dtw_encoder;

/* Number of float32 parameters (62,144). */
int32_t dtw_encoder_num_params(void);

/* Workspace for series of length T and up to max_batch series per call
 * (training batches and embedding batches).  Parameters start at zero: load
 * them with dtw_encoder_set_params.  Errors: DTW_EINVAL (T not a multiple of
 * 64 or outside [64, 832], max_batch < 2), DTW_ENOMEM. */
int dtw_encoder_create(int32_t T, int32_t max_batch, dtw_encoder **out);

/* Load the float32 master parameters (host) and reset Adam's moments and
 * step count; synchronous. */
int dtw_encoder_set_params(dtw_encoder *enc, const float *host_params);

/* Initialise the parameters on the device and reset Adam's state:
 * parameter i = std * z_i with z_i standard normal by Box-Muller from outputs
 * 2i+1 and 2i+2 of the splitmix64 stream of `seed` (Steele, Lea & Flood
 * 2014); std = sqrt(2/7) for W1, sqrt(2/448) for W2 and W3, 1/8 for Wl; biases
 * zero.  Synchronous. */
int dtw_encoder_init_params(dtw_encoder *enc, uint64_t seed);

/* Copy the float32 master parameters to the host; synchronous. */
int dtw_encoder_get_params(const dtw_encoder *enc, float *host_params);

/* Gradient of the loss at the parameters of the last training step (before
 * its Adam update), float32, to the host; synchronous. */
int dtw_encoder_get_grads(const dtw_encoder *enc, float *host_grads);

/* Embeddings of B series: x [B][T] float32 -> emb [B][64] float32.
 * Errors: DTW_EINVAL for B < 1 or B > max_batch. */
int dtw_encoder_embed(dtw_encoder *enc, const float *x, int32_t B, float *emb, void *stream);

/* `steps` full-batch training steps on S series x [S][T] with targets [S][S];
 * the loss of every step is written to loss_dev[step] (device).  With
 * use_graph != 0 one step is captured into a CUDA graph on the first call for
 * these buffers and replayed.  lr_dev is a device float read by every step
 * (it can be changed between calls).  loss_dev must hold `steps` floats.
 * Errors: DTW_EINVAL for S < 2 or S > max_batch. */
int dtw_encoder_train(dtw_encoder *enc, const float *x, int32_t S, const float *targets,
                      const float *lr_dev, int32_t steps, float *loss_dev, int32_t use_graph,
                      void *stream);

/* Regression targets from a DTW matrix D [S][S] (device):
 * targets[a][b] = sqrt(D[a][b]) / mean_{a != b} sqrt(D[a][b]), zero diagonal.
 * sqrt because the paper's DTW cost is a sum of squared differences; the
 * scale makes the targets unit-mean.  Asynchronous. */
int dtw_encoder_targets(const float *D, int32_t S, float *targets, void *stream);

/* Tensors of the last training step, for checking the network layer by layer
 * (dtw_encoder_get_tensor).  Activations are [S][T][64] (series, step,
 * channel); the embeddings e and their loss gradient dL/de are [S][64]. */
#define DTW_ENC_Z1 0  /* conv1 pre-activation, bfloat16 values */
#define DTW_ENC_H1 1  /* GELU(z1), bfloat16 */
#define DTW_ENC_Z2 2
#define DTW_ENC_H2 3
#define DTW_ENC_Z3 4
#define DTW_ENC_H3 5
#define DTW_ENC_DZ3 6 /* dL/dz3, bfloat16 */
#define DTW_ENC_DZ2 7
#define DTW_ENC_DZ1 8
#define DTW_ENC_E 9   /* embeddings, float32 */
#define DTW_ENC_DE 10 /* dL/de, float32 */

/* Copy tensor `which` (DTW_ENC_*) of the last dtw_encoder_train call's last
 * step to host_out as float32 in the layout above (S of that call; bfloat16
 * values widened exactly).  Synchronises the device.  Errors: DTW_EINVAL for
 * an unknown tensor or before any training step. */
int dtw_encoder_get_tensor(const dtw_encoder *enc, int32_t which, float *host_out);

/* Synchronises the device and reports whether a tensor-core kernel of this
 * encoder gave up waiting for its MMAs to complete (then DTW_ETIMEOUT: the
 * outputs of the calls since the last check are invalid); clears the flag. */
int dtw_encoder_check(dtw_encoder *enc);

void dtw_encoder_destroy(dtw_encoder *enc);

#ifdef __cplusplus
}
#endif

#endif /* DTWGB_ENCODER_H */
