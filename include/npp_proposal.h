/* npp_proposal.h -- learned sampling proposal and the BF16 tensor-core GEMM.
 *
 * The paper draws the controller parameters isotropically, theta ~ N(0, I)
 * per sampling time (Sect. II-D "Fourth"), and names guiding the sampling
 * with pre-encoded knowledge as future work (Sect. V).  This interface adds
 * that guide without changing the method: a network maps a scene encoding
 * to the mean and standard deviation of a diagonal Gaussian over theta; a
 * plan step may draw its first N_prop samples from it, the rest stay
 * isotropic, and every sample is judged by the same exact rollout cost, so
 * the plain sampler wins whenever the proposal's samples are worse.
 *
 * Network: 72 inputs (64-bin polar obstacle histogram + the 8 rollout
 * inputs at h = 0) -> 256 ReLU -> 256 ReLU -> 900 = (mean, log-std) of the
 * 450 parameters of the 8-16-16-2 controller; log-std clamped to
 * [ls_min, ls_max].  BF16 weights and activations with FP32 accumulation
 * on the tensor cores (tcgen05), FP32 master weights, Adam.
 *
 * All device pointers are caller-owned unless stated; calls are
 * asynchronous on `stream` (a cudaStream_t, NULL for the legacy stream)
 * unless stated.  Errors: npp_last_error(NULL) holds the message.
 */
#ifndef NPP_PROPOSAL_H
#define NPP_PROPOSAL_H

#include <stdint.h>

#include "npp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NPP_PROP_NIN 72
#define NPP_PROP_HIDDEN 256
#define NPP_PROP_NTHETA 450

typedef struct npp_proposal npp_proposal;

typedef struct {
    int32_t batch;          /* rows per training step / most rows per forward: a multiple of 128 */
    float ls_min, ls_max;   /* clamp of the predicted log-std (ls_min < ls_max) */
    float beta1, beta2;     /* Adam moment decays in [0, 1) */
    float eps;              /* Adam denominator term, > 0 */
    int32_t device;         /* CUDA device */
} npp_proposal_config;

/* Allocates the network (parameters zero), its Adam state and activation
 * buffers for `batch` rows on the device.  NPP_INVALID_ARG for a bad
 * config, NPP_CUDA_ERROR when allocation or tensor-map set-up fails. */
npp_status npp_proposal_create(const npp_proposal_config* cfg, npp_proposal** out);
npp_status npp_proposal_destroy(npp_proposal* P);

/* Number of floats of the packed parameter layout: W1[256][72], b1[256],
 * W2[256][256], b2[256], W3[900][256], b3[900] (rows = outputs). */
int32_t npp_proposal_n_params(void);

/* Host copies in the packed layout (synchronous).  set_params also resets
 * the Adam moments and step count; NPP_INVALID_ARG for a non-finite value.
 * get_grads returns the gradient of the last training step's loss.  Both
 * getters return NPP_DEVICE_TIMEOUT if a GEMM pipeline wait timed out. */
npp_status npp_proposal_set_params(npp_proposal* P, const float* params_host);
npp_status npp_proposal_get_params(npp_proposal* P, float* params_host);
npp_status npp_proposal_get_grads(npp_proposal* P, float* grads_host);

/* Scene encodings x_dev[S][72] for S scene descriptors (a device array of
 * npp_scene, as for npp_plan_batch: state, goal, T, M, obs_offset) over the
 * world-frame points obs_dev (16-byte aligned [*][4]).  The feature scaling
 * is the planner handle's.  Histogram bin k of 64 covers headings
 * [-pi + k 2pi/64, -pi + (k+1) 2pi/64) in the EV-aligned frame at t; a point
 * at distance d adds max(0, 1 - d / 20 m); entry k is h_k / (1 + h_k). */
npp_status npp_proposal_encode(const npp_handle* h, const npp_scene* scenes_dev, int32_t S,
                               const float* obs_dev, float* x_dev, void* stream);

/* Proposal of n <= batch scenes: mean_dev[n][450], std_dev[n][450]. */
npp_status npp_proposal_forward(npp_proposal* P, const float* x_dev, int32_t n, float* mean_dev,
                                float* std_dev, void* stream);

/* One Adam step on the mean Gaussian negative log-likelihood of
 * theta_dev[batch][450] under the proposal of x_dev[batch][72]; the loss
 * before the update goes to loss_dev (one float, may be NULL). */
npp_status npp_proposal_train_step(npp_proposal* P, const float* x_dev, const float* theta_dev,
                                   float lr, float* loss_dev, void* stream);

/* npp_plan_step whose samples n < N_prop are drawn from the proposal:
 * theta_n,i = fma(std_dev[i], eps_n,i, mean_dev[i]) rounded once to FP32,
 * eps the normals of Philox stream 1 (same counter layout as the isotropic
 * samples, stream field 1); samples n >= N_prop are the isotropic samples
 * of npp_plan_step, and warm_dev still replaces sample 0.  mean_dev and
 * std_dev hold n_theta floats.  0 <= N_prop <= N. */
npp_status npp_plan_step_proposal(npp_handle* h, const npp_state* state, const npp_goal* goal,
                                  const float* obs_dev, int32_t M, int32_t N, int32_t T,
                                  uint64_t seed, uint32_t t_index, const float* warm_dev,
                                  const float* mean_dev, const float* std_dev, int32_t N_prop,
                                  const npp_outputs* out, void* stream);

/* C_dev[M][N] (FP32, row-major) = A_dev[M][K] B_dev[N][K]^T with BF16
 * operands given as raw 16-bit patterns, rows K-contiguous, FP32
 * accumulation on the tensor cores.  M, N multiples of 128, K of 64; all
 * pointers 16-byte aligned.  NPP_INVALID_ARG otherwise. */
npp_status npp_gemm_bf16(const uint16_t* A_dev, const uint16_t* B_dev, float* C_dev, int32_t M,
                         int32_t N, int32_t K, void* stream);

/* Synchronous: NPP_DEVICE_TIMEOUT (and clears it) if a pipeline wait of an
 * npp_gemm_bf16 launch timed out since the last call, else NPP_OK. */
npp_status npp_gemm_status(void);

#ifdef __cplusplus
}
#endif

#endif
