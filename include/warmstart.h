/*
 * warmstart.h -- learned warm start for child nodes (C ABI, sm_103a).
 *
 * In branch and bound every child node starts from its parent's solution
 * (Sec. 5.3).  The learned start keeps that and adds a correction predicted
 * per coordinate j by a small network f:
 *
 *     beta0_j = b_j + f(x_j),
 *     x_j = [ b_j, (X' grad F(X b))_j, fix_j, ||X_j||_2, |corr(X_j, y)| ],
 *
 * where b is the parent's solution beta^P with the child's J0 coordinates set
 * to zero (so the gradient at b shows how the branching moves every other
 * coordinate) and fix_j the child's fixing (-1 J0, 0 free, +1 J1).
 *
 * f: 5 -> 64 -> 64 -> 1, ReLU after both hidden layers, inputs standardised as
 * (x - shift) / scale.  Trained on (parent, child) pairs of solved nodes by
 * minimising the mean squared error between b_j + f(x_j) and the child's
 * converged beta_j.  A network whose output layer is zero gives exactly the
 * parent warm start.
 *
 * Parameters: one device float vector theta[RELAX_MLP_NPARAM], in this order
 *   W1 [64][5] (row = hidden unit), b1 [64], W2 [64][64] (row = output unit of
 *   layer 2), b2 [64], w3 [64], b3 [1]                 -> RELAX_MLP_NTRAIN trained
 *   shift [5], scale [5]                               -> fixed standardisation
 * bf16 != 0: the kernels evaluate the network with the trained entries rounded
 * to BF16 (round to nearest even), accumulating in FP32; bf16 = 0: FP32 weights.
 *
 * Conventions as in relax.h: "device" pointers are owned by the caller; work is
 * enqueued on `stream` (cudaStream_t as void*, NULL = legacy default stream);
 * errors are relax_status codes.
 */
#ifndef RELAX_WARMSTART_H
#define RELAX_WARMSTART_H

#include <stdint.h>

#include "relax.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RELAX_MLP_NTRAIN 4609
#define RELAX_MLP_NPARAM 4619

/* Features of a child node's coordinates.
 *   beta_parent: device p (handle dtype), the parent's solution.
 *   fixings: device int8[p] of the CHILD (as in relax_solve), NULL = none fixed.
 *   feat_out: device float[p][5], row j = x_j above; column 0 is b, the base
 *   that relax_mlp_forward adds the correction to.
 * The gradient at b is one fused pass over X (relax_xpass); the column norms
 * and correlations are computed in FP64 on the first call and kept by the
 * handle.  Synchronizes the handle's stream. */
relax_status relax_mlp_features(relax_handle* h, const void* beta_parent, const int8_t* fixings,
                                float* feat_out);

/* The start of a child: out[r] = 0 where feat[r][2] = -1 (the child's J0),
 * base[r] + f(feat[r]) elsewhere; base NULL: out[r] = f(feat[r]) for every r.
 *   theta: device float[RELAX_MLP_NPARAM]; feat: device float[rows][5];
 *   base, out: device float[rows].  rows = 0 is a no-op. */
relax_status relax_mlp_forward(const float* theta, int32_t bf16, const float* feat,
                               const float* base, int64_t rows, float* out, void* stream);

/* Gradient of L = mean_r (base[r] + f(feat[r]) - target[r])^2 with respect to theta.
 *   grad: device float[RELAX_MLP_NPARAM] (zero on shift and scale);
 *   loss: device float[1] receiving L, or NULL.  rows >= 1.
 * Per-CTA partial sums are added in a fixed order: the result is reproducible
 * bit for bit for a given rows and device.  Scratch is taken from the
 * stream-ordered allocator and returned before the call's work completes. */
relax_status relax_mlp_grad(const float* theta, int32_t bf16, const float* feat, const float* base,
                            const float* target, int64_t rows, float* grad, float* loss, void* stream);

/* One Adam step (Kingma and Ba, 2015) on the trained entries of theta:
 *   m, v: device float[RELAX_MLP_NTRAIN] moments (zero before step 1);
 *   t: step number, >= 1 (bias corrections 1 - beta1^t, 1 - beta2^t, and the
 *   complements 1 - beta, formed in FP64); 0 <= beta1, beta2 < 1, eps >= 0. */
relax_status relax_mlp_adam(float* theta, const float* grad, float* m, float* v, int32_t t, double lr,
                            double beta1, double beta2, double eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RELAX_WARMSTART_H */
