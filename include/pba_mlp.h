/*
 * pba_mlp.h — learned inverse-depth proposal for the photometric bundle
 * adjustment library (C ABI; include/pba.h holds the context API).
 *
 * Not part of the paper: the paper starts every inverse depth from a base
 * solution (Sec. 4). This addition proposes each point's initial inverse
 * depth with a small MLP from its template patch and samples along its
 * epipolar lines, trained on the inverse depths the bundle adjustment itself
 * converges to; the constant-depth initialisation stays the fallback.
 *
 * Features of a point (pixel (u, v) in its bundle's reference frame 0),
 * PBA_MLP_IN = 96 FP32 values:
 *   [0, 64)   the 8 x 8 template patch I_0(u + dx, v + dy), dx, dy in -3..4,
 *             row-major in dy then dx (coordinates clamped into the image),
 *             as (I - mu) / (sigma + 1/255) with the patch's own mean mu and
 *             population standard deviation sigma;
 *   [64, 96)  16 matching costs along the epipolar line in each of two
 *             target frames: the first two frames (in frame order) that
 *             observe the point (one such frame: used twice; none: 4.0
 *             everywhere). Inverse depths d_m = 0.5 + (m + 1/2) 1.5 / 256,
 *             m = 0..255, place every pixel x_j of the point's P-pixel
 *             pattern at q = R x~_j + d_m t with the frame's current pose;
 *             the cost of d_m is the mean over j of (I(f_x q_x / q_z + c_x,
 *             f_y q_y / q_z + c_y), bilinear, normalised as the patch, minus
 *             the template's normalised value at x_j)^2, 4.0 when a
 *             projection is behind the camera or its 2 x 2 footprint leaves
 *             the image; value k of a frame is the least cost of
 *             d_m, m = 16 k .. 16 k + 15.
 * Network: 96 -> 128 -> 128 -> 128 -> 1, GELU (x Phi(x)) after each hidden
 * layer, output = inverse depth. Parameters, PBA_MLP_NPARAMS FP32 values in
 * this order: W1 [128][96] (row = output unit), b1 [128], W2 [128][128],
 * b2 [128], W3 [128][128], b3 [128], w4 [128], b4 [1].
 * Training loss: mean over the batch of (y - target)^2 / 2; Adam with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8.
 *
 * All pointers below are device pointers unless stated otherwise; nothing is
 * allocated by the library. Work is enqueued on cuda_stream (NULL = legacy
 * default stream) or, for the calls taking a context, the context's stream.
 */
#ifndef PBA_MLP_H
#define PBA_MLP_H

#include <stddef.h>

#include "pba.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PBA_MLP_IN 96
#define PBA_MLP_HIDDEN 128
#define PBA_MLP_NPARAMS 45569
/* inference layout: BF16 W1, W2, W3 (the tensor cores' shared-memory
 * layout), then FP32 b1, b2, b3, w4, b4 */
#define PBA_MLP_PACKED_BYTES 92176

/* Features of every point of `bundle` at the context's current poses
 * (normally p_0, before pba_precompute_ic). features: N_b x 96 FP32 rows in
 * the caller's point order of that bundle. Requires the workspace. */
pba_status pba_depth_features(pba_ctx* ctx, int bundle, float* features);

/* FP32 parameters (PBA_MLP_NPARAMS) -> the inference layout
 * (PBA_MLP_PACKED_BYTES, 16-byte aligned). Not synchronised. */
pba_status pba_mlp_pack(const float* params, void* packed, void* cuda_stream);

/* Inference on the tensor cores (tcgen05, BF16 weights and activations,
 * FP32 accumulation): out[i] = MLP(features[i]) for i < n. dev_flag: one
 * device int the call clears and the kernel sets if a tensor-core wait gives
 * up. Synchronises the stream; PBA_ERR_TIMEOUT when the flag was set. */
pba_status pba_mlp_infer(const void* packed, int n, const float* features, float* out, int* dev_flag,
                         void* cuda_stream);

/* Exercises the give-up path that every bounded device wait of the library
 * takes (the tensor-core completion waits above): one warp waits on a
 * barrier phase that nothing completes, gives up after its bound (a few
 * milliseconds at most), sets the error bit in dev_flag (one device int,
 * cleared first) and exits normally, leaving the context usable.
 * Synchronises the stream; returns PBA_ERR_TIMEOUT when the give-up reached
 * the host (the expected result), PBA_ERR_CUDA on a launch or copy error. */
pba_status pba_wait_selftest(int* dev_flag, void* cuda_stream);

/* Training scratch for a batch of n samples, in floats. */
size_t pba_mlp_scratch_floats(int n);

/* Gradient of the loss over n samples (FP32): grad (PBA_MLP_NPARAMS) and,
 * when loss is non-NULL, the batch's summed (y - t)^2 / 2 (one float).
 * params are not changed. Not synchronised. */
pba_status pba_mlp_grad(const float* params, int n, const float* features, const float* targets, float* grad,
                        float* loss, float* scratch, void* cuda_stream);

/* One Adam step (step counts from 1) on params with moments m, v
 * (PBA_MLP_NPARAMS each, zero before step 1) over a batch of n samples;
 * loss as for pba_mlp_grad. Not synchronised. */
pba_status pba_mlp_train_step(float* params, float* m, float* v, int step, float lr, int n,
                              const float* features, const float* targets, float* scratch, float* loss,
                              void* cuda_stream);

/* Proposes the inverse depths of `bundle` from its features at the current
 * poses and replaces the bundle's current inverse depths with them (clamped
 * into [0.05, 20]); points without matching data (no observing target frame,
 * or all 32 costs 4.0) keep their current inverse depth, the constant
 * initialisation being the fallback. Call pba_precompute_ic (or
 * pba_solve_ic) afterwards. scratch: N_b * 97 floats. Synchronises the
 * context's stream. */
pba_status pba_propose_depths(pba_ctx* ctx, int bundle, const void* packed, float* scratch);

#ifdef __cplusplus
}
#endif

#endif /* PBA_MLP_H */
