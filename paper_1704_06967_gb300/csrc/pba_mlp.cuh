// Constants and launchers of the learned inverse-depth proposal
// (pba_mlp.cu). The feature definition and the parameter order are those of
// include/pba_mlp.h.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/pba_mlp.h"
#include "pba_internal.cuh"

namespace pba {

constexpr int kMlpPatch = 8;        // 8 x 8 template patch
constexpr int kMlpPatchLo = -3;     // offsets -3 .. 4
constexpr int kMlpFrames = 2;       // target frames sampled along the epipolar line
constexpr int kMlpSamples = 16;     // matching-cost bins per frame
constexpr int kMlpSub = 16;         // inverse depths per bin
constexpr float kMlpNoData = 4.0f;  // cost where the pattern leaves the image
constexpr float kMlpDLo = 0.5f;     // inverse-depth range of the samples
constexpr float kMlpDHi = 2.0f;
constexpr float kMlpEps = 1.0f / 255.0f;
constexpr float kMlpDMin = 0.05f;   // proposals are clamped into [kMlpDMin, kMlpDMax]
constexpr float kMlpDMax = 20.0f;
constexpr int kMlpIn = PBA_MLP_IN;          // 96
constexpr int kMlpHidden = PBA_MLP_HIDDEN;  // 128
constexpr int kMlpTileM = 128;              // points per tensor-core tile (MMA M)
constexpr int kMlpParams = PBA_MLP_NPARAMS;

// offsets of the FP32 parameter vector: W1 b1 W2 b2 W3 b3 w4 b4
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpHidden * kMlpIn;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpHidden;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpHidden * kMlpHidden;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpHidden;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpHidden * kMlpHidden;
constexpr int kMlpOffW4 = kMlpOffB3 + kMlpHidden;
constexpr int kMlpOffB4 = kMlpOffW4 + kMlpHidden;
static_assert(kMlpOffB4 + 1 == kMlpParams, "parameter count");

// inference layout: BF16 W1, W2, W3 in the tensor cores' canonical shared-
// memory layout, then FP32 b1, b2, b3, w4, b4
constexpr uint32_t kMlpPackedWeightBytes = (kMlpHidden * kMlpIn + 2 * kMlpHidden * kMlpHidden) * 2;
constexpr int kMlpBiasFloats = 4 * kMlpHidden + 1;
static_assert(PBA_MLP_PACKED_BYTES >= kMlpPackedWeightBytes + kMlpBiasFloats * 4, "packed size");

cudaError_t launch_mlp_features(const DevProblem& pb, const float* fconst, const int* slot_caller, int tile0,
                                int ntiles, float* out, cudaStream_t st);
cudaError_t launch_mlp_propose(const int* slot_caller, int slot0, int nslots, const float* X, const float* y,
                               double* d64, cudaStream_t st);
cudaError_t launch_mlp_pack(const float* params, uint8_t* packed, cudaStream_t st);
cudaError_t launch_mlp_infer(const uint8_t* packed, int n, const float* X, float* out, int* err, cudaStream_t st);
size_t mlp_grad_scratch_floats(int n);
// gradient of the mean squared loss over n samples into grad (nullable) and,
// with m and v, one Adam step (step counts from 1) on params
cudaError_t launch_mlp_grad_adam(float* params, int n, const float* X, const float* T, float* scratch,
                                 float* grad, float* m, float* v, int step, float lr, float* loss,
                                 cudaStream_t st);

}  // namespace pba
