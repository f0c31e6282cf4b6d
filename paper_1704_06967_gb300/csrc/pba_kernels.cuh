// Kernel-level state structs and launcher declarations shared by the
// library's translation units.
#pragma once

#include "pba_internal.cuh"

namespace pba {

// Per-frame state used by the pass kernels.
struct FrameState {
    float* fc;        // F * kFrameConst FP32 constants of the current poses
    float* fc_prev;   // F * 12 FP32 R|t of the previous poses
    float* dtheta32;  // F * 6 last update (FP32)
};

// Per-point state of one method (IC or FC) for the depth back-substitution.
struct DepthState {
    double* d64;          // current inverse depths (sorted order)
    const double* d0_64;  // p_0 inverse depths (IC rule)
    float* gn;            // g_d of the last linearisation / pass
    float* Hnn;           // H_dd of the system in use
    const float* Hfd;     // H_fd of the system in use (compact pairs)
    double* dd_last;      // last applied depth update
    int* err;
};

// IC precompute products.
struct IcStore {
    float4* J4;  // pairs * NC float4 chunks
    float* Hfd;  // pairs * 6
    float* Hnn;  // Npad
};

struct LaunchCtx {
    DevProblem pb;
    FrameState fs;
    DepthState ds_ic, ds_fc;
    IcStore ic;
    float* Hfd_fc;
    float* ent_part;
    TileStats* tstats;
    float* dthsq;     // F
    double* stats;    // slots * kStats
    const double* poses0;  // F*12 FP64 poses at p_0
    cudaStream_t stream;
};

size_t pass_smem_bytes(int F);
cudaError_t set_pass_smem_limits(int F);
cudaError_t launch_ic_precompute(const LaunchCtx& L);
cudaError_t launch_ic_pass(const LaunchCtx& L, bool accum, int apply, int have_prev);
cudaError_t launch_fc_pass(const LaunchCtx& L, bool accum, int apply, int have_prev);
cudaError_t launch_frame_reduce(const LaunchCtx& L, int off, int ncomp, double* out, int slot_cur,
                                int slot_prev, bool frames);

// linear algebra (pba_linalg.cu)
struct SolveArgs {
    int F, n6;
    const int* pat;
    int P;
    double fx, fy;
    double* poses64;        // F*12 current
    const double* poses0;   // F*12 p_0
    double* dtheta64;       // F*6
    float* dtheta32;        // F*6
    float* fc;              // F*kFrameConst
    float* fc_prev;         // F*12
    float* dthsq;           // F
    int* err;
    const int* active;      // [0] anchor frame, [f] frame has residuals
    const double* tanchor;  // F*12 poses whose t define the gauge direction
};

cudaError_t launch_schur_offdiag(const DevProblem& pb, const float* Hfd, const float* Hnn,
                                 const int2* frame_pairs, int n_pairs, double* Soff,
                                 cudaStream_t st);
cudaError_t launch_assemble_S(int F, const double* Hff, int hff_stride, const double* Soff,
                              const double* anchor_t, double gauge_w, double* S, int* active,
                              cudaStream_t st);
cudaError_t launch_cholesky(double* A, int n, int* err, cudaStream_t st);
cudaError_t launch_chol_inverse(const double* L, double* Sinv, int n, cudaStream_t st);
cudaError_t launch_ic_solve_update(const SolveArgs& a, const double* Sinv, const double* y,
                                   int y_stride, int y_off, cudaStream_t st);
cudaError_t launch_fc_solve_update(const SolveArgs& a, const double* L, const double* y,
                                   int y_stride, int y_off, cudaStream_t st);

// setup kernels (pba_runtime.cu)
cudaError_t launch_setup(const DevProblem& pb, float* gx, float* gy, float* I0p, cudaStream_t st);

}  // namespace pba
