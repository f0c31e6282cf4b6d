// Kernel-level state structs and launcher declarations shared by the
// library's translation units.
#pragma once

#include "pba_internal.cuh"

namespace pba {

// Per-frame state used by the pass kernels.
struct FrameState {
    float* fc;               // F * kFrameConst FP32 constants of the current poses
    float* fc_prev;          // F * 12 FP32 R|t of the previous poses
    float* dtheta32;         // F * 6 last update (FP32)
    const double* dtheta64;  // F * 6 last update (FP64)
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
    double fx, fy, inv_fx, inv_fy;
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

// Schur complement (pba_schur.cu)
// Co-visibility lists of the sparse Schur complement (device pointers):
// pair_fg[2p..2p+1] = frame pair (f <= g); the pair's chunks are
// [pair_chunk[p], pair_chunk[p+1]); chunk c covers items [chunk_start[c],
// chunk_start[c+1]) of pair chunk_pair[c]; an item is (entry of f, entry of
// g) of one tile that sees both frames.
struct SchurLists {
    const int* pair_fg;
    const int* pair_chunk;
    const int* chunk_pair;
    const int* chunk_start;
    const int2* items;
    int n_pairs, n_chunks;
};
constexpr int kSchurChunk = 16;
cudaError_t launch_schur_sparse(const DevProblem& pb, const float* Hfd, const float* Hnn,
                                const SchurLists& sl, float2* part, double* Soff,
                                cudaStream_t st, int* launches);
cudaError_t launch_assemble_S(int F, const double* Hff, int hff_stride, const double* Soff,
                              const double* anchor_t, double gauge_w, double* S, int* active,
                              cudaStream_t st);
// FP64 Cholesky (pba_chol.cu): A (consumed) -> L (lower, with L^T in the
// upper triangle) and inv_diag = 1/L_ii
cudaError_t launch_cholesky(double* A, double* L, double* inv_diag, int n, int* err,
                            cudaStream_t st, int* launches);
cudaError_t launch_chol_inverse(const double* L, const double* inv_diag, double* Sinv, int n,
                                cudaStream_t st);
cudaError_t launch_ic_solve_update(const SolveArgs& a, const double* Sinv, const double* y,
                                   int y_stride, int y_off, cudaStream_t st);
cudaError_t launch_fc_solve_update(const SolveArgs& a, const double* L, const double* inv_diag,
                                   const double* y, int y_stride, int y_off, cudaStream_t st);

// setup kernels (pba_runtime.cu)
cudaError_t launch_setup(const DevProblem& pb, float* gx, float* gy, float* I0p, cudaStream_t st);

}  // namespace pba
