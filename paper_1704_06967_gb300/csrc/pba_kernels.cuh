// Kernel-level state structs and launcher declarations shared by the
// library's translation units.
#pragma once

#include <utility>

#include "pba_df.cuh"
#include "pba_internal.cuh"

namespace pba {

// Launch with programmatic stream serialisation (the kernel must call
// pdl_wait() before reading what the previous kernel on the stream wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Per-frame state used by the pass kernels.
struct FrameState {
    float* fc;               // F * kFrameConst FP32 constants of the current poses
    float* fc_prev;          // F * 12 FP32 R|t of the previous poses
    float2* dth2;            // F * 6 last update as FP32 pairs (hi, lo = v - hi)
    const double* dtheta64;  // F * 6 last update (FP64)
};

// Buffers of the per-entry iteration kernels (pba_iter.cu).
struct IterBufs {
    float* dcur;     // Npad FP32 depths the residual kernels use
    float* dprev;    // Npad FP32 depths before the last update
    float* gpart;    // E * 32 per-(entry, lane) J_d^T w r (FC: E * 64: that, then J_d^T w J_d)
    float4* estats;  // E (energy, r^2, count, max displacement)
    float* ddsq_t;   // T sum of Dd^2 of the last depth update
    float2* G0p;     // T * P * 32 template gradients (g_u, g_v) at the pattern pixels
};

// Per-point state of one method (IC or FC) for the depth back-substitution.
struct DepthState {
    double* d64;          // current inverse depths (sorted order)
    const double* d0_64;  // p_0 inverse depths (IC rule)
    float* gn;            // g_d of the last linearisation / pass
    float* Hnn;           // H_dd of the system in use
    const float* Hfd;     // H_fd of the system in use (compact pairs)
    const float* Had;     // joint brightness (IC): J_d^T W_0 [I_0, 1] per pair; null otherwise
    double* dd_last;      // last applied depth update
    int* err;
};

// IC precompute products.
struct IcStore {
    float4* J4;       // pairs * NC float4 chunks
    float* Hfd;       // pairs * 6
    float* Hnn;       // Npad
    double* inv_hnn;  // Npad 1 / H_dd (0 where H_dd = 0)
    double* inv_d0;   // Npad 1 / d_0
    float* part;      // E rows of kEntryPartial: the entry's 21 H_ff sums (kept for window updates)
    float* hpart;     // E * 32 per-(entry, lane) J_d^T W_0 J_d (kept for window updates)
    float* Had;       // joint brightness: pairs * 2 (J_d^T W_0 [I_0, 1]); null otherwise
    unsigned* vmask0; // joint brightness: pairs, pattern pixels valid at p_0
};

struct LaunchCtx {
    DevProblem pb;
    FrameState fs;
    DepthState ds_ic, ds_fc;
    IcStore ic;
    float* Hfd_fc;
    float* Had_fc;    // joint brightness (FC): pairs * 2, J_d^T W [-v, -1]
    float* aff_part;  // joint brightness (FC): E rows of kEntryPartial, the 15 H_pa / H_aa sums
    float* ent_part;
    TileStats* tstats;
    IterBufs it;
    float* dthsq;     // F
    double* stats;    // slots * kStats
    const double* poses0;  // F*12 FP64 poses at p_0
    cudaStream_t stream;
    int res_warps;         // warps per CTA of the accumulating IC residual pass (4, 8, 16)
    int photo;             // affine brightness: 0 off, 1 moment fit (the residual passes write its
                           // sums), 2 joint unknowns (IC: g_a sums and the Schur corrections)
};

// IC precompute of the entries of the frames with todo[f] != 0 (all when
// todo is null), then H_dd and its reciprocals for every point
cudaError_t launch_ic_precompute(const LaunchCtx& L, const unsigned char* todo = nullptr);
cudaError_t launch_ic_residual(const LaunchCtx& L, bool accum, int have_prev);
// out[f * ncomp + k] = sum over frame f's entries of part[off + k]
// (minus part[sub + k - sub_from] for k >= sub_from when sub >= 0)
cudaError_t launch_frame_reduce(const LaunchCtx& L, int off, int ncomp, double* out, int slot_cur,
                                int slot_prev, bool frames, int sub = -1, int sub_from = 0,
                                const float* src = nullptr);
cudaError_t launch_fc_residual(const LaunchCtx& L, bool accum, int have_prev);

// The bundles of a launch over reduced camera systems: B bundles described
// by the device array bund, or (bund null) the one bundle `one`.
struct BundleSet {
    int B;
    const BundleDesc* bund;
    BundleDesc one;
    int n6max;  // largest 6 (F - 1) of the bundles
    int nb;     // unknowns per frame of the factorised system (6, or 8 with the brightness pair)
};

__device__ __forceinline__ BundleDesc bundle_at(const BundleSet& s, int b)
{
    return s.bund ? s.bund[b] : s.one;
}

// linear algebra (pba_linalg.cu)
struct SolveArgs {
    int F, n6;              // total frames; largest 6 (F_b - 1) of the bundles
    int B, Fmax;            // bundles; largest frame count of a bundle
    const BundleDesc* bund;        // B bundles (device)
    const int* frame_bundle;       // F bundle of each global frame
    const int* pat;
    int P;
    double fx, fy, inv_fx, inv_fy;
    double* poses64;        // F*12 current
    const double* poses0;   // F*12 p_0
    double* dtheta64;       // F*6
    float2* dth2;           // F*6 (hi, lo) pairs
    float* fc;              // F*kFrameConst
    float* fc_prev;         // F*12
    float* dthsq;           // F
    int* err;
    const int* active;      // per bundle at fo: [0] anchor frame, [f] frame has residuals
    const int* cmap;        // per bundle at co: [f] compact index of an active frame or -1,
                            // [F_b] their number
    const double* tanchor;  // F*12 poses whose t define the gauge direction
    const double* photo_sums;  // F*5 brightness fit sums of the step (null: model off)
    // joint brightness unknowns (IC): the last increments (da, db) per frame
    // (composed into the pairs by the pose-update CTAs of the next depth
    // update), the frame sums H_pa / H_aa and the prior weight
    double* dab64;          // F*2
    float2* dab2;           // F*2 (hi, lo) pairs
    const double* red_aff;  // F*kAffComp
    double photo_prior;
};

// Affine brightness of frame f from its fit sums (w, w v, w v^2, w I_0,
// w I_0^2): v takes the template's weighted mean and spread,
// alpha = sqrt(var(I_0) / var(v)), beta = mean(I_0) - alpha mean(v); the
// pair is kept without residuals or without spread (FP64).
__device__ inline void photo_update_frame(const double* s, float* fc_f)
{
    if (!(s[0] > 0.0)) return;
    const double mv = s[1] / s[0], m0 = s[3] / s[0];
    const double vv = s[2] / s[0] - mv * mv, v0 = s[4] / s[0] - m0 * m0;
    if (!(vv > 1e-12) || !(v0 > 1e-12)) return;
    const double alpha = sqrt(v0 / vv);
    fc_f[kFrameAlpha] = (float)alpha;
    fc_f[kFrameAlpha + 1] = (float)(m0 - alpha * mv);
}

// depth back-substitution (when apply) of the last update and, in extra
// CTAs, every frame's pose update with it (a.active / tanchor unused)
cudaError_t launch_depth_update(const LaunchCtx& L, const SolveArgs& a, bool ic_rule, int apply);
// FP32 constants and previous R|t of frames [f0, f0 + nf) from a.poses64;
// init_photo also resets their brightness pairs to (1, 0)
cudaError_t launch_frame_consts(const SolveArgs& a, int f0, int nf, cudaStream_t st, int init_photo = 0);
cudaError_t launch_ic_point(const LaunchCtx& L, bool accum);
cudaError_t launch_fc_point(const LaunchCtx& L, bool accum);
// Dtheta = -S^-1 y (per bundle the compact S^-1 at so, y per global frame as
// written by the frame reduction), the gauge constraint and every frame's update
cudaError_t launch_ic_solve(const SolveArgs& a, const dfloat* Sinv, const double* y, cudaStream_t st);

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
constexpr int kSchurChunk = 32;
// tile_todo (nullable): form only the chunks with an item of a flagged tile
// and keep the other chunks' sums in part
cudaError_t launch_schur_sparse(const DevProblem& pb, const float* Hfd, const float* Hnn,
                                const SchurLists& sl, float2* part, double* Soff,
                                cudaStream_t st, int* launches, const unsigned char* tile_todo = nullptr);

// Schur complement on the tensor cores (pba_schur_tc.cu). Tiles are grouped
// into super-tiles of kStTiles consecutive tiles of one bundle (K = 128
// points); a super-tile's rows are 6 per frame that any of its tiles sees.
constexpr int kStTiles = 4;
constexpr int kSchurTcM = 128;  // rows of an output block (tensor-memory lanes)
constexpr int kSchurTcN = 80;   // columns of an output block
struct StRow {
    int f;               // global frame
    int e[kStTiles];     // the frame's entry in each tile of the super-tile (-1: none)
};
struct SchurTcLists {
    const int4* st;      // per super-tile: (first row, frames, first tile, tiles)
    const StRow* rows;   // the super-tiles' frames, in frame order within a super-tile
    const int4* items;   // output blocks: (super-tile, 128-row block, 80-column block, 0)
    short* ea;           // 6 per row: exponent bounding |H_fd| over the super-tile's points
    short* eb;           // 6 per row: the same for |H_fd / H_dd|
    long long* acc;      // fixed-point sums of S_off (per bundle at so, n6 x n6); zero between formations
    int n_st, n_items;
};
// S_off[f][g] = sum_n H_fd(n,f) H_fd(n,g)^T / H_dd(n) for f <= g with the
// operands split into exact BF16 slices (tcgen05.mma), written like
// launch_schur_sparse. red: the frame sums whose first 21 components per
// frame (stride red_stride) are the packed H_ff blocks (their diagonals
// bound the fixed-point scale).
cudaError_t launch_schur_tc(const DevProblem& pb, const float* Hfd, const float* Hnn, const SchurTcLists& tl,
                            const SchurLists& sl, const double* red, int red_stride, double* Soff, int* err,
                            cudaStream_t st, int* launches);
// once per process and device, before any capture
cudaError_t schur_tc_setup();
// Per bundle (arrays at the bundle's offsets; Hff, anchor_t, rhs and active
// indexed by global frame): S (FP64) and, when S2 is given, its double-float
// copy over the active frames only (compact order, cmap[f] = compact index
// or -1, cmap[F_b] = their number; the factorisation's working matrix; with
// rhs, one extra row b = -y taken from rhs[f * rhs_stride + rhs_off + a])
cudaError_t launch_assemble_S(const BundleSet& bs, const double* Hff, int hff_stride, const double* Soff,
                              const double* anchor_t, double gauge_w, double damping, double* S, int* active,
                              cudaStream_t st, dfloat* S2 = nullptr, int* cmap = nullptr,
                              const double* rhs = nullptr, int rhs_stride = 0, int rhs_off = 0);
// double-float LDL^T (pba_chol.cu), one thread-block cluster per bundle:
// A ((n + aug) x n, consumed) -> L (unit lower with L^T in the upper
// triangle; with aug, row n = D^-1 L^-1 b), Linv (inverses of the 32 x 32
// diagonal blocks and their transposes), dpiv = d_j, rpiv = 1 / d_j.
// The order n = 6 * cmap[F_b] is read on the device (the active frames).
// cluster: CTAs per bundle (0: the default chosen by ldl_setup)
cudaError_t launch_ldl(const BundleSet& bs, dfloat* A, dfloat* L, dfloat* Linv, dfloat* dpiv, dfloat* rpiv,
                       const int* cmap, int aug, int* err, cudaStream_t st, int cluster = 0);
// once per process and device, before any capture: cluster size of the
// factorisation, shared-memory limits of the solves
cudaError_t ldl_setup();
cudaError_t iter_setup();
cudaError_t linalg_setup();
int ldl_max_cluster();    // the largest cluster size ldl_setup found usable (8 or 16)
// S^-1 over the active frames (compact nc x nc, nc = 6 cmap[F_b]) per bundle
cudaError_t launch_ldl_inverse(const BundleSet& bs, const dfloat* L, const dfloat* Linv, const dfloat* rpiv,
                               const int* cmap, dfloat* Sinv, cudaStream_t st);
// Joint brightness unknowns (pba_affine.cu; IC, one bundle). Sums over the
// points of H_fd(n,f) H_a(n,g)^T / H_dd(n) (6 x 2 per frame pair, S_pa) and
// H_a(n,f) H_a(n,g)^T / H_dd(n) (2 x 2, S_aa) as fixed-point integers (acc:
// n6 * n2 then n2 * n2, zero on entry); the scale comes from the frame
// sums (red_ic: 21 per frame, red_aff: 15 per frame).
cudaError_t launch_affine_schur(const DevProblem& pb, const float* Hfd, const float* Had, const float* Hnn,
                                const double* red_ff, int ff_stride, const double* red_aff, long long* acc,
                                int F, cudaStream_t st);
// The factorisation's working matrix of the 8 (F - 1) system over the
// active frames, poses first (6 per active frame, the order of S) then the
// pairs (2 per active frame): S (FP64, assembled), H_pa and H_aa from
// red_aff, minus the fixed-point sums of launch_affine_schur.
cudaError_t launch_assemble_affine(const double* S, const double* red_ff, int ff_stride, const double* red_aff,
                                   const long long* acc, const int* cmap, int F, double damping, double prior,
                                   dfloat* A8, cudaStream_t st, const double* rhs = nullptr, int rhs_stride = 0,
                                   int rhs_off = 0, const double* yph = nullptr);
// FC with the pairs as unknowns: the backward substitution of the factorised
// 8 (F - 1) system (its augmented row), the gauge constraint on the
// translations, every frame's pose update and (da, db) (one CTA)
cudaError_t launch_fc_solve_affine(const SolveArgs& a, const dfloat* L8, const dfloat* Linv8, cudaStream_t st);
// Delta = -S8^-1 [y_theta; y_a] per target frame (y_a from the brightness
// columns of the frame reduction and the prior), the gauge constraint on the
// translations, the pose update written like launch_ic_solve and (da, db)
cudaError_t launch_ic_solve_affine(const SolveArgs& a, const dfloat* Sinv8, const double* y,
                                   const double* yph, cudaStream_t st);
// once per process and device, before any capture
cudaError_t affine_setup();

// one CTA per bundle
cudaError_t launch_fc_solve_update(const SolveArgs& a, const dfloat* L, const dfloat* Linv,
                                   cudaStream_t st);

// setup kernels (pba_runtime.cu); tile_f0[t] = reference frame of tile t
cudaError_t launch_setup(const DevProblem& pb, const int* tile_f0, float* gx, float* gy, float* I0p,
                         float2* G0p, cudaStream_t st);

}  // namespace pba
