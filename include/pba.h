/*
 * pba.h — C ABI of the GB300 (sm_103a) photometric bundle adjustment library.
 *
 * Inverse compositional photometric bundle adjustment with proxy templates
 * (IC) and the forwards compositional form (FC) beside it, after Ham, Lucey
 * and Singh, "Proxy Templates for Inverse Compositional Photometric Bundle
 * Adjustment", ICCV 2017 (arXiv 1704.06967).
 *
 * Model (Sec. 3, Eq. energy and Eq. warp). Frame 0 is the reference (template)
 * with the identity pose. Every point n has an integer pixel u_n in frame 0,
 * one inverse depth d_n shared by its P pattern pixels u_n + o_j, and a
 * visibility flag per target frame f = 1..F-1. With normalised coordinates
 * x = ((u - c_x)/f_x, (v - c_y)/f_y) the warp is W(x; p_fn) = <R_f x~ + d_n t_f>
 * and each residual is r = I_0(x) - I_f(W(x; p_fn)), sampled bilinearly.
 * The energy is the Huber norm of the residuals over (point, pattern pixel,
 * target frame).
 *
 * Poses are 12 doubles per frame, row-major [R | t] with R the 3x3 rotation
 * (row-major, 9 values) followed by t (3 values), mapping reference-frame
 * points X to frame-f points R X + t. Frame 0 must be the identity.
 * Inverse depths are doubles. All arrays passed from the host use the
 * caller's point order; the library reorders internally and maps back.
 *
 * Memory. The library allocates no device memory. The caller asks for the
 * workspace size (pba_workspace_size) once frames and points are set and
 * hands over one device buffer (pba_set_workspace) that must outlive the
 * context or the next pba_set_workspace. Device images passed with
 * PBA_MEM_DEVICE are borrowed and must outlive the context; host images
 * (PBA_MEM_HOST) are copied into the workspace by pba_set_workspace. All
 * device work is enqueued on the configured CUDA stream; a call returns
 * before its kernels finish unless it returns data to the host (statistics,
 * parameters, updates, systems), in which case it synchronises that stream.
 *
 * Errors. Every call returns a pba_status; no exception or exit crosses the
 * ABI. On failure pba_last_error() describes it. Kernels never trap; they set
 * a device error word that the next synchronising call reports
 * (PBA_ERR_NOT_PD for a non-positive pivot of the reduced camera system,
 * PBA_ERR_NONFINITE for a non-finite update). A context is not thread safe;
 * distinct contexts are independent.
 */
#ifndef PBA_H
#define PBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PBA_MAX_PATTERN 16
#define PBA_MAX_BUNDLES 65535

typedef struct pba_ctx pba_ctx;

typedef enum {
    PBA_OK = 0,
    PBA_ERR_ARG = 1,        /* invalid argument (null pointer, size, range) */
    PBA_ERR_STATE = 2,      /* call out of order (e.g. iterate before precompute) */
    PBA_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    PBA_ERR_NOMEM = 4,      /* workspace too small / host allocation failed */
    PBA_ERR_NOT_PD = 5,     /* reduced camera system not positive definite */
    PBA_ERR_NONFINITE = 6,  /* non-finite update or statistic */
    PBA_ERR_TIMEOUT = 7,    /* a bounded device wait gave up */
    PBA_ERR_TOO_LARGE = 8   /* problem exceeds a fixed capacity (no-allocation entry point) */
} pba_status;

typedef enum { PBA_F32 = 0, PBA_F16 = 1, PBA_BF16 = 2 } pba_dtype;

typedef enum { PBA_MEM_DEVICE = 0, PBA_MEM_HOST = 1 } pba_memory;

typedef struct {
    double huber_k;          /* Huber constant k of ||.||_gamma (Eq. energy); > 0 */
    int pattern_size;        /* P, 1..PBA_MAX_PATTERN */
    const int32_t* pattern;  /* host, P*2 pixel offsets (dx, dy), copied at create */
    double gauge_anchor_w;   /* scale-gauge prior weight relative to mean diag(S); 0 -> 1 */
    double conv_px;          /* convergence threshold of Sec. 4.1 in pixels; 0 -> 5e-3 */
    int n_bundles;           /* independent bundles solved together, 1..PBA_MAX_BUNDLES
                                (0 -> 1). Their frames, points and residuals are
                                concatenated, so every kernel of an iteration runs over
                                all bundles in one launch; each bundle keeps its own
                                reference frame, gauge and reduced camera system
                                (factored by its own thread-block cluster). The bundles
                                share the camera: image size, pitch, element type, memory
                                kind and intrinsics. Statistics are summed over them. */
    void* cuda_stream;       /* cudaStream_t for all work; NULL = legacy default stream */
    int use_graphs;          /* non-zero (and cuda_stream non-NULL): pba_precompute_ic,
                                pba_iterate and pba_solve_fc submit their kernels by
                                replaying a CUDA graph captured on the first call with
                                the same iteration count and timing mask (one
                                cudaGraphLaunch per call instead of one launch per
                                kernel); the graphs hold workspace pointers and are
                                dropped by pba_set_workspace. Ignored with a NULL
                                stream (the legacy stream cannot be captured). */
    int max_stats_iters;     /* capacity of the per-iteration statistics; 0 -> 256 */
    int autotune;            /* non-zero: the first pba_precompute_ic times the candidate
                                launch shapes on this problem and keeps the fastest: warps
                                per CTA of the IC residual pass (4, 8, 16: the number of
                                (tile, frame) entries a CTA takes) and CTAs per bundle of
                                the cluster that factors the reduced camera system (1, 2,
                                4, 8, 16); a candidate replaces the current shape only when
                                more than 3 % faster. Results do not depend on the choice
                                (every sum keeps its order); see pba_get_tuning /
                                pba_set_tuning. */
    double damping;          /* Levenberg-Marquardt lambda >= 0; 0 = Gauss-Newton as in the
                                paper (Sec. 3.5). lambda > 0 scales every diagonal entry of
                                the frame blocks H_ff and of H_dd by 1 + lambda in the
                                solve (IC: in the system fixed at p_0; FC: every
                                iteration), replaces the scale-gauge prior (the damped
                                system is definite) and keeps the exact gauge constraint
                                t_a . Delta t_a = 0. pba_get_system returns the undamped
                                blocks and the S that was factorised. */
    int photometric;         /* affine brightness per target frame (an option beyond the
                                paper, whose Sec. 2 notes that direct methods must model
                                lighting): residual r = I_0 - (alpha_f I_f + beta_f),
                                pairs starting at (1, 0); see pba_get_brightness.
                                1: after every IC/FC step each frame's pair is set from
                                that step's residuals so that the warped samples take the
                                template's Huber-weighted mean and spread (alpha =
                                sqrt(var I_0 / var v), beta = mean I_0 - alpha mean v).
                                2: the pairs are unknowns of the Gauss-Newton system
                                (8 x 8 frame blocks, an 8 (F - 1) reduced system). IC: the
                                template-side increment (1 + da) I_0 + db adds the fixed
                                columns I_0 and 1, formed and inverted once at p_0 with
                                the rest of the IC system (Sec. 3.5), and a step composes
                                alpha' = alpha / (1 + da), beta' = (beta - db) / (1 +
                                da). FC: the columns -I_f and -1 at the current
                                parameters, every iteration, and (alpha, beta) += (da,
                                db). One bundle per context (pba_set_window and the
                                sharded steps return PBA_ERR_ARG). Other values:
                                PBA_ERR_ARG. */
    double photo_prior;      /* photometric = 2, IC: weight lambda >= 0 of a prior that pulls
                                the pairs toward (1, 0), lambda W_f ((ln alpha_f)^2 +
                                beta_f^2) / 2 with W_f the sum of the frame's Huber
                                weights at p_0 (fixed with the IC system: lambda W_f on
                                the pair's diagonal, its gradient at the current pair
                                every step). The template-side pairs are exact at zero
                                residual but, far from alignment, move toward
                                var(I_0) / cov(I_0, I_f) and can drift; 0.01 keeps them
                                bounded. 0: no prior. Negative or non-finite:
                                PBA_ERR_ARG. */
} pba_config;

/* Statistics of one iteration (Sec. 4.1): Huber energy, RMS and count of the
 * residuals valid at the iteration's parameters, the largest pattern-centre
 * reprojection displacement of the step (pixels), and the norms of the update. */
typedef struct {
    double energy;
    double rms;
    double n_valid;
    double max_disp_px;
    double dtheta_norm;
    double dd_norm;
} pba_iter_stats;

/* Creates a context. cfg and cfg->pattern are copied. */
pba_status pba_create(const pba_config* cfg, pba_ctx** out);

/* Destroys a context (synchronises its stream; NULL is a no-op). */
void pba_destroy(pba_ctx* ctx);

/* Text of the last error of this context (never NULL; valid until the next call). */
const char* pba_last_error(const pba_ctx* ctx);

/* Sets the images, the initial poses p_0 and the pinhole intrinsics.
 * images: F frames of height h, row pitch pitch_elems >= w elements of dtype,
 *   frame-major (frame f at images + f*h*pitch_elems elements); frame 0 is the
 *   template I_0. Device pointer (borrowed) or host pointer (copied by
 *   pba_set_workspace) according to mem.
 * poses: host, F*12 doubles (p_0), frame 0 = identity. Copied.
 * intrinsics: host, {f_x, f_y, c_x, c_y}. Copied.
 * Requires 0 <= bundle < n_bundles, 2 <= F <= 1024, w, h >= 4, and (all
 * bundles together) fewer than 2^32 image elements; the camera (w, h,
 * pitch_elems, dtype, mem, intrinsics) must equal that of the other bundles
 * already set. Invalidates the precompute and the workspace layout. */
pba_status pba_set_frames(pba_ctx* ctx, int bundle, int n_frames, int w, int h, int pitch_elems,
                          pba_dtype dtype, pba_memory mem, const void* images,
                          const double* poses, const double* intrinsics);

/* Sets the points (Sec. 3: one inverse depth per point in the reference frame).
 * uv: host, N*2 int32 pixel centres in frame 0; every pattern pixel and its
 *   central-difference neighbours must lie inside frame 0.
 * inv_depth: host, N doubles (d_0), > 0.
 * vis: host, N*F bytes (vis[n*F + f] != 0: point n observed in frame f;
 *   column 0 ignored), or NULL for all visible. Copied.
 * Invalidates the precompute and the workspace layout. */
pba_status pba_set_points(pba_ctx* ctx, int bundle, int n_points, const int32_t* uv,
                          const double* inv_depth, const uint8_t* vis);

/* Device workspace bytes needed for the current frames and points. */
pba_status pba_workspace_size(pba_ctx* ctx, size_t* bytes);

/* Hands over the device workspace (>= pba_workspace_size bytes, 256-byte
 * aligned) and uploads frames, points and parameters into it. */
pba_status pba_set_workspace(pba_ctx* ctx, void* dev_ptr, size_t bytes);

/* IC precompute at the current parameters, which become p_0 (Sec. 3.5):
 * per residual the proxy-template Jacobian row J = grad I_0 dphi/dDelta p
 * (Sec. 3.4), initial residual and Huber weight W_0; H = J^T W_0 J in frame,
 * frame-point and point blocks; the Schur complement S of the point block
 * with the scale-gauge prior, its LDL^T factor (double-float arithmetic,
 * ~48 bits, over the frames that have residuals) and inverse.
 * PBA_ERR_NOT_PD: the system of a bundle (pba_bundle_errors says which) had
 * a non-positive pivot, replaced by 1; the precompute still counts as done,
 * so the other bundles of a batch can iterate. */
pba_status pba_precompute_ic(pba_ctx* ctx);

/* Sliding window over a bundle's frames (the dynamic Hessian the paper
 * suggests for windows of keyframes, Sec. 4.2). in_window: host, F_b flags
 * (frame 0 ignored: the reference is always in). Frames outside the window
 * keep their images, poses and stored products, but none of their residuals
 * enters any sum (IC, FC, statistics). After a change pba_iterate needs
 * pba_update_ic (PBA_ERR_STATE otherwise); pba_solve_ic and pba_solve_fc
 * work on the window as it is. All frames are in the window initially. */
pba_status pba_set_window(pba_ctx* ctx, int bundle, const uint8_t* in_window);

/* Brings the IC system up to date with the window without a full
 * precompute: the Jacobian rows and H products of the entering frames are
 * formed (anchored at their current poses; every point keeps its d_0),
 * those of the frames already in are reused from the workspace, H_dd and
 * the frame blocks are formed again from the stored products, the sums of
 * the Schur complement are formed again only for the points of tiles that
 * see a frame that entered or left (the rest are kept), and S, its factor
 * and S^-1 follow. The result equals a full pba_precompute_ic whose p_0
 * holds the same anchors, bit for bit. Before any precompute it runs the
 * full one. */
pba_status pba_update_ic(pba_ctx* ctx);

/* Runs n_iters IC iterations (Sec. 3.5 steps 1-4 with the Sec. 3.6 update):
 * Huber weights from the current residuals, g = J^T W r, Delta p = -H^-1 g by
 * the Schur complement, then R <- R R0^T exp(omega)^T R0, t <- t - R R0^T Dt,
 * d <- d (d0 - Dd)/d0. stats (host, nullable): n_iters+1 entries, entry k for
 * the parameters p_k (the last one has no update). PBA_ERR_STATE before
 * pba_precompute_ic. */
pba_status pba_iterate(pba_ctx* ctx, int n_iters, pba_iter_stats* stats);

/* A whole IC solve in one call: the precompute at the current parameters,
 * then n_iters IC iterations (as pba_iterate) with re-anchoring: after every
 * reanchor_every iterations (0: never) the parameters reached become the new
 * p_0 and J, W_0, H, S and S^-1 are formed there again (the precompute of
 * Sec. 3.5 at the new linearisation point; an option beyond the paper, for
 * bundles where the Hessian fixed at the first p_0 stops describing the
 * problem). With reanchor_every = 0 the result equals pba_precompute_ic +
 * pba_iterate bit for bit. stats as for pba_iterate. Replayed from one CUDA
 * graph per (n_iters, reanchor_every, timing mask) under cfg.use_graphs. */
pba_status pba_solve_ic(pba_ctx* ctx, int n_iters, int reanchor_every, pba_iter_stats* stats);

/* Runs n_iters FC iterations: Jacobians from the target-image gradients, the
 * Hessian blocks, the Schur complement and its LDL^T factor (double-float)
 * rebuilt every iteration, then T <- exp([upsilon, omega]) T, d <- d + Dd (Sec. 3,
 * the boxplus operator). stats as for pba_iterate. Needs no precompute. */
pba_status pba_solve_fc(pba_ctx* ctx, int n_iters, pba_iter_stats* stats);

/* Current parameters: poses F*12 doubles, inv_depth N doubles (host, nullable each). */
pba_status pba_get_params(pba_ctx* ctx, int bundle, double* poses, double* inv_depth);

/* Replaces the current parameters (not p_0; the IC precompute is kept). */
pba_status pba_set_params(pba_ctx* ctx, int bundle, const double* poses, const double* inv_depth);

/* Update of the last iteration: dtheta F*6 doubles ([Dt, omega] for IC,
 * [upsilon, omega] for FC; frame 0 zero), dd N doubles (host, nullable each). */
pba_status pba_get_last_update(pba_ctx* ctx, int bundle, double* dtheta, double* dd);

/* The last linear system: Hff F*36 (row-major 6x6 per frame, frame 0 zero),
 * Hfd N*F*6 (caller point order), Hdd N, and S (6(F-1))^2 row-major as
 * factorised (with the gauge prior). fc != 0 selects the last FC system.
 * Host arrays, nullable each. With the brightness pairs as unknowns
 * (photometric = 2) these are the pose blocks of the 8-per-frame system;
 * its brightness border is not returned. */
pba_status pba_get_system(pba_ctx* ctx, int bundle, int fc, double* Hff, double* Hfd,
                          double* Hdd, double* S);

/* Residual count of the bundle (visible (point, frame) pairs times P). */
pba_status pba_num_residuals(pba_ctx* ctx, int bundle, int64_t* n);

/* Kernel timing. pba_enable_timing(ctx, mask) records a CUDA event pair on
 * the context's stream around every kernel launch of the slots whose bit is
 * set in mask (-1: all slots, 0: none) and resets the counters.
 * pba_last_timing synchronises the stream and fills out[2 * PBA_TIMING_SLOTS
 * + 1]: out[s] = accumulated device ms of slot s, out[PBA_TIMING_SLOTS] =
 * kernel launches since the reset (counted whether or not timing is on),
 * out[PBA_TIMING_SLOTS + 1 + s] = timed launches of slot s. Slots: 0 setup /
 * IC precompute, 1 residual pass (the kernel that samples the images), 2
 * per-frame reduction, 3 Schur complement + assembly (FC), 4 factorisation /
 * solve / pose update, 5 final evaluation, 6 per-point kernels of the
 * iteration (depth back-substitution, point sums and Schur right-hand side). */
#define PBA_TIMING_SLOTS 7
pba_status pba_enable_timing(pba_ctx* ctx, int mask);
pba_status pba_last_timing(pba_ctx* ctx, double* out);

/* Per-bundle device errors seen by the last call that synchronised (bit 0:
 * reduced camera system not positive definite, bit 1: non-finite update).
 * When a call returns PBA_ERR_NOT_PD or PBA_ERR_NONFINITE, the bundles whose
 * flags are 0 were solved normally (bundles never share a sum). flags: host,
 * n_bundles ints. */
pba_status pba_bundle_errors(pba_ctx* ctx, int* flags);

/* Affine brightness pairs of a bundle's frames: ab host, F_b x 2 doubles
 * (alpha_f, beta_f; frame 0 is (1, 0)), stored as FP32 on the device. They
 * are used in every residual (an identity pair changes nothing) and fitted
 * (photometric = 1) or solved for (photometric = 2) by the steps when
 * cfg.photometric is set. With photometric = 2 a step's pair update is
 * applied with its pose update (at the next iteration's start or at the end
 * of the call), so the pairs read after a call belong to its final
 * parameters. */
pba_status pba_get_brightness(pba_ctx* ctx, int bundle, double* ab);
pba_status pba_set_brightness(pba_ctx* ctx, int bundle, const double* ab);

/* Launch shapes in use (after autotuning, or the defaults 8 and the largest
 * cluster the device co-schedules): res_warps = warps per CTA of the IC
 * residual pass, ldl_cluster = CTAs per bundle of the factorisation. Host,
 * nullable each. */
pba_status pba_get_tuning(pba_ctx* ctx, int* res_warps, int* ldl_cluster);

/* Sets the launch shapes (e.g. those pba_get_tuning returned for another
 * context of the same shape, so that a fresh context need not autotune):
 * res_warps in {4, 8, 16}; ldl_cluster a power of two from 1 to the largest
 * cluster the device co-schedules (16, else 8). Results do not depend on
 * them. PBA_ERR_ARG for other values (nothing changes). The captured graphs
 * are discarded, and a context with cfg.autotune keeps these shapes (its
 * first precompute times no candidates). Needs the CUDA device. */
pba_status pba_set_tuning(pba_ctx* ctx, int res_warps, int ldl_cluster);

/* ------------------------------------------------------------------------
 * Point sharding of one bundle across processes, one GPU each. Every rank
 * creates a context of the whole bundle's frames, images and poses with its
 * own share of the points (n_bundles = 1, cfg.photometric = 0). A point's
 * residuals, H_fd, H_dd, g_d and depth update never leave its rank; the
 * quantities that couple the points are sums over points (Sec. 3.5: the
 * H_ff blocks, S_off = H_pd H_dd^-1 H_dp and the right-hand side
 * g_theta - H_pd H_dd^-1 g_d), so each call below has two halves and the
 * caller sums the named buffers over the ranks in between (an all-reduce):
 *
 *   pba_shard_ic_precompute(ctx, 0)   J, W_0, H blocks at p_0 = the current
 *       parameters; fills PBA_SHARD_IC_FRAME_SUMS and PBA_SHARD_SOFF with
 *       this rank's sums.
 *   pba_shard_ic_precompute(ctx, 1)   S (with the gauge prior), its factor
 *       and S^-1 from the summed buffers (identical on every rank).
 *   pba_shard_ic_step(ctx, k, 0)      IC iteration k: (k > 0) the update of
 *       iteration k - 1 applied, J^T W r of this rank's residuals; fills
 *       PBA_SHARD_IC_RHS (frame sums of the Schur right-hand side).
 *   pba_shard_ic_step(ctx, k, 1)      the update from the summed right-hand
 *       side (identical frame updates on every rank).
 *   pba_shard_fc_step(ctx, k, 0)      FC iteration k: (k > 0) the last update
 *       applied, the linearisation of this rank's residuals; fills
 *       PBA_SHARD_FC_FRAME_SUMS (H_ff, g_theta and the Schur corrections per
 *       frame) and PBA_SHARD_SOFF.
 *   pba_shard_fc_step(ctx, k, 1)      S, its factorisation and the update.
 *   pba_shard_eval(ctx, fc, n)        after n iterations: the last update
 *       applied and the statistics of slot n (IC with fc = 0, FC with 1).
 *
 * k counts iterations from 0 (k <= cfg.max_stats_iters); the statistics of
 * iteration k land in slot k (pba_shard_stats). The buffers are FP64 device
 * arrays inside the workspace: pba_shard_count gives their length,
 * pba_shard_export copies one to a caller device array (dev_dst, count
 * doubles, on the context's stream) and pba_shard_import copies the summed
 * array back. Errors: PBA_ERR_ARG (several bundles, brightness model on,
 * bad half, k or buffer), PBA_ERR_STATE (no workspace, step before the
 * precompute), and the statuses of the solves. */
#define PBA_SHARD_IC_FRAME_SUMS 0  /* F x 21 packed H_ff blocks of the IC precompute */
#define PBA_SHARD_SOFF 1           /* (6 (F - 1))^2 S_off, both triangles */
#define PBA_SHARD_IC_RHS 2         /* F x 6 Schur right-hand side of an IC iteration */
#define PBA_SHARD_FC_FRAME_SUMS 3  /* F x 27: 21 packed H_ff, 6 right-hand side of an FC iteration */
pba_status pba_shard_ic_precompute(pba_ctx* ctx, int half);
pba_status pba_shard_ic_step(pba_ctx* ctx, int k, int half);
pba_status pba_shard_fc_step(pba_ctx* ctx, int k, int half);
pba_status pba_shard_eval(pba_ctx* ctx, int fc, int k);
pba_status pba_shard_count(pba_ctx* ctx, int which, int64_t* count);
pba_status pba_shard_export(pba_ctx* ctx, int which, double* dev_dst);
pba_status pba_shard_import(pba_ctx* ctx, int which, const double* dev_src);
/* Raw statistics of slots 0 .. n_slots - 1 of this rank's residuals, 6
 * doubles per slot: energy (sum of Huber rho), sum r^2, valid residual
 * count, largest pattern-centre displacement of the step (px), |Dtheta|^2
 * (the same on every rank), sum Dd^2. Sum over ranks, except the
 * displacement (max) and |Dtheta|^2 (any rank). raw: host. Synchronises. */
pba_status pba_shard_stats(pba_ctx* ctx, int n_slots, double* raw);

/* How the Schur complement S_off = H_pd H_dd^-1 H_dp of the reduced camera
 * system (Sec. 3.5 step 3) is formed, once per pba_precompute_ic and every
 * FC iteration:
 *  PBA_SCHUR_AUTO (default): the tensor cores when the bundle set has at
 *    least four of the tensor path's 128 x 80 output blocks per SM, else the
 *    SIMT products (the faster of the two on small bundles); the choice
 *    depends only on the problem's structure and the device's SM count.
 *  PBA_SCHUR_TENSOR: on the tensor cores (tcgen05.mma) over
 *    super-tiles of 128 points, with every H_fd row and every product
 *    H_fd / H_dd split exactly into BF16 digit slices whose FP32
 *    accumulation is exact; the sums are added as 64-bit fixed-point
 *    integers, so the result does not depend on the order of the work.
 *  PBA_SCHUR_SIMT: exact FP32 products (TwoProduct) with compensated sums on
 *    the SIMT pipes, over the co-visible (tile, frame pair) items.
 * Both form sum_n H_fd H_fd^T w_n of the FP32 blocks with the same FP32
 * w_n = 1 / (H_dd (1 + lambda)); they agree to ~1e-14 of the largest entry
 * and each is deterministic run to run. The captured graphs are discarded.
 * PBA_ERR_ARG for another value. */
#define PBA_SCHUR_TENSOR 0
#define PBA_SCHUR_SIMT 1
#define PBA_SCHUR_AUTO 2
pba_status pba_set_schur_path(pba_ctx* ctx, int path);

/* Bytes this context copied host->device and device->host since it was
 * created (uploads of images, points, structure and parameters; downloads of
 * statistics, parameters, updates and systems). Host, nullable each. */
pba_status pba_transfer_bytes(pba_ctx* ctx, int64_t* h2d, int64_t* d2h);

/* One level of an image pyramid (coarse-to-fine solving; an addition beyond
 * the paper): dst[f][y][x] = mean of src[f][2y .. 2y+1][2x .. 2x+1], FP32,
 * floor(w/2) x floor(h/2) per frame, rows of floor(w/2) elements. Pixel
 * centres map as x_coarse = (x_fine + 0.5) / 2 - 0.5, so a camera's
 * intrinsics become f / 2 and (c + 0.5) / 2 - 0.5. src: device, n_frames x h
 * rows of pitch_elems elements of dtype; dst: device. Enqueued on
 * cuda_stream (NULL = legacy default), not synchronised. */
pba_status pba_downsample(const void* src, pba_dtype dtype, int n_frames, int w, int h, int pitch_elems,
                          float* dst, void* cuda_stream);

/* Coarse-to-fine solve of one bundle over an image pyramid (an addition
 * beyond the paper: a direct method's basin widens at coarse levels). Level
 * l (0 = full resolution) halves the images l times (pba_downsample, FP32)
 * with intrinsics f / 2^l and (c + 0.5) / 2^l - 0.5. A point keeps its
 * inverse depth at every level and takes the nearest level pixel, (u + 0.5)
 * / 2^l - 0.5 rounded to nearest (ties to even); a point whose pattern (and
 * the pattern's central-difference neighbours) would leave a level's
 * reference image sits that level out. From the coarsest level to level 0,
 * a context of the level (cfg with one bundle) solves iters[i] iterations
 * (i = 0 for the coarsest), method 0 = IC (pba_solve_ic with
 * reanchor_every) or 1 = FC (pba_solve_fc); the poses and inverse depths it
 * reaches start the next level (a point driven to a non-positive or
 * non-finite inverse depth keeps the one it entered the level with).
 *
 * levels: 1..8, every level at least 4 x 4 pixels and with at least one
 * point. images: device, n_frames x h rows of pitch_elems elements of dtype.
 * poses (n_frames x 12, R row-major then t) and inv_depth (n_points): host,
 * in: the initial values, out: the result. intrinsics, uv (n_points x 2),
 * vis (n_points x n_frames, nullable = all visible): host, as for
 * pba_set_frames / pba_set_points. workspace: device, 256-byte aligned, at
 * least the size pba_pyramid_workspace_size gives for the same problem (the
 * coarser levels' images, then the region each level's context uses in
 * turn); its contents are scratch. stats: host, nullable, sum(iters[i] + 1)
 * entries, each level's pba_solve_ic / pba_solve_fc statistics in turn.
 * level_ms: host, nullable, `levels` entries (coarsest first): the device
 * time of each level's solve call (CUDA events on the stream around it; the
 * level's image reduction and context set-up excluded). Runs on
 * cfg->cuda_stream and returns when the result is on the host.
 * Errors: PBA_ERR_ARG (invalid arguments, cfg with several bundles, a level
 * too small or without points) and PBA_ERR_NOMEM (workspace smaller than
 * the size query's), both before anything is solved, and any status of a
 * level's calls (the solve stops at that level; poses and inv_depth then
 * hold the last completed level's result). */
pba_status pba_pyramid_workspace_size(const pba_config* cfg, int levels, int n_frames, int w, int h,
                                      const double* poses, const double* intrinsics, int n_points,
                                      const int32_t* uv, const double* inv_depth, const uint8_t* vis,
                                      size_t* bytes);
pba_status pba_solve_pyramid(const pba_config* cfg, int levels, const int* iters, int method, int reanchor_every,
                             const void* images, pba_dtype dtype, int n_frames, int w, int h, int pitch_elems,
                             double* poses, const double* intrinsics, int n_points, const int32_t* uv,
                             double* inv_depth, const uint8_t* vis, void* workspace, size_t ws_bytes,
                             pba_iter_stats* stats, double* level_ms);

/* Reduced camera system without any allocation, for callers that cannot
 * allocate device memory (code running inside a fixed pre-reserved memory
 * arena, runtimes that forbid cudaMalloc after start-up, frameworks that
 * hand an operation only its input and output tensors). The paper has no
 * counterpart: it is a deployment form of the Schur-complement step.
 *
 * Builds the anchored reduced camera system from dense Hessian blocks:
 *   S = blockdiag(Hff) - sum_n Hfd(n,.) Hfd(n,.)^T / Hdd(n)   (points with
 *   Hdd(n) <= 0 skipped), frames whose Hff has zero trace replaced by an
 *   identity block, and the scale-gauge prior gauge_anchor_w * mu * t t^T on
 *   the translation block of the first active frame (t = unit translation of
 *   that frame in poses, mu = mean diagonal of the active frames) -- the same
 *   system pba_get_system returns.
 * All pointers are device pointers, caller owned: Hff F*36 (row-major 6x6
 * per frame, frame 0 ignored), Hfd N*F*6 (zero where a point is not
 * observed), Hdd N, poses F*12 ([R|t] rows, only t is read), S output
 * (6(F-1))^2 row-major. gauge_anchor_w 0 means 1. Work is enqueued on
 * cuda_stream (NULL = legacy default stream) and not synchronised.
 * Scratch lives in one static device array sized for n_frames <=
 * PBA_NOALLOC_MAX_FRAMES (about 1.2 MB, held by every GPU that loads the
 * library until exit); larger problems return PBA_ERR_TOO_LARGE without
 * touching the GPU. The function calls no cudaMalloc/cudaFree. Its first
 * call in a CUDA context of a device looks up the array's device address in
 * that context (make that first call before any stream capture; a later
 * context on the device, e.g. after cudaDeviceReset, gets its own lookup on
 * its first call). Every call on a device shares the array:
 * calls that overlap on the GPU (concurrent streams) race and must be
 * serialised by the caller. Returns PBA_ERR_ARG for invalid arguments and
 * PBA_ERR_CUDA when a launch fails. */
#define PBA_NOALLOC_MAX_FRAMES 65
pba_status pba_reduced_system_noalloc(int n_frames, int n_points, const double* Hff,
                                      const double* Hfd, const double* Hdd, const double* poses,
                                      double gauge_anchor_w, double* S, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PBA_H */
