// Reduced camera system (Sec. 3.5 step 3): assembly of S with the
// scale-gauge prior, the IC solve (explicit FP64 S^-1 applied as a GEMV, the
// factorisation being done once), the FC solve (substitutions with the FP64
// Cholesky factor, every iteration), and the FP64 pose updates of Sec. 3.6
// (IC) and of the boxplus operator (FC).
#include <algorithm>

#include "pba_chol.cuh"

namespace pba {

// ---------------------------------------------------------------------------
// S = blockdiag(H_ff) - S_off, then: frames without residuals (zero H_ff
// trace) get an identity block; mu = mean diagonal over the active frames;
// the prior gauge_w * mu * that that^T goes on the translation block of the
// first active frame (that = unit translation of that frame in anchor_t).
// H_ff comes as 21 upper-triangle values per frame at Hff[f*stride].
// active[f] (f >= 1) receives the frame flags, active[0] the anchor frame;
// cmap[f] the compact index of an active frame (-1 otherwise) and cmap[F]
// their number.
// Every CTA recomputes the flags, mu and the anchor (a few hundred FP64
// operations) and fills its share of S.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int upper_index(int a, int b)
{
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
    return a * 6 - a * (a - 1) / 2 + (b - a);
}

constexpr int kAssembleThreads = 256;

__global__ void __launch_bounds__(kAssembleThreads)
assemble_S_kernel(int F, const double* Hff, int stride, const double* Soff,
                  const double* anchor_t, double gauge_w, double* S, int* active, dfloat* S2,
                  int* cmap, const double* rhs, int rhs_stride, int rhs_off)
{
    __shared__ int s_act[1024];
    __shared__ int s_cidx[1024];  // compact index of an active frame
    __shared__ int s_nact;
    __shared__ double s_red[kAssembleThreads / 32];
    __shared__ int s_anchor;
    __shared__ double s_mu;
    const int n6 = 6 * (F - 1), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int f = 1 + tid; f < F; f += blockDim.x) {
        const double* h = Hff + (size_t)f * stride;
        double tr = 0.0;
        for (int a = 0; a < 6; ++a) tr += h[upper_index(a, a)];
        s_act[f] = tr > 0.0;
    }
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < n6; i += blockDim.x) {
        const int f = i / 6 + 1;
        if (s_act[f]) part += Hff[(size_t)f * stride + upper_index(i % 6, i % 6)] - Soff[(size_t)i * n6 + i];
    }
    part = warp_sum1d(part);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    if (tid == 0) {
        double mu = 0.0;
        for (int w = 0; w < kAssembleThreads / 32; ++w) mu += s_red[w];
        int cnt = 0, anchor = -1;
        for (int f = 1; f < F; ++f) {
            s_cidx[f] = s_act[f] ? cnt / 6 : -1;
            if (!s_act[f]) continue;
            if (anchor < 0) anchor = f;
            cnt += 6;
        }
        s_mu = cnt ? gauge_w * mu / cnt : 0.0;
        s_anchor = anchor;
        s_nact = cnt / 6;
        if (blockIdx.x == 0) {
            active[0] = anchor;
            for (int f = 1; f < F; ++f) active[f] = s_act[f];
            if (cmap) {
                for (int f = 1; f < F; ++f) cmap[f] = s_cidx[f];
                cmap[0] = -1;
                cmap[F] = s_nact;
            }
        }
    }
    __syncthreads();
    const int anchor = s_anchor;
    double th[3] = {0.0, 0.0, 0.0};
    if (anchor > 0) {
        const double* ta = anchor_t + 12 * anchor + 9;
        const double nt = sqrt(ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2]);
        if (nt > 0.0)
            for (int a = 0; a < 3; ++a) th[a] = ta[a] / nt;
    }
    const size_t total = (size_t)n6 * n6;
    const int nc = 6 * s_nact;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + tid; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n6), j = (int)(idx % n6);
        const int fi = i / 6 + 1, fj = j / 6 + 1;
        double v;
        if (!s_act[fi] || !s_act[fj]) {
            v = (i == j) ? 1.0 : 0.0;
        } else {
            v = -Soff[idx];
            if (fi == fj) {
                v += Hff[(size_t)fi * stride + upper_index(i % 6, j % 6)];
                const int a = i % 6, b = j % 6;
                if (fi == anchor && a < 3 && b < 3) v += s_mu * (th[a] * th[b]);
            }
        }
        S[idx] = v;
        // the double-float working copy holds the active frames only
        // (compact order, row stride nc): frames without residuals have
        // identity blocks and a zero update, so they are left out of the
        // factorisation
        if (S2 && s_act[fi] && s_act[fj])
            S2[(size_t)(6 * s_cidx[fi] + i % 6) * nc + 6 * s_cidx[fj] + j % 6] = df_from_double(v);
    }
    // augmented row nc of the double-float copy: b = -y, eliminated with the
    // matrix by the factorisation
    if (S2 && rhs)
        for (int j = blockIdx.x * blockDim.x + tid; j < n6; j += gridDim.x * blockDim.x) {
            const int f = j / 6 + 1;
            if (s_act[f])
                S2[(size_t)nc * nc + 6 * s_cidx[f] + j % 6] =
                    df_from_double(-rhs[(size_t)f * rhs_stride + rhs_off + j % 6]);
        }
}

cudaError_t launch_assemble_S(int F, const double* Hff, int hff_stride, const double* Soff,
                              const double* anchor_t, double gauge_w, double* S, int* active,
                              cudaStream_t st, dfloat* S2, int* cmap, const double* rhs,
                              int rhs_stride, int rhs_off)
{
    if (S2 && !cmap) return cudaErrorInvalidValue;
    const int n6 = 6 * (F - 1);
    if (F > 1024) return cudaErrorInvalidValue;
    const int blocks = std::max(1, std::min(148, (n6 * n6 + 4 * kAssembleThreads - 1) / (4 * kAssembleThreads)));
    assemble_S_kernel<<<blocks, kAssembleThreads, 0, st>>>(F, Hff, hff_stride, Soff, anchor_t,
                                                            gauge_w, S, active, S2, cmap, rhs,
                                                            rhs_stride, rhs_off);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pose updates (FP64). GB300 issues an FP64 warp instruction at a small
// fraction of the FP32 rate whatever the number of active lanes, so the 3x3
// products are spread over lanes of one warp instead of one thread.
// ---------------------------------------------------------------------------
// C = A B for 3x3 matrices in shared memory; lanes 0..8 each one entry.
__device__ __forceinline__ void mat3_mul_lanes(const double* A, const double* B, double* C, int lane)
{
    if (lane < 9) {
        const int i = lane / 3, j = lane % 3;
        C[lane] = fma(A[3 * i], B[j], fma(A[3 * i + 1], B[3 + j], A[3 * i + 2] * B[6 + j]));
    }
    __syncwarp();
}

// Writes the new pose of frame f (lanes of one warp; Rn, tn in shared
// memory), its FP32 pass constants, the previous R|t and the update.
__device__ void write_frame_lanes(const SolveArgs& a, int f, const double* pose_old, const double* Rn,
                                  const double* tn, const double* dth, int lane)
{
    double* pose = a.poses64 + 12 * f;
    float* prev = a.fc_prev + 12 * f;
    if (lane < 12) prev[lane] = (float)pose_old[lane];
    __syncwarp();
    if (lane < 9) pose[lane] = Rn[lane];
    if (lane < 3) pose[9 + lane] = tn[lane];
    __syncwarp();
    float* out = a.fc + (size_t)f * kFrameConst;
    if (lane < 12) out[lane] = (float)(lane < 9 ? Rn[lane] : tn[lane - 9]);
    for (int q = lane; q < 3 * a.P; q += 32) {
        const int j = q / 3, r = q % 3;
        const double ox = a.pat[2 * j] * a.inv_fx, oy = a.pat[2 * j + 1] * a.inv_fy;
        out[12 + q] = (float)(ox * Rn[3 * r] + oy * Rn[3 * r + 1]);
    }
    float q = 0.0f;
    if (lane < 6) {
        const double v = dth[lane];
        const float hi = (float)v;
        a.dtheta64[6 * f + lane] = v;
        a.dth2[6 * f + lane] = make_float2(hi, (float)(v - (double)hi));
        q = hi * hi;  // |Dtheta_f|^2 is a convergence statistic: FP32 is enough
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) a.dthsq[f] = q;
}

// Rodrigues coefficients of omega: A = sin/th, B = (1-cos)/th^2,
// C = (th-sin)/th^3. Updates are small rotations, so below th = 0.5 the
// coefficients come from their Taylor series in x = th^2 (Horner, eight
// terms: the first omitted one is below 1e-19 there); FP64 sincos and three
// FP64 divisions on one lane cost several microseconds on GB300.
__device__ void rodrigues_coeffs(const double* w, double* ABC, int lane)
{
    if (lane == 0) {
        const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        if (th2 < 0.25) {
            // 1/(2k+1)!, 1/(2k+2)!, 1/(2k+3)! for k = 7 .. 0, in powers of -x
            const double y = -th2;
            double A = 1.0 / 1307674368000.0, B = 1.0 / 20922789888000.0, C = 1.0 / 355687428096000.0;
            A = fma(A, y, 1.0 / 6227020800.0);
            B = fma(B, y, 1.0 / 87178291200.0);
            C = fma(C, y, 1.0 / 1307674368000.0);
            A = fma(A, y, 1.0 / 39916800.0);
            B = fma(B, y, 1.0 / 479001600.0);
            C = fma(C, y, 1.0 / 6227020800.0);
            A = fma(A, y, 1.0 / 362880.0);
            B = fma(B, y, 1.0 / 3628800.0);
            C = fma(C, y, 1.0 / 39916800.0);
            A = fma(A, y, 1.0 / 5040.0);
            B = fma(B, y, 1.0 / 40320.0);
            C = fma(C, y, 1.0 / 362880.0);
            A = fma(A, y, 1.0 / 120.0);
            B = fma(B, y, 1.0 / 720.0);
            C = fma(C, y, 1.0 / 5040.0);
            A = fma(A, y, 1.0 / 6.0);
            B = fma(B, y, 1.0 / 24.0);
            C = fma(C, y, 1.0 / 120.0);
            A = fma(A, y, 1.0);
            B = fma(B, y, 0.5);
            C = fma(C, y, 1.0 / 6.0);
            ABC[0] = A;
            ABC[1] = B;
            ABC[2] = C;
        } else {
            const double th = sqrt(th2);
            double sn, cs;
            sincos(th, &sn, &cs);
            ABC[0] = sn / th;
            ABC[1] = (1.0 - cs) / th2;
            ABC[2] = (th - sn) / (th2 * th);
        }
    }
    __syncwarp();
}

// Entry e (0..8) of I + p [w]x + q [w]x^2 with [w]x^2 = w w^T - |w|^2 I.
__device__ __forceinline__ double rodrigues_entry(const double* w, double p, double q, int e)
{
    const int i = e / 3, j = e % 3;
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double K = 0.0;  // [w]x (i, j)
    if (i != j) {
        const int k = 3 - i - j;
        K = ((j - i + 3) % 3 == 1) ? -w[k] : w[k];
    }
    return (i == j ? 1.0 : 0.0) + p * K + q * (w[i] * w[j] - (i == j ? th2 : 0.0));
}

// Sec. 3.6: R <- R R0^T exp(omega)^T R0, t <- t - R R0^T Dt (old R on the
// right-hand sides). pose, p0: the frame's current and p_0 poses (12 each,
// shared memory); sh: 48 doubles of warp-private shared memory.
__device__ void ic_pose_update_warp(const SolveArgs& a, int f, const double* pose, const double* p0,
                                    const double* dth, double* sh, int lane)
{
    double *R = sh, *R0t = sh + 9, *A = sh + 18, *E = sh + 27, *B = sh + 36, *t = sh + 45;
    double ABC[3];
    if (lane < 9) {
        R[lane] = pose[lane];
        R0t[lane] = p0[3 * (lane % 3) + lane / 3];
    }
    double* coef = B;  // scratch until B is formed
    rodrigues_coeffs(dth + 3, coef, lane);
    for (int k = 0; k < 3; ++k) ABC[k] = coef[k];
    __syncwarp();
    if (lane < 9) {
        const double mw[3] = {-dth[3], -dth[4], -dth[5]};
        E[lane] = rodrigues_entry(mw, ABC[0], ABC[1], lane);  // exp(omega)^T = exp(-omega)
    }
    __syncwarp();
    mat3_mul_lanes(R, R0t, A, lane);   // A = R R0^T
    mat3_mul_lanes(A, E, B, lane);     // B = A exp(-omega)
    double* Rn = E;                    // E no longer needed
    if (lane < 9) {
        const int i = lane / 3, j = lane % 3;
        Rn[lane] = fma(B[3 * i], p0[j], fma(B[3 * i + 1], p0[3 + j], B[3 * i + 2] * p0[6 + j]));
    }
    if (lane < 3)
        t[lane] = pose[9 + lane] - fma(A[3 * lane], dth[0], fma(A[3 * lane + 1], dth[1], A[3 * lane + 2] * dth[2]));
    __syncwarp();
    write_frame_lanes(a, f, pose, Rn, t, dth, lane);
}

// Boxplus: T <- exp([upsilon, omega]) T.
__device__ void fc_pose_update_warp(const SolveArgs& a, int f, const double* dth, double* sh, int lane)
{
    double *E = sh, *V = sh + 9, *Rn = sh + 18, *R = sh + 27, *t = sh + 36, *ABC = sh + 39;
    double* pose = sh + 42;  // 12 (sh holds 54 doubles)
    if (lane < 12) pose[lane] = a.poses64[12 * f + lane];
    __syncwarp();
    if (lane < 9) R[lane] = pose[lane];
    rodrigues_coeffs(dth + 3, ABC, lane);
    if (lane < 9) E[lane] = rodrigues_entry(dth + 3, ABC[0], ABC[1], lane);
    else if (lane < 18) V[lane - 9] = rodrigues_entry(dth + 3, ABC[1], ABC[2], lane - 9);
    __syncwarp();
    mat3_mul_lanes(E, R, Rn, lane);
    if (lane < 3)
        t[lane] = fma(E[3 * lane], pose[9], fma(E[3 * lane + 1], pose[10], E[3 * lane + 2] * pose[11])) +
                  fma(V[3 * lane], dth[0], fma(V[3 * lane + 1], dth[1], V[3 * lane + 2] * dth[2]));
    __syncwarp();
    write_frame_lanes(a, f, pose, Rn, t, dth, lane);
}

// Scale gauge (the one free direction of the system, Delta t_f = -t_f,
// Delta d_n = d_n): the prior mu that that^T selects the solution with
// that . Delta t_anchor = 0, but in floating point the prior pins that
// component only to cond(S) * eps. Adding alpha times the null vector leaves
// H Delta p unchanged, so the constraint is imposed exactly:
//   alpha = (t_a . Delta t_a) / |t_a|^2,  Delta t_f -= alpha t_f (active f),
// and the depth back-substitution carries the matching alpha d_n.
__device__ __forceinline__ double gauge_alpha(const double* ta, const double* dta)
{
    const double n2 = ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2];
    return n2 > 0.0 ? (ta[0] * dta[0] + ta[1] * dta[1] + ta[2] * dta[2]) / n2 : 0.0;
}

// IC step 3 + 4: Dtheta = -S^-1 y (one CTA per target frame, one warp per
// row, FP64 dot products; warps 6-8 also form the anchor frame's Delta t for
// the gauge constraint), then the frame's pose update by warp 0. Everything
// the update reads besides Dtheta is fetched at the start, beside the rows.
__global__ void __launch_bounds__(9 * 32) ic_solve_update_kernel(SolveArgs a, const double* Sinv,
                                                                 const double* y, int y_stride,
                                                                 int y_off)
{
    __shared__ double dth[9];
    __shared__ double d[6];
    __shared__ double sh[48];
    __shared__ double s_pose[12], s_p0[12], s_ta[3], s_tf[3];
    __shared__ int s_act;
    const int f = blockIdx.x + 1, tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
    const int n6 = a.n6;
    const int anchor = a.active[0];
    if (row == 8) {
        if (lane < 12) s_pose[lane] = a.poses64[12 * f + lane];
        else if (lane < 24) s_p0[lane - 12] = a.poses0[12 * f + lane - 12];
        else if (lane < 27) s_tf[lane - 24] = a.tanchor[12 * f + 9 + lane - 24];
        else if (lane < 30) s_ta[lane - 27] = anchor > 0 ? a.tanchor[12 * anchor + 9 + lane - 27] : 0.0;
        else if (lane == 30) s_act = a.active[f];
    }
    const int rr = row < 6 ? 6 * (f - 1) + row : (anchor > 0 ? 6 * (anchor - 1) + row - 6 : -1);
    if (rr >= 0) {
        const double* Sr = Sinv + (size_t)rr * n6;
        double s0 = 0.0, s1 = 0.0;  // two chains halve the dependent FP64 latency
        int c = lane;
        for (; c + 32 < n6; c += 64) {
            s0 = fma(Sr[c], y[(size_t)(c / 6 + 1) * y_stride + y_off + c % 6], s0);
            s1 = fma(Sr[c + 32], y[(size_t)((c + 32) / 6 + 1) * y_stride + y_off + (c + 32) % 6], s1);
        }
        if (c < n6) s0 = fma(Sr[c], y[(size_t)(c / 6 + 1) * y_stride + y_off + c % 6], s0);
        const double s = warp_sum1d(s0 + s1);
        if (lane == 0) dth[row] = -s;
    }
    __syncthreads();
    if (row != 0) return;
    if (lane < 6) {
        double v = dth[lane];
        if (lane < 3 && anchor > 0 && s_act) {
            const double alpha = gauge_alpha(s_ta, dth + 6);
            v = fma(-alpha, s_tf[lane], v);
        }
        d[lane] = v;
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, lane >= 6 || isfinite(d[lane]));
    if (!ok) {
        if (lane == 0) atomicOr(a.err, kErrNonFinite);
        if (lane < 6) d[lane] = 0.0;
        __syncwarp();
    }
    ic_pose_update_warp(a, f, s_pose, s_p0, d, sh, lane);
}

cudaError_t launch_ic_solve_update(const SolveArgs& a, const double* Sinv, const double* y,
                                   int y_stride, int y_off, cudaStream_t st)
{
    ic_solve_update_kernel<<<a.F - 1, 9 * 32, 0, st>>>(a, Sinv, y, y_stride, y_off);
    return cudaGetLastError();
}

// FC: the factorisation has eliminated b = -y with the matrix, so row n of L
// holds D^-1 L^-1 b; the backward substitution L^T Dtheta = that row gives
// Dtheta = -S^-1 y (double-float, one CTA). Then the exact gauge constraint
// and every frame's boxplus update (one warp per frame, FP64).
constexpr int kFcSolveWarps = 32;  // one warp per frame's update (F <= 33 in one round)

__global__ void __launch_bounds__(kFcSolveWarps * 32) fc_solve_update_kernel(SolveArgs a, const dfloat* L,
                                                                           const dfloat* Linv)
{
    extern __shared__ dfloat xs[];
    __shared__ dfloat tb[kLdlBlock];
    double* x = reinterpret_cast<double*>(xs + a.n6);
    __shared__ double s_alpha;
    __shared__ double sh[kFcSolveWarps][54];
    __shared__ double dsh[kFcSolveWarps][6];
    const int n = a.n6, nc = 6 * a.cmap[a.F], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nc; i += blockDim.x) xs[i] = L[(size_t)nc * nc + i];
    __syncthreads();
    ldl_backward_smem(L, Linv, nc, xs, tb);
    // back to the full frame order (frames left out get no update)
    for (int i = tid; i < n; i += blockDim.x) {
        const int k = a.cmap[i / 6 + 1];
        x[i] = k >= 0 ? df_to_double(xs[6 * k + i % 6]) : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        const int anchor = a.active[0];
        s_alpha = anchor > 0 ? gauge_alpha(a.tanchor + 12 * anchor + 9, x + 6 * (anchor - 1)) : 0.0;
    }
    __syncthreads();
    for (int f = 1 + warp; f < a.F; f += blockDim.x >> 5) {
        double* d = dsh[warp];
        if (lane < 6) {
            double v = x[6 * (f - 1) + lane];
            if (lane < 3 && a.active[f]) v = fma(-s_alpha, a.tanchor[12 * f + 9 + lane], v);
            d[lane] = v;
        }
        __syncwarp();
        const bool ok = __all_sync(0xffffffffu, lane >= 6 || isfinite(d[lane]));
        if (!ok) {
            if (lane == 0) atomicOr(a.err, kErrNonFinite);
            if (lane < 6) d[lane] = 0.0;
            __syncwarp();
        }
        fc_pose_update_warp(a, f, d, sh[warp], lane);
        __syncwarp();
    }
}

cudaError_t launch_fc_solve_update(const SolveArgs& a, const dfloat* L, const dfloat* Linv,
                                   cudaStream_t st)
{
    fc_solve_update_kernel<<<1, kFcSolveWarps * 32, (sizeof(dfloat) + sizeof(double)) * a.n6, st>>>(a, L, Linv);
    return cudaGetLastError();
}

}  // namespace pba
