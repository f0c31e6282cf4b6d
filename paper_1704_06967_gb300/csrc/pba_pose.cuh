// FP64 pose updates (Sec. 3.6 for IC, the boxplus T <- exp(xi) T for FC),
// one warp per frame, and the exact scale-gauge constraint. The solves write
// the update; the pose updates run one frame per CTA in the next launch
// (FP64 issues slowly: thirty frames on one SM would take ~30 x longer).
#pragma once

#include "pba_kernels.cuh"

namespace pba {

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
// memory), its FP32 pass constants and the previous R|t.
__device__ inline void write_frame_lanes(const SolveArgs& a, int f, const double* pose_old, const double* Rn,
                                         const double* tn, int lane)
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
}

// Writes the update of frame f (lanes 0..5 hold dth[lane]): FP64, as FP32
// pairs (hi, lo = v - hi) for the depth back-substitution, and |Dtheta_f|^2.
__device__ inline void write_update_lanes(const SolveArgs& a, int f, const double* dth, int lane)
{
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
__device__ inline void rodrigues_coeffs(const double* w, double* ABC, int lane)
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
__device__ inline void ic_pose_update_warp(const SolveArgs& a, int f, const double* pose, const double* p0,
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
    write_frame_lanes(a, f, pose, Rn, t, lane);
}

// Boxplus: T <- exp([upsilon, omega]) T.
__device__ inline void fc_pose_update_warp(const SolveArgs& a, int f, const double* dth, double* sh, int lane)
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
    write_frame_lanes(a, f, pose, Rn, t, lane);
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

}  // namespace pba
