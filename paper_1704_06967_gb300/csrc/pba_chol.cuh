// Substitutions with the FP64 Cholesky factor of the reduced camera system
// (Sec. 3.5 step 3). L holds the factor in its lower triangle and L^T in its
// upper triangle; inv_diag holds 1 / L_ii (FP64 division is slow on GB300, so
// the substitutions only multiply).
#pragma once

#include "pba_kernels.cuh"

namespace pba {

// L L^T x = b with x in shared memory (in: b, out: x), one CTA. Blocks of 32
// rows: the off-diagonal part is a warp-per-row GEMV along rows of the lower
// (forward) or upper = L^T (backward) triangle; the 32x32 diagonal triangle
// is solved by one warp with shuffles.
__device__ inline void chol_solve_smem(const double* L, const double* inv_diag, int n, double* x)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int nb = min(32, n - b0);
        for (int r = warp; r < nb; r += nw) {
            const double* Lr = L + (size_t)(b0 + r) * n;
            double s = 0.0;
            for (int j = lane; j < b0; j += 32) s = fma(Lr[j], x[j], s);
            s = warp_sum1d(s);
            if (lane == 0) x[b0 + r] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            double xi = lane < nb ? x[b0 + lane] : 0.0;
            const double ri = lane < nb ? inv_diag[b0 + lane] : 0.0;
            for (int c = 0; c < nb; ++c) {
                if (lane == c) xi *= ri;
                const double xc = __shfl_sync(0xffffffffu, xi, c);
                if (lane > c && lane < nb) xi = fma(-L[(size_t)(b0 + lane) * n + b0 + c], xc, xi);
            }
            if (lane < nb) x[b0 + lane] = xi;
        }
        __syncthreads();
    }
    for (int b0 = ((n - 1) / 32) * 32; b0 >= 0; b0 -= 32) {
        const int nb = min(32, n - b0);
        for (int r = warp; r < nb; r += nw) {
            const double* Ur = L + (size_t)(b0 + r) * n;  // row of L^T (upper triangle)
            double s = 0.0;
            for (int j = b0 + nb + lane; j < n; j += 32) s = fma(Ur[j], x[j], s);
            s = warp_sum1d(s);
            if (lane == 0) x[b0 + r] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            double xi = lane < nb ? x[b0 + lane] : 0.0;
            const double ri = lane < nb ? inv_diag[b0 + lane] : 0.0;
            for (int c = nb - 1; c >= 0; --c) {
                if (lane == c) xi *= ri;
                const double xc = __shfl_sync(0xffffffffu, xi, c);
                // L^T(lane, c) = L(c, lane), read from the lower triangle
                if (lane < c) xi = fma(-L[(size_t)(b0 + c) * n + b0 + lane], xc, xi);
            }
            if (lane < nb) x[b0 + lane] = xi;
        }
        __syncthreads();
    }
}

}  // namespace pba
