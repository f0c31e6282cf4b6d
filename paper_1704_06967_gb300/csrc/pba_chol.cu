// FP64 Cholesky factorisation of the reduced camera system and the
// substitutions that use it (Sec. 3.5 step 3: Delta p = -H^-1 g through the
// Schur complement S).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so a factorisation on
// one SM is slow; the blocked right-looking algorithm spreads the trailing
// updates over all SMs. The working copy A is consumed; the factor goes to a
// separate matrix L. Per block column k (NB x NB blocks):
//   panel:  every CTA factors the diagonal block A_kk in shared memory (a
//           redundant 16x16 or 32x32 Cholesky), then CTA i > k solves
//           L_ik = A_ik L_kk^-T; results go to the lower triangle of L and,
//           transposed, to its upper triangle (so the backward substitution
//           reads rows);
//   update: one CTA per trailing tile (i, j), k < j <= i:
//           A_ij -= L_ik L_jk^T.
// Each launch reads one matrix and writes the other, so no CTA reads what
// another CTA of the same launch writes; the launches on the stream order the
// steps and no CTA waits on another. A non-positive pivot sets kErrNotPD and
// is replaced by 1.
#include "pba_chol.cuh"

namespace pba {

template <int NB>
__global__ void __launch_bounds__(NB * NB)
chol_panel_kernel(const double* A, double* L, double* inv_diag, int n, int k, int* err)
{
    __shared__ double D[NB][NB + 1];
    __shared__ double P[NB][NB + 1];
    __shared__ double rd[NB];
    const int tid = threadIdx.x, r = tid / NB, c = tid % NB;
    const int k0 = k * NB, nk = min(NB, n - k0);
    const int ib = k + blockIdx.x, i0 = ib * NB, ni = min(NB, n - i0);
    // the lower triangle of A_kk is current (updates touch only c <= r there)
    D[r][c] = (r < nk && c < nk) ? A[(size_t)(k0 + max(r, c)) * n + k0 + min(r, c)]
                                 : (r == c ? 1.0 : 0.0);
    if (blockIdx.x > 0) P[r][c] = (r < ni && c < nk) ? A[(size_t)(i0 + r) * n + k0 + c] : 0.0;
    __syncthreads();
    // unblocked right-looking factorisation of the diagonal block; one
    // division per column (FP64 division is slow), the rest multiplies
    for (int j = 0; j < NB; ++j) {
        if (tid == 0) {
            double v = D[j][j];
            if (!(v > 0.0)) {
                if (j < nk) atomicOr(err, kErrNotPD);
                v = 1.0;
            }
            // 1/sqrt(v) by Newton-Raphson from an FP32 seed: y <- y (3 - v y^2) / 2
            // (two steps take the ~23-bit seed past double precision); far
            // fewer dependent FP64 operations than a square root and a division
            double y = (double)rsqrtf((float)v);
            y = y * fma(-0.5 * v, y * y, 1.5);
            y = y * fma(-0.5 * v, y * y, 1.5);
            D[j][j] = v * y;
            rd[j] = y;
        }
        __syncthreads();
        if (c == j && r > j) D[r][j] *= rd[j];
        __syncthreads();
        if (r > j && c > j && c <= r) D[r][c] = fma(-D[r][j], D[c][j], D[r][c]);
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        if (r < nk && c <= r) {
            L[(size_t)(k0 + r) * n + k0 + c] = D[r][c];
            L[(size_t)(k0 + c) * n + k0 + r] = D[r][c];
        }
        if (tid < nk) inv_diag[k0 + tid] = rd[tid];
        return;
    }
    // X L_kk^T = P, right-looking over the columns: every (row, column)
    // element in parallel
    for (int j = 0; j < NB; ++j) {
        if (c == j) P[r][j] *= rd[j];
        __syncthreads();
        if (c > j) P[r][c] = fma(-P[r][j], D[c][j], P[r][c]);
        __syncthreads();
    }
    if (r < ni && c < nk) {
        L[(size_t)(i0 + r) * n + k0 + c] = P[r][c];
        L[(size_t)(k0 + c) * n + i0 + r] = P[r][c];
    }
}

template <int NB>
__global__ void __launch_bounds__(NB * NB)
chol_update_kernel(double* A, const double* L, int n, int k, int nblk)
{
    __shared__ double Li[NB][NB + 1];
    __shared__ double Lj[NB][NB + 1];
    // tile (i, j), k < j <= i < nblk, from the block index
    int t = blockIdx.x, j = k + 1, cnt = nblk - j;
    while (t >= cnt) {
        t -= cnt;
        ++j;
        cnt = nblk - j;
    }
    const int i = j + t;
    const int tid = threadIdx.x, r = tid / NB, c = tid % NB;
    const int k0 = k * NB, nk = min(NB, n - k0);
    const int i0 = i * NB, ni = min(NB, n - i0);
    const int j0 = j * NB, nj = min(NB, n - j0);
    Li[r][c] = (r < ni && c < nk) ? L[(size_t)(i0 + r) * n + k0 + c] : 0.0;
    Lj[r][c] = (r < nj && c < nk) ? L[(size_t)(j0 + r) * n + k0 + c] : 0.0;
    __syncthreads();
    if (r < ni && c < nj && (i > j || c <= r)) {
        double s = A[(size_t)(i0 + r) * n + j0 + c];
#pragma unroll
        for (int q = 0; q < NB; ++q) s = fma(-Li[r][q], Lj[c][q], s);
        A[(size_t)(i0 + r) * n + j0 + c] = s;
    }
}

template <int NB>
static cudaError_t chol_blocked(double* A, double* L, double* inv_diag, int n, int* err,
                               cudaStream_t st, int* launches)
{
    const int nblk = (n + NB - 1) / NB;
    for (int k = 0; k < nblk; ++k) {
        chol_panel_kernel<NB><<<nblk - k, NB * NB, 0, st>>>(A, L, inv_diag, n, k, err);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int rem = nblk - k - 1;
        if (rem > 0) {
            chol_update_kernel<NB><<<rem * (rem + 1) / 2, NB * NB, 0, st>>>(A, L, n, k, nblk);
            ++*launches;
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_cholesky(double* A, double* L, double* inv_diag, int n, int* err,
                            cudaStream_t st, int* launches)
{
    return n <= 256 ? chol_blocked<16>(A, L, inv_diag, n, err, st, launches)
                    : chol_blocked<32>(A, L, inv_diag, n, err, st, launches);
}

// S^-1 = L^-T L^-1, one column (= row, S^-1 is symmetric) per CTA.
__global__ void __launch_bounds__(256)
chol_inverse_kernel(const double* L, const double* inv_diag, double* Sinv, int n)
{
    extern __shared__ double x[];
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    chol_solve_smem(L, inv_diag, n, x);
    for (int i = threadIdx.x; i < n; i += blockDim.x) Sinv[(size_t)c * n + i] = x[i];
}

cudaError_t launch_chol_inverse(const double* L, const double* inv_diag, double* Sinv, int n,
                                cudaStream_t st)
{
    chol_inverse_kernel<<<n, 256, sizeof(double) * n, st>>>(L, inv_diag, Sinv, n);
    return cudaGetLastError();
}

}  // namespace pba
