// Substitutions with the LDL^T factor of the reduced camera system (Sec. 3.5
// step 3), in double-float arithmetic. L (unit lower, row-major n x n of
// dfloat) holds the factor in its lower triangle and L^T in its upper
// triangle, so both substitutions read rows; Linv holds the inverses of its
// 32 x 32 diagonal blocks (block b at Linv + b * 2048: the inverse, then its
// transpose), so a block's triangular solve is a matrix-vector product
// instead of 32 dependent steps.
#pragma once

#include "pba_df.cuh"
#include "pba_kernels.cuh"

namespace pba {

constexpr int kLdlBlock = 32;
constexpr int kLinvStride = 2 * kLdlBlock * kLdlBlock;  // dfloats per diagonal block in Linv

// y[r] = sum_{c in [c0, c1)} M[r * ldm + c] x[c] for the rows r < nr of a
// block (warp w takes rows w, w + nw, ...; lanes take columns; four rows at
// a time, their sums interleaved), written as out[r] = base[r] - y[r]
// (sub = true) or out[r] = y[r].
__device__ __forceinline__ void block_gemv(const dfloat* M, int ldm, int nr, int c0, int c1,
                                           const dfloat* x, dfloat* out, bool sub)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < nr; r += 4 * nw) {
        DfAcc acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int rr = r + u * nw;
            if (rr < nr) {
                const dfloat* Mr = M + (size_t)rr * ldm;
                for (int c = c0 + lane; c < c1; c += 32) acc[u].add_prod(Mr[c], x[c]);
            }
        }
        dfloat s[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = df_warp_sum(acc[u].value());
        if (lane < 4) {
            const int rr = r + lane * nw;
            dfloat v = s[0];
#pragma unroll
            for (int u = 1; u < 4; ++u) v = lane == u ? s[u] : v;
            if (rr < nr) out[rr] = sub ? df_sub(out[rr], v) : v;
        }
    }
}

// x <- L^-1 x (forward substitution, unit diagonal), x in shared memory,
// one CTA; blocks before block b_first are known to be zero on entry.
// t: 32 dfloats of shared scratch.
__device__ inline void ldl_forward_smem(const dfloat* L, const dfloat* Linv, int n, dfloat* x,
                                        dfloat* t, int b_first)
{
    for (int b0 = b_first * kLdlBlock; b0 < n; b0 += kLdlBlock) {
        const int nb = min(kLdlBlock, n - b0);
        const dfloat* Li = Linv + (size_t)(b0 / kLdlBlock) * kLinvStride;
        if (b0 > b_first * kLdlBlock)
            block_gemv(L + (size_t)b0 * n, n, nb, b_first * kLdlBlock, b0, x, x + b0, true);
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x) t[i] = x[b0 + i];
        __syncthreads();
        block_gemv(Li, kLdlBlock, nb, 0, nb, t, x + b0, false);
        __syncthreads();
    }
}

// x <- L^-T x (backward substitution), same layout.
__device__ inline void ldl_backward_smem(const dfloat* L, const dfloat* Linv, int n, dfloat* x,
                                         dfloat* t)
{
    for (int b0 = ((n - 1) / kLdlBlock) * kLdlBlock; b0 >= 0; b0 -= kLdlBlock) {
        const int nb = min(kLdlBlock, n - b0);
        const dfloat* LiT = Linv + (size_t)(b0 / kLdlBlock) * kLinvStride + kLdlBlock * kLdlBlock;
        if (b0 + nb < n) block_gemv(L + (size_t)b0 * n, n, nb, b0 + nb, n, x, x + b0, true);
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x) t[i] = x[b0 + i];
        __syncthreads();
        block_gemv(LiT, kLdlBlock, nb, 0, nb, t, x + b0, false);
        __syncthreads();
    }
}

}  // namespace pba
