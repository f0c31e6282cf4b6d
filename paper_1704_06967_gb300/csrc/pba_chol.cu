// LDL^T factorisation of the reduced camera system (Sec. 3.5 step 3:
// Delta p = -H^-1 g through the Schur complement S) in double-float
// arithmetic, and the IC inverse S^-1 = L^-T D^-1 L^-1.
//
// GB300 issues FP64 at 1/64 of the FP32 rate and its dependent FP64 latency
// is ~14x the FP32 one; a factorisation of a 174 x 174 system is a chain of
// 174 dependent pivots, so its FP64 form is latency-bound at tens of
// microseconds and throughput-bound on any single SM. Here the matrix is held
// as double-float pairs (about 48 bits; the system's condition number,
// ~3e7 on the helix bundle, leaves ~1e-7 relative error in the solution,
// well inside the 1e-4 step tolerance) and factored by one thread-block
// cluster: blocked right-looking LDL^T with 32 x 32 blocks, where per block
// column k
//   every CTA factors the diagonal block A_kk in shared memory (redundantly,
//     so no CTA waits for it) and, in the same steps, eliminates its share
//     of the rows below (W_ik L_kk^T = A_ik, W = L D): one barrier per pivot,
//     the reciprocal of the next pivot formed by the thread that updated it;
//     it stores L_ik = W_ik D_k^-1;
//   cluster barrier; the trailing tiles (i, j), k < j <= i, are dealt
//     round-robin to the CTAs: A_ij -= (L_ik D_k) L_jk^T;
//   cluster barrier.
// The cluster barriers order the global-memory writes of one step before the
// reads of the next (release / acquire at cluster scope); no CTA spins.
// A non-positive pivot sets kErrNotPD and is replaced by 1.
//
// Augmented right-hand side: with aug = 1 the input has one extra row n
// holding b^T; it is eliminated like any other row, so on exit row n of L
// holds (D^-1 L^-1 b)^T and only the backward substitution remains.
#include <cooperative_groups.h>

#include "pba_chol.cuh"

namespace cg = cooperative_groups;

namespace pba {

namespace {

constexpr int kNB = 32;
constexpr int kCholThreads = 1024;  // one thread per element of a 32 x 32 block
// cluster size: 16 CTAs (non-portable, allowed on sm_103a) when the device
// can co-schedule them, else the portable 8; chosen once by ldl_setup()
int g_chol_cluster = 8;

struct CholSmem {
    dfloat D[kNB][kNB + 1];   // diagonal block: W below the diagonal, pivots d_j on it
    dfloat r[kNB];            // 1 / d_j
    unsigned short tri[kNB * (kNB - 1) / 2];  // packed index -> (i', m') of the trailing triangle
    dfloat T0[kNB][kNB + 1];  // rows being eliminated / rows i of a trailing tile (L D)
    dfloat T1[kNB][kNB + 1];  // rows j of a trailing tile (L)
};

// reciprocal of a pivot; a non-positive one (of a real row) is flagged and
// replaced by 1
__device__ __forceinline__ dfloat pivot_recip(dfloat& d, bool real, int* err, int bundle)
{
    if (!(d.x > 0.0f)) {
        if (real) flag_error(err, bundle, kErrNotPD);
        d = df_make(1.0f, 0.0f);
    }
    return df_recip(d);
}

// One thread per element of a 32 x 32 block (1024 threads: warp = row,
// lane = column) for loads, stores and the trailing tiles. In elimination
// step j the diagonal block's active elements (j < m <= i) are packed onto
// the first (31-j)(32-j)/2 threads through a table, and the rows below use
// the top warps, so no issue slot goes to an element that is already done.
// Cluster c of the grid factors bundle c's system.
__global__ void __launch_bounds__(kCholThreads)
ldl_cluster_kernel(BundleSet bs, dfloat* A, dfloat* L, dfloat* Linv, dfloat* dpiv, dfloat* rpiv,
                   const int* cmap, int aug, int* err)
{
    __shared__ CholSmem sm;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
    const int bundle = (int)blockIdx.x / C;
    const BundleDesc bd = bundle_at(bs, bundle);
    A += bd.ao;
    L += bd.ao;
    Linv += bd.lo;
    dpiv += bd.po;
    rpiv += bd.po;
    const int n = bs.nb * cmap[bd.co + bd.F];  // active frames only (the same value in every CTA)
    const int tid = threadIdx.x, wi = tid >> 5, lm = tid & 31;
    const int nrow = n + aug;  // rows of A / L (the last one is b^T when aug)
    const int nblk = (n + kNB - 1) / kNB;
    const int nblk_r = (nrow + kNB - 1) / kNB;
    // triangle enumeration, column-major from the bottom-right corner:
    // e = m'(m'+1)/2 + i', 0 <= i' <= m', element (31 - i', 31 - m'); the
    // first s(s+1)/2 entries are the triangle left after step 31 - s
    if (tid < kNB * (kNB - 1) / 2) {
        int mp = (int)((sqrtf(8.0f * tid + 1.0f) - 1.0f) * 0.5f);
        while (mp * (mp + 1) / 2 > tid) --mp;
        while ((mp + 1) * (mp + 2) / 2 <= tid) ++mp;
        const int ip = tid - mp * (mp + 1) / 2;
        sm.tri[tid] = (unsigned short)(ip | (mp << 8));
    }
    for (int k = 0; k < nblk; ++k) {
        const int k0 = k * kNB, nk = min(kNB, n - k0);
        // rows below the block are split over the CTAs; this CTA eliminates
        // its share (32 rows at a time) together with the diagonal block
        const int below = nrow - k0 - nk;
        const int per = (below + C - 1) / C;
        const int a0 = k0 + nk + rank * per, a1 = min(nrow, a0 + per);
        for (int r0 = a0; r0 < max(a1, a0 + 1); r0 += kNB) {
            const int nr = max(0, min(kNB, a1 - r0));
            const bool first = r0 == a0;
            // ---- load: diagonal block (lower triangle current, identity
            // outside nk) on the first chunk, and this chunk of rows below
            if (first) {
                dfloat v = df_make(wi == lm ? 1.0f : 0.0f, 0.0f);
                if (wi < nk && lm <= wi) v = A[(size_t)(k0 + wi) * n + k0 + lm];
                sm.D[wi][lm] = v;
            }
            sm.T0[wi][lm] = (wi < nr && lm < nk) ? A[(size_t)(r0 + wi) * n + k0 + lm] : df_make(0.0f, 0.0f);
            __syncthreads();
            if (first && tid == 0) sm.r[0] = pivot_recip(sm.D[0][0], nk > 0, err, bundle);
            __syncthreads();
            // ---- right-looking elimination, one barrier per pivot: the
            // diagonal block (first chunk only; later chunks reuse its
            // factor) and the rows below, A_im -= (A_ij / d_j) A_mj
            for (int j = 0; j < kNB - 1; ++j) {
                const int s = kNB - 1 - j;  // trailing triangle size
                if (first && tid < s * (s + 1) / 2) {
                    const unsigned short te = sm.tri[tid];
                    const int i = kNB - 1 - (te & 0xff), m = kNB - 1 - (te >> 8);
                    const dfloat lij = df_mul(sm.D[i][j], sm.r[j]);
                    dfloat v = df_fnms(lij, sm.D[m][j], sm.D[i][m]);
                    // the owner of (j+1, j+1) has just formed it: next reciprocal
                    // straight from the register
                    if (i == j + 1 && m == j + 1) sm.r[j + 1] = pivot_recip(v, j + 1 < nk, err, bundle);
                    sm.D[i][m] = v;
                }
                const int ra = kNB - 1 - wi;  // rows below on the top warps
                if (ra < nr && lm > j && lm < nk) {
                    const dfloat wj = df_mul(sm.T0[ra][j], sm.r[j]);
                    sm.T0[ra][lm] = df_fnms(wj, sm.D[lm][j], sm.T0[ra][lm]);
                }
                __syncthreads();
            }
            if (first && rank == 0) {
                if (wi < nk && lm < nk && lm <= wi) {
                    const dfloat l = lm < wi ? df_mul(sm.D[wi][lm], sm.r[lm]) : df_make(1.0f, 0.0f);
                    L[(size_t)(k0 + wi) * n + k0 + lm] = l;
                    L[(size_t)(k0 + lm) * n + k0 + wi] = l;
                }
                if (tid < nk) {
                    dpiv[k0 + tid] = sm.D[tid][tid];
                    rpiv[k0 + tid] = sm.r[tid];
                }
            }
            // L_ik = W_ik D_k^-1 of this chunk
            if (wi < nr && lm < nk) {
                const dfloat l = df_mul(sm.T0[wi][lm], sm.r[lm]);
                L[(size_t)(r0 + wi) * n + k0 + lm] = l;
                if (r0 + wi < n) L[(size_t)(k0 + lm) * n + r0 + wi] = l;
            }
            __syncthreads();
        }
        cl.sync();
        // ---- trailing tiles (bi, bj), k < bj <= bi, round-robin over the CTAs
        const int nt = nblk - k - 1;     // trailing block columns
        const int ntr = nblk_r - k - 1;  // trailing block rows (one more with b^T in a new block)
        const int tiles = nt * (nt + 1) / 2 + (ntr > nt ? nt : 0);
        for (int tt = rank; tt < tiles; tt += C) {
            int bi, bj;
            if (tt < nt * (nt + 1) / 2) {
                int t = tt;
                bi = k + 1;
                while (t > bi - k - 1) {
                    t -= bi - k;
                    ++bi;
                }
                bj = k + 1 + t;
            } else {  // the block row that holds only b^T
                bi = nblk;
                bj = k + 1 + (tt - nt * (nt + 1) / 2);
            }
            const int i0 = bi * kNB, j0 = bj * kNB;
            const int ni = min(kNB, nrow - i0), nj = min(kNB, n - j0);
            {
                dfloat a = df_make(0.0f, 0.0f), b = df_make(0.0f, 0.0f);
                if (lm < nk) {
                    if (wi < ni) a = df_mul(L[(size_t)(i0 + wi) * n + k0 + lm], sm.D[lm][lm]);
                    if (wi < nj) b = L[(size_t)(j0 + wi) * n + k0 + lm];
                }
                sm.T0[wi][lm] = a;
                sm.T1[wi][lm] = b;
            }
            __syncthreads();
            if (wi < ni && lm < nj && (bi > bj || lm <= wi)) {
                DfAcc acc;
#pragma unroll 8
                for (int j = 0; j < nk; ++j) acc.add_prod(sm.T0[wi][j], sm.T1[lm][j]);
                dfloat* p = A + (size_t)(i0 + wi) * n + j0 + lm;
                *p = df_sub(*p, acc.value());
            }
            __syncthreads();
        }
        cl.sync();
    }
    // ---- inverses of the diagonal blocks (unit lower), block b by CTA
    // b mod C: X = I, then X_i -= L_ij X_j for i > j, one barrier per column
    for (int b = rank; b < nblk; b += C) {
        const int b0 = b * kNB, nb = min(kNB, n - b0);
        sm.D[wi][lm] = (wi < nb && lm < wi) ? L[(size_t)(b0 + wi) * n + b0 + lm] : df_make(0.0f, 0.0f);
        sm.T0[wi][lm] = df_make(wi == lm ? 1.0f : 0.0f, 0.0f);
        __syncthreads();
        for (int j = 0; j < kNB - 1; ++j) {
            if (wi > j && lm <= j) sm.T0[wi][lm] = df_fnms(sm.D[wi][j], sm.T0[j][lm], sm.T0[wi][lm]);
            __syncthreads();
        }
        dfloat* out = Linv + (size_t)b * kLinvStride;
        out[wi * kNB + lm] = sm.T0[wi][lm];
        out[kNB * kNB + lm * kNB + wi] = sm.T0[wi][lm];
        __syncthreads();
    }
}

// S^-1 = L^-T D^-1 L^-1 over the active frames (compact nc x nc order,
// double-float), one column (= row) per CTA: the column's forward
// substitution (starting at its block), scaling and backward substitution.
// blockIdx.y is the bundle; CTAs beyond its nc (the grid is sized for all
// frames of the largest bundle) return at once.
__global__ void __launch_bounds__(256)
ldl_inverse_kernel(BundleSet bs, const dfloat* L, const dfloat* Linv, const dfloat* rpiv, const int* cmap,
                   dfloat* Sinv)
{
    extern __shared__ dfloat xs[];
    __shared__ dfloat t[kLdlBlock];
    const BundleDesc bd = bundle_at(bs, blockIdx.y);
    const int nc = bs.nb * cmap[bd.co + bd.F], c = blockIdx.x;
    if (c >= nc) return;
    L += bd.ao;
    Linv += bd.lo;
    rpiv += bd.po;
    Sinv += bd.so;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) xs[i] = df_make(i == c ? 1.0f : 0.0f, 0.0f);
    __syncthreads();
    ldl_forward_smem(L, Linv, nc, xs, t, c / kLdlBlock);
    for (int i = threadIdx.x; i < nc; i += blockDim.x) xs[i] = df_mul(xs[i], rpiv[i]);
    __syncthreads();
    ldl_backward_smem(L, Linv, nc, xs, t);
    for (int j = threadIdx.x; j < nc; j += blockDim.x) Sinv[(size_t)c * nc + j] = xs[j];
}

}  // namespace

cudaError_t launch_ldl(const BundleSet& bs, dfloat* A, dfloat* L, dfloat* Linv, dfloat* dpiv, dfloat* rpiv,
                       const int* cmap, int aug, int* err, cudaStream_t st, int cluster)
{
    const int C = cluster > 0 ? cluster : g_chol_cluster;
    if (C > g_chol_cluster || (C & (C - 1)) || bs.B < 1 || (bs.nb != 6 && bs.nb != 8)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * bs.B);
    cfg.blockDim = dim3(kCholThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ldl_cluster_kernel, bs, A, L, Linv, dpiv, rpiv, cmap, aug, err);
}

int ldl_max_cluster() { return g_chol_cluster; }

cudaError_t ldl_setup()
{
    cudaError_t e = cudaFuncSetAttribute(ldl_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kCholThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, ldl_cluster_kernel, &cfg);
    g_chol_cluster = (e == cudaSuccess && nclusters > 0) ? 16 : 8;
    cudaGetLastError();  // a refused query leaves the portable size
    return cudaSuccess;
}

cudaError_t launch_ldl_inverse(const BundleSet& bs, const dfloat* L, const dfloat* Linv, const dfloat* rpiv,
                               const int* cmap, dfloat* Sinv, cudaStream_t st)
{
    if (bs.nb != 6 && bs.nb != 8) return cudaErrorInvalidValue;
    const int n = bs.n6max / 6 * bs.nb;
    if (n > 8 * 1023 || n < 1 || bs.B < 1 || bs.B > 65535) return cudaErrorInvalidValue;
    ldl_inverse_kernel<<<dim3(n, bs.B), 256, sizeof(dfloat) * n, st>>>(bs, L, Linv, rpiv, cmap, Sinv);
    return cudaGetLastError();
}

}  // namespace pba
