// Reduced camera system (Sec. 3.5 step 3): assembly of S with the
// scale-gauge prior, the IC solve (explicit FP64 S^-1 applied as a GEMV, the
// factorisation being done once), the FC solve (substitutions with the FP64
// Cholesky factor, every iteration), and the FP64 pose updates of Sec. 3.6
// (IC) and of the boxplus operator (FC).
#include <algorithm>

#include "pba_chol.cuh"
#include "pba_pose.cuh"

namespace pba {

// ---------------------------------------------------------------------------
// S = blockdiag(H_ff) - S_off, then: frames without residuals (zero H_ff
// trace) get an identity block; mu = mean diagonal over the active frames;
// the prior gauge_w * mu * that that^T goes on the translation block of the
// first active frame (that = unit translation of that frame in anchor_t).
// With Levenberg-Marquardt damping lambda > 0 the diagonal entries of H_ff
// are scaled by 1 + lambda (S_off already holds the damped H_dd) and the
// prior is left out: the damped system is definite without it.
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

// Bundle blockIdx.y of bs, gridDim.x CTAs per bundle.
__global__ void __launch_bounds__(kAssembleThreads)
assemble_S_kernel(BundleSet bs, const double* Hff, int stride, const double* Soff,
                  const double* anchor_t, double gauge_w, double damping, double* S, int* active, dfloat* S2,
                  int* cmap, const double* rhs, int rhs_stride, int rhs_off)
{
    __shared__ int s_act[1024];
    __shared__ int s_cidx[1024];  // compact index of an active frame
    __shared__ int s_nact;
    __shared__ double s_red[kAssembleThreads / 32];
    __shared__ int s_anchor;
    __shared__ double s_mu;
    const BundleDesc bd = bundle_at(bs, blockIdx.y);
    const int F = bd.F;
    Hff += (size_t)bd.fo * stride;
    anchor_t += (size_t)12 * bd.fo;
    active += bd.fo;
    Soff += bd.so;
    S += bd.so;
    if (S2) S2 += bd.ao;
    if (cmap) cmap += bd.co;
    if (rhs) rhs += (size_t)bd.fo * rhs_stride;
    const int n6 = 6 * (F - 1), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double ld = 1.0 + damping;  // Levenberg-Marquardt: diagonal entries x (1 + lambda)
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
        if (s_act[f])
            part += Hff[(size_t)f * stride + upper_index(i % 6, i % 6)] * ld - Soff[(size_t)i * n6 + i];
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
                v += Hff[(size_t)fi * stride + upper_index(i % 6, j % 6)] * (i == j ? ld : 1.0);
                const int a = i % 6, b = j % 6;
                // the damped system is definite without the gauge prior
                if (fi == anchor && a < 3 && b < 3 && damping == 0.0) v += s_mu * (th[a] * th[b]);
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

cudaError_t launch_assemble_S(const BundleSet& bs, const double* Hff, int hff_stride, const double* Soff,
                              const double* anchor_t, double gauge_w, double damping, double* S, int* active,
                              cudaStream_t st, dfloat* S2, int* cmap, const double* rhs,
                              int rhs_stride, int rhs_off)
{
    if (S2 && !cmap) return cudaErrorInvalidValue;
    const int n6 = bs.n6max;
    if (n6 > 6 * 1023 || bs.B < 1 || bs.B > 65535) return cudaErrorInvalidValue;
    // one element per thread on up to 148 SMs (the FP64 -> double-float
    // conversions go to the slow FP64 pipe), spread over the bundles
    const int per_bundle = std::max(1, 1184 / bs.B);
    const int blocks =
        std::max(1, std::min(std::min(148, per_bundle), (n6 * n6 + kAssembleThreads - 1) / kAssembleThreads));
    assemble_S_kernel<<<dim3(blocks, bs.B), kAssembleThreads, 0, st>>>(bs, Hff, hff_stride, Soff, anchor_t,
                                                                       gauge_w, damping, S, active, S2, cmap,
                                                                       rhs, rhs_stride, rhs_off);
    return cudaGetLastError();
}

// FC: the factorisation has eliminated b = -y with the matrix, so row n of L
// holds D^-1 L^-1 b; the backward substitution L^T Dtheta = that row gives
// Dtheta = -S^-1 y (double-float, one CTA per bundle). Then the exact gauge
// constraint; the update is written per frame (the reference frame's is
// zero) and the boxplus pose updates run in the next launch, one frame per
// CTA.
constexpr int kFcSolveWarps = 32;  // one warp per frame's update

__global__ void __launch_bounds__(kFcSolveWarps * 32) fc_solve_update_kernel(SolveArgs a, const dfloat* L,
                                                                           const dfloat* Linv)
{
    extern __shared__ dfloat xs[];
    __shared__ dfloat tb[kLdlBlock];
    __shared__ double s_alpha;
    __shared__ double dsh[kFcSolveWarps][6];
    const BundleDesc bd = a.bund[blockIdx.x];
    const int F = bd.F, fo = bd.fo;
    const int* cmap = a.cmap + bd.co;
    const int* active = a.active + fo;
    const double* tanchor = a.tanchor + (size_t)12 * fo;
    L += bd.ao;
    Linv += bd.lo;
    double* x = reinterpret_cast<double*>(xs + a.n6);
    const int n = 6 * (F - 1), nc = 6 * cmap[F], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the brightness pairs from this step's residuals
    if (a.photo_sums)
        for (int f = 1 + tid; f < F; f += blockDim.x)
            photo_update_frame(a.photo_sums + (size_t)5 * (fo + f), a.fc + (size_t)(fo + f) * kFrameConst);
    for (int i = tid; i < nc; i += blockDim.x) xs[i] = L[(size_t)nc * nc + i];
    __syncthreads();
    ldl_backward_smem(L, Linv, nc, xs, tb);
    // back to the full frame order (frames left out get no update)
    for (int i = tid; i < n; i += blockDim.x) {
        const int k = cmap[i / 6 + 1];
        x[i] = k >= 0 ? df_to_double(xs[6 * k + i % 6]) : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        const int anchor = active[0];
        s_alpha = anchor > 0 ? gauge_alpha(tanchor + 12 * anchor + 9, x + 6 * (anchor - 1)) : 0.0;
    }
    __syncthreads();
    for (int f = warp; f < F; f += blockDim.x >> 5) {
        double* d = dsh[warp];
        if (lane < 6) {
            double v = f > 0 ? x[6 * (f - 1) + lane] : 0.0;
            if (lane < 3 && f > 0 && active[f]) v = fma(-s_alpha, tanchor[12 * f + 9 + lane], v);
            d[lane] = v;
        }
        __syncwarp();
        const bool ok = __all_sync(0xffffffffu, lane >= 6 || isfinite(d[lane]));
        if (!ok) {
            if (lane == 0) flag_error(a.err, blockIdx.x, kErrNonFinite);
            if (lane < 6) d[lane] = 0.0;
            __syncwarp();
        }
        write_update_lanes(a, fo + f, d, lane);
        __syncwarp();
    }
}

cudaError_t linalg_setup()
{
    // dynamic shared memory above the default 48 KB for the largest systems
    // (1024 frames: 6138 rows)
    return cudaFuncSetAttribute(fc_solve_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((sizeof(dfloat) + sizeof(double)) * 6 * 1023));
}

cudaError_t launch_fc_solve_update(const SolveArgs& a, const dfloat* L, const dfloat* Linv,
                                   cudaStream_t st)
{
    fc_solve_update_kernel<<<a.B, kFcSolveWarps * 32, (sizeof(dfloat) + sizeof(double)) * a.n6, st>>>(a, L,
                                                                                                     Linv);
    return cudaGetLastError();
}

}  // namespace pba
