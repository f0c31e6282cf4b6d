// Affine brightness pairs as unknowns of the Gauss-Newton system (an option
// beyond the paper, whose Sec. 2 notes that direct methods must model
// lighting; cfg.photometric = 2, one bundle per context). IC and FC share
// the border formation and the 8 (F - 1) assembly below; FC's columns are
// -I_f and -1 at the current parameters, re-formed every iteration, and its
// pairs are updated additively.
//
// Each target frame's block gains (da, db): the template-side increment
// (1 + da) I_0 + db, whose Jacobian columns I_0 and 1 are fixed like the
// rest of the IC system (Sec. 3.5), so the frame blocks are 8 x 8 and the
// reduced camera system has 8 unknowns per frame. The pose part of S is
// formed exactly as without the pairs (tensor-core or SIMT former,
// assemble_S_kernel); this file adds the border:
//   S_pa[f][g] = delta_fg H_pa(f) - sum_n H_fd(n,f) H_a(n,g)^T / H_dd(n)
//   S_aa[f][g] = delta_fg H_aa(f) - sum_n H_a(n,f) H_a(n,g)^T / H_dd(n)
// (H_a(n,f) = J_d^T W_0 [I_0, 1] per pair), assembles the 8 (F - 1) system
// for the double-float LDL^T and S^-1 of pba_chol.cu, and solves each
// iteration with that S^-1. The pair update composes the increment:
// alpha' = alpha / (1 + da), beta' = (beta - db) / (1 + da) (in the pose
// CTAs of the next depth update, so no kernel reads a pair while another
// CTA writes it). An optional prior lambda W_f ((ln alpha)^2 + beta^2) / 2
// (W_f = the frame's sum of W_0) adds lambda W_f to the pair's diagonal and
// -lambda W_f (ln alpha, beta) to its gradient.
#include <algorithm>

#include "pba_chol.cuh"
#include "pba_kernels.cuh"
#include "pba_pose.cuh"
#include "pba_reduce.cuh"

namespace pba {

namespace {

constexpr int kAffWarps = 4;

__device__ __forceinline__ int lane_rank(unsigned mask, int lane)
{
    return __popc(mask & ((1u << lane) - 1u));
}

// Fixed-point scale of the border sums: every partial sum of
// sum_n u_n v_n / H_dd(n) (u, v entries of H_fd or H_a of two frames) is
// bounded by sqrt(H_ff,aa H_aa,bb) (Cauchy-Schwarz per point, H_dd being at
// least the frame's share), so by m = the largest diagonal entry of the
// frame blocks; the sums are kept as integers of 2^(58 - e) units, 2^e > m.
// Every caller computes the same value from the same frame sums.
__device__ inline double affine_scale(const double* red_ff, int ff_stride, const double* red_aff, int F)
{
    double m = 0.0;
    for (int f = 1; f < F; ++f) {
        for (int a = 0; a < 6; ++a) m = fmax(m, red_ff[(size_t)f * ff_stride + a * 6 - a * (a - 1) / 2]);
        m = fmax(m, red_aff[(size_t)f * kAffComp + 12]);
        m = fmax(m, red_aff[(size_t)f * kAffComp + 14]);
    }
    if (!(m > 0.0) || !isfinite(m)) return 0.0;
    return ldexp(1.0, 58 - (ilogb(m) + 1));
}

}  // namespace

// One CTA per tile; warp w takes the tile's entries w, w + 4, ... as the
// left frame f and pairs each with every entry of the tile (frame g): the
// 12 + 4 sums over the lanes that both frames see are formed by
// reduce-scatter (sum q on lanes 2q, 2q + 1) and added to the integer
// accumulators (integer sums do not depend on the order of the additions,
// so the result is the same run to run).
__global__ void __launch_bounds__(kAffWarps * 32)
affine_schur_kernel(DevProblem pb, const float* __restrict__ Hfd, const float* __restrict__ Had,
                    const float* __restrict__ Hnn, const double* __restrict__ red_ff, int ff_stride,
                    const double* __restrict__ red_aff, long long* __restrict__ acc, int F)
{
    __shared__ double s_scale;
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_scale = affine_scale(red_ff, ff_stride, red_aff, F);
    __syncthreads();
    const double scale = s_scale;
    if (scale == 0.0 || t >= pb.T) return;
    const int n2 = 2 * (F - 1), n6 = 6 * (F - 1);
    unsigned long long* pa = reinterpret_cast<unsigned long long*>(acc);
    unsigned long long* aa = pa + (size_t)n6 * n2;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    const int n = t * kTile + lane;
    // 1 / H_dd of the solved system (H_dd = 0: a point without residuals)
    const float hn = Hnn[n];
    const float ih = hn > 0.0f ? 1.0f / (hn * pb.damp1) : 0.0f;
    for (int i = e0 + warp; i < e1; i += kAffWarps) {
        const Entry ei = pb.entries[i];
        const bool vi = (ei.mask >> lane) & 1u;
        const int ri = vi ? lane_rank(ei.mask, lane) : 0, nvi = __popc(ei.mask);
        float u[6], ai[2];
#pragma unroll
        for (int a = 0; a < 6; ++a) u[a] = vi ? Hfd[(size_t)ei.pair_off * 6 + ri + a * nvi] * ih : 0.0f;
#pragma unroll
        for (int a = 0; a < 2; ++a) ai[a] = vi ? Had[(size_t)ei.pair_off * 2 + ri + a * nvi] * ih : 0.0f;
        for (int j = e0; j < e1; ++j) {
            const Entry ej = pb.entries[j];
            const bool vj = (ej.mask >> lane) & 1u;
            const int rj = vj ? lane_rank(ej.mask, lane) : 0, nvj = __popc(ej.mask);
            float aj[2];
#pragma unroll
            for (int b = 0; b < 2; ++b) aj[b] = vj ? Had[(size_t)ej.pair_off * 2 + rj + b * nvj] : 0.0f;
            float v[16];
#pragma unroll
            for (int q = 0; q < 12; ++q) v[q] = u[q >> 1] * aj[q & 1];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[12 + q] = ai[q >> 1] * aj[q & 1];
            scatter_level<8>(v, lane, 16);
            scatter_level<4>(v, lane, 8);
            scatter_level<2>(v, lane, 4);
            scatter_level<1>(v, lane, 2);
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            if ((lane & 1) == 0) {
                const int q = lane >> 1;
                const unsigned long long x = (unsigned long long)llrint((double)v[0] * scale);
                if (q < 12)
                    atomicAdd(pa + (size_t)(6 * (ei.f - 1) + (q >> 1)) * n2 + 2 * (ej.f - 1) + (q & 1), x);
                else
                    atomicAdd(aa + (size_t)(2 * (ei.f - 1) + ((q - 12) >> 1)) * n2 + 2 * (ej.f - 1) + (q & 1), x);
            }
        }
    }
}

// A8 (8 nact x 8 nact, row-major, double-float): the pose rows of the
// assembled S over the active frames (compact order, as the 6 (F - 1)
// system's working copy), then the pair rows; grid-stride over elements.
__global__ void __launch_bounds__(256)
assemble_affine_kernel(const double* __restrict__ S, const double* __restrict__ red_ff, int ff_stride,
                       const double* __restrict__ red_aff, const long long* __restrict__ acc,
                       const int* __restrict__ cmap, int F, double damping, double prior,
                       dfloat* __restrict__ A8, const double* __restrict__ rhs, int rhs_stride, int rhs_off,
                       const double* __restrict__ yph)
{
    __shared__ int frame_of[1024];
    __shared__ double s_scale;
    const int nact = cmap[F], n6 = 6 * (F - 1), n2 = 2 * (F - 1), nc = 8 * nact, np = 6 * nact;
    for (int f = 1 + threadIdx.x; f < F; f += blockDim.x)
        if (cmap[f] >= 0) frame_of[cmap[f]] = f;
    if (threadIdx.x == 0) s_scale = affine_scale(red_ff, ff_stride, red_aff, F);
    __syncthreads();
    const double inv = s_scale > 0.0 ? 1.0 / s_scale : 0.0;  // a power of two: exact
    const long long* pa = acc;
    const long long* aa = acc + (size_t)n6 * n2;
    const double ld = 1.0 + damping;
    const size_t total = (size_t)nc * nc;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / nc), j = (int)(idx % nc);
        const bool pi = i < np, pj = j < np;
        const int fi = frame_of[pi ? i / 6 : (i - np) / 2], fj = frame_of[pj ? j / 6 : (j - np) / 2];
        const int a = pi ? i % 6 : (i - np) % 2, b = pj ? j % 6 : (j - np) % 2;
        double v;
        if (pi && pj) {
            v = S[(size_t)(6 * (fi - 1) + a) * n6 + 6 * (fj - 1) + b];
        } else if (pi) {
            v = -(double)pa[(size_t)(6 * (fi - 1) + a) * n2 + 2 * (fj - 1) + b] * inv;
            if (fi == fj) v += red_aff[(size_t)fi * kAffComp + 2 * a + b];
        } else if (pj) {
            v = -(double)pa[(size_t)(6 * (fj - 1) + b) * n2 + 2 * (fi - 1) + a] * inv;
            if (fi == fj) v += red_aff[(size_t)fi * kAffComp + 2 * b + a];
        } else {
            v = -(double)aa[(size_t)(2 * (fi - 1) + a) * n2 + 2 * (fj - 1) + b] * inv;
            if (fi == fj) {
                // H_aa = [[sum w0 I_0^2, sum w0 I_0], [sum w0 I_0, sum w0]],
                // + lambda sum w0 on the diagonal (the prior)
                const double* h = red_aff + (size_t)fi * kAffComp + 12;
                v += (a == b ? (h[2 * a] + prior * h[2]) * ld : h[1]);
            }
        }
        A8[idx] = df_from_double(v);
    }
    // FC: augmented row nc, b = -[y_theta; y_a], eliminated with the matrix
    if (rhs)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
            double y;
            if (j < np) {
                y = rhs[(size_t)frame_of[j / 6] * rhs_stride + rhs_off + j % 6];
            } else {
                const int g = frame_of[(j - np) / 2], b = (j - np) % 2;
                y = yph[(size_t)g * 5 + b] - yph[(size_t)g * 5 + 2 + b];
            }
            A8[(size_t)nc * nc + j] = df_from_double(-y);
        }
}

// One CTA per target frame (one bundle): warps 0-5 its pose rows of S8^-1,
// 6-7 its pair rows, 8-10 the anchor frame's translation rows (for the
// gauge constraint of ic_solve_kernel), each a double-float GEMV against
// y = [y_theta (compact, 6 per active frame); y_a (2 per active frame)],
// y_a = g_a - sum_n H_a g_n / H_dd (brightness columns 0-1 minus 2-3 of
// the frame reduction) - lambda W_f (ln alpha, beta). Then Dtheta = -that
// with the exact gauge constraint, written like ic_solve_kernel, and
// (da, db) = -that for the depth back-substitution and the pair update.
__global__ void __launch_bounds__(11 * 32)
ic_solve_affine_kernel(SolveArgs a, const dfloat* __restrict__ Sinv, const double* __restrict__ y,
                       const double* __restrict__ yph)
{
    extern __shared__ dfloat ys[];  // nc, then F ints
    __shared__ double dth[11], d[6];
    const int f = blockIdx.x + 1, lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int F = a.F;
    pdl_trigger();
    const int* cmap = a.cmap;
    const int nact = cmap[F], nc = 8 * nact, np = 6 * nact, kf = cmap[f], anchor = a.active[0];
    int* frame_of = reinterpret_cast<int*>(ys + nc);
    const int r = row < 6 ? 6 * kf + row
                          : row < 8 ? np + 2 * kf + row - 6 : (anchor > 0 ? 6 * cmap[anchor] + row - 8 : -1);
    for (int g = 1 + threadIdx.x; g < F; g += blockDim.x)
        if (cmap[g] >= 0) frame_of[cmap[g]] = g;
    pdl_wait();
    if (kf < 0) {
        if (row == 0) {
            if (lane < 6) d[lane] = 0.0;
            __syncwarp();
            write_update_lanes(a, f, d, lane);
            if (lane < 2) {
                a.dab64[2 * f + lane] = 0.0;
                a.dab2[2 * f + lane] = make_float2(0.0f, 0.0f);
            }
        }
        return;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        double v;
        if (c < np) {
            v = y[(size_t)frame_of[c / 6] * 6 + c % 6];
        } else {
            const int g = frame_of[(c - np) / 2], b = (c - np) % 2;
            v = yph[(size_t)g * 5 + b] - yph[(size_t)g * 5 + 2 + b];
            if (a.photo_prior > 0.0) {
                const double w = a.photo_prior * a.red_aff[(size_t)g * kAffComp + 14];
                const float* fcg = a.fc + (size_t)g * kFrameConst + kFrameAlpha;
                v -= w * (b == 0 ? log((double)fcg[0]) : (double)fcg[1]);
            }
        }
        ys[c] = df_from_double(v);
    }
    __syncthreads();
    if (r >= 0) {
        const dfloat* Sr = Sinv + (size_t)r * nc;
        DfAcc acc;
        for (int c = lane; c < nc; c += 32) acc.add_prod(Sr[c], ys[c]);
        float ss = acc.s, cc = acc.c;
        warp_sum_pair(ss, cc);
        if (lane == 0) dth[row] = -((double)ss + (double)cc);
    }
    __syncthreads();
    if (row != 0) return;
    const double* tanchor = a.tanchor;
    if (lane < 6) {
        double v = dth[lane];
        if (lane < 3 && anchor > 0) v = fma(-gauge_alpha(tanchor + 12 * anchor + 9, dth + 8), tanchor[12 * f + 9 + lane], v);
        d[lane] = v;
    }
    __syncwarp();
    const double da = dth[6], db = dth[7];
    const bool ok = __all_sync(0xffffffffu, lane >= 6 || isfinite(d[lane])) && isfinite(da) && isfinite(db) &&
                    1.0 + da > 0.0;
    if (!ok) {
        if (lane == 0) flag_error(a.err, 0, kErrNonFinite);
        if (lane < 6) d[lane] = 0.0;
        __syncwarp();
    }
    write_update_lanes(a, f, d, lane);
    if (lane < 2) {
        const double v = ok ? (lane == 0 ? da : db) : 0.0;
        const float hi = (float)v;
        a.dab64[2 * f + lane] = v;
        a.dab2[2 * f + lane] = make_float2(hi, (float)(v - (double)hi));
    }
}

cudaError_t launch_affine_schur(const DevProblem& pb, const float* Hfd, const float* Had, const float* Hnn,
                                const double* red_ff, int ff_stride, const double* red_aff, long long* acc,
                                int F, cudaStream_t st)
{
    if (F < 2 || F > 1024 || pb.T < 1) return cudaErrorInvalidValue;
    affine_schur_kernel<<<pb.T, kAffWarps * 32, 0, st>>>(pb, Hfd, Had, Hnn, red_ff, ff_stride, red_aff, acc, F);
    return cudaGetLastError();
}

cudaError_t launch_assemble_affine(const double* S, const double* red_ff, int ff_stride, const double* red_aff,
                                   const long long* acc, const int* cmap, int F, double damping, double prior,
                                   dfloat* A8, cudaStream_t st, const double* rhs, int rhs_stride, int rhs_off,
                                   const double* yph)
{
    if (F < 2 || F > 1024 || (rhs && !yph)) return cudaErrorInvalidValue;
    const int n8 = 8 * (F - 1);
    const int blocks = std::max(1, std::min(148, (n8 * n8 + 255) / 256));
    assemble_affine_kernel<<<blocks, 256, 0, st>>>(S, red_ff, ff_stride, red_aff, acc, cmap, F, damping, prior,
                                                   A8, rhs, rhs_stride, rhs_off, yph);
    return cudaGetLastError();
}

// FC: row nc of L8 holds D^-1 L^-1 b (b = -y), so the backward
// substitution gives Delta = -S8^-1 y; then the pose part takes the exact
// gauge constraint and every frame's update is written (warp per frame),
// the pair part (da, db) for the depth back-substitution and the additive
// pair update of the next depth update. One CTA.
constexpr int kFcAffWarps = 32;

__global__ void __launch_bounds__(kFcAffWarps * 32)
fc_solve_affine_kernel(SolveArgs a, const dfloat* __restrict__ L, const dfloat* __restrict__ Linv)
{
    extern __shared__ dfloat xs[];  // nc, then 8 (F - 1) doubles
    __shared__ dfloat tb[kLdlBlock];
    __shared__ double s_alpha;
    __shared__ double dsh[kFcAffWarps][6];
    const int F = a.F;
    const int* cmap = a.cmap;
    const int nact = cmap[F], nc = 8 * nact, np = 6 * nact, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* x = reinterpret_cast<double*>(xs + 8 * (F - 1));
    for (int i = tid; i < nc; i += blockDim.x) xs[i] = L[(size_t)nc * nc + i];
    __syncthreads();
    ldl_backward_smem(L, Linv, nc, xs, tb);
    // back to frame order, 8 per frame [pose 6, pair 2]; frames left out of
    // the system get no update
    for (int i = tid; i < 8 * (F - 1); i += blockDim.x) {
        const int f = i / 8 + 1, q = i % 8, k = cmap[f];
        x[i] = k < 0 ? 0.0 : df_to_double(q < 6 ? xs[6 * k + q] : xs[np + 2 * k + q - 6]);
    }
    __syncthreads();
    const int anchor = a.active[0];
    const double* tanchor = a.tanchor;
    if (tid == 0) {
        double dta[3] = {0.0, 0.0, 0.0};
        if (anchor > 0)
            for (int q = 0; q < 3; ++q) dta[q] = x[8 * (anchor - 1) + q];
        s_alpha = anchor > 0 ? gauge_alpha(tanchor + 12 * anchor + 9, dta) : 0.0;
    }
    __syncthreads();
    for (int f = warp; f < F; f += blockDim.x >> 5) {
        double* d = dsh[warp];
        if (lane < 6) {
            double v = f > 0 ? x[8 * (f - 1) + lane] : 0.0;
            if (lane < 3 && f > 0 && a.active[f]) v = fma(-s_alpha, tanchor[12 * f + 9 + lane], v);
            d[lane] = v;
        }
        __syncwarp();
        double dab = (f > 0 && lane < 2) ? x[8 * (f - 1) + 6 + lane] : 0.0;
        const bool ok = __all_sync(0xffffffffu, (lane >= 6 || isfinite(d[lane])) && isfinite(dab));
        if (!ok) {
            if (lane == 0) flag_error(a.err, 0, kErrNonFinite);
            if (lane < 6) d[lane] = 0.0;
            dab = 0.0;
            __syncwarp();
        }
        write_update_lanes(a, f, d, lane);
        if (lane < 2) {
            const float hi = (float)dab;
            a.dab64[2 * f + lane] = dab;
            a.dab2[2 * f + lane] = make_float2(hi, (float)(dab - (double)hi));
        }
        __syncwarp();
    }
}

cudaError_t launch_fc_solve_affine(const SolveArgs& a, const dfloat* L8, const dfloat* Linv8, cudaStream_t st)
{
    if (a.F < 2 || a.F > 1024 || a.B != 1) return cudaErrorInvalidValue;
    const size_t smem = (sizeof(dfloat) + sizeof(double)) * 8 * (a.F - 1);
    fc_solve_affine_kernel<<<1, kFcAffWarps * 32, smem, st>>>(a, L8, Linv8);
    return cudaGetLastError();
}

cudaError_t launch_ic_solve_affine(const SolveArgs& a, const dfloat* Sinv8, const double* y, const double* yph,
                                   cudaStream_t st)
{
    if (a.F < 2 || a.F > 1024 || a.B != 1) return cudaErrorInvalidValue;
    const size_t smem = sizeof(dfloat) * 8 * (a.F - 1) + sizeof(int) * a.F;
    return launch_pdl(ic_solve_affine_kernel, a.F - 1, 11 * 32, smem, st, a, Sinv8, y, yph);
}

cudaError_t affine_setup()
{
    // up to 1023 target frames: 8 * 1023 double-float values + the frame
    // map, or + as many doubles
    cudaError_t e = cudaFuncSetAttribute(ic_solve_affine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(dfloat) * 8 * 1023 + sizeof(int) * 1024));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fc_solve_affine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((sizeof(dfloat) + sizeof(double)) * 8 * 1023));
}

}  // namespace pba
