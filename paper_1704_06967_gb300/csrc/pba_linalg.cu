// Reduced camera system (Sec. 3.5 step 3): Schur complement of the point
// block, assembly with the scale-gauge prior, FP64 Cholesky factorisation,
// explicit inverse (IC: factorised once, applied every iteration as a GEMV),
// triangular solves (FC: every iteration), and the FP64 pose updates of
// Sec. 3.6 (IC) and of the boxplus operator (FC).
#include "pba_kernels.cuh"

namespace pba {

// ---------------------------------------------------------------------------
// S_off[f][g] = sum_n H_fd(n,f) H_fd(n,g)^T / H_dd(n) for one frame pair per
// CTA (f <= g, both target frames). Warps walk the tiles; a lane adds its
// point when it is visible in both frames. The products and sums are FP64:
// S = blockdiag(H_ff) - S_off cancels along the near-null directions of the
// reduced system, where FP32 products would lose cond(S) * 2^-24. Fixed-order
// reduction: deterministic.
// ---------------------------------------------------------------------------
constexpr int kSchurWarps = 4;

__global__ void __launch_bounds__(32 * kSchurWarps)
schur_offdiag_kernel(DevProblem pb, const float* Hfd, const float* Hnn, const int2* pairs,
                     double* Soff, int n6)
{
    __shared__ double red[kSchurWarps][36];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 fg = pairs[blockIdx.x];
    const int f = fg.x, g = fg.y;
    double s[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) s[k] = 0.0;
    for (int t = warp; t < pb.T; t += kSchurWarps) {
        const int ea = pb.ent_of[(size_t)t * pb.F + f];
        const int eb = pb.ent_of[(size_t)t * pb.F + g];
        if (ea < 0 || eb < 0) continue;
        const Entry A = pb.entries[ea], B = pb.entries[eb];
        if (!((A.mask & B.mask) >> lane & 1u)) continue;
        const int n = t * kTile + lane;
        const float h = Hnn[n];
        if (!(h > 0.0f)) continue;
        const double ih = 1.0 / (double)h;
        const int na = __popc(A.mask), ra = __popc(A.mask & ((1u << lane) - 1u));
        const int nb = __popc(B.mask), rb = __popc(B.mask & ((1u << lane) - 1u));
        const float* pa = Hfd + (size_t)A.pair_off * 6 + ra;
        const float* pbp = Hfd + (size_t)B.pair_off * 6 + rb;
        double ha[6], hb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            ha[k] = (double)pa[k * na];
            hb[k] = (double)pbp[k * nb];
        }
        // (h_a h_b) / H_dd: the product commutes, so diagonal blocks come out
        // exactly symmetric
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) s[6 * a + b] = fma(ha[a] * hb[b], ih, s[6 * a + b]);
    }
    // fixed-order reduction: lanes (butterfly), then warps
#pragma unroll
    for (int k = 0; k < 36; ++k) {
        double v = warp_sum1d(s[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 36 && (f != g || threadIdx.x / 6 <= threadIdx.x % 6)) {
        const int k = threadIdx.x, a = k / 6, b = k % 6;
        double v = 0.0;
        for (int w = 0; w < kSchurWarps; ++w) v += red[w][k];
        const int i = 6 * (f - 1) + a, j = 6 * (g - 1) + b;
        Soff[(size_t)i * n6 + j] = v;
        Soff[(size_t)j * n6 + i] = v;
    }
}

cudaError_t launch_schur_offdiag(const DevProblem& pb, const float* Hfd, const float* Hnn,
                                 const int2* frame_pairs, int n_pairs, double* Soff,
                                 cudaStream_t st)
{
    if (n_pairs == 0) return cudaSuccess;
    schur_offdiag_kernel<<<n_pairs, 32 * kSchurWarps, 0, st>>>(pb, Hfd, Hnn, frame_pairs, Soff,
                                                               6 * (pb.F - 1));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S = blockdiag(H_ff) - S_off, then: frames without residuals (zero H_ff
// trace) get an identity block; mu = mean diagonal over the active frames;
// the prior gauge_w * mu * that that^T goes on the translation block of the
// first active frame (that = unit translation of that frame in anchor_t).
// H_ff comes as 21 upper-triangle values per frame at Hff[f*stride].
// active[f] (f >= 1) receives the frame flags, active[0] the anchor frame.
// ---------------------------------------------------------------------------
__global__ void assemble_S_kernel(int F, const double* Hff, int stride, const double* Soff,
                                  const double* anchor_t, double gauge_w, double* S, int* active)
{
    extern __shared__ double sh[];
    const int n6 = 6 * (F - 1);
    double* diag = sh;  // n6
    __shared__ int s_anchor;
    __shared__ double s_mu;
    for (int f = 1 + threadIdx.x; f < F; f += blockDim.x) {
        const double* h = Hff + (size_t)f * stride;
        // trace of the 6x6 block from the upper-triangle layout
        double tr = 0.0;
        int q = 0;
        for (int a = 0; a < 6; ++a)
            for (int b = a; b < 6; ++b, ++q)
                if (a == b) tr += h[q];
        active[f] = tr > 0.0;
    }
    __syncthreads();
    for (size_t idx = threadIdx.x; idx < (size_t)n6 * n6; idx += blockDim.x) {
        const int i = (int)(idx / n6), j = (int)(idx % n6);
        const int fi = i / 6 + 1, fj = j / 6 + 1;
        double v;
        if (!active[fi] || !active[fj]) {
            v = (i == j) ? 1.0 : 0.0;
        } else {
            v = -Soff[idx];
            if (fi == fj) {
                int a = i % 6, b = j % 6;
                if (a > b) { int tmp = a; a = b; b = tmp; }
                const int q = a * 6 - a * (a - 1) / 2 + (b - a);
                v += Hff[(size_t)fi * stride + q];
            }
        }
        S[idx] = v;
        if (i == j) diag[i] = active[fi] ? v : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mu = 0.0;
        int cnt = 0, anchor = -1;
        for (int f = 1; f < F; ++f) {
            if (!active[f]) continue;
            if (anchor < 0) anchor = f;
            for (int a = 0; a < 6; ++a) mu += diag[6 * (f - 1) + a];
            cnt += 6;
        }
        s_mu = cnt ? gauge_w * mu / cnt : 0.0;
        s_anchor = anchor;
        active[0] = anchor;  // first active frame, -1 if none
    }
    __syncthreads();
    if (s_anchor > 0 && threadIdx.x < 9) {
        const double* ta = anchor_t + 12 * s_anchor + 9;
        const double nt = sqrt(ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2]);
        if (nt > 0.0) {
            const int a = threadIdx.x / 3, b = threadIdx.x % 3;
            const int base = 6 * (s_anchor - 1);
            S[(size_t)(base + a) * n6 + base + b] += s_mu * ((ta[a] / nt) * (ta[b] / nt));
        }
    }
}

cudaError_t launch_assemble_S(int F, const double* Hff, int hff_stride, const double* Soff,
                              const double* anchor_t, double gauge_w, double* S, int* active,
                              cudaStream_t st)
{
    const int n6 = 6 * (F - 1);
    assemble_S_kernel<<<1, 1024, sizeof(double) * n6, st>>>(F, Hff, hff_stride, Soff, anchor_t,
                                                             gauge_w, S, active);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 Cholesky A = L L^T in place (lower triangle, row-major), one CTA,
// left-looking by columns. A non-positive pivot sets kErrNotPD and is
// replaced by 1 so the factorisation finishes without non-finite values.
// ---------------------------------------------------------------------------
constexpr int kCholThreads = 1024;

__global__ void __launch_bounds__(kCholThreads) cholesky_kernel(double* A, int n, int* err)
{
    __shared__ double red[kCholThreads / 32];
    __shared__ double s_ljj;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < n; ++j) {
        const double* Lj = A + (size_t)j * n;
        double p = 0.0;
        for (int k = tid; k < j; k += kCholThreads) p = fma(Lj[k], Lj[k], p);
        p = warp_sum1d(p);
        if (lane == 0) red[warp] = p;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < kCholThreads / 32; ++w) s += red[w];
            double v = A[(size_t)j * n + j] - s;
            if (!(v > 0.0)) {
                atomicOr(err, kErrNotPD);
                v = 1.0;
            }
            const double l = sqrt(v);
            A[(size_t)j * n + j] = l;
            s_ljj = l;
        }
        __syncthreads();
        const double ljj = s_ljj;
        for (int i = j + 1 + tid; i < n; i += kCholThreads) {
            const double* Li = A + (size_t)i * n;
            double t = Li[j];
            for (int k = 0; k < j; ++k) t = fma(-Li[k], Lj[k], t);
            A[(size_t)i * n + j] = t / ljj;
        }
        __syncthreads();
    }
}

cudaError_t launch_cholesky(double* A, int n, int* err, cudaStream_t st)
{
    cholesky_kernel<<<1, kCholThreads, 0, st>>>(A, n, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S^-1 from its Cholesky factor: CTA c solves L y = e_c, L^T x = y for
// column c (forward substitution starts at row c).
// ---------------------------------------------------------------------------
__global__ void chol_inverse_kernel(const double* L, double* Sinv, int n)
{
    extern __shared__ double y[];
    const int c = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) y[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = c; k < n; ++k) {
        const double yk = y[k] / L[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) y[k] = yk;
        for (int i = k + 1 + tid; i < n; i += blockDim.x) y[i] = fma(-L[(size_t)i * n + k], yk, y[i]);
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        const double xk = y[k] / L[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) y[k] = xk;
        for (int i = tid; i < k; i += blockDim.x) y[i] = fma(-L[(size_t)k * n + i], xk, y[i]);
        __syncthreads();
    }
    for (int i = tid; i < n; i += blockDim.x) Sinv[(size_t)i * n + c] = y[i];
}

cudaError_t launch_chol_inverse(const double* L, double* Sinv, int n, cudaStream_t st)
{
    chol_inverse_kernel<<<n, 256, sizeof(double) * n, st>>>(L, Sinv, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pose updates (FP64)
// ---------------------------------------------------------------------------
__device__ void write_frame(const SolveArgs& a, int f, const double* Rn, const double* tn,
                            const double* dth)
{
    double* pose = a.poses64 + 12 * f;
    float* prev = a.fc_prev + 12 * f;
    for (int i = 0; i < 12; ++i) prev[i] = (float)pose[i];
    for (int i = 0; i < 9; ++i) pose[i] = Rn[i];
    for (int i = 0; i < 3; ++i) pose[9 + i] = tn[i];
    frame_consts(pose, a.pat, a.P, a.fx, a.fy, a.fc + (size_t)f * kFrameConst);
    double q = 0.0;
    for (int k = 0; k < 6; ++k) {
        a.dtheta64[6 * f + k] = dth[k];
        a.dtheta32[6 * f + k] = (float)dth[k];
        q += dth[k] * dth[k];
    }
    a.dthsq[f] = (float)q;
}

// Sec. 3.6: R <- R R0^T exp(omega)^T R0, t <- t - R R0^T Dt (old R on the right).
__device__ void ic_pose_update(const SolveArgs& a, int f, const double* dth)
{
    const double* pose = a.poses64 + 12 * f;
    const double* p0 = a.poses0 + 12 * f;
    double mw[3] = {-dth[3], -dth[4], -dth[5]};
    double Et[9], R0t[9], A[9], B[9], Rn[9], tn[3];
    so3_exp_d(mw, Et);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R0t[3 * i + j] = p0[3 * j + i];
    mat3_mul_d(pose, R0t, A);
    mat3_mul_d(A, Et, B);
    mat3_mul_d(B, p0, Rn);
    for (int i = 0; i < 3; ++i)
        tn[i] = pose[9 + i] - (A[3 * i] * dth[0] + A[3 * i + 1] * dth[1] + A[3 * i + 2] * dth[2]);
    write_frame(a, f, Rn, tn, dth);
}

// Boxplus: T <- exp([upsilon, omega]) T.
__device__ void fc_pose_update(const SolveArgs& a, int f, const double* dth)
{
    const double* pose = a.poses64 + 12 * f;
    double E[9], V[9], Rn[9], tn[3];
    so3_exp_d(dth + 3, E);
    so3_left_jacobian_d(dth + 3, V);
    mat3_mul_d(E, pose, Rn);
    for (int i = 0; i < 3; ++i)
        tn[i] = E[3 * i] * pose[9] + E[3 * i + 1] * pose[10] + E[3 * i + 2] * pose[11] +
                V[3 * i] * dth[0] + V[3 * i + 1] * dth[1] + V[3 * i + 2] * dth[2];
    write_frame(a, f, Rn, tn, dth);
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
// the gauge constraint), then the frame's pose update.
__global__ void ic_solve_update_kernel(SolveArgs a, const double* Sinv, const double* y,
                                       int y_stride, int y_off)
{
    __shared__ double dth[9];
    const int f = blockIdx.x + 1, lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int n6 = a.n6;
    const int anchor = a.active[0];
    const int rr = row < 6 ? 6 * (f - 1) + row : (anchor > 0 ? 6 * (anchor - 1) + row - 6 : -1);
    if (rr >= 0) {
        const double* Sr = Sinv + (size_t)rr * n6;
        double s = 0.0;
        for (int c = lane; c < n6; c += 32) s = fma(Sr[c], y[(size_t)(c / 6 + 1) * y_stride + y_off + c % 6], s);
        s = warp_sum1d(s);
        if (lane == 0) dth[row] = -s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d[6];
        bool ok = true;
        for (int k = 0; k < 6; ++k) {
            d[k] = dth[k];
            ok = ok && isfinite(d[k]);
        }
        if (anchor > 0 && a.active[f]) {
            const double* ta = a.tanchor + 12 * anchor + 9;
            const double alpha = gauge_alpha(ta, dth + 6);
            const double* tf = a.tanchor + 12 * f + 9;
            for (int k = 0; k < 3; ++k) d[k] -= alpha * tf[k];
        }
        if (!ok) {
            atomicOr(a.err, kErrNonFinite);
            for (int k = 0; k < 6; ++k) d[k] = 0.0;
        }
        ic_pose_update(a, f, d);
    }
}

cudaError_t launch_ic_solve_update(const SolveArgs& a, const double* Sinv, const double* y,
                                   int y_stride, int y_off, cudaStream_t st)
{
    ic_solve_update_kernel<<<a.F - 1, 9 * 32, 0, st>>>(a, Sinv, y, y_stride, y_off);
    return cudaGetLastError();
}

// FC: solve L L^T Dtheta = -y (one CTA, column-oriented substitutions), the
// exact gauge constraint, then every frame's boxplus update.
__global__ void __launch_bounds__(1024) fc_solve_update_kernel(SolveArgs a, const double* L,
                                                               const double* y, int y_stride,
                                                               int y_off)
{
    extern __shared__ double x[];
    const int n = a.n6, tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) x[i] = -y[(size_t)(i / 6 + 1) * y_stride + y_off + i % 6];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double xk = x[k] / L[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) x[k] = xk;
        for (int i = k + 1 + tid; i < n; i += blockDim.x) x[i] = fma(-L[(size_t)i * n + k], xk, x[i]);
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        const double xk = x[k] / L[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) x[k] = xk;
        for (int i = tid; i < k; i += blockDim.x) x[i] = fma(-L[(size_t)k * n + i], xk, x[i]);
        __syncthreads();
    }
    __shared__ double s_alpha;
    if (tid == 0) {
        const int anchor = a.active[0];
        s_alpha = anchor > 0 ? gauge_alpha(a.tanchor + 12 * anchor + 9, x + 6 * (anchor - 1)) : 0.0;
    }
    __syncthreads();
    for (int f = 1 + tid; f < a.F; f += blockDim.x) {
        double d[6];
        bool ok = true;
        for (int k = 0; k < 6; ++k) {
            d[k] = x[6 * (f - 1) + k];
            ok = ok && isfinite(d[k]);
        }
        if (a.active[f])
            for (int k = 0; k < 3; ++k) d[k] -= s_alpha * a.tanchor[12 * f + 9 + k];
        if (!ok) {
            atomicOr(a.err, kErrNonFinite);
            for (int k = 0; k < 6; ++k) d[k] = 0.0;
        }
        fc_pose_update(a, f, d);
    }
}

cudaError_t launch_fc_solve_update(const SolveArgs& a, const double* L, const double* y,
                                   int y_stride, int y_off, cudaStream_t st)
{
    fc_solve_update_kernel<<<1, 1024, sizeof(double) * a.n6, st>>>(a, L, y, y_stride, y_off);
    return cudaGetLastError();
}

}  // namespace pba
