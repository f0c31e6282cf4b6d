// Residual-pass kernels: IC precompute (Sec. 3.5: J, W_0, H blocks), the IC
// iteration pass (Sec. 3.5 steps 1-2 plus the Schur right-hand side and the
// depth back-substitution of the previous step), the FC linearisation pass
// and the fixed-order per-frame reductions.
//
// One CTA owns one tile of 32 points (lane = point). Its warps take the
// tile's entries (target frames that see at least one of the tile's points)
// round-robin, so every sum over a point's frames completes inside the CTA
// and every per-frame sum is written once per entry, then reduced across
// entries in a fixed order: results are deterministic run to run.
#include "pba_kernels.cuh"

namespace pba {

__device__ __forceinline__ int lane_rank(unsigned mask, int lane)
{
    return __popc(mask & ((1u << lane) - 1u));
}

// Depth back-substitution of the previous step (Sec. 3.5 step 3 for the
// point block): Dd_n = -(g_n + sum_f H_fd^T Dtheta_f) / H_dd, then the IC
// rule d <- d (d0 - Dd)/d0 (Sec. 3.6) or the FC rule d <- d + Dd. Returns the
// updated depth of the lane's point (rounded to FP32, as the pass uses it);
// all warps of the CTA call it.
__device__ double depth_backsub(const DevProblem& pb, const DepthState& ds, const float* s_dth,
                                float* s_red, int t, int e0, int e1, bool ic_rule, float& ddsq)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    float s = 0.0f;
    for (int e = e0 + warp; e < e1; e += kPassWarps) {
        const Entry en = pb.entries[e];
        if ((en.mask >> lane) & 1u) {
            const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
            const float* h = ds.Hfd + (size_t)en.pair_off * 6 + rank;
            const float* dt = s_dth + 6 * en.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s = fmaf(h[k * nvis], dt[k], s);
        }
    }
    s_red[warp * 32 + lane] = s;
    __syncthreads();
    double d = ds.d64[n];
    if (warp == 0) {
        float tot = 0.0f;
        for (int w = 0; w < kPassWarps; ++w) tot += s_red[w * 32 + lane];
        const float hnn = ds.Hnn[n];
        double dd = 0.0;
        if (pb.valid_pt[n] && hnn > 0.0f) {
            dd = -((double)ds.gn[n] + (double)tot) / (double)hnn;
            double dn = ic_rule ? d * (ds.d0_64[n] - dd) / ds.d0_64[n] : d + dd;
            if (isfinite(dn)) {
                d = dn;
                ds.d64[n] = d;
            } else {
                atomicOr(ds.err, kErrNonFinite);
            }
        }
        ds.dd_last[n] = dd;
        ddsq = (float)(dd * dd);
        s_red[kPassWarps * 32 + lane] = (float)d;
    }
    __syncthreads();
    // every warp continues with the updated depth (FP32 is what the pass uses)
    return (double)s_red[kPassWarps * 32 + lane];
}

// Block-wide statistics of a tile: sums of energy, r^2, count, dd^2 and the
// max displacement; written once per tile.
__device__ void tile_stats_write(TileStats* out, int t, float energy, float sumsq, float cnt,
                                 float maxdisp, float ddsq, float* s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    energy = warp_sum1(energy);
    sumsq = warp_sum1(sumsq);
    cnt = warp_sum1(cnt);
    ddsq = warp_sum1(ddsq);
    maxdisp = warp_max1(maxdisp);
    __syncthreads();
    if (lane == 0) {
        s_red[warp * 5 + 0] = energy;
        s_red[warp * 5 + 1] = sumsq;
        s_red[warp * 5 + 2] = cnt;
        s_red[warp * 5 + 3] = maxdisp;
        s_red[warp * 5 + 4] = ddsq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        TileStats ts = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < kPassWarps; ++w) {
            ts.energy += s_red[w * 5 + 0];
            ts.sumsq += s_red[w * 5 + 1];
            ts.count += s_red[w * 5 + 2];
            ts.maxdisp = fmaxf(ts.maxdisp, s_red[w * 5 + 3]);
            ts.ddsq += s_red[w * 5 + 4];
        }
        out[t] = ts;
    }
}

// Pattern-centre reprojection displacement between the previous and the
// current parameters of one (point, frame) (convergence rule of Sec. 4.1).
__device__ __forceinline__ float centre_disp(const DevProblem& pb, const float* c, const float* cp,
                                             float2 xc, float d, float dprev)
{
    float qx = fmaf(c[0], xc.x, fmaf(c[1], xc.y, fmaf(d, c[9], c[2])));
    float qy = fmaf(c[3], xc.x, fmaf(c[4], xc.y, fmaf(d, c[10], c[5])));
    float qz = fmaf(c[6], xc.x, fmaf(c[7], xc.y, fmaf(d, c[11], c[8])));
    float px = fmaf(cp[0], xc.x, fmaf(cp[1], xc.y, fmaf(dprev, cp[9], cp[2])));
    float py = fmaf(cp[3], xc.x, fmaf(cp[4], xc.y, fmaf(dprev, cp[10], cp[5])));
    float pz = fmaf(cp[6], xc.x, fmaf(cp[7], xc.y, fmaf(dprev, cp[11], cp[8])));
    float du = pb.fx * (qx / qz - px / pz), dv = pb.fy * (qy / qz - py / pz);
    return sqrtf(du * du + dv * dv);
}

// Shared-memory carve-up of the pass kernels (floats).
struct PassSmem {
    float* fc;    // F * kFrameConst current constants
    float* prev;  // F * 12 previous R|t
    float* dth;   // F * 6 last update
    float* ent;   // F * 32 per local entry accumulators
    float* red;   // kPassWarps * 32 + 32 scratch
    __device__ PassSmem(float* s, int F)
    {
        fc = s;
        prev = fc + F * kFrameConst;
        dth = prev + F * 12;
        ent = dth + F * 6;
        red = ent + F * kEntryPartial;
    }
};

size_t pass_smem_bytes(int F)
{
    return sizeof(float) * ((size_t)F * (kFrameConst + 12 + 6 + kEntryPartial) + 3 * kPassWarps * 32 + 64);
}

__device__ void load_frame_smem(const PassSmem& sm, const FrameState& fs, int F, bool prev,
                                bool dth)
{
    for (int i = threadIdx.x; i < F * kFrameConst; i += blockDim.x) sm.fc[i] = fs.fc[i];
    if (prev)
        for (int i = threadIdx.x; i < F * 12; i += blockDim.x) sm.prev[i] = fs.fc_prev[i];
    if (dth)
        for (int i = threadIdx.x; i < F * 6; i += blockDim.x) sm.dth[i] = fs.dtheta32[i];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// IC precompute (Sec. 3.4-3.5) at the current parameters p_0, evaluated in
// FP64 once and stored in FP32. Per residual: template gradient (central
// differences at the integer template pixel), the proxy-warp Jacobian row in
// pixel units
//   c = (1/zbar0) (g_u f_x, g_v f_y, -(g_u f_x x + g_v f_y y)),
//   m = zbar0 R0 c - e_z (t0 . R0 c)            (m = M^T c),
//   J = [d0 m, (R0 x~) x m, m . t0],
// the residual and Huber weight at p_0 (J = 0 when invalid there), and the
// H blocks: H_fd per pair, H_dd per point, H_ff (21 unique) per entry.
// ---------------------------------------------------------------------------
template <int PMAX>
__global__ void __launch_bounds__(kTile * kPassWarps)
ic_precompute_kernel(DevProblem pb, const double* poses0, DepthState ds, IcStore ic,
                     float* ent_part, TileStats* tstats)
{
    extern __shared__ float smraw[];
    double* s_pose = reinterpret_cast<double*>(smraw);   // F * 12 FP64 poses at p_0
    float* s_red = smraw + 2 * 12 * pb.F;
    for (int i = threadIdx.x; i < 12 * pb.F; i += blockDim.x) s_pose[i] = poses0[i];
    __syncthreads();
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    const int P = pb.P, NC = (7 * P + 3) / 4;
    const double d0 = ds.d64[n];
    const double fx = pb.fx, fy = pb.fy, cx = pb.cx, cy = pb.cy;
    const int ux = pb.uvs[2 * n], uy = pb.uvs[2 * n + 1];
    float I0[PMAX], gu[PMAX], gv[PMAX];
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        if (j < P) {
            I0[j] = pb.I0p[((size_t)t * P + j) * kTile + lane];
            const int px = ux + pb.pat[2 * j], py = uy + pb.pat[2 * j + 1];
            const size_t b = (size_t)py * pb.pitch + px;
            gu[j] = 0.5f * (load_px(pb.img, pb.dtype, b + 1) - load_px(pb.img, pb.dtype, b - 1));
            gv[j] = 0.5f * (load_px(pb.img, pb.dtype, b + pb.pitch) -
                            load_px(pb.img, pb.dtype, b - pb.pitch));
        }
    }
    float hnn = 0.0f, energy = 0.0f, sumsq = 0.0f, cnt = 0.0f;
    for (int e = e0 + warp; e < e1; e += kPassWarps) {
        const Entry en = pb.entries[e];
        const double* R = s_pose + 12 * en.f;
        const double* t0 = R + 9;
        float hff[21];
#pragma unroll
        for (int k = 0; k < 21; ++k) hff[k] = 0.0f;
        if ((en.mask >> lane) & 1u) {
            const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
            float Jr[7 * PMAX + 4];
            double hfd[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < PMAX; ++j) {
                if (j >= P) break;
                float* J = Jr + 7 * j;
                const double x = (ux + pb.pat[2 * j] - cx) / fx;
                const double y = (uy + pb.pat[2 * j + 1] - cy) / fy;
                const double a0 = R[0] * x + R[1] * y + R[2];
                const double a1 = R[3] * x + R[4] * y + R[5];
                const double a2 = R[6] * x + R[7] * y + R[8];
                const double qx = a0 + d0 * t0[0], qy = a1 + d0 * t0[1], qz = a2 + d0 * t0[2];
                bool valid = qz > 0.0;
                float val = 0.f, wa, wb;
                int bx, by;
                if (valid) {
                    const float u = (float)(fx * qx / qz + cx), v = (float)(fy * qy / qz + cy);
                    valid = bilinear(pb, en.f, u, v, val, wa, wb, bx, by);
                }
                if (!valid) {
#pragma unroll
                    for (int k = 0; k < 7; ++k) J[k] = 0.0f;
                    continue;
                }
                const float r0 = I0[j] - val;
                const double w0 = (double)huber_w(r0, pb.huber_k);
                energy += huber_rho(r0, pb.huber_k);
                sumsq += r0 * r0;
                cnt += 1.0f;
                const double zb = qz / d0;
                const double gx = (double)gu[j] * fx, gy = (double)gv[j] * fy;
                const double c0 = gx / zb, c1 = gy / zb, c2 = -(gx * x + gy * y) / zb;
                const double cp0 = R[0] * c0 + R[1] * c1 + R[2] * c2;
                const double cp1 = R[3] * c0 + R[4] * c1 + R[5] * c2;
                const double cp2 = R[6] * c0 + R[7] * c1 + R[8] * c2;
                const double tc = t0[0] * cp0 + t0[1] * cp1 + t0[2] * cp2;
                const double m0 = zb * cp0, m1 = zb * cp1, m2 = zb * cp2 - tc;
                double Jd[7];
                Jd[0] = d0 * m0;
                Jd[1] = d0 * m1;
                Jd[2] = d0 * m2;
                Jd[3] = a1 * m2 - a2 * m1;
                Jd[4] = a2 * m0 - a0 * m2;
                Jd[5] = a0 * m1 - a1 * m0;
                Jd[6] = m0 * t0[0] + m1 * t0[1] + m2 * t0[2];
                // H from the stored (FP32-rounded) row, so H = J^T W0 J holds
                // exactly for the J the iterations use
#pragma unroll
                for (int k = 0; k < 7; ++k) J[k] = (float)Jd[k];
                int q = 0;
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const double wja = w0 * (double)J[a];
#pragma unroll
                    for (int b = a; b < 6; ++b) {
                        hff[q] += (float)(wja * (double)J[b]);
                        ++q;
                    }
                    hfd[a] += wja * (double)J[6];
                }
                hnn += (float)(w0 * (double)J[6] * (double)J[6]);
            }
#pragma unroll
            for (int k = 0; k < 7 * PMAX + 4; ++k)
                if (k >= 7 * P) Jr[k] = 0.0f;
            float4* dst = ic.J4 + (size_t)en.pair_off * NC + rank;
#pragma unroll
            for (int ch = 0; ch < (7 * PMAX + 3) / 4; ++ch)
                if (ch < NC)
                    dst[(size_t)ch * nvis] =
                        make_float4(Jr[4 * ch], Jr[4 * ch + 1], Jr[4 * ch + 2], Jr[4 * ch + 3]);
            float* hd = ic.Hfd + (size_t)en.pair_off * 6 + rank;
#pragma unroll
            for (int k = 0; k < 6; ++k) hd[k * nvis] = (float)hfd[k];
        }
        warp_sum<21>(hff);
        if (lane == 0) {
            float* out = ent_part + (size_t)e * kEntryPartial;
#pragma unroll
            for (int k = 0; k < 21; ++k) out[k] = hff[k];
        }
    }
    s_red[warp * 32 + lane] = hnn;
    __syncthreads();
    if (warp == 0) {
        float tot = 0.0f;
        for (int w = 0; w < kPassWarps; ++w) tot += s_red[w * 32 + lane];
        ic.Hnn[n] = pb.valid_pt[n] ? tot : 0.0f;
    }
    tile_stats_write(tstats, t, energy, sumsq, cnt, 0.0f, 0.0f, s_red);
}

// ---------------------------------------------------------------------------
// IC iteration pass (Sec. 3.5 steps 1-2): prologue = depth back-substitution
// and update of the previous step; main = warp, bilinear sample, residual,
// Huber weight, g_f += J_theta w r and g_n += J_d w r; epilogue = Schur
// right-hand side y_f = g_f - sum_n H_fd g_n / H_dd per entry.
// kAccum = false evaluates statistics only (after the last step).
// ---------------------------------------------------------------------------
template <int PMAX, bool kAccum>
__global__ void __launch_bounds__(kTile * kPassWarps)
ic_pass_kernel(DevProblem pb, FrameState fs, DepthState ds, IcStore ic, float* ent_part,
               TileStats* tstats, int apply, int have_prev)
{
    extern __shared__ float smraw[];
    PassSmem sm(smraw, pb.F);
    load_frame_smem(sm, fs, pb.F, have_prev, apply);
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    const int P = pb.P, NC = (7 * P + 3) / 4;
    float ddsq = 0.0f;
    const float dprev = (float)ds.d64[n];
    float d = dprev;
    if (apply) d = (float)depth_backsub(pb, ds, sm.dth, sm.red, t, e0, e1, true, ddsq);
    const float2 xc = pb.xn[n];
    float I0[PMAX];
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
        if (j < P) I0[j] = pb.I0p[((size_t)t * P + j) * kTile + lane];
    float gpart = 0.0f, energy = 0.0f, sumsq = 0.0f, cnt = 0.0f, maxdisp = 0.0f;
    const float k = pb.huber_k;
    for (int e = e0 + warp; e < e1; e += kPassWarps) {
        const Entry en = pb.entries[e];
        const float* c = sm.fc + en.f * kFrameConst;
        float acc[6] = {0, 0, 0, 0, 0, 0};
        if ((en.mask >> lane) & 1u) {
            const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
            float Jr[kAccum ? 7 * PMAX + 4 : 4];
            if (kAccum) {
                const float4* src = ic.J4 + (size_t)en.pair_off * NC + rank;
#pragma unroll
                for (int ch = 0; ch < (7 * PMAX + 3) / 4; ++ch) {
                    if (ch < NC) {
                        const float4 v = __ldg(src + (size_t)ch * nvis);
                        Jr[4 * ch] = v.x;
                        Jr[4 * ch + 1] = v.y;
                        Jr[4 * ch + 2] = v.z;
                        Jr[4 * ch + 3] = v.w;
                    }
                }
            }
            const float qcx = fmaf(c[0], xc.x, fmaf(c[1], xc.y, fmaf(d, c[9], c[2])));
            const float qcy = fmaf(c[3], xc.x, fmaf(c[4], xc.y, fmaf(d, c[10], c[5])));
            const float qcz = fmaf(c[6], xc.x, fmaf(c[7], xc.y, fmaf(d, c[11], c[8])));
#pragma unroll
            for (int j = 0; j < PMAX; ++j) {
                if (j >= P) break;
                const float qx = qcx + c[12 + 3 * j], qy = qcy + c[13 + 3 * j], qz = qcz + c[14 + 3 * j];
                if (!(qz > 0.0f)) continue;
                const float iz = 1.0f / qz;
                const float u = fmaf(pb.fx * qx, iz, pb.cx), v = fmaf(pb.fy * qy, iz, pb.cy);
                float val, wa, wb;
                int bx, by;
                if (!bilinear(pb, en.f, u, v, val, wa, wb, bx, by)) continue;
                const float r = I0[j] - val;
                energy += huber_rho(r, k);
                sumsq = fmaf(r, r, sumsq);
                cnt += 1.0f;
                if (kAccum) {
                    const float wr = huber_w(r, k) * r;
#pragma unroll
                    for (int a = 0; a < 6; ++a) acc[a] = fmaf(Jr[7 * j + a], wr, acc[a]);
                    gpart = fmaf(Jr[7 * j + 6], wr, gpart);
                }
            }
            if (have_prev)
                maxdisp = fmaxf(maxdisp, centre_disp(pb, c, sm.prev + 12 * en.f, xc, d, dprev));
        }
        if (kAccum) {
            warp_sum<6>(acc);
            if (lane == 0) {
                float* o = sm.ent + (e - e0) * kEntryPartial;
#pragma unroll
                for (int a = 0; a < 6; ++a) o[a] = acc[a];
            }
        }
    }
    if (kAccum) {
        sm.red[warp * 32 + lane] = gpart;
        __syncthreads();
        if (warp == 0) {
            float g = 0.0f;
            for (int w = 0; w < kPassWarps; ++w) g += sm.red[w * 32 + lane];
            const float hnn = ic.Hnn[n];
            const bool ok = pb.valid_pt[n] && hnn > 0.0f;
            ds.gn[n] = ok ? g : 0.0f;
            sm.red[kPassWarps * 32 + lane] = ok ? g / hnn : 0.0f;
        }
        __syncthreads();
        const float sn = sm.red[kPassWarps * 32 + lane];
        for (int e = e0 + warp; e < e1; e += kPassWarps) {
            const Entry en = pb.entries[e];
            float acc[6] = {0, 0, 0, 0, 0, 0};
            if ((en.mask >> lane) & 1u) {
                const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
                const float* h = ic.Hfd + (size_t)en.pair_off * 6 + rank;
#pragma unroll
                for (int a = 0; a < 6; ++a) acc[a] = h[a * nvis] * sn;
            }
            warp_sum<6>(acc);
            if (lane == 0) {
                const float* o = sm.ent + (e - e0) * kEntryPartial;
                float* out = ent_part + (size_t)e * kEntryPartial;
#pragma unroll
                for (int a = 0; a < 6; ++a) out[a] = o[a] - acc[a];
            }
        }
    }
    tile_stats_write(tstats, t, energy, sumsq, cnt, maxdisp, ddsq, sm.red);
}

// ---------------------------------------------------------------------------
// FC linearisation pass: prologue = FC depth back-substitution (d <- d + Dd);
// main = per residual r, the target-image gradient (bilinear of the central-
// difference gradient images) and the row
//   c3 = -(1/q_z) (g_u f_x, g_v f_y, -(g_u f_x q_x + g_v f_y q_y)/q_z),
//   J = [d c3, q x c3, c3 . t]      ([upsilon, omega, d] of T <- exp(xi) T),
// accumulating H_ff (21) and g_f per entry, H_fd per pair, H_dd and g_d per
// point with the current Huber weights; epilogue = Schur right-hand side.
// ---------------------------------------------------------------------------
template <int PMAX, bool kAccum>
__global__ void __launch_bounds__(kTile * kPassWarps)
fc_pass_kernel(DevProblem pb, FrameState fs, DepthState ds, float* Hfd_out, float* ent_part,
               TileStats* tstats, int apply, int have_prev)
{
    extern __shared__ float smraw[];
    PassSmem sm(smraw, pb.F);
    load_frame_smem(sm, fs, pb.F, have_prev, apply);
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    const int P = pb.P;
    float ddsq = 0.0f;
    const float dprev = (float)ds.d64[n];
    float d = dprev;
    if (apply) d = (float)depth_backsub(pb, ds, sm.dth, sm.red, t, e0, e1, false, ddsq);
    __syncthreads();  // the prologue read H_fd / g / H_dd that this pass rewrites
    const float2 xc = pb.xn[n];
    float I0[PMAX];
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
        if (j < P) I0[j] = pb.I0p[((size_t)t * P + j) * kTile + lane];
    float gpart = 0.0f, hnn = 0.0f, energy = 0.0f, sumsq = 0.0f, cnt = 0.0f, maxdisp = 0.0f;
    const float k = pb.huber_k;
    for (int e = e0 + warp; e < e1; e += kPassWarps) {
        const Entry en = pb.entries[e];
        const float* c = sm.fc + en.f * kFrameConst;
        float acc[27];
#pragma unroll
        for (int a = 0; a < 27; ++a) acc[a] = 0.0f;
        if ((en.mask >> lane) & 1u) {
            const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
            float hfd[6] = {0, 0, 0, 0, 0, 0};
            const float qcx = fmaf(c[0], xc.x, fmaf(c[1], xc.y, fmaf(d, c[9], c[2])));
            const float qcy = fmaf(c[3], xc.x, fmaf(c[4], xc.y, fmaf(d, c[10], c[5])));
            const float qcz = fmaf(c[6], xc.x, fmaf(c[7], xc.y, fmaf(d, c[11], c[8])));
#pragma unroll
            for (int j = 0; j < PMAX; ++j) {
                if (j >= P) break;
                const float qx = qcx + c[12 + 3 * j], qy = qcy + c[13 + 3 * j], qz = qcz + c[14 + 3 * j];
                if (!(qz > 0.0f)) continue;
                const float iz = 1.0f / qz;
                const float u = fmaf(pb.fx * qx, iz, pb.cx), v = fmaf(pb.fy * qy, iz, pb.cy);
                float val, wa, wb;
                int bx, by;
                if (!bilinear(pb, en.f, u, v, val, wa, wb, bx, by)) continue;
                const float r = I0[j] - val;
                energy += huber_rho(r, k);
                sumsq = fmaf(r, r, sumsq);
                cnt += 1.0f;
                if (!kAccum) continue;
                // bilinear of the gradient images (same footprint)
                const size_t gb = ((size_t)en.f * pb.H + by) * pb.W + bx;
                const float* GX = pb.gx + gb;
                const float* GY = pb.gy + gb;
                const float gxt = fmaf(wa, __ldg(GX + 1) - __ldg(GX), __ldg(GX));
                const float gxb = fmaf(wa, __ldg(GX + pb.W + 1) - __ldg(GX + pb.W), __ldg(GX + pb.W));
                const float gyt = fmaf(wa, __ldg(GY + 1) - __ldg(GY), __ldg(GY));
                const float gyb = fmaf(wa, __ldg(GY + pb.W + 1) - __ldg(GY + pb.W), __ldg(GY + pb.W));
                const float gxv = fmaf(wb, gxb - gxt, gxt) * pb.fx;
                const float gyv = fmaf(wb, gyb - gyt, gyt) * pb.fy;
                const float c0 = -gxv * iz, c1 = -gyv * iz;
                const float c2 = (gxv * qx + gyv * qy) * iz * iz;
                float J[7];
                J[0] = d * c0;
                J[1] = d * c1;
                J[2] = d * c2;
                J[3] = qy * c2 - qz * c1;
                J[4] = qz * c0 - qx * c2;
                J[5] = qx * c1 - qy * c0;
                J[6] = fmaf(c0, c[9], fmaf(c1, c[10], c2 * c[11]));
                const float w = huber_w(r, k);
                const float wr = w * r;
                int q = 0;
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const float wja = w * J[a];
#pragma unroll
                    for (int b = a; b < 6; ++b) {
                        acc[q] = fmaf(wja, J[b], acc[q]);
                        ++q;
                    }
                    acc[21 + a] = fmaf(J[a], wr, acc[21 + a]);
                    hfd[a] = fmaf(wja, J[6], hfd[a]);
                }
                hnn = fmaf(w * J[6], J[6], hnn);
                gpart = fmaf(J[6], wr, gpart);
            }
            if (kAccum) {
                float* hd = Hfd_out + (size_t)en.pair_off * 6 + rank;
#pragma unroll
                for (int a = 0; a < 6; ++a) hd[a * nvis] = hfd[a];
            }
            if (have_prev)
                maxdisp = fmaxf(maxdisp, centre_disp(pb, c, sm.prev + 12 * en.f, xc, d, dprev));
        }
        if (kAccum) {
            warp_sum<27>(acc);
            if (lane == 0) {
                float* o = sm.ent + (e - e0) * kEntryPartial;
#pragma unroll
                for (int a = 0; a < 27; ++a) o[a] = acc[a];
            }
        }
    }
    if (kAccum) {
        sm.red[warp * 32 + lane] = gpart;
        sm.red[(kPassWarps + warp) * 32 + lane] = hnn;
        __syncthreads();
        if (warp == 0) {
            float g = 0.0f, h = 0.0f;
            for (int w = 0; w < kPassWarps; ++w) {
                g += sm.red[w * 32 + lane];
                h += sm.red[(kPassWarps + w) * 32 + lane];
            }
            const bool ok = pb.valid_pt[n] && h > 0.0f;
            ds.gn[n] = ok ? g : 0.0f;
            ds.Hnn[n] = ok ? h : 0.0f;
            sm.red[2 * kPassWarps * 32 + lane] = ok ? g / h : 0.0f;
        }
        __syncthreads();
        const float sn = sm.red[2 * kPassWarps * 32 + lane];
        for (int e = e0 + warp; e < e1; e += kPassWarps) {
            const Entry en = pb.entries[e];
            float acc[6] = {0, 0, 0, 0, 0, 0};
            if ((en.mask >> lane) & 1u) {
                const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
                const float* h = Hfd_out + (size_t)en.pair_off * 6 + rank;
#pragma unroll
                for (int a = 0; a < 6; ++a) acc[a] = h[a * nvis] * sn;
            }
            warp_sum<6>(acc);
            if (lane == 0) {
                const float* o = sm.ent + (e - e0) * kEntryPartial;
                float* out = ent_part + (size_t)e * kEntryPartial;
#pragma unroll
                for (int a = 0; a < 21; ++a) out[a] = o[a];
#pragma unroll
                for (int a = 0; a < 6; ++a) out[21 + a] = o[21 + a] - acc[a];
            }
        }
    }
    tile_stats_write(tstats, t, energy, sumsq, cnt, maxdisp, ddsq, sm.red);
}

// ---------------------------------------------------------------------------
// Fixed-order per-frame reduction of entry partials (Neumaier-compensated
// FP32 per thread, fixed tree across threads, FP64 result), plus one extra
// block that folds the tile statistics into the statistics slots.
// out[f * ncomp + k] = sum over the entries of frame f of part[e][off + k].
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 128;

__global__ void __launch_bounds__(kReduceThreads)
frame_reduce_kernel(DevProblem pb, const float* ent_part, int off, int ncomp, double* out,
                    const TileStats* tstats, const float* dthsq, double* stats, int slot_cur,
                    int slot_prev, int nframes_blocks)
{
    __shared__ double red[kReduceThreads];
    const int tid = threadIdx.x;
    if ((int)blockIdx.x < nframes_blocks) {
        const int f = blockIdx.x + 1;
        const int s0 = pb.frame_entry[f], s1 = pb.frame_entry[f + 1];
        for (int k = 0; k < ncomp; ++k) {
            float s = 0.0f, cmp = 0.0f;
            for (int i = s0 + tid; i < s1; i += kReduceThreads)
                neumaier_add(s, cmp, ent_part[(size_t)pb.frame_entries[i] * kEntryPartial + off + k]);
            red[tid] = (double)s + (double)cmp;
            __syncthreads();
            for (int h = kReduceThreads / 2; h > 0; h >>= 1) {
                if (tid < h) red[tid] += red[tid + h];
                __syncthreads();
            }
            if (tid == 0) out[(size_t)f * ncomp + k] = red[0];
            __syncthreads();
        }
        return;
    }
    // statistics block
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = tid; i < pb.T; i += kReduceThreads) {
        const TileStats s = tstats[i];
        acc[0] += s.energy;
        acc[1] += s.sumsq;
        acc[2] += s.count;
        acc[3] = fmax(acc[3], (double)s.maxdisp);
        acc[4] += s.ddsq;
    }
    for (int k = 0; k < 5; ++k) {
        red[tid] = acc[k];
        __syncthreads();
        for (int h = kReduceThreads / 2; h > 0; h >>= 1) {
            if (tid < h) red[tid] = (k == 3) ? fmax(red[tid], red[tid + h]) : red[tid] + red[tid + h];
            __syncthreads();
        }
        acc[k] = red[0];
        __syncthreads();
    }
    if (tid == 0) {
        if (slot_cur >= 0) {
            double* s = stats + (size_t)slot_cur * kStats;
            s[0] = acc[0];
            s[1] = acc[2] > 0 ? sqrt(acc[1] / acc[2]) : 0.0;
            s[2] = acc[2];
        }
        if (slot_prev >= 0) {
            double* s = stats + (size_t)slot_prev * kStats;
            s[3] = acc[3];
            s[5] = sqrt(acc[4]);
            double q = 0.0;
            for (int f = 0; f < pb.F; ++f) q += dthsq[f];
            s[4] = sqrt(q);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int PMAX>
static cudaError_t launch_ic_precompute_p(const LaunchCtx& L)
{
    size_t sm = pass_smem_bytes(L.pb.F);
    ic_precompute_kernel<PMAX><<<L.pb.T, kTile * kPassWarps, sm, L.stream>>>(
        L.pb, L.poses0, L.ds_ic, L.ic, L.ent_part, L.tstats);
    return cudaGetLastError();
}

cudaError_t launch_ic_precompute(const LaunchCtx& L)
{
    return L.pb.P <= 8 ? launch_ic_precompute_p<8>(L) : launch_ic_precompute_p<16>(L);
}

template <int PMAX>
static cudaError_t launch_ic_pass_p(const LaunchCtx& L, bool accum, int apply, int have_prev)
{
    size_t sm = pass_smem_bytes(L.pb.F);
    if (accum)
        ic_pass_kernel<PMAX, true><<<L.pb.T, kTile * kPassWarps, sm, L.stream>>>(
            L.pb, L.fs, L.ds_ic, L.ic, L.ent_part, L.tstats, apply, have_prev);
    else
        ic_pass_kernel<PMAX, false><<<L.pb.T, kTile * kPassWarps, sm, L.stream>>>(
            L.pb, L.fs, L.ds_ic, L.ic, L.ent_part, L.tstats, apply, have_prev);
    return cudaGetLastError();
}

cudaError_t launch_ic_pass(const LaunchCtx& L, bool accum, int apply, int have_prev)
{
    return L.pb.P <= 8 ? launch_ic_pass_p<8>(L, accum, apply, have_prev)
                       : launch_ic_pass_p<16>(L, accum, apply, have_prev);
}

template <int PMAX>
static cudaError_t launch_fc_pass_p(const LaunchCtx& L, bool accum, int apply, int have_prev)
{
    size_t sm = pass_smem_bytes(L.pb.F);
    if (accum)
        fc_pass_kernel<PMAX, true><<<L.pb.T, kTile * kPassWarps, sm, L.stream>>>(
            L.pb, L.fs, L.ds_fc, L.Hfd_fc, L.ent_part, L.tstats, apply, have_prev);
    else
        fc_pass_kernel<PMAX, false><<<L.pb.T, kTile * kPassWarps, sm, L.stream>>>(
            L.pb, L.fs, L.ds_fc, L.Hfd_fc, L.ent_part, L.tstats, apply, have_prev);
    return cudaGetLastError();
}

cudaError_t launch_fc_pass(const LaunchCtx& L, bool accum, int apply, int have_prev)
{
    return L.pb.P <= 8 ? launch_fc_pass_p<8>(L, accum, apply, have_prev)
                       : launch_fc_pass_p<16>(L, accum, apply, have_prev);
}

cudaError_t launch_frame_reduce(const LaunchCtx& L, int off, int ncomp, double* out, int slot_cur,
                                int slot_prev, bool frames)
{
    const int nfb = frames ? L.pb.F - 1 : 0;
    frame_reduce_kernel<<<nfb + 1, kReduceThreads, 0, L.stream>>>(
        L.pb, L.ent_part, off, ncomp, out, L.tstats, L.dthsq, L.stats, slot_cur, slot_prev, nfb);
    return cudaGetLastError();
}

cudaError_t set_pass_smem_limits(int F)
{
    size_t sm = pass_smem_bytes(F);
    if (sm <= 48 * 1024) return cudaSuccess;
    cudaError_t e;
#define PBA_SMEM(kern)                                                                     \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    if (e != cudaSuccess) return e;
    PBA_SMEM(ic_precompute_kernel<8>)
    PBA_SMEM(ic_precompute_kernel<16>)
    PBA_SMEM((ic_pass_kernel<8, true>))
    PBA_SMEM((ic_pass_kernel<8, false>))
    PBA_SMEM((ic_pass_kernel<16, true>))
    PBA_SMEM((ic_pass_kernel<16, false>))
    PBA_SMEM((fc_pass_kernel<8, true>))
    PBA_SMEM((fc_pass_kernel<8, false>))
    PBA_SMEM((fc_pass_kernel<16, true>))
    PBA_SMEM((fc_pass_kernel<16, false>))
#undef PBA_SMEM
    return cudaSuccess;
}

}  // namespace pba
