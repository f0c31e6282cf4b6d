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
__device__ double depth_backsub(const DevProblem& pb, const DepthState& ds, const Entry* s_ents,
                                const double* s_dth, float* s_red, int t, int e0, int e1,
                                bool ic_rule, float& ddsq)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    // g_n + sum_f H_fd^T Dtheta_f nearly cancels for well-determined points:
    // the dot products use the FP64 update and FP64 sums
    double s = 0.0;
    for (int le = warp; le < e1 - e0; le += kPassWarps) {
        const Entry en = s_ents[le];
        if ((en.mask >> lane) & 1u) {
            const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
            const float* h = ds.Hfd + (size_t)en.pair_off * 6 + rank;
            const double* dt = s_dth + 6 * le;
#pragma unroll
            for (int k = 0; k < 6; ++k) s = fma((double)h[k * nvis], dt[k], s);
        }
    }
    double* s_red64 = reinterpret_cast<double*>(s_red);
    s_red64[warp * 32 + lane] = s;
    __syncthreads();
    double d = ds.d64[n];
    if (warp == 0) {
        double tot = 0.0;
        for (int w = 0; w < kPassWarps; ++w) tot += s_red64[w * 32 + lane];
        const float hnn = ds.Hnn[n];
        double dd = 0.0;
        if (pb.valid_pt[n] && hnn > 0.0f) {
            dd = -((double)ds.gn[n] + tot) / (double)hnn;
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
    }
    __syncthreads();  // all warps have read s_red64 before it is reused
    if (warp == 0) s_red[2 * kPassWarps * 32 + lane] = (float)d;
    __syncthreads();
    // every warp continues with the updated depth (FP32 is what the pass uses)
    return (double)s_red[2 * kPassWarps * 32 + lane];
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

// Shared-memory carve-up of the pass kernels, per local entry le = e - e0 of
// the tile (at most F - 1): the entry record, the FP32 constants of its frame
// (R, t, rotated pattern offsets), the previous R|t, the FP64 update, and a
// 32-float accumulator; then scratch.
struct PassSmem {
    double* dth;  // ne * 6
    Entry* ents;  // ne
    float* fc;    // ne * kFrameConst
    float* prev;  // ne * 12
    float* ent;   // ne * kEntryPartial
    float* red;   // 3 * kPassWarps * 32 + 64 scratch
    __device__ PassSmem(float* s, int F)
    {
        dth = reinterpret_cast<double*>(s);
        ents = reinterpret_cast<Entry*>(s + 12 * F);
        fc = s + 16 * F;
        prev = fc + F * kFrameConst;
        ent = prev + F * 12;
        red = ent + F * kEntryPartial;
    }
};

size_t pass_smem_bytes(int F)
{
    return sizeof(float) * ((size_t)F * (16 + kFrameConst + 12 + kEntryPartial) + 3 * kPassWarps * 32 + 64);
}

// Stages the tile's entries and their frames' constants (the first 12 + 3P
// floats of each) in shared memory.
__device__ void load_tile_smem(const PassSmem& sm, const DevProblem& pb, const FrameState& fs,
                               int e0, int ne, bool prev, bool dth)
{
    for (int i = threadIdx.x; i < ne; i += blockDim.x) sm.ents[i] = pb.entries[e0 + i];
    __syncthreads();
    const int nc = 12 + 3 * pb.P;
    for (int i = threadIdx.x; i < ne * nc; i += blockDim.x) {
        const int le = i / nc, k = i % nc;
        sm.fc[le * kFrameConst + k] = fs.fc[sm.ents[le].f * kFrameConst + k];
    }
    if (prev)
        for (int i = threadIdx.x; i < ne * 12; i += blockDim.x)
            sm.prev[i] = fs.fc_prev[sm.ents[i / 12].f * 12 + i % 12];
    if (dth)
        for (int i = threadIdx.x; i < ne * 6; i += blockDim.x)
            sm.dth[i] = fs.dtheta64[sm.ents[i / 6].f * 6 + i % 6];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// IC precompute (Sec. 3.4-3.5) at the current parameters p_0. Per residual:
// template gradient (central differences at the integer template pixel), the
// proxy-warp Jacobian row in pixel units
//   c = (1/zbar0) (g_u f_x, g_v f_y, -(g_u f_x x + g_v f_y y)),
//   m = zbar0 R0 c - e_z (t0 . R0 c)            (m = M^T c),
//   J = [d0 m, (R0 x~) x m, m . t0],
// the residual and Huber weight at p_0 (J = 0 when invalid there), and the
// H blocks from the stored rows: H_fd per pair, H_dd per point, H_ff (21
// unique) per entry. FP32 throughout (GB300's FP64 issue rate would make
// this pass FP64-bound); J is stored in FP32 either way and H is formed from
// the stored rows, so H = J^T W_0 J holds for the J the iterations use.
// ---------------------------------------------------------------------------
template <int PMAX, int DT>
__global__ void __launch_bounds__(kTile * kPassWarps, 4)
ic_precompute_kernel(DevProblem pb, FrameState fs, DepthState ds, IcStore ic, float* ent_part,
                     TileStats* tstats)
{
    extern __shared__ float smraw[];
    PassSmem sm(smraw, pb.F);
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    load_tile_smem(sm, pb, fs, e0, e1 - e0, false, false);
    const int P = pb.P, NC = (7 * P + 3) / 4;
    const float d0 = (float)ds.d64[n];
    const float2 xc = pb.xn[n];
    const int ux = pb.uvs[2 * n], uy = pb.uvs[2 * n + 1];
    float I0[PMAX], gu[PMAX], gv[PMAX];
#pragma unroll
    for (int j = 0; j < PMAX; ++j) {
        if (j < P) {
            I0[j] = pb.I0p[((size_t)t * P + j) * kTile + lane];
            const int px = ux + pb.pat[2 * j], py = uy + pb.pat[2 * j + 1];
            const size_t b = (size_t)py * pb.pitch + px;
            gu[j] = 0.5f * (load_px_t<DT>(pb.img, (unsigned)(b + 1)) - load_px_t<DT>(pb.img, (unsigned)(b - 1)));
            gv[j] = 0.5f * (load_px_t<DT>(pb.img, (unsigned)(b + pb.pitch)) -
                            load_px_t<DT>(pb.img, (unsigned)(b - pb.pitch)));
        }
    }
    float hnn = 0.0f, energy = 0.0f, sumsq = 0.0f, cnt = 0.0f;
    for (int le = warp; le < e1 - e0; le += kPassWarps) {
        const Entry en = sm.ents[le];
        const float* c = sm.fc + le * kFrameConst;
        float hff[21];
#pragma unroll
        for (int k = 0; k < 21; ++k) hff[k] = 0.0f;
        if ((en.mask >> lane) & 1u) {
            const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
            float Jr[7 * PMAX + 4];
            float hfd[6] = {0, 0, 0, 0, 0, 0};
            const float ax = fmaf(c[0], xc.x, fmaf(c[1], xc.y, c[2]));
            const float ay = fmaf(c[3], xc.x, fmaf(c[4], xc.y, c[5]));
            const float az = fmaf(c[6], xc.x, fmaf(c[7], xc.y, c[8]));
            const float t0x = c[9], t0y = c[10], t0z = c[11];
#pragma unroll
            for (int j = 0; j < PMAX; ++j) {
                if (j >= P) break;
                const float a0 = ax + c[12 + 3 * j], a1 = ay + c[13 + 3 * j], a2 = az + c[14 + 3 * j];
                const float qx = fmaf(d0, t0x, a0), qy = fmaf(d0, t0y, a1), qz = fmaf(d0, t0z, a2);
                float val = 0.f, wa, wb;
                int bx, by;
                bool valid = qz > 0.0f;
                if (valid) {
                    const float iz = 1.0f / qz;
                    valid = bilinear_t<DT>(pb, en.f, fmaf(pb.fx * qx, iz, pb.cx),
                                     fmaf(pb.fy * qy, iz, pb.cy), val, wa, wb, bx, by);
                }
                float J[7] = {0, 0, 0, 0, 0, 0, 0};
                if (valid) {
                    const float r0 = I0[j] - val;
                    const float w0 = huber_w(r0, pb.huber_k);
                    energy += huber_rho(r0, pb.huber_k);
                    sumsq = fmaf(r0, r0, sumsq);
                    cnt += 1.0f;
                    const float x = xc.x + pb.pat[2 * j] / pb.fx, y = xc.y + pb.pat[2 * j + 1] / pb.fy;
                    const float zb = qz / d0;
                    const float izb = 1.0f / zb;
                    const float gx = gu[j] * pb.fx, gy = gv[j] * pb.fy;
                    const float c0 = gx * izb, c1 = gy * izb, c2 = -fmaf(gx, x, gy * y) * izb;
                    const float cp0 = fmaf(c[0], c0, fmaf(c[1], c1, c[2] * c2));
                    const float cp1 = fmaf(c[3], c0, fmaf(c[4], c1, c[5] * c2));
                    const float cp2 = fmaf(c[6], c0, fmaf(c[7], c1, c[8] * c2));
                    const float tc = fmaf(t0x, cp0, fmaf(t0y, cp1, t0z * cp2));
                    const float m0 = zb * cp0, m1 = zb * cp1, m2 = fmaf(zb, cp2, -tc);
                    J[0] = d0 * m0;
                    J[1] = d0 * m1;
                    J[2] = d0 * m2;
                    J[3] = fmaf(a1, m2, -a2 * m1);
                    J[4] = fmaf(a2, m0, -a0 * m2);
                    J[5] = fmaf(a0, m1, -a1 * m0);
                    J[6] = fmaf(m0, t0x, fmaf(m1, t0y, m2 * t0z));
                    int q = 0;
#pragma unroll
                    for (int a = 0; a < 6; ++a) {
                        const float wja = w0 * J[a];
#pragma unroll
                        for (int b = a; b < 6; ++b) {
                            hff[q] = fmaf(wja, J[b], hff[q]);
                            ++q;
                        }
                        hfd[a] = fmaf(wja, J[6], hfd[a]);
                    }
                    hnn = fmaf(w0 * J[6], J[6], hnn);
                }
#pragma unroll
                for (int k = 0; k < 7; ++k) Jr[7 * j + k] = J[k];
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
            for (int k = 0; k < 6; ++k) hd[k * nvis] = hfd[k];
        }
        warp_sum<21>(hff);
        if (lane == 0) {
            float* out = ent_part + (size_t)pb.entry_slot[e0 + le] * kEntryPartial;
#pragma unroll
            for (int k = 0; k < 21; ++k) out[k] = hff[k];
        }
    }
    sm.red[warp * 32 + lane] = hnn;
    __syncthreads();
    if (warp == 0) {
        float tot = 0.0f;
        for (int w = 0; w < kPassWarps; ++w) tot += sm.red[w * 32 + lane];
        ic.Hnn[n] = pb.valid_pt[n] ? tot : 0.0f;
    }
    tile_stats_write(tstats, t, energy, sumsq, cnt, 0.0f, 0.0f, sm.red);
}

// ---------------------------------------------------------------------------
// IC iteration pass (Sec. 3.5 steps 1-2): prologue = depth back-substitution
// and update of the previous step; main = warp, bilinear sample, residual,
// Huber weight, g_f += J_theta w r and g_n += J_d w r; epilogue = Schur
// right-hand side y_f = g_f - sum_n H_fd g_n / H_dd per entry.
// kAccum = false evaluates statistics only (after the last step).
// ---------------------------------------------------------------------------
template <int PMAX, bool kAccum, int DT>
__global__ void __launch_bounds__(kTile * kPassWarps, 5)
ic_pass_kernel(DevProblem pb, FrameState fs, DepthState ds, IcStore ic, float* ent_part,
               TileStats* tstats, int apply, int have_prev)
{
    extern __shared__ float smraw[];
    PassSmem sm(smraw, pb.F);
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    load_tile_smem(sm, pb, fs, e0, e1 - e0, have_prev, apply);
    const int P = pb.P, NC = (7 * P + 3) / 4;
    float ddsq = 0.0f;
    const float dprev = (float)ds.d64[n];
    float d = dprev;
    if (apply) d = (float)depth_backsub(pb, ds, sm.ents, sm.dth, sm.red, t, e0, e1, true, ddsq);
    const float2 xc = pb.xn[n];
    float I0[PMAX];
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
        if (j < P) I0[j] = pb.I0p[((size_t)t * P + j) * kTile + lane];
    float gpart = 0.0f, energy = 0.0f, sumsq = 0.0f, cnt = 0.0f, maxdisp = 0.0f;
    const float k = pb.huber_k;
    for (int le = warp; le < e1 - e0; le += kPassWarps) {
        const Entry en = sm.ents[le];
        const float* c = sm.fc + le * kFrameConst;
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
                if (!bilinear_t<DT>(pb, en.f, u, v, val, wa, wb, bx, by)) continue;
                const float r = I0[j] - val;
                energy += huber_rho(r, k);
                sumsq = fmaf(r, r, sumsq);
                cnt += 1.0f;
                if (kAccum) {
                    // w r with w = min(1, k/|r|): r, or k sign(r) (exact, no division)
                    const float wr = fabsf(r) <= k ? r : copysignf(k, r);
#pragma unroll
                    for (int a = 0; a < 6; ++a) acc[a] = fmaf(Jr[7 * j + a], wr, acc[a]);
                    gpart = fmaf(Jr[7 * j + 6], wr, gpart);
                }
            }
            if (have_prev)
                maxdisp = fmaxf(maxdisp, centre_disp(pb, c, sm.prev + 12 * le, xc, d, dprev));
        }
        if (kAccum) {
            warp_sum<6>(acc);
            if (lane == 0) {
                float* o = sm.ent + le * kEntryPartial;
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
        for (int le = warp; le < e1 - e0; le += kPassWarps) {
            const Entry en = sm.ents[le];
            float acc[6] = {0, 0, 0, 0, 0, 0};
            if ((en.mask >> lane) & 1u) {
                const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
                const float* h = ic.Hfd + (size_t)en.pair_off * 6 + rank;
#pragma unroll
                for (int a = 0; a < 6; ++a) acc[a] = h[a * nvis] * sn;
            }
            warp_sum<6>(acc);
            if (lane == 0) {
                const float* o = sm.ent + le * kEntryPartial;
                float* out = ent_part + (size_t)pb.entry_slot[e0 + le] * kEntryPartial;
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
template <int PMAX, bool kAccum, int DT>
__global__ void __launch_bounds__(kTile * kPassWarps)
fc_pass_kernel(DevProblem pb, FrameState fs, DepthState ds, float* Hfd_out, float* ent_part,
               TileStats* tstats, int apply, int have_prev)
{
    extern __shared__ float smraw[];
    PassSmem sm(smraw, pb.F);
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    load_tile_smem(sm, pb, fs, e0, e1 - e0, have_prev, apply);
    const int P = pb.P;
    float ddsq = 0.0f;
    const float dprev = (float)ds.d64[n];
    float d = dprev;
    if (apply) d = (float)depth_backsub(pb, ds, sm.ents, sm.dth, sm.red, t, e0, e1, false, ddsq);
    __syncthreads();  // the prologue read H_fd / g / H_dd that this pass rewrites
    const float2 xc = pb.xn[n];
    float I0[PMAX];
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
        if (j < P) I0[j] = pb.I0p[((size_t)t * P + j) * kTile + lane];
    float gpart = 0.0f, hnn = 0.0f, energy = 0.0f, sumsq = 0.0f, cnt = 0.0f, maxdisp = 0.0f;
    const float k = pb.huber_k;
    for (int le = warp; le < e1 - e0; le += kPassWarps) {
        const Entry en = sm.ents[le];
        const float* c = sm.fc + le * kFrameConst;
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
                if (!bilinear_t<DT>(pb, en.f, u, v, val, wa, wb, bx, by)) continue;
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
                maxdisp = fmaxf(maxdisp, centre_disp(pb, c, sm.prev + 12 * le, xc, d, dprev));
        }
        if (kAccum) {
            warp_sum<27>(acc);
            if (lane == 0) {
                float* o = sm.ent + le * kEntryPartial;
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
        for (int le = warp; le < e1 - e0; le += kPassWarps) {
            const Entry en = sm.ents[le];
            float acc[6] = {0, 0, 0, 0, 0, 0};
            if ((en.mask >> lane) & 1u) {
                const int nvis = __popc(en.mask), rank = lane_rank(en.mask, lane);
                const float* h = Hfd_out + (size_t)en.pair_off * 6 + rank;
#pragma unroll
                for (int a = 0; a < 6; ++a) acc[a] = h[a * nvis] * sn;
            }
            warp_sum<6>(acc);
            if (lane == 0) {
                const float* o = sm.ent + le * kEntryPartial;
                float* out = ent_part + (size_t)pb.entry_slot[e0 + le] * kEntryPartial;
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
// Fixed-order per-frame reduction of entry partials, plus one extra block that
// folds the tile statistics into the statistics slots. Sums are kept as
// unevaluated FP32 pairs (s, c): Neumaier accumulation per lane, then a
// butterfly whose additions are error-free two-sums (Knuth), converted to
// FP64 once at the end. GB300 issues FP64 slowly; this keeps the reductions
// on the FP32 pipes while carrying about 48 bits.
// out[f * ncomp + k] = sum over the entries of frame f of part[e][off + k].
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 128;

__device__ __forceinline__ void two_sum_add(float& s, float& c, float s2, float c2)
{
    const float t = s + s2;
    const float bb = t - s;
    const float e = (s - (t - bb)) + (s2 - bb);
    s = t;
    c = c + c2 + e;
}

__device__ __forceinline__ void warp_sum_pair(float& s, float& c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        two_sum_add(s, c, s2, c2);
    }
}

__global__ void __launch_bounds__(kReduceThreads)
frame_reduce_kernel(DevProblem pb, const float* ent_part, int off, int ncomp, double* out,
                    const TileStats* tstats, const float* dthsq, double* stats, int slot_cur,
                    int slot_prev, int nframes_blocks)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kReduceThreads / 32;
    if ((int)blockIdx.x < nframes_blocks) {
        const int f = blockIdx.x + 1;
        const int s0 = pb.frame_entry[f], s1 = pb.frame_entry[f + 1];
        for (int k = warp; k < ncomp; k += nw) {
            float s = 0.0f, c = 0.0f;
#pragma unroll 8
            for (int i = s0 + lane; i < s1; i += 32)
                neumaier_add(s, c, ent_part[(size_t)i * kEntryPartial + off + k]);
            warp_sum_pair(s, c);
            if (lane == 0) out[(size_t)f * ncomp + k] = (double)s + (double)c;
        }
        return;
    }
    // statistics block: every thread folds a strided share of the tiles
    // (energy, r^2, count, dd^2 as unevaluated pairs; max displacement), then
    // warps and the block combine them in a fixed order
    __shared__ double res[5];
    __shared__ float sh_s[4][nw], sh_c[4][nw], sh_m[nw];
    float s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0}, m = 0.0f;
#pragma unroll 4
    for (int i = tid; i < pb.T; i += kReduceThreads) {
        const TileStats ts = tstats[i];
        neumaier_add(s[0], c[0], ts.energy);
        neumaier_add(s[1], c[1], ts.sumsq);
        neumaier_add(s[2], c[2], ts.count);
        neumaier_add(s[3], c[3], ts.ddsq);
        m = fmaxf(m, ts.maxdisp);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) warp_sum_pair(s[q], c[q]);
    m = warp_max1(m);
    if (lane == 0) {
        for (int q = 0; q < 4; ++q) {
            sh_s[q][warp] = s[q];
            sh_c[q][warp] = c[q];
        }
        sh_m[warp] = m;
    }
    __syncthreads();
    if (tid < 4) {
        float vs = sh_s[tid][0], vc = sh_c[tid][0];
        for (int w = 1; w < nw; ++w) two_sum_add(vs, vc, sh_s[tid][w], sh_c[tid][w]);
        res[tid == 3 ? 4 : tid] = (double)vs + (double)vc;
    }
    if (tid == 4) {
        float mm = 0.0f;
        for (int w = 0; w < nw; ++w) mm = fmaxf(mm, sh_m[w]);
        res[3] = mm;
    }
    __syncthreads();
    if (tid == 0) {
        if (slot_cur >= 0) {
            double* st = stats + (size_t)slot_cur * kStats;
            st[0] = res[0];
            st[1] = res[2] > 0 ? sqrt(res[1] / res[2]) : 0.0;
            st[2] = res[2];
        }
        if (slot_prev >= 0) {
            double* st = stats + (size_t)slot_prev * kStats;
            st[3] = res[3];
            st[5] = sqrt(res[4]);
            float q = 0.0f, qc = 0.0f;
            for (int f = 0; f < pb.F; ++f) neumaier_add(q, qc, dthsq[f]);
            st[4] = sqrt((double)q + (double)qc);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers (dispatch on the pattern capacity and the image storage type)
// ---------------------------------------------------------------------------
#define PBA_DISPATCH_DT(dtype, CALL) \
    ((dtype) == PBA_F32 ? CALL(PBA_F32) : (dtype) == PBA_F16 ? CALL(PBA_F16) : CALL(PBA_BF16))

template <int PMAX, int DT>
static cudaError_t ic_precompute_p(const LaunchCtx& L)
{
    ic_precompute_kernel<PMAX, DT><<<L.pb.T, kTile * kPassWarps, pass_smem_bytes(L.pb.F), L.stream>>>(
        L.pb, L.fs, L.ds_ic, L.ic, L.ent_part, L.tstats);
    return cudaGetLastError();
}

cudaError_t launch_ic_precompute(const LaunchCtx& L)
{
#define PBA_C8(DT) ic_precompute_p<8, DT>(L)
#define PBA_C16(DT) ic_precompute_p<16, DT>(L)
    return L.pb.P <= 8 ? PBA_DISPATCH_DT(L.pb.dtype, PBA_C8) : PBA_DISPATCH_DT(L.pb.dtype, PBA_C16);
#undef PBA_C8
#undef PBA_C16
}

template <int PMAX, bool A, int DT>
static cudaError_t ic_pass_p(const LaunchCtx& L, int apply, int have_prev)
{
    ic_pass_kernel<PMAX, A, DT><<<L.pb.T, kTile * kPassWarps, pass_smem_bytes(L.pb.F), L.stream>>>(
        L.pb, L.fs, L.ds_ic, L.ic, L.ent_part, L.tstats, apply, have_prev);
    return cudaGetLastError();
}

cudaError_t launch_ic_pass(const LaunchCtx& L, bool accum, int apply, int have_prev)
{
#define PBA_C(PM, A) \
    [&]() { \
        switch (L.pb.dtype) { \
        case PBA_F32: return ic_pass_p<PM, A, PBA_F32>(L, apply, have_prev); \
        case PBA_F16: return ic_pass_p<PM, A, PBA_F16>(L, apply, have_prev); \
        default: return ic_pass_p<PM, A, PBA_BF16>(L, apply, have_prev); \
        } \
    }()
    if (L.pb.P <= 8) return accum ? PBA_C(8, true) : PBA_C(8, false);
    return accum ? PBA_C(16, true) : PBA_C(16, false);
#undef PBA_C
}

template <int PMAX, bool A, int DT>
static cudaError_t fc_pass_p(const LaunchCtx& L, int apply, int have_prev)
{
    fc_pass_kernel<PMAX, A, DT><<<L.pb.T, kTile * kPassWarps, pass_smem_bytes(L.pb.F), L.stream>>>(
        L.pb, L.fs, L.ds_fc, L.Hfd_fc, L.ent_part, L.tstats, apply, have_prev);
    return cudaGetLastError();
}

cudaError_t launch_fc_pass(const LaunchCtx& L, bool accum, int apply, int have_prev)
{
#define PBA_C(PM, A) \
    [&]() { \
        switch (L.pb.dtype) { \
        case PBA_F32: return fc_pass_p<PM, A, PBA_F32>(L, apply, have_prev); \
        case PBA_F16: return fc_pass_p<PM, A, PBA_F16>(L, apply, have_prev); \
        default: return fc_pass_p<PM, A, PBA_BF16>(L, apply, have_prev); \
        } \
    }()
    if (L.pb.P <= 8) return accum ? PBA_C(8, true) : PBA_C(8, false);
    return accum ? PBA_C(16, true) : PBA_C(16, false);
#undef PBA_C
}

cudaError_t launch_frame_reduce(const LaunchCtx& L, int off, int ncomp, double* out, int slot_cur,
                                int slot_prev, bool frames)
{
    const int nfb = frames ? L.pb.F - 1 : 0;
    frame_reduce_kernel<<<nfb + 1, kReduceThreads, 0, L.stream>>>(
        L.pb, L.ent_part, off, ncomp, out, L.tstats, L.dthsq, L.stats, slot_cur, slot_prev, nfb);
    return cudaGetLastError();
}

template <int PM, int DT>
static cudaError_t smem_limits_pd(int sm)
{
    cudaError_t e;
#define PBA_SMEM(...)                                                                                     \
    e = cudaFuncSetAttribute(__VA_ARGS__, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); \
    if (e != cudaSuccess) return e;
    PBA_SMEM(ic_precompute_kernel<PM, DT>)
    PBA_SMEM(ic_pass_kernel<PM, true, DT>)
    PBA_SMEM(ic_pass_kernel<PM, false, DT>)
    PBA_SMEM(fc_pass_kernel<PM, true, DT>)
    PBA_SMEM(fc_pass_kernel<PM, false, DT>)
#undef PBA_SMEM
    return cudaSuccess;
}

cudaError_t set_pass_smem_limits(int F)
{
    const size_t sm = pass_smem_bytes(F);
    if (sm <= 48 * 1024) return cudaSuccess;
    cudaError_t e;
    if ((e = smem_limits_pd<8, PBA_F32>((int)sm)) != cudaSuccess) return e;
    if ((e = smem_limits_pd<8, PBA_F16>((int)sm)) != cudaSuccess) return e;
    if ((e = smem_limits_pd<8, PBA_BF16>((int)sm)) != cudaSuccess) return e;
    if ((e = smem_limits_pd<16, PBA_F32>((int)sm)) != cudaSuccess) return e;
    if ((e = smem_limits_pd<16, PBA_F16>((int)sm)) != cudaSuccess) return e;
    return smem_limits_pd<16, PBA_BF16>((int)sm);
}

}  // namespace pba
