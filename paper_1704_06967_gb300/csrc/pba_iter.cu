// IC iteration kernels (Sec. 3.5 steps 1-3 with the J, W_0 and H fixed by
// the precompute at p_0), none of which waits on another part of the grid:
//   depth_update_kernel  one CTA per tile: back-substitution of the previous
//                        step's depth update (Sec. 3.5 step 3, point block)
//                        and the depth rule (IC: Sec. 3.6; FC: d <- d + Dd);
//   ic_residual_kernel   one warp per (tile, frame) entry: warp, bilinear
//                        sample, residual, Huber weight, and the entry's
//                        share of g_f = sum J_theta^T w r and of g_d;
//   ic_point_kernel      one CTA per tile: g_d per point (entries added in
//                        tile order), the Schur right-hand-side correction
//                        sum_n H_fd g_d / H_dd per entry, the tile
//                        statistics;
// then the frame reduction of y (pba_pass.cu) and ic_solve_kernel (CTA per
// frame: Dtheta = -S^-1 y). The pose updates of a step run in the next
// depth_update_kernel, one frame per CTA.
// A tile has about ten entries, so a CTA per tile (earlier design) left its
// warps waiting at barriers between the phases; a warp per entry gives the
// scheduler ~6k independent warps whose image taps are all in flight at once.
// Every sum has a fixed order: results are deterministic run to run.
#include "pba_kernels.cuh"
#include "pba_pose.cuh"
#include "pba_reduce.cuh"

namespace pba {

namespace {

constexpr int kResWarps = 8;    // warps (entries) per CTA of the residual kernels
constexpr int kTileWarps = 4;   // warps per CTA of the per-tile kernels

__device__ __forceinline__ int rank_of(unsigned mask, int lane)
{
    return __popc(mask & ((1u << lane) - 1u));
}

// Sums of v[0 .. 7] over the warp's lanes by reduce-scatter (nine exchanges
// instead of forty): at strides 16, 8, 4 a lane keeps half of its values and
// adds its partner's copy of them, then two butterfly levels; sum q ends in
// v[0] of lanes 4q .. 4q + 3.
__device__ __forceinline__ void lane_sums8(float (&v)[8], int lane)
{
    scatter_level<4>(v, lane, 16);
    scatter_level<2>(v, lane, 8);
    scatter_level<1>(v, lane, 4);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// (s, c) += h (t.x + t.y): h t.x split exactly by TwoProduct (Ogita, Rump
// and Oishi 2005), the sum carried by Knuth's two-sum; t = (hi, lo) is an
// FP64 value as an unevaluated pair of floats.
__device__ __forceinline__ void dot_pair_add(float& s, float& c, float h, float2 t)
{
    const float p = h * t.x;
    const float e = fmaf(h, t.x, -p);
    const float tail = fmaf(h, t.y, e);
    const float u = s + p;
    const float bb = u - s;
    const float err = (s - (u - bb)) + (p - bb);
    s = u;
    c += err + tail;
}

}  // namespace

// ---------------------------------------------------------------------------
// Depth back-substitution: Dd_n = -(g_n + sum_f H_fd^T Dtheta_f) / H_dd
// (with the brightness pairs as unknowns, + sum_f H_a^T (da_f, db_f)).
// g_n + sum H_fd^T Dtheta nearly cancels for well-determined points, so the
// dot products are carried as unevaluated FP32 pairs (about 48 bits) and the
// quotient and the depth rule are FP64 (IC: 1/H_dd and 1/d_0 come from the
// precompute, so no FP64 division is left). One CTA per tile; warp w takes
// the tile's entries w, w + 4, ... (their records loaded one per lane, so no
// load waits on another), then warp 0 adds the four partial sums in order.
// Writes the FP32 depth the residual kernels use (dcur), the one before this
// update (dprev) and the tile's sum of Dd^2. apply = 0 only refreshes
// dcur/dprev from the FP64 depths.
// ---------------------------------------------------------------------------
template <bool kIcRule, bool kAff = false>
__global__ void __launch_bounds__(kTileWarps * 32)
depth_update_kernel(DevProblem pb, DepthState ds, const float2* __restrict__ dth2,
                    const double* __restrict__ inv_hnn, const double* __restrict__ inv_d0,
                    float* __restrict__ dcur, float* __restrict__ dprev, float* __restrict__ ddsq_t,
                    int apply, SolveArgs a)
{
    __shared__ float2 red[kTileWarps][32];
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_trigger();
    if (t >= pb.T) {
        pdl_wait();
        // CTA T + f - 1: pose update of frame f with the update the solve
        // wrote (FP64; one frame per CTA, spread over the SMs)
        __shared__ double sh[54], d[6];
        const int f = t - pb.T + 1;
        if (warp != 0) return;
        if (lane < 6) d[lane] = a.dtheta64[6 * f + lane];
        if (kAff && lane == 0) {
            // the brightness pair: IC composes alpha' = alpha / (1 + da),
            // beta' = (beta - db) / (1 + da); FC adds (da, db)
            const double da = a.dab64[2 * f], db = a.dab64[2 * f + 1];
            if (da != 0.0 || db != 0.0) {
                float* fcf = a.fc + (size_t)f * kFrameConst + kFrameAlpha;
                const double al = (double)fcf[0], be = (double)fcf[1];
                if (kIcRule) {
                    const double s = 1.0 + da;
                    fcf[0] = (float)(al / s);
                    fcf[1] = (float)((be - db) / s);
                } else {
                    fcf[0] = (float)(al + da);
                    fcf[1] = (float)(be + db);
                }
            }
        }
        __syncwarp();
        // a zero update (a bundle's reference frame, a frame without
        // residuals) leaves the pose exactly as it is
        if (__all_sync(0xffffffffu, lane >= 6 || d[lane] == 0.0)) {
            if (lane < 12) a.fc_prev[12 * f + lane] = (float)a.poses64[12 * f + lane];
            return;
        }
        if (kIcRule) ic_pose_update_warp(a, f, a.poses64 + 12 * f, a.poses0 + 12 * f, d, sh, lane);
        else fc_pose_update_warp(a, f, d, sh, lane);
        return;
    }
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], ne = pb.tile_entry[t + 1] - e0, cnt0 = min(32, ne);
    // Before the wait: the tile's entry records and, for IC, what the
    // precompute fixed (H_fd rows of each warp's first kDepthPre entries,
    // H_dd, 1/H_dd, d_0, 1/d_0); no kernel of the iteration writes them.
    constexpr int kDepthPre = 4;
    double d = 0.0, d0 = 0.0, ih = 0.0, id0 = 0.0;
    float gn = 0.0f, hnn = 0.0f;
    bool valid = false;
    Entry mine = {0, 0u, 0, 0};
    float hpre[kDepthPre][6];
    if (apply) {
        if (lane < ne) mine = pb.entries[e0 + lane];
        if (warp == 0) {
            valid = pb.valid_pt[n];
            if (kIcRule) {
                hnn = ds.Hnn[n];
                d0 = ds.d0_64[n];
                ih = inv_hnn[n];
                id0 = inv_d0[n];
            }
        }
        if (kIcRule) {
#pragma unroll
            for (int r = 0; r < kDepthPre; ++r) {
                const int i = warp + kTileWarps * r;
                const unsigned mask = __shfl_sync(0xffffffffu, mine.mask, i);
                const int po = __shfl_sync(0xffffffffu, mine.pair_off, i);
                const bool vis = i < cnt0 && ((mask >> lane) & 1u);
                const int nvis = __popc(mask);
                const float* h = ds.Hfd + (size_t)po * 6 + (vis ? rank_of(mask, lane) : 0);
#pragma unroll
                for (int k = 0; k < 6; ++k) hpre[r][k] = vis ? h[k * nvis] : 0.0f;
            }
        }
    }
    pdl_wait();
    if (warp == 0) {
        d = ds.d64[n];
        if (apply) {
            gn = ds.gn[n];
            if (!kIcRule) hnn = ds.Hnn[n];
        }
    }
    if (apply) {
        float s = 0.0f, c = 0.0f;
        // entry i of the current batch (hv: its prefetched H_fd values, or
        // null to load them)
        auto add_entry = [&](int i, const float* hv) {
            const int f = __shfl_sync(0xffffffffu, mine.f, i);
            const unsigned mask = __shfl_sync(0xffffffffu, mine.mask, i);
            const int po = __shfl_sync(0xffffffffu, mine.pair_off, i);
            const bool vis = (mask >> lane) & 1u;
            const int nvis = __popc(mask);
            const float* h = ds.Hfd + (size_t)po * 6 + (vis ? rank_of(mask, lane) : 0);
            const float2* th = dth2 + 6 * f;
#pragma unroll
            for (int k = 0; k < 6; ++k) dot_pair_add(s, c, vis ? (hv ? hv[k] : h[k * nvis]) : 0.0f, th[k]);
            if (kAff) {
                // joint brightness: + H_a^T (da, db) of the frame (H_a: the
                // IC or FC system's, ds.Had)
                const float* ha = ds.Had + (size_t)po * 2 + (vis ? rank_of(mask, lane) : 0);
                const float2* tb = a.dab2 + 2 * f;
                dot_pair_add(s, c, vis ? ha[0] : 0.0f, tb[0]);
                dot_pair_add(s, c, vis ? ha[nvis] : 0.0f, tb[1]);
            }
        };
        int i = warp;
        if (kIcRule) {
#pragma unroll
            for (int r = 0; r < kDepthPre; ++r, i += kTileWarps)
                if (i < cnt0) add_entry(i, hpre[r]);
        }
#pragma unroll 2
        for (; i < cnt0; i += kTileWarps) add_entry(i, nullptr);
        for (int b = 32; b < ne; b += 32) {
            mine = Entry{0, 0u, 0, 0};
            if (b + lane < ne) mine = pb.entries[e0 + b + lane];
            const int cnt = min(32, ne - b);
#pragma unroll 2
            for (int j = warp; j < cnt; j += kTileWarps) add_entry(j, nullptr);
        }
        red[warp][lane] = make_float2(s, c);
    }
    __syncthreads();
    if (warp != 0) return;
    const float dold = (float)d;
    float ddsq = 0.0f;
    if (apply) {
        float s = red[0][lane].x, c = red[0][lane].y;
        for (int w = 1; w < kTileWarps; ++w) {
            const float2 v = red[w][lane];
            const float u = s + v.x, bb = u - s;
            c += v.y + ((s - (u - bb)) + (v.x - bb));
            s = u;
        }
        double dd = 0.0;
        if (valid && hnn > 0.0f) {
            const double num = (double)gn + ((double)s + (double)c);
            dd = kIcRule ? -num * ih : -num / ((double)hnn * (double)pb.damp1);
            const double dn = kIcRule ? d * ((d0 - dd) * id0) : d + dd;
            if (isfinite(dn)) {
                d = dn;
                ds.d64[n] = d;
            } else {
                flag_error(ds.err, pb.frame_bundle[pb.tile_f0[t]], kErrNonFinite);
            }
        }
        ds.dd_last[n] = dd;
        ddsq = (float)(dd * dd);
    }
    dcur[n] = (float)d;
    dprev[n] = dold;
    ddsq = warp_sum1(ddsq);
    if (lane == 0) ddsq_t[t] = ddsq;
}

// Statistics of tile t from its entries' (energy, r^2, count, max
// displacement) and the tile's sum of Dd^2; lanes take entries, then a
// butterfly (fixed order).
__device__ __forceinline__ void tile_stats_from_entries(const DevProblem& pb, const float4* estats,
                                                        const float* ddsq_t, TileStats* out, int t,
                                                        int e0, int e1, int lane)
{
    float s[3] = {0, 0, 0}, m = 0.0f;
    for (int e = e0 + lane; e < e1; e += 32) {
        const float4 v = __ldcg(estats + e);
        s[0] += v.x;
        s[1] += v.y;
        s[2] += v.z;
        m = fmaxf(m, v.w);
    }
    warp_sum<3>(s);
    m = warp_max1(m);
    if (lane == 0) out[t] = TileStats{s[0], s[1], s[2], m, ddsq_t[t], 0, 0, 0};
}


// ---------------------------------------------------------------------------
// IC residuals of one entry (Sec. 3.5 steps 1-2). Lane l is point 32 t + l of
// the entry's tile; lanes whose point the frame does not see stay idle.
// Phase 1 projects the P pattern pixels (q = R x~_c + d t + delta_j) and
// forms their bilinear footprints; a footprint outside [1, W-2] x [1, H-2]
// (or behind the camera) marks the residual invalid and is clamped into the
// image, so phase 2 can issue every tap of every pattern pixel at once with
// no branch in between. Phase 3 forms r = I_0 - I(W(x)), the Huber terms and
// w r (r, or k sign r: exact, no division); phase 4 streams the stored rows
// J and adds J_theta w r into the frame sum and J_d w r into the point's.
// ---------------------------------------------------------------------------
template <int PMAX, bool kAccum, int DT, int WARPS, bool kJoint = false>
__global__ void __launch_bounds__(WARPS * 32, (PMAX <= 8 ? 32 : 16) / WARPS)
ic_residual_kernel(DevProblem pb, const float* __restrict__ fconst, const float* __restrict__ fprev,
                   const float* __restrict__ dcur, const float* __restrict__ dprev,
                   const float4* __restrict__ J4, float* __restrict__ ent_part,
                   float* __restrict__ gpart, float4* __restrict__ estats, int have_prev, int photo)
{
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * WARPS + (threadIdx.x >> 5);
    pdl_trigger();
    pdl_wait();
    if (e >= pb.E) return;
    const Entry en = pb.entries[e];
    const int P = pb.P;
    const float k = pb.huber_k;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // g_f (6), energy, r^2
    float cnt = 0.0f;
    float ph[5] = {0, 0, 0, 0, 0};  // photo: brightness fit sums (w, w v, w v^2, w I_0, w I_0^2);
                                    // kJoint: g_a = (sum I_0 w r, sum w r) over the rows valid at p_0
    float gp = 0.0f, disp = 0.0f;
    if ((en.mask >> lane) & 1u) {
        const int n = en.tile * kTile + lane;
        const unsigned vm0 = (kAccum && kJoint) ? pb.vmask0[en.pair_off + rank_of(en.mask, lane)] : 0u;
        const float* c = fconst + (size_t)en.f * kFrameConst;
        const float alpha = c[kFrameAlpha], beta = c[kFrameAlpha + 1];
        const float d = dcur[n];
        const float2 xc = pb.xn[n];
        float I0[PMAX];
#pragma unroll
        for (int j = 0; j < PMAX; ++j)
            if (j < P) I0[j] = pb.I0p[((size_t)en.tile * P + j) * kTile + lane];
        const float qcx = fmaf(c[0], xc.x, fmaf(c[1], xc.y, fmaf(d, c[9], c[2])));
        const float qcy = fmaf(c[3], xc.x, fmaf(c[4], xc.y, fmaf(d, c[10], c[5])));
        const float qcz = fmaf(c[6], xc.x, fmaf(c[7], xc.y, fmaf(d, c[11], c[8])));
        const float umax = (float)(pb.W - 3), vmax = (float)(pb.H - 3);
        const unsigned row0 = (unsigned)en.f * (unsigned)pb.H, pitch = (unsigned)pb.pitch;
        unsigned base[PMAX], ok = 0;
        float wa[PMAX], wb[PMAX];
#pragma unroll
        for (int j = 0; j < PMAX; ++j) {
            if (j < P) {
                const float qx = qcx + c[12 + 3 * j], qy = qcy + c[13 + 3 * j], qz = qcz + c[14 + 3 * j];
                const float iz = rcp_approx(qz);
                const float u = fmaf(pb.fx * qx, iz, pb.cx), v = fmaf(pb.fy * qy, iz, pb.cy);
                const float fu = floorf(u), fv = floorf(v);
                // (a NaN coordinate fails the test and clamps to 1)
                if (qz > 0.0f && fu >= 1.0f && fu <= umax && fv >= 1.0f && fv <= vmax) ok |= 1u << j;
                const float xu = fminf(fmaxf(fu, 1.0f), umax), yv = fminf(fmaxf(fv, 1.0f), vmax);
                wa[j] = u - fu;
                wb[j] = v - fv;
                base[j] = (row0 + (unsigned)(int)yv) * pitch + (unsigned)(int)xu;
            }
        }
        float val[PMAX];
#pragma unroll
        for (int j = 0; j < PMAX; ++j) {
            if (j < P) {
                const unsigned b = base[j];
                const float i00 = load_px_t<DT>(pb.img, b), i10 = load_px_t<DT>(pb.img, b + 1);
                const float i01 = load_px_t<DT>(pb.img, b + pitch), i11 = load_px_t<DT>(pb.img, b + pitch + 1);
                const float top = fmaf(wa[j], i10 - i00, i00);
                const float bot = fmaf(wa[j], i11 - i01, i01);
                val[j] = fmaf(wb[j], bot - top, top);
            }
        }
        float wr[PMAX];
#pragma unroll
        for (int j = 0; j < PMAX; ++j) {
            wr[j] = 0.0f;
            if (j < P && ((ok >> j) & 1u)) {
                // affine brightness: the template sees alpha I_f + beta (1, 0: exact no-op)
                const float r = I0[j] - fmaf(alpha, val[j], beta);
                acc[6] += huber_rho(r, k);
                acc[7] = fmaf(r, r, acc[7]);
                cnt += 1.0f;
                wr[j] = fabsf(r) <= k ? r : copysignf(k, r);
                if (kAccum && kJoint) {
                    if ((vm0 >> j) & 1u) {
                        ph[0] = fmaf(I0[j], wr[j], ph[0]);
                        ph[1] += wr[j];
                    }
                } else if (kAccum && photo) {
                    const float w = huber_w(r, k);
                    ph[0] += w;
                    ph[1] = fmaf(w, val[j], ph[1]);
                    ph[2] = fmaf(w * val[j], val[j], ph[2]);
                    ph[3] = fmaf(w, I0[j], ph[3]);
                    ph[4] = fmaf(w * I0[j], I0[j], ph[4]);
                }
            }
        }
        if (kAccum) {
            const int NC = (7 * P + 3) / 4, nvis = __popc(en.mask);
            const float4* src = J4 + (size_t)en.pair_off * NC + rank_of(en.mask, lane);
            const uint64_t pol = l2_evict_first_policy();
            // rows of four pattern pixels (seven float4 chunks) at a time,
            // loaded after the taps are consumed (register pressure)
#pragma unroll
            for (int g = 0; g < PMAX / 4; ++g) {
                if (4 * g < P) {
                    asm volatile("" ::: "memory");
                    float Jr[28];
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (7 * g + q < NC) v = ld_stream4(src + (size_t)(7 * g + q) * nvis, pol);
                        Jr[4 * q] = v.x;
                        Jr[4 * q + 1] = v.y;
                        Jr[4 * q + 2] = v.z;
                        Jr[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * g + jj;
                        if (j < P) {
#pragma unroll
                            for (int a = 0; a < 6; ++a) acc[a] = fmaf(Jr[7 * jj + a], wr[j], acc[a]);
                            gp = fmaf(Jr[7 * jj + 6], wr[j], gp);
                        }
                    }
                }
            }
        }
        if (have_prev) {
            // pattern-centre displacement since the previous parameters
            // (convergence rule of Sec. 4.1)
            const float* cp = fprev + 12 * en.f;
            const float dp = dprev[n];
            const float px = fmaf(cp[0], xc.x, fmaf(cp[1], xc.y, fmaf(dp, cp[9], cp[2])));
            const float py = fmaf(cp[3], xc.x, fmaf(cp[4], xc.y, fmaf(dp, cp[10], cp[5])));
            const float pz = fmaf(cp[6], xc.x, fmaf(cp[7], xc.y, fmaf(dp, cp[11], cp[8])));
            const float iq = rcp_approx(qcz), ip = rcp_approx(pz);
            const float du = pb.fx * fmaf(qcx, iq, -px * ip), dv = pb.fy * fmaf(qcy, iq, -py * ip);
            disp = fmaf(du, du, dv * dv);  // squared: the square root of the warp's maximum is taken once
        }
    }
    disp = sqrtf(warp_max1(disp));
    if (kAccum) {
        gpart[(size_t)e * kTile + lane] = gp;
        // g_f (6), energy and r^2 by reduce-scatter (sum q on lanes 4q ..
        // 4q + 3), the count by a butterfly
        lane_sums8(acc, lane);
        cnt = warp_sum1(cnt);
        if (kJoint) {
            float g2[2] = {ph[0], ph[1]};
            warp_sum(g2);
            ph[0] = g2[0];
            ph[1] = g2[1];
        } else if (photo) {
            warp_sum<5>(ph);
        }
        float* o = ent_part + (size_t)pb.entry_slot[e] * kEntryPartial;
        float* es = reinterpret_cast<float*>(estats + e);
        if ((lane & 3) == 0) {
            if (lane < 24) o[lane >> 2] = acc[0];
            else es[(lane - 24) >> 2] = acc[0];  // energy, r^2
        }
        if (lane == 0) {
            es[2] = cnt;
            es[3] = disp;
            if (kJoint) {
                o[kPhotoColIc] = ph[0];
                o[kPhotoColIc + 1] = ph[1];
            } else if (photo) {
#pragma unroll
                for (int a = 0; a < 5; ++a) o[kPhotoColIc + a] = ph[a];
            }
        }
    } else {
        float st[3] = {acc[6], acc[7], cnt};
        warp_sum<3>(st);
        if (lane == 0) estats[e] = make_float4(st[0], st[1], st[2], disp);
    }
}

// ---------------------------------------------------------------------------
// FC linearisation of one entry: per residual the target-image gradient
// (bilinear of the central-difference gradient images, same footprint as the
// intensity) and the row
//   c3 = -(1/q_z) (g_u f_x, g_v f_y, -(g_u f_x q_x + g_v f_y q_y)/q_z),
//   J = [d c3, q x c3, c3 . t]      ([upsilon, omega, d] of T <- exp(xi) T),
// with the current Huber weight w: the entry's H_ff (21 upper entries) and
// g_f = J_theta^T w r, H_fd of each pair, and per lane J_d^T w r and
// J_d^T w J_d. Pattern pixels go in groups of kFcGroup, each group's twelve
// taps per pixel issued together (register pressure bounds the group).
// ---------------------------------------------------------------------------
constexpr int kFcGroup = 2;

template <int PMAX, bool kAccum, int DT, bool kJoint = false>
__global__ void __launch_bounds__(kResWarps * 32, 2)
fc_residual_kernel(DevProblem pb, const float* __restrict__ fconst, const float* __restrict__ fprev,
                   const float* __restrict__ dcur, const float* __restrict__ dprev,
                   float* __restrict__ Hfd_out, float* __restrict__ ent_part,
                   float* __restrict__ gpart, float4* __restrict__ estats, int have_prev, int photo,
                   float* __restrict__ Had_out, float* __restrict__ aff_part)
{
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * kResWarps + (threadIdx.x >> 5);
    pdl_trigger();
    pdl_wait();
    if (e >= pb.E) return;
    const Entry en = pb.entries[e];
    const int P = pb.P;
    const float k = pb.huber_k;
    float acc[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) acc[q] = 0.0f;
    float hfd[6] = {0, 0, 0, 0, 0, 0};
    float st[3] = {0, 0, 0};
    float ph[5] = {0, 0, 0, 0, 0};  // brightness fit sums (w, w v, w v^2, w I_0, w I_0^2);
                                    // kJoint: g_a = (sum -v w r, sum -w r)
    // kJoint (the pairs as unknowns, columns -v and -1): H_pa ([a][alpha,
    // beta]), H_aa (v^2, v, 1) weighted sums, and the pair's J_d^T W [-v, -1]
    float aff[kAffComp], had[2] = {0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < kAffComp; ++q) aff[q] = 0.0f;
    float gp = 0.0f, hnn = 0.0f, disp = 0.0f;
    if ((en.mask >> lane) & 1u) {
        const int n = en.tile * kTile + lane;
        const float* c = fconst + (size_t)en.f * kFrameConst;
        const float alpha = c[kFrameAlpha], beta = c[kFrameAlpha + 1];
        const float d = dcur[n];
        const float2 xc = pb.xn[n];
        const float qcx = fmaf(c[0], xc.x, fmaf(c[1], xc.y, fmaf(d, c[9], c[2])));
        const float qcy = fmaf(c[3], xc.x, fmaf(c[4], xc.y, fmaf(d, c[10], c[5])));
        const float qcz = fmaf(c[6], xc.x, fmaf(c[7], xc.y, fmaf(d, c[11], c[8])));
        const float t0 = c[9], t1 = c[10], t2 = c[11];
        const float umax = (float)(pb.W - 3), vmax = (float)(pb.H - 3);
        const unsigned row0 = (unsigned)en.f * (unsigned)pb.H, pitch = (unsigned)pb.pitch;
        const unsigned W = (unsigned)pb.W;
#pragma unroll
        for (int g = 0; g < PMAX; g += kFcGroup) {
            if (g < P) {
                asm volatile("" ::: "memory");
                unsigned ib[kFcGroup], gb[kFcGroup], ok = 0;
                float wa[kFcGroup], wb[kFcGroup], qx[kFcGroup], qy[kFcGroup], qz[kFcGroup],
                    iz[kFcGroup], I0[kFcGroup];
#pragma unroll
                for (int jj = 0; jj < kFcGroup; ++jj) {
                    const int j = g + jj;
                    if (j < P) {
                        I0[jj] = pb.I0p[((size_t)en.tile * P + j) * kTile + lane];
                        qx[jj] = qcx + c[12 + 3 * j];
                        qy[jj] = qcy + c[13 + 3 * j];
                        qz[jj] = qcz + c[14 + 3 * j];
                        iz[jj] = 1.0f / qz[jj];
                        const float u = fmaf(pb.fx * qx[jj], iz[jj], pb.cx);
                        const float v = fmaf(pb.fy * qy[jj], iz[jj], pb.cy);
                        const float fu = floorf(u), fv = floorf(v);
                        if (qz[jj] > 0.0f && fu >= 1.0f && fu <= umax && fv >= 1.0f && fv <= vmax)
                            ok |= 1u << jj;
                        const unsigned x = (unsigned)(int)fminf(fmaxf(fu, 1.0f), umax);
                        const unsigned y = (unsigned)(int)fminf(fmaxf(fv, 1.0f), vmax);
                        wa[jj] = u - fu;
                        wb[jj] = v - fv;
                        ib[jj] = (row0 + y) * pitch + x;
                        gb[jj] = (row0 + y) * W + x;
                    }
                }
                float val[kFcGroup], gxv[kFcGroup], gyv[kFcGroup];
#pragma unroll
                for (int jj = 0; jj < kFcGroup; ++jj) {
                    if (g + jj < P) {
                        const unsigned b = ib[jj];
                        const float i00 = load_px_t<DT>(pb.img, b), i10 = load_px_t<DT>(pb.img, b + 1);
                        const float i01 = load_px_t<DT>(pb.img, b + pitch);
                        const float i11 = load_px_t<DT>(pb.img, b + pitch + 1);
                        const float top = fmaf(wa[jj], i10 - i00, i00);
                        const float bot = fmaf(wa[jj], i11 - i01, i01);
                        val[jj] = fmaf(wb[jj], bot - top, top);
                        if (kAccum) {
                            const float* GX = pb.gx + gb[jj];
                            const float* GY = pb.gy + gb[jj];
                            const float gxt = fmaf(wa[jj], __ldg(GX + 1) - __ldg(GX), __ldg(GX));
                            const float gxb = fmaf(wa[jj], __ldg(GX + W + 1) - __ldg(GX + W), __ldg(GX + W));
                            const float gyt = fmaf(wa[jj], __ldg(GY + 1) - __ldg(GY), __ldg(GY));
                            const float gyb = fmaf(wa[jj], __ldg(GY + W + 1) - __ldg(GY + W), __ldg(GY + W));
                            gxv[jj] = fmaf(wb[jj], gxb - gxt, gxt) * (pb.fx * alpha);
                            gyv[jj] = fmaf(wb[jj], gyb - gyt, gyt) * (pb.fy * alpha);
                        }
                    }
                }
#pragma unroll
                for (int jj = 0; jj < kFcGroup; ++jj) {
                    if (g + jj < P && ((ok >> jj) & 1u)) {
                        const float r = I0[jj] - fmaf(alpha, val[jj], beta);
                        st[0] += huber_rho(r, k);
                        st[1] = fmaf(r, r, st[1]);
                        st[2] += 1.0f;
                        if (kAccum && !kJoint && photo) {
                            const float w = huber_w(r, k);
                            ph[0] += w;
                            ph[1] = fmaf(w, val[jj], ph[1]);
                            ph[2] = fmaf(w * val[jj], val[jj], ph[2]);
                            ph[3] = fmaf(w, I0[jj], ph[3]);
                            ph[4] = fmaf(w * I0[jj], I0[jj], ph[4]);
                        }
                        if (kAccum) {
                            const float c0 = -gxv[jj] * iz[jj], c1 = -gyv[jj] * iz[jj];
                            const float c2 = (gxv[jj] * qx[jj] + gyv[jj] * qy[jj]) * iz[jj] * iz[jj];
                            float J[7];
                            J[0] = d * c0;
                            J[1] = d * c1;
                            J[2] = d * c2;
                            J[3] = qy[jj] * c2 - qz[jj] * c1;
                            J[4] = qz[jj] * c0 - qx[jj] * c2;
                            J[5] = qx[jj] * c1 - qy[jj] * c0;
                            J[6] = fmaf(c0, t0, fmaf(c1, t1, c2 * t2));
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
                            gp = fmaf(J[6], wr, gp);
                            if (kJoint) {
                                const float wv = w * val[jj];
#pragma unroll
                                for (int a = 0; a < 6; ++a) {
                                    aff[2 * a] = fmaf(-wv, J[a], aff[2 * a]);
                                    aff[2 * a + 1] = fmaf(-w, J[a], aff[2 * a + 1]);
                                }
                                aff[12] = fmaf(wv, val[jj], aff[12]);
                                aff[13] += wv;
                                aff[14] += w;
                                ph[0] = fmaf(-val[jj], wr, ph[0]);
                                ph[1] -= wr;
                                had[0] = fmaf(-wv, J[6], had[0]);
                                had[1] = fmaf(-w, J[6], had[1]);
                            }
                        }
                    }
                }
            }
        }
        if (kAccum) {
            const int nvis = __popc(en.mask);
            float* hd = Hfd_out + (size_t)en.pair_off * 6 + rank_of(en.mask, lane);
#pragma unroll
            for (int a = 0; a < 6; ++a) hd[a * nvis] = hfd[a];
            if (kJoint) {
                float* ha = Had_out + (size_t)en.pair_off * 2 + rank_of(en.mask, lane);
                ha[0] = had[0];
                ha[nvis] = had[1];
            }
        }
        if (have_prev) {
            const float* cp = fprev + 12 * en.f;
            const float dp = dprev[n];
            const float px = fmaf(cp[0], xc.x, fmaf(cp[1], xc.y, fmaf(dp, cp[9], cp[2])));
            const float py = fmaf(cp[3], xc.x, fmaf(cp[4], xc.y, fmaf(dp, cp[10], cp[5])));
            const float pz = fmaf(cp[6], xc.x, fmaf(cp[7], xc.y, fmaf(dp, cp[11], cp[8])));
            const float du = pb.fx * (qcx / qcz - px / pz), dv = pb.fy * (qcy / qcz - py / pz);
            disp = sqrtf(du * du + dv * dv);
        }
    }
    if (kAccum) {
        gpart[(size_t)e * 2 * kTile + lane] = gp;
        gpart[(size_t)e * 2 * kTile + kTile + lane] = hnn;
        warp_sum<27>(acc);
        if (photo) warp_sum<5>(ph);
        if (kJoint) warp_sum<kAffComp>(aff);
    }
    warp_sum<3>(st);
    disp = warp_max1(disp);
    if (lane == 0) {
        if (kAccum) {
            float* o = ent_part + (size_t)pb.entry_slot[e] * kEntryPartial;
#pragma unroll
            for (int q = 0; q < 27; ++q) o[q] = acc[q];
            if (photo)
#pragma unroll
                for (int a = 0; a < 5; ++a) o[kPhotoColFc + a] = ph[a];
            if (kJoint) {
                float* oa = aff_part + (size_t)pb.entry_slot[e] * kEntryPartial;
#pragma unroll
                for (int q = 0; q < kAffComp; ++q) oa[q] = aff[q];
            }
        }
        estats[e] = make_float4(st[0], st[1], st[2], disp);
    }
}

// ---------------------------------------------------------------------------
// Per tile: g_n = sum over the tile's entries of J_d^T w r (fixed entry
// order; FC also sums H_dd = J_d^T w J_d the same way), then the Schur
// right-hand-side correction c_e = sum_n H_fd(n, f) g_n / H_dd(n) of every
// entry e, written beside the entry's g_f partial at coff (the frame
// reduction forms y_f = sum_e (g_f,e - c_e), Sec. 3.5 step 3). Every warp
// forms g_n itself (a few independent loads) and takes entries round-robin,
// their records loaded one per lane, so no warp waits on another.
// kFc: per-lane partials are E x 64 (g then H_dd) and H_dd is written out.
// Before the wait each warp loads the tile's entry records and (IC) the H_fd
// rows of its first kPointPre entries and H_dd: the precompute wrote them and
// no kernel of the iteration does (FC forms H_fd and H_dd in the residual
// pass just before, so FC reads them after the wait).
// ---------------------------------------------------------------------------
constexpr int kPointPre = 4;

template <bool kAccum, bool kFc, bool kAff = false>
__global__ void __launch_bounds__(kTileWarps * 32)
point_kernel(DevProblem pb, const float* __restrict__ gpart, const float* __restrict__ Hfd,
             float* __restrict__ Hnn, float* __restrict__ gn, float* __restrict__ ent_part, int coff,
             const float4* __restrict__ estats, const float* __restrict__ ddsq_t,
             TileStats* __restrict__ tstats, const float* __restrict__ Had, int acol)
{
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_trigger();
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1], ne = e1 - e0;
    const int n = t * kTile + lane;
    const int cnt0 = min(32, ne);
    Entry mine = {0, 0u, 0, 0};
    int slot = 0;
    bool valid = false;
    float hnn = 0.0f;
    float hpre[kPointPre][6];
    if (kAccum) {
        if (lane < ne) {
            mine = pb.entries[e0 + lane];
            slot = pb.entry_slot[e0 + lane];
        }
        valid = pb.valid_pt[n];
        if (!kFc) {
            hnn = Hnn[n];
#pragma unroll
            for (int r = 0; r < kPointPre; ++r) {
                const int i = warp + kTileWarps * r;
                const unsigned mask = __shfl_sync(0xffffffffu, mine.mask, i);
                const int po = __shfl_sync(0xffffffffu, mine.pair_off, i);
                const bool vis = i < cnt0 && ((mask >> lane) & 1u);
                const int nvis = __popc(mask);
                const float* h = Hfd + (size_t)po * 6 + (vis ? rank_of(mask, lane) : 0);
#pragma unroll
                for (int q = 0; q < 6; ++q) hpre[r][q] = vis ? h[q * nvis] : 0.0f;
            }
        }
    }
    pdl_wait();
    if (kAccum) {
        // g_n (FC: and H_dd): warp w adds the tile's entries w, w + 4, ...,
        // then every warp adds the four partial sums in warp order
        const int stride = kFc ? 2 * kTile : kTile;
        __shared__ float red_g[kTileWarps][kTile], red_h[kTileWarps][kTile];
        float g = 0.0f, hsum = 0.0f;
        for (int e = e0 + warp; e < e1; e += 8 * kTileWarps) {
            float v[8], h[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int eu = e + u * kTileWarps;
                const bool in = eu < e1;
                v[u] = in ? gpart[(size_t)eu * stride + lane] : 0.0f;
                h[u] = (kFc && in) ? gpart[(size_t)eu * stride + kTile + lane] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                g += v[u];
                if (kFc) hsum += h[u];
            }
        }
        red_g[warp][lane] = g;
        if (kFc) red_h[warp][lane] = hsum;
        __syncthreads();
        g = red_g[0][lane];
        if (kFc) hnn = red_h[0][lane];
#pragma unroll
        for (int w = 1; w < kTileWarps; ++w) {
            g += red_g[w][lane];
            if (kFc) hnn += red_h[w][lane];
        }
        const bool ok = valid && hnn > 0.0f;
        const float sn = ok ? g / (hnn * pb.damp1) : 0.0f;
        if (warp == 0) {
            gn[n] = ok ? g : 0.0f;
            if (kFc) Hnn[n] = ok ? hnn : 0.0f;
        }
        // the correction of entry i of the current batch (hv: its prefetched
        // H_fd values, or null to load them)
        auto correct = [&](int i, const float* hv) {
            const unsigned mask = __shfl_sync(0xffffffffu, mine.mask, i);
            const int po = __shfl_sync(0xffffffffu, mine.pair_off, i);
            const int sl = __shfl_sync(0xffffffffu, slot, i);
            const bool vis = (mask >> lane) & 1u;
            const int nvis = __popc(mask);
            const float* h = Hfd + (size_t)po * 6 + (vis ? rank_of(mask, lane) : 0);
            float v[8];
#pragma unroll
            for (int q = 0; q < 6; ++q) v[q] = vis ? (hv ? hv[q] : h[q * nvis]) * sn : 0.0f;
            v[6] = v[7] = 0.0f;
            if (kAff && vis) {
                // joint brightness: the pair's correction sum_n H_a g_n / H_dd
                const float* ha = Had + (size_t)po * 2 + rank_of(mask, lane);
                v[6] = ha[0] * sn;
                v[7] = ha[nvis] * sn;
            }
            // sums over the lanes by reduce-scatter (nine exchanges instead
            // of thirty): at strides 16, 8, 4 a lane keeps half of its values
            // and adds its partner's copy of them, then two butterfly levels;
            // value q ends on lanes 4q .. 4q + 3
            scatter_level<4>(v, lane, 16);
            scatter_level<2>(v, lane, 8);
            scatter_level<1>(v, lane, 4);
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            if ((lane & 3) == 0 && lane < 24) ent_part[(size_t)sl * kEntryPartial + coff + (lane >> 2)] = v[0];
            else if (kAff && (lane & 3) == 0)
                ent_part[(size_t)sl * kEntryPartial + acol + ((lane - 24) >> 2)] = v[0];
        };
        int i = warp;
        if (!kFc) {
#pragma unroll
            for (int r = 0; r < kPointPre; ++r, i += kTileWarps)
                if (i < cnt0) correct(i, hpre[r]);
        }
#pragma unroll 2
        for (; i < cnt0; i += kTileWarps) correct(i, nullptr);
        for (int b = 32; b < ne; b += 32) {
            mine = Entry{0, 0u, 0, 0};
            slot = 0;
            if (b + lane < ne) {
                mine = pb.entries[e0 + b + lane];
                slot = pb.entry_slot[e0 + b + lane];
            }
            const int cnt = min(32, ne - b);
#pragma unroll 2
            for (int j = warp; j < cnt; j += kTileWarps) correct(j, nullptr);
        }
    }
    if (warp == kTileWarps - 1) tile_stats_from_entries(pb, estats, ddsq_t, tstats, t, e0, e1, lane);
}

// ---------------------------------------------------------------------------
// IC solve (Sec. 3.5 step 4): Dtheta = -S^-1 y, one CTA per target frame:
// nine warps take the frame's six rows and the anchor frame's three
// translation rows of the compact S^-1 (double-float GEMV against y), then
// the exact gauge constraint and the frame's update are written (the pose
// update itself follows in the next launch, one frame per CTA). Frames
// without residuals get a zero update.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(9 * 32)
ic_solve_kernel(SolveArgs a, const dfloat* __restrict__ Sinv, const double* __restrict__ y)
{
    extern __shared__ dfloat ys[];  // nc, compact order; then F ints
    __shared__ double dth[9], d[6];
    const int fg = blockIdx.x + 1, lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    pdl_trigger();
    // Before the wait: the reduced system's layout and the row of S^-1 this
    // warp multiplies (the first kSinvPre elements per lane, in registers).
    // The precompute, which ends with an ordinary launch, wrote them; no
    // kernel of the iteration writes them.
    const BundleDesc bd = a.bund[a.frame_bundle[fg]];
    const int F = bd.F, f = fg - bd.fo;
    const int* cmap = a.cmap + bd.co;
    const double* tanchor = a.tanchor + (size_t)12 * bd.fo;
    Sinv += bd.so;
    y += (size_t)6 * bd.fo;
    // the reference frame of a bundle (f = 0) and frames without residuals
    // get a zero update
    const int kf = f > 0 ? cmap[f] : -1, nc = 6 * cmap[F], anchor = a.active[bd.fo];
    int* frame_of = reinterpret_cast<int*>(ys + 6 * (F - 1));
    const int r = row < 6 ? 6 * kf + row : (anchor > 0 ? 6 * cmap[anchor] + row - 6 : -1);
    const dfloat* Sr = Sinv + (size_t)(r >= 0 ? r : 0) * nc;
    constexpr int kSinvPre = 8;
    dfloat pre[kSinvPre];
#pragma unroll
    for (int q = 0; q < kSinvPre; ++q) {
        const int c = lane + 32 * q;
        pre[q] = (kf >= 0 && r >= 0 && c < nc) ? Sr[c] : df_make(0.0f, 0.0f);
    }
    if (kf >= 0) {
        for (int g = 1 + threadIdx.x; g < F; g += blockDim.x) {
            const int k = cmap[g];
            if (k >= 0) frame_of[k] = g;
        }
    }
    pdl_wait();
    // the frame's brightness pair from this step's residuals (the next
    // residual pass reads it)
    if (a.photo_sums && f > 0 && threadIdx.x == 0)
        photo_update_frame(a.photo_sums + (size_t)5 * fg, a.fc + (size_t)fg * kFrameConst);
    if (kf < 0) {
        if (row == 0) {
            if (lane < 6) d[lane] = 0.0;
            __syncwarp();
            write_update_lanes(a, fg, d, lane);
        }
        return;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
        ys[c] = df_from_double(y[(size_t)frame_of[c / 6] * 6 + c % 6]);
    __syncthreads();
    if (r >= 0) {
        DfAcc acc;
#pragma unroll
        for (int q = 0; q < kSinvPre; ++q) {
            const int c = lane + 32 * q;
            if (c < nc) acc.add_prod(pre[q], ys[c]);
        }
        for (int c = lane + 32 * kSinvPre; c < nc; c += 32) acc.add_prod(Sr[c], ys[c]);
        float ss = acc.s, cc = acc.c;
        warp_sum_pair(ss, cc);
        if (lane == 0) dth[row] = -((double)ss + (double)cc);
    }
    __syncthreads();
    if (row != 0) return;
    if (lane < 6) {
        double v = dth[lane];
        if (lane < 3 && anchor > 0) v = fma(-gauge_alpha(tanchor + 12 * anchor + 9, dth + 6), tanchor[12 * f + 9 + lane], v);
        d[lane] = v;
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, lane >= 6 || isfinite(d[lane]));
    if (!ok) {
        if (lane == 0) flag_error(a.err, a.frame_bundle[fg], kErrNonFinite);
        if (lane < 6) d[lane] = 0.0;
        __syncwarp();
    }
    write_update_lanes(a, fg, d, lane);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_depth_update(const LaunchCtx& L, const SolveArgs& a, bool ic_rule, int apply)
{
    const DepthState& ds = ic_rule ? L.ds_ic : L.ds_fc;
    const int grid = L.pb.T + (apply ? L.pb.F - 1 : 0);  // + one CTA per frame's pose update
    if (ic_rule)
        return launch_pdl(ds.Had ? depth_update_kernel<true, true> : depth_update_kernel<true, false>, grid,
                          kTileWarps * 32, 0, L.stream, L.pb, ds, L.fs.dth2, L.ic.inv_hnn, L.ic.inv_d0, L.it.dcur,
                          L.it.dprev, L.it.ddsq_t, apply, a);
    else
        return launch_pdl(ds.Had ? depth_update_kernel<false, true> : depth_update_kernel<false, false>, grid,
                          kTileWarps * 32, 0, L.stream, L.pb, ds, L.fs.dth2, (const double*)nullptr,
                          (const double*)nullptr, L.it.dcur, L.it.dprev, L.it.ddsq_t, apply, a);
    return cudaGetLastError();
}

template <int PMAX, bool A, int DT, int WARPS, bool J = false>
static cudaError_t ic_residual_w(const LaunchCtx& L, int have_prev)
{
    const int blocks = (L.pb.E + WARPS - 1) / WARPS;
    return launch_pdl(ic_residual_kernel<PMAX, A, DT, WARPS, J>, blocks, WARPS * 32, 0, L.stream, L.pb, L.fs.fc,
                      L.fs.fc_prev, L.it.dcur, L.it.dprev, L.ic.J4, L.ent_part, L.it.gpart, L.it.estats,
                      have_prev, L.photo);
}

// warps (entries) per CTA: the autotuner's choice for the accumulating pass
// (4, 8 or 16); the evaluation pass keeps 8
template <int PMAX, bool A, int DT>
static cudaError_t ic_residual_p(const LaunchCtx& L, int have_prev)
{
    // the brightness pairs as unknowns: their own instance, 8 warps
    if (A && L.photo == 2) return ic_residual_w<PMAX, A, DT, kResWarps, A>(L, have_prev);
    if (A && L.res_warps == 4) return ic_residual_w<PMAX, A, DT, 4>(L, have_prev);
    if (A && L.res_warps == 16) return ic_residual_w<PMAX, A, DT, 16>(L, have_prev);
    return ic_residual_w<PMAX, A, DT, kResWarps>(L, have_prev);
}

cudaError_t launch_ic_residual(const LaunchCtx& L, bool accum, int have_prev)
{
    if (L.pb.E == 0) return cudaSuccess;
#define PBA_C(PM, A)                                                           \
    [&]() {                                                                    \
        switch (L.pb.dtype) {                                                  \
        case PBA_F32: return ic_residual_p<PM, A, PBA_F32>(L, have_prev);      \
        case PBA_F16: return ic_residual_p<PM, A, PBA_F16>(L, have_prev);      \
        default: return ic_residual_p<PM, A, PBA_BF16>(L, have_prev);          \
        }                                                                      \
    }()
    if (L.pb.P <= 8) return accum ? PBA_C(8, true) : PBA_C(8, false);
    return accum ? PBA_C(16, true) : PBA_C(16, false);
#undef PBA_C
}

template <int PMAX, bool A, int DT>
static cudaError_t fc_residual_p(const LaunchCtx& L, int have_prev)
{
    const int blocks = (L.pb.E + kResWarps - 1) / kResWarps;
    // the brightness pairs as unknowns: their own instance
    auto k = (A && L.photo == 2) ? fc_residual_kernel<PMAX, A, DT, A> : fc_residual_kernel<PMAX, A, DT, false>;
    return launch_pdl(k, blocks, kResWarps * 32, 0, L.stream, L.pb, L.fs.fc, L.fs.fc_prev, L.it.dcur, L.it.dprev,
                      L.Hfd_fc, L.ent_part, L.it.gpart, L.it.estats, have_prev, L.photo, L.Had_fc, L.aff_part);
}

cudaError_t launch_fc_residual(const LaunchCtx& L, bool accum, int have_prev)
{
    if (L.pb.E == 0) return cudaSuccess;
#define PBA_C(PM, A)                                                           \
    [&]() {                                                                    \
        switch (L.pb.dtype) {                                                  \
        case PBA_F32: return fc_residual_p<PM, A, PBA_F32>(L, have_prev);      \
        case PBA_F16: return fc_residual_p<PM, A, PBA_F16>(L, have_prev);      \
        default: return fc_residual_p<PM, A, PBA_BF16>(L, have_prev);          \
        }                                                                      \
    }()
    if (L.pb.P <= 8) return accum ? PBA_C(8, true) : PBA_C(8, false);
    return accum ? PBA_C(16, true) : PBA_C(16, false);
#undef PBA_C
}

cudaError_t launch_ic_point(const LaunchCtx& L, bool accum)
{
    const bool aff = accum && L.photo == 2;
    auto k = aff ? point_kernel<true, false, true> : accum ? point_kernel<true, false> : point_kernel<false, false>;
    return launch_pdl(k, L.pb.T, kTileWarps * 32, 0, L.stream, L.pb, L.it.gpart, L.ic.Hfd, L.ic.Hnn,
                      L.ds_ic.gn, L.ent_part, 6, L.it.estats, L.it.ddsq_t, L.tstats,
                      (const float*)(L.photo == 2 ? L.ic.Had : nullptr), kPhotoColIc + 2);
}

cudaError_t launch_fc_point(const LaunchCtx& L, bool accum)
{
    const bool aff = accum && L.photo == 2;
    auto k = aff ? point_kernel<true, true, true> : accum ? point_kernel<true, true> : point_kernel<false, true>;
    return launch_pdl(k, L.pb.T, kTileWarps * 32, 0, L.stream, L.pb, L.it.gpart, L.Hfd_fc, L.ds_fc.Hnn,
                      L.ds_fc.gn, L.ent_part, 27, L.it.estats, L.it.ddsq_t, L.tstats,
                      (const float*)(L.photo == 2 ? L.Had_fc : nullptr), kPhotoColFc + 2);
}

// FP32 pass constants and previous R|t of frames [f0, f0 + nf) from their
// FP64 poses (set-up and pba_set_params), one warp per frame: the same
// arithmetic as the pose updates, so a state restored from its FP64
// parameters continues exactly as the uninterrupted run.
__global__ void frame_consts_kernel(SolveArgs a, int f0, int nf, int init_photo)
{
    __shared__ double sh[4][12];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, f = f0 + blockIdx.x * 4 + w;
    if (f >= f0 + nf) return;
    double* p = sh[w];
    if (lane < 12) p[lane] = a.poses64[12 * f + lane];
    __syncwarp();
    write_frame_lanes(a, f, p, p, p + 9, lane);
    if (init_photo && lane < 2) a.fc[(size_t)f * kFrameConst + kFrameAlpha + lane] = lane == 0 ? 1.0f : 0.0f;
}

cudaError_t launch_frame_consts(const SolveArgs& a, int f0, int nf, cudaStream_t st, int init_photo)
{
    if (nf <= 0) return cudaSuccess;
    frame_consts_kernel<<<(nf + 3) / 4, 128, 0, st>>>(a, f0, nf, init_photo);
    return cudaGetLastError();
}

cudaError_t launch_ic_solve(const SolveArgs& a, const dfloat* Sinv, const double* y, cudaStream_t st)
{
    return launch_pdl(ic_solve_kernel, a.F - 1, 9 * 32, sizeof(dfloat) * a.n6 + sizeof(int) * a.Fmax, st, a,
                      Sinv, y);
}

cudaError_t iter_setup()
{
    // dynamic shared memory above the default 48 KB for the largest systems
    // (1024 frames: 6138 rows)
    cudaError_t e = cudaFuncSetAttribute(ic_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(dfloat) * 6 * 1023 + sizeof(int) * 1024));
    return e;
}

}  // namespace pba
