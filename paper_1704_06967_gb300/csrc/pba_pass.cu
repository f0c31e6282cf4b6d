// IC precompute (Sec. 3.5: J, W_0, H blocks at p_0) and the fixed-order
// per-frame reductions. The per-iteration kernels (IC and FC) are in
// pba_iter.cu.
//
// One CTA owns one tile of 32 points (lane = point). Its warps take the
// tile's entries (target frames that see at least one of the tile's points)
// round-robin, so every sum over a point's frames completes inside the CTA
// and every per-frame sum is written once per entry, then reduced across
// entries in a fixed order: results are deterministic run to run.
#include "pba_kernels.cuh"
#include "pba_reduce.cuh"

namespace pba {

namespace {

constexpr int kPreWarps = 8;   // entries per CTA of the precompute
constexpr int kTileWarps = 4;  // warps per CTA of the per-tile kernels

__device__ __forceinline__ int rank_in(unsigned mask, int lane)
{
    return __popc(mask & ((1u << lane) - 1u));
}

}  // namespace

// ---------------------------------------------------------------------------
// IC precompute (Sec. 3.4-3.5) at the current parameters p_0, one warp per
// (tile, frame) entry, lane = point. Per residual: the template gradient
// (central differences at the integer template pixel, gathered at set-up),
// the proxy-warp Jacobian row in pixel units
//   c = (1/zbar0) (g_u f_x, g_v f_y, -(g_u f_x x + g_v f_y y)),
//   m = zbar0 R0 c - e_z (t0 . R0 c)            (m = M^T c),
//   J = [d0 m, (R0 x~) x m, m . t0],
// the residual and Huber weight at p_0 (J = 0 when invalid there), and the
// H blocks from the stored rows: H_fd per pair, H_ff (21 unique) per entry,
// and each lane's share of H_dd (summed over the tile's entries by
// ic_hdd_kernel). FP32 throughout (GB300's FP64 issue rate would make this
// pass FP64-bound); J is stored in FP32 either way and H is formed from the
// stored rows, so H = J^T W_0 J holds for the J the iterations use. Pattern
// pixels go in groups of four: their taps are issued together and their
// rows are exactly seven float4 chunks, stored as soon as they are formed.
// kAff (the brightness pairs as unknowns): the frame block gains the columns
// I_0 and 1 (the template-side increment (1 + da) I_0 + db), so per entry
// also H_pa (12 sums: sum w0 J_a I_0, sum w0 J_a), H_aa (sum w0 I_0^2,
// sum w0 I_0, sum w0) and per pair J_d^T W_0 [I_0, 1] and the mask of the
// pattern pixels valid at p_0 (the iterations' brightness gradient keeps
// the residual set of p_0, like the stored rows).
// ---------------------------------------------------------------------------
template <int PMAX, int DT, bool kAff>
__global__ void __launch_bounds__(kPreWarps * 32, 2)
ic_precompute_kernel(DevProblem pb, const float* __restrict__ fconst, const double* __restrict__ d0_64,
                     const float2* __restrict__ G0p, IcStore ic, const unsigned char* __restrict__ todo)
{
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * kPreWarps + (threadIdx.x >> 5);
    if (e >= pb.E) return;
    const Entry en = pb.entries[e];
    if (todo && !todo[en.f]) return;  // window update: only the frames that entered
    float* ent_part = ic.part;
    float* hpart = ic.hpart;
    const int P = pb.P, NC = (7 * P + 3) / 4;
    const float k = pb.huber_k;
    float hff[21];
#pragma unroll
    for (int q = 0; q < 21; ++q) hff[q] = 0.0f;
    float hnn = 0.0f;
    float aff[kAffComp];  // kAff: H_pa (a-major: [a][I_0, 1]), H_aa (I_0^2, I_0, 1)
#pragma unroll
    for (int q = 0; q < kAffComp; ++q) aff[q] = 0.0f;
    if ((en.mask >> lane) & 1u) {
        const int n = en.tile * kTile + lane;
        const int nvis = __popc(en.mask), rank = rank_in(en.mask, lane);
        float had[2] = {0.0f, 0.0f};
        unsigned vm = 0u;
        const float* c = fconst + (size_t)en.f * kFrameConst;
        const float d0 = (float)d0_64[n];
        const float2 xc = pb.xn[n];
        const float ax = fmaf(c[0], xc.x, fmaf(c[1], xc.y, c[2]));
        const float ay = fmaf(c[3], xc.x, fmaf(c[4], xc.y, c[5]));
        const float az = fmaf(c[6], xc.x, fmaf(c[7], xc.y, c[8]));
        const float t0x = c[9], t0y = c[10], t0z = c[11];
        const float umax = (float)(pb.W - 3), vmax = (float)(pb.H - 3);
        const unsigned row0 = (unsigned)en.f * (unsigned)pb.H, pitch = (unsigned)pb.pitch;
        float hfd[6] = {0, 0, 0, 0, 0, 0};
        float4* dst = ic.J4 + (size_t)en.pair_off * NC + rank;
#pragma unroll
        for (int g = 0; g < PMAX; g += 4) {
            if (g < P) {
                asm volatile("" ::: "memory");
                unsigned base[4], ok = 0;
                float wa[4], wb[4], I0[4], gu[4], gv[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int j = g + jj;
                    if (j < P) {
                        const size_t ti = ((size_t)en.tile * P + j) * kTile + lane;
                        I0[jj] = pb.I0p[ti];
                        const float2 gg = G0p[ti];
                        gu[jj] = gg.x;
                        gv[jj] = gg.y;
                        const float a0 = ax + c[12 + 3 * j], a1 = ay + c[13 + 3 * j], a2 = az + c[14 + 3 * j];
                        const float qx = fmaf(d0, t0x, a0), qy = fmaf(d0, t0y, a1), qz = fmaf(d0, t0z, a2);
                        const float iz = 1.0f / qz;
                        const float u = fmaf(pb.fx * qx, iz, pb.cx), v = fmaf(pb.fy * qy, iz, pb.cy);
                        const float fu = floorf(u), fv = floorf(v);
                        if (qz > 0.0f && fu >= 1.0f && fu <= umax && fv >= 1.0f && fv <= vmax) ok |= 1u << jj;
                        const unsigned x = (unsigned)(int)fminf(fmaxf(fu, 1.0f), umax);
                        const unsigned y = (unsigned)(int)fminf(fmaxf(fv, 1.0f), vmax);
                        wa[jj] = u - fu;
                        wb[jj] = v - fv;
                        base[jj] = (row0 + y) * pitch + x;
                    }
                }
                float val[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    if (g + jj < P) {
                        const unsigned b = base[jj];
                        const float i00 = load_px_t<DT>(pb.img, b), i10 = load_px_t<DT>(pb.img, b + 1);
                        const float i01 = load_px_t<DT>(pb.img, b + pitch);
                        const float i11 = load_px_t<DT>(pb.img, b + pitch + 1);
                        const float top = fmaf(wa[jj], i10 - i00, i00);
                        const float bot = fmaf(wa[jj], i11 - i01, i01);
                        val[jj] = fmaf(wb[jj], bot - top, top);
                    }
                }
                float Jr[28];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int j = g + jj;
                    float J[7] = {0, 0, 0, 0, 0, 0, 0};
                    if (j < P && ((ok >> jj) & 1u)) {
                        const float a0 = ax + c[12 + 3 * j], a1 = ay + c[13 + 3 * j], a2 = az + c[14 + 3 * j];
                        const float qz = fmaf(d0, t0z, a2);
                        const float r0 = I0[jj] - fmaf(c[kFrameAlpha], val[jj], c[kFrameAlpha + 1]);
                        const float w0 = huber_w(r0, k);
                        const float x = xc.x + pb.pat[2 * j] / pb.fx, y = xc.y + pb.pat[2 * j + 1] / pb.fy;
                        const float zb = qz / d0;
                        const float izb = 1.0f / zb;
                        const float gx = gu[jj] * pb.fx, gy = gv[jj] * pb.fy;
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
                        if (kAff) {
                            const float wi = w0 * I0[jj];
#pragma unroll
                            for (int a = 0; a < 6; ++a) {
                                aff[2 * a] = fmaf(wi, J[a], aff[2 * a]);
                                aff[2 * a + 1] = fmaf(w0, J[a], aff[2 * a + 1]);
                            }
                            aff[12] = fmaf(wi, I0[jj], aff[12]);
                            aff[13] += wi;
                            aff[14] += w0;
                            had[0] = fmaf(wi, J[6], had[0]);
                            had[1] = fmaf(w0, J[6], had[1]);
                            vm |= 1u << j;
                        }
                    }
#pragma unroll
                    for (int a = 0; a < 7; ++a) Jr[7 * jj + a] = J[a];
                }
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const int ch = 7 * (g / 4) + q;
                    if (ch < NC)
                        dst[(size_t)ch * nvis] = make_float4(Jr[4 * q], Jr[4 * q + 1], Jr[4 * q + 2], Jr[4 * q + 3]);
                }
            }
        }
        float* hd = ic.Hfd + (size_t)en.pair_off * 6 + rank;
#pragma unroll
        for (int a = 0; a < 6; ++a) hd[a * nvis] = hfd[a];
        if (kAff) {
            float* ha = ic.Had + (size_t)en.pair_off * 2 + rank;
            ha[0] = had[0];
            ha[nvis] = had[1];
            ic.vmask0[en.pair_off + rank] = vm;
        }
    }
    hpart[(size_t)e * kTile + lane] = hnn;
    // the entry's 21 H_ff sums over the lanes by reduce-scatter (25
    // exchanges instead of 105): sums 0-15 end on lanes 2q, 2q + 1, sums
    // 16-20 on lanes 4q .. 4q + 3
    float a[16], b[8];
#pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = hff[q];
#pragma unroll
    for (int q = 0; q < 8; ++q) b[q] = q < 5 ? hff[16 + q] : 0.0f;
    scatter_level<8>(a, lane, 16);
    scatter_level<4>(a, lane, 8);
    scatter_level<2>(a, lane, 4);
    scatter_level<1>(a, lane, 2);
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
    scatter_level<4>(b, lane, 16);
    scatter_level<2>(b, lane, 8);
    scatter_level<1>(b, lane, 4);
    b[0] += __shfl_xor_sync(0xffffffffu, b[0], 2);
    b[0] += __shfl_xor_sync(0xffffffffu, b[0], 1);
    float* o = ent_part + (size_t)pb.entry_slot[e] * kEntryPartial;
    if ((lane & 1) == 0) o[lane >> 1] = a[0];
    if ((lane & 3) == 0 && lane < 20) o[16 + (lane >> 2)] = b[0];
    if (kAff) {
        warp_sum<kAffComp>(aff);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < kAffComp; ++q) o[kAffCol + q] = aff[q];
    }
}

// H_dd per point (entries of its tile added in order; entries of frames
// outside the window have no visible lanes) and the FP64 reciprocals 1/H_dd
// and 1/d_0 that the depth back-substitution multiplies by.
__global__ void __launch_bounds__(kTileWarps * 32)
ic_hdd_kernel(DevProblem pb, const float* __restrict__ hpart, const double* __restrict__ d64, IcStore ic)
{
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * kTileWarps + (threadIdx.x >> 5);
    if (t >= pb.T) return;
    const int n = t * kTile + lane;
    const int e0 = pb.tile_entry[t], e1 = pb.tile_entry[t + 1];
    const bool valid = pb.valid_pt[n];
    const double d0 = d64[n];
    float tot = 0.0f;
    for (int e = e0; e < e1; e += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = (e + u < e1 && ((pb.entries[e + u].mask >> lane) & 1u)) ? hpart[(size_t)(e + u) * kTile + lane]
                                                                           : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) tot += v[u];
    }
    const bool ok = valid && tot > 0.0f;
    ic.Hnn[n] = valid ? tot : 0.0f;
    ic.inv_hnn[n] = ok ? 1.0 / ((double)tot * (double)pb.damp1) : 0.0;
    ic.inv_d0[n] = 1.0 / d0;
}

// ---------------------------------------------------------------------------
// Fixed-order per-frame reduction of entry partials (one CTA per frame), plus
// one extra block that folds the tile statistics into the statistics slots
// (pba_reduce.cuh).
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 512;

template <int NCOMP, int SUB, int SUB_FROM>
__global__ void __launch_bounds__(kReduceThreads)
frame_reduce_kernel(DevProblem pb, const float* __restrict__ ent_part, double* __restrict__ out,
                    const TileStats* __restrict__ tstats, const float* __restrict__ dthsq,
                    double* __restrict__ stats, int slot_cur, int slot_prev, int nframes_blocks)
{
    pdl_trigger();
    if ((int)blockIdx.x < nframes_blocks) {
        const int f = blockIdx.x + 1;
        // the frame's slot range is fixed at set-up: read before the wait
        const int s0 = pb.frame_entry[f], s1 = pb.frame_entry[f + 1];
        pdl_wait();
        float vs, vc;
        frame_rows_sum<NCOMP, SUB, SUB_FROM, kReduceThreads>(ent_part, s0, s1, vs, vc);
        if (threadIdx.x < NCOMP) out[(size_t)f * NCOMP + threadIdx.x] = (double)vs + (double)vc;
        return;
    }
    pdl_wait();
    stats_block<kReduceThreads>(pb, tstats, dthsq, stats, slot_cur, slot_prev);
}

// ---------------------------------------------------------------------------
// launchers (dispatch on the pattern capacity and the image storage type)
// ---------------------------------------------------------------------------
#define PBA_DISPATCH_DT(dtype, CALL) \
    ((dtype) == PBA_F32 ? CALL(PBA_F32) : (dtype) == PBA_F16 ? CALL(PBA_F16) : CALL(PBA_BF16))

template <int PMAX, int DT>
static cudaError_t ic_precompute_p(const LaunchCtx& L, const unsigned char* todo)
{
    const int blocks = (L.pb.E + kPreWarps - 1) / kPreWarps;
    if (L.ic.Had)
        ic_precompute_kernel<PMAX, DT, true><<<blocks, kPreWarps * 32, 0, L.stream>>>(
            L.pb, L.fs.fc, L.ds_ic.d0_64, L.it.G0p, L.ic, todo);
    else
        ic_precompute_kernel<PMAX, DT, false><<<blocks, kPreWarps * 32, 0, L.stream>>>(
            L.pb, L.fs.fc, L.ds_ic.d0_64, L.it.G0p, L.ic, todo);
    return cudaGetLastError();
}

cudaError_t launch_ic_precompute(const LaunchCtx& L, const unsigned char* todo)
{
    cudaError_t e = cudaSuccess;
    if (L.pb.E > 0) {
#define PBA_C8(DT) ic_precompute_p<8, DT>(L, todo)
#define PBA_C16(DT) ic_precompute_p<16, DT>(L, todo)
        e = L.pb.P <= 8 ? PBA_DISPATCH_DT(L.pb.dtype, PBA_C8) : PBA_DISPATCH_DT(L.pb.dtype, PBA_C16);
#undef PBA_C8
#undef PBA_C16
        if (e != cudaSuccess) return e;
    }
    ic_hdd_kernel<<<(L.pb.T + kTileWarps - 1) / kTileWarps, kTileWarps * 32, 0, L.stream>>>(
        L.pb, L.ic.hpart, L.ds_ic.d0_64, L.ic);
    return cudaGetLastError();
}

cudaError_t launch_frame_reduce(const LaunchCtx& L, int off, int ncomp, double* out, int slot_cur,
                                int slot_prev, bool frames, int sub, int sub_from, const float* src)
{
    const int nfb = frames ? L.pb.F - 1 : 0;
    const dim3 grid(nfb + 1), block(kReduceThreads);
    if (off != 0) return cudaErrorInvalidValue;
    const float* rows = src ? src : L.ent_part;
#define PBA_R(NC, SB, SF)                                                                           \
    launch_pdl(frame_reduce_kernel<NC, SB, SF>, grid, block, 0, L.stream, L.pb, rows, out, L.tstats, \
               L.dthsq, L.stats, slot_cur, slot_prev, nfb)
    if (!frames || (ncomp == 6 && sub == 6 && sub_from == 0)) return PBA_R(6, 6, 0);
    if (ncomp == 21 && sub < 0) return PBA_R(21, -1, 0);
    if (ncomp == 5 && sub < 0) return PBA_R(5, -1, 0);
    if (ncomp == kAffComp && sub < 0) return PBA_R(kAffComp, -1, 0);
    if (ncomp == 27 && sub == 27 && sub_from == 21) return PBA_R(27, 27, 21);
    return cudaErrorInvalidValue;
#undef PBA_R
}

}  // namespace pba
