// Fixed-order reductions shared by the per-frame kernels. Sums are kept as
// unevaluated FP32 pairs (s, c): Knuth's two-sum per added value (branch-free
// and error-free), then pair additions across lanes and warps, converted to
// FP64 (or normalised to double-float) once at the end. GB300 issues FP64
// slowly; this keeps the reductions on the FP32 pipes while carrying about
// 48 bits. Every sum has a fixed order: results are deterministic.
#pragma once

#include "pba_kernels.cuh"

namespace pba {

__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v)
{
    const float t = s + v;
    const float bb = t - s;
    c += (s - (t - bb)) + (v - bb);
    s = t;
}

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

// Sum over the entry rows [s0, s1) of a frame (its slots frame_entry[f] ..
// frame_entry[f + 1]) of
// row[k] (minus row[SUB + k - SUB_FROM] for k >= SUB_FROM when SUB >= 0),
// k < NCOMP. Thread t takes rows t, t + THREADS, ... and loads each row's
// partials as float4 chunks, so a frame of up to THREADS entries is read in
// one latency round. Thread k < NCOMP receives component k as (vs, vc).
// All threads of the CTA must call it.
template <int NCOMP, int SUB, int SUB_FROM, int THREADS>
__device__ inline void frame_rows_sum(const float* __restrict__ ent_part, int s0, int s1, float& vs, float& vc)
{
    constexpr int kWarps = THREADS / 32;
    constexpr int kLast = SUB < 0 ? NCOMP - 1
                                  : (NCOMP - 1 > SUB + NCOMP - 1 - SUB_FROM ? NCOMP - 1
                                                                            : SUB + NCOMP - 1 - SUB_FROM);
    constexpr int kChunks = kLast / 4 + 1;
    static_assert(4 * kChunks <= kEntryPartial, "row chunks");
    __shared__ float red_s[kWarps][NCOMP], red_c[kWarps][NCOMP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float s[NCOMP], c[NCOMP];
#pragma unroll
    for (int k = 0; k < NCOMP; ++k) s[k] = c[k] = 0.0f;
    for (int i = s0 + tid; i < s1; i += THREADS) {
        const float4* row = reinterpret_cast<const float4*>(ent_part + (size_t)i * kEntryPartial);
        float v[4 * kChunks];
#pragma unroll
        for (int q = 0; q < kChunks; ++q) {
            const float4 x = row[q];
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
#pragma unroll
        for (int k = 0; k < NCOMP; ++k)
            two_sum_acc(s[k], c[k], (SUB >= 0 && k >= SUB_FROM) ? v[k] - v[SUB + k - SUB_FROM] : v[k]);
    }
#pragma unroll
    for (int k = 0; k < NCOMP; ++k) {
        warp_sum_pair(s[k], c[k]);
        if (lane == 0) {
            red_s[warp][k] = s[k];
            red_c[warp][k] = c[k];
        }
    }
    __syncthreads();
    vs = vc = 0.0f;
    if (tid < NCOMP) {
        vs = red_s[0][tid];
        vc = red_c[0][tid];
        for (int w = 1; w < kWarps; ++w) two_sum_add(vs, vc, red_s[w][tid], red_c[w][tid]);
    }
}

// Statistics of a pass into the slots (raw sums: energy, r^2, count of the
// current pass; max displacement, |Dtheta|^2, Dd^2 of the previous update):
// every thread folds a strided share of the tiles, then warps and the block
// combine them in a fixed order. All threads of the CTA must call it.
template <int THREADS>
__device__ inline void stats_block(const DevProblem& pb, const TileStats* __restrict__ tstats,
                                   const float* __restrict__ dthsq, double* __restrict__ stats,
                                   int slot_cur, int slot_prev)
{
    constexpr int kWarps = THREADS / 32;
    __shared__ double res[6];
    __shared__ float sh_s[4][kWarps], sh_c[4][kWarps], sh_m[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0}, m = 0.0f;
    for (int i0 = tid; i0 < pb.T; i0 += THREADS * 4) {
        TileStats ts[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + THREADS * u;
            ts[u] = i < pb.T ? tstats[i] : TileStats{0, 0, 0, 0, 0, 0, 0, 0};
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            two_sum_acc(s[0], c[0], ts[u].energy);
            two_sum_acc(s[1], c[1], ts[u].sumsq);
            two_sum_acc(s[2], c[2], ts[u].count);
            two_sum_acc(s[3], c[3], ts[u].ddsq);
            m = fmaxf(m, ts[u].maxdisp);
        }
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
        for (int w = 1; w < kWarps; ++w) two_sum_add(vs, vc, sh_s[tid][w], sh_c[tid][w]);
        res[tid == 3 ? 4 : tid] = (double)vs + (double)vc;
    }
    if (tid == 4) {
        float mm = 0.0f;
        for (int w = 0; w < kWarps; ++w) mm = fmaxf(mm, sh_m[w]);
        res[3] = mm;
    }
    if (warp == 1 && slot_prev >= 0) {
        // |Dtheta|^2 over the frames: lanes take frames, then a butterfly
        float q = 0.0f, qc = 0.0f;
        for (int f = lane; f < pb.F; f += 32) two_sum_acc(q, qc, dthsq[f]);
        warp_sum_pair(q, qc);
        if (lane == 0) res[5] = (double)q + (double)qc;
    }
    __syncthreads();
    // raw sums only (the host forms the RMS and the norms): no FP64 square
    // root or division on the device
    if (tid == 0) {
        if (slot_cur >= 0) {
            double* st = stats + (size_t)slot_cur * kStats;
            st[0] = res[0];
            st[1] = res[1];
            st[2] = res[2];
        }
        if (slot_prev >= 0) {
            double* st = stats + (size_t)slot_prev * kStats;
            st[3] = res[3];
            st[5] = res[4];
            st[4] = res[5];
        }
    }
}

}  // namespace pba
