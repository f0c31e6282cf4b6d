// Learned inverse-depth proposal (an addition to the paper, which starts
// every inverse depth from a base solution): a 96 -> 128 -> 128 -> 128 -> 1
// MLP with GELU maps a point's template patch and samples along its
// epipolar lines in two target frames to an initial inverse depth. It is
// trained on the inverse depths the bundle adjustment converges to.
//
//   mlp_features_kernel   warp per point: the 8 x 8 normalised template
//                         patch and 2 x 16 epipolar matching costs (96 FP32
//                         values)
//   mlp_infer_tc_kernel   inference on the 5th-generation tensor cores:
//                         BF16 weights and activations in shared memory,
//                         tcgen05.mma with the FP32 accumulator in tensor
//                         memory, bias + GELU epilogue from tcgen05.ld
//   mlp_grad_kernel       training: forward and backward of 64 samples per
//                         CTA in FP32 on the SIMT pipes (partial gradients)
//   mlp_adam_kernel       fixed-order sum of the partial gradients and the
//                         Adam update of the FP32 master weights
#include <cmath>
#include <cstdint>

#include "pba_kernels.cuh"
#include "pba_mlp.cuh"
#include "pba_tc.cuh"

namespace pba {

namespace {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool bilinear_any(const DevProblem& pb, int f, float u, float v, float& val)
{
    const float fu = floorf(u), fv = floorf(v);
    if (!(fu >= 0.0f && fu <= (float)(pb.W - 2) && fv >= 0.0f && fv <= (float)(pb.H - 2))) return false;
    const int x = (int)fu, y = (int)fv;
    const float a = u - fu, b = v - fv;
    const size_t base = ((size_t)f * pb.H + y) * pb.pitch + x;
    const float i00 = load_px(pb.img, pb.dtype, base), i10 = load_px(pb.img, pb.dtype, base + 1);
    const float i01 = load_px(pb.img, pb.dtype, base + pb.pitch);
    const float i11 = load_px(pb.img, pb.dtype, base + pb.pitch + 1);
    const float top = (1.0f - a) * i00 + a * i10, bot = (1.0f - a) * i01 + a * i11;
    val = (1.0f - b) * top + b * bot;
    return true;
}

// One warp per point of tiles [tile0, tile0 + ntiles). Lanes share the 8 x 8
// patch (two pixels each, mean and deviation by butterflies); lane
// 16 s + k then takes bin k of frame s: the least mean squared difference
// between the normalised pattern and the target frame over the bin's 16
// inverse depths.
__global__ void __launch_bounds__(128)
mlp_features_kernel(DevProblem pb, const float* __restrict__ fconst, const int* __restrict__ slot_caller,
                    int tile0, int ntiles, float* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int slot = (blockIdx.x * 4 + (threadIdx.x >> 5));
    if (slot >= ntiles * kTile) return;
    const int t = tile0 + slot / kTile, pl = slot % kTile, n = t * kTile + pl;
    const int caller = slot_caller[n];
    if (caller < 0) return;
    float* o = out + (size_t)caller * kMlpIn;
    const int f0 = pb.tile_f0[t];
    const int u = pb.uvs[2 * n], v = pb.uvs[2 * n + 1];
    const size_t ref = (size_t)f0 * pb.H;
    float p[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h, i = k / kMlpPatch, j = k % kMlpPatch;
        const int y = min(max(v + kMlpPatchLo + i, 0), pb.H - 1);
        const int x = min(max(u + kMlpPatchLo + j, 0), pb.W - 1);
        p[h] = load_px(pb.img, pb.dtype, (ref + y) * pb.pitch + x);
    }
    const float mu = warp_sum1(p[0] + p[1]) * (1.0f / (kMlpPatch * kMlpPatch));
    const float ss = warp_sum1((p[0] - mu) * (p[0] - mu) + (p[1] - mu) * (p[1] - mu));
    const float scale = 1.0f / (sqrtf(ss * (1.0f / (kMlpPatch * kMlpPatch))) + kMlpEps);
    o[lane] = (p[0] - mu) * scale;
    o[lane + 32] = (p[1] - mu) * scale;
    // the first two target frames (in frame order) that observe the point:
    // a tile's entries are stored in frame order
    int g[2] = {-1, -1}, found = 0;
    for (int e = pb.tile_entry[t]; e < pb.tile_entry[t + 1] && found < 2; ++e) {
        const Entry en = pb.entries[e];
        if ((en.mask >> pl) & 1u) g[found++] = en.f;
    }
    if (found == 0) {
        o[kMlpPatch * kMlpPatch + lane] = kMlpNoData;
        return;
    }
    if (found == 1) g[1] = g[0];
    const int P = pb.P, s = lane >> 4, k = lane & 15;
    float tm[PBA_MAX_PATTERN], xx[PBA_MAX_PATTERN], xy[PBA_MAX_PATTERN];
    for (int j = 0; j < P; ++j) {
        const int ox = pb.pat[2 * j], oy = pb.pat[2 * j + 1];
        tm[j] = (load_px(pb.img, pb.dtype, (ref + v + oy) * pb.pitch + u + ox) - mu) * scale;
        xx[j] = ((float)(u + ox) - pb.cx) / pb.fx;
        xy[j] = ((float)(v + oy) - pb.cy) / pb.fy;
    }
    const float* c = fconst + (size_t)g[s] * kFrameConst;
    const float step = (kMlpDHi - kMlpDLo) / (kMlpSamples * kMlpSub);
    float best = 3.0e38f;
    for (int i = 0; i < kMlpSub; ++i) {
        const float d = kMlpDLo + ((float)(kMlpSub * k + i) + 0.5f) * step;
        float cost = 0.0f;
        bool ok = true;
        for (int j = 0; j < P && ok; ++j) {
            const float qx = fmaf(c[0], xx[j], fmaf(c[1], xy[j], fmaf(d, c[9], c[2])));
            const float qy = fmaf(c[3], xx[j], fmaf(c[4], xy[j], fmaf(d, c[10], c[5])));
            const float qz = fmaf(c[6], xx[j], fmaf(c[7], xy[j], fmaf(d, c[11], c[8])));
            float val = 0.0f;
            ok = qz > 0.0f && bilinear_any(pb, g[s], pb.fx * qx / qz + pb.cx, pb.fy * qy / qz + pb.cy, val);
            const float r = (val - mu) * scale - tm[j];
            cost = fmaf(r, r, cost);
        }
        best = fminf(best, ok ? cost / (float)P : kMlpNoData);
    }
    o[kMlpPatch * kMlpPatch + lane] = best;
}

// Writes the proposals (clamped to a positive range) as the inverse depths
// of the bundle's points. Pads, and points without any matching data (no
// target frame observes them, or every hypothesis leaves the image), keep
// their inverse depth: the constant-depth initialisation is the fallback.
__global__ void mlp_propose_kernel(const int* __restrict__ slot_caller, int slot0, int nslots,
                                   const float* __restrict__ X, const float* __restrict__ y,
                                   double* __restrict__ d64)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nslots) return;
    const int caller = slot_caller[slot0 + i];
    if (caller < 0) return;
    const float* m = X + (size_t)caller * kMlpIn + kMlpPatch * kMlpPatch;
    bool any = false;
    for (int k = 0; k < kMlpFrames * kMlpSamples; ++k) any |= m[k] != kMlpNoData;
    if (!any) return;
    const float v = y[caller];
    if (isfinite(v)) d64[slot0 + i] = (double)fminf(fmaxf(v, kMlpDMin), kMlpDMax);
}

// ---------------------------------------------------------------------------
// tensor-core inference
// ---------------------------------------------------------------------------
// Instruction descriptor of the layers: FP32 accumulator, BF16 A and B,
// both K-major, N = 128, M = 128.
constexpr uint32_t kIdescBf16 = idesc_bf16(kMlpTileM, kMlpHidden);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    mma_bf16_id(tmem_d, a, b, kIdescBf16, accumulate);
}

// The give-up path of the bounded waits, exercised on purpose: one warp
// waits on a barrier phase that nothing completes (no arrival is ever
// made), gives up after the bound, reports kErrTimeout through the flag and
// exits normally.
__global__ void wait_selftest_kernel(int* err)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t mbar = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait(mbar, 0);
    __syncwarp();
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(err, kErrTimeout);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
    }
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// Shared-memory plan of the inference kernel (bytes).
constexpr uint32_t kOffW1 = 0;
constexpr uint32_t kOffW2 = kOffW1 + kMlpHidden * kMlpIn * 2;
constexpr uint32_t kOffW3 = kOffW2 + kMlpHidden * kMlpHidden * 2;
constexpr uint32_t kOffA = kOffW3 + kMlpHidden * kMlpHidden * 2;
constexpr uint32_t kOffBias = kOffA + kMlpTileM * kMlpHidden * 2;
constexpr uint32_t kOffBar = kOffBias + kMlpBiasFloats * 4 + 12;  // 8-byte aligned below
constexpr uint32_t kInferSmem = ((kOffBar + 7) & ~7u) + 16;

static_assert(kMlpPackedWeightBytes == kOffA, "packed layout = shared-memory image of the weights");

// One CTA of 128 threads takes tiles of 128 points in turn (persistent over
// the tiles); thread r of the CTA owns row r of a tile (TMEM lane r).
__global__ void __launch_bounds__(128, 1)
mlp_infer_tc_kernel(const uint8_t* __restrict__ packed, int n, const float* __restrict__ X,
                    float* __restrict__ out, int* err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    float* bias = reinterpret_cast<float*>(sm + kOffBias);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + ((kOffBar + 7) & ~7u));
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    const uint32_t mbar = smem_u32(bar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kMlpHidden)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights (already in the canonical layout) and the FP32 biases
    {
        const uint4* src = reinterpret_cast<const uint4*>(packed);
        uint4* dst = reinterpret_cast<uint4*>(sm);
        for (uint32_t i = tid; i < kMlpPackedWeightBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
        const float* b = reinterpret_cast<const float*>(packed + kMlpPackedWeightBytes);
        for (int i = tid; i < kMlpBiasFloats; i += blockDim.x) bias[i] = __ldg(b + i);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sA = smem_u32(sm + kOffA);
    const uint32_t sW[3] = {smem_u32(sm + kOffW1), smem_u32(sm + kOffW2), smem_u32(sm + kOffW3)};
    const int Kl[3] = {kMlpIn, kMlpHidden, kMlpHidden};
    uint32_t phase = 0;
    bool ok = true;
    const int ntiles = (n + kMlpTileM - 1) / kMlpTileM;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 TMEM lanes
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int row = tile * kMlpTileM + tid;
        // features of row tid -> BF16, canonical K-major (K = 96)
        {
            const float4* xr = reinterpret_cast<const float4*>(X + (size_t)row * kMlpIn);
#pragma unroll
            for (int c = 0; c < kMlpIn / 8; ++c) {
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                if (row < n) {
                    a = __ldg(xr + 2 * c);
                    b = __ldg(xr + 2 * c + 1);
                }
                const uint4 w = make_uint4(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w), pack_bf16x2(b.x, b.y),
                                           pack_bf16x2(b.z, b.w));
                *reinterpret_cast<uint4*>(sm + kOffA + canon_offset(tid, 8 * c, kMlpIn)) = w;
            }
        }
        float y = 0.0f;
        for (int layer = 0; layer < 3 && ok; ++layer) {
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            if (tid == 0) {
                const int K = Kl[layer];
                const uint32_t sbo = (uint32_t)(K / 8) * 128;
                for (int ks = 0; ks < K / 16; ++ks)
                    mma_bf16(tmem, smem_desc(sA + ks * 256, 128, sbo), smem_desc(sW[layer] + ks * 256, 128, sbo),
                             ks > 0);
                mma_commit(mbar);
            }
            ok = __syncthreads_and(mbar_wait(mbar, phase));
            phase ^= 1;
            if (!ok) break;
            fence_after_sync();
            const float* bl = bias + layer * kMlpHidden;
#pragma unroll 1
            for (int c = 0; c < kMlpHidden / 32; ++c) {
                float v[32];
                tmem_ld32(taddr + c * 32, v);
                if (layer < 2) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float h[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) h[e] = gelu_f(v[8 * q + e] + bl[32 * c + 8 * q + e]);
                        const uint4 w = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                                                   pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
                        *reinterpret_cast<uint4*>(sm + kOffA + canon_offset(tid, 32 * c + 8 * q, kMlpHidden)) = w;
                    }
                } else {
                    const float* w4 = bias + 3 * kMlpHidden;
#pragma unroll
                    for (int e = 0; e < 32; ++e) y = fmaf(gelu_f(v[e] + bl[32 * c + e]), w4[32 * c + e], y);
                }
            }
        }
        if (ok && row < n) out[row] = y + bias[4 * kMlpHidden];
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    }
    if (!ok) {
        // a wait gave up: the outputs of this CTA are undefined (the host
        // sees kErrTimeout). The committed MMAs may still be running and
        // writing this CTA's tensor memory, so wait for that phase again
        // (bounded, longer) before the memory is freed.
        if (tid == 0) atomicOr(err, kErrTimeout);
        mbar_wait(mbar, phase ^ 1u, 1 << 20);
        fence_after_sync();
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kMlpHidden);
    if (tid == 0) mbar_inval(mbar);
}

// FP32 masters -> the inference layout (BF16 weights in the canonical
// layout, FP32 biases and output weights).
__global__ void mlp_pack_kernel(const float* __restrict__ params, uint8_t* __restrict__ packed)
{
    const int total = kMlpHidden * kMlpIn + 2 * kMlpHidden * kMlpHidden;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total + kMlpBiasFloats; i += gridDim.x * blockDim.x) {
        if (i < total) {
            int layer, r, k, K;
            uint32_t base;
            float w;
            if (i < kMlpHidden * kMlpIn) {
                layer = 0;
                K = kMlpIn;
                r = i / K;
                k = i % K;
                base = kOffW1;
                w = params[kMlpOffW1 + i];
            } else {
                const int j = i - kMlpHidden * kMlpIn;
                layer = 1 + j / (kMlpHidden * kMlpHidden);
                K = kMlpHidden;
                r = (j % (kMlpHidden * kMlpHidden)) / K;
                k = j % K;
                base = layer == 1 ? kOffW2 : kOffW3;
                w = params[(layer == 1 ? kMlpOffW2 : kMlpOffW3) + r * K + k];
            }
            *reinterpret_cast<__nv_bfloat16*>(packed + base + canon_offset(r, k, K)) = __float2bfloat16_rn(w);
        } else {
            const int j = i - total;  // b1 b2 b3 w4 b4
            const int src = j < kMlpHidden          ? kMlpOffB1 + j
                            : j < 2 * kMlpHidden    ? kMlpOffB2 + j - kMlpHidden
                            : j < 3 * kMlpHidden    ? kMlpOffB3 + j - 2 * kMlpHidden
                            : j < 4 * kMlpHidden    ? kMlpOffW4 + j - 3 * kMlpHidden
                                                    : kMlpOffB4;
            reinterpret_cast<float*>(packed + kMlpPackedWeightBytes)[j] = params[src];
        }
    }
}

// ---------------------------------------------------------------------------
// training (FP32, SIMT)
// ---------------------------------------------------------------------------
constexpr int kGradRows = 64;      // samples per CTA
constexpr int kGradThreads = 256;
constexpr size_t kGradSmem = (size_t)kGradRows * (kMlpIn + 4 * kMlpHidden) * 4 + kGradRows * 4 * 2;

__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// H = GELU(Z) over the CTA's rows
__device__ __forceinline__ void act_gelu(const float* Z, float* H)
{
    for (int q = threadIdx.x; q < kGradRows * kMlpHidden; q += blockDim.x) H[q] = gelu_f(Z[q]);
}

// Z[s][o] = b[o] + sum_i A[s][i] W[o][i] for the CTA's rows
__device__ __forceinline__ void dense_fwd(const float* A, int K, const float* __restrict__ W,
                                          const float* __restrict__ b, float* Z)
{
    for (int q = threadIdx.x; q < kGradRows * kMlpHidden; q += blockDim.x) {
        const int s = q / kMlpHidden, o = q % kMlpHidden;
        const float* a = A + s * K;
        const float* w = W + (size_t)o * K;
        float acc = __ldg(b + o);
        for (int i = 0; i < K; ++i) acc = fmaf(a[i], __ldg(w + i), acc);
        Z[q] = acc;
    }
}

// dW[o][i] = sum_s dZ[s][o] A[s][i], db[o] = sum_s dZ[s][o] (the first `rows` rows)
__device__ __forceinline__ void dense_wgrad(const float* dZ, const float* A, int K, int rows, float* __restrict__ gW,
                                            float* __restrict__ gb)
{
    for (int q = threadIdx.x; q < kMlpHidden * K; q += blockDim.x) {
        const int o = q / K, i = q % K;
        float acc = 0.0f;
        for (int s = 0; s < rows; ++s) acc = fmaf(dZ[s * kMlpHidden + o], A[s * K + i], acc);
        gW[q] = acc;
    }
    for (int o = threadIdx.x; o < kMlpHidden; o += blockDim.x) {
        float acc = 0.0f;
        for (int s = 0; s < rows; ++s) acc += dZ[s * kMlpHidden + o];
        gb[o] = acc;
    }
}

// dZprev[s][i] = (sum_o dZ[s][o] W[o][i]) GELU'(Zprev[s][i]), in place over Zprev
__device__ __forceinline__ void dense_dgrad(const float* dZ, const float* __restrict__ W, float* Zprev)
{
    for (int q = threadIdx.x; q < kGradRows * kMlpHidden; q += blockDim.x) {
        const int s = q / kMlpHidden, i = q % kMlpHidden;
        float acc = 0.0f;
        for (int o = 0; o < kMlpHidden; ++o)
            acc = fmaf(dZ[s * kMlpHidden + o], __ldg(W + (size_t)o * kMlpHidden + i), acc);
        Zprev[q] = acc * gelu_grad_f(Zprev[q]);
    }
}

// CTA c takes samples [64 c, 64 c + 64) of n; writes its partial gradient
// (kMlpParams floats, same order as the parameters) and its partial loss
// sum to part[c] and loss_part[c].
__global__ void __launch_bounds__(kGradThreads)
mlp_grad_kernel(const float* __restrict__ P, int n, const float* __restrict__ X, const float* __restrict__ T,
                float* __restrict__ part, float* __restrict__ loss_part)
{
    extern __shared__ float gs[];
    float* Xs = gs;                               // rows x 96
    float* Z1 = Xs + kGradRows * kMlpIn;          // rows x 128 pre-activations (then dZ1)
    float* Z2 = Z1 + kGradRows * kMlpHidden;      // (then dZ2)
    float* Z3 = Z2 + kGradRows * kMlpHidden;      // (then dZ3)
    float* Hs = Z3 + kGradRows * kMlpHidden;      // one layer's activations
    float* dy = Hs + kGradRows * kMlpHidden;      // rows
    float* lv = dy + kGradRows;                   // rows
    const int s0 = blockIdx.x * kGradRows, rows = min(kGradRows, n - s0);
    float* G = part + (size_t)blockIdx.x * kMlpParams;
    for (int q = threadIdx.x; q < kGradRows * kMlpIn; q += blockDim.x) {
        const int s = q / kMlpIn;
        Xs[q] = s < rows ? X[(size_t)(s0 + s) * kMlpIn + q % kMlpIn] : 0.0f;
    }
    __syncthreads();
    dense_fwd(Xs, kMlpIn, P + kMlpOffW1, P + kMlpOffB1, Z1);
    __syncthreads();
    act_gelu(Z1, Hs);
    __syncthreads();
    dense_fwd(Hs, kMlpHidden, P + kMlpOffW2, P + kMlpOffB2, Z2);
    __syncthreads();
    act_gelu(Z2, Hs);
    __syncthreads();
    dense_fwd(Hs, kMlpHidden, P + kMlpOffW3, P + kMlpOffB3, Z3);
    __syncthreads();
    // output, loss and dy = (y - t) / n (Hs keeps GELU(Z2) for dW3)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = warp; s < kGradRows; s += kGradThreads / 32) {
        float acc = 0.0f;
        for (int o = lane; o < kMlpHidden; o += 32)
            acc = fmaf(gelu_f(Z3[s * kMlpHidden + o]), __ldg(P + kMlpOffW4 + o), acc);
        acc = warp_sum1(acc);
        if (lane == 0) {
            const float y = acc + __ldg(P + kMlpOffB4);
            const float r = s < rows ? y - T[s0 + s] : 0.0f;
            lv[s] = 0.5f * r * r;
            dy[s] = r / (float)n;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float l = 0.0f;
        for (int s = 0; s < rows; ++s) l += lv[s];
        loss_part[blockIdx.x] = l;
    }
    for (int o = threadIdx.x; o < kMlpHidden; o += blockDim.x) {
        float acc = 0.0f;
        for (int s = 0; s < rows; ++s) acc = fmaf(dy[s], gelu_f(Z3[s * kMlpHidden + o]), acc);
        G[kMlpOffW4 + o] = acc;
    }
    if (threadIdx.x == 0) {
        float acc = 0.0f;
        for (int s = 0; s < rows; ++s) acc += dy[s];
        G[kMlpOffB4] = acc;
    }
    __syncthreads();
    // dZ3 = dy w4 GELU'(Z3), in place
    for (int q = threadIdx.x; q < kGradRows * kMlpHidden; q += blockDim.x) {
        const int s = q / kMlpHidden, o = q % kMlpHidden;
        Z3[q] = dy[s] * __ldg(P + kMlpOffW4 + o) * gelu_grad_f(Z3[q]);
    }
    __syncthreads();
    dense_wgrad(Z3, Hs, kMlpHidden, rows, G + kMlpOffW3, G + kMlpOffB3);
    __syncthreads();
    dense_dgrad(Z3, P + kMlpOffW3, Z2);
    act_gelu(Z1, Hs);
    __syncthreads();
    dense_wgrad(Z2, Hs, kMlpHidden, rows, G + kMlpOffW2, G + kMlpOffB2);
    __syncthreads();
    dense_dgrad(Z2, P + kMlpOffW2, Z1);
    __syncthreads();
    dense_wgrad(Z1, Xs, kMlpIn, rows, G + kMlpOffW1, G + kMlpOffB1);
}

// grad[i] = sum over the parts in order; then (when m, v are given) Adam.
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ part, int nparts,
                                float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                                float lr, float c1, float c2, const float* __restrict__ loss_part,
                                float* __restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss) {
        float l = 0.0f;
        for (int k = 0; k < nparts; ++k) l += loss_part[k];
        *loss = l;
    }
    if (i >= kMlpParams) return;
    float g = 0.0f;
    for (int k = 0; k < nparts; ++k) g += part[(size_t)k * kMlpParams + i];
    if (grad) grad[i] = g;
    if (!m) return;
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

}  // namespace

cudaError_t launch_mlp_features(const DevProblem& pb, const float* fconst, const int* slot_caller, int tile0,
                                int ntiles, float* out, cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;
    mlp_features_kernel<<<(ntiles * kTile + 3) / 4, 128, 0, st>>>(pb, fconst, slot_caller, tile0, ntiles, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_propose(const int* slot_caller, int slot0, int nslots, const float* X, const float* y,
                               double* d64, cudaStream_t st)
{
    if (nslots <= 0) return cudaSuccess;
    mlp_propose_kernel<<<(nslots + 255) / 256, 256, 0, st>>>(slot_caller, slot0, nslots, X, y, d64);
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float* params, uint8_t* packed, cudaStream_t st)
{
    mlp_pack_kernel<<<128, 256, 0, st>>>(params, packed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const uint8_t* packed, int n, const float* X, float* out, int* err, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kInferSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + kMlpTileM - 1) / kMlpTileM;
    const int grid = tiles < sms ? tiles : sms;
    mlp_infer_tc_kernel<<<grid, 128, kInferSmem, st>>>(packed, n, X, out, err);
    return cudaGetLastError();
}

size_t mlp_grad_scratch_floats(int n)
{
    const size_t parts = (size_t)(n + kGradRows - 1) / kGradRows;
    return parts * kMlpParams + parts;
}

cudaError_t launch_mlp_grad_adam(float* params, int n, const float* X, const float* T, float* scratch,
                                 float* grad, float* m, float* v, int step, float lr, float* loss,
                                 cudaStream_t st)
{
    if (n <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGradSmem);
    if (e != cudaSuccess) return e;
    const int parts = (n + kGradRows - 1) / kGradRows;
    float* part = scratch;
    float* loss_part = scratch + (size_t)parts * kMlpParams;
    mlp_grad_kernel<<<parts, kGradThreads, kGradSmem, st>>>(params, n, X, T, part, loss_part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float c1 = 1.0f, c2 = 1.0f;
    if (m) {
        c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)step)));
        c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)step)));
    }
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(params, part, parts, grad, m, v, lr, c1, c2,
                                                               loss_part, loss);
    return cudaGetLastError();
}

}  // namespace pba

// ===========================================================================
// C ABI (context-free part; pba_depth_features and pba_propose_depths live
// with the context in pba_runtime.cu)
// ===========================================================================
extern "C" {

pba_status pba_mlp_pack(const float* params, void* packed, void* cuda_stream)
{
    if (!params || !packed || ((uintptr_t)packed & 15)) return PBA_ERR_ARG;
    return pba::launch_mlp_pack(params, static_cast<uint8_t*>(packed), static_cast<cudaStream_t>(cuda_stream)) ==
                   cudaSuccess
               ? PBA_OK
               : PBA_ERR_CUDA;
}

pba_status pba_mlp_infer(const void* packed, int n, const float* features, float* out, int* dev_flag,
                         void* cuda_stream)
{
    if (!packed || n < 0 || (n > 0 && (!features || !out)) || !dev_flag || ((uintptr_t)packed & 15) ||
        ((uintptr_t)features & 15))
        return PBA_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(dev_flag, 0, sizeof(int), st) != cudaSuccess) return PBA_ERR_CUDA;
    if (pba::launch_mlp_infer(static_cast<const uint8_t*>(packed), n, features, out, dev_flag, st) != cudaSuccess)
        return PBA_ERR_CUDA;
    int flag = 0;
    if (cudaMemcpyAsync(&flag, dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PBA_ERR_CUDA;
    return flag ? PBA_ERR_TIMEOUT : PBA_OK;
}

size_t pba_mlp_scratch_floats(int n) { return n > 0 ? pba::mlp_grad_scratch_floats(n) : 0; }

pba_status pba_wait_selftest(int* dev_flag, void* cuda_stream)
{
    if (!dev_flag) return PBA_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(dev_flag, 0, sizeof(int), st) != cudaSuccess) return PBA_ERR_CUDA;
    pba::wait_selftest_kernel<<<1, 32, 0, st>>>(dev_flag);
    int flag = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&flag, dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PBA_ERR_CUDA;
    return flag ? PBA_ERR_TIMEOUT : PBA_OK;
}

pba_status pba_mlp_grad(const float* params, int n, const float* features, const float* targets, float* grad,
                        float* loss, float* scratch, void* cuda_stream)
{
    if (!params || n < 1 || !features || !targets || !grad || !scratch) return PBA_ERR_ARG;
    return pba::launch_mlp_grad_adam(const_cast<float*>(params), n, features, targets, scratch, grad, nullptr,
                                     nullptr, 0, 0.0f, loss, static_cast<cudaStream_t>(cuda_stream)) ==
                   cudaSuccess
               ? PBA_OK
               : PBA_ERR_CUDA;
}

pba_status pba_mlp_train_step(float* params, float* m, float* v, int step, float lr, int n,
                              const float* features, const float* targets, float* scratch, float* loss,
                              void* cuda_stream)
{
    if (!params || !m || !v || step < 1 || !(lr > 0.0f) || n < 1 || !features || !targets || !scratch)
        return PBA_ERR_ARG;
    return pba::launch_mlp_grad_adam(params, n, features, targets, scratch, nullptr, m, v, step, lr, loss,
                                     static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
               ? PBA_OK
               : PBA_ERR_CUDA;
}

}  // extern "C"
