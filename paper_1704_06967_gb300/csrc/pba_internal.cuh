// Internal device layout and helpers of the GB300 photometric bundle
// adjustment library (IC with proxy templates, FC beside it).
//
// Data layout in HBM (all inside the caller's workspace):
//  * points are reordered (Morton order of their reference pixel) and grouped
//    in tiles of 32: lane l of tile t is sorted point 32 t + l. A CTA of the
//    pass kernels owns one tile, so a point's sums over frames complete on chip.
//  * an "entry" is a (tile, target frame) pair with at least one visible lane;
//    entries are stored tile-major. Entry e owns the pairs pair_off .. pair_off
//    + popc(mask) - 1 (visible lanes in lane order, "rank" = popc below lane).
//  * per pair: the IC Jacobian rows of its P pattern pixels (7 floats each,
//    pattern-major, packed into float4 chunks and stored chunk-major inside
//    the entry so a warp's loads are contiguous) and the 6-float frame-point
//    Hessian block H_fd (component-major inside the entry).
//  * per frame: FP64 master pose, FP32 constants for the pass (R, t and the
//    pattern offsets rotated into the frame).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pba.h"

namespace pba {

constexpr int kTile = 32;             // points per tile (= lanes of a warp)
constexpr int kPassWarps = 4;         // warps per CTA of the pass kernels
constexpr int kFrameConst = 64;       // floats of FP32 constants per frame
constexpr int kEntryPartial = 44;     // floats of partial sums per entry (FC: 21 H_ff, 6 g_f, 6 corrections)
constexpr int kPhotoColIc = 12;       // brightness fit sums of an entry (IC), 5 floats, 16-byte aligned
constexpr int kPhotoColFc = 36;       // the same for FC
constexpr int kFrameAlpha = 60;       // frame constants [60], [61]: affine brightness alpha, beta
constexpr int kAffCol = 24;           // IC precompute rows, joint brightness: 12 H_pa, 3 H_aa sums
constexpr int kAffComp = 15;
constexpr int kStats = 8;             // doubles per statistics slot

// device error word values (bit flags); the error words are err[0] for the
// whole context and err[1 + b] for bundle b
constexpr int kErrNotPD = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrTimeout = 4;

__device__ __forceinline__ void flag_error(int* err, int bundle, int bits)
{
    atomicOr(err, bits);
    atomicOr(err + 1 + bundle, bits);
}

struct Entry {
    int f;          // target frame (1..F-1)
    unsigned mask;  // visible lanes
    int pair_off;   // first pair of the entry
    int tile;
};

// One bundle of a context (a context solves one or several independent
// bundles; their frames, tiles and entries are concatenated, so the
// per-entry, per-tile and per-frame kernels run over all bundles in one
// launch). Its frames are the global frames fo .. fo + F - 1, fo being its
// reference frame; its reduced camera system (order n6 = 6 (F - 1)) sits at
// element offset so of the S, S_off and S^-1 arrays, its factorisation
// matrices ((n6 + 1) x n6) at ao, the inverses of its diagonal blocks at lo,
// its pivots at po and the compact frame map of its frames (F + 1 ints) at co.
struct BundleDesc {
    int fo, F, co, po;
    long long so, ao, lo;
};

// Per-tile statistics partials (FP32 sums of one tile).
struct TileStats {
    float energy, sumsq, count, maxdisp, ddsq, pad0, pad1, pad2;
};

// Everything the kernels need, passed by value.
struct DevProblem {
    int F, N, Npad, T, E, P, W, H, pitch, dtype;  // F, N, T, E: totals over the bundles
    float fx, fy, cx, cy, huber_k;
    float damp1;                // 1 + Levenberg-Marquardt lambda (scales every H_dd that is solved with)
    const void* img;            // F frames, H rows of `pitch` elements
    const float* gx;            // FC gradient images (F*H*W), nullable for IC
    const float* gy;
    const int* pat;             // P*2 offsets (device copy)
    const Entry* entries;       // E, tile-major
    const int* tile_entry;      // T+1 offsets into entries
    const int* frame_entry;     // F+1 offsets of each frame's partial-sum rows
    const int* entry_slot;      // E partial-sum row of each entry (frame-major order)
    const int* frame_bundle;    // F bundle of each global frame
    const BundleDesc* bund;     // bundles
    const int* tile_f0;         // T reference frame of each tile's bundle
    const int* uvs;             // Npad*2 sorted pixels (pad: copy of a real point)
    const float2* xn;           // Npad normalised centre coordinates
    const float* I0p;           // T*P*32 template intensities [tile][j][lane]
    unsigned char* valid_pt;    // Npad (1 = real point)
    // joint brightness unknowns (IC, cfg.photometric = 2; null otherwise):
    const unsigned* vmask0;     // per pair: bit j set when pattern pixel j was valid at p_0
    const float* Had;           // per pair, 2 values (compact like H_fd): J_d^T W_0 [I_0, 1]
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch. A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while the previous kernel
// on the stream is still finishing: it calls pdl_wait() before it reads
// anything an earlier kernel wrote (the wait returns once the previous grid
// has completed and its memory is visible, and at once for an ordinary
// launch). pdl_trigger() lets the next such kernel be scheduled early.
// Every kernel triggers at its start, so a kernel's code before its wait may
// run beside any earlier kernel of the chain back to the last ordinary
// launch or copy on the stream: there it reads only data that no kernel of
// the chain writes (the set-up's topology; in IC the J, H and S^-1 that the
// precompute, which ends with an ordinary launch, fixed).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// a 16-byte read-only load of data streamed once per pass (the stored J
// rows): not allocated in L1 and, with an evict-first L2 policy
// (l2_evict_first_policy()), the first to leave L2, so that it does not push
// the image lines the gathers reuse out of either cache
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ float4 ld_stream4(const float4* p, uint64_t pol)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

// ---------------------------------------------------------------------------
// image access (offsets are unsigned 32-bit: the host checks that the whole
// stack, F * H * pitch elements over all bundles, stays below 2^32)
// ---------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ float load_px_t(const void* img, unsigned idx)
{
    if (DT == PBA_F32) return __ldg(reinterpret_cast<const float*>(img) + idx);
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(img) + idx);
    if (DT == PBA_F16) return __half2float(__ushort_as_half(b));
    return __uint_as_float(((unsigned)b) << 16);
}

__device__ __forceinline__ float load_px(const void* img, int dtype, size_t idx)
{
    if (dtype == PBA_F32) return load_px_t<PBA_F32>(img, (unsigned)idx);
    if (dtype == PBA_F16) return load_px_t<PBA_F16>(img, (unsigned)idx);
    return load_px_t<PBA_BF16>(img, (unsigned)idx);
}

// Bilinear sample at pixel coordinates (pixel centres on integers); valid
// iff the 2x2 footprint lies in [1, W-2] x [1, H-2] (gradients defined).
template <int DT>
__device__ __forceinline__ bool bilinear_t(const DevProblem& pb, int f, float u, float v,
                                           float& val, float& a, float& b, int& x, int& y)
{
    const float fu = floorf(u), fv = floorf(v);
    // float range test first (also rejects NaN and values beyond int range)
    if (!(fu >= 1.0f && fu <= (float)(pb.W - 3) && fv >= 1.0f && fv <= (float)(pb.H - 3)))
        return false;
    x = (int)fu;
    y = (int)fv;
    a = u - fu;
    b = v - fv;
    const unsigned base = ((unsigned)f * (unsigned)pb.H + (unsigned)y) * (unsigned)pb.pitch + (unsigned)x;
    const float i00 = load_px_t<DT>(pb.img, base);
    const float i10 = load_px_t<DT>(pb.img, base + 1);
    const float i01 = load_px_t<DT>(pb.img, base + pb.pitch);
    const float i11 = load_px_t<DT>(pb.img, base + pb.pitch + 1);
    const float top = fmaf(a, i10 - i00, i00);
    const float bot = fmaf(a, i11 - i01, i01);
    val = fmaf(b, bot - top, top);
    return true;
}

// ---------------------------------------------------------------------------
// warp reductions (butterfly: every lane ends with the same total)
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void warp_sum(float (&v)[K])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// 1 / x by the hardware approximation (rcp.approx.ftz: within 1 ulp)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One reduce-scatter level over the lanes at stride o: a lane keeps values
// [0, M) (lane bit o clear) or [M, 2M) (set) of v, moved to v[0 .. M), and
// adds its partner's copy of them.
template <int M, int N>
__device__ __forceinline__ void scatter_level(float (&v)[N], int lane, int o)
{
    static_assert(2 * M <= N, "scatter level");
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const float send = up ? v[q] : v[q + M];
        const float keep = up ? v[q + M] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}

__device__ __forceinline__ float warp_sum1(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum1d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max1(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Neumaier compensated accumulation (Neumaier 1974)
__device__ __forceinline__ void neumaier_add(float& s, float& c, float x)
{
    float t = s + x;
    if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

__device__ __forceinline__ float huber_w(float r, float k)
{
    float a = fabsf(r);
    return a <= k ? 1.0f : k / a;
}

__device__ __forceinline__ float huber_rho(float r, float k)
{
    float a = fabsf(r);
    return a <= k ? 0.5f * r * r : k * a - 0.5f * k * k;
}

}  // namespace pba
