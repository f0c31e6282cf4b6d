// Schur complement of the point block (Sec. 3.5 step 3):
//   S_off[f][g] = sum_n H_fd(n,f) H_fd(n,g)^T / H_dd(n),
// summed over the points that frames f and g both observe.
//
// A precomputed list holds, per frame pair f <= g, the tiles that see both
// frames (items in tile order: the fixed summation order), cut into chunks
// of at most kChunk items so that large pairs do not serialise on one SM.
// One CTA per chunk (a lane adds its point) writes its sums; a second kernel
// adds a pair's chunks in order. The visibility structure is sparse (on the helix bundle
// about a fifth of the (point, frame) pairs exist), so this touches only the
// products that are not zero, where a dense B B^T would do ~20x the work.
//
// S = blockdiag(H_ff) - S_off cancels along the near-null directions of the
// reduced system, so the sum must not lose accuracy. GB300 issues FP64
// slowly, so the products and sums stay on the FP32 pipes but are carried
// exactly: each product a*b is split error-free into p + e with
// e = fma(a, b, -p) (TwoProduct, Ogita, Rump and Oishi 2005), and p is added
// into an unevaluated pair (s, c) with Knuth's error-free two-sum; the pairs
// are reduced across lanes and warps the same way and converted to FP64 once.
// The only rounding left is that of 1/H_dd(n), a factor common to a point.
// Deterministic; diagonal blocks come out exactly symmetric (the (a,b) and
// (b,a) products are identical).
#include "pba_kernels.cuh"

namespace pba {

// (s, c) += a b w: a b = p + e exactly (TwoProduct), p w = q + g exactly,
// q added by two-sum, the small terms g + e w into c. The only rounding
// left is that of w = 1/H_dd, a per-point factor common to all 36 entries.
__device__ __forceinline__ void acc_product(float& s, float& c, float a, float b, float w)
{
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float q = p * w;
    const float g = fmaf(p, w, -q);
    const float t = s + q;
    const float bb = t - s;
    const float err = (s - (t - bb)) + (q - bb);
    s = t;
    c += err + fmaf(e, w, g);
}

__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2)
{
    const float t = s + s2;
    const float bb = t - s;
    const float e = (s - (t - bb)) + (s2 - bb);
    s = t;
    c = c + c2 + e;
}

constexpr int kSchurWarps = 4;

// Lane-sums of the 36 unevaluated pairs of a warp, in a fixed order. The
// first 32 go through a reduce-scatter (at each of the five levels a lane
// keeps half of its values and adds its partner's copy of them: 31 pair
// exchanges instead of 32 x 5); the last 4 through butterflies. Lane l ends
// with value l of the first 32 (returned in *v0, its index in *k0) and, on
// every lane, values 32..35 in s[32..35], c[32..35].
__device__ __forceinline__ void warp_reduce_36(float (&s)[36], float (&c)[36], int lane, float2* v0,
                                               int* k0)
{
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int o = 16 >> lvl, half = 16 >> lvl;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            // keep k (lower) or k + half (upper); send the other
            const float ss = up ? s[k] : s[k + half], sc = up ? c[k] : c[k + half];
            const float ks = up ? s[k + half] : s[k], kc = up ? c[k + half] : c[k];
            const float rs = __shfl_xor_sync(0xffffffffu, ss, o);
            const float rc = __shfl_xor_sync(0xffffffffu, sc, o);
            float a = ks, b = kc;
            // the lower lane adds (its value, partner's) and the upper lane
            // (partner's, its value) in the same order
            if (up) {
                a = rs;
                b = rc;
                pair_add(a, b, ks, kc);
            } else {
                pair_add(a, b, rs, rc);
            }
            s[k] = a;
            c[k] = b;
        }
    }
    // level with stride o kept the upper half iff lane bit o is set, so
    // after the five levels lane l holds value index l
    *v0 = make_float2(s[0], c[0]);
    *k0 = lane;
#pragma unroll
    for (int k = 32; k < 36; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float a2 = __shfl_xor_sync(0xffffffffu, s[k], o);
            const float b2 = __shfl_xor_sync(0xffffffffu, c[k], o);
            if (lane & o) {
                float a = a2, b = b2;
                pair_add(a, b, s[k], c[k]);
                s[k] = a;
                c[k] = b;
            } else {
                pair_add(s[k], c[k], a2, b2);
            }
        }
    }
}

// chunk c covers items [chunk_start[c], chunk_start[c+1]) of one frame pair;
// it writes 36 unevaluated pairs (s, c) to part[c]. With tile_todo, a chunk
// none of whose items lies in a flagged tile keeps part[c] as it is.
__global__ void __launch_bounds__(32 * kSchurWarps)
schur_chunk_kernel(DevProblem pb, const float* Hfd, const float* Hnn, const int* chunk_start,
                   const int2* items, float2* part, const unsigned char* tile_todo)
{
    __shared__ float2 red[kSchurWarps][36];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ch = blockIdx.x;
    const int i0 = chunk_start[ch], i1 = chunk_start[ch + 1];
    if (tile_todo) {
        bool todo = false;
        for (int it = i0 + (int)threadIdx.x; it < i1; it += blockDim.x)
            todo |= tile_todo[pb.entries[items[it].x].tile] != 0;
        if (!__syncthreads_or(todo)) return;
    }
    float s[36], c[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) s[k] = c[k] = 0.0f;
    for (int it = i0 + warp; it < i1; it += kSchurWarps) {
        const int2 ee = items[it];
        const Entry A = pb.entries[ee.x], B = pb.entries[ee.y];
        if (!((A.mask & B.mask) >> lane & 1u)) continue;
        const int n = A.tile * kTile + lane;
        const float h = Hnn[n];
        if (!(h > 0.0f)) continue;
        const float ih = 1.0f / (h * pb.damp1);
        const int na = __popc(A.mask), ra = __popc(A.mask & ((1u << lane) - 1u));
        const int nb = __popc(B.mask), rb = __popc(B.mask & ((1u << lane) - 1u));
        const float* pa = Hfd + (size_t)A.pair_off * 6 + ra;
        const float* pq = Hfd + (size_t)B.pair_off * 6 + rb;
        float ha[6], hb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            ha[k] = pa[k * na];
            hb[k] = pq[k * nb];
        }
        // a b = b a exactly, so diagonal blocks (ha == hb) come out symmetric
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) acc_product(s[6 * a + b], c[6 * a + b], ha[a], hb[b], ih);
    }
    float2 v0;
    int k0;
    warp_reduce_36(s, c, lane, &v0, &k0);
    red[warp][k0] = v0;
    if (lane < 4) {
        float a = s[32], b = c[32];
#pragma unroll
        for (int k = 33; k < 36; ++k)
            if (lane == k - 32) {
                a = s[k];
                b = c[k];
            }
        red[warp][32 + lane] = make_float2(a, b);
    }
    __syncthreads();
    if (threadIdx.x < 36) {
        const int k = threadIdx.x;
        float vs = red[0][k].x, vc = red[0][k].y;
        for (int w = 1; w < kSchurWarps; ++w) pair_add(vs, vc, red[w][k].x, red[w][k].y);
        part[(size_t)ch * 36 + k] = make_float2(vs, vc);
    }
}

// S_off blocks from the chunk sums, chunks of a pair added in order; a
// pair's frames belong to one bundle, whose block of S_off it fills.
__global__ void schur_pair_reduce_kernel(const int* pair_fg, const int* pair_chunk, const int* frame_bundle,
                                         const BundleDesc* bund, const float2* part, int n_pairs,
                                         double* Soff)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_pairs * 36) return;
    const int p = idx / 36, k = idx % 36, a = k / 6, b = k % 6;
    const int f = pair_fg[2 * p], g = pair_fg[2 * p + 1];
    if (f == g && a > b) return;
    float vs = 0.0f, vc = 0.0f;
    for (int ch = pair_chunk[p]; ch < pair_chunk[p + 1]; ++ch) {
        const float2 v = part[(size_t)ch * 36 + k];
        pair_add(vs, vc, v.x, v.y);
    }
    const double v = (double)vs + (double)vc;
    const BundleDesc bd = bund[frame_bundle[f]];
    const size_t n6 = 6 * (bd.F - 1);
    const int i = 6 * (f - bd.fo - 1) + a, j = 6 * (g - bd.fo - 1) + b;
    Soff[bd.so + i * n6 + j] = v;
    Soff[bd.so + j * n6 + i] = v;
}

cudaError_t launch_schur_sparse(const DevProblem& pb, const float* Hfd, const float* Hnn,
                                const SchurLists& sl, float2* part, double* Soff,
                                cudaStream_t st, int* launches, const unsigned char* tile_todo)
{
    if (sl.n_pairs == 0) return cudaSuccess;
    if (sl.n_chunks > 0) {
        schur_chunk_kernel<<<sl.n_chunks, 32 * kSchurWarps, 0, st>>>(
            pb, Hfd, Hnn, sl.chunk_start, sl.items, part, tile_todo);
        ++*launches;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    schur_pair_reduce_kernel<<<(sl.n_pairs * 36 + 255) / 256, 256, 0, st>>>(
        sl.pair_fg, sl.pair_chunk, pb.frame_bundle, pb.bund, part, sl.n_pairs, Soff);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace pba
