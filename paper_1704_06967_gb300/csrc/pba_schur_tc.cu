// Schur complement of the point block (Sec. 3.5 step 3) on the tensor cores:
//   S_off[f][g] = sum_n H_fd(n,f) H_fd(n,g)^T / H_dd(n)   (f <= g),
// the one dense contraction of the method, formed as a sum of products
// A B^T over super-tiles of 128 points (four consecutive Morton tiles of one
// bundle): the rows of A are the H_fd components (6 per frame that any of
// the super-tile's points sees), those of B the same components times
// w_n = 1 / (H_dd(n) (1 + lambda)), the columns the points.
//
// Error-free splitting. S cancels along the near-null directions of the
// reduced system, so the products are not rounded: every row of A and of B
// is written in fixed point with its own power-of-two scale 2^E (|value| <
// 2^E over the super-tile's points) as 48-bit integers X (the FP32 values
// of A exactly, the 48-bit products u w of B exactly, down to 2^(E-47)),
// and X as six balanced base-256 digits, |q| <= 128. A digit is exact in
// BF16; a product of two digits is an integer of at most 2^14, and the
// accumulator of the pairs (s, t) with s + t = k (at most six pairs over
// 128 points) stays below 6 * 2^14 * 128 < 2^24, so the tcgen05.mma FP32
// accumulation is exact in any order. The 21 pairs with s + t <= 5 are
// kept (the dropped ones lie below 2^-56 of the row scales, 128 points
// each). Each output element is then the exact integer
// V = sum_k D_k 256^(5-k) (|V| < 2^62) times 2^(E_A + E_B - 54).
//
// Deterministic accumulation. Every contribution is rounded once to a
// fixed point whose unit is 2^(G_i + G_j - 62), G_i from the frame's H_ff
// diagonal (2^G_i >= 2 sqrt(H_ff,ii) >= 2 sqrt(S_off,ii), which bounds
// every partial sum by 2^60 units), and added with 64-bit integer atomics:
// integer sums do not depend on order, so the result is the same run to
// run. The rounding left is 2^-62 of the bound per super-tile.
//
// One persistent CTA per SM takes output blocks (super-tile, 128 rows, 80
// columns) of the upper block triangle in turn: the 256 threads write the
// digit slices of a 32-point chunk into shared memory (two buffers) while
// one thread issues the previous chunk's 42 MMAs (M = 128, N = 80, K = 16,
// six accumulators of 80 columns in tensor memory); the epilogue reads the
// accumulators with tcgen05.ld, forms V and adds it at the block's place.
#include "pba_kernels.cuh"
#include "pba_tc.cuh"

namespace pba {

namespace {

constexpr int kTcM = kSchurTcM;                    // output rows per block (TMEM lanes)
constexpr int kTcN = kSchurTcN;                    // output columns per block
constexpr int kTcSl = 6;                           // digits (slices) per operand
constexpr int kTcKc = kTile;                       // points per K chunk (one tile)
constexpr int kTcThreads = 256;
constexpr int kTcCols = 512;                       // tensor-memory columns allocated (6 x 80 used)
constexpr uint32_t kTcASlice = kTcM * kTcKc * 2;   // bytes of one BF16 slice of A (8 KB)
constexpr uint32_t kTcBSlice = kTcN * kTcKc * 2;   // of B (5 KB)
constexpr uint32_t kTcStage = kTcSl * (kTcASlice + kTcBSlice);
constexpr uint32_t kTcSbo = (kTcKc / 8) * 128;     // stride between 8-row core-matrix groups
constexpr int kTcNoRow = -1;
constexpr short kTcZeroExp = -32768;               // exponent of a row that is zero on the super-tile
constexpr uint32_t kTcIdesc = idesc_bf16(kTcM, kTcN);

// row metadata of an output block (shared memory)
struct TcRow {
    int g;    // row of the bundle's S (6 (f - f0 - 1) + a), kTcNoRow when padding
    int eg;   // global scale exponent G of the row
    int e;    // super-tile exponent (E_A for rows, E_B for columns)
    int fl;   // frame position within the super-tile (upper-triangle test)
};

constexpr uint32_t kTcOffW = 2 * kTcStage;                          // 128 floats: w of the points
constexpr uint32_t kTcOffRows = kTcOffW + kStTiles * kTile * 4;     // TcRow[kTcM + kTcN]
constexpr uint32_t kTcOffBar = kTcOffRows + (kTcM + kTcN) * sizeof(TcRow);
constexpr uint32_t kTcSmem = kTcOffBar + 3 * 8 + 8;                 // two barriers, tmem slot, pad

// the exponent E with m < 2^E of a non-negative FP32 m (zero and
// subnormals: the zero-row mark)
__device__ __forceinline__ short tc_bound_exp(float m)
{
    const uint32_t b = __float_as_uint(m);
    const int e = (int)((b >> 23) & 255u);
    return e == 0 ? kTcZeroExp : (short)(e - 126);  // m in [2^(e-127), 2^(e-126))
}

// G with 2^G >= 2 sqrt(h): h < 2^eh gives sqrt(h) < 2^ceil(eh / 2)
__device__ __forceinline__ int tc_global_exp(double h, bool* ok)
{
    if (!(h > 0.0)) {
        *ok = false;
        return 0;
    }
    int eh;
    frexp(h, &eh);
    *ok = true;
    return ((eh + 1) >> 1) + 1;
}

// X = round(u 2^(47 - E)) for an FP32 u with |u| < 2^E (subnormals as zero)
__device__ __forceinline__ long long tc_fix_a(float u, int E)
{
    const uint32_t b = __float_as_uint(u);
    const int e = (int)((b >> 23) & 255u);
    if (e == 0) return 0;
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);  // u = m 2^(e - 150)
    const int sh = 103 + E - e;                                      // X = m 2^-sh, sh >= -23
    long long X;
    if (sh <= 0) X = m << (-sh);
    else if (sh >= 40) X = 0;  // m < 2^24: rounds to 0 from sh = 26
    else X = (m + (1ll << (sh - 1))) >> sh;
    return (b >> 31) ? -X : X;
}

// X = round(u w 2^(47 - E)) of the exact product (48-bit integer mantissa)
__device__ __forceinline__ long long tc_fix_b(float u, float w, int E)
{
    const uint32_t bu = __float_as_uint(u), bw = __float_as_uint(w);
    const int eu = (int)((bu >> 23) & 255u), ew = (int)((bw >> 23) & 255u);
    if (eu == 0 || ew == 0) return 0;
    const unsigned long long m = (unsigned long long)((bu & 0x7FFFFFu) | 0x800000u) *
                                 (unsigned long long)((bw & 0x7FFFFFu) | 0x800000u);  // [2^46, 2^48)
    const int sh = 253 + E - eu - ew;  // X = m 2^-sh, sh >= 0 when |u w| < 2^E
    long long X;
    if (sh >= 50) X = 0;
    else if (sh <= 0) X = (long long)(m << (-sh));  // sh < 0 is not reached for a valid E
    else X = (long long)((m + (1ull << (sh - 1))) >> sh);
    return ((bu ^ bw) >> 31) ? -X : X;
}

// balanced base-256 digits of |X| <= 2^47, most significant first
__device__ __forceinline__ void tc_digits(long long X, int (&q)[kTcSl])
{
#pragma unroll
    for (int i = kTcSl - 1; i > 0; --i) {
        const int d = (int)((X + 128) & 255) - 128;
        q[i] = d;
        X = (X - d) >> 8;
    }
    q[0] = (int)X;
}

}  // namespace

// Per super-tile and row: the exponents E_A (of |H_fd|) and E_B (of
// |H_fd w|) over the super-tile's points. A warp per frame of the
// super-tile, lane = point of a tile, its tiles in turn.
__global__ void __launch_bounds__(256)
schur_tc_scale_kernel(DevProblem pb, const float* __restrict__ Hfd, const float* __restrict__ Hnn,
                      const int4* __restrict__ st, const StRow* __restrict__ rows, short* __restrict__ ea,
                      short* __restrict__ eb)
{
    const int s = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 info = st[s];  // first row, frames, first tile, tiles
    for (int fl = warp; fl < info.y; fl += 8) {
        const StRow r = rows[info.x + fl];
        float ma[6] = {0, 0, 0, 0, 0, 0}, mb[6] = {0, 0, 0, 0, 0, 0};
        for (int c = 0; c < info.w; ++c) {
            const int e = r.e[c];
            if (e < 0) continue;
            const Entry en = pb.entries[e];
            if (!((en.mask >> lane) & 1u)) continue;
            const int nvis = __popc(en.mask), rank = __popc(en.mask & ((1u << lane) - 1u));
            const float h = Hnn[(size_t)en.tile * kTile + lane];
            const float w = h > 0.0f ? 1.0f / (h * pb.damp1) : 0.0f;
            const float* hp = Hfd + (size_t)en.pair_off * 6 + rank;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const float u = fabsf(hp[a * nvis]);
                ma[a] = fmaxf(ma[a], u);
                mb[a] = fmaxf(mb[a], u * w);
            }
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            ma[a] = warp_max1(ma[a]);
            mb[a] = warp_max1(mb[a]);
        }
        if (lane < 6) {
            float va = ma[0], vb = mb[0];
#pragma unroll
            for (int a = 1; a < 6; ++a)
                if (lane == a) {
                    va = ma[a];
                    vb = mb[a];
                }
            ea[(size_t)(info.x + fl) * 6 + lane] = tc_bound_exp(va);
            eb[(size_t)(info.x + fl) * 6 + lane] = tc_bound_exp(vb);
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
schur_tc_kernel(DevProblem pb, const float* __restrict__ Hfd, const float* __restrict__ Hnn,
                const int4* __restrict__ st, const StRow* __restrict__ rows, const int4* __restrict__ items,
                int n_items, const short* __restrict__ ea, const short* __restrict__ eb,
                const double* __restrict__ red, int red_stride, unsigned long long* __restrict__ acc,
                int* __restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* wsm = reinterpret_cast<float*>(sm + kTcOffW);
    TcRow* mrow = reinterpret_cast<TcRow*>(sm + kTcOffRows);
    TcRow* nrow = mrow + kTcM;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTcOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    const uint32_t mbar[2] = {smem_u32(bar), smem_u32(bar + 1)};
    if (warp == 0) tmem_alloc(tmem_slot, kTcCols);
    if (tid == 0) {
        mbar_init(mbar[0], 1);
        mbar_init(mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sbase = smem_u32(sm);
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;

    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        const int4 item = items[it];
        const int4 info = st[item.x];  // first row, frames, first tile, tiles
        const int nrows = 6 * info.y;
        const BundleDesc bd = pb.bund[pb.frame_bundle[rows[info.x].f]];
        const int n6 = 6 * (bd.F - 1);
        // weights of the super-tile's points and the block's row metadata
        if (tid < kStTiles * kTile) {
            float w = 0.0f;
            if (tid < info.w * kTile) {
                const float h = Hnn[(size_t)(info.z + tid / kTile) * kTile + (tid % kTile)];
                w = h > 0.0f ? 1.0f / (h * pb.damp1) : 0.0f;
            }
            wsm[tid] = w;
        }
        if (tid < kTcM + kTcN) {
            const bool is_m = tid < kTcM;
            const int rr = is_m ? item.y * kTcM + tid : item.z * kTcN + (tid - kTcM);
            TcRow m{kTcNoRow, 0, 0, 0};
            if (rr < nrows) {
                const int fl = rr / 6, a = rr - 6 * fl;
                const int f = rows[info.x + fl].f;
                bool have;
                const int q = a * 6 - (a * (a - 1)) / 2;  // packed H_ff diagonal (a, a)
                const int eg = tc_global_exp(red[(size_t)f * red_stride + q], &have);
                const short e = (is_m ? ea : eb)[(size_t)info.x * 6 + rr];
                if (have && e != kTcZeroExp) m = TcRow{6 * (f - bd.fo - 1) + a, eg, (int)e, fl};
            }
            (is_m ? mrow[tid] : nrow[tid - kTcM]) = m;
        }
        __syncthreads();

        // K chunks (the super-tile's tiles): slices into buffer c & 1, then
        // one thread issues the chunk's MMAs
        for (int c = 0; c < info.w; ++c) {
            const int buf = c & 1;
            if (c >= 2) {
                ok = __syncthreads_and(mbar_wait(mbar[buf], phase[buf]));
                phase[buf] ^= 1u;
                if (!ok) break;
            }
            uint8_t* sA = sm + buf * kTcStage;
            uint8_t* sB = sA + kTcSl * kTcASlice;
            for (int task = tid; task < (kTcM + kTcN) * 4; task += kTcThreads) {
                const bool is_a = task < kTcM * 4;
                const int tt = is_a ? task : task - kTcM * 4;
                const int r = tt >> 2, g = tt & 3;  // operand row, group of 8 points
                const int rr = is_a ? item.y * kTcM + r : item.z * kTcN + r;
                int q[8][kTcSl];
#pragma unroll
                for (int j = 0; j < 8; ++j)
#pragma unroll
                    for (int s = 0; s < kTcSl; ++s) q[j][s] = 0;
                const TcRow meta = is_a ? mrow[r] : nrow[r];
                if (meta.g != kTcNoRow) {
                    const int fl = rr / 6, a = rr - 6 * fl;
                    const int e = rows[info.x + fl].e[c];
                    if (e >= 0) {
                        const Entry en = pb.entries[e];
                        const int nvis = __popc(en.mask);
                        const float* hp = Hfd + (size_t)en.pair_off * 6 + (size_t)a * nvis;
                        const unsigned below = en.mask & ((1u << (8 * g)) - 1u);
                        int rank = __popc(below);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int l = 8 * g + j;
                            if ((en.mask >> l) & 1u) {
                                const float u = __ldg(hp + rank);
                                ++rank;
                                const long long X = is_a ? tc_fix_a(u, meta.e)
                                                         : tc_fix_b(u, wsm[c * kTile + l], meta.e);
                                tc_digits(X, q[j]);
                            }
                        }
                    }
                }
                uint8_t* dst = (is_a ? sA : sB) + (r >> 3) * kTcSbo + g * 128 + (r & 7) * 16;
                const uint32_t sl = is_a ? kTcASlice : kTcBSlice;
#pragma unroll
                for (int s = 0; s < kTcSl; ++s)
                    *reinterpret_cast<uint4*>(dst + s * sl) =
                        make_uint4(pack_bf16x2((float)q[0][s], (float)q[1][s]), pack_bf16x2((float)q[2][s], (float)q[3][s]),
                                   pack_bf16x2((float)q[4][s], (float)q[5][s]), pack_bf16x2((float)q[6][s], (float)q[7][s]));
            }
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            if (tid == 0) {
                const uint32_t a0 = sbase + buf * kTcStage, b0 = a0 + kTcSl * kTcASlice;
#pragma unroll
                for (int ks = 0; ks < kTcKc / 16; ++ks)
#pragma unroll
                    for (int k = 0; k < kTcSl; ++k)
#pragma unroll
                        for (int s = 0; s <= k; ++s) {
                            const int t = k - s;
                            mma_bf16_id(tmem + k * kTcN, smem_desc(a0 + s * kTcASlice + ks * 256, 128, kTcSbo),
                                        smem_desc(b0 + t * kTcBSlice + ks * 256, 128, kTcSbo), kTcIdesc,
                                        (c > 0 || ks > 0 || s > 0) ? 1u : 0u);
                        }
                mma_commit(mbar[buf]);
            }
        }
        // every outstanding commit (the last chunk's, and the one before it)
        for (int c = (info.w >= 2 ? info.w - 2 : 0); c < info.w && ok; ++c) {
            const int buf = c & 1;
            ok = __syncthreads_and(mbar_wait(mbar[buf], phase[buf]));
            phase[buf] ^= 1u;
        }
        if (!ok) break;
        fence_after_sync();

        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the block's
        // rows) and the 16-column groups w / 4, w / 4 + 2, ...
        {
            const int r = 32 * (warp & 3) + lane;
            const TcRow mr = mrow[r];
            const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
            for (int cg = warp >> 2; cg < kTcN / 16; cg += 2) {
                const int col0 = 16 * cg;
                float D[kTcSl][16];
#pragma unroll
                for (int k = 0; k < kTcSl; ++k) tmem_ld16(trow + k * kTcN + col0, D[k]);
                tmem_wait_ld();
                if (mr.g == kTcNoRow) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const TcRow nc = nrow[col0 + j];
                    if (nc.g == kTcNoRow) continue;
                    // upper block triangle; in a diagonal block a <= b
                    if (mr.fl > nc.fl || (mr.fl == nc.fl && mr.g > nc.g)) continue;
                    long long V = (long long)__float2int_rn(D[0][j]);
#pragma unroll
                    for (int k = 1; k < kTcSl; ++k) V = V * 256 + (long long)__float2int_rn(D[k][j]);
                    if (V == 0) continue;
                    const int dl = mr.e + nc.e - mr.eg - nc.eg + 8;  // V 2^dl in units 2^(G_i + G_j - 62)
                    long long I;
                    if (dl >= 0) {
                        const long long lim = dl >= 62 ? 0 : (1ll << (62 - dl));
                        if (!(V < lim && V > -lim)) {
                            atomicOr(err, kErrNonFinite);  // the scale bound does not hold
                            continue;
                        }
                        I = V << dl;
                    } else {
                        const int n = -dl;
                        I = n >= 62 ? 0 : ((V + (1ll << (n - 1))) >> n);
                    }
                    if (I != 0)
                        atomicAdd(acc + bd.so + (size_t)mr.g * n6 + nc.g, (unsigned long long)I);
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok) {
        // a wait gave up: report it and let the MMAs in flight finish (a
        // second, longer bound) before the tensor memory is freed
        if (tid == 0) atomicOr(err, kErrTimeout);
        mbar_wait(mbar[0], phase[0], 1 << 20);
        mbar_wait(mbar[1], phase[1], 1 << 20);
        fence_after_sync();
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTcCols);
    if (tid == 0) {
        mbar_inval(mbar[0]);
        mbar_inval(mbar[1]);
    }
}

// S_off of every frame pair f <= g from the fixed-point sums (both
// triangles), which are reset to zero for the next formation.
__global__ void schur_tc_finish_kernel(const int* __restrict__ pair_fg, int n_pairs,
                                       const int* __restrict__ frame_bundle, const BundleDesc* __restrict__ bund,
                                       const double* __restrict__ red, int red_stride,
                                       unsigned long long* __restrict__ acc, double* __restrict__ Soff)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_pairs * 36) return;
    const int p = idx / 36, k = idx % 36, a = k / 6, b = k % 6;
    const int f = pair_fg[2 * p], g = pair_fg[2 * p + 1];
    if (f == g && a > b) return;
    const BundleDesc bd = bund[frame_bundle[f]];
    const size_t n6 = 6 * (bd.F - 1);
    const int i = 6 * (f - bd.fo - 1) + a, j = 6 * (g - bd.fo - 1) + b;
    const size_t at = bd.so + i * n6 + j;
    const long long I = (long long)acc[at];
    acc[at] = 0ull;
    double v = 0.0;
    if (I != 0) {
        bool hi, hj;
        const int gi = tc_global_exp(red[(size_t)f * red_stride + a * 6 - (a * (a - 1)) / 2], &hi);
        const int gj = tc_global_exp(red[(size_t)g * red_stride + b * 6 - (b * (b - 1)) / 2], &hj);
        v = ldexp((double)I, gi + gj - 62);
    }
    Soff[bd.so + i * n6 + j] = v;
    Soff[bd.so + j * n6 + i] = v;
}

namespace {
int g_sm_count[64] = {0};
}

cudaError_t schur_tc_setup()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    e = cudaFuncSetAttribute(schur_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    return cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
}

cudaError_t launch_schur_tc(const DevProblem& pb, const float* Hfd, const float* Hnn, const SchurTcLists& tl,
                            const SchurLists& sl, const double* red, int red_stride, double* Soff, int* err,
                            cudaStream_t st, int* launches)
{
    if (sl.n_pairs == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int nsm = (dev >= 0 && dev < 64 && g_sm_count[dev] > 0) ? g_sm_count[dev] : 1;
    if (tl.n_items > 0) {
        schur_tc_scale_kernel<<<tl.n_st, 256, 0, st>>>(pb, Hfd, Hnn, tl.st, tl.rows, tl.ea, tl.eb);
        ++*launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int grid = tl.n_items < nsm ? tl.n_items : nsm;
        schur_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(pb, Hfd, Hnn, tl.st, tl.rows, tl.items, tl.n_items,
                                                          tl.ea, tl.eb, red, red_stride,
                                                          reinterpret_cast<unsigned long long*>(tl.acc), err);
        ++*launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    schur_tc_finish_kernel<<<(sl.n_pairs * 36 + 255) / 256, 256, 0, st>>>(
        sl.pair_fg, sl.n_pairs, pb.frame_bundle, pb.bund, red, red_stride,
        reinterpret_cast<unsigned long long*>(tl.acc), Soff);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace pba
