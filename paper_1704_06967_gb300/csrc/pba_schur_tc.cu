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
constexpr int kTcRows = kTcM + kTcN;               // operand rows of a block (A then B)
constexpr int kTcSl = 6;                           // digits (slices) per operand
constexpr int kTcKc = kTile;                       // points per K chunk (one tile)
constexpr int kTcThreads = 512;
constexpr int kTcCols = 512;                       // tensor-memory columns allocated (6 x 80 used)
constexpr uint32_t kTcASlice = kTcM * kTcKc * 2;   // bytes of one BF16 slice of A (8 KB)
constexpr uint32_t kTcBSlice = kTcN * kTcKc * 2;   // of B (5 KB)
constexpr uint32_t kTcStage = kTcSl * (kTcASlice + kTcBSlice);
constexpr uint32_t kTcSbo = (kTcKc / 8) * 128;     // stride between 8-row core-matrix groups
constexpr int kTcNoRow = -1;
constexpr short kTcZeroExp = -32768;               // exponent of a row that is zero on the super-tile
constexpr int kTcExpLo = -80, kTcExpHi = 100;      // row exponents the FP32 splitting covers
constexpr uint32_t kTcIdesc = idesc_bf16(kTcM, kTcN);
// frames a block's rows can touch: 128 rows span at most 23 frames, 80 at most 15
constexpr int kTcMFrames = 23, kTcNFrames = 15, kTcSlots = kTcMFrames + kTcNFrames;

// row metadata of an output block (shared memory)
struct TcRow {
    int g;    // row of the bundle's S (6 (f - f0 - 1) + a), kTcNoRow when padding
    int eg;   // global scale exponent G of the row
    int e;    // super-tile exponent (E_A for rows, E_B for columns)
    int fl;   // frame position within the super-tile (upper-triangle test)
};

// shared-memory plan (bytes)
constexpr uint32_t kTcStg = kTcRows * kTcKc * 4;                        // FP32 staging of one chunk
constexpr uint32_t kTcOffStg = 2 * kTcStage;                           // two staging buffers
constexpr uint32_t kTcOffW = kTcOffStg + 2 * kTcStg;                   // 128 floats: w of the points
constexpr uint32_t kTcOffRows = kTcOffW + kStTiles * kTile * 4;        // TcRow[kTcRows]
constexpr uint32_t kTcOffTab = kTcOffRows + kTcRows * sizeof(TcRow);   // int2[kTcSlots][kStTiles]
constexpr uint32_t kTcOffBar = kTcOffTab + kTcSlots * kStTiles * 8;
constexpr uint32_t kTcSmem = kTcOffBar + 8 * 8;                        // six barriers, tmem slot, abort flag

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

__device__ __forceinline__ float tc_pow2(int e) { return __int_as_float((e + 127) << 23); }  // e in [-126, 127]

// Digits of an FP32 u with |u| < 2^E (E in [kTcExpLo, kTcExpHi]): slice s
// is u's residual rounded to a multiple of 2^(E - 7 - 8 s) by the addition
// of 1.5 * 2^(E + 16 - 8 s) (exact: the residual stays below that scale),
// the residual updated exactly, the digit q 2^(7 + 8 s - E) an integer with
// |q| <= 128.
__device__ __forceinline__ void tc_split_a(float u, int E, float (&d)[kTcSl])
{
#pragma unroll
    for (int s = 0; s < kTcSl; ++s) {
        const float sig = 1.5f * tc_pow2(E + 16 - 8 * s);
        const float q = (u + sig) - sig;
        u -= q;
        d[s] = q * tc_pow2(7 + 8 * s - E);
    }
}

// Digits of the exact product u w (48-bit integer mantissa) with
// |u w| < 2^E: X = round(u w 2^(47 - E)) as a 64-bit integer, cut into a
// high and a balanced low 24-bit half (both exact in FP32), each split into
// three digits by the same rounding additions (units 2^16, 2^8, 1).
__device__ __forceinline__ void tc_split_b(float u, float w, int E, float (&d)[kTcSl])
{
    const uint32_t bu = __float_as_uint(u), bw = __float_as_uint(w);
    const int eu = (int)((bu >> 23) & 255u), ew = (int)((bw >> 23) & 255u);
    long long X = 0;
    if (eu != 0 && ew != 0) {
        const unsigned long long m = (unsigned long long)((bu & 0x7FFFFFu) | 0x800000u) *
                                     (unsigned long long)((bw & 0x7FFFFFu) | 0x800000u);  // [2^46, 2^48)
        const int sh = 253 + E - eu - ew;  // X = m 2^-sh, sh >= 0 when |u w| < 2^E
        if (sh <= 0) X = (long long)(m << (-sh));
        else if (sh < 50) X = (long long)((m + (1ull << (sh - 1))) >> sh);
        if ((bu ^ bw) >> 31) X = -X;
    }
    const long long hi = (X + (1ll << 23)) >> 24;  // |hi| <= 2^23
    float fh = (float)(int)hi;
    float fl = (float)(int)(X - (hi << 24));       // in [-2^23, 2^23)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const float sig = 1.5f * tc_pow2(39 - 8 * s);  // unit 2^(16 - 8 s)
        float q = (fh + sig) - sig;
        fh -= q;
        d[s] = q * tc_pow2(8 * s - 16);
        q = (fl + sig) - sig;
        fl -= q;
        d[s + 3] = q * tc_pow2(8 * s - 16);
    }
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

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

// Converter warps: all but the last warp of the CTA. The last warp issues
// the MMAs (its lane 0) and owns the tensor memory.
constexpr int kTcConv = kTcThreads;  // converter threads (16 warps)
constexpr int kTcMmaWarp = kTcConv / 32;

__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTcConv) : "memory"); }

// converter barrier that also ANDs a flag over the converter threads
__device__ __forceinline__ bool conv_sync_and(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kTcConv)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__global__ void __launch_bounds__(kTcThreads + 32, 1)
schur_tc_kernel(DevProblem pb, const float* __restrict__ Hfd, const float* __restrict__ Hnn,
                const int4* __restrict__ st, const StRow* __restrict__ rows, const int4* __restrict__ items,
                int n_items, const short* __restrict__ ea, const short* __restrict__ eb,
                const double* __restrict__ red, int red_stride, unsigned long long* __restrict__ acc,
                int* __restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* wsm = reinterpret_cast<float*>(sm + kTcOffW);
    TcRow* meta = reinterpret_cast<TcRow*>(sm + kTcOffRows);  // A rows, then B rows
    int2* tab = reinterpret_cast<int2*>(sm + kTcOffTab);      // (first H_fd float, mask) per frame slot and tile
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTcOffBar);
    // full[b]: chunk in buffer b formed (one arrival per converter warp);
    // empty[b]: its MMAs done (commit); tfree: the epilogue has read the
    // accumulators (one arrival per converter warp); fin: every MMA done
    const uint32_t full0 = smem_u32(bar), empty0 = smem_u32(bar + 2), tfree = smem_u32(bar + 4),
                   fin = smem_u32(bar + 5);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 6);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 7);
    if (warp == kTcMmaWarp) tmem_alloc(tmem_slot, kTcCols);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full0 + 8 * b, kTcConv / 32);
            mbar_init(empty0 + 8 * b, 1);
        }
        mbar_init(tfree, kTcConv / 32);
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sbase = smem_u32(sm);

    if (warp == kTcMmaWarp) {
        // MMA issuer: per chunk q (counted over this CTA's items) wait until
        // buffer q & 1 holds it, before an item's first chunk until the
        // previous item's accumulators were read, then 42 MMAs and a commit
        if (lane == 0) {
            int q = 0, k = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++k) {
                const int nt = st[items[it].x].w;
                for (int c = 0; c < nt && ok; ++c, ++q) {
                    const int buf = q & 1;
                    ok = mbar_wait(full0 + 8 * buf, (uint32_t)((q >> 1) & 1), 1 << 22) && !*abort_flag;
                    if (ok && c == 0 && k > 0) ok = mbar_wait(tfree, (uint32_t)((k - 1) & 1), 1 << 22) && !*abort_flag;
                    if (!ok) break;
                    fence_after_sync();
                    const uint32_t a0 = sbase + buf * kTcStage, b0 = a0 + kTcSl * kTcASlice;
#pragma unroll
                    for (int ks = 0; ks < kTcKc / 16; ++ks)
#pragma unroll
                        for (int kk = 0; kk < kTcSl; ++kk)
#pragma unroll
                            for (int s = 0; s <= kk; ++s) {
                                const int t = kk - s;
                                mma_bf16_id(tmem + kk * kTcN,
                                            smem_desc(a0 + s * kTcASlice + ks * 256, 128, kTcSbo),
                                            smem_desc(b0 + t * kTcBSlice + ks * 256, 128, kTcSbo), kTcIdesc,
                                            (c > 0 || ks > 0 || s > 0) ? 1u : 0u);
                            }
                    mma_commit(empty0 + 8 * buf);
                }
            }
            if (!ok) {
                atomicOr(err, kErrTimeout);
                *abort_flag = 1;
            }
            // every MMA issued has finished before the tensor memory is freed
            mma_commit(fin);
            mbar_wait(fin, 0u, 1 << 22);
        }
        __syncwarp();
    } else {
        // converters: stage, form the digit slices, read the accumulators
        int q0 = 0;                  // this item's first chunk, counted over the CTA's items
        uint32_t consumed[2] = {0u, 0u};  // commits on empty[b] waited for
        bool ok = true;
        // chunk j's MMAs are done (its commit is number j >> 1 on empty[j & 1])
        auto ensure_done = [&](int j) -> bool {
            const int b = j & 1;
            while ((int)consumed[b] <= (j >> 1)) {
                const bool w = mbar_wait(empty0 + 8 * b, consumed[b] & 1u, 1 << 22) && !*abort_flag;
                if (!w) return false;
                ++consumed[b];
            }
            return true;
        };
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const int4 item = items[it];
            const int4 info = st[item.x];  // first row, frames, first tile, tiles
            const int nrows = 6 * info.y;
            const BundleDesc bd = pb.bund[pb.frame_bundle[rows[info.x].f]];
            const int n6 = 6 * (bd.F - 1);
            const int flm0 = (item.y * kTcM) / 6, fln0 = (item.z * kTcN) / 6;  // first frames of the blocks
            // weights of the points, row metadata, each frame slot's entries
            if (tid < kStTiles * kTile) {
                float w = 0.0f;
                if (tid < info.w * kTile) {
                    const float h = Hnn[(size_t)(info.z + tid / kTile) * kTile + (tid % kTile)];
                    w = h > 0.0f ? 1.0f / (h * pb.damp1) : 0.0f;
                }
                wsm[tid] = w;
            } else if (tid < kStTiles * kTile + kTcRows) {
                const int r = tid - kStTiles * kTile;
                const bool is_m = r < kTcM;
                const int rr = is_m ? item.y * kTcM + r : item.z * kTcN + (r - kTcM);
                TcRow m{kTcNoRow, 0, 0, 0};
                if (rr < nrows) {
                    const int fl = rr / 6, a = rr - 6 * fl;
                    const int f = rows[info.x + fl].f;
                    bool have;
                    const int qd = a * 6 - (a * (a - 1)) / 2;  // packed H_ff diagonal (a, a)
                    const int eg = tc_global_exp(red[(size_t)f * red_stride + qd], &have);
                    const short e = (is_m ? ea : eb)[(size_t)info.x * 6 + rr];
                    if (have && e != kTcZeroExp) {
                        if (e < kTcExpLo || e > kTcExpHi) atomicOr(err, kErrNonFinite);  // beyond the FP32 splitting
                        else m = TcRow{6 * (f - bd.fo - 1) + a, eg, (int)e, fl};
                    }
                }
                meta[r] = m;
            } else if (tid < kStTiles * kTile + kTcRows + kTcSlots * kStTiles) {
                const int j = tid - kStTiles * kTile - kTcRows, slot = j / kStTiles, c = j % kStTiles;
                const int fl = slot < kTcMFrames ? flm0 + slot : fln0 + slot - kTcMFrames;
                int2 t = make_int2(0, 0);
                if (fl < info.y && c < info.w) {
                    const int e = rows[info.x + fl].e[c];
                    if (e >= 0) {
                        const Entry en = pb.entries[e];
                        t = make_int2(en.pair_off * 6, (int)en.mask);
                    }
                }
                tab[j] = t;
            }
            conv_sync();

            // FP32 staging of chunk c (one tile): element (row, lane) of the
            // block's operand rows, zero where the lane does not see the frame
            auto stage = [&](int c) {
                float* stg = reinterpret_cast<float*>(sm + kTcOffStg + (c & 1) * kTcStg);
                const uint32_t sdst = smem_u32(stg);
                for (int i = tid; i < kTcRows * kTile; i += kTcConv) {
                    const int r = i >> 5, l = i & 31;
                    const TcRow mr = meta[r];
                    const float* src = Hfd;
                    bool valid = false;
                    if (mr.g != kTcNoRow) {
                        const int rr = r < kTcM ? item.y * kTcM + r : item.z * kTcN + (r - kTcM);
                        const int fl = rr / 6, a = rr - 6 * fl;
                        const int slot = r < kTcM ? fl - flm0 : kTcMFrames + fl - fln0;
                        const int2 t = tab[slot * kStTiles + c];
                        const unsigned mask = (unsigned)t.y;
                        if ((mask >> l) & 1u) {
                            src = Hfd + t.x + a * __popc(mask) + __popc(mask & ((1u << l) - 1u));
                            valid = true;
                        }
                    }
                    cp_async4(sdst + 4u * i, src, valid);
                }
                cp_async_commit();
            };
            // chunk c + 1 is staged while chunk c's digits are formed into
            // buffer (q0 + c) & 1, once that buffer's previous MMAs are done;
            // one converter barrier per chunk (after it, chunk c's staging is
            // visible and staging buffer (c + 1) & 1 is free)
            stage(0);
            for (int c = 0; c < info.w && ok; ++c) {
                const int q = q0 + c, buf = q & 1;
                cp_async_wait_all();
                bool w = true;
                if (q >= 2) w = ensure_done(q - 2);
                if (!conv_sync_and(w)) {
                    ok = false;
                    break;
                }
                if (c + 1 < info.w) stage(c + 1);
                const float* stg = reinterpret_cast<const float*>(sm + kTcOffStg + (c & 1) * kTcStg);
                uint8_t* sA = sm + buf * kTcStage;
                uint8_t* sB = sA + kTcSl * kTcASlice;
                for (int task = tid; task < kTcRows * 4; task += kTcConv) {
                    const int r = task >> 2, g = task & 3;  // operand row, group of 8 points
                    const bool is_a = r < kTcM;
                    const int e = meta[r].e;
                    const float4* sp = reinterpret_cast<const float4*>(stg + r * kTile + 8 * g);
                    const float4 u0 = sp[0], u1 = sp[1];
                    const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                    float d[8][kTcSl];
                    if (is_a) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) tc_split_a(u[j], e, d[j]);
                    } else {
                        const float4* wp = reinterpret_cast<const float4*>(wsm + c * kTile + 8 * g);
                        const float4 w0 = wp[0], w1 = wp[1];
                        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                        for (int j = 0; j < 8; ++j) tc_split_b(u[j], w[j], e, d[j]);
                    }
                    const int rl = is_a ? r : r - kTcM;
                    uint8_t* dst = (is_a ? sA : sB) + (rl >> 3) * kTcSbo + g * 128 + (rl & 7) * 16;
                    const uint32_t sl = is_a ? kTcASlice : kTcBSlice;
#pragma unroll
                    for (int s = 0; s < kTcSl; ++s)
                        *reinterpret_cast<uint4*>(dst + s * sl) =
                            make_uint4(pack_bf16x2(d[0][s], d[1][s]), pack_bf16x2(d[2][s], d[3][s]),
                                       pack_bf16x2(d[4][s], d[5][s]), pack_bf16x2(d[6][s], d[7][s]));
                }
                // the slices are visible to the tensor cores, then the MMA
                // warp is told (one arrival per warp)
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(full0 + 8 * buf);
            }
            if (ok) ok = conv_sync_and(ensure_done(q0 + info.w - 1));  // the item's MMAs are done
            if (!ok) {
                cp_async_wait_all();
                break;
            }
            q0 += info.w;
            fence_after_sync();

            // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the block's
            // rows) and the 8-column groups w / 4, w / 4 + 4, ...
            {
                const int r = 32 * (warp & 3) + lane;
                const TcRow mr = meta[r];
                const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
                for (int cg = warp >> 2; cg < kTcN / 8; cg += kTcConv / 128) {
                    const int col0 = 8 * cg;
                    float D[kTcSl][8];
#pragma unroll
                    for (int k = 0; k < kTcSl; ++k) tmem_ld8(trow + k * kTcN + col0, D[k]);
                    tmem_wait_ld();
                    if (mr.g == kTcNoRow) continue;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const TcRow nc = meta[kTcM + col0 + j];
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
            // the accumulators are read: the MMA warp may start the next item
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(tfree);
            conv_sync();
        }
        if (!ok && tid == 0) {
            atomicOr(err, kErrTimeout);
            *abort_flag = 1;
        }
    }
    __syncthreads();
    if (warp == kTcMmaWarp) tmem_dealloc(tmem, kTcCols);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_inval(full0 + 8 * b);
            mbar_inval(empty0 + 8 * b);
        }
        mbar_inval(tfree);
        mbar_inval(fin);
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
        schur_tc_kernel<<<grid, kTcThreads + 32, kTcSmem, st>>>(pb, Hfd, Hnn, tl.st, tl.rows, tl.items, tl.n_items,
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
