// Double-float arithmetic: a value is an unevaluated pair (hi, lo) of FP32
// numbers with |lo| <= ulp(hi)/2, carrying about 48 significant bits.
// GB300 issues FP64 at 1/64 of its FP32 rate with a ~14x longer dependent
// latency, so the dense reduced-camera-system kernels run on the FP32 pipes
// in this format. The building blocks are the error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum) and the FMA form of Dekker's product
// (Ogita, Rump and Oishi 2005); the composite operations follow the usual
// double-word algorithms (Dekker 1971; Joldes, Muller and Popescu 2017).
#pragma once

#include <cuda_runtime.h>

namespace pba {

using dfloat = float2;  // x = hi, y = lo

__device__ __forceinline__ dfloat df_make(float hi, float lo) { return make_float2(hi, lo); }

// exact s + e = a + b (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// exact s + e = a + b given |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ dfloat df_norm(float s, float e)
{
    float h, l;
    fast_two_sum(s, e, h, l);
    return df_make(h, l);
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b)
{
    float s, e, t, f;
    two_sum(a.x, b.x, s, e);
    two_sum(a.y, b.y, t, f);
    e += t;
    float s2, e2;
    fast_two_sum(s, e, s2, e2);
    e2 += f;
    return df_norm(s2, e2);
}

__device__ __forceinline__ dfloat df_neg(dfloat a) { return df_make(-a.x, -a.y); }

__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) { return df_add(a, df_neg(b)); }

// a * b: the exact product of the high parts plus the cross terms
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return df_norm(p, e);
}

// c - a b with one normalisation: the product is split exactly (plus cross
// terms) and its high part subtracted by two-sum; the remaining small terms
// are added without a second two-sum, so the error is ~2^-48 (|c| + |a b|)
// (the bound a backward-stable elimination step needs)
__device__ __forceinline__ dfloat df_fnms(dfloat a, dfloat b, dfloat c)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    float s, t;
    two_sum(c.x, -p, s, t);
    t += c.y - e;
    return df_norm(s, t);
}

// 1 / a: FP32 reciprocal refined by one Newton step carried in double-float,
// y1 = y + y (1 - a y); the seed's relative error (~2^-23) is squared
__device__ __forceinline__ dfloat df_recip(dfloat a)
{
    // hardware reciprocal approximation as the seed (the Newton step below
    // squares its ~2^-22 relative error)
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.x));
    // 1 - a y with a = hi + lo: fma gives 1 - hi y exactly rounded once
    const float r = fmaf(-a.x, y, 1.0f) - a.y * y;
    return df_norm(y, y * r);
}

// Accumulator for sums of products a_k b_k of double-float operands: the
// high products are split exactly and added by two-sum into (s, c); the
// cross terms and rounding errors go into c. Normalised once at the end.
struct DfAcc {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add_prod(dfloat a, dfloat b)
    {
        const float p = a.x * b.x;
        float e = fmaf(a.x, b.x, -p);
        e = fmaf(a.x, b.y, e);
        e = fmaf(a.y, b.x, e);
        float t, err;
        two_sum(s, p, t, err);
        s = t;
        c += err + e;
    }
    __device__ __forceinline__ void add(dfloat a)
    {
        float t, err;
        two_sum(s, a.x, t, err);
        s = t;
        c += err + a.y;
    }
    __device__ __forceinline__ dfloat value() const { return df_norm(s, c); }
};

// FP64 <-> double-float (two FP64-pipe conversions and one subtraction)
__device__ __forceinline__ dfloat df_from_double(double v)
{
    const float hi = (float)v;
    return df_make(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.x + (double)a.y; }

// butterfly sum of a double-float over the lanes of a warp (fixed order)
__device__ __forceinline__ dfloat df_warp_sum(dfloat v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfloat w;
        w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = df_add(v, w);
    }
    return v;
}

}  // namespace pba
