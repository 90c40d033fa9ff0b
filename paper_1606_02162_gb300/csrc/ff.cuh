// Double-float arithmetic for the FP64-class quality reductions of FP32
// placements (shared by the reduction kernels of layout.cu and blocked.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gila {

// Double-float arithmetic: a value held as an unevaluated sum hi + lo of
// two FP32 numbers (|lo| at most half an ulp of hi), 48 significant bits.
// The building blocks are the exact error-free transformations of Knuth
// (two-sum) and Dekker (two-product, here through a fused multiply-add);
// every FP32 operation below is an explicitly rounded intrinsic, so the
// compiler neither contracts nor reorders them.
struct Ff {
    float hi, lo;
};

__device__ __forceinline__ Ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ Ff ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ Ff ff_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ Ff ff_from_double(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ Ff ff_add(Ff a, Ff b)
{
    const Ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ Ff ff_mul(Ff a, Ff b)
{
    const Ff p = ff_two_prod(a.hi, b.hi);
    const float c = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return ff_fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}

// |x_u - x_v|^2 from FP32 coordinates: the differences are exact as
// double-floats (two-sum), their squares exact as double-floats
// (two-product); only the square of each difference's low part (below
// 2^-48 of the result) is left out.
__device__ __forceinline__ Ff ff_dist2(float ax, float ay, float bx, float by)
{
    const Ff dx = ff_two_sum(ax, -bx);
    const Ff dy = ff_two_sum(ay, -by);
    const Ff px = ff_two_prod(dx.hi, dx.hi);
    const Ff py = ff_two_prod(dy.hi, dy.hi);
    const Ff s = ff_two_sum(px.hi, py.hi);
    const float cross = __fmaf_rn(2.0f * dx.hi, dx.lo, __fmul_rn(2.0f * dy.hi, dy.lo));
    const float low = __fadd_rn(__fadd_rn(s.lo, __fadd_rn(px.lo, py.lo)), cross);
    return ff_fast_two_sum(s.hi, low);
}

// 1 / sqrt(r2) for r2 = hi + lo > 0: the hardware's approximate reciprocal
// square root y0 of hi (relative error below 2^-22) refined by the series
// y = y0 (1 + e/2 + 3e^2/8) of y0 / sqrt(1 - e), with e = 1 - r2 y0^2 formed
// exactly up to the rounding of its low parts (the classical Newton step for
// the inverse square root carried one order further). ff_rsqrt_pow then
// takes q double-float products, (1 / sqrt(r2))^q (q >= 0); for q = 1 its
// product 1 * y equals y exactly (y is normalised).
__device__ __forceinline__ Ff ff_rsqrt(Ff r2)
{
    float y0;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(y0) : "f"(r2.hi));
    const Ff y2 = ff_two_prod(y0, y0);
    const Ff t = ff_two_prod(r2.hi, y2.hi);
    const float tl = __fadd_rn(t.lo, __fmaf_rn(r2.hi, y2.lo, __fmul_rn(r2.lo, y2.hi)));
    const float e = __fsub_rn(__fsub_rn(1.0f, t.hi), tl);  // 1 - t.hi is exact near 1
    const float corr = __fmul_rn(y0, __fmaf_rn(0.375f * e, e, 0.5f * e));
    return ff_fast_two_sum(y0, corr);
}

__device__ __forceinline__ Ff ff_rsqrt_pow(Ff r2, int q)
{
    const Ff y = ff_rsqrt(r2);
    Ff r = {1.0f, 0.0f};
    for (int i = 0; i < q; ++i) r = ff_mul(r, y);
    return r;
}


}  // namespace gila
