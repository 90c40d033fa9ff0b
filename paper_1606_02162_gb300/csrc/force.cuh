// Device helpers shared by the iteration kernels (single graph, tiled and
// batched): position vector types, streaming id loads, the per-pair force
// term, compensated accumulators, row traversal and the capped move.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device_util.cuh"
#include "gila_impl.h"

namespace gila {

template <class T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

enum Model { kFR = 0, kGeneric = 1 };


// Streaming load of four ids: read once per iteration, kept out of L1 so
// that L1 serves the position gathers.
__device__ __forceinline__ uint4 ld_ids4(const uint4* p)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ld_id(const uint32_t* p)
{
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

template <class T>
__device__ __forceinline__ T ipow_(T x, int e)
{
    T r = T(1);
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fsqrt(float r2) { return r2 * rsqrtf(r2); }
__device__ __forceinline__ double fsqrt(double r2) { return sqrt(r2); }

// Force accumulator; COMP adds a running compensation term per component
// (two-sum), which removes the rounding error of long float sums.
template <class T, bool COMP>
struct Acc {
    T sx = T(0), sy = T(0), cx = T(0), cy = T(0);

    __device__ __forceinline__ static void two_sum(T& s, T& c, T x)
    {
        const T t = s + x;
        const T bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ void add(T x, T y)
    {
        if (COMP) {
            two_sum(sx, cx, x);
            two_sum(sy, cy, y);
        } else {
            sx += x;
            sy += y;
        }
    }
    __device__ __forceinline__ void merge(T ox, T oy, T ocx, T ocy)
    {
        if (COMP) {
            two_sum(sx, cx, ox);
            two_sum(sy, cy, oy);
            cx += ocx;
            cy += ocy;
        } else {
            sx += ox;
            sy += oy;
        }
    }
    __device__ __forceinline__ void group_reduce(int width)
    {
        for (int o = width >> 1; o > 0; o >>= 1) {
            const T ox = __shfl_xor_sync(kFull, sx, o, width);
            const T oy = __shfl_xor_sync(kFull, sy, o, width);
            const T ocx = COMP ? __shfl_xor_sync(kFull, cx, o, width) : T(0);
            const T ocy = COMP ? __shfl_xor_sync(kFull, cy, o, width) : T(0);
            merge(ox, oy, ocx, ocy);
        }
    }
    __device__ __forceinline__ T fx() const { return COMP ? sx + cx : sx; }
    __device__ __forceinline__ T fy() const { return COMP ? sy + cy : sy; }
};

// Where a kernel reads positions from.
enum Src {
    kSrcGlobal = 0,   // the whole placement, read-only for the launch (ld.global.nc)
    kSrcShared = 1,   // a shared-memory tile of ids [base, base + size), 32-bit addresses
    kSrcGeneric = 2   // a buffer of ids [base, base + size) in shared or global memory
};

// 1/x in FP64 by Newton-Raphson iteration for the reciprocal: the hardware's
// approximate reciprocal as the seed, then two steps y <- y + y (1 - x y),
// each squaring the seed's relative error (below 2^-22 at the start), so the
// result is within about an ulp of 1/x at a third of an IEEE division's
// FP64 operations. For x > 0 (x = 0 gives no finite result; callers test).
__device__ __forceinline__ double rcp_newton(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// Reciprocal square root, one approximate MUFU operation (denormals flushed).
__device__ __forceinline__ float rsqrt_fast(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Squared distance beyond which the generic force model takes a term as zero.
template <class T> __device__ __forceinline__ T far_r2();
template <> __device__ __forceinline__ float far_r2<float>() { return 1.0e38f; }
template <> __device__ __forceinline__ double far_r2<double>() { return 1.0e300; }

// Reciprocal, one approximate MUFU operation (denormals flushed; +inf at 0).
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Position of id v for a kernel reading from `SRC`.
template <class T, int SRC>
struct PosSource {
    using P2 = typename V2<T>::type;
    const P2* __restrict__ pos = nullptr;  // kSrcGlobal / kSrcGeneric
    uint32_t base = 0;                     // first id held (kSrcShared / kSrcGeneric)
    const P2* shp = nullptr;               // kSrcShared: tile shifted so that shp[v] is id v

    // kSrcShared: `tile` holds ids [first, ...). Plain indexing (not inline
    // ld.shared) leaves the compiler free to schedule the gathers.
    __device__ __forceinline__ void set_shared(const P2* tile, uint32_t first)
    {
        base = first;
        shp = tile - first;
    }
    __device__ __forceinline__ P2 operator()(uint32_t v) const
    {
        if (SRC == kSrcShared) return shp[v];
        if (SRC == kSrcGeneric) return pos[v - base];
        return __ldg(pos + v);
    }
};

// Repulsion of one k-hop entry v on u (Section 3.1 with the repelling set
// of Section 4.5): adds c (x_u - x_v) with c = d^2 / delta^(q+1). For
// Fruchterman-Reingold (q = 1) in FP32 that is d^2 * rsqrt(r^2)^2, or
// rcp(r^2) unscaled: one MUFU, no divide. A pair at distance 0 adds nothing. With
// UNSCALED the factor d^2 is left out (the caller multiplies the row's sum
// by it once). With WEIGHTED the term is multiplied by wt[v], the repulsion
// weight of the repelling vertex (Section 4.6).
template <class T, int MODEL, bool COMP, int SRC = kSrcGlobal, bool UNSCALED = false,
          bool WEIGHTED = false>
struct Rep {
    using P2 = typename V2<T>::type;
    PosSource<T, SRC> src;
    T xu, yu, d2;
    int q;
    const T* __restrict__ wt = nullptr;

    template <bool C = COMP>
    __device__ __forceinline__ void operator()(uint32_t v, Acc<T, C>& a) const
    {
        if constexpr (sizeof(T) == 4 && MODEL == kFR && UNSCALED && !WEIGHTED && SRC == kSrcShared) {
            // the blocked kernel's FP32 term with packed two-lane FP32
            // arithmetic (sm_100 and later): one subtraction forms
            // (dx, dy) and one fused multiply-add accumulates c (dx, dy)
            const P2 pv = src(v);
            uint64_t pu, pp, dd, cc, ac;
            asm("mov.b64 %0, {%1, %2};" : "=l"(pu) : "f"(xu), "f"(yu));
            asm("mov.b64 %0, {%1, %2};" : "=l"(pp) : "f"(pv.x), "f"(pv.y));
            asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dd) : "l"(pu), "l"(pp));
            float dx, dy;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(dx), "=f"(dy) : "l"(dd));
            const float c = rep_fr1(dx, dy);
            asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
            asm("mov.b64 %0, {%1, %2};" : "=l"(ac) : "f"(a.sx), "f"(a.sy));
            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(ac) : "l"(cc), "l"(dd));
            asm("mov.b64 {%0, %1}, %2;" : "=f"(a.sx), "=f"(a.sy) : "l"(ac));
            return;
        }
        const P2 pv = src(v);
        const T dx = xu - pv.x, dy = yu - pv.y;
        T c;
        if (MODEL == kFR) {
            c = UNSCALED ? rep_fr1(dx, dy) : rep_fr(d2, dx * dx + dy * dy);
        } else {
            const T r2 = dx * dx + dy * dy;
            c = T(0);
            // beyond r^2 = 1e38 (FP32) or 1e300 (FP64) the term is taken as
            // zero (padding entries of the blocked layout lie there)
            if (r2 > T(0) && r2 < far_r2<T>()) {
                const T dl = sqrt(r2);
                c = (UNSCALED ? T(1) : d2) / (ipow_(dl, q) * dl);
            }
        }
        if (WEIGHTED) c *= __ldg(wt + v);
        a.add(c * dx, c * dy);
    }

    // (the plain kernels: rsqrt squared measured 4% faster there than rcp)
    __device__ __forceinline__ static float rep_fr(float d2, float r2)
    {
        const float r = rsqrt_fast(r2);
        return r2 > 0.0f ? d2 * (r * r) : 0.0f;
    }
    __device__ __forceinline__ static double rep_fr(double d2, double r2)
    {
        return r2 > 0.0 ? d2 * rcp_newton(r2) : 0.0;
    }
    // 1 / r^2 in FP32: one approximate reciprocal of r^2 + 2^-100. The added
    // 2^-100 is less than half an ulp of any r^2 >= 2^-75 (far below any
    // distance of a placement), so it changes such an r^2 by at most its
    // rounding; at r^2 = 0
    // (coincident vertices) it keeps the factor finite (2^100), and the
    // factor then multiplies dx = dy = 0 exactly: the pair adds nothing.
    __device__ __forceinline__ static float rep_fr1(float dx, float dy)
    {
        return rcp_fast(fmaf(dx, dx, fmaf(dy, dy, 0x1p-100f)));
    }
    __device__ __forceinline__ static double rep_fr1(double dx, double dy)
    {
        const double r2 = dx * dx + dy * dy;
        return r2 > 0.0 ? rcp_newton(r2) : 0.0;
    }
};

// Attraction of a neighbour v of u: adds -c (x_u - x_v) with
// c = delta^(p-1) / d (delta / d for p = 2).
template <class T, int MODEL, bool COMP, int SRC = kSrcGlobal>
struct Att {
    using P2 = typename V2<T>::type;
    PosSource<T, SRC> src;
    T xu, yu, inv_d;
    int p;

    __device__ __forceinline__ void operator()(uint32_t v, Acc<T, COMP>& a) const
    {
        const P2 pv = src(v);
        const T dx = xu - pv.x, dy = yu - pv.y;
        const T r2 = dx * dx + dy * dy;
        if (r2 > T(0)) {
            T c;
            if (MODEL == kFR) {
                c = fsqrt(r2) * inv_d;
            } else {
                const T dl = sqrt(r2);
                c = ipow_(dl, p) / dl * inv_d;
            }
            a.add(-c * dx, -c * dy);
        }
    }
};

// Entries [s, e) of kcol, lanes gl = 0..G-1 of a group (G >= 4): an
// unaligned head of at most 3 entries, 16-byte vector loads of 4 ids,
// then a tail of at most 3 entries. Which lane takes which entry depends on
// the row's position modulo 4 in kcol (fixed for a given list).
template <class F, class A>
__device__ __forceinline__ void row_sum(const uint32_t* __restrict__ kcol, int64_t s, int64_t e,
                                        int gl, int G, const F& f, A& a)
{
    int64_t s4 = (s + 3) & ~int64_t(3);
    if (s4 > e) s4 = e;
    int64_t e4 = e & ~int64_t(3);
    if (e4 < s4) e4 = s4;
    if (s + gl < s4) f(ld_id(kcol + s + gl), a);
    const uint4* k4 = reinterpret_cast<const uint4*>(kcol + s4);
    const int n4 = (int)((e4 - s4) >> 2);
#pragma unroll 4
    for (int c = gl; c < n4; c += G) {
        const uint4 w = ld_ids4(k4 + c);
        f(w.x, a);
        f(w.y, a);
        f(w.z, a);
        f(w.w, a);
    }
    if (e4 + gl < e) f(ld_id(kcol + e4 + gl), a);
}

// Entries [s, e) with lane gl taking entries s + gl, s + gl + G, ...: the
// assignment depends only on the position inside the row.
template <class F, class A>
__device__ __forceinline__ void row_sum_rel(const uint32_t* __restrict__ ids, int64_t s, int64_t e,
                                            int gl, int G, const F& f, A& a)
{
    const uint32_t* p = ids + s;
    const int len = (int)(e - s);
    for (int j = gl; j < len; j += G) f(ld_id(p + j), a);
}

template <class T>
__device__ __forceinline__ void apply_move(double t_, void* pos_out, void* disp_out, int64_t u,
                                           T xu, T yu, T fx, T fy)
{
    using P2 = typename V2<T>::type;
    const T t = (T)t_;
    const T fn = sqrt(fx * fx + fy * fy);
    T mx = fx, my = fy;
    if (fn > t) {
        const T sc = t / fn;
        mx = fx * sc;
        my = fy * sc;
    }
    P2 o;
    o.x = xu + mx;
    o.y = yu + my;
    reinterpret_cast<P2*>(pos_out)[u] = o;
    if (disp_out) {
        P2 m;
        m.x = mx;
        m.y = my;
        reinterpret_cast<P2*>(disp_out)[u] = m;
    }
}

}  // namespace gila
