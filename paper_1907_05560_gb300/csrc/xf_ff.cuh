// xf_ff.cuh -- float-float numbers for the per-bin arithmetic of the
// XF_FP32X2 precision.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (about 48 significant bits, unit roundoff near 2^-47).  The operations
// follow the double-float arithmetic of Dekker (1971): Knuth's TwoSum for
// the exact error of a sum, the fused multiply-add for the exact error of a
// product, and a final renormalisation (Dekker's Fast2Sum).  On GB300 a warp
// issues 64 float operations per FP64 one, so a float-float operation of
// 5-15 float instructions costs a fraction of an FP64 operation while keeping
// most of its precision.
//
// The device code uses the *_rn intrinsics for every rounding step that must
// stay a separate operation: the compiler never fuses them into an FMA,
// which would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

#include <math.h>

#if defined(__CUDACC__)
#define XF_FF_NOINLINE __noinline__
#else
#define XF_FF_NOINLINE __attribute__((noinline))
#endif

namespace xf {

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float ff_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ff_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ff_mul(float a, float b) { return __fmul_rn(a, b); }
#else
inline float ff_add(float a, float b) { return a + b; }
inline float ff_sub(float a, float b) { return a - b; }
inline float ff_mul(float a, float b) { return a * b; }
#endif

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ ff(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ ff(int i) : hi((float)i), lo(0.0f) {} // the small literals of the templates
    // the double rounded to float, and the rest rounded to float
    __host__ __device__ ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__host__ __device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }

// s + e == a + b exactly, s = fl(a + b) (Knuth's TwoSum)
__host__ __device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = ff_add(a, b);
    const float bb = ff_sub(s, a);
    e = ff_add(ff_sub(a, ff_sub(s, bb)), ff_sub(b, bb));
}
// the same when |a| >= |b| (Dekker's Fast2Sum): the renormalisation step
__host__ __device__ __forceinline__ ff fast_two_sum_f(float a, float b)
{
    const float s = ff_add(a, b);
    return ff(s, ff_sub(b, ff_sub(s, a)));
}

__host__ __device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ ff operator+(ff a, ff b)
{
    float s, e;
    two_sum_f(a.hi, b.hi, s, e);
    e = ff_add(e, ff_add(a.lo, b.lo));
    return fast_two_sum_f(s, e);
}
__host__ __device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__host__ __device__ __forceinline__ ff operator*(ff a, ff b)
{
    const float p = ff_mul(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p); // the product's rounding error, exact
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum_f(p, e);
}
__host__ __device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
__host__ __device__ __forceinline__ ff &operator-=(ff &a, ff b) { return a = a - b; }
__host__ __device__ __forceinline__ ff &operator*=(ff &a, ff b) { return a = a * b; }

// a b + c without the final renormalisation: hi + lo is the sum, lo not
// bounded by ulp(hi)/2 (an input of another fma_r, which takes c.hi and c.lo
// apart anyway)
__host__ __device__ __forceinline__ ff fma_nr(ff a, ff b, ff c)
{
    const float p = ff_mul(a.hi, b.hi);
    const float pe = fmaf(a.hi, b.hi, -p);
    float s, se;
    two_sum_f(p, c.hi, s, se);
    const float t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, c.lo));
    return ff(s, ff_add(ff_add(pe, se), t));
}

// a b + c with one renormalisation
__host__ __device__ __forceinline__ ff fma_r(ff a, ff b, ff c)
{
    const float p = ff_mul(a.hi, b.hi);
    const float pe = fmaf(a.hi, b.hi, -p);
    float s, se;
    two_sum_f(p, c.hi, s, se);
    const float t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, c.lo));
    return fast_two_sum_f(s, ff_add(ff_add(pe, se), t));
}

__host__ __device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__host__ __device__ __forceinline__ bool operator<(ff a, ff b) { return b > a; }
__host__ __device__ __forceinline__ bool operator>=(ff a, ff b) { return !(b > a); }
__host__ __device__ __forceinline__ bool operator<=(ff a, ff b) { return !(a > b); }
__host__ __device__ __forceinline__ ff abs_r(ff a) { return a.hi < 0.0f ? -a : a; }

// 1/sqrt(x) for x > 0 in the normal float range: the float reciprocal square
// root y (two ulps), then one third-order correction in float-float:
// with e = 1 - x y^2, 1/sqrt(x) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + O(e^3)),
// and |e| < 2^-21 leaves O(e^3) below 2^-60.
__host__ __device__ __forceinline__ ff rsqrt_r(ff x)
{
#ifdef __CUDA_ARCH__
    const float y = rsqrtf(x.hi);
#else
    const float y = 1.0f / sqrtf(x.hi);
#endif
    // t = x y^2 in float-float (a float times a float-float, twice)
    auto mulf = [](ff a, float b) {
        const float p = ff_mul(a.hi, b);
        float e = fmaf(a.hi, b, -p);
        e = fmaf(a.lo, b, e);
        return fast_two_sum_f(p, e);
    };
    const ff t = mulf(mulf(x, y), y);
    const float e = ff_sub(ff_sub(1.0f, t.hi), t.lo); // 1 - t.hi is exact (t.hi near 1)
    const float c = e * fmaf(0.375f, e, 0.5f);
    const float p = ff_mul(y, c);
    const float pe = fmaf(y, c, -p);
    return fast_two_sum_f(y, ff_add(p, pe));
}

// The step's path length: a double, rounded to float-float for the phase.
template <typename Real> struct StepLen;
template <> struct StepLen<ff> {
    double v;
};
__host__ __device__ __forceinline__ StepLen<ff> make_step_len(double dl, ff *) { return {dl}; }
__host__ __device__ __forceinline__ ff step_len_value(StepLen<ff> d) { return ff(d.v); }

// a float-float constant from a double literal, at compile time
__host__ __device__ constexpr ff ff_const(double d) { return ff((float)d, (float)(d - (double)(float)d)); }
// a float-float times a float
__host__ __device__ __forceinline__ ff mul_f(ff a, float b)
{
    const float p = ff_mul(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum_f(p, e);
}

// sin r and cos r for |r| <= pi/4 (plus the reduction's rounding) from their
// Taylor series about 0: float-float Horner steps for the terms above
// 1e-8 of the result, plain float for the tail (through r^17 and r^16; the
// first omitted terms are below 1e-16 there).
__host__ __device__ __forceinline__ void sincos_octant_ff(ff r, ff *s, ff *c)
{
    const ff r2 = r * r;
    const float q = r2.hi;
    // sin r = r + r^3 (c3 + r2 (c5 + r2 (c7 + r2 (c9 + r2 tail))))
    const float ts = fmaf(q, fmaf(q, fmaf(q, (float)(1.0 / 355687428096000.0), (float)(-1.0 / 1307674368000.0)),
                                  (float)(1.0 / 6227020800.0)), (float)(-1.0 / 39916800.0));
    ff ps = fma_r(r2, ff(ts), ff_const(1.0 / 362880.0));
    ps = fma_r(r2, ps, ff_const(-1.0 / 5040.0));
    ps = fma_r(r2, ps, ff_const(1.0 / 120.0));
    ps = fma_r(r2, ps, ff_const(-1.0 / 6.0));
    *s = fma_r(r * r2, ps, r);
    // cos r = 1 + r2 (c2 + r2 (c4 + r2 (c6 + r2 (c8 + r2 tail))))
    const float tc = fmaf(q, fmaf(q, fmaf(q, (float)(1.0 / 20922789888000.0), (float)(-1.0 / 87178291200.0)),
                                  (float)(1.0 / 479001600.0)), (float)(-1.0 / 3628800.0));
    ff pc = fma_r(r2, ff(tc), ff_const(1.0 / 40320.0));
    pc = fma_r(r2, pc, ff_const(-1.0 / 720.0));
    pc = fma_r(r2, pc, ff_const(1.0 / 24.0));
    pc = fma_r(r2, pc, ff_const(-0.5));
    *c = fma_r(r2, pc, ff(1.0f));
}

// (sin, cos) of the phase lam * dl.  The product in float-float, reduced to
// [-pi/4, pi/4] and a quadrant by Cody and Waite's method (pi/2 in three
// floats: 1.5703125 with 8 significant bits, so k * 1.5703125 is exact for
// |k| < 2^16, the next part's product kept exact by the FMA, the last one
// rounded), then the polynomials above: no FP64 instruction (the FP64 pipe
// carries the conversions of the state; with the FP64 library sine-cosine
// here the three-flavor workload ran 7 % and the ensemble 8 % slower).
// Phases beyond 2^15 rad take the FP64 library sine-cosine.
__host__ __device__ __forceinline__ void phase_sincos(ff lam, StepLen<ff> d, ff *s, ff *c)
{
    if (!(fabsf(lam.hi * (float)d.v) < 32768.0f)) {
        double sd, cd;
        sincos(to_double(lam) * d.v, &sd, &cd);
        *s = ff(sd);
        *c = ff(cd);
        return;
    }
    const ff x = lam * ff(d.v);
    const float k = rintf(x.hi * 0.636619772367581343f); // 2 / pi
    ff r = x + ff(-k * 1.5703125f);
    const float p2 = ff_mul(k, 4.838267923332751e-4f); // float(pi/2 - 1.5703125)
    r = r + (-ff(p2, fmaf(k, 4.838267923332751e-4f, -p2)));
    r = r + ff(-k * 2.5633440682570896e-12f); // pi/2 - 1.5703125 - that float
    ff sr, cr;
    sincos_octant_ff(r, &sr, &cr);
    const int qd = (int)k;
    const ff sv = (qd & 1) ? cr : sr, cv = (qd & 1) ? sr : cr;
    *s = (qd & 2) ? -sv : sv;
    *c = ((qd + 1) & 2) ? -cv : cv;
}

// Complex products and sums of products on float-float parts, as calls: one
// copy of each in the code.  Inlined like the rest, the propagator's code
// overflows the instruction cache (hit rate 55 %, issue on 20 % of cycles);
// as calls the three-flavor workload ran 1.35x and the ensemble 1.6x faster.
// Overloads of the templates in xf_math.cuh, preferred as exact matches.  The
// inner product-sum of each component is not renormalised (the outer one
// takes it apart anyway): 2-3 % faster, no change in the host check.
static __host__ __device__ XF_FF_NOINLINE cx<ff> cfma(cx<ff> a, cx<ff> b, cx<ff> acc)
{
    return {fma_r(a.r, b.r, fma_nr(-a.i, b.i, acc.r)), fma_r(a.r, b.i, fma_nr(a.i, b.r, acc.i))};
}
static __host__ __device__ XF_FF_NOINLINE cx<ff> cfmac(cx<ff> a, cx<ff> b, cx<ff> acc)
{
    return {fma_r(a.r, b.r, fma_nr(a.i, b.i, acc.r)), fma_r(a.i, b.r, fma_nr(-a.r, b.i, acc.i))};
}
// a conj(b) and a b
static __host__ __device__ XF_FF_NOINLINE cx<ff> mulc(cx<ff> a, cx<ff> b)
{
    return {fma_r(a.r, b.r, a.i * b.i), fma_r(a.i, b.r, -(a.r * b.i))};
}
static __host__ __device__ XF_FF_NOINLINE cx<ff> operator*(cx<ff> a, cx<ff> b)
{
    return {fma_r(a.r, b.r, -(a.i * b.i)), fma_r(a.r, b.i, a.i * b.r)};
}

template <typename Real> struct JacobiTol;
// Sweeps stop at an off-diagonal norm of 1e-13 of the matrix's: a few units
// of the float-float rounding, past which a sweep only chases rounding.
template <> struct JacobiTol<ff> {
    static constexpr float rel2 = 1e-26f;
    static constexpr int sweeps = 8;
};

} // namespace xf
