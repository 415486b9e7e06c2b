// xf_math.cuh -- per-bin arithmetic of the flavor-evolution path on packed,
// traceless Hermitian components (device side).
//
// A density matrix or Hamiltonian is stored as its traceless part; the trace
// of rho is constant (d tr rho/dr = tr(-i[H,rho]) = 0) and the trace of H
// drops out of every commutator and of U rho U^dagger.
//
//   2 flavors, S = 3:  T = [[a, x + i y], [x - i y, -a]]
//                      comps (a, x, y)
//   3 flavors, S = 8:  T = [[t1, z12, z13], [., t2, z23], [., ., -t1-t2]]
//                      comps (t1, t2, Re z12, Im z12, Re z13, Im z13, Re z23, Im z23)
//
// Equations: d rho/dl = -i [H, rho] (Eq. 3.2/3.4 written for rho); the
// propagator exp(-i H dl) of Eq. 3.10-3.12.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <math.h>

namespace xf {

template <int NF> struct Comp;
template <> struct Comp<2> { static constexpr int S = 3; };
template <> struct Comp<3> { static constexpr int S = 8; };

// ---------------------------------------------------------------- helpers
__host__ __device__ __forceinline__ void sincos_r(double x, double *s, double *c) { sincos(x, s, c); }
__host__ __device__ __forceinline__ void sincos_r(float x, float *s, float *c) { sincosf(x, s, c); }
__host__ __device__ __forceinline__ double abs_r(double x) { return fabs(x); }
__host__ __device__ __forceinline__ float abs_r(float x) { return fabsf(x); }
__host__ __device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
// 1/sqrt(x): the device's reciprocal square root (1 ulp in FP64, 2 in FP32);
// the host build (used only to count operations) divides.
__host__ __device__ __forceinline__ double rsqrt_r(double x)
{
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}
__host__ __device__ __forceinline__ float rsqrt_r(float x)
{
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}

// Step path length in the precision of the phase arithmetic: FP64 for the
// FP64 path; for FP32 an unevaluated sum hi + lo of two floats (about 48
// significant bits), so that the phase lam * dl of a long step keeps FP64-like
// accuracy without FP64 instructions (a warp-wide FP64 instruction occupies
// this GPU's FP64 pipe for 16 cycles).
template <typename Real> struct StepLen;
template <> struct StepLen<double> {
    double v;
};
template <> struct StepLen<float> {
    float hi, lo;
};
__host__ __device__ __forceinline__ StepLen<double> make_step_len(double dl, double *) { return {dl}; }
__host__ __device__ __forceinline__ StepLen<float> make_step_len(double dl, float *)
{
    float hi = (float)dl;
    return {hi, (float)(dl - (double)hi)};
}
__host__ __device__ __forceinline__ double step_len_value(StepLen<double> d) { return d.v; }
__host__ __device__ __forceinline__ float step_len_value(StepLen<float> d) { return d.hi; }

// sin r and cos r for |r| <= pi/4 (plus the reduction's rounding) from their
// Taylor series about 0, through r^9 and r^10: the first omitted terms,
// r^11/11! and r^12/12!, are below 2e-9 there, under FP32's half-ulp.
__host__ __device__ __forceinline__ void sincos_octant(float r, float *s, float *c)
{
    const float r2 = r * r;
    float ps = fmaf(r2, (float)(1.0 / 362880.0), (float)(-1.0 / 5040.0));
    ps = fmaf(r2, ps, (float)(1.0 / 120.0));
    ps = fmaf(r2, ps, (float)(-1.0 / 6.0));
    *s = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, (float)(-1.0 / 3628800.0), (float)(1.0 / 40320.0));
    pc = fmaf(r2, pc, (float)(-1.0 / 720.0));
    pc = fmaf(r2, pc, (float)(1.0 / 24.0));
    pc = fmaf(r2, pc, -0.5f);
    *c = fmaf(r2, pc, 1.0f);
}

// (sin, cos) of the phase lam * dl.
//  FP64: directly.
//  FP32: the product in float-float (exact product by FMA, plus lam * lo),
//  reduced to r in [-pi/4, pi/4] and a quadrant k mod 4 by Cody and Waite's
//  method: pi/2 split in three parts (1.5703125 has 8 significant bits, so
//  k * 1.5703125 is exact for |k| < 2^16; the next two parts are pi/2 minus
//  the parts before it, rounded to float).  Phases beyond 2^14 rad take an
//  FP64 reduction.  Then the Taylor polynomials above and the quadrant's
//  swap and signs: no library call, so no slow-path reduction in the loop.
__host__ __device__ __forceinline__ void phase_sincos(double lam, StepLen<double> d, double *s, double *c)
{
    sincos(lam * d.v, s, c);
}
__host__ __device__ __forceinline__ void phase_sincos(float lam, StepLen<float> d, float *s, float *c)
{
    const float p = lam * d.hi;
    float e = fmaf(lam, d.hi, -p); // rounding error of the product, exact
    e = fmaf(lam, d.lo, e);
    float red;
    int q;
    if (fabsf(p) < 16384.0f) {
        const float k = rintf(p * 0.636619772367581343f); // 2 / pi
        red = fmaf(-k, 1.5703125f, p);
        red = fmaf(-k, 4.838267923332751e-4f, red);  // float(pi/2 - 1.5703125)
        red = fmaf(-k, 2.5633440682570896e-12f, red); // pi/2 - 1.5703125 - that float
        red += e;
        q = (int)k;
    } else {
        const double half_pi = 1.5707963267948966192313216916398;
        const double ph = (double)p + (double)e;
        const double k = rint(ph * (1.0 / half_pi));
        red = (float)fma(-k, half_pi, ph);
        const double k4 = k - 4.0 * floor(0.25 * k); // k mod 4, exact for |k| < 2^53
        q = (k4 >= 0.0 && k4 < 4.0) ? (int)k4 : 0;   // 0 for a non-finite phase
    }
    float sr, cr;
    sincos_octant(red, &sr, &cr);
    // sin(r + q pi/2), cos(r + q pi/2): q odd swaps sin and cos; the signs
    // follow the quadrant
    const float sv = (q & 1) ? cr : sr, cv = (q & 1) ? sr : cr;
    *s = (q & 2) ? -sv : sv;
    *c = ((q + 1) & 2) ? -cv : cv;
}

// ---------------------------------------------------------------- 2 flavors
// The Bloch rotation's angle: lam = |h| and, per path length dl, sin(lam dl),
// cos(lam dl) and sigma = sin(lam dl)/lam (dl when lam = 0).  FP64: lam and
// sigma from one reciprocal square root (rl; no square root, no division);
// FP32: the square root and the division, which measured faster there (a
// two-flavor FP32 pack ran 1.5x faster with them).
template <typename Real>
__host__ __device__ __forceinline__ void rotation_lambda(const Real *h, Real *lam, Real *rl)
{
    const Real lam2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    if constexpr (!std::is_same<Real, float>::value) {
        *rl = (lam2 > Real(0)) ? rsqrt_r(lam2) : Real(0);
        *lam = lam2 * *rl;
    } else {
        *lam = sqrt_r(lam2);
        *rl = Real(0); // unused
    }
}
template <typename Real>
__host__ __device__ __forceinline__ void rotation_phase(Real lam, Real rl, StepLen<Real> dl, Real *sn, Real *cs,
                                                        Real *sig)
{
    phase_sincos(lam, dl, sn, cs);
    if constexpr (!std::is_same<Real, float>::value) *sig = (lam > Real(0)) ? *sn * rl : step_len_value(dl);
    else *sig = (lam > Real(0)) ? *sn / lam : step_len_value(dl);
}
template <typename Real>
__host__ __device__ __forceinline__ void rotation_angle(const Real *h, StepLen<Real> dl, Real *sn, Real *cs, Real *sig)
{
    Real lam, rl;
    rotation_lambda(h, &lam, &rl);
    rotation_phase(lam, rl, dl, sn, cs, sig);
}

// -i[H, T] for traceless 2x2 H = (hz, hx, hy), T = (a, x, y):
//   da = 2 (hy x - hx y),  dx = 2 (hz y - a hy),  dy = 2 (a hx - hz x)
template <typename Real>
__host__ __device__ __forceinline__ void comm2(const Real *h, const Real *t, Real *d)
{
    d[0] = Real(2) * (h[2] * t[1] - h[1] * t[2]);
    d[1] = Real(2) * (h[0] * t[2] - t[0] * h[2]);
    d[2] = Real(2) * (t[0] * h[1] - h[0] * t[1]);
}

// T' = U T U^dagger with U = exp(-i H dl) (Eq. 3.11): a rotation of the Bloch
// vector of T about the Bloch vector of H by the angle 2 lam dl,
// lam = sqrt(h11^2 + |h12|^2) (Eq. 3.12).  With W = (1/2)(-i[H,T]) and
// Q the same map applied to W (Rodrigues' formula):
//   T' = T + 2 sigma C W + 2 sigma^2 Q,  sigma = sin(lam dl)/lam, C = cos(lam dl)
template <typename Real>
__host__ __device__ __forceinline__ void prop2(const Real *h, StepLen<Real> dl, const Real *t, Real *out)
{
    Real sn, cs, sig;
    rotation_angle(h, dl, &sn, &cs, &sig);
    Real w[3], q[3];
    w[0] = h[2] * t[1] - h[1] * t[2];
    w[1] = h[0] * t[2] - t[0] * h[2];
    w[2] = t[0] * h[1] - h[0] * t[1];
    q[0] = h[2] * w[1] - h[1] * w[2];
    q[1] = h[0] * w[2] - w[0] * h[2];
    q[2] = w[0] * h[1] - h[0] * w[1];
    Real c1 = Real(2) * sig * cs, c2 = Real(2) * sig * sig;
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k] = t[k] + c1 * w[k] + c2 * q[k];
}

// ---------------------------------------------------------------- 3 flavors
template <typename Real> struct cx {
    Real r, i;
};
template <typename Real> __host__ __device__ __forceinline__ cx<Real> mk(Real r, Real i) { return {r, i}; }
template <typename Real> __host__ __device__ __forceinline__ cx<Real> operator+(cx<Real> a, cx<Real> b)
{
    return {a.r + b.r, a.i + b.i};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> operator-(cx<Real> a, cx<Real> b)
{
    return {a.r - b.r, a.i - b.i};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> operator*(cx<Real> a, cx<Real> b)
{
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> operator*(Real a, cx<Real> b)
{
    return {a * b.r, a * b.i};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> cj(cx<Real> a) { return {a.r, -a.i}; }
// a * conj(b)
template <typename Real> __host__ __device__ __forceinline__ cx<Real> mulc(cx<Real> a, cx<Real> b)
{
    return {a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> neg(cx<Real> a) { return {-a.r, -a.i}; }

__host__ __device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
// acc + a b, acc + a conj(b) and acc + s a (s real) with the products fused
// into the sum: two FMA per component, where a complex product and then a
// complex sum take a multiply, an FMA and an add per component.
template <typename Real> __host__ __device__ __forceinline__ cx<Real> cfma(cx<Real> a, cx<Real> b, cx<Real> acc)
{
    return {fma_r(a.r, b.r, fma_r(-a.i, b.i, acc.r)), fma_r(a.r, b.i, fma_r(a.i, b.r, acc.i))};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> cfmac(cx<Real> a, cx<Real> b, cx<Real> acc)
{
    return {fma_r(a.r, b.r, fma_r(a.i, b.i, acc.r)), fma_r(a.i, b.r, fma_r(-a.r, b.i, acc.i))};
}
template <typename Real> __host__ __device__ __forceinline__ cx<Real> rfma(Real s, cx<Real> a, cx<Real> acc)
{
    return {fma_r(s, a.r, acc.r), fma_r(s, a.i, acc.i)};
}

// -i[H, T] for traceless Hermitian 3x3 (comps layout above).  With X = H T:
//   D_kk = 2 Im X_kk,   D_jk = -i (X_jk - conj(X_kj))  (j < k)
// written out so that real diagonal entries never multiply zero imaginary parts.
template <typename Real>
__host__ __device__ __forceinline__ void comm3(const Real *h, const Real *t, Real *d)
{
    const Real h1 = h[0], h2 = h[1], h3 = -(h[0] + h[1]);
    const Real r1 = t[0], r2 = t[1], r3 = -(t[0] + t[1]);
    const cx<Real> h12 = mk(h[2], h[3]), h13 = mk(h[4], h[5]), h23 = mk(h[6], h[7]);
    const cx<Real> r12 = mk(t[2], t[3]), r13 = mk(t[4], t[5]), r23 = mk(t[6], t[7]);
    // Im(a conj b) = a.i b.r - a.r b.i
    Real d11 = Real(2) * ((h12.i * r12.r - h12.r * r12.i) + (h13.i * r13.r - h13.r * r13.i));
    Real d22 = Real(2) * ((h12.r * r12.i - h12.i * r12.r) + (h23.i * r23.r - h23.r * r23.i));
    // Z12 = (h1 - h2) r12 - (r1 - r2) h12 + h13 conj(r23) - conj(h23) r13
    cx<Real> z12 = (h1 - h2) * r12 - (r1 - r2) * h12 + mulc(h13, r23) - mulc(r13, h23);
    // Z13 = (h1 - h3) r13 - (r1 - r3) h13 + h12 r23 - h23 r12
    cx<Real> z13 = (h1 - h3) * r13 - (r1 - r3) * h13 + h12 * r23 - h23 * r12;
    // Z23 = (h2 - h3) r23 - (r2 - r3) h23 + conj(h12) r13 - h13 conj(r12)
    cx<Real> z23 = (h2 - h3) * r23 - (r2 - r3) * h23 + mulc(r13, h12) - mulc(h13, r12);
    d[0] = d11;
    d[1] = d22;
    // -i Z = (Z.i, -Z.r)
    d[2] = z12.i;
    d[3] = -z12.r;
    d[4] = z13.i;
    d[5] = -z13.r;
    d[6] = z23.i;
    d[7] = -z23.r;
}

// index of the stored upper entry (a, b), a < b: (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
__host__ __device__ constexpr int oidx(int a, int b) { return a == 0 ? b - 1 : 2; }

// One Jacobi rotation on pivot (P, Q) of the Hermitian matrix held as diag
// dg[3] and upper entries o[3], accumulating V <- V J with
// J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] on rows/cols (P, Q),
// e^{i phi} = A_PQ / |A_PQ| and theta the smaller rotation angle that zeroes
// the (P, Q) entry: with d = (A_QQ - A_PP)/2 and D = sqrt(d^2 + |A_PQ|^2),
//   tan(theta) = sgn(d) |A_PQ| / (|d| + D),  c^2 = (1 + |d|/D) / 2,
// from which (using 1/(|d| + D) = 1/(2 D c^2))
//   s e^{i phi} = sgn(d) A_PQ / (2 D c),  t |A_PQ| = sgn(d) |A_PQ|^2 / (2 D c^2),
// and A_PP -> A_PP - t |A_PQ|, A_QQ -> A_QQ + t |A_PQ|.  With rD = 1/D and
// rc = 1/c from two reciprocal square roots, the rotation needs no division
// and no square root.
// ZR: which entry of the third row R is exactly zero on entry (the pivot the
// previous rotation of a cyclic (0,1), (0,2), (1,2) sweep zeroed): 0 none,
// 1 A_RP, 2 A_RQ; its terms are left out (x * 0 is not folded in IEEE
// arithmetic).
template <typename Real, int P, int Q, int ZR = 0>
__host__ __device__ __forceinline__ bool jacobi_angles(Real *dg, cx<Real> *o, Real *c_out, cx<Real> *se_out)
{
    constexpr int R = 3 - P - Q;
    cx<Real> g = o[oidx(P, Q)];
    Real ag2 = g.r * g.r + g.i * g.i;
    if (!(ag2 > Real(0))) {
        *c_out = Real(1);
        *se_out = mk(Real(0), Real(0));
        return false;
    }
    const Real d = Real(0.5) * (dg[Q] - dg[P]);
    const Real rD = rsqrt_r(d * d + ag2);
    const Real u = Real(0.5) + Real(0.5) * abs_r(d) * rD; // c^2, in [1/2, 1]
    const Real rc = rsqrt_r(u);
    const Real c = u * rc;
    const Real h = (d >= Real(0) ? Real(0.5) : Real(-0.5)) * rD * rc; // sgn(d) / (2 D c)
    const Real tg = h * rc * ag2;                                     // t |A_PQ|
    const cx<Real> se = mk(h * g.r, h * g.i), sec = mk(h * g.r, -h * g.i); // s e^{+-i phi}
    dg[P] -= tg;
    dg[Q] += tg;
    o[oidx(P, Q)] = mk(Real(0), Real(0));
    // A_RP and A_RQ: stored when R is the row of an upper entry, else conjugated
    cx<Real> aRP = (R < P) ? o[oidx(R, P)] : cj(o[oidx(P, R)]);
    cx<Real> aRQ = (R < Q) ? o[oidx(R, Q)] : cj(o[oidx(Q, R)]);
    // (J^dagger A J)_RP = c A_RP - s e^{-i phi} A_RQ,  (.)_RQ = s e^{i phi} A_RP + c A_RQ
    cx<Real> nRP, nRQ;
    if constexpr (ZR == 1) {
        const cx<Real> m = sec * aRQ;
        nRP = mk(-m.r, -m.i);
        nRQ = c * aRQ;
    } else if constexpr (ZR == 2) {
        nRP = c * aRP;
        nRQ = se * aRP;
    } else {
        nRP = cfma(neg(sec), aRQ, c * aRP);
        nRQ = cfma(se, aRP, c * aRQ);
    }
    if (R < P) o[oidx(R, P)] = nRP;
    else o[oidx(P, R)] = cj(nRP);
    if (R < Q) o[oidx(R, Q)] = nRQ;
    else o[oidx(Q, R)] = cj(nRQ);
    *c_out = c;
    *se_out = se;
    return true;
}

template <typename Real, int P, int Q, int ZR = 0>
__host__ __device__ __forceinline__ void jacobi_rot(Real *dg, cx<Real> *o, cx<Real> (*V)[3])
{
    Real c;
    cx<Real> se;
    if (!jacobi_angles<Real, P, Q, ZR>(dg, o, &c, &se)) return;
    const cx<Real> sec = cj(se);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cx<Real> vp = V[k][P], vq = V[k][Q];
        V[k][P] = cfma(neg(sec), vq, c * vp);
        V[k][Q] = cfma(se, vp, c * vq);
    }
}

// Sweeps stop once the off-diagonal part's squared norm is below rel2 times
// the matrix's.  FP32: 1e-13 (off-diagonal below 3.2e-7 of the norm, a few
// ulps; once there, what is left changes T' = U T U^dagger by less than the
// float rounding of the phases).  A tighter bound spends sweeps on rounding
// noise: on the batched ensemble's three-flavor Hamiltonians 1e-15 took 2.39
// sweeps on average and 2.55 as the maximum over runs of 32 energies, 1e-13
// 2.27 and 2.39, while the propagated T' moved by under 1 % of its FP32 error.
template <typename Real> struct JacobiTol;
template <> struct JacobiTol<double> {
    static constexpr double rel2 = 1e-34;
    static constexpr int sweeps = 8;
};
template <> struct JacobiTol<float> {
    static constexpr float rel2 = 1e-13f;
    static constexpr int sweeps = 6;
};

// T' = U T U^dagger with U = exp(-i H dl), H traceless Hermitian 3x3:
// H = V diag(lam) V^dagger by cyclic Jacobi (eig3), then
// T' = V (E o (V^dagger T V)) V^dagger with E_jk = exp(-i (lam_j - lam_k) dl)
// (apply3); prop3 is the two in sequence.
template <typename Real>
__host__ __device__ __forceinline__ void eig3(const Real *h, Real *dg, cx<Real> (*V)[3])
{
    dg[0] = h[0];
    dg[1] = h[1];
    dg[2] = -(h[0] + h[1]);
    cx<Real> o[3] = {mk(h[2], h[3]), mk(h[4], h[5]), mk(h[6], h[7])};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) V[a][b] = mk(Real(a == b ? 1 : 0), Real(0));
    const Real scale2 = dg[0] * dg[0] + dg[1] * dg[1] + dg[2] * dg[2] +
                        Real(2) * (o[0].r * o[0].r + o[0].i * o[0].i + o[1].r * o[1].r +
                                   o[1].i * o[1].i + o[2].r * o[2].r + o[2].i * o[2].i);
    // cyclic sweeps until the off-diagonal part is below the tolerance; the
    // first sweep is written out so that it starts from the constant V = I
    auto converged = [&]() {
        const Real off2 = o[0].r * o[0].r + o[0].i * o[0].i + o[1].r * o[1].r + o[1].i * o[1].i +
                          o[2].r * o[2].r + o[2].i * o[2].i;
        return !(off2 > JacobiTol<Real>::rel2 * scale2);
    };
    if (converged()) return;
    {
        // the first sweep from V = I, with its structural zeros and real
        // entries written out (x * 0 is not folded in IEEE arithmetic)
        Real c1, c2, c3;
        cx<Real> s1, s2, s3;
        jacobi_angles<Real, 0, 1>(dg, o, &c1, &s1); // V = [[c1, s1, 0], [-s1*, c1, 0], [0, 0, 1]]
        jacobi_angles<Real, 0, 2, 1>(dg, o, &c2, &s2); // columns 0 and 2
        const cx<Real> m1 = mk(-s1.r, s1.i); // -conj(s1)
        const Real v00 = c2 * c1;
        const cx<Real> v10 = c2 * m1, v02 = c1 * s2;
        const cx<Real> v12 = m1 * s2, v20 = mk(-s2.r, s2.i);
        // V = [[v00, s1, v02], [v10, c1, v12], [v20, 0, c2]]
        jacobi_angles<Real, 1, 2, 2>(dg, o, &c3, &s3); // columns 1 and 2
        const cx<Real> s3c = cj(s3);
        V[0][0] = mk(v00, Real(0));
        V[1][0] = v10;
        V[2][0] = v20;
        V[0][1] = cfma(neg(s3c), v02, c3 * s1);
        V[0][2] = cfma(s3, s1, c3 * v02);
        V[1][1] = mk(fma_r(-s3c.r, v12.r, fma_r(s3c.i, v12.i, c3 * c1)), fma_r(-s3c.r, v12.i, -(s3c.i * v12.r)));
        V[1][2] = rfma(c1, s3, c3 * v12);
        V[2][1] = mk(-(c2 * s3c.r), -(c2 * s3c.i));
        V[2][2] = mk(c3 * c2, Real(0));
    }
    for (int sweep = 1; sweep < JacobiTol<Real>::sweeps; ++sweep) {
        if (converged()) break;
        jacobi_rot<Real, 0, 1, 2>(dg, o, V);
        jacobi_rot<Real, 0, 2, 1>(dg, o, V);
        jacobi_rot<Real, 1, 2, 2>(dg, o, V);
    }
}

template <typename Real>
__host__ __device__ __forceinline__ void apply3(const Real *dg, const cx<Real> (*V)[3], StepLen<Real> dl, const Real *t,
                                                Real *out)
{
    // T: real diagonal Td, off-diagonal To[a][b] (a != b; To[b][a] = conj To[a][b])
    const Real Td[3] = {t[0], t[1], -(t[0] + t[1])};
    const cx<Real> To[3][3] = {{mk(Real(0), Real(0)), mk(t[2], t[3]), mk(t[4], t[5])},
                               {mk(t[2], -t[3]), mk(Real(0), Real(0)), mk(t[6], t[7])},
                               {mk(t[4], -t[5]), mk(t[6], -t[7]), mk(Real(0), Real(0))}};
    // W = T V, the diagonal term as real x complex
    cx<Real> W[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
            W[a][k] = cfma(To[a][b2], V[b2][k], cfma(To[a][b1], V[b1][k], Td[a] * V[a][k]));
        }
    // R = V^dagger W (Hermitian): diag real, upper entries
    Real Rd[3];
    cx<Real> Ro[3]; // (0,1), (0,2), (1,2)
#pragma unroll
    for (int j = 0; j < 3; ++j)
        Rd[j] = V[0][j].r * W[0][j].r + V[0][j].i * W[0][j].i + V[1][j].r * W[1][j].r +
                V[1][j].i * W[1][j].i + V[2][j].r * W[2][j].r + V[2][j].i * W[2][j].i;
    Ro[0] = cfmac(W[2][1], V[2][0], cfmac(W[1][1], V[1][0], mulc(W[0][1], V[0][0])));
    Ro[1] = cfmac(W[2][2], V[2][0], cfmac(W[1][2], V[1][0], mulc(W[0][2], V[0][0])));
    Ro[2] = cfmac(W[2][2], V[2][1], cfmac(W[1][2], V[1][1], mulc(W[0][2], V[0][1])));
    // phases exp(-i (lam_j - lam_k) dl) on the upper entries; the (0,2) phase
    // is the product of the (0,1) and (1,2) ones (two sine-cosine pairs, not three)
    {
        Real s01, c01, s12, c12;
        phase_sincos(dg[0] - dg[1], dl, &s01, &c01);
        phase_sincos(dg[1] - dg[2], dl, &s12, &c12);
        const cx<Real> e01 = mk(c01, -s01), e12 = mk(c12, -s12);
        Ro[0] = Ro[0] * e01;
        Ro[1] = Ro[1] * (e01 * e12);
        Ro[2] = Ro[2] * e12;
    }
    const cx<Real> Rm[3][3] = {{mk(Real(0), Real(0)), Ro[0], Ro[1]},
                               {cj(Ro[0]), mk(Real(0), Real(0)), Ro[2]},
                               {cj(Ro[1]), cj(Ro[2]), mk(Real(0), Real(0))}};
    // Z = V R' (the diagonal of R' real), T' = Z V^dagger
    cx<Real> Z[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int j1 = k == 0 ? 1 : 0, j2 = k == 2 ? 1 : 2;
            Z[a][k] = cfma(V[a][j2], Rm[j2][k], cfma(V[a][j1], Rm[j1][k], Rd[k] * V[a][k]));
        }
    Real o00 = Z[0][0].r * V[0][0].r + Z[0][0].i * V[0][0].i + Z[0][1].r * V[0][1].r +
               Z[0][1].i * V[0][1].i + Z[0][2].r * V[0][2].r + Z[0][2].i * V[0][2].i;
    Real o11 = Z[1][0].r * V[1][0].r + Z[1][0].i * V[1][0].i + Z[1][1].r * V[1][1].r +
               Z[1][1].i * V[1][1].i + Z[1][2].r * V[1][2].r + Z[1][2].i * V[1][2].i;
    cx<Real> o01 = cfmac(Z[0][2], V[1][2], cfmac(Z[0][1], V[1][1], mulc(Z[0][0], V[1][0])));
    cx<Real> o02 = cfmac(Z[0][2], V[2][2], cfmac(Z[0][1], V[2][1], mulc(Z[0][0], V[2][0])));
    cx<Real> o12 = cfmac(Z[1][2], V[2][2], cfmac(Z[1][1], V[2][1], mulc(Z[1][0], V[2][0])));
    // keep the result exactly traceless in the packed form: t3 is implied
    out[0] = o00;
    out[1] = o11;
    out[2] = o01.r;
    out[3] = o01.i;
    out[4] = o02.r;
    out[5] = o02.i;
    out[6] = o12.r;
    out[7] = o12.i;
}

template <typename Real>
__host__ __device__ __forceinline__ void prop3(const Real *h, StepLen<Real> dl, const Real *t, Real *out)
{
    Real dg[3];
    cx<Real> V[3][3];
    eig3<Real>(h, dg, V);
    apply3<Real>(dg, V, dl, t, out);
}

// ---------------------------------------------------------------- dispatch
template <int NF, typename Real>
__host__ __device__ __forceinline__ void comm(const Real *h, const Real *t, Real *d)
{
    if constexpr (NF == 2) comm2<Real>(h, t, d);
    else comm3<Real>(h, t, d);
}
template <int NF, typename Real>
__host__ __device__ __forceinline__ void prop(const Real *h, StepLen<Real> dl, const Real *t, Real *out)
{
    if constexpr (NF == 2) prop2<Real>(h, dl, t, out);
    else prop3<Real>(h, dl, t, out);
}

// Two propagations of the same T under the same H for two path lengths
// (one eigendecomposition / one Bloch-vector rotation axis for both).
template <int NF, typename Real>
__host__ __device__ __forceinline__ void prop_pair(const Real *h, StepLen<Real> dl1, StepLen<Real> dl2, const Real *t,
                                                   Real *out1, Real *out2)
{
    if constexpr (NF == 2) {
        Real lam, rl;
        rotation_lambda(h, &lam, &rl);
        Real w[3], q[3];
        w[0] = h[2] * t[1] - h[1] * t[2];
        w[1] = h[0] * t[2] - t[0] * h[2];
        w[2] = t[0] * h[1] - h[0] * t[1];
        q[0] = h[2] * w[1] - h[1] * w[2];
        q[1] = h[0] * w[2] - w[0] * h[2];
        q[2] = w[0] * h[1] - h[0] * w[1];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const StepLen<Real> dl = i ? dl2 : dl1;
            Real sn, cs, sig;
            rotation_phase(lam, rl, dl, &sn, &cs, &sig);
            Real c1 = Real(2) * sig * cs, c2 = Real(2) * sig * sig;
            Real *o = i ? out2 : out1;
#pragma unroll
            for (int k = 0; k < 3; ++k) o[k] = t[k] + c1 * w[k] + c2 * q[k];
        }
    } else {
        Real dg[3];
        cx<Real> V[3][3];
        eig3<Real>(h, dg, V);
        apply3<Real>(dg, V, dl1, t, out1);
        apply3<Real>(dg, V, dl2, t, out2);
    }
}

// Traceless components of rho_nu - conj(rho_nubar): conjugation flips the
// sign of every imaginary part.
template <int NF, typename Real>
__host__ __device__ __forceinline__ void nu_minus_conj_nubar(const Real *tn, const Real *tb, Real *d)
{
    if constexpr (NF == 2) {
        d[0] = tn[0] - tb[0];
        d[1] = tn[1] - tb[1];
        d[2] = tn[2] + tb[2];
    } else {
        d[0] = tn[0] - tb[0];
        d[1] = tn[1] - tb[1];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            d[2 + 2 * k] = tn[2 + 2 * k] - tb[2 + 2 * k];
            d[3 + 2 * k] = tn[3 + 2 * k] + tb[3 + 2 * k];
        }
    }
}

// Hamiltonians of the two species of one (u, E) pair (traceless comps):
//   H_nu = H_vac + A P_e + G,   H_nubar = H_vac - A P_e - conj(G)
// P_e = diag(1, 0[, 0]) has traceless part (1/2)(1,-1) or (2/3, -1/3, -1/3).
template <int NF, typename Real>
__host__ __device__ __forceinline__ void hamiltonians(const Real *hv, Real A, const Real *g, Real *hn, Real *hb)
{
    constexpr int S = Comp<NF>::S;
#pragma unroll
    for (int k = 0; k < S; ++k) hn[k] = hv[k] + g[k];
    // conj(G) flips the imaginary parts: those of hb take +g
    if constexpr (NF == 2) {
        hb[0] = hv[0] - g[0];
        hb[1] = hv[1] - g[1];
        hb[2] = hv[2] + g[2];
        const Real a = Real(0.5) * A;
        hn[0] += a;
        hb[0] -= a;
    } else {
        hb[0] = hv[0] - g[0];
        hb[1] = hv[1] - g[1];
#pragma unroll
        for (int k = 2; k < S; k += 2) {
            hb[k] = hv[k] - g[k];
            hb[k + 1] = hv[k + 1] + g[k + 1];
        }
        const Real a1 = A * Real(2) / Real(3), a2 = A / Real(3);
        hn[0] += a1;
        hn[1] -= a2;
        hb[0] -= a1;
        hb[1] += a2;
    }
}

// tr(T^2) of a traceless Hermitian matrix T in packed form (2(a^2 + x^2 + y^2)
// in two flavors; with the trace fixed, tr(rho^2) and |P| follow from it).
template <int NF, typename Real>
__host__ __device__ __forceinline__ Real purity(const Real *t)
{
    if constexpr (NF == 2) {
        return Real(2) * (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    } else {
        const Real t3 = -(t[0] + t[1]);
        Real q = t[0] * t[0] + t[1] * t[1] + t3 * t3;
#pragma unroll
        for (int c = 2; c < 8; ++c) q += Real(2) * t[c] * t[c];
        return q;
    }
}

// Scale the traceless part back to the initial tr(T^2) = ref (the exact flow
// conserves it; the FP32 update lets it drift).
template <int NF, typename Real>
__host__ __device__ __forceinline__ void renormalise(Real *t, Real ref)
{
    constexpr int S = Comp<NF>::S;
    const Real q = purity<NF, Real>(t);
    if (q > Real(0) && ref > Real(0)) {
        const Real f = sqrt_r(ref / q);
#pragma unroll
        for (int c = 0; c < S; ++c) t[c] *= f;
    }
}

} // namespace xf

// float-float numbers (the XF_FP32X2 per-bin arithmetic) for the templates above
#include "xf_ff.cuh"
