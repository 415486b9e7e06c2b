// Host check of the float-float arithmetic (xf_ff.cuh) and of the library's
// 3x3 and 2x2 propagators run on it (the XF_FP32X2 per-bin arithmetic),
// against long double and against the same templates in double.  Prints the
// largest errors found over seeded inputs:
//   add_rel, mul_rel, fma_rel: relative error of +, x and a b + c
//     (operands of random sign and of magnitudes 2^-40 .. 2^40);
//   rsqrt_rel: relative error of rsqrt_r over 2^-60 .. 2^60;
//   prop3_abs, prop2_abs: max |T'_ff - T'_double| over the packed components
//     for |T| <= 1, Hamiltonians with eigenvalue spreads 1e-3 .. 1e4 and
//     path lengths 0.01 .. 0.3 (phases up to 3e3 rad);
//   phase_over: the phase sine-cosine's largest error in units of the
//     float-float rounding of the phase itself (|phase| 2^-47 + 1e-15).
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "xf_math.cuh"

using namespace xf;

static uint64_t g_s = 0x2545F4914F6CDD1Dull;
static double uniform01()
{
    // SplitMix64 (Steele, Lea & Flood 2014)
    uint64_t z = (g_s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}
static double signed_mag(int lo, int hi)
{
    const double m = std::ldexp(1.0 + uniform01(), lo + (int)((hi - lo) * uniform01()));
    return uniform01() < 0.5 ? -m : m;
}
static long double exact(ff a) { return (long double)a.hi + (long double)a.lo; }
static ff round_ff(long double x)
{
    const float h = (float)x;
    return ff(h, (float)(x - (long double)h));
}

int main()
{
    double add_rel = 0, mul_rel = 0, fma_rel = 0, rsqrt_rel = 0, prop3_abs = 0, prop2_abs = 0;
    for (int i = 0; i < 1000000; ++i) {
        const ff a = round_ff(signed_mag(-40, 40)), b = round_ff(signed_mag(-40, 40)), c = round_ff(signed_mag(-40, 40));
        // same-sign and opposite-sign sums: error relative to |a| + |b|
        const long double s = exact(a) + exact(b);
        add_rel = std::fmax(add_rel, (double)(std::fabs(exact(a + b) - s) / (std::fabs(exact(a)) + std::fabs(exact(b)))));
        const long double p = exact(a) * exact(b);
        mul_rel = std::fmax(mul_rel, (double)(std::fabs(exact(a * b) - p) / std::fabs(p)));
        const long double f = p + exact(c);
        fma_rel = std::fmax(fma_rel, (double)(std::fabs(exact(fma_r(a, b, c)) - f) / (std::fabs(p) + std::fabs(exact(c)))));
        const double x = std::ldexp(1.0 + uniform01(), -60 + (int)(120 * uniform01()));
        const ff r = rsqrt_r(ff(x));
        rsqrt_rel = std::fmax(rsqrt_rel, (double)std::fabs(exact(r) * std::sqrt((long double)x) - 1.0L));
    }
    for (int i = 0; i < 200000; ++i) {
        const double scale = std::pow(10.0, -3.0 + 7.0 * uniform01());
        const double dl = 0.01 + 0.29 * uniform01();
        double h[8], t[8];
        for (int k = 0; k < 8; ++k) h[k] = scale * (2.0 * uniform01() - 1.0) * (k < 2 ? 1.0 : std::pow(10.0, -4.0 * uniform01()));
        for (int k = 0; k < 8; ++k) t[k] = 0.5 * (2.0 * uniform01() - 1.0) * (k < 2 ? 1.0 : 1e-2);
        ff hf[8], tf[8], of[8];
        double hd[8], td[8], od[8];
        for (int k = 0; k < 8; ++k) {
            hf[k] = ff(h[k]);
            tf[k] = ff(t[k]);
            hd[k] = to_double(hf[k]);
            td[k] = to_double(tf[k]);
        }
        prop3<ff>(hf, make_step_len(dl, (ff *)nullptr), tf, of);
        prop3<double>(hd, make_step_len(dl, (double *)nullptr), td, od);
        for (int k = 0; k < 8; ++k) prop3_abs = std::fmax(prop3_abs, std::fabs(to_double(of[k]) - od[k]));
        prop2<ff>(hf, make_step_len(dl, (ff *)nullptr), tf, of);
        prop2<double>(hd, make_step_len(dl, (double *)nullptr), td, od);
        for (int k = 0; k < 3; ++k) prop2_abs = std::fmax(prop2_abs, std::fabs(to_double(of[k]) - od[k]));
    }
    // the phase sine-cosine: error relative to the float-float rounding of
    // the phase itself (|phase| 2^-47, plus 1e-15), phases 1e-6 .. 2e4 rad
    double phase_over = 0;
    for (int i = 0; i < 1000000; ++i) {
        const double dl = 0.001 + 0.3 * uniform01();
        const double mag = std::ldexp(1.0, -20 + (int)(34 * uniform01())) * (1.0 + uniform01());
        const ff lam((uniform01() < 0.5 ? -mag : mag) / dl);
        ff s, c;
        phase_sincos(lam, make_step_len(dl, (ff *)nullptr), &s, &c);
        const long double ph = exact(lam) * (long double)dl;
        const long double e = std::fmax(std::fabs(std::sin(ph) - exact(s)), std::fabs(std::cos(ph) - exact(c)));
        phase_over = std::fmax(phase_over, (double)(e / (std::fabs(ph) * 7.1e-15L + 1e-15L)));
    }
    std::printf("add_rel %.3e\nmul_rel %.3e\nfma_rel %.3e\nrsqrt_rel %.3e\nprop3_abs %.3e\nprop2_abs %.3e\n"
                "phase_over %.3f\n", add_rel, mul_rel, fma_rel, rsqrt_rel, prop3_abs, prop2_abs, phase_over);
    return 0;
}
