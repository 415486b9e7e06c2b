// Host check of the FP32 phase sine-cosine (phase_sincos in xf_math.cuh):
// Cody-Waite reduction by pi/2 of a float-float phase, Taylor polynomials on
// [-pi/4, pi/4], quadrant swap and signs.  Prints the largest absolute error
// of sin and cos against the double-precision library's values of the exact
// phase lam * (hi + lo), over seeded phases of every magnitude the kernels
// meet (a few microradians to 2^16 rad, both signs, and the quadrant
// boundaries), and the worst case found.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "xf_math.cuh"

using namespace xf;

static uint64_t g_s = 0x9E3779B97F4A7C15ull;
static double uniform01()
{
    // SplitMix64 (Steele, Lea & Flood 2014)
    uint64_t z = (g_s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

int main()
{
    double worst_s = 0.0, worst_c = 0.0, at = 0.0;
    long long n = 0;
    auto check = [&](float lam, double dl) {
        const StepLen<float> d = make_step_len(dl, (float *)nullptr);
        float s, c;
        phase_sincos(lam, d, &s, &c);
        const long double ph = (long double)lam * ((long double)d.hi + (long double)d.lo);
        const double es = std::fabs((double)(std::sin(ph) - (long double)s));
        const double ec = std::fabs((double)(std::cos(ph) - (long double)c));
        if (es > worst_s || ec > worst_c) at = (double)ph;
        if (es > worst_s) worst_s = es;
        if (ec > worst_c) worst_c = ec;
        ++n;
    };
    // phases over 2^-20 .. 2^16 rad, log-uniform, both signs, seeded path lengths
    for (int i = 0; i < 2000000; ++i) {
        const double mag = std::ldexp(1.0, -20 + (int)(36 * uniform01())) * (1.0 + uniform01());
        const double dl = 0.001 + 0.1 * uniform01();
        const float lam = (float)((uniform01() < 0.5 ? -mag : mag) / dl);
        check(lam, dl);
    }
    // near the quadrant boundaries k pi/4 (octant edges of the polynomial)
    for (int k = -4000; k <= 4000; ++k)
        for (int j = -3; j <= 3; ++j) {
            const double dl = 0.0495;
            const float lam = (float)((k * 0.78539816339744830962 + j * 1e-6) / dl);
            check(lam, dl);
        }
    std::printf("samples %lld\nmax_abs_err_sin %.3e\nmax_abs_err_cos %.3e\nworst_phase %.9g\n", n, worst_s, worst_c, at);
    return 0;
}
