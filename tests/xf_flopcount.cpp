// xf_flopcount.cpp -- counts the floating-point work per bin-step of the
// library's per-bin formulas, the figures behind bench.py's roofline.
//
// The per-bin templates of the CUDA path (xf_math.cuh, xf_psi.cuh) are
// __host__ __device__ and templated on the number type.  Here they run on
// the host with a counting type, Cnt, in the order in which the kernels'
// per-pair loops call them (stage_tile, psi_stage_tile and the three stages
// of the error-controlled step): per (angle, energy) pair and stage the nu-nu
// term G = mu (M0 - cos M1), the two Hamiltonians, the update of the neutrino
// and the antineutrino matrix, the averages, and the pair's contribution to
// the next stage's sums.  Per-angle and per-problem work (tables, moment
// totals, barriers) is not per-bin work and is left out.
//
// Counting rules: + - * / and sqrt count 1 each, a fused multiply-add 2, a
// reciprocal square root 1; sine-cosine pairs, comparisons, fabs and
// negation count nothing.  An operation with a structural zero (a literal 0
// of the source: a product with it, a sum with it) is no work of the method
// and is dropped, even where IEEE rules keep a compiler from folding it.
// The Jacobi eigensolver's sweep count depends on the Hamiltonian, so the
// three-flavor figures are given at a stated sweep count, taken from
// Hamiltonians of the regime in question (matter-dominated: two sweeps;
// vacuum-dominated: three).
//
// Build (host only): g++ -O1 -std=c++17 -I<cuda>/include -I<csrc> xf_flopcount.cpp
// Output: one "key value" line per figure.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

// ---- the counting number type ------------------------------------------------
static long long g_flops = 0, g_rsqrt = 0;

struct Cnt {
    double v = 0.0;
    bool z = false; // a structural (literal) zero
    Cnt() = default;
    // constants written in the source: a literal 0 is structural
    Cnt(double x) : v(x), z(x == 0.0) {}
    Cnt(int x) : v(x), z(x == 0) {}
    // a value computed or read at run time (never structural)
    static Cnt in(double x)
    {
        Cnt c;
        c.v = x;
        c.z = false;
        return c;
    }
};
static inline Cnt val(double x) { return Cnt::in(x); }

static inline Cnt operator+(Cnt a, Cnt b)
{
    if (a.z) return b;
    if (b.z) return a;
    ++g_flops;
    return val(a.v + b.v);
}
static inline Cnt operator-(Cnt a) { return a.z ? a : val(-a.v); }
static inline Cnt operator-(Cnt a, Cnt b)
{
    if (b.z) return a;
    if (a.z) return -b;
    ++g_flops;
    return val(a.v - b.v);
}
static inline Cnt operator*(Cnt a, Cnt b)
{
    if (a.z || b.z) return Cnt(0.0);
    ++g_flops;
    return val(a.v * b.v);
}
static inline Cnt operator/(Cnt a, Cnt b)
{
    if (a.z) return Cnt(0.0);
    ++g_flops;
    return val(a.v / b.v);
}
static inline Cnt &operator+=(Cnt &a, Cnt b) { return a = a + b; }
static inline Cnt &operator-=(Cnt &a, Cnt b) { return a = a - b; }
static inline Cnt &operator*=(Cnt &a, Cnt b) { return a = a * b; }
static inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
static inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
static inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
static inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
static inline Cnt fabs(Cnt a) { return a.z ? a : val(std::fabs(a.v)); }
static inline Cnt abs_r(Cnt a) { return fabs(a); }
static inline Cnt fmax(Cnt a, Cnt b) { return val(std::fmax(a.v, b.v)); }

#include "xf_math.cuh"

namespace xf {
template <> struct StepLen<Cnt> {
    Cnt v;
};
template <> struct JacobiTol<Cnt> {
    static constexpr double rel2 = JacobiTol<double>::rel2;
    static constexpr int sweeps = JacobiTol<double>::sweeps;
};
} // namespace xf

// The templates call these unqualified; with Cnt arguments argument-dependent
// lookup finds them here, in Cnt's (the global) namespace.
static inline Cnt step_len_value(xf::StepLen<Cnt> d) { return d.v; }
static inline Cnt sqrt_r(Cnt x)
{
    if (x.z) return x;
    ++g_flops;
    return val(std::sqrt(x.v));
}
static inline Cnt rsqrt_r(Cnt x)
{
    ++g_flops;
    ++g_rsqrt;
    return val(1.0 / std::sqrt(x.v));
}
static inline Cnt fma_r(Cnt a, Cnt b, Cnt c)
{
    if (a.z || b.z) return c;
    if (c.z) return a * b;
    g_flops += 2;
    return val(std::fma(a.v, b.v, c.v));
}
// the phase lam * dl is work; its sine-cosine pair is not counted
static inline void phase_sincos(Cnt lam, xf::StepLen<Cnt> d, Cnt *s, Cnt *c)
{
    const Cnt ph = lam * d.v;
    *s = val(std::sin(ph.v));
    *c = val(std::cos(ph.v));
}

#include "xf_psi.cuh"

using namespace xf;
using R = Cnt;

// ---- inputs of the workload's regimes -----------------------------------------
// Traceless packed Hamiltonian pieces and states with every entry non-zero,
// so that no run-time value is mistaken for a structural zero.
template <int NF> struct Regime {
    static constexpr int S = Comp<NF>::S;
    R hv[S], M0[S], M1[S], t[2][S], A, gam, wa, wb, kap, cy, cb, dl, half, trace;
};

// Three flavors: the vacuum term of the 1000 x 200 bulb workload at 20 MeV
// (PMNS angles 0.59 / 0.15 / 0.72, dm2 7.5e-5 / 2.4e-3 eV^2, in km^-1), the
// nu-nu term and a state with entries of order 1e-3 .. 1; `matter` is the
// potential A (km^-1): 2.4e4 at 30 km on the r^-3 profile (matter-dominated,
// two Jacobi sweeps), 0 far out (vacuum-dominated).
static Regime<3> regime3(double matter, double mu_scale)
{
    Regime<3> g;
    const double hv[8] = {-0.0508, -0.0139, 0.0122, 0.0, 0.0309, 0.0, 0.0645, 0.0};
    // the vacuum term of a CP-conserving H is real: its imaginary parts are
    // written as run-time zeros (they are table entries, not literals)
    for (int c = 0; c < 8; ++c) g.hv[c] = val(hv[c]);
    const double m0[8] = {0.31, -0.12, 0.021, -0.013, 0.017, 0.009, -0.011, 0.006};
    const double m1[8] = {0.17, -0.07, 0.012, -0.008, 0.010, 0.005, -0.007, 0.004};
    for (int c = 0; c < 8; ++c) {
        g.M0[c] = val(mu_scale * m0[c]);
        g.M1[c] = val(mu_scale * m1[c]);
    }
    const double tn[8] = {0.33, -0.11, 1.1e-3, -0.7e-3, 0.9e-3, 0.4e-3, -0.6e-3, 0.8e-3};
    const double tb[8] = {0.21, -0.07, 0.8e-3, 0.5e-3, -0.6e-3, 0.9e-3, 0.3e-3, -0.4e-3};
    for (int c = 0; c < 8; ++c) {
        g.t[0][c] = val(tn[c]);
        g.t[1][c] = val(tb[c]);
    }
    g.A = val(matter);
    g.gam = val(0.83);
    g.wa = val(2.1e-4);
    g.wb = val(1.7e-4);
    g.kap = val(1.21);
    g.cy = val(0.025);
    g.cb = val(0.0083);
    g.dl = val(0.0503);
    g.half = val(0.0251);
    g.trace = val(1.37);
    return g;
}

static Regime<2> regime2()
{
    Regime<2> g;
    const double hv[3] = {-0.119, 0.012, 0.0};
    for (int c = 0; c < 3; ++c) g.hv[c] = val(hv[c]);
    const double m0[3] = {0.41, 0.031, -0.017}, m1[3] = {0.23, 0.017, -0.009};
    for (int c = 0; c < 3; ++c) {
        g.M0[c] = val(m0[c]);
        g.M1[c] = val(m1[c]);
    }
    const double tn[3] = {0.29, 1.3e-3, -0.8e-3}, tb[3] = {0.19, 0.7e-3, 0.5e-3};
    for (int c = 0; c < 3; ++c) {
        g.t[0][c] = val(tn[c]);
        g.t[1][c] = val(tb[c]);
    }
    g.A = val(0.0);
    g.gam = val(0.83);
    g.wa = val(2.1e-4);
    g.wb = val(1.7e-4);
    g.kap = val(1.21);
    g.cy = val(0.005);
    g.cb = val(0.0017);
    g.dl = val(0.0101);
    g.half = val(0.0050);
    g.trace = val(1.37);
    return g;
}

// ---- per-pair pieces, in the kernels' order ------------------------------------
template <int NF> static void nu_nu_term(const Regime<NF> &g, R *gg)
{
    for (int c = 0; c < Comp<NF>::S; ++c) gg[c] = g.M0[c] - g.gam * g.M1[c];
}
// accum: the weighted sums of one pair's stage output (xf_run.cuh)
template <int NF> static void accumulate(const Regime<NF> &g, const R *tn, const R *tb, R *m)
{
    constexpr int S = Comp<NF>::S;
    R d[S];
    nu_minus_conj_nubar<NF, R>(tn, tb, d);
    for (int c = 0; c < S; ++c) {
        m[c] += g.wa * d[c];
        m[S + c] += g.wb * d[c];
    }
}
template <int NF> static void fresh_sums(R *m)
{
    for (int c = 0; c < 2 * Comp<NF>::S; ++c) m[c] = val(1e-3 * (c + 1)); // running sums, not literals
}

// One predictor-corrector step of one pair (two stages), rho form.
template <int NF> static long long exph_pair(const Regime<NF> &g)
{
    constexpr int S = Comp<NF>::S;
    const long long f0 = g_flops;
    const StepLen<R> dl{g.dl};
    for (int st = 0; st < 2; ++st) {
        R gg[S], hn[S], hb[S], m[2 * S], on[S], ob[S];
        fresh_sums<NF>(m);
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R pr[S];
            prop<NF, R>(s == 0 ? hn : hb, dl, g.t[s], pr);
            R *o = s == 0 ? on : ob;
            if (st == 0)
                for (int c = 0; c < S; ++c) o[c] = pr[c];
            else
                for (int c = 0; c < S; ++c) o[c] = R(0.5) * (g.t[1 - s][c] + pr[c]);
        }
        accumulate<NF>(g, on, ob, m);
    }
    return g_flops - f0;
}

// One RK4 step of one pair (four stages), rho form.
template <int NF> static long long rk4_pair(const Regime<NF> &g)
{
    constexpr int S = Comp<NF>::S;
    const long long f0 = g_flops;
    for (int st = 0; st < 4; ++st) {
        R gg[S], hn[S], hb[S], m[2 * S], on[S], ob[S];
        fresh_sums<NF>(m);
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R kk[S], bb[S];
            const R *y = g.t[s], *rn = g.t[1 - s];
            comm<NF, R>(s == 0 ? hn : hb, y, kk);
            for (int c = 0; c < S; ++c) kk[c] *= g.kap;
            if (st == 0)
                for (int c = 0; c < S; ++c) bb[c] = y[c] + g.cb * kk[c];
            else
                for (int c = 0; c < S; ++c) {
                    bb[c] = rn[c];
                    bb[c] += g.cb * kk[c];
                }
            R *o = s == 0 ? on : ob;
            if (st < 3)
                for (int c = 0; c < S; ++c) o[c] = rn[c] + g.cy * kk[c];
            else
                for (int c = 0; c < S; ++c) o[c] = bb[c];
        }
        accumulate<NF>(g, on, ob, m);
    }
    return g_flops - f0;
}

// max_entry of the error-controlled kernel (xf_adapt.cuh)
template <int NF> static R max_entry_count(const R *d)
{
    if constexpr (NF == 2) {
        return fmax(fabs(d[0]), sqrt_r(d[1] * d[1] + d[2] * d[2]));
    } else {
        R m = fmax(fmax(fabs(d[0]), fabs(d[1])), fabs(d[0] + d[1]));
        m = fmax(m, sqrt_r(d[2] * d[2] + d[3] * d[3]));
        m = fmax(m, sqrt_r(d[4] * d[4] + d[5] * d[5]));
        return fmax(m, sqrt_r(d[6] * d[6] + d[7] * d[7]));
    }
}

// One attempt of the error-controlled step for one pair: stages A, B, C.
template <int NF> static long long adaptive_pair(const Regime<NF> &g)
{
    constexpr int S = Comp<NF>::S;
    const long long f0 = g_flops;
    const StepLen<R> dlf{g.dl}, dlh{g.half};
    R gg[S], hn[S], hb[S];
    { // A: H0 -> full and half steps from one eigendecomposition; two sets of sums
        R m[4 * S], fn[S], fb[S], hn_[S], hb_[S];
        fresh_sums<NF>(m);
        fresh_sums<NF>(m + 2 * S);
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s)
            prop_pair<NF, R>(s ? hb : hn, dlf, dlh, g.t[s], s ? fb : fn, s ? hb_ : hn_);
        accumulate<NF>(g, fn, fb, m);
        accumulate<NF>(g, hn_, hb_, m + 2 * S);
    }
    { // B: H1 -> coarse result; H2 -> fine path's second half
        R m[2 * S], o5n[S], o5b[S];
        fresh_sums<NF>(m);
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R r3[S], r2[S];
            prop<NF, R>(s ? hb : hn, dlf, g.t[s], r3);
            for (int c = 0; c < S; ++c) r2[c] = R(0.5) * (g.t[1 - s][c] + r3[c]);
        }
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) prop<NF, R>(s ? hb : hn, dlh, g.t[s], s ? o5b : o5n);
        accumulate<NF>(g, o5n, o5b, m);
    }
    { // C: H3 -> fine result, the error against the coarse one, sums of the coarse result
        R m[2 * S];
        fresh_sums<NF>(m);
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R r6[S], d[S];
            prop<NF, R>(s ? hb : hn, dlf, g.t[s], r6);
            for (int c = 0; c < S; ++c) d[c] = g.t[s][c] - R(0.5) * (g.t[1 - s][c] + r6[c]);
            R e = max_entry_count<NF>(d) / fabs(g.trace);
            (void)e;
        }
        accumulate<NF>(g, g.t[0], g.t[1], m);
    }
    return g_flops - f0;
}

// Wavefunction form: one wavefunction per initial flavor, rho's traceless part
// rebuilt from them for the sums (psi_stage_tile).
template <int NF> static void psi_state(R *x)
{
    constexpr int SS = PsiComp<NF>::SS;
    for (int c = 0; c < SS; ++c) x[c] = val(0.05 + 0.9 / (c + 1)); // every component non-zero
}
template <int NF> static long long psi_pair(const Regime<NF> &g, bool rk4)
{
    constexpr int S = Comp<NF>::S, SS = PsiComp<NF>::SS;
    const long long f0 = g_flops;
    const StepLen<R> dl{g.dl};
    R x[SS];
    psi_state<NF>(x);
    const R w0 = val(0.71), w1 = val(0.43);
    for (int st = 0; st < (rk4 ? 4 : 2); ++st) {
        R gg[S], hn[S], hb[S], m[2 * S], tr_[2][S];
        fresh_sums<NF>(m);
        nu_nu_term<NF>(g, gg);
        hamiltonians<NF, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R o[SS], tr;
            if (rk4) {
                R k[SS], bb[SS];
                rhs_psi<NF, R>(s == 0 ? hn : hb, g.kap, x, k);
                if (st == 0)
                    for (int c = 0; c < SS; ++c) bb[c] = x[c] + g.cb * k[c];
                else
                    for (int c = 0; c < SS; ++c) {
                        bb[c] = x[c];
                        bb[c] += g.cb * k[c];
                    }
                if (st < 3)
                    for (int c = 0; c < SS; ++c) o[c] = x[c] + g.cy * k[c];
                else
                    for (int c = 0; c < SS; ++c) o[c] = bb[c];
            } else {
                R u[SS];
                prop_psi<NF, R>(s == 0 ? hn : hb, dl, x, u);
                if (st == 0)
                    for (int c = 0; c < SS; ++c) o[c] = u[c];
                else
                    for (int c = 0; c < SS; ++c) o[c] = R(0.5) * (x[c] + u[c]);
            }
            psi_rho<NF, R>(o, w0, w1, tr_[s], &tr);
        }
        accumulate<NF>(g, tr_[0], tr_[1], m);
    }
    return g_flops - f0;
}

// The extended bulb model (Eq. 3.18, four moments): stage_tile with NMOM = 4,
// per pair and stage two more terms in G and two more running sums.
static long long exph_azimuth_pair(const Regime<2> &g)
{
    constexpr int S = 3;
    const long long f0 = g_flops;
    const StepLen<R> dl{g.dl};
    const R g2 = val(0.31), g3 = val(-0.27), M2[S] = {val(0.021), val(-0.013), val(0.004)},
            M3[S] = {val(0.017), val(0.009), val(-0.006)}, wc = val(1.1e-4), wd = val(0.9e-4);
    for (int st = 0; st < 2; ++st) {
        R gg[S], hn[S], hb[S], m[4 * S], on[S], ob[S], d[S];
        for (int c = 0; c < 4 * S; ++c) m[c] = val(1e-3 * (c + 1));
        nu_nu_term<2>(g, gg);
        for (int c = 0; c < S; ++c) gg[c] = gg[c] - g2 * M2[c] - g3 * M3[c];
        hamiltonians<2, R>(g.hv, g.A, gg, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R pr[S];
            prop<2, R>(s == 0 ? hn : hb, dl, g.t[s], pr);
            R *o = s == 0 ? on : ob;
            for (int c = 0; c < S; ++c) o[c] = st == 0 ? pr[c] : R(0.5) * (g.t[1 - s][c] + pr[c]);
        }
        nu_minus_conj_nubar<2, R>(on, ob, d); // accum4
        for (int c = 0; c < S; ++c) {
            m[c] += g.wa * d[c];
            m[S + c] += g.wb * d[c];
            m[2 * S + c] += wc * d[c];
            m[3 * S + c] += wd * d[c];
        }
    }
    return g_flops - f0;
}

// The cylinder model's per-bin update (xf_cyl.cuh): G comes per trajectory
// from the angle-pair sum (counted separately, per trajectory), so a pair
// takes the Hamiltonians, the update and a plain trajectory sum.
static long long exph_cylinder_pair(const Regime<2> &g)
{
    constexpr int S = 3;
    const long long f0 = g_flops;
    const StepLen<R> dl{g.dl};
    for (int st = 0; st < 2; ++st) {
        R hn[S], hb[S], on[S], ob[S], dd[S], d[S] = {val(1e-3), val(2e-3), val(3e-3)};
        hamiltonians<2, R>(g.hv, g.A, g.M0, hn, hb);
        for (int s = 0; s < 2; ++s) {
            R pr[S];
            prop<2, R>(s == 0 ? hn : hb, dl, g.t[s], pr);
            R *o = s == 0 ? on : ob;
            for (int c = 0; c < S; ++c) o[c] = st == 0 ? pr[c] : R(0.5) * (g.t[1 - s][c] + pr[c]);
        }
        nu_minus_conj_nubar<2, R>(on, ob, dd);
        for (int c = 0; c < S; ++c) d[c] += dd[c];
    }
    return g_flops - f0;
}

// Jacobi sweeps that eig3 took on a Hamiltonian (two reciprocal square roots
// per rotation, three rotations per sweep).
static int sweeps_of(const Regime<3> &g)
{
    R gg[8], hn[8], hb[8], dg[3];
    cx<R> V[3][3];
    nu_nu_term<3>(g, gg);
    hamiltonians<3, R>(g.hv, g.A, gg, hn, hb);
    const long long r0 = g_rsqrt;
    eig3<R>(hn, dg, V);
    return (int)((g_rsqrt - r0) / 6);
}

static long long prop3_count(const Regime<3> &g)
{
    R gg[8], hn[8], hb[8], out[8];
    nu_nu_term<3>(g, gg);
    hamiltonians<3, R>(g.hv, g.A, gg, hn, hb);
    const long long f0 = g_flops;
    prop<3, R>(hn, StepLen<R>{g.dl}, g.t[0], out);
    return g_flops - f0;
}

static long long eig3_count(const Regime<3> &g)
{
    R gg[8], hn[8], hb[8], dg[3];
    cx<R> V[3][3];
    nu_nu_term<3>(g, gg);
    hamiltonians<3, R>(g.hv, g.A, gg, hn, hb);
    const long long f0 = g_flops;
    eig3<R>(hn, dg, V);
    return g_flops - f0;
}

// Sweep counts of eig3 on traceless Hamiltonians read from a file of doubles,
// eight per Hamiltonian in the packed layout (t1, t2, Re/Im z12, z13, z23):
// prints the mean and the count for each number of sweeps.
static int sweep_histogram(const char *path)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return 1;
    double h[8];
    long long n = 0, hist[16] = {0};
    while (std::fread(h, sizeof(double), 8, f) == 8) {
        R hh[8], dg[3];
        cx<R> V[3][3];
        for (int c = 0; c < 8; ++c) hh[c] = val(h[c]);
        const long long r0 = g_rsqrt;
        eig3<R>(hh, dg, V);
        const int sw = (int)((g_rsqrt - r0) / 6);
        ++hist[sw < 15 ? sw : 15];
        ++n;
    }
    std::fclose(f);
    double mean = 0.0;
    for (int k = 0; k < 16; ++k) mean += k * (double)hist[k];
    std::printf("hamiltonians %lld\nmean_sweeps %.4f\n", n, n ? mean / n : 0.0);
    for (int k = 0; k < 16; ++k)
        if (hist[k]) std::printf("sweeps_%d %lld\n", k, hist[k]);
    return 0;
}

int main(int argc, char **argv)
{
    if (argc == 3 && std::strcmp(argv[1], "--sweeps") == 0) return sweep_histogram(argv[2]);
    const Regime<3> m3 = regime3(2.4e4, 1.0); // matter-dominated: two sweeps
    const Regime<3> v3 = regime3(0.0, 0.05);  // vacuum-dominated: three sweeps
    const Regime<2> g2 = regime2();
    std::printf("sweeps_matter %d\n", sweeps_of(m3));
    std::printf("sweeps_vacuum %d\n", sweeps_of(v3));
    std::printf("prop3 %lld\n", prop3_count(m3));
    std::printf("eig3_extra_sweep %lld\n", eig3_count(v3) - eig3_count(m3));
    // per bin-step (two bins, nu and nubar, per pair)
    std::printf("exph_3 %lld\n", exph_pair<3>(m3) / 2);
    std::printf("rk4_3 %lld\n", rk4_pair<3>(m3) / 2);
    std::printf("exph_2 %lld\n", exph_pair<2>(g2) / 2);
    std::printf("rk4_2 %lld\n", rk4_pair<2>(g2) / 2);
    std::printf("attempt_3 %lld\n", adaptive_pair<3>(m3) / 2);
    std::printf("attempt_2 %lld\n", adaptive_pair<2>(g2) / 2);
    std::printf("psi_exph_3 %lld\n", psi_pair<3>(m3, false) / 2);
    std::printf("psi_rk4_3 %lld\n", psi_pair<3>(m3, true) / 2);
    std::printf("psi_exph_2 %lld\n", psi_pair<2>(g2, false) / 2);
    std::printf("psi_rk4_2 %lld\n", psi_pair<2>(g2, true) / 2);
    std::printf("azimuth_exph_2 %lld\n", exph_azimuth_pair(g2) / 2);
    std::printf("cylinder_exph_2 %lld\n", exph_cylinder_pair(g2) / 2);
    // the parts of one 3x3 propagation (matter-dominated, two sweeps)
    {
        const long long r0 = g_rsqrt;
        prop3_count(m3);
        std::printf("prop3_rsqrt %lld\nprop3_sincos_pairs 2\n", g_rsqrt - r0);
    }
    return 0;
}
