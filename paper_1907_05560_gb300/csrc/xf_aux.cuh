// xf_aux.cuh -- non-hot-path device kernels: seeded initial state, packed <->
// component-major layout conversion, full moments, per-bin outputs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xf_math.cuh"
#include "xf_psi.cuh"

namespace xf {

// SplitMix64 (Steele, Lea & Flood 2014): the i-th output of the stream
// seeded with `seed`, computed from the counter alone.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct LayoutArgs {
    int n_E, n_u, n_pairs, npad;
    const double *phi;  // [4][n_E] number-flux weights (nu_e, nubar_e, nu_x, nubar_x)
    double eps;
    uint64_t seed;
    int *bad;           // set to 1 if an input value is not finite
};

// Bin b = (s n_u + j) n_E + e  <->  species s, pair p = j n_E + e.
__device__ __forceinline__ void bin_split(const LayoutArgs &a, long long b, int *s, int *p)
{
    long long per = (long long)a.n_u * a.n_E;
    *s = (int)(b / per);
    *p = (int)(b - (long long)(*s) * per);
}

// Seeded initial state (one thread per bin): rho = diag(phi_e, phi_x[, phi_x])
// plus eps sqrt(rho_ii rho_jj) exp(2 pi i U) on each upper entry.
// ref (may be NULL): receives tr(T^2) of each bin's traceless part, the
// quantity the renormalising variant restores after every step.
template <int NF, typename Real>
__global__ void init_state_kernel(LayoutArgs a, Real *state, double *trace, Real *ref)
{
    constexpr int S = Comp<NF>::S, NOFF = NF * (NF - 1) / 2;
    const long long nb = 2ll * a.n_pairs;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        const int e = p % a.n_E;
        const double pe = a.phi[(s == 0 ? 0 : 1) * a.n_E + e];
        const double px = a.phi[(s == 0 ? 2 : 3) * a.n_E + e];
        double dg[3] = {pe, px, px};
        double tr = pe + (NF - 1) * px;
        double t[S];
        if constexpr (NF == 2) {
            t[0] = 0.5 * (pe - px);
        } else {
            double tau = tr / 3.0;
            t[0] = pe - tau;
            t[1] = px - tau;
        }
        int k = 0;
        for (int i = 0; i < NF; ++i)
            for (int j = i + 1; j < NF; ++j) {
                uint64_t z = splitmix64(a.seed, (uint64_t)b * NOFF + k);
                double U = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                double sn, cs;
                sincos(6.283185307179586476925286766559 * U, &sn, &cs);
                double amp = a.eps * sqrt(dg[i] * dg[j]);
                t[NF - 1 + 2 * k] = amp * cs;
                t[NF + 2 * k] = amp * sn;
                ++k;
            }
#pragma unroll
        for (int c = 0; c < S; ++c) state[(size_t)(c * 2 + s) * a.npad + p] = (Real)t[c];
        trace[(size_t)s * a.npad + p] = tr;
        if (ref) ref[(size_t)s * a.npad + p] = (Real)purity<NF, double>(t);
    }
}

// packed host layout -> traceless components + trace (+ tr(T^2) into ref)
template <int NF, typename Real>
__global__ void pack_to_state_kernel(LayoutArgs a, const double *packed, Real *state, double *trace, Real *ref)
{
    constexpr int S = Comp<NF>::S, M = NF * NF;
    const long long nb = 2ll * a.n_pairs;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        const double *x = packed + (size_t)b * M;
        bool ok = true;
        for (int c = 0; c < M; ++c) ok = ok && isfinite(x[c]);
        if (!ok) *a.bad = 1;
        double t[S], tr;
        if constexpr (NF == 2) {
            tr = x[0] + x[1];
            t[0] = 0.5 * (x[0] - x[1]);
            t[1] = x[2];
            t[2] = x[3];
        } else {
            tr = x[0] + x[1] + x[2];
            double tau = tr / 3.0;
            t[0] = x[0] - tau;
            t[1] = x[1] - tau;
            for (int c = 0; c < 6; ++c) t[2 + c] = x[3 + c];
        }
#pragma unroll
        for (int c = 0; c < S; ++c) state[(size_t)(c * 2 + s) * a.npad + p] = (Real)t[c];
        trace[(size_t)s * a.npad + p] = tr;
        if (ref) ref[(size_t)s * a.npad + p] = (Real)purity<NF, double>(t);
    }
}

// traceless components + trace -> packed host layout
template <int NF, typename Real>
__global__ void state_to_pack_kernel(LayoutArgs a, const Real *state, const double *trace, double *packed)
{
    constexpr int S = Comp<NF>::S, M = NF * NF;
    const long long nb = 2ll * a.n_pairs;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        double t[S];
#pragma unroll
        for (int c = 0; c < S; ++c) t[c] = (double)state[(size_t)(c * 2 + s) * a.npad + p];
        const double tr = trace[(size_t)s * a.npad + p];
        double *x = packed + (size_t)b * M;
        if constexpr (NF == 2) {
            const double tau = 0.5 * tr;
            x[0] = tau + t[0];
            x[1] = tau - t[0];
            x[2] = t[1];
            x[3] = t[2];
        } else {
            const double tau = tr / 3.0;
            x[0] = tau + t[0];
            x[1] = tau + t[1];
            x[2] = tau - t[0] - t[1];
            for (int c = 0; c < 6; ++c) x[3 + c] = t[2 + c];
        }
    }
}

// Per-bin outputs: survival probability, trace, tr(T^2) of the traceless part.
template <int NF, typename Real>
__global__ void outputs_kernel(LayoutArgs a, const Real *state, const double *trace, double *p_surv,
                               double *trace_out, double *purity_out)
{
    constexpr int S = Comp<NF>::S;
    const long long nb = 2ll * a.n_pairs;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        const int e = p % a.n_E;
        double t[S];
#pragma unroll
        for (int c = 0; c < S; ++c) t[c] = (double)state[(size_t)(c * 2 + s) * a.npad + p];
        const double tr = trace[(size_t)s * a.npad + p];
        const double ree = (NF == 2 ? 0.5 * tr : tr / 3.0) + t[0];
        const double pur = purity<NF, double>(t);
        const double pe = a.phi[(s == 0 ? 0 : 1) * a.n_E + e];
        const double px = a.phi[(s == 0 ? 2 : 3) * a.n_E + e];
        if (p_surv) p_surv[b] = (pe != px) ? (ree - px) / (pe - px) : (double)NAN;
        if (trace_out) trace_out[b] = tr;
        if (purity_out) purity_out[b] = pur;
    }
}

// Full nu-nu moments of a state at radius r (fixed-order, two kernels):
// CTA b sums pairs [b * chunk, (b+1) * chunk) -> part[b][NV + 2], where the
// last two entries carry the trace sums (trace of rho_nu - rho_nubar) for the
// a- and b-weights; a single CTA then sums the partials in order and writes
// the packed Hermitian M0, M1 (trace restored on the diagonal).
struct MomArgs {
    int n_E, n_u, n_phi, n_pairs, npad, geometry, chunk, pad_;
    double R, du, dE, r;
};

// Weights of trajectory t = j n_phi + k for the moments M0..M3 at radius m.r
// (Eq. 3.13-3.15 and, with azimuth bins, Eq. 3.18: each bin carries 1/n_phi
// of its zenith bin's weight, M2 / M3 weighted by sin th' cos / sin ph'; the
// cylinder model's latitude-averaged moments, Eq. 3.20).
__device__ __forceinline__ void mom_weights(const MomArgs &m, int t, double *w)
{
    const int j = t / m.n_phi, k = t - j * m.n_phi;
    w[0] = m.du;
    w[1] = w[2] = w[3] = 0.0;
    if (m.geometry == 4) { // cylinder (Eq. 3.20): latitude averages of w, w cos(alpha), w sin(alpha)
        const double pi = 3.14159265358979323846;
        double st, ct;
        sincos(-0.5 * pi + (j + 0.5) * pi / m.n_u, &st, &ct);
        const double sa = (m.R / m.r) * st, ca = sqrt(1.0 - sa * sa);
        const double wc = ct / ca * (pi / m.n_u);
        w[0] = wc / m.n_phi;
        w[1] = wc * ca / m.n_phi;
        w[2] = wc * sa / m.n_phi;
        return;
    }
    if (m.geometry == 0 || m.geometry == 1) {
        double x = m.R / m.r, x2 = x * x, u = (j + 0.5) * m.du;
        double c = sqrt(1.0 - x2 * u);
        if (m.geometry == 0) {
            double a = x2 * m.du / (2.0 * c);
            w[0] = a / m.n_phi;
            w[1] = a * c / m.n_phi;
            if (m.n_phi > 1) {
                double sn = sqrt(x2 * u), sp, cp;
                sincos((k + 0.5) * 2.0 * 3.14159265358979323846 / m.n_phi, &sp, &cp);
                w[2] = a * sn * cp / m.n_phi;
                w[3] = a * sn * sp / m.n_phi;
            }
        } else {
            w[1] = m.du * c;
        }
    }
}

// FP64 sums of the four moments over chunks of pairs: per component the
// traceless parts (4 S values) and the trace parts (4 values).
template <int NF, typename Real, int NT>
__global__ void __launch_bounds__(NT) moments_partial_kernel(MomArgs m, const Real *state,
                                                             const double *trace, double *part)
{
    constexpr int S = Comp<NF>::S, NV = 4 * S + 4;
    __shared__ double s_w[NT / 32][NV];
    double acc[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] = 0.0;
    const int p0 = blockIdx.x * m.chunk, p1 = min(p0 + m.chunk, m.n_pairs);
    for (int p = p0 + threadIdx.x; p < p1; p += NT) {
        const int t = p / m.n_E;
        double w[4];
        mom_weights(m, t, w);
        Real tn[S], tb[S], d[S];
#pragma unroll
        for (int c = 0; c < S; ++c) {
            tn[c] = state[(size_t)(c * 2 + 0) * m.npad + p];
            tb[c] = state[(size_t)(c * 2 + 1) * m.npad + p];
        }
        nu_minus_conj_nubar<NF, Real>(tn, tb, d);
        const double dtr = trace[p] - trace[(size_t)m.npad + p];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int c = 0; c < S; ++c) acc[q * S + c] += w[q] * (double)d[c];
            acc[4 * S + q] += w[q] * dtr;
        }
    }
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        double v = acc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int q = 0; q < NT / 32; ++q) s += s_w[q][threadIdx.x];
        part[(size_t)blockIdx.x * NV + threadIdx.x] = s;
    }
}

// Sum the chunk partials in order; M[q] (q = 0..3) packed like a bin, times dE.
template <int NF>
__global__ void moments_final_kernel(const double *part, int G, double dE, double *M)
{
    constexpr int S = Comp<NF>::S, NV = 4 * S + 4, MM = NF * NF;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot[NV];
    for (int c = 0; c < NV; ++c) tot[c] = 0.0;
    for (int g = 0; g < G; ++g)
        for (int c = 0; c < NV; ++c) tot[c] += part[(size_t)g * NV + c];
    for (int q = 0; q < 4; ++q) {
        const double *t = tot + q * S;
        const double tau = tot[4 * S + q] / NF * dE;
        double *x = M + q * MM;
        if constexpr (NF == 2) {
            x[0] = tau + t[0] * dE;
            x[1] = tau - t[0] * dE;
            x[2] = t[1] * dE;
            x[3] = t[2] * dE;
        } else {
            x[0] = tau + t[0] * dE;
            x[1] = tau + t[1] * dE;
            x[2] = tau - (t[0] + t[1]) * dE;
            for (int c = 0; c < 6; ++c) x[3 + c] = t[2 + c] * dE;
        }
    }
}

// Dump mode 2 (Sec. 4.2.4): the flavor state of each trajectory averaged over
// its energy bins.  One block per (s, trajectory); threads stride the
// energies, sum the packed entries in FP64, then the block adds the threads'
// sums in a fixed order.  out[(s n_traj + t) NF^2 + c] (a.n_u = trajectories).
template <int NF, typename Real, int NT>
__global__ void __launch_bounds__(NT) angle_average_kernel(LayoutArgs a, const Real *state, const double *trace,
                                                           double *out)
{
    constexpr int S = Comp<NF>::S, M = NF * NF;
    __shared__ double sm[NT][M];
    const int s = blockIdx.x / a.n_u, j = blockIdx.x % a.n_u;
    double acc[M];
#pragma unroll
    for (int c = 0; c < M; ++c) acc[c] = 0.0;
    for (int e = threadIdx.x; e < a.n_E; e += NT) {
        const int p = j * a.n_E + e;
        double t[S];
#pragma unroll
        for (int c = 0; c < S; ++c) t[c] = (double)state[(size_t)(c * 2 + s) * a.npad + p];
        const double tau = trace[(size_t)s * a.npad + p] / NF;
        if constexpr (NF == 2) {
            acc[0] += tau + t[0];
            acc[1] += tau - t[0];
            acc[2] += t[1];
            acc[3] += t[2];
        } else {
            acc[0] += tau + t[0];
            acc[1] += tau + t[1];
            acc[2] += tau - (t[0] + t[1]);
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[3 + c] += t[2 + c];
        }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) sm[threadIdx.x][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < M) {
        double v = 0.0;
        for (int q = 0; q < NT; ++q) v += sm[q][threadIdx.x];
        out[(size_t)blockIdx.x * M + threadIdx.x] = v / a.n_E;
    }
}

// ---- wavefunction form (one psi per initial flavor; 2 n_f^2 reals per bin,
// component c = (a n_f + i) 2 + re/im at (c 2 + s) npad + p) ---------------

// Seeded wavefunctions: psi_a = (e_a + eps sum_{b != a} exp(2 pi i U_ab) e_b)
// / sqrt(1 + (n_f - 1) eps^2), U_ab the SplitMix64 uniform number at counter
// bin n_f (n_f - 1) + k, k running over (a, b != a) in row order.
template <int NF, typename Real>
__global__ void psi_init_kernel(LayoutArgs a, Real *state)
{
    constexpr int NPERM = NF * (NF - 1);
    const long long nb = 2ll * a.n_pairs;
    const double norm = 1.0 / sqrt(1.0 + (NF - 1) * a.eps * a.eps);
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        int k = 0;
        for (int fa = 0; fa < NF; ++fa)
            for (int i = 0; i < NF; ++i) {
                double re = 0.0, im = 0.0;
                if (i == fa) {
                    re = norm;
                } else {
                    uint64_t z = splitmix64(a.seed, (uint64_t)b * NPERM + k);
                    double U = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                    double sn, cs;
                    sincos(6.283185307179586476925286766559 * U, &sn, &cs);
                    re = norm * a.eps * cs;
                    im = norm * a.eps * sn;
                    ++k;
                }
                const int c = (fa * NF + i) * 2;
                state[(size_t)(c * 2 + s) * a.npad + p] = (Real)re;
                state[(size_t)((c + 1) * 2 + s) * a.npad + p] = (Real)im;
            }
    }
}

// Density matrices of the wavefunction state (rho = sum_a phi_a psi_a psi_a^+)
// into a traceless plane and the FP64 trace, for the outputs and moments.
template <int NF, typename Real>
__global__ void psi_to_rho_kernel(LayoutArgs a, const Real *psi, Real *state, double *trace)
{
    constexpr int S = Comp<NF>::S, SS = 2 * NF * NF;
    const long long nb = 2ll * a.n_pairs;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        const int e = p % a.n_E;
        double x[SS], t[S], tr;
#pragma unroll
        for (int c = 0; c < SS; ++c) x[c] = (double)psi[(size_t)(c * 2 + s) * a.npad + p];
        const double w0 = a.phi[(s == 0 ? 0 : 1) * a.n_E + e], w1 = a.phi[(s == 0 ? 2 : 3) * a.n_E + e];
        psi_rho<NF, double>(x, w0, w1, t, &tr);
#pragma unroll
        for (int c = 0; c < S; ++c) state[(size_t)(c * 2 + s) * a.npad + p] = (Real)t[c];
        trace[(size_t)s * a.npad + p] = tr;
    }
}

// packed host wavefunctions [s][t][E][a][i](re, im) <-> planes
template <int NF, typename Real>
__global__ void psi_pack_kernel(LayoutArgs a, const double *packed, Real *state, int to_device)
{
    constexpr int SS = 2 * NF * NF;
    const long long nb = 2ll * a.n_pairs;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        int s, p;
        bin_split(a, b, &s, &p);
        double *x = (double *)packed + (size_t)b * SS;
        for (int c = 0; c < SS; ++c) {
            Real &y = state[(size_t)(c * 2 + s) * a.npad + p];
            if (to_device) {
                if (!isfinite(x[c])) *a.bad = 1;
                y = (Real)x[c];
            } else {
                x[c] = (double)y;
            }
        }
    }
}

} // namespace xf
