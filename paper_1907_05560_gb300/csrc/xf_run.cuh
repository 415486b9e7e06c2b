// xf_run.cuh -- the persistent fused integrator kernel.
//
// One cooperative launch advances one problem by n_steps fixed radial steps.
// Every integrator stage is one pass over the CTA's (u, E) pairs (both species
// of a pair are handled by the same thread):
//
//   1. each thread updates its pairs (Hamiltonian assembly + RK4 stage or
//      exact propagator) from the moments M0, M1 of the stage input, and
//      accumulates the weighted nu-nu sums of the stage output (Eq. 3.13)
//   2. fixed-order reduction: per thread (pairs in index order) -> warp
//      shuffle tree -> CTA (warps in order) -> one partial per CTA in global
//   3. grid barrier (bounded spin on a global counter; times out with an
//      error flag instead of hanging)
//   4. every CTA sums all CTA partials in the same fixed order, so every CTA
//      holds bitwise identical M0, M1 for the next stage
//
// RK4 needs 4 stages per step, the predictor-corrector (Sec. 4.2.3, Listing
// 5.1 S1-S3) needs 2.  The reduction tree depends only on the launch shape,
// so results are deterministic run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xf_math.cuh"

namespace xf {

enum { GEOM_BULB = 0, GEOM_MU_R4 = 1, GEOM_SA = 2, GEOM_CONST = 3 };
enum { MAT_NONE = 0, MAT_POWER = 1, MAT_EXP = 2 };
enum { STEP_RK4 = 0, STEP_EXPH = 1 };
enum { ERR_NONFINITE = 1, ERR_BARRIER = 2 };

// Kernel arguments (one problem).  State planes are component-major:
// element (c, s, p) of a state buffer is at ((c * 2 + s) * npad + p).
struct RunArgs {
    int n_E, n_u, n_pairs, npad;
    int geometry, matter;
    int pairs_per_cta, span_max;
    double R, mu0, du, dE;
    double ne_ref, r_ref, ne_power, nb0, h_ns, Ye, gf; // gf = sqrt(2) G_F in km^-1 cm^3
    double r0, h;             // step k of this launch starts at r0 + (k0 + k) h
    long long k0, n_steps;
    int cur;                  // buffer (0/1) holding the input state
    const void *hvac;         // Real [n_E][S]
    void *rho0, *rho1, *aux;  // Real state buffers
    double *partials;         // [2][grid][2S]
    double *mom_out;          // [2S] M0 | M1 of the final state (dE applied)
    unsigned *bar;            // barrier counter, zero at launch
    int *err;                 // error bits
    unsigned long long *steps_done; // running total, incremented by CTA 0 at exit
    unsigned long long timeout_ns;
    int skip_cta;             // test hook: this CTA leaves at its first barrier (-1: none)
};

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier number k (1-based) of this launch: wait until all CTAs
// have arrived k times.  The spin is bounded by a time limit and an
// iteration limit; on expiry it sets ERR_BARRIER and every CTA leaves.
// Returns false when the run must stop.
__device__ __forceinline__ bool grid_barrier(const RunArgs &a, unsigned k, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if ((int)blockIdx.x == a.skip_cta) {
            ok = 0; // leave without arriving: the other CTAs' waits run out
        } else if (gridDim.x > 1) {
            __threadfence();
            red_release_add_u32(a.bar, 1u);
            const unsigned target = k * gridDim.x;
            const unsigned long long t0 = gtimer();
            unsigned iter = 0;
            while (ld_acquire_u32(a.bar) < target) {
                ++iter;
                if ((iter & 255u) == 0) {
                    if (*(volatile int *)a.err) {
                        ok = 0;
                        break;
                    }
                    if (gtimer() - t0 > a.timeout_ns || iter > (1u << 30)) {
                        atomicOr(a.err, ERR_BARRIER);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ double matter_A(const RunArgs &a, double r)
{
    if (a.matter == MAT_POWER) return a.gf * a.ne_ref * pow(a.r_ref / r, a.ne_power);
    if (a.matter == MAT_EXP) return a.gf * a.Ye * a.nb0 * exp(-(r - a.R) / a.h_ns);
    return 0.0;
}

__device__ __forceinline__ double mu_eff(const RunArgs &a, double r)
{
    double x = a.R / r, x2 = x * x;
    if (a.geometry == GEOM_MU_R4) return a.mu0 * x2 * x2;
    if (a.geometry == GEOM_SA) {
        double t = 1.0 - sqrt(1.0 - x2); // Eq. 3.17
        return a.mu0 * 0.5 * t * t;
    }
    return a.mu0;
}

// cos(theta) of trajectory j at radius r (Eq. 3.14), u_j = (j + 1/2) du.
__device__ __forceinline__ double cos_u(const RunArgs &a, int j, double r)
{
    double x = a.R / r;
    return sqrt(1.0 - x * x * ((j + 0.5) * a.du));
}

// Table slots (each span_max doubles): 0 gamma (G = mu (M0 - gamma M1)),
// 1 kappa = dl/dr, 2 weight a (M0), 3 weight b (M1), 4 dl (step path length).
__device__ inline void build_rhs_table(const RunArgs &a, double *tb, int j_lo, int span, double r)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        int j = j_lo + q;
        double g = 0.0, k = 1.0;
        if (a.geometry == GEOM_BULB || a.geometry == GEOM_MU_R4) {
            double c = cos_u(a, j, r);
            g = c;
            k = 1.0 / c;
        }
        tb[0 * a.span_max + q] = g;
        tb[1 * a.span_max + q] = k;
    }
}
// weights of the nu-nu sums at radius r (Eq. 3.13-3.15)
__device__ inline void build_weight_table(const RunArgs &a, double *tb, int j_lo, int span, double r)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        int j = j_lo + q;
        double wa = a.du, wb = 0.0;
        if (a.geometry == GEOM_BULB) {
            double x = a.R / r, x2 = x * x;
            double c = sqrt(1.0 - x2 * ((j + 0.5) * a.du));
            wa = x2 * a.du / (2.0 * c);
            wb = wa * c;
        } else if (a.geometry == GEOM_MU_R4) {
            wb = a.du * cos_u(a, j, r);
        }
        tb[2 * a.span_max + q] = wa;
        tb[3 * a.span_max + q] = wb;
    }
}
// exact path length from r to r + h along trajectory j (Eq. 3.3, l = r cos):
// l(r+h) - l(r) = h (2r + h) / (l(r) + l(r+h)), free of cancellation.
__device__ inline void build_dl_table(const RunArgs &a, double *tb, int j_lo, int span, double r, double h)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        int j = j_lo + q;
        double dl = h;
        if (a.geometry == GEOM_BULB || a.geometry == GEOM_MU_R4) {
            double l0 = r * cos_u(a, j, r), l1 = (r + h) * cos_u(a, j, r + h);
            dl = h * (2.0 * r + h) / (l0 + l1);
        }
        tb[4 * a.span_max + q] = dl;
    }
}

// Reduce per-thread partial sums m[NV] over the CTA in fixed order and write
// the CTA partial to part[blockIdx.x * NV + c].
template <int NV, int NT>
__device__ __forceinline__ void cta_partial(double *m, double (*s_w)[NV], double *part)
{
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        double v = m[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        m[c] = v;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) s_w[w][c] = m[c];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) s += s_w[q][threadIdx.x];
        __stcg(part + (size_t)blockIdx.x * NV + threadIdx.x, s);
    }
}

// Sum the CTA partials of all CTAs in fixed order; result (times dE) in s_M.
template <int NV, int NT>
__device__ __forceinline__ void grid_total(const double *part, int G, double dE, double *s_M,
                                           double *s_scr)
{
    constexpr int LG = NT / NV; // threads per component
    const int t = threadIdx.x, c = t / LG, k = t % LG;
    double acc = 0.0;
    if (c < NV)
        for (int g = k; g < G; g += LG) acc += __ldcg(part + (size_t)g * NV + c);
    s_scr[t] = acc;
    __syncthreads();
    if (t < NV) {
        double s = 0.0;
        for (int q = 0; q < LG; ++q) s += s_scr[t * LG + q];
        s_M[t] = s * dE;
    }
    __syncthreads();
}

template <int NV>
__device__ __forceinline__ bool all_finite(const double *s_M)
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NV; ++c) ok = ok && isfinite(s_M[c]);
    return ok;
}

template <typename Real, int S>
__device__ __forceinline__ void load_state(const Real *buf, int npad, int s, int p, Real *t)
{
#pragma unroll
    for (int c = 0; c < S; ++c) t[c] = buf[(size_t)(c * 2 + s) * npad + p];
}
template <typename Real, int S>
__device__ __forceinline__ void store_state(Real *buf, int npad, int s, int p, const Real *t)
{
#pragma unroll
    for (int c = 0; c < S; ++c) buf[(size_t)(c * 2 + s) * npad + p] = t[c];
}

// Accumulate the weighted nu-nu sums of one pair's stage output.
template <int NF, typename Real>
__device__ __forceinline__ void accum(const Real *tn, const Real *tb, double wa, double wb, double *m)
{
    constexpr int S = Comp<NF>::S;
    Real d[S];
    nu_minus_conj_nubar<NF, Real>(tn, tb, d);
#pragma unroll
    for (int c = 0; c < S; ++c) {
        double dc = (double)d[c];
        m[c] += wa * dc;
        m[S + c] += wb * dc;
    }
}

template <int NF, int STEP, typename Real, int NT>
__global__ void __launch_bounds__(NT) xf_run_kernel(RunArgs a)
{
    constexpr int S = Comp<NF>::S, NV = 2 * S;
    extern __shared__ double s_tab[];
    __shared__ double s_M[NV];
    __shared__ double s_scr[NT];
    __shared__ double s_w[NT / 32][NV];
    __shared__ int s_flag;

    const int G = gridDim.x;
    const int p_begin = blockIdx.x * a.pairs_per_cta;
    const int p_end = min(p_begin + a.pairs_per_cta, a.n_pairs);
    const int j_lo = (p_begin < a.n_pairs) ? p_begin / a.n_E : 0;
    const int span = (p_begin < p_end) ? (p_end - 1) / a.n_E - j_lo + 1 : 0;
    const Real *hvac = (const Real *)a.hvac;
    Real *const buf0 = (Real *)a.rho0, *const buf1 = (Real *)a.rho1;
    Real *aux = (Real *)a.aux;
    unsigned nbar = 0;

    // an earlier launch on this ctx failed: leave the state untouched
    if (threadIdx.x == 0) s_flag = *(volatile int *)a.err;
    __syncthreads();
    if (s_flag) return;

    // ---- prologue: moments of the input state at r0
    {
        build_weight_table(a, s_tab, j_lo, span, a.r0 + (double)a.k0 * a.h);
        __syncthreads();
        double m[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) m[c] = 0.0;
        const Real *in = a.cur ? buf1 : buf0;
        for (int p = p_begin + threadIdx.x; p < p_end; p += NT) {
            const int q = p / a.n_E - j_lo;
            Real tn[S], tb[S];
            load_state<Real, S>(in, a.npad, 0, p, tn);
            load_state<Real, S>(in, a.npad, 1, p, tb);
            accum<NF, Real>(tn, tb, s_tab[2 * a.span_max + q], s_tab[3 * a.span_max + q], m);
        }
        cta_partial<NV, NT>(m, s_w, a.partials);
        if (!grid_barrier(a, ++nbar, &s_flag)) return;
        grid_total<NV, NT>(a.partials, G, a.dE, s_M, s_scr);
        if (!all_finite<NV>(s_M)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.err, ERR_NONFINITE);
            return;
        }
    }

    constexpr int NSTAGE = (STEP == STEP_RK4) ? 4 : 2;
    for (long long k = 0; k < a.n_steps; ++k) {
        // radii from the global step index, so that a run split over several
        // launches evaluates the same radii as one launch
        const double kk = (double)(a.k0 + k), h = a.h;
        const double r = a.r0 + kk * h, r_half = a.r0 + (kk + 0.5) * h, r_next = a.r0 + (kk + 1.0) * h;
        const bool odd = ((a.cur + (int)(k & 1)) & 1) != 0;
        const Real *cur = odd ? buf1 : buf0;
        Real *nxt = odd ? buf0 : buf1;
#pragma unroll 1
        for (int st = 0; st < NSTAGE; ++st) {
            // radius of the right-hand side and of the stage output
            double r_rhs, r_out;
            if constexpr (STEP == STEP_RK4) {
                r_rhs = (st == 0) ? r : (st == 3 ? r_next : r_half);
                r_out = (st <= 1) ? r_half : r_next;
            } else {
                r_rhs = (st == 0) ? r : r_next;
                r_out = r_next;
            }
            __syncthreads();
            build_rhs_table(a, s_tab, j_lo, span, r_rhs);
            build_weight_table(a, s_tab, j_lo, span, r_out);
            if (STEP == STEP_EXPH && st == 0) build_dl_table(a, s_tab, j_lo, span, r, h);
            const double mu = mu_eff(a, r_rhs);
            const Real A = (Real)matter_A(a, r_rhs);
            __syncthreads();
            Real M0[S], M1[S];
#pragma unroll
            for (int c = 0; c < S; ++c) {
                M0[c] = (Real)(mu * s_M[c]);
                M1[c] = (Real)(mu * s_M[S + c]);
            }
            double m[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) m[c] = 0.0;

            for (int p = p_begin + threadIdx.x; p < p_end; p += NT) {
                const int j = p / a.n_E, e = p - j * a.n_E, q = j - j_lo;
                const Real gam = (Real)s_tab[q];
                Real g[S], hv[S], hn[S], hb[S];
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    g[c] = M0[c] - gam * M1[c];
                    hv[c] = hvac[(size_t)e * S + c];
                }
                hamiltonians<NF, Real>(hv, A, g, hn, hb);
                Real on[S], ob[S]; // stage outputs (nu, nubar)
                if constexpr (STEP == STEP_RK4) {
                    const Real kap = (Real)s_tab[a.span_max + q];
                    const Real cy = (Real)((st == 2) ? h : 0.5 * h);
                    const Real cb = (Real)((st == 0 || st == 3) ? h / 6.0 : h / 3.0);
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        Real y[S], kk[S], rn[S], bb[S];
                        if (st == 0) load_state<Real, S>(cur, a.npad, s, p, y);
                        else load_state<Real, S>(aux, a.npad, s, p, y);
                        comm<NF, Real>(s == 0 ? hn : hb, y, kk);
#pragma unroll
                        for (int c = 0; c < S; ++c) kk[c] *= kap;
                        if (st == 0) {
#pragma unroll
                            for (int c = 0; c < S; ++c) rn[c] = y[c];
                        } else if (st < 3) {
                            load_state<Real, S>(cur, a.npad, s, p, rn);
                        }
                        if (st == 0) {
#pragma unroll
                            for (int c = 0; c < S; ++c) bb[c] = rn[c] + cb * kk[c];
                        } else {
                            load_state<Real, S>(nxt, a.npad, s, p, bb);
#pragma unroll
                            for (int c = 0; c < S; ++c) bb[c] += cb * kk[c];
                        }
                        store_state<Real, S>(nxt, a.npad, s, p, bb);
                        Real *o = (s == 0) ? on : ob;
                        if (st < 3) {
#pragma unroll
                            for (int c = 0; c < S; ++c) o[c] = rn[c] + cy * kk[c];
                            store_state<Real, S>(aux, a.npad, s, p, o);
                        } else {
#pragma unroll
                            for (int c = 0; c < S; ++c) o[c] = bb[c];
                        }
                    }
                } else {
                    const double dl = s_tab[4 * a.span_max + q];
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        Real rn[S], pr[S];
                        load_state<Real, S>(cur, a.npad, s, p, rn);
                        prop<NF, Real>(s == 0 ? hn : hb, dl, rn, pr);
                        Real *o = (s == 0) ? on : ob;
                        if (st == 0) {
#pragma unroll
                            for (int c = 0; c < S; ++c) o[c] = pr[c];
                            store_state<Real, S>(aux, a.npad, s, p, o);
                        } else {
                            Real pp[S];
                            load_state<Real, S>(aux, a.npad, s, p, pp);
#pragma unroll
                            for (int c = 0; c < S; ++c) o[c] = Real(0.5) * (pp[c] + pr[c]);
                            store_state<Real, S>(nxt, a.npad, s, p, o);
                        }
                    }
                }
                accum<NF, Real>(on, ob, s_tab[2 * a.span_max + q], s_tab[3 * a.span_max + q], m);
            }
            cta_partial<NV, NT>(m, s_w, a.partials + (size_t)(nbar & 1) * G * NV);
            if (!grid_barrier(a, ++nbar, &s_flag)) return;
            grid_total<NV, NT>(a.partials + (size_t)((nbar - 1) & 1) * G * NV, G, a.dE, s_M, s_scr);
            if (!all_finite<NV>(s_M)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    atomicOr(a.err, ERR_NONFINITE);
                    atomicAdd(a.steps_done, (unsigned long long)k);
                }
                return;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(a.steps_done, (unsigned long long)a.n_steps);
        for (int c = 0; c < NV; ++c) a.mom_out[c] = s_M[c];
    }
}

} // namespace xf
