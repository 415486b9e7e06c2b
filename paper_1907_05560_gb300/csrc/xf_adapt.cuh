// xf_adapt.cuh -- the error-controlled step of Sec. 4.2.3 (Fig. 4.8-4.9;
// sections S1-S5 of Listings 5.1-5.3) as one persistent kernel.
//
// An attempt from rho0 at r with step h needs four Hamiltonians, H0 from
// rho0 at r, H1 from the full-step predictor at r + h, H2 from the half-step
// predictor at r + h/2, H3 from the fine path's end point at r + h.  H1 and
// H2 come from one fused reduction (the paper's third loop order), so an
// attempt takes three grid-synchronised stages:
//   A  (H0)      rho2 = U(H0; r, h) rho0, rho1 = U(H0; r, h/2) rho0 (one
//                eigendecomposition); moments of rho2 at r + h and of rho1 at
//                r + h/2
//   B  (H1, H2)  rho_c = (rho2 + U(H1; r, h) rho0) / 2 (the coarse result),
//                rho5 = U(H2; r + h/2, h/2) rho1; moments of rho5 at r + h
//   C  (H3)      rho_f = (rho5 + U(H3; r, h) rho0) / 2; per-bin error
//                max |rho_c - rho_f| / tr rho; moments of rho_c at r + h
// and the accept / reject decision opens the next attempt's stage A: with
// err <= eps0 the coarse result becomes the state, and the next step is
// ksi h (eps0/err)^(1/2) trimmed to dr_max.  A rejected attempt leaves rho0
// and its moments untouched.
//
// Buffers: the instance's three state planes rotate, cur = rho0, X = cur + 1
// (rho2, then rho_c), Y = cur + 2 (rho1, then rho5); accepting makes X the
// new cur.  Partial sums (stride APS doubles per tile) sit in four slots:
// in_slot (0 or 3) holds the moments of rho0, 1 the stage A pair, 2 stage B,
// 3 - in_slot stage C (moments of rho_c and the error), which becomes in_slot
// on acceptance.
#pragma once

#include "xf_run.cuh"

namespace xf {

constexpr int APS = 2 * NVMAX + 4; // doubles per tile and slot: two moment sets, the error, padding
constexpr int AERR = 2 * NVMAX;    // index of the error in a slot

// Shared per-angle tables of the error-controlled kernel, span_max entries
// each: 0 gamma_a, 1 gamma_b, 2-3 weights (a, b) of set 1, 4-5 weights of set
// 2, then two step lengths (one slot each in FP64, hi + lo in FP32).
template <typename Real> struct ASlots;
template <> struct ASlots<double> { static constexpr int dl1 = 6, dl2 = 7, n = 8; };
template <> struct ASlots<float> { static constexpr int dl1 = 6, dl2 = 8, n = 10; };

__device__ __forceinline__ void store_dl_at(double *tb, int smax, int slot, int q, double dl) { tb[slot * smax + q] = dl; }
__device__ __forceinline__ void store_dl_at(float *tb, int smax, int slot, int q, double dl)
{
    const StepLen<float> d = make_step_len(dl, (float *)nullptr);
    tb[slot * smax + q] = d.hi;
    tb[(slot + 1) * smax + q] = d.lo;
}
__device__ __forceinline__ StepLen<double> load_dl_at(const double *tb, int smax, int slot, int q)
{
    return {tb[slot * smax + q]};
}
__device__ __forceinline__ StepLen<float> load_dl_at(const float *tb, int smax, int slot, int q)
{
    return {tb[slot * smax + q], tb[(slot + 1) * smax + q]};
}

struct SharedA {
    double M[2 * NVMAX];     // instance totals (dE applied) of the slot being read
    double scr[256];         // reduction scratch (>= NT)
    double w[8][2 * NVMAX];  // per-warp sums (NT <= 256)
    double ew[8];            // per-warp error maxima
    double err;              // instance error maximum
    double mu[2], A[2];      // stage scalars (H1 / H2 in stage B)
    AdaptPos ts;             // the current tile's copy of its instance's progress
    int flag;
};

// max that lets a NaN through (a NaN error must reject, not vanish)
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }

// Totals over an instance's tiles [t0, t1) of the first nv components of a
// slot (in tile order, times dE) into sh.M; with want_err also the maximum
// of the tiles' errors into sh.err.
template <int NT>
__device__ __forceinline__ void adapt_total(const double *slot, int t0, int t1, int nv, double dE, bool want_err,
                                            SharedA &sh)
{
    constexpr int LG = NT / (2 * NVMAX); // threads per component
    const int t = threadIdx.x, c = t / LG, k = t % LG;
    double acc = 0.0;
    if (c < nv)
        for (int g = t0 + k; g < t1; g += LG) acc += __ldcg(slot + (size_t)g * APS + c);
    sh.scr[t] = acc;
    __syncthreads();
    if (t < nv) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < LG; ++q) s += sh.scr[t * LG + q];
        sh.M[t] = s * dE;
    }
    if (want_err && t < 32) {
        double e = 0.0;
        for (int g = t0 + t; g < t1; g += 32) e = nanmax(e, __ldcg(slot + (size_t)g * APS + AERR));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e = nanmax(e, __shfl_down_sync(0xffffffffu, e, off));
        if (t == 0) sh.err = e;
    }
    __syncthreads();
}

// CTA maximum of per-thread errors into part[AERR].
template <int NT>
__device__ __forceinline__ void cta_max(double e, SharedA &sh, double *part)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = nanmax(e, __shfl_down_sync(0xffffffffu, e, off));
    if ((threadIdx.x & 31) == 0) sh.ew[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) m = nanmax(m, sh.ew[q]);
        __stcg(part + AERR, m);
    }
    __syncthreads();
}

// Largest entry modulus of the packed traceless difference d (3 or 8 reals).
template <int NF, typename Real>
__device__ __forceinline__ Real max_entry(const Real *d)
{
    if constexpr (NF == 2) {
        return fmax(fabs(d[0]), sqrt_r(d[1] * d[1] + d[2] * d[2]));
    } else {
        Real m = fmax(fmax(fabs(d[0]), fabs(d[1])), fabs(d[0] + d[1]));
        m = fmax(m, sqrt_r(d[2] * d[2] + d[3] * d[3]));
        m = fmax(m, sqrt_r(d[4] * d[4] + d[5] * d[5]));
        return fmax(m, sqrt_r(d[6] * d[6] + d[7] * d[7]));
    }
}

// The decision after an attempt (identical on every tile of the instance).
__device__ __forceinline__ void adapt_decide(const Inst &in, AdaptPos &ts, double err, bool finite)
{
    ts.err = err;
    ts.iters_left -= 1;
    if (!finite || !(err == err) || isinf(err)) { // rho0 stays the last accepted state
        ts.status = AD_NONFINITE;
        return;
    }
    if (err <= in.eps0) {
        ts.cur = (ts.cur + 1) % 3;
        ts.r = ts.last ? ts.r_end : ts.r + ts.ht;
        ts.in_slot = 3 - ts.in_slot;
        ++ts.n_acc;
    } else {
        ++ts.n_rej;
    }
    const double hn = (err > 0.0) ? in.ksi * ts.ht * sqrt(in.eps0 / err) : in.dr_max;
    ts.h = hn < in.dr_max ? hn : in.dr_max;
    if (!(ts.r_end - ts.r > 1e-12 * ts.r_end)) {
        ts.status = AD_DONE;
        ts.r = ts.r_end;
    } else if (ts.iters_left <= 0) {
        ts.status = AD_BUDGET;
    } else if (ts.h < 1e-12 * ts.r) {
        ts.status = AD_STEPSIZE;
    }
}

template <typename Real>
struct AdaptView {
    const Real *hvac;
    const double *trace;
    Real *b0, *bx, *by; // rho0, X, Y
    int n_E, npad, p0, p1, j_lo;
};

template <typename Real>
__device__ __forceinline__ AdaptView<Real> adapt_view(const RunArgs &a, const Inst &in, const Tile &tl, int cur)
{
    AdaptView<Real> v;
    Real *const base = (Real *)a.arena;
    v.b0 = base + in.off[cur];
    v.bx = base + in.off[(cur + 1) % 3];
    v.by = base + in.off[(cur + 2) % 3];
    v.hvac = base + in.hvac_off;
    v.trace = (const double *)a.arena + in.trace_off;
    v.n_E = in.n_E;
    v.npad = in.npad;
    v.p0 = tl.p0;
    v.p1 = tl.p0 + tl.np;
    v.j_lo = tl.p0 / in.n_E;
    return v;
}

// Per-tile G = mu (M0 - gamma M1) inputs: the moments scaled by mu.
template <int S, typename Real>
__device__ __forceinline__ void scaled_moments(const double *M, double mu, Real *M0, Real *M1)
{
#pragma unroll
    for (int c = 0; c < S; ++c) {
        M0[c] = (Real)(mu * M[c]);
        M1[c] = (Real)(mu * M[S + c]);
    }
}

// Stage A of one tile: H0 from sh.M at r (gamma slot 0, mu/A [0]).
template <int NF, typename Real, int NT>
__device__ __forceinline__ void adapt_stage_a(const AdaptView<Real> v, int smax, const Real *tb, SharedA &sh,
                                              double *part_out)
{
    constexpr int S = Comp<NF>::S, NV = 2 * S;
    Real M0[S], M1[S];
    scaled_moments<S, Real>(sh.M, sh.mu[0], M0, M1);
    const Real A = (Real)sh.A[0];
    Real m[2 * NV];
#pragma unroll
    for (int c = 0; c < 2 * NV; ++c) m[c] = Real(0);
    for (int p = v.p0 + threadIdx.x; p < v.p1; p += NT) {
        const int j = p / v.n_E, e = p - j * v.n_E, q = j - v.j_lo;
        const Real gam = tb[q];
        Real g[S], hv[S], hn[S], hb[S];
#pragma unroll
        for (int c = 0; c < S; ++c) {
            g[c] = M0[c] - gam * M1[c];
            hv[c] = v.hvac[(size_t)e * S + c];
        }
        hamiltonians<NF, Real>(hv, A, g, hn, hb);
        const StepLen<Real> dlf = load_dl_at(tb, smax, ASlots<Real>::dl1, q);
        const StepLen<Real> dlh = load_dl_at(tb, smax, ASlots<Real>::dl2, q);
        Real fn[S], fb[S], hn_[S], hb_[S]; // full and half step outputs (nu, nubar)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Real r0[S];
            load_state<Real, S>(v.b0, v.npad, s, p, r0);
            Real *full = s ? fb : fn, *half = s ? hb_ : hn_;
            prop_pair<NF, Real>(s ? hb : hn, dlf, dlh, r0, full, half);
            store_state<Real, S>(v.bx, v.npad, s, p, full);
            store_state<Real, S>(v.by, v.npad, s, p, half);
        }
        accum<NF, Real, Real>(fn, fb, tb[2 * smax + q], tb[3 * smax + q], m);
        accum<NF, Real, Real>(hn_, hb_, tb[4 * smax + q], tb[5 * smax + q], m + NV);
    }
    cta_partial<2 * NV, NT, Real>(m, sh, part_out);
}

// Stage B of one tile: H1 from sh.M[0, NV) at r + h (gamma slot 0, [0]),
// H2 from sh.M[NV, 2 NV) at r + h/2 (gamma slot 1, [1]).
template <int NF, typename Real, int NT>
__device__ __forceinline__ void adapt_stage_b(const AdaptView<Real> v, int smax, const Real *tb, SharedA &sh,
                                              double *part_out)
{
    constexpr int S = Comp<NF>::S, NV = 2 * S;
    Real m[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) m[c] = Real(0);
    for (int p = v.p0 + threadIdx.x; p < v.p1; p += NT) {
        const int j = p / v.n_E, e = p - j * v.n_E, q = j - v.j_lo;
        Real hv[S];
#pragma unroll
        for (int c = 0; c < S; ++c) hv[c] = v.hvac[(size_t)e * S + c];
        Real o5n[S], o5b[S];
        {
            // coarse result with H1
            Real M0[S], M1[S], g[S], hn[S], hb[S];
            scaled_moments<S, Real>(sh.M, sh.mu[0], M0, M1);
            const Real gam = tb[q];
#pragma unroll
            for (int c = 0; c < S; ++c) g[c] = M0[c] - gam * M1[c];
            hamiltonians<NF, Real>(hv, (Real)sh.A[0], g, hn, hb);
            const StepLen<Real> dlf = load_dl_at(tb, smax, ASlots<Real>::dl1, q);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                Real r0[S], r3[S], r2[S];
                load_state<Real, S>(v.b0, v.npad, s, p, r0);
                prop<NF, Real>(s ? hb : hn, dlf, r0, r3);
                load_state<Real, S>(v.bx, v.npad, s, p, r2);
#pragma unroll
                for (int c = 0; c < S; ++c) r2[c] = Real(0.5) * (r2[c] + r3[c]);
                store_state<Real, S>(v.bx, v.npad, s, p, r2);
            }
        }
        {
            // fine path, midpoint to end with H2
            Real M0[S], M1[S], g[S], hn[S], hb[S];
            scaled_moments<S, Real>(sh.M + NV, sh.mu[1], M0, M1);
            const Real gam = tb[smax + q];
#pragma unroll
            for (int c = 0; c < S; ++c) g[c] = M0[c] - gam * M1[c];
            hamiltonians<NF, Real>(hv, (Real)sh.A[1], g, hn, hb);
            const StepLen<Real> dlm = load_dl_at(tb, smax, ASlots<Real>::dl2, q);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                Real r1[S];
                load_state<Real, S>(v.by, v.npad, s, p, r1);
                Real *o = s ? o5b : o5n;
                prop<NF, Real>(s ? hb : hn, dlm, r1, o);
                store_state<Real, S>(v.by, v.npad, s, p, o);
            }
        }
        accum<NF, Real, Real>(o5n, o5b, tb[2 * smax + q], tb[3 * smax + q], m);
    }
    cta_partial<NV, NT, Real>(m, sh, part_out);
}

// Stage C of one tile: H3 from sh.M at r + h (gamma slot 0, [0]); error of
// the attempt; moments of the coarse result.
template <int NF, typename Real, int NT>
__device__ __forceinline__ void adapt_stage_c(const AdaptView<Real> v, int smax, const Real *tb, SharedA &sh,
                                              double *part_out)
{
    constexpr int S = Comp<NF>::S, NV = 2 * S;
    Real M0[S], M1[S];
    scaled_moments<S, Real>(sh.M, sh.mu[0], M0, M1);
    const Real A = (Real)sh.A[0];
    Real m[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) m[c] = Real(0);
    double emax = 0.0;
    for (int p = v.p0 + threadIdx.x; p < v.p1; p += NT) {
        const int j = p / v.n_E, e = p - j * v.n_E, q = j - v.j_lo;
        const Real gam = tb[q];
        Real g[S], hv[S], hn[S], hb[S];
#pragma unroll
        for (int c = 0; c < S; ++c) {
            g[c] = M0[c] - gam * M1[c];
            hv[c] = v.hvac[(size_t)e * S + c];
        }
        hamiltonians<NF, Real>(hv, A, g, hn, hb);
        const StepLen<Real> dlf = load_dl_at(tb, smax, ASlots<Real>::dl1, q);
        Real cn[S], cb[S];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Real r0[S], r6[S], r5[S];
            Real *rc = s ? cb : cn;
            load_state<Real, S>(v.b0, v.npad, s, p, r0);
            prop<NF, Real>(s ? hb : hn, dlf, r0, r6);
            load_state<Real, S>(v.by, v.npad, s, p, r5);
            load_state<Real, S>(v.bx, v.npad, s, p, rc);
            Real d[S];
#pragma unroll
            for (int c = 0; c < S; ++c) d[c] = rc[c] - Real(0.5) * (r5[c] + r6[c]);
            const double tr = v.trace[(size_t)s * v.npad + p];
            emax = nanmax(emax, (double)max_entry<NF, Real>(d) / fabs(tr));
        }
        accum<NF, Real, Real>(cn, cb, tb[2 * smax + q], tb[3 * smax + q], m);
    }
    cta_partial<NV, NT, Real>(m, sh, part_out);
    cta_max<NT>(emax, sh, part_out);
}

template <typename Real>
__device__ inline void adapt_tables(const Inst &in, Real *tb, int smax, int j_lo, int span, double rg_a, double rg_b,
                                    double rw1, double rw2, double rd1, double hd1, double rd2, double hd2)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        const int j = j_lo + q;
        double g, k, wa, wb;
        gamma_kappa(in, j, rg_a, &g, &k);
        tb[0 * smax + q] = (Real)g;
        if (rg_b > 0) {
            gamma_kappa(in, j, rg_b, &g, &k);
            tb[1 * smax + q] = (Real)g;
        }
        nu_weights(in, j, rw1, &wa, &wb);
        tb[2 * smax + q] = (Real)wa;
        tb[3 * smax + q] = (Real)wb;
        if (rw2 > 0) {
            nu_weights(in, j, rw2, &wa, &wb);
            tb[4 * smax + q] = (Real)wa;
            tb[5 * smax + q] = (Real)wb;
        }
        store_dl_at(tb, smax, ASlots<Real>::dl1, q, path_length(in, j, rd1, hd1));
        if (hd2 > 0) store_dl_at(tb, smax, ASlots<Real>::dl2, q, path_length(in, j, rd2, hd2));
    }
}

// Load the tile's progress copy into shared memory (all threads see it).
__device__ __forceinline__ void load_ts(const RunArgs &a, int t, SharedA &sh)
{
    __syncthreads();
    if (threadIdx.x == 0) sh.ts = a.tstate[t];
    __syncthreads();
}
__device__ __forceinline__ void store_ts(const RunArgs &a, int t, SharedA &sh)
{
    if (threadIdx.x == 0) a.tstate[t] = sh.ts;
    __syncthreads();
}

// Decide the attempt whose stage C partials sit in the slot 3 - in_slot.
template <int NT>
__device__ __forceinline__ void adapt_decide_tile(const RunArgs &a, const Inst &in, int t, int nv, SharedA &sh)
{
    const double *slotc = a.partials + (size_t)(3 - sh.ts.in_slot) * a.n_tiles * APS;
    adapt_total<NT>(slotc, in.tile_begin, in.tile_end, nv, in.dE, true, sh);
    if (threadIdx.x == 0) adapt_decide(in, sh.ts, sh.err, moments_finite(sh.M, nv));
    store_ts(a, t, sh);
}

// Resident CTAs per SM the register allocation is fitted to: stage A keeps
// two moment sets per thread, so the FP64 kernel stays at 2 (a third would
// spill about 1 KB per thread); FP32 fits 3; the 256-thread kernels 2.
__host__ __device__ constexpr int adapt_min_blocks(int nt, int real_bytes)
{
    return nt == 128 ? (real_bytes == 8 ? 2 : 3) : 2;
}

// NFM: 2 or 3 (all instances) or 0 (mixed pack).  a.n_steps = attempts in this launch.
template <int NFM, typename Real, int NT>
__global__ void __launch_bounds__(NT, adapt_min_blocks(NT, sizeof(Real))) xf_adapt_kernel(RunArgs a)
{
    extern __shared__ double s_dyn[];
    Real *const tb = (Real *)s_dyn;
    __shared__ SharedA sh;
    const int t_begin = a.cta_tiles[blockIdx.x], t_end = a.cta_tiles[blockIdx.x + 1];
    const int smax = a.span_max;
    const size_t slot_sz = (size_t)a.n_tiles * APS;
    unsigned nbar = 0;

    if (threadIdx.x == 0) sh.flag = *(volatile int *)a.err;
    __syncthreads();
    if (sh.flag) return;

    // ---- prologue: every tile copies its instance's progress; moments of rho0 at r into slot 0
    for (int t = t_begin; t < t_end; ++t) {
        const Tile tl = a.tiles[t];
        const Inst &in = a.inst[tl.inst];
        __syncthreads();
        if (threadIdx.x == 0) {
            sh.ts = a.apos[tl.inst];
            sh.ts.in_slot = 0;
            sh.ts.ran = (sh.ts.status == AD_RUN);
        }
        store_ts(a, t, sh);
        if (sh.ts.status != AD_RUN) continue;
        const int nf = NFM ? NFM : in.nf;
        const AdaptView<Real> v = adapt_view<Real>(a, in, tl, sh.ts.cur);
        const int span = (v.p1 - 1) / in.n_E - v.j_lo + 1;
        build_weight_table(in, tb, smax, v.j_lo, span, sh.ts.r);
        __syncthreads();
        TileView<Real> tv;
        tv.cur = v.b0;
        tv.n_E = v.n_E;
        tv.npad = v.npad;
        tv.p0 = v.p0;
        tv.p1 = v.p1;
        tv.j_lo = v.j_lo;
        double *out = a.partials + (size_t)t * APS;
        if (nf == 2) {
            if constexpr (NFM != 3) prologue_tile<2, Real, NT, VAR_PLAIN>(tv, smax, tb, sh, out);
        } else {
            if constexpr (NFM != 2) prologue_tile<3, Real, NT, VAR_PLAIN>(tv, smax, tb, sh, out);
        }
    }
    if (!grid_barrier(a, ++nbar, &sh.flag)) return;

    for (long long it = 0; it < a.n_steps; ++it) {
        // ---- stage A (opened by the decision on the previous attempt)
        for (int t = t_begin; t < t_end; ++t) {
            const Tile tl = a.tiles[t];
            const Inst &in = a.inst[tl.inst];
            const int nf = NFM ? NFM : in.nf, nv = 2 * (nf * nf - 1);
            load_ts(a, t, sh);
            if (sh.ts.status != AD_RUN) continue;
            if (it > 0) adapt_decide_tile<NT>(a, in, t, nv, sh);
            if (sh.ts.status != AD_RUN) continue;
            adapt_total<NT>(a.partials + (size_t)sh.ts.in_slot * slot_sz, in.tile_begin, in.tile_end, nv, in.dE,
                            false, sh);
            if (threadIdx.x == 0) {
                if (!moments_finite(sh.M, nv)) {
                    sh.ts.status = AD_NONFINITE;
                } else {
                    sh.ts.last = (sh.ts.h >= sh.ts.r_end - sh.ts.r);
                    sh.ts.ht = sh.ts.last ? sh.ts.r_end - sh.ts.r : sh.ts.h;
                    sh.mu[0] = mu_eff(in, sh.ts.r);
                    sh.A[0] = matter_A(in, sh.ts.r);
                }
            }
            store_ts(a, t, sh);
            if (sh.ts.status != AD_RUN) continue;
            const double r = sh.ts.r, h = sh.ts.ht;
            const AdaptView<Real> v = adapt_view<Real>(a, in, tl, sh.ts.cur);
            const int span = (v.p1 - 1) / in.n_E - v.j_lo + 1;
            adapt_tables(in, tb, smax, v.j_lo, span, r, -1.0, r + h, r + 0.5 * h, r, h, r, 0.5 * h);
            __syncthreads();
            double *out = a.partials + 1 * slot_sz + (size_t)t * APS;
            if (nf == 2) {
                if constexpr (NFM != 3) adapt_stage_a<2, Real, NT>(v, smax, tb, sh, out);
            } else {
                if constexpr (NFM != 2) adapt_stage_a<3, Real, NT>(v, smax, tb, sh, out);
            }
        }
        if (!grid_barrier(a, ++nbar, &sh.flag)) return;

        // ---- stage B
        for (int t = t_begin; t < t_end; ++t) {
            const Tile tl = a.tiles[t];
            const Inst &in = a.inst[tl.inst];
            const int nf = NFM ? NFM : in.nf, nv = 2 * (nf * nf - 1);
            load_ts(a, t, sh);
            if (sh.ts.status != AD_RUN) continue;
            adapt_total<NT>(a.partials + 1 * slot_sz, in.tile_begin, in.tile_end, 2 * nv, in.dE, false, sh);
            const double r = sh.ts.r, h = sh.ts.ht;
            if (threadIdx.x == 0) {
                if (!moments_finite(sh.M, 2 * nv)) {
                    sh.ts.status = AD_NONFINITE;
                } else {
                    sh.mu[0] = mu_eff(in, r + h);
                    sh.A[0] = matter_A(in, r + h);
                    sh.mu[1] = mu_eff(in, r + 0.5 * h);
                    sh.A[1] = matter_A(in, r + 0.5 * h);
                }
            }
            store_ts(a, t, sh);
            if (sh.ts.status != AD_RUN) continue;
            // the stage A pair came out as [H1 set | H2 set], each nv long
            const AdaptView<Real> v = adapt_view<Real>(a, in, tl, sh.ts.cur);
            const int span = (v.p1 - 1) / in.n_E - v.j_lo + 1;
            adapt_tables(in, tb, smax, v.j_lo, span, r + h, r + 0.5 * h, r + h, -1.0, r, h, r + 0.5 * h, 0.5 * h);
            __syncthreads();
            double *out = a.partials + 2 * slot_sz + (size_t)t * APS;
            if (nf == 2) {
                if constexpr (NFM != 3) adapt_stage_b<2, Real, NT>(v, smax, tb, sh, out);
            } else {
                if constexpr (NFM != 2) adapt_stage_b<3, Real, NT>(v, smax, tb, sh, out);
            }
        }
        if (!grid_barrier(a, ++nbar, &sh.flag)) return;

        // ---- stage C
        for (int t = t_begin; t < t_end; ++t) {
            const Tile tl = a.tiles[t];
            const Inst &in = a.inst[tl.inst];
            const int nf = NFM ? NFM : in.nf, nv = 2 * (nf * nf - 1);
            load_ts(a, t, sh);
            if (sh.ts.status != AD_RUN) continue;
            adapt_total<NT>(a.partials + 2 * slot_sz, in.tile_begin, in.tile_end, nv, in.dE, false, sh);
            const double r = sh.ts.r, h = sh.ts.ht;
            if (threadIdx.x == 0) {
                if (!moments_finite(sh.M, nv)) {
                    sh.ts.status = AD_NONFINITE;
                } else {
                    sh.mu[0] = mu_eff(in, r + h);
                    sh.A[0] = matter_A(in, r + h);
                }
            }
            store_ts(a, t, sh);
            if (sh.ts.status != AD_RUN) continue;
            const AdaptView<Real> v = adapt_view<Real>(a, in, tl, sh.ts.cur);
            const int span = (v.p1 - 1) / in.n_E - v.j_lo + 1;
            adapt_tables(in, tb, smax, v.j_lo, span, r + h, -1.0, r + h, -1.0, r, h, 0.0, -1.0);
            __syncthreads();
            double *out = a.partials + (size_t)(3 - sh.ts.in_slot) * slot_sz + (size_t)t * APS;
            if (nf == 2) {
                if constexpr (NFM != 3) adapt_stage_c<2, Real, NT>(v, smax, tb, sh, out);
            } else {
                if constexpr (NFM != 2) adapt_stage_c<3, Real, NT>(v, smax, tb, sh, out);
            }
        }
        if (!grid_barrier(a, ++nbar, &sh.flag)) return;
    }

    // ---- epilogue: decide the last attempt; the owner tile publishes progress and moments
    for (int t = t_begin; t < t_end; ++t) {
        const Tile tl = a.tiles[t];
        const Inst &in = a.inst[tl.inst];
        const int nf = NFM ? NFM : in.nf, nv = 2 * (nf * nf - 1);
        load_ts(a, t, sh);
        if (sh.ts.status == AD_RUN && a.n_steps > 0) adapt_decide_tile<NT>(a, in, t, nv, sh);
        if (t != in.tile_begin || !sh.ts.ran) continue;
        if (sh.ts.status != AD_NONFINITE) {
            adapt_total<NT>(a.partials + (size_t)sh.ts.in_slot * slot_sz, in.tile_begin, in.tile_end, nv, in.dE,
                            false, sh);
            if (threadIdx.x < nv) a.mom_out[(size_t)tl.inst * NVMAX + threadIdx.x] = sh.M[threadIdx.x];
        }
        if (threadIdx.x == 0) a.apos[tl.inst] = sh.ts;
        __syncthreads();
    }
}

} // namespace xf
