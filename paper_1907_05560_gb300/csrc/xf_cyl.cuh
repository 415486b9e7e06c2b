// xf_cyl.cuh -- the integrator kernel of the cylinder/line model (Sec. 3.2.5,
// Eq. 3.20): an infinite cylinder of radius R emits perpendicular to its
// axis; trajectory t = j n_phi + k leaves latitude Phi_k = (k + 1/2) 2 pi/n_phi
// at the angle theta_j = -pi/2 + (j + 1/2) pi/n_u from the outward normal
// (positive clockwise).  At radius r it runs at alpha_j = asin(x sin theta_j)
// to the radial direction (x = R/r), so dl/dr = 1/cos(alpha_j), and
//   G_t = mu0 x dE sum_j' w_j' [1 - cos(alpha_j - alpha_j')] D(Phi', j'),
//   w_j' = cos(theta_j') / cos(alpha_j') dtheta,
//   Phi' = Phi_k + (theta_j' - alpha_j') - (theta_j - alpha_j),
// with D(k, j') = sum_E (rho_nu - conj rho_nubar) of trajectory (j', k) and
// D(Phi', j') read by periodic linear interpolation between latitude bins.
//
// G is not a sum of a few moments: every trajectory couples to every angle
// bin at its own latitude offset.  So a stage is: per trajectory, G from the
// previous stage's per-trajectory sums D (FP64, L2-resident, read with
// .cg loads), the per-bin update of its 2 n_E bins, and its new D; one grid
// barrier per stage as in the bulb kernel.  A warp owns a trajectory: lanes
// split the angle sum of G, then the energy bins; both warp sums run in a
// fixed shuffle tree, so runs are bitwise reproducible.  One problem per
// launch; CTA c owns the trajectories of tile c.
#pragma once

#include "xf_run.cuh"

namespace xf {

constexpr int CYL_MAX_U = 2048; // angle bins held in the shared-memory table (4 doubles each)
constexpr int CYL_DS = 8;       // doubles per trajectory sum (S <= 8)
constexpr int CYL_NT = 128;

// Angle bin j at radius r: beta = theta - alpha, the coupling weight
// wc = cos(theta) / cos(alpha) dtheta, cos(alpha), sin(alpha).
__device__ __forceinline__ void cyl_angle(const Inst &a, int j, double r, double *beta, double *wc, double *ca,
                                          double *sa)
{
    const double pi = 3.14159265358979323846;
    const double th = -0.5 * pi + (j + 0.5) * pi / a.n_u;
    double st, ct;
    sincos(th, &st, &ct);
    const double s = (a.R / r) * st, c = sqrt(1.0 - s * s);
    *beta = th - asin(s);
    *wc = ct / c * (pi / a.n_u);
    *ca = c;
    *sa = s;
}

// Path length from r to r + h on a ray of impact parameter b = R sin(theta_j):
// l = sqrt(r^2 - b^2), so l(r + h) - l(r) = h (2r + h) / (l(r) + l(r + h)).
__device__ __forceinline__ double cyl_path_length(const Inst &a, int j, double r, double h)
{
    const double pi = 3.14159265358979323846;
    const double b = a.R * sin(-0.5 * pi + (j + 0.5) * pi / a.n_u), b2 = b * b;
    return h * (2.0 * r + h) / (sqrt(r * r - b2) + sqrt((r + h) * (r + h) - b2));
}

// Sum over the warp's lanes into every lane (fixed tree to lane 0, then broadcast).
template <int N>
__device__ __forceinline__ void warp_sum_bcast(double *x)
{
#pragma unroll
    for (int c = 0; c < N; ++c) {
        double v = x[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        x[c] = __shfl_sync(0xffffffffu, v, 0);
    }
}

// One stage of one bin pair (nu, nubar at pair p): the bulb kernel's RK4 or
// predictor-corrector stage; on / ob receive the stage outputs.
template <int NF, int STEP, typename Real>
__device__ __forceinline__ void cyl_pair_stage(const TileView<Real> &v, int st, int p, const Real *hn, const Real *hb,
                                               Real kap, StepLen<Real> dl, Real cy, Real cb, Real *on, Real *ob)
{
    constexpr int S = Comp<NF>::S;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        Real *o = (s == 0) ? on : ob;
        if constexpr (STEP == STEP_RK4) {
            Real y[S], kk[S], rn[S], bb[S];
            if (st == 0) load_state<Real, S>(v.cur, v.npad, s, p, y);
            else load_state<Real, S>(v.aux, v.npad, s, p, y);
            comm<NF, Real>(s == 0 ? hn : hb, y, kk);
#pragma unroll
            for (int c = 0; c < S; ++c) kk[c] *= kap;
            if (st == 0) {
#pragma unroll
                for (int c = 0; c < S; ++c) rn[c] = y[c];
            } else if (st < 3) {
                load_state<Real, S>(v.cur, v.npad, s, p, rn);
            }
            if (st == 0) {
#pragma unroll
                for (int c = 0; c < S; ++c) bb[c] = rn[c] + cb * kk[c];
            } else {
                load_state<Real, S>(v.nxt, v.npad, s, p, bb);
#pragma unroll
                for (int c = 0; c < S; ++c) bb[c] += cb * kk[c];
            }
            store_state<Real, S>(v.nxt, v.npad, s, p, bb);
            if (st < 3) {
#pragma unroll
                for (int c = 0; c < S; ++c) o[c] = rn[c] + cy * kk[c];
                store_state<Real, S>(v.aux, v.npad, s, p, o);
            } else {
#pragma unroll
                for (int c = 0; c < S; ++c) o[c] = bb[c];
            }
        } else {
            Real rn[S], pr[S];
            load_state<Real, S>(v.cur, v.npad, s, p, rn);
            prop<NF, Real>(s == 0 ? hn : hb, dl, rn, pr);
            if (st == 0) {
#pragma unroll
                for (int c = 0; c < S; ++c) o[c] = pr[c];
                store_state<Real, S>(v.aux, v.npad, s, p, o);
            } else {
                Real pp[S];
                load_state<Real, S>(v.aux, v.npad, s, p, pp);
#pragma unroll
                for (int c = 0; c < S; ++c) o[c] = Real(0.5) * (pp[c] + pr[c]);
                store_state<Real, S>(v.nxt, v.npad, s, p, o);
            }
        }
    }
}

// Write trajectory t's sum (lane 0) and flag a non-finite one with the
// barrier number after which it is read.
template <int S>
__device__ __forceinline__ void cyl_store_sum(const RunArgs &a, double *Dout, int t, const double *d, unsigned nb)
{
    if ((threadIdx.x & 31) == 0) {
        bool ok = true;
#pragma unroll
        for (int c = 0; c < S; ++c) {
            __stcg(Dout + (size_t)t * CYL_DS + c, d[c]);
            ok = ok && isfinite(d[c]);
        }
        if (!ok) atomicMin(a.first_bad, nb);
    }
}

template <int NF, int STEP, typename Real>
__global__ void __launch_bounds__(CYL_NT, min_blocks(128, sizeof(Real))) xf_cyl_kernel(RunArgs a)
{
    constexpr int S = Comp<NF>::S, NT = CYL_NT, NW = NT / 32;
    extern __shared__ double s_dyn[];
    __shared__ int s_flag;
    const Inst &in = a.inst[0];
    const int nu = in.n_u, nphi = in.n_phi;
    double *const tb_beta = s_dyn, *const tb_wc = s_dyn + nu, *const tb_ca = s_dyn + 2 * nu,
                  *const tb_sa = s_dyn + 3 * nu;
    const Tile tl = a.tiles[blockIdx.x];
    const int t_a = tl.p0 / in.n_E, t_b = (tl.p0 + tl.np) / in.n_E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned nbar = 0;

    // an earlier launch on these buffers failed at a barrier: touch nothing
    if (threadIdx.x == 0) s_flag = *(volatile int *)a.err;
    __syncthreads();
    if (s_flag) return;
    const InstPos ps = a.pos[0];
    const long long n = launch_steps(a, ps);
    if (n <= 0) return; // every CTA sees the same n
    double *const Dbuf[2] = {a.partials, a.partials + (size_t)nu * nphi * CYL_DS};
    const double inv_dphi = nphi / (2.0 * 3.14159265358979323846);

    // ---- prologue: per-trajectory sums of the input state
    {
        const TileView<Real> v = make_view<Real>(a, in, ps, tl, 0);
        for (int t = t_a + warp; t < t_b; t += NW) {
            double d[S];
#pragma unroll
            for (int c = 0; c < S; ++c) d[c] = 0.0;
            for (int e = lane; e < in.n_E; e += 32) {
                const int p = t * in.n_E + e;
                Real tn[S], tb[S], dd[S];
                load_state<Real, S>(v.cur, v.npad, 0, p, tn);
                load_state<Real, S>(v.cur, v.npad, 1, p, tb);
                nu_minus_conj_nubar<NF, Real>(tn, tb, dd);
#pragma unroll
                for (int c = 0; c < S; ++c) d[c] += (double)dd[c];
            }
            warp_sum_bcast<S>(d);
            cyl_store_sum<S>(a, Dbuf[0], t, d, 1u);
        }
    }
    if (!grid_barrier(a, ++nbar, &s_flag)) return;

    constexpr int NSTAGE = (STEP == STEP_RK4) ? 4 : 2;
    for (long long k = 0; k < n; ++k) {
#pragma unroll 1
        for (int st = 0; st < NSTAGE; ++st) {
            // the stage input's sums were written before barrier nbar: a
            // non-finite one stops the run (every CTA reads the same value)
            if (*(volatile unsigned *)a.first_bad <= nbar) {
                if (blockIdx.x == 0 && threadIdx.x == 0)
                    advance(a.pos, (st == 0) ? (k > 0 ? k - 1 : 0) : k, ERR_NONFINITE);
                return;
            }
            const double kk = (double)(ps.k0 + k), h = in.h;
            const double r = in.r0 + kk * h, r_half = in.r0 + (kk + 0.5) * h, r_next = in.r0 + (kk + 1.0) * h;
            double r_rhs;
            if constexpr (STEP == STEP_RK4) r_rhs = (st == 0) ? r : (st == 3 ? r_next : r_half);
            else r_rhs = (st == 0) ? r : r_next;
            const double mu = mu_eff(in, r_rhs) * in.dE;
            const Real A = (Real)matter_A(in, r_rhs);
            const Real cy = (Real)((st == 2) ? h : 0.5 * h);
            const Real cb = (Real)((st == 0 || st == 3) ? h / 6.0 : h / 3.0);
            __syncthreads(); // the previous stage's readers of the table are done
            for (int j = threadIdx.x; j < nu; j += NT) cyl_angle(in, j, r_rhs, tb_beta + j, tb_wc + j, tb_ca + j, tb_sa + j);
            __syncthreads();
            const TileView<Real> v = make_view<Real>(a, in, ps, tl, k);
            const double *const Din = Dbuf[(nbar - 1) & 1];
            double *const Dout = Dbuf[nbar & 1];
            for (int t = t_a + warp; t < t_b; t += NW) {
                const int j = t / nphi, kl = t - j * nphi;
                const double beta_j = tb_beta[j], ca_j = tb_ca[j], sa_j = tb_sa[j];
                // G of the trajectory: lanes split the angle bins j'
                double g[S];
#pragma unroll
                for (int c = 0; c < S; ++c) g[c] = 0.0;
                for (int jp = lane; jp < nu; jp += 32) {
                    const double pos = kl + (tb_beta[jp] - beta_j) * inv_dphi;
                    const double fl = floor(pos), f = pos - fl;
                    int i0 = (int)fl % nphi;
                    if (i0 < 0) i0 += nphi;
                    const int i1 = (i0 + 1 == nphi) ? 0 : i0 + 1;
                    const double K = tb_wc[jp] * (1.0 - (ca_j * tb_ca[jp] + sa_j * tb_sa[jp]));
                    const double K0 = K * (1.0 - f), K1 = K * f;
                    const double *d0 = Din + (size_t)(jp * nphi + i0) * CYL_DS;
                    const double *d1 = Din + (size_t)(jp * nphi + i1) * CYL_DS;
#pragma unroll
                    for (int c = 0; c < S; ++c) g[c] += K0 * __ldcg(d0 + c) + K1 * __ldcg(d1 + c);
                }
                warp_sum_bcast<S>(g);
                Real gr[S];
#pragma unroll
                for (int c = 0; c < S; ++c) gr[c] = (Real)(mu * g[c]);
                const Real kap = (Real)(1.0 / ca_j);
                const StepLen<Real> dl = make_step_len(STEP == STEP_EXPH ? cyl_path_length(in, j, r, h) : 0.0,
                                                       (Real *)nullptr);
                // the trajectory's bins: lanes split the energies
                double d[S];
#pragma unroll
                for (int c = 0; c < S; ++c) d[c] = 0.0;
                for (int e = lane; e < in.n_E; e += 32) {
                    const int p = t * in.n_E + e;
                    Real hv[S], hn[S], hb[S], on[S], ob[S], dd[S];
#pragma unroll
                    for (int c = 0; c < S; ++c) hv[c] = v.hvac[(size_t)e * S + c];
                    hamiltonians<NF, Real>(hv, A, gr, hn, hb);
                    cyl_pair_stage<NF, STEP, Real>(v, st, p, hn, hb, kap, dl, cy, cb, on, ob);
                    nu_minus_conj_nubar<NF, Real>(on, ob, dd);
#pragma unroll
                    for (int c = 0; c < S; ++c) d[c] += (double)dd[c];
                }
                warp_sum_bcast<S>(d);
                cyl_store_sum<S>(a, Dout, t, d, nbar + 1);
            }
            if (!grid_barrier(a, ++nbar, &s_flag)) return;
        }
    }
    // the last stage's sums: a non-finite one leaves the last step's input
    // as the last finite state
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const bool bad = *(volatile unsigned *)a.first_bad <= nbar;
        advance(a.pos, bad ? n - 1 : n, bad ? ERR_NONFINITE : 0);
    }
}

} // namespace xf
