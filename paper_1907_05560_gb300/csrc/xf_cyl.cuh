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
// bin at its own latitude offset.  A stage runs, per chunk of up to 128 of the
// CTA's trajectories:
//   1. when the chunk's trajectories have at most two distinct angle bins j
//      (always when n_phi >= 127), their coupling rows: per background bin j'
//      the weights K (1 - f), K f and the latitude offset floor(x) of
//      x = (Phi' - Phi) / dPhi, in shared memory (else each thread computes
//      its own);
//   2. G of every trajectory of the chunk, one thread each, from the previous
//      stage's per-trajectory sums D (FP64, component-major [c][t] so that
//      neighbouring latitudes read neighbouring words; L2-resident, read with
//      .cg loads because other SMs wrote them);
//   3. the chunk's bins, one warp per trajectory, lanes over the energies, the
//      bulb kernel's per-bin update, and the trajectory's new D from a fixed
//      shuffle tree (so runs are bitwise reproducible);
// then one grid barrier, as in the bulb kernel.  One problem per launch; CTA c
// owns the trajectories of tile c.
#pragma once

#include "xf_run.cuh"

namespace xf {

constexpr int CYL_MAX_U = 2048; // angle bins held in the shared-memory tables (9 doubles each)
constexpr int CYL_DS = 8;       // components of a trajectory sum slot (S <= 8); D[slot][c][T]
constexpr int CYL_NT = 128;
constexpr int CYL_ROWS = 2;     // coupling rows held per chunk

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

// Coupling of angle bin j to background bin jp from the angle table: the
// interpolation weights K (1 - f), K f and the latitude offset floor(x) mod
// n_phi, x = (Phi' - Phi) / dPhi = ((theta' - alpha') - (theta - alpha)) / dPhi.
__device__ __forceinline__ void cyl_coupling(const double *tb_beta, const double *tb_wc, const double *tb_ca,
                                             const double *tb_sa, int nu, int nphi, double inv_dphi, int j, int jp,
                                             double *K0, double *K1, int *off)
{
    const double x = (tb_beta[jp] - tb_beta[j]) * inv_dphi;
    const double fl = floor(x), f = x - fl;
    int o = (int)fl % nphi;
    if (o < 0) o += nphi;
    const double K = tb_wc[jp] * (1.0 - (tb_ca[j] * tb_ca[jp] + tb_sa[j] * tb_sa[jp]));
    *K0 = K * (1.0 - f);
    *K1 = K * f;
    *off = o;
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
__device__ __forceinline__ void cyl_store_sum(const RunArgs &a, double *Dout, int T, int t, const double *d,
                                              unsigned nb)
{
    if ((threadIdx.x & 31) == 0) {
        bool ok = true;
#pragma unroll
        for (int c = 0; c < S; ++c) {
            __stcg(Dout + (size_t)c * T + t, d[c]);
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
    __shared__ double s_G[NT][S]; // G of the chunk's trajectories (mu dE applied)
    __shared__ int s_flag;
    const Inst &in = a.inst[0];
    const int nu = in.n_u, nphi = in.n_phi, T = nu * nphi;
    // dynamic shared memory: the angle table (4 nu doubles), then the
    // coupling rows (2 CYL_ROWS nu doubles, CYL_ROWS nu ints)
    double *const tb_beta = s_dyn, *const tb_wc = s_dyn + nu, *const tb_ca = s_dyn + 2 * nu,
                  *const tb_sa = s_dyn + 3 * nu;
    double *const rK0 = s_dyn + 4 * nu, *const rK1 = s_dyn + (4 + CYL_ROWS) * nu;
    int *const rOff = (int *)(s_dyn + (4 + 2 * CYL_ROWS) * nu);
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
    double *const Dbuf[2] = {a.partials, a.partials + (size_t)CYL_DS * T};
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
            cyl_store_sum<S>(a, Dbuf[0], T, t, d, 1u);
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
            __syncthreads(); // the previous stage's readers of the tables are done
            for (int j = threadIdx.x; j < nu; j += NT) cyl_angle(in, j, r_rhs, tb_beta + j, tb_wc + j, tb_ca + j, tb_sa + j);
            __syncthreads();
            const TileView<Real> v = make_view<Real>(a, in, ps, tl, k);
            const double *const Din = Dbuf[(nbar - 1) & 1];
            double *const Dout = Dbuf[nbar & 1];
            for (int c0 = t_a; c0 < t_b; c0 += NT) {
                const int c1 = min(c0 + NT, t_b);
                const int j_lo = c0 / nphi, rows = (c1 - 1) / nphi - j_lo + 1;
                const bool tab = rows <= CYL_ROWS;
                // 1. the chunk's coupling rows
                if (tab)
                    for (int q = threadIdx.x; q < rows * nu; q += NT) {
                        const int row = q / nu, jp = q - row * nu;
                        cyl_coupling(tb_beta, tb_wc, tb_ca, tb_sa, nu, nphi, inv_dphi, j_lo + row, jp,
                                     rK0 + row * nu + jp, rK1 + row * nu + jp, rOff + row * nu + jp);
                    }
                __syncthreads();
                // 2. G, one thread per trajectory
                const int t = c0 + (int)threadIdx.x;
                if (t < c1) {
                    const int j = t / nphi, kl = t - j * nphi, row = j - j_lo;
                    double g[S];
#pragma unroll
                    for (int c = 0; c < S; ++c) g[c] = 0.0;
                    for (int jp = 0; jp < nu; ++jp) {
                        double K0, K1;
                        int off;
                        if (tab) {
                            K0 = rK0[row * nu + jp];
                            K1 = rK1[row * nu + jp];
                            off = rOff[row * nu + jp];
                        } else {
                            cyl_coupling(tb_beta, tb_wc, tb_ca, tb_sa, nu, nphi, inv_dphi, j, jp, &K0, &K1, &off);
                        }
                        int i0 = kl + off;
                        if (i0 >= nphi) i0 -= nphi;
                        const int i1 = (i0 + 1 == nphi) ? 0 : i0 + 1;
                        const double *const Dj = Din + (size_t)jp * nphi;
#pragma unroll
                        for (int c = 0; c < S; ++c)
                            g[c] = fma(K0, __ldcg(Dj + (size_t)c * T + i0), fma(K1, __ldcg(Dj + (size_t)c * T + i1), g[c]));
                    }
#pragma unroll
                    for (int c = 0; c < S; ++c) s_G[threadIdx.x][c] = mu * g[c];
                }
                __syncthreads();
                // 3. the bins, one warp per trajectory
                for (int tt = c0 + warp; tt < c1; tt += NW) {
                    const int j = tt / nphi;
                    Real gr[S];
#pragma unroll
                    for (int c = 0; c < S; ++c) gr[c] = (Real)s_G[tt - c0][c];
                    const Real kap = (Real)(1.0 / tb_ca[j]);
                    const StepLen<Real> dl = make_step_len(STEP == STEP_EXPH ? cyl_path_length(in, j, r, h) : 0.0,
                                                           (Real *)nullptr);
                    double d[S];
#pragma unroll
                    for (int c = 0; c < S; ++c) d[c] = 0.0;
                    for (int e = lane; e < in.n_E; e += 32) {
                        const int p = tt * in.n_E + e;
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
                    cyl_store_sum<S>(a, Dout, T, tt, d, nbar + 1);
                }
                __syncthreads(); // the chunk's G and rows are consumed
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
