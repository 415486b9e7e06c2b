// xf_psi.cuh -- the wavefunction form of the per-bin update (Eq. 3.1, 3.4,
// 3.9-3.11): each bin carries one wavefunction psi_a (n_f complex components)
// per initial flavor a, rho = sum_a phi_a psi_a psi_a^+ with phi_a the flavor's
// number-flux weight, and every psi evolves with the Hamiltonian of rho.
//
// State: 2 n_f^2 reals per bin (8 or 18), component c = (a n_f + i) 2 + re/im,
// stored like the density-matrix form's planes: element (c, s, p) at
// (c 2 + s) npad + p.  Packed Hamiltonians follow the density-matrix packing:
// (a, x, y) is [[a, x + i y], [x - i y, -a]]; in three flavors (d0, d1, Re/Im
// of the (0,1), (0,2), (1,2) entries), d2 = -(d0 + d1).
#pragma once

#include "xf_math.cuh"

namespace xf {

template <int NF> struct PsiComp { static constexpr int SS = 2 * NF * NF; };

// y = H x for one complex vector (re/im interleaved), H packed traceless.
template <int NF, typename Real>
__host__ __device__ __forceinline__ void h_apply(const Real *h, const Real *x, Real *y)
{
    if constexpr (NF == 2) {
        // (a p + (hx + i hy) q, (hx - i hy) p - a q)
        const Real pr = x[0], pi = x[1], qr = x[2], qi = x[3];
        y[0] = h[0] * pr + h[1] * qr - h[2] * qi;
        y[1] = h[0] * pi + h[1] * qi + h[2] * qr;
        y[2] = h[1] * pr + h[2] * pi - h[0] * qr;
        y[3] = h[1] * pi - h[2] * pr - h[0] * qi;
    } else {
        const cx<Real> H01 = mk(h[2], h[3]), H02 = mk(h[4], h[5]), H12 = mk(h[6], h[7]);
        const Real d2 = -(h[0] + h[1]);
        const cx<Real> x0 = mk(x[0], x[1]), x1 = mk(x[2], x[3]), x2 = mk(x[4], x[5]);
        const cx<Real> y0 = h[0] * x0 + H01 * x1 + H02 * x2;
        const cx<Real> y1 = cj(H01) * x0 + h[1] * x1 + H12 * x2;
        const cx<Real> y2 = cj(H02) * x0 + cj(H12) * x1 + d2 * x2;
        y[0] = y0.r;
        y[1] = y0.i;
        y[2] = y1.r;
        y[3] = y1.i;
        y[4] = y2.r;
        y[5] = y2.i;
    }
}

// psi' = exp(-i H dl) psi for the NF wavefunctions of one bin.
//   2 flavors (Eq. 3.11): cos(lam dl) psi - i sin(lam dl)/lam H psi, lam^2 = a^2 + |H01|^2;
//   3 flavors: H = V diag(lam) V^+ (cyclic Jacobi), psi' = V (exp(-i lam dl) o (V^+ psi)).
template <int NF, typename Real>
__host__ __device__ __forceinline__ void prop_psi(const Real *h, StepLen<Real> dl, const Real *x, Real *y)
{
    constexpr int N2 = 2 * NF;
    if constexpr (NF == 2) {
        Real sn, cs, sig;
        rotation_angle(h, dl, &sn, &cs, &sig);
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            Real hx[N2];
            h_apply<NF, Real>(h, x + a * N2, hx);
#pragma unroll
            for (int i = 0; i < NF; ++i) { // cs x - i sig (Hx)
                y[a * N2 + 2 * i] = cs * x[a * N2 + 2 * i] + sig * hx[2 * i + 1];
                y[a * N2 + 2 * i + 1] = cs * x[a * N2 + 2 * i + 1] - sig * hx[2 * i];
            }
        }
    } else {
        Real dg[3];
        cx<Real> V[3][3];
        eig3<Real>(h, dg, V);
        cx<Real> e[3];
        // exp(-i lam_j dl) for j = 0, 1; lam_2 = -(lam_0 + lam_1) (H traceless)
        // gives the third as conj(e_0 e_1)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            Real sn, cs;
            phase_sincos(dg[j], dl, &sn, &cs);
            e[j] = mk(cs, -sn);
        }
        e[2] = cj(e[0] * e[1]);
#pragma unroll
        for (int a = 0; a < NF; ++a) {
            const cx<Real> x0 = mk(x[a * N2 + 0], x[a * N2 + 1]), x1 = mk(x[a * N2 + 2], x[a * N2 + 3]),
                           x2 = mk(x[a * N2 + 4], x[a * N2 + 5]);
            cx<Real> w[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) w[j] = e[j] * cfmac(x2, V[2][j], cfmac(x1, V[1][j], mulc(x0, V[0][j])));
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const cx<Real> z = cfma(V[i][2], w[2], cfma(V[i][1], w[1], V[i][0] * w[0]));
                y[a * N2 + 2 * i] = z.r;
                y[a * N2 + 2 * i + 1] = z.i;
            }
        }
    }
}

// k = -i kappa H psi for the NF wavefunctions of one bin.
template <int NF, typename Real>
__host__ __device__ __forceinline__ void rhs_psi(const Real *h, Real kappa, const Real *x, Real *k)
{
    constexpr int N2 = 2 * NF;
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        Real hx[N2];
        h_apply<NF, Real>(h, x + a * N2, hx);
#pragma unroll
        for (int i = 0; i < NF; ++i) { // -i (u + i v) = v - i u
            k[a * N2 + 2 * i] = kappa * hx[2 * i + 1];
            k[a * N2 + 2 * i + 1] = -kappa * hx[2 * i];
        }
    }
}

// Traceless packed part of rho = sum_a w_a psi_a psi_a^+ (w_0: the e flavor's
// weight, w_1: the others'); *tr = its trace.
template <int NF, typename Real>
__host__ __device__ __forceinline__ void psi_rho(const Real *x, Real w0, Real w1, Real *t, Real *tr)
{
    constexpr int N2 = 2 * NF;
    Real d[NF];
    cx<Real> o[3] = {mk(Real(0), Real(0)), mk(Real(0), Real(0)), mk(Real(0), Real(0))};
#pragma unroll
    for (int i = 0; i < NF; ++i) d[i] = Real(0);
#pragma unroll
    for (int a = 0; a < NF; ++a) {
        const Real w = a == 0 ? w0 : w1;
        const Real *v = x + a * N2;
#pragma unroll
        for (int i = 0; i < NF; ++i) d[i] += w * (v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1]);
        // upper entries psi_i conj(psi_j): (0,1), (0,2), (1,2)
        o[0] = o[0] + w * mulc(mk(v[0], v[1]), mk(v[2], v[3]));
        if constexpr (NF == 3) {
            o[1] = o[1] + w * mulc(mk(v[0], v[1]), mk(v[4], v[5]));
            o[2] = o[2] + w * mulc(mk(v[2], v[3]), mk(v[4], v[5]));
        }
    }
    if constexpr (NF == 2) {
        *tr = d[0] + d[1];
        t[0] = Real(0.5) * (d[0] - d[1]);
        t[1] = o[0].r;
        t[2] = o[0].i;
    } else {
        *tr = d[0] + d[1] + d[2];
        const Real tau = *tr / Real(3);
        t[0] = d[0] - tau;
        t[1] = d[1] - tau;
        t[2] = o[0].r;
        t[3] = o[0].i;
        t[4] = o[1].r;
        t[5] = o[1].i;
        t[6] = o[2].r;
        t[7] = o[2].i;
    }
}

} // namespace xf
