/*
 * xf_oracle.c -- plain FP64 CPU oracle for multi-angle collective neutrino
 * flavor evolution in the neutrino bulb model (XFLAT, arXiv 1907.05560).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path.  Only
 * tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py may build, load or call it.  It shares no code, header, table or
 * constant with the CUDA library: every formula below is written out again
 * from the paper.
 *
 * Representation: every density matrix is a full n_f x n_f complex matrix
 * (C99 double complex), trace included, exactly as Eq. 3.8-3.9 use it.  Bins
 * are ordered [s][u][E] with s = 0 for neutrinos and s = 1 for antineutrinos.
 *
 * What is computed (section / equation of the paper):
 *   - vacuum Hamiltonian      Eq. 3.5-3.6 (2 flavors); 3 flavors: the same
 *                             mass-basis form (1/2E) U diag(0, dm21, dm31) U^T
 *   - matter potential        Eq. 3.7, profiles Eq. 4.3 (power law) / Eq. 4.4
 *   - antineutrino rule       A -> -A, B -> -B, B_et -> -B_et*  (after Eq. 3.4)
 *   - nu-nu potential         Eq. 3.13 with the bulb geometry Eq. 3.14-3.15;
 *                             single-angle form Eq. 3.16-3.17; the extended
 *                             bulb Eq. 3.18; the cylinder/line model Eq. 3.20
 *   - trajectory length       Eq. 3.3 (l = r cos(theta))
 *   - spectra                 Eq. 4.1-4.2 (Fermi-Dirac, 1/(exp(E/T-eta)+1))
 *   - propagator              Eq. 3.10-3.12 (2 flavors); 3 flavors: spectral
 *                             exponential from a complex Jacobi eigensolver
 *   - integrators             classic RK4 on d(rho)/dr = -i[H,rho] dl/dr, and
 *                             the fixed-step coarse predictor-corrector of
 *                             Sec. 4.2.3 / Listing 5.1 (S1-S3) in rho form;
 *                             either optionally renormalised after each step
 *                             to the entry tr(T^2) (a constant of Eq. 3.10)
 *
 * Readings taken where the paper is silent:
 *   angle variable u = sin^2(theta_0) on a midpoint grid; energy midpoint grid;
 *   rho's diagonal carries the number-flux weights phi_a(E) relative to nu_e;
 *   mu0 absorbs the normalisation of Eq. 3.8; the predictor-corrector averages
 *   density matrices; the step path length is the exact chord of Eq. 3.3.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
#define NFMAX 3

/* ---- parameters (layout mirrored by oracle/oracle.py) ------------------- */
enum { ORC_RK4 = 0, ORC_EXPH = 1 };
enum { ORC_BULB = 0, ORC_MU_R4 = 1, ORC_SINGLE_ANGLE = 2, ORC_CONST = 3, ORC_CYLINDER = 4 };
enum { ORC_MATTER_NONE = 0, ORC_MATTER_POWER = 1, ORC_MATTER_EXP = 2 };

typedef struct {
    int32_t n_E, n_u, n_f, stepper, geometry, hierarchy, matter, n_threads;
    int32_t renorm;   /* 1: after every step, scale each bin's traceless part back to
                         the tr(T^2) it had on entry (see renormalise()) */
    int32_t n_phi;    /* azimuth bins of the extended bulb model (Eq. 3.18), or latitude
                         bins of the cylinder model (Eq. 3.20); 0 or 1: none */
    double R_nu;      /* neutrinosphere radius, km */
    double mu0;       /* nu-nu coupling, km^-1 */
    double E_min, E_max; /* MeV */
    double dm2[2];    /* eV^2, magnitudes: 2 fl dm2[0]; 3 fl dm2_21, dm2_31 */
    double theta[3];  /* rad: 2 fl theta[0]; 3 fl theta12, theta13, theta23 */
    double ne_ref, r_ref, ne_power; /* power law n_e = ne_ref (r_ref/r)^p, cm^-3 */
    double nb0, h_ns, Ye;           /* exponential n_b = nb0 exp(-(r-R)/h_ns) */
    double T[4], eta[4], L[4];      /* nu_e, nubar_e, nu_x, nubar_x */
    double eps;       /* off-diagonal seed amplitude */
    uint64_t seed;
    double eps0;      /* error-controlled step: tolerance on max |rho_c - rho_f| / tr rho */
    double ksi;       /* safety factor of the step-size update, 0 < ksi <= 1 */
    double dr_max;    /* largest step, km */
} orc_params;

/* ---- physical constants, stated here from CODATA 2018 / PDG ------------- */
static const double HBARC_EV_KM = 1.973269804e-10; /* hbar c in eV km */
static const double HBARC_EV_CM = 1.973269804e-5;  /* hbar c in eV cm */
static const double GF_EV2 = 1.1663787e-23;        /* Fermi constant, eV^-2 */
static const double PI = 3.14159265358979323846;

/* dm^2 [eV^2] / (2 E [MeV]) expressed in km^-1, per unit dm^2/E (Eq. 3.6). */
double orc_vac_coeff(void) { return 1.0 / (2.0 * 1.0e6 * HBARC_EV_KM); }
/* sqrt(2) G_F n_e in km^-1 for n_e = 1 cm^-3 (Eq. 3.7). */
double orc_matter_coeff(void)
{
    return sqrt(2.0) * GF_EV2 * HBARC_EV_CM * HBARC_EV_CM * HBARC_EV_CM / HBARC_EV_KM;
}

/* ---- Fermi-Dirac integral, Eq. 4.2, by composite Simpson quadrature ----- */
static double fd_quadrature(int k, double eta)
{
    double b = (eta > 0 ? eta : 0.0) + 80.0;
    int n = 400000; /* even */
    double h = b / n, s = 0.0, comp = 0.0;
    for (int i = 0; i <= n; ++i) {
        double x = i * h, xk = 1.0;
        for (int q = 0; q < k; ++q) xk *= x;
        double f = xk / (exp(x - eta) + 1.0);
        double wgt = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        /* compensated (Kahan) summation: 4e5 terms would otherwise lose ~1e-13 */
        double y = wgt * f - comp;
        double t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    return s * h / 3.0;
}
/* small memo: the same few (k, eta) pairs are asked for on every set-up */
double orc_fd_integral(int k, double eta)
{
    static int nmemo = 0;
    static int mk[16];
    static double me[16], mv[16];
    double v;
#pragma omp critical(orc_fd_memo)
    {
        int hit = -1;
        for (int i = 0; i < nmemo; ++i)
            if (mk[i] == k && me[i] == eta) hit = i;
        if (hit >= 0) v = mv[hit];
        else {
            v = fd_quadrature(k, eta);
            if (nmemo < 16) {
                mk[nmemo] = k;
                me[nmemo] = eta;
                mv[nmemo] = v;
                ++nmemo;
            }
        }
    }
    return v;
}

/* ---- SplitMix64 (Steele, Lea, Flood 2014), i-th output of the stream
 *      seeded with `seed`, evaluated directly from the counter. ------------ */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static double uniform01(uint64_t seed, uint64_t i)
{
    return (double)(splitmix64_at(seed, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- small dense complex matrix helpers (n <= 3) ------------------------ */
static void mat_mul(int n, const cplx *A, const cplx *B, cplx *C)
{
    cplx T[NFMAX * NFMAX];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx s = 0;
            for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
            T[i * n + j] = s;
        }
    memcpy(C, T, sizeof(cplx) * n * n);
}
static void mat_adjoint(int n, const cplx *A, cplx *B)
{
    cplx T[NFMAX * NFMAX];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) T[i * n + j] = conj(A[j * n + i]);
    memcpy(B, T, sizeof(cplx) * n * n);
}
/* rho' = U rho U^dagger */
static void conjugate_by(int n, const cplx *U, const cplx *rho, cplx *out)
{
    cplx Ud[NFMAX * NFMAX], T[NFMAX * NFMAX];
    mat_adjoint(n, U, Ud);
    mat_mul(n, U, rho, T);
    mat_mul(n, T, Ud, out);
}

/* ---- packed Hermitian <-> full matrix ------------------------------------
 * packed: n diagonal reals, then (Re, Im) of the upper triangle in row order */
static void unpack(int n, const double *p, cplx *M)
{
    for (int i = 0; i < n; ++i) M[i * n + i] = p[i];
    int k = n;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            cplx z = p[k] + I * p[k + 1];
            M[i * n + j] = z;
            M[j * n + i] = conj(z);
            k += 2;
        }
}
static void pack(int n, const cplx *M, double *p)
{
    for (int i = 0; i < n; ++i) p[i] = creal(M[i * n + i]);
    int k = n;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            p[k] = creal(M[i * n + j]);
            p[k + 1] = cimag(M[i * n + j]);
            k += 2;
        }
}

/* ---- complex Hermitian Jacobi eigensolver: A = V diag(w) V^dagger -------- */
int orc_eigh(int n, const double *Hp, double *w, double *Vri)
{
    cplx A[NFMAX * NFMAX], V[NFMAX * NFMAX];
    unpack(n, Hp, A);
    for (int i = 0; i < n * n; ++i) V[i] = 0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1;
    double scale = 0;
    for (int i = 0; i < n * n; ++i) scale += creal(A[i] * conj(A[i]));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += creal(A[p * n + q] * conj(A[p * n + q]));
        if (off <= 1e-34 * scale || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                cplx g = A[p * n + q];
                double ag = cabs(g);
                if (ag == 0.0) continue;
                cplx ph = g / ag; /* e^{i phi} */
                double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
                double tau = (aqq - app) / (2.0 * ag);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* J = identity except the (p,q) block [[c, s],[-s conj(ph), c conj(ph)]]:
                 * a phase on column q makes the pivot real, then a real rotation. */
                cplx J[NFMAX * NFMAX], Jd[NFMAX * NFMAX];
                for (int i = 0; i < n * n; ++i) J[i] = 0;
                for (int i = 0; i < n; ++i) J[i * n + i] = 1;
                J[p * n + p] = c;
                J[p * n + q] = s;
                J[q * n + p] = -s * conj(ph);
                J[q * n + q] = c * conj(ph);
                mat_adjoint(n, J, Jd);
                mat_mul(n, Jd, A, A);
                mat_mul(n, A, J, A);
                mat_mul(n, V, J, V);
                A[p * n + q] = 0; /* zero by construction; drop rounding residue */
                A[q * n + p] = 0;
            }
    }
    for (int i = 0; i < n; ++i) w[i] = creal(A[i * n + i]);
    for (int i = 0; i < n * n; ++i) {
        Vri[2 * i] = creal(V[i]);
        Vri[2 * i + 1] = cimag(V[i]);
    }
    return 0;
}

/* U = exp(-i H t).  2 flavors: the closed form of Eq. 3.10-3.12 applied to
 * the traceless part of H (the trace is a global phase that cancels in
 * U rho U^dagger, so it is dropped).  3 flavors: spectral form from the
 * Jacobi eigensolver. */
static void expm_minus_iHt(int n, const cplx *H, double t, cplx *U)
{
    if (n == 2) {
        double tr2 = 0.5 * creal(H[0] + H[3]);
        double h11 = creal(H[0]) - tr2;
        cplx h12 = H[1];
        double lam = sqrt(h11 * h11 + creal(h12 * conj(h12)));
        double cs = cos(lam * t);
        double sn_over = (lam > 0.0) ? sin(lam * t) / lam : t;
        U[0] = cs - I * h11 * sn_over;
        U[1] = -I * h12 * sn_over;
        U[2] = -I * conj(h12) * sn_over;
        U[3] = cs + I * h11 * sn_over;
        return;
    }
    double Hp[NFMAX * NFMAX], w[NFMAX], Vri[2 * NFMAX * NFMAX];
    cplx H0[NFMAX * NFMAX];
    double trn = 0;
    for (int i = 0; i < n; ++i) trn += creal(H[i * n + i]) / n;
    memcpy(H0, H, sizeof(cplx) * n * n);
    for (int i = 0; i < n; ++i) H0[i * n + i] -= trn;
    pack(n, H0, Hp);
    orc_eigh(n, Hp, w, Vri);
    cplx V[NFMAX * NFMAX], Vd[NFMAX * NFMAX], D[NFMAX * NFMAX];
    for (int i = 0; i < n * n; ++i) V[i] = Vri[2 * i] + I * Vri[2 * i + 1];
    mat_adjoint(n, V, Vd);
    for (int i = 0; i < n * n; ++i) D[i] = 0;
    for (int k = 0; k < n; ++k) D[k * n + k] = cexp(-I * w[k] * t);
    mat_mul(n, V, D, U);
    mat_mul(n, U, Vd, U);
}

/* exported for tests: U = exp(-i H t), H packed, U as (re, im) pairs */
int orc_expm(int n, const double *Hp, double t, double *Uri)
{
    cplx H[NFMAX * NFMAX], U[NFMAX * NFMAX];
    unpack(n, Hp, H);
    expm_minus_iHt(n, H, t, U);
    for (int i = 0; i < n * n; ++i) {
        Uri[2 * i] = creal(U[i]);
        Uri[2 * i + 1] = cimag(U[i]);
    }
    return 0;
}

/* ---- problem set-up -------------------------------------------------------- */
typedef struct {
    orc_params p;
    int n, nE, nu, nphi, nt, nbins, m; /* m = n*n; nt = nu * nphi trajectories */
    double dE, du;
    double *E, *u, *phi; /* phi[a*nE + e], a = nu_e, nubar_e, nu_x, nubar_x */
    double *th;          /* cylinder: emission angles theta_j in (-pi/2, pi/2) */
    cplx *Hvac;          /* [nE][n][n] */
} orc_ctx;

static int ctx_init(orc_ctx *c, const orc_params *p)
{
    memset(c, 0, sizeof(*c));
    if (p->n_E <= 0 || p->n_u <= 0 || (p->n_f != 2 && p->n_f != 3)) return -1;
    c->p = *p;
    c->n = p->n_f;
    c->m = p->n_f * p->n_f;
    c->nE = p->n_E;
    c->nu = p->n_u;
    c->nphi = p->n_phi > 1 ? p->n_phi : 1;
    if (c->nphi > 1 && p->geometry != ORC_BULB && p->geometry != ORC_CYLINDER)
        return -1; /* azimuth (or latitude) bins belong to the bulb (or cylinder) model only */
    c->nt = c->nu * c->nphi;
    c->nbins = 2 * c->nt * p->n_E;
    c->dE = (p->E_max - p->E_min) / p->n_E;
    c->du = 1.0 / p->n_u;
    c->E = malloc(sizeof(double) * c->nE);
    c->u = malloc(sizeof(double) * c->nu);
    c->phi = malloc(sizeof(double) * 4 * c->nE);
    c->Hvac = malloc(sizeof(cplx) * c->nE * c->m);
    c->th = malloc(sizeof(double) * c->nu);
    if (!c->E || !c->u || !c->phi || !c->Hvac || !c->th) return -2;
    for (int e = 0; e < c->nE; ++e) c->E[e] = p->E_min + (e + 0.5) * c->dE;
    for (int j = 0; j < c->nu; ++j) c->u[j] = (j + 0.5) * c->du;
    for (int j = 0; j < c->nu; ++j) c->th[j] = -0.5 * PI + (j + 0.5) * PI / c->nu;

    /* Eq. 4.1-4.2: f_a(E) = E^2 / (F2(eta) T^3 (exp(E/T - eta) + 1)), and the
     * number flux weight L_a/<E_a> relative to nu_e, <E> = T F3/F2. */
    double ref = 0;
    for (int a = 0; a < 4; ++a) {
        double F2 = orc_fd_integral(2, p->eta[a]);
        double F3 = orc_fd_integral(3, p->eta[a]);
        double Tm = p->T[a];
        double meanE = Tm * F3 / F2;
        double flux = p->L[a] / meanE;
        if (a == 0) ref = flux;
        for (int e = 0; e < c->nE; ++e) {
            double E = c->E[e];
            double f = E * E / (F2 * Tm * Tm * Tm * (exp(E / Tm - p->eta[a]) + 1.0));
            c->phi[a * c->nE + e] = (flux / ref) * f;
        }
    }

    /* vacuum Hamiltonian per energy bin, km^-1 */
    double K = orc_vac_coeff();
    for (int e = 0; e < c->nE; ++e) {
        cplx *H = c->Hvac + (size_t)e * c->m;
        if (c->n == 2) {
            double dm2 = p->hierarchy * p->dm2[0];
            double Delta = K * dm2 / c->E[e]; /* Eq. 3.6 */
            double c2 = cos(2 * p->theta[0]), s2 = sin(2 * p->theta[0]);
            H[0] = -0.5 * Delta * c2; /* Eq. 3.5 */
            H[1] = 0.5 * Delta * s2;
            H[2] = 0.5 * Delta * s2;
            H[3] = 0.5 * Delta * c2;
        } else {
            double s12 = sin(p->theta[0]), c12 = cos(p->theta[0]);
            double s13 = sin(p->theta[1]), c13 = cos(p->theta[1]);
            double s23 = sin(p->theta[2]), c23 = cos(p->theta[2]);
            /* standard mixing matrix with delta_CP = 0 (rows e, mu, tau) */
            double U[9] = {c12 * c13, s12 * c13, s13,
                           -s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13,
                           s12 * s23 - c12 * c23 * s13, -c12 * s23 - s12 * c23 * s13, c23 * c13};
            double m2[3] = {0.0, p->dm2[0], p->hierarchy * p->dm2[1]};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0;
                    for (int k = 0; k < 3; ++k) s += U[i * 3 + k] * m2[k] * U[j * 3 + k];
                    H[i * 3 + j] = K * s / c->E[e];
                }
        }
    }
    return 0;
}
static void ctx_free(orc_ctx *c)
{
    free(c->E);
    free(c->u);
    free(c->phi);
    free(c->Hvac);
    free(c->th);
}

/* Eq. 3.7 with the configured n_e(r) */
static double matter_A(const orc_ctx *c, double r)
{
    const orc_params *p = &c->p;
    double ne = 0;
    if (p->matter == ORC_MATTER_POWER) ne = p->ne_ref * pow(p->r_ref / r, p->ne_power);
    else if (p->matter == ORC_MATTER_EXP) ne = p->Ye * p->nb0 * exp(-(r - p->R_nu) / p->h_ns);
    return orc_matter_coeff() * ne;
}

/* Per-trajectory geometry at one radius.  Trajectory t = j n_phi + k (zenith
 * bin j, azimuth bin k).  The moments are M_q = dE sum_t w_q(t) S_t, q = 0..3,
 * and G_t = mu_eff (M0 - g1_t M1 - g2_t M2 - g3_t M3); kap[t] = dl/dr.
 * BULB: Eq. 3.13-3.15 with u = sin^2(theta_0):  cos(theta') = sqrt(1 - x^2 u),
 *       d cos(theta') = x^2 du / (2 cos(theta')), and l = r cos(theta) (Eq. 3.3)
 *       gives dl/dr = 1/cos(theta).
 * Extended bulb (Eq. 3.18, n_phi > 1): 1 - cos(gamma) = 1 - cos(th) cos(th')
 *       - sin(th) sin(th') (cos(ph) cos(ph') + sin(ph) sin(ph')), with
 *       sin(theta') = x sqrt(u) and azimuth midpoints ph_k = (k + 1/2) 2 pi / n_phi
 *       of weight 1/n_phi: four moments.  With one azimuth bin the model is the
 *       azimuthally symmetric bulb (M2 = M3 = 0).
 * CYLINDER (Sec. 3.2.5, Eq. 3.20): an infinite cylinder of radius R emits
 *       perpendicular to its axis; trajectory t = j n_phi + k leaves latitude
 *       Phi_k = (k + 1/2) 2 pi / n_phi at angle theta_j (midpoints of
 *       (-pi/2, pi/2), measured from the outward normal, positive clockwise).
 *       At radius r it makes the angle alpha_j = asin(x sin(theta_j)) with
 *       the radial direction, so dl/dr = 1/cos(alpha_j) and l = r cos(alpha_j).
 *       G_t is not a sum of a few moments when n_phi > 1 (cyl_G below); the
 *       moments M0..M2 here are the latitude averages with the weights
 *       cos(theta') / cos(alpha') dtheta', times 1, cos(alpha'), sin(alpha'),
 *       for which G = mu (M0 - cos(alpha) M1 - sin(alpha) M2) when the state is
 *       the same at every latitude; mu_eff = mu0 x (a line source thins as 1/r). */
typedef struct {
    double *w[4], *g1, *g2, *g3, *kap;
    double *alpha, *wc;  /* cylinder: alpha_t and cos(theta)/cos(alpha) dtheta of trajectory t */
    const cplx *S;       /* per-trajectory sums of the state the moments were taken from */
} geom_t;

static void geometry(const orc_ctx *c, double r, geom_t *g, double *mu_eff)
{
    const orc_params *p = &c->p;
    double x = p->R_nu / r, x2 = x * x;
    for (int t = 0; t < c->nt; ++t) {
        const int j = t / c->nphi, k = t % c->nphi;
        double cth = sqrt(1.0 - x2 * c->u[j]);
        g->w[2][t] = g->w[3][t] = g->g2[t] = g->g3[t] = 0.0;
        switch (p->geometry) {
        case ORC_BULB: {
            double a = x2 * c->du / (2.0 * cth);
            g->w[0][t] = a / c->nphi;
            g->w[1][t] = a * cth / c->nphi;
            g->g1[t] = cth;
            g->kap[t] = 1.0 / cth;
            if (c->nphi > 1) {
                double sth = sqrt(x2 * c->u[j]);
                double ph = (k + 0.5) * 2.0 * PI / c->nphi;
                g->w[2][t] = a * sth * cos(ph) / c->nphi;
                g->w[3][t] = a * sth * sin(ph) / c->nphi;
                g->g2[t] = sth * cos(ph);
                g->g3[t] = sth * sin(ph);
            }
            break;
        }
        case ORC_CYLINDER: {
            double sa = x * sin(c->th[j]), ca = sqrt(1.0 - sa * sa);
            double wc = cos(c->th[j]) / ca * (PI / c->nu);
            g->alpha[t] = asin(sa);
            g->wc[t] = wc;
            g->w[0][t] = wc / c->nphi;
            g->w[1][t] = wc * ca / c->nphi;
            g->w[2][t] = wc * sa / c->nphi;
            g->g1[t] = ca;
            g->g2[t] = sa;
            g->kap[t] = 1.0 / ca;
            break;
        }
        case ORC_MU_R4:
            g->w[0][t] = c->du;
            g->w[1][t] = c->du * cth;
            g->g1[t] = cth;
            g->kap[t] = 1.0 / cth;
            break;
        default: /* single-angle and constant-coupling modes: radial, no angle factor */
            g->w[0][t] = c->du;
            g->w[1][t] = 0.0;
            g->g1[t] = 0.0;
            g->kap[t] = 1.0;
            break;
        }
    }
    if (p->geometry == ORC_MU_R4) *mu_eff = p->mu0 * x2 * x2;
    else if (p->geometry == ORC_CYLINDER) *mu_eff = p->mu0 * x;
    else if (p->geometry == ORC_SINGLE_ANGLE) {
        double t = 1.0 - sqrt(1.0 - x2); /* Eq. 3.17 */
        *mu_eff = p->mu0 * 0.5 * t * t;
    } else *mu_eff = p->mu0;
}

/* Exact path length along trajectory t from r to r+h (Eq. 3.3, l = r cos):
 * l(r+h) - l(r) = ((r+h)^2 - r^2) / (l(r+h) + l(r)), since l^2 = r^2 - b^2 with
 * b the impact parameter; written this way it has no cancellation.  It depends
 * on the zenith bin only. */
static double path_length(const orc_ctx *c, int t, double r, double h)
{
    const int j = t / c->nphi;
    double R = c->p.R_nu;
    if (c->p.geometry == ORC_CYLINDER) { /* l = sqrt(r^2 - R^2 sin^2(theta_j)) */
        double b2 = R * R * sin(c->th[j]) * sin(c->th[j]);
        return h * (2.0 * r + h) / (sqrt(r * r - b2) + sqrt((r + h) * (r + h) - b2));
    }
    if (c->p.geometry != ORC_BULB && c->p.geometry != ORC_MU_R4) return h;
    double x0 = R / r, x1 = R / (r + h);
    double l0 = r * sqrt(1.0 - x0 * x0 * c->u[j]);
    double l1 = (r + h) * sqrt(1.0 - x1 * x1 * c->u[j]);
    return h * (2.0 * r + h) / (l0 + l1);
}

/* nu-nu moments (Eq. 3.13 / 3.18): S_t = sum_e (rho_nu - conj(rho_nubar)) per
 * trajectory, M_q = dE sum_t w_q(t) S_t.  Sequential sums in index order; the
 * trajectory loop may run in parallel (each S_t is one thread's).  M[2], M[3]
 * are zero without azimuth bins. */
typedef cplx mom_t[4][NFMAX * NFMAX];

static void moments(const orc_ctx *c, const cplx *rho, geom_t *g, mom_t M, cplx *Sbuf)
{
    int m = c->m, nE = c->nE, nt = c->nt;
    const int nmom = (c->nphi > 1 || c->p.geometry == ORC_CYLINDER) ? 4 : 2;
    g->S = Sbuf;
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nt; ++t) {
        cplx S[NFMAX * NFMAX];
        for (int k = 0; k < m; ++k) S[k] = 0;
        for (int e = 0; e < nE; ++e) {
            const cplx *rn = rho + ((size_t)(0 * nt + t) * nE + e) * m;
            const cplx *ra = rho + ((size_t)(1 * nt + t) * nE + e) * m;
            for (int k = 0; k < m; ++k) S[k] += rn[k] - conj(ra[k]);
        }
        memcpy(Sbuf + (size_t)t * m, S, sizeof(cplx) * m);
    }
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < m; ++k) M[q][k] = 0;
    for (int t = 0; t < nt; ++t)
        for (int q = 0; q < nmom; ++q)
            for (int k = 0; k < m; ++k) M[q][k] += g->w[q][t] * Sbuf[(size_t)t * m + k];
    for (int q = 0; q < nmom; ++q)
        for (int k = 0; k < m; ++k) M[q][k] *= c->dE;
}

/* Cylinder model, Eq. 3.20, for trajectory t = (theta_j, Phi_k):
 *   G_t = mu dE sum_j' w_j' [1 - cos(alpha_j - alpha_j')] S(Phi', theta_j'),
 *   w_j' = cos(theta_j') / cos(alpha_j') dtheta,
 *   Phi' = Phi_k + theta_j' - theta_j + alpha_j - alpha_j'  (the background
 *          trajectory that crosses t's point at radius r left from latitude Phi'),
 * S(Phi', .) by periodic linear interpolation between the two latitude bins
 * around Phi' (the paper does not say how Phi' off the grid is read). */
static void cyl_G(const orc_ctx *c, const geom_t *g, int t, double mu, cplx *G)
{
    const int m = c->m, nphi = c->nphi, j = t / nphi, k = t % nphi;
    const double dphi = 2.0 * PI / nphi;
    for (int q = 0; q < m; ++q) G[q] = 0;
    for (int jp = 0; jp < c->nu; ++jp) {
        double a = g->alpha[j * nphi], ap = g->alpha[jp * nphi];
        double shift = c->th[jp] - c->th[j] + a - ap; /* Phi' - Phi_k */
        double pos = k + shift / dphi;                /* Phi' in units of the latitude grid */
        double fl = floor(pos), f = pos - fl;
        int i0 = ((int)fl % nphi + nphi) % nphi, i1 = (i0 + 1) % nphi;
        double K = g->wc[jp * nphi] * (1.0 - cos(a - ap));
        const cplx *S0 = g->S + (size_t)(jp * nphi + i0) * m, *S1 = g->S + (size_t)(jp * nphi + i1) * m;
        for (int q = 0; q < m; ++q) G[q] += K * ((1.0 - f) * S0[q] + f * S1[q]);
    }
    for (int q = 0; q < m; ++q) G[q] *= mu * c->dE;
}

/* G_t = mu (M0 - g1_t M1 - g2_t M2 - g3_t M3); the cylinder model with
 * latitude bins from the state's per-trajectory sums (cyl_G). */
static void g_of(const orc_ctx *c, const geom_t *g, int t, double mu, mom_t M, cplx *G)
{
    if (c->p.geometry == ORC_CYLINDER && c->nphi > 1) {
        cyl_G(c, g, t, mu, G);
        return;
    }
    for (int k = 0; k < c->m; ++k)
        G[k] = mu * (M[0][k] - g->g1[t] * M[1][k] - g->g2[t] * M[2][k] - g->g3[t] * M[3][k]);
}

static int moments_finite(const orc_ctx *c, mom_t M)
{
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < c->m; ++k)
            if (!isfinite(creal(M[q][k])) || !isfinite(cimag(M[q][k]))) return 0;
    return 1;
}

/* Hamiltonian of bin (s, j, e):  nu:    H_vac + A P_e + G_j
 *                                nubar: H_vac - A P_e - conj(G_j) */
static void hamiltonian(const orc_ctx *c, int s, int e, const cplx *G, double A, cplx *H)
{
    int m = c->m, n = c->n;
    const cplx *Hv = c->Hvac + (size_t)e * m;
    for (int k = 0; k < m; ++k) H[k] = Hv[k] + (s == 0 ? G[k] : -conj(G[k]));
    H[0] += (s == 0 ? A : -A);
    (void)n;
}

static int all_finite(int m, const cplx *M)
{
    for (int k = 0; k < m; ++k)
        if (!isfinite(creal(M[k])) || !isfinite(cimag(M[k]))) return 0;
    return 1;
}

typedef struct {
    geom_t g;
    cplx *Sbuf;
} scratch_t;

static int scratch_alloc(const orc_ctx *c, scratch_t *w)
{
    memset(w, 0, sizeof(*w));
    for (int q = 0; q < 4; ++q) w->g.w[q] = malloc(sizeof(double) * c->nt);
    w->g.g1 = malloc(sizeof(double) * c->nt);
    w->g.g2 = malloc(sizeof(double) * c->nt);
    w->g.g3 = malloc(sizeof(double) * c->nt);
    w->g.kap = malloc(sizeof(double) * c->nt);
    w->g.alpha = malloc(sizeof(double) * c->nt);
    w->g.wc = malloc(sizeof(double) * c->nt);
    w->Sbuf = malloc(sizeof(cplx) * c->nt * c->m);
    return w->g.w[3] && w->g.kap && w->g.alpha && w->g.wc && w->Sbuf ? 0 : -2;
}

static void scratch_free(scratch_t *w)
{
    for (int q = 0; q < 4; ++q) free(w->g.w[q]);
    free(w->g.g1);
    free(w->g.g2);
    free(w->g.g3);
    free(w->g.kap);
    free(w->g.alpha);
    free(w->g.wc);
    free(w->Sbuf);
}

/* d(rho)/dr = -i [H, rho] dl/dr for every bin; returns 0 if the moments were
 * not finite. */
static int rhs(const orc_ctx *c, scratch_t *w, double r, const cplx *rho, cplx *K)
{
    int n = c->n, m = c->m, nE = c->nE, nt = c->nt;
    double mu;
    geometry(c, r, &w->g, &mu);
    mom_t M;
    moments(c, rho, &w->g, M, w->Sbuf);
    if (!moments_finite(c, M)) return 0;
    double A = matter_A(c, r);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < c->nbins; ++b) {
        int s = b / (nt * nE), t = (b / nE) % nt, e = b % nE;
        cplx G[NFMAX * NFMAX], H[NFMAX * NFMAX], X[NFMAX * NFMAX], Y[NFMAX * NFMAX];
        g_of(c, &w->g, t, mu, M, G);
        hamiltonian(c, s, e, G, A, H);
        const cplx *rb = rho + (size_t)b * m;
        mat_mul(n, H, rb, X);
        mat_mul(n, rb, H, Y);
        for (int k = 0; k < m; ++k) K[(size_t)b * m + k] = -I * (X[k] - Y[k]) * w->g.kap[t];
    }
    return 1;
}

static int step_rk4(const orc_ctx *c, scratch_t *w, cplx *rho, double r, double h, cplx *Y,
                    cplx *K, cplx *acc)
{
    size_t N = (size_t)c->nbins * c->m;
    /* k1 */
    if (!rhs(c, w, r, rho, K)) return 0;
    for (size_t i = 0; i < N; ++i) {
        acc[i] = K[i];
        Y[i] = rho[i] + (0.5 * h) * K[i];
    }
    /* k2 */
    if (!rhs(c, w, r + 0.5 * h, Y, K)) return 0;
    for (size_t i = 0; i < N; ++i) {
        acc[i] += 2.0 * K[i];
        Y[i] = rho[i] + (0.5 * h) * K[i];
    }
    /* k3 */
    if (!rhs(c, w, r + 0.5 * h, Y, K)) return 0;
    for (size_t i = 0; i < N; ++i) {
        acc[i] += 2.0 * K[i];
        Y[i] = rho[i] + h * K[i];
    }
    /* k4 */
    if (!rhs(c, w, r + h, Y, K)) return 0;
    for (size_t i = 0; i < N; ++i) Y[i] = rho[i] + (h / 6.0) * (acc[i] + K[i]);
    return 1;
}

/* Coarse predictor-corrector of Sec. 4.2.3 / Listing 5.1 (S1-S3), rho form:
 *   H0 from rho_n at r;     rho_p = U(H0) rho_n U(H0)^+            (predictor)
 *   H1 from rho_p at r + h; rho_{n+1} = (rho_p + U(H1) rho_n U(H1)^+) / 2
 * U(H) = exp(-i H dl_j) with dl_j the path length of trajectory j. */
static int step_exph(const orc_ctx *c, scratch_t *w, const cplx *rho, double r, double h,
                     cplx *rp, cplx *out)
{
    int n = c->n, m = c->m, nE = c->nE, nt = c->nt;
    double mu;
    mom_t M;
    double *dl = malloc(sizeof(double) * nt);
    for (int t = 0; t < nt; ++t) dl[t] = path_length(c, t, r, h);
    for (int pass = 0; pass < 2; ++pass) {
        double rr = (pass == 0) ? r : r + h;
        const cplx *src = (pass == 0) ? rho : rp;
        geometry(c, rr, &w->g, &mu);
        moments(c, src, &w->g, M, w->Sbuf);
        if (!moments_finite(c, M)) {
            free(dl);
            return 0;
        }
        double A = matter_A(c, rr);
#pragma omp parallel for schedule(static)
        for (int b = 0; b < c->nbins; ++b) {
            int s = b / (nt * nE), t = (b / nE) % nt, e = b % nE;
            cplx G[NFMAX * NFMAX], H[NFMAX * NFMAX], U[NFMAX * NFMAX], X[NFMAX * NFMAX];
            g_of(c, &w->g, t, mu, M, G);
            hamiltonian(c, s, e, G, A, H);
            expm_minus_iHt(n, H, dl[t], U);
            conjugate_by(n, U, rho + (size_t)b * m, X);
            if (pass == 0) memcpy(rp + (size_t)b * m, X, sizeof(cplx) * m);
            else
                for (int k = 0; k < m; ++k)
                    out[(size_t)b * m + k] = 0.5 * (rp[(size_t)b * m + k] + X[k]);
        }
    }
    free(dl);
    return 1;
}

/* Renormalised method: the exact flow d(rho)/dr = -i[H, rho] dl/dr (Eq. 3.2,
 * 3.10) is a unitary conjugation per bin, so it keeps tr(rho), and with it
 * tr(T^2) of the traceless part T = rho - tr(rho)/n I (|P|^2 / 2 in two
 * flavors).  Neither RK4 nor the averaged predictor-corrector keeps tr(T^2);
 * this variant of either method restores it after every step:
 *     rho <- tr(rho)/n I + sqrt(q0 / q) T,   q = tr(T^2), q0 its value on entry. */
static void purity_of(int n, const cplx *rho, double *q)
{
    double tau = 0;
    for (int i = 0; i < n; ++i) tau += creal(rho[i * n + i]);
    tau /= n;
    double s = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx t = rho[i * n + j] - (i == j ? tau : 0.0);
            s += creal(t) * creal(t) + cimag(t) * cimag(t);
        }
    *q = s;
}

static void renormalise(int n, cplx *rho, double q0)
{
    double q;
    purity_of(n, rho, &q);
    if (!(q > 0) || !(q0 > 0)) return;
    double tau = 0;
    for (int i = 0; i < n; ++i) tau += creal(rho[i * n + i]);
    tau /= n;
    double f = sqrt(q0 / q);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx d = (i == j) ? tau : 0.0;
            rho[i * n + j] = d + f * (rho[i * n + j] - d);
        }
}

/* One attempt of the error-controlled step of Sec. 4.2.3 (Fig. 4.9; the
 * sections S1-S5 of Listings 5.1-5.3), in rho form.  From rho0 at r with
 * step h, U(H; r, h) = exp(-i H dl_j(r, h)) along trajectory j:
 *   S1  H0 from rho0 at r
 *   S2  rho1 = U(H0; r, h/2) rho0 U^+ (half step), rho2 = U(H0; r, h) rho0 U^+
 *       (full step); H1 from rho2 at r + h, H2 from rho1 at r + h/2
 *   S3  rho3 = U(H1; r, h) rho0 U^+, coarse result rho_c = (rho2 + rho3) / 2
 *   S4  rho5 = U(H2; r + h/2, h/2) rho1 U^+ (midpoint to r + h); H3 from rho5
 *       at r + h
 *   S5  rho6 = U(H3; r, h) rho0 U^+, fine result rho_f = (rho5 + rho6) / 2;
 *       err = max over bins b and packed entries of |rho_c - rho_f| / tr rho0_b
 * Writes rho_c to out.  Returns 0 if a moment or a result was not finite. */
static int hamiltonians_at(const orc_ctx *c, scratch_t *w, geom_t *gsave, const cplx *src, double r, mom_t M,
                           double *mu, double *A)
{
    geometry(c, r, gsave, mu);
    moments(c, src, gsave, M, w->Sbuf);
    *A = matter_A(c, r);
    return moments_finite(c, M);
}

/* rho_out[b] = U rho_in[b] U^+ for every bin, U = exp(-i H_b dl_t), H_b from
 * the moments M with the geometry g and the scalars mu, A. */
static void propagate_all(const orc_ctx *c, mom_t M, double mu, double A, const geom_t *g, const double *dl,
                          const cplx *rho_in, cplx *rho_out)
{
    int n = c->n, m = c->m, nE = c->nE, nt = c->nt;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < c->nbins; ++b) {
        int s = b / (nt * nE), t = (b / nE) % nt, e = b % nE;
        cplx G[NFMAX * NFMAX], H[NFMAX * NFMAX], U[NFMAX * NFMAX];
        g_of(c, g, t, mu, M, G);
        hamiltonian(c, s, e, G, A, H);
        expm_minus_iHt(n, H, dl[t], U);
        conjugate_by(n, U, rho_in + (size_t)b * m, rho_out + (size_t)b * m);
    }
}

typedef struct {
    cplx *r1, *r2, *r3, *r5, *r6;
    double *dl_full, *dl_half, *dl_mid;
} adapt_buf;

static int adapt_alloc(const orc_ctx *c, adapt_buf *B)
{
    size_t N = (size_t)c->nbins * c->m;
    B->r1 = malloc(sizeof(cplx) * N);
    B->r2 = malloc(sizeof(cplx) * N);
    B->r3 = malloc(sizeof(cplx) * N);
    B->r5 = malloc(sizeof(cplx) * N);
    B->r6 = malloc(sizeof(cplx) * N);
    B->dl_full = malloc(sizeof(double) * c->nt);
    B->dl_half = malloc(sizeof(double) * c->nt);
    B->dl_mid = malloc(sizeof(double) * c->nt);
    return B->r6 && B->dl_mid ? 0 : -2;
}

static void adapt_free(adapt_buf *B)
{
    free(B->r1);
    free(B->r2);
    free(B->r3);
    free(B->r5);
    free(B->r6);
    free(B->dl_full);
    free(B->dl_half);
    free(B->dl_mid);
}

static int attempt_adaptive(const orc_ctx *c, scratch_t *w, adapt_buf *B, const cplx *rho0, double r, double h,
                            cplx *out, double *err)
{
    int m = c->m, nt = c->nt;
    size_t N = (size_t)c->nbins * m;
    mom_t M;
    double mu, A;
    geom_t *g = &w->g;
    for (int t = 0; t < nt; ++t) {
        B->dl_full[t] = path_length(c, t, r, h);
        B->dl_half[t] = path_length(c, t, r, 0.5 * h);
        B->dl_mid[t] = path_length(c, t, r + 0.5 * h, 0.5 * h);
    }
    /* S1 */
    if (!hamiltonians_at(c, w, g, rho0, r, M, &mu, &A)) return 0;
    /* S2 */
    propagate_all(c, M, mu, A, g, B->dl_half, rho0, B->r1);
    propagate_all(c, M, mu, A, g, B->dl_full, rho0, B->r2);
    /* S3: H1 from rho2 at r + h */
    if (!hamiltonians_at(c, w, g, B->r2, r + h, M, &mu, &A)) return 0;
    propagate_all(c, M, mu, A, g, B->dl_full, rho0, B->r3);
    for (size_t i = 0; i < N; ++i) out[i] = 0.5 * (B->r2[i] + B->r3[i]);
    /* S4: H2 from rho1 at r + h/2 */
    if (!hamiltonians_at(c, w, g, B->r1, r + 0.5 * h, M, &mu, &A)) return 0;
    propagate_all(c, M, mu, A, g, B->dl_mid, B->r1, B->r5);
    /* S5: H3 from rho5 at r + h */
    if (!hamiltonians_at(c, w, g, B->r5, r + h, M, &mu, &A)) return 0;
    propagate_all(c, M, mu, A, g, B->dl_full, rho0, B->r6);
    double e = 0.0;
    for (int b = 0; b < c->nbins; ++b) {
        double tr = 0.0;
        for (int i = 0; i < c->n; ++i) tr += creal(rho0[(size_t)b * m + i * c->n + i]);
        for (int k = 0; k < m; ++k) {
            size_t i = (size_t)b * m + k;
            cplx f = 0.5 * (B->r5[i] + B->r6[i]);
            double d = cabs(out[i] - f) / fabs(tr);
            if (!(d <= e)) e = d; /* a NaN difference propagates */
        }
    }
    *err = e;
    for (size_t i = 0; i < N; ++i)
        if (!isfinite(creal(out[i])) || !isfinite(cimag(out[i]))) return 0;
    return 1;
}

/* ---- exported entry points (ctypes) --------------------------------------- */

/* Tables for inspection: E[nE], u[nu], phi[4*nE], Hvac[nE*n*n] packed. */
int orc_tables(const orc_params *p, double *E, double *u, double *phi, double *Hvac_packed)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
    memcpy(E, c.E, sizeof(double) * c.nE);
    memcpy(u, c.u, sizeof(double) * c.nu);
    memcpy(phi, c.phi, sizeof(double) * 4 * c.nE);
    for (int e = 0; e < c.nE; ++e) pack(c.n, c.Hvac + (size_t)e * c.m, Hvac_packed + (size_t)e * c.m);
    ctx_free(&c);
    return 0;
}

/* Seeded initial state, packed [s][u][E][n*n]:
 * rho_nu = diag(phi_nue, phi_nux[, phi_nux]), rho_nubar likewise with the
 * antineutrino spectra; each off-diagonal (i<j) gets
 * eps sqrt(rho_ii rho_jj) exp(2 pi i U), U the SplitMix64 uniform number with
 * counter b * n_off + k (k-th upper entry in row order). */
int orc_init_state(const orc_params *p, double *rho_packed)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
    int n = c.n, m = c.m, noff = n * (n - 1) / 2;
    for (int b = 0; b < c.nbins; ++b) {
        int s = b / (c.nt * c.nE), e = b % c.nE;
        double pe = c.phi[(s == 0 ? 0 : 1) * c.nE + e];
        double px = c.phi[(s == 0 ? 2 : 3) * c.nE + e];
        cplx M[NFMAX * NFMAX];
        for (int k = 0; k < m; ++k) M[k] = 0;
        M[0] = pe;
        for (int i = 1; i < n; ++i) M[i * n + i] = px;
        int k = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double ph = 2.0 * PI * uniform01(p->seed, (uint64_t)b * noff + k);
                double amp = p->eps * sqrt(creal(M[i * n + i]) * creal(M[j * n + j]));
                M[i * n + j] = amp * cexp(I * ph);
                M[j * n + i] = conj(M[i * n + j]);
                ++k;
            }
        pack(n, M, rho_packed + (size_t)b * m);
    }
    ctx_free(&c);
    return 0;
}

/* Advance rho (packed, in/out) by n_steps fixed steps of size h from r0.
 * Returns 0 on success, 1 if a non-finite moment appeared (rho is then left
 * at the last step whose state was finite; *steps_done tells which), <0 on
 * argument errors. */
int orc_evolve(const orc_params *p, double *rho_packed, double r0, double h, int64_t n_steps,
               int64_t *steps_done)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
#ifdef _OPENMP
    if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#endif
    size_t N = (size_t)c.nbins * c.m;
    cplx *rho = malloc(sizeof(cplx) * N), *Y = malloc(sizeof(cplx) * N);
    cplx *K = malloc(sizeof(cplx) * N), *acc = malloc(sizeof(cplx) * N);
    scratch_t w;
    scratch_alloc(&c, &w);
    for (int b = 0; b < c.nbins; ++b) unpack(c.n, rho_packed + (size_t)b * c.m, rho + (size_t)b * c.m);
    double *q0 = NULL;
    if (p->renorm) {
        q0 = malloc(sizeof(double) * c.nbins);
        for (int b = 0; b < c.nbins; ++b) purity_of(c.n, rho + (size_t)b * c.m, &q0[b]);
    }
    int status = 0;
    int64_t done = 0;
    for (int64_t st = 0; st < n_steps; ++st) {
        double r = r0 + (double)st * h;
        int ok = (p->stepper == ORC_RK4) ? step_rk4(&c, &w, rho, r, h, Y, K, acc)
                                         : step_exph(&c, &w, rho, r, h, K, Y);
        if (ok) {
            for (size_t i = 0; i < N && ok; ++i)
                if (!isfinite(creal(Y[i])) || !isfinite(cimag(Y[i]))) ok = 0;
        }
        if (!ok) {
            status = 1;
            break;
        }
        cplx *t = rho;
        rho = Y;
        Y = t;
        if (q0)
            for (int b = 0; b < c.nbins; ++b) renormalise(c.n, rho + (size_t)b * c.m, q0[b]);
        ++done;
    }
    free(q0);
    for (int b = 0; b < c.nbins; ++b) pack(c.n, rho + (size_t)b * c.m, rho_packed + (size_t)b * c.m);
    if (steps_done) *steps_done = done;
    free(rho);
    free(Y);
    free(K);
    free(acc);
    scratch_free(&w);
    ctx_free(&c);
    return status;
}

/* Step-size update after an attempt with error err at step h (Sec. 4.2.3 and
 * the eps0 / ksi / max_dr keywords of Appendix A.3): the error estimate of
 * one attempt scales as h^2 (measured; see the tests), so the step that would
 * just meet eps0 is h (eps0 / err)^(1/2); ksi < 1 keeps the next try on the
 * safe side, and dr_max trims it.  err = 0 gives dr_max. */
static double next_step(const orc_params *p, double h, double err)
{
    double hn = (err > 0.0) ? p->ksi * h * sqrt(p->eps0 / err) : p->dr_max;
    return hn < p->dr_max ? hn : p->dr_max;
}

/* Error-controlled evolution from r0 to r_end (Fig. 4.8-4.9): repeat
 * attempts; an attempt with err <= eps0 is accepted (rho <- rho_c, r <- r + h),
 * otherwise rho and r stay; either way h <- next_step(h, err).  The last step
 * is shortened to land on r_end, and a radius within 1e-12 r_end of r_end
 * counts as arrived (and is set to r_end).  Stops at r_end (status 0), after max_iters
 * attempts (status 2), at a non-finite attempt (status 1; rho is the last
 * accepted state) or when h falls below 1e-12 r (status 3).  r_out, h_out:
 * final radius and the next step size; n_acc / n_rej: accepted and rejected
 * attempts. */
int orc_evolve_adaptive(const orc_params *p, double *rho_packed, double r0, double r_end, double h0,
                        int64_t max_iters, double *r_out, double *h_out, int64_t *n_acc, int64_t *n_rej)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
    if (!(h0 > 0) || !(r_end >= r0) || !(p->eps0 > 0) || !(p->ksi > 0) || !(p->dr_max > 0)) {
        ctx_free(&c);
        return -1;
    }
#ifdef _OPENMP
    if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#endif
    size_t N = (size_t)c.nbins * c.m;
    cplx *rho = malloc(sizeof(cplx) * N), *out = malloc(sizeof(cplx) * N);
    adapt_buf B;
    adapt_alloc(&c, &B);
    scratch_t w;
    scratch_alloc(&c, &w);
    for (int b = 0; b < c.nbins; ++b) unpack(c.n, rho_packed + (size_t)b * c.m, rho + (size_t)b * c.m);
    double r = r0, h = h0 < p->dr_max ? h0 : p->dr_max;
    int64_t acc = 0, rej = 0, it = 0;
    int status = 0;
    /* arrival: within 1e-12 r_end of the end (the accumulated radius of many
     * steps lands a few ulps short of it) */
    while (r_end - r > 1e-12 * r_end) {
        if (it >= max_iters) {
            status = 2;
            break;
        }
        if (h < 1e-12 * r) {
            status = 3;
            break;
        }
        const int last = (h >= r_end - r);
        const double ht = last ? r_end - r : h;
        double err = 0.0;
        ++it;
        if (!attempt_adaptive(&c, &w, &B, rho, r, ht, out, &err) || !isfinite(err)) {
            status = 1;
            break;
        }
        if (err <= p->eps0) {
            cplx *t = rho;
            rho = out;
            out = t;
            r = last ? r_end : r + ht;
            ++acc;
        } else {
            ++rej;
        }
        h = next_step(p, ht, err);
    }
    if (status == 0) r = r_end;
    for (int b = 0; b < c.nbins; ++b) pack(c.n, rho + (size_t)b * c.m, rho_packed + (size_t)b * c.m);
    if (r_out) *r_out = r;
    if (h_out) *h_out = h;
    if (n_acc) *n_acc = acc;
    if (n_rej) *n_rej = rej;
    free(rho);
    free(out);
    adapt_free(&B);
    scratch_free(&w);
    ctx_free(&c);
    return status;
}

/* One attempt only (no acceptance logic): rho_packed <- rho_c; *err as above;
 * *fine (optional, packed) <- rho_f.  Returns 0, or 1 if not finite. */
int orc_attempt_adaptive(const orc_params *p, double *rho_packed, double r, double h, double *err, double *fine)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
#ifdef _OPENMP
    if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#endif
    size_t N = (size_t)c.nbins * c.m;
    cplx *rho = malloc(sizeof(cplx) * N), *out = malloc(sizeof(cplx) * N);
    adapt_buf B;
    adapt_alloc(&c, &B);
    scratch_t w;
    scratch_alloc(&c, &w);
    for (int b = 0; b < c.nbins; ++b) unpack(c.n, rho_packed + (size_t)b * c.m, rho + (size_t)b * c.m);
    int ok = attempt_adaptive(&c, &w, &B, rho, r, h, out, err);
    for (int b = 0; b < c.nbins; ++b) pack(c.n, out + (size_t)b * c.m, rho_packed + (size_t)b * c.m);
    if (fine)
        for (int b = 0; b < c.nbins; ++b) {
            cplx f[NFMAX * NFMAX];
            for (int k = 0; k < c.m; ++k) f[k] = 0.5 * (B.r5[(size_t)b * c.m + k] + B.r6[(size_t)b * c.m + k]);
            pack(c.n, f, fine + (size_t)b * c.m);
        }
    free(rho);
    free(out);
    adapt_free(&B);
    scratch_free(&w);
    ctx_free(&c);
    return ok ? 0 : 1;
}

/* ---- wavefunction form (Eq. 3.1, 3.4, 3.9-3.11; Fig. 4.9) ----------------
 * Each bin carries one wavefunction psi_a (n complex components) per initial
 * flavor a, and its density matrix is rho = sum_a phi_a psi_a psi_a^+ with
 * phi_a the number-flux weight of flavor a (nu_e, or nu_x for the others; the
 * antineutrino spectra for nubar bins).  Each psi evolves with the same
 * Hamiltonian as rho: psi' = exp(-i H dl) psi (Eq. 3.10-3.11).  The
 * predictor-corrector averages wavefunctions (Sec. 4.2.3: "averaging between
 * two flavor states"): psi_p = U(H0) psi_n, psi_{n+1} = (psi_p + U(H1) psi_n)/2,
 * with no renormalisation.  RK4 integrates d(psi)/dr = -i H psi dl/dr.
 * Packed layout: [s][t][E][a][i] complex, as (Re, Im) doubles, 2 n^2 per bin. */

static double flux_weight(const orc_ctx *c, int s, int e, int a)
{
    return c->phi[(s == 0 ? (a == 0 ? 0 : 2) : (a == 0 ? 1 : 3)) * c->nE + e];
}

/* rho of every bin from the wavefunctions (psi: [b][a][i]). */
static void psi_to_rho(const orc_ctx *c, const cplx *psi, cplx *rho)
{
    int n = c->n, m = c->m, nE = c->nE, nt = c->nt;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < c->nbins; ++b) {
        int s = b / (nt * nE), e = b % nE;
        cplx *R = rho + (size_t)b * m;
        for (int k = 0; k < m; ++k) R[k] = 0;
        for (int a = 0; a < n; ++a) {
            const cplx *v = psi + ((size_t)b * n + a) * n;
            double w = flux_weight(c, s, e, a);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) R[i * n + j] += w * v[i] * conj(v[j]);
        }
    }
}

/* out_a = U in_a for every bin and flavor, U = exp(-i H_b dl_t). */
static void propagate_psi(const orc_ctx *c, mom_t M, double mu, double A, const geom_t *g, const double *dl,
                          const cplx *in, cplx *out)
{
    int n = c->n, m = c->m, nE = c->nE, nt = c->nt;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < c->nbins; ++b) {
        int s = b / (nt * nE), t = (b / nE) % nt, e = b % nE;
        cplx G[NFMAX * NFMAX], H[NFMAX * NFMAX], U[NFMAX * NFMAX];
        g_of(c, g, t, mu, M, G);
        hamiltonian(c, s, e, G, A, H);
        expm_minus_iHt(n, H, dl[t], U);
        for (int a = 0; a < n; ++a) {
            const cplx *v = in + ((size_t)b * n + a) * n;
            cplx *o = out + ((size_t)b * n + a) * n;
            for (int i = 0; i < n; ++i) {
                cplx z = 0;
                for (int j = 0; j < n; ++j) z += U[i * n + j] * v[j];
                o[i] = z;
            }
        }
    }
    (void)m;
}

/* d(psi)/dr = -i H psi dl/dr for every bin and flavor, H taken traceless as
 * in the propagator of Eq. 3.11 (its trace would only turn every wavefunction
 * of the bin by one common phase, which rho = sum phi psi psi^+ never sees). */
static int rhs_psi(const orc_ctx *c, scratch_t *w, cplx *rho_scr, double r, const cplx *psi, cplx *K)
{
    int n = c->n, nE = c->nE, nt = c->nt;
    double mu;
    geometry(c, r, &w->g, &mu);
    psi_to_rho(c, psi, rho_scr);
    mom_t M;
    moments(c, rho_scr, &w->g, M, w->Sbuf);
    if (!moments_finite(c, M)) return 0;
    double A = matter_A(c, r);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < c->nbins; ++b) {
        int s = b / (nt * nE), t = (b / nE) % nt, e = b % nE;
        cplx G[NFMAX * NFMAX], H[NFMAX * NFMAX];
        g_of(c, &w->g, t, mu, M, G);
        hamiltonian(c, s, e, G, A, H);
        double trn = 0.0;
        for (int i = 0; i < n; ++i) trn += creal(H[i * n + i]) / n;
        for (int i = 0; i < n; ++i) H[i * n + i] -= trn;
        for (int a = 0; a < n; ++a) {
            const cplx *v = psi + ((size_t)b * n + a) * n;
            cplx *k = K + ((size_t)b * n + a) * n;
            for (int i = 0; i < n; ++i) {
                cplx z = 0;
                for (int j = 0; j < n; ++j) z += H[i * n + j] * v[j];
                k[i] = -I * z * w->g.kap[t];
            }
        }
    }
    return 1;
}

int orc_init_psi(const orc_params *p, double *psi_packed)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
    int n = c.n, nperm = n * (n - 1);
    /* psi_a = (e_a + eps sum_{b != a} exp(2 pi i U_ab) e_b) / sqrt(1 + (n-1) eps^2),
     * U_ab the SplitMix64 uniform number at counter bin * n(n-1) + k, k running
     * over (a, b != a) in row order */
    double norm = 1.0 / sqrt(1.0 + (n - 1) * p->eps * p->eps);
    for (int b = 0; b < c.nbins; ++b) {
        int k = 0;
        for (int a = 0; a < n; ++a) {
            double *v = psi_packed + ((size_t)b * n + a) * 2 * n;
            for (int i = 0; i < n; ++i) {
                cplx z;
                if (i == a) z = norm;
                else {
                    double ph = 2.0 * PI * uniform01(p->seed, (uint64_t)b * nperm + k);
                    z = norm * p->eps * cexp(I * ph);
                    ++k;
                }
                v[2 * i] = creal(z);
                v[2 * i + 1] = cimag(z);
            }
        }
    }
    ctx_free(&c);
    return 0;
}

int orc_psi_to_rho(const orc_params *p, const double *psi_packed, double *rho_packed)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
    size_t NP = (size_t)c.nbins * c.n * c.n, N = (size_t)c.nbins * c.m;
    cplx *psi = malloc(sizeof(cplx) * NP), *rho = malloc(sizeof(cplx) * N);
    for (size_t i = 0; i < NP; ++i) psi[i] = psi_packed[2 * i] + I * psi_packed[2 * i + 1];
    psi_to_rho(&c, psi, rho);
    for (int b = 0; b < c.nbins; ++b) pack(c.n, rho + (size_t)b * c.m, rho_packed + (size_t)b * c.m);
    free(psi);
    free(rho);
    ctx_free(&c);
    return 0;
}

/* Advance the wavefunctions (packed, in/out) by n_steps fixed steps of size h
 * from r0 with the configured stepper.  Status as orc_evolve. */
int orc_evolve_psi(const orc_params *p, double *psi_packed, double r0, double h, int64_t n_steps,
                   int64_t *steps_done)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
#ifdef _OPENMP
    if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#endif
    const int n = c.n, nt = c.nt;
    size_t NP = (size_t)c.nbins * n * n, N = (size_t)c.nbins * c.m;
    cplx *psi = malloc(sizeof(cplx) * NP), *nxt = malloc(sizeof(cplx) * NP);
    cplx *Y = malloc(sizeof(cplx) * NP), *K = malloc(sizeof(cplx) * NP), *acc = malloc(sizeof(cplx) * NP);
    cplx *rho = malloc(sizeof(cplx) * N);
    double *dl = malloc(sizeof(double) * nt);
    scratch_t w;
    scratch_alloc(&c, &w);
    for (size_t i = 0; i < NP; ++i) psi[i] = psi_packed[2 * i] + I * psi_packed[2 * i + 1];
    int status = 0;
    int64_t done = 0;
    for (int64_t st = 0; st < n_steps; ++st) {
        const double r = r0 + (double)st * h;
        int ok = 1;
        if (p->stepper == ORC_RK4) {
            ok = rhs_psi(&c, &w, rho, r, psi, K);
            for (size_t i = 0; ok && i < NP; ++i) {
                acc[i] = K[i];
                Y[i] = psi[i] + (0.5 * h) * K[i];
            }
            ok = ok && rhs_psi(&c, &w, rho, r + 0.5 * h, Y, K);
            for (size_t i = 0; ok && i < NP; ++i) {
                acc[i] += 2.0 * K[i];
                Y[i] = psi[i] + (0.5 * h) * K[i];
            }
            ok = ok && rhs_psi(&c, &w, rho, r + 0.5 * h, Y, K);
            for (size_t i = 0; ok && i < NP; ++i) {
                acc[i] += 2.0 * K[i];
                Y[i] = psi[i] + h * K[i];
            }
            ok = ok && rhs_psi(&c, &w, rho, r + h, Y, K);
            for (size_t i = 0; ok && i < NP; ++i) nxt[i] = psi[i] + (h / 6.0) * (acc[i] + K[i]);
        } else {
            for (int t = 0; t < nt; ++t) dl[t] = path_length(&c, t, r, h);
            for (int pass = 0; pass < 2 && ok; ++pass) {
                const double rr = pass == 0 ? r : r + h;
                double mu;
                mom_t M;
                geometry(&c, rr, &w.g, &mu);
                psi_to_rho(&c, pass == 0 ? psi : Y, rho);
                moments(&c, rho, &w.g, M, w.Sbuf);
                if (!moments_finite(&c, M)) {
                    ok = 0;
                    break;
                }
                const double A = matter_A(&c, rr);
                if (pass == 0) propagate_psi(&c, M, mu, A, &w.g, dl, psi, Y); /* predictor */
                else {
                    propagate_psi(&c, M, mu, A, &w.g, dl, psi, K);
                    for (size_t i = 0; i < NP; ++i) nxt[i] = 0.5 * (Y[i] + K[i]);
                }
            }
        }
        for (size_t i = 0; ok && i < NP; ++i)
            if (!isfinite(creal(nxt[i])) || !isfinite(cimag(nxt[i]))) ok = 0;
        if (!ok) {
            status = 1;
            break;
        }
        cplx *tmp = psi;
        psi = nxt;
        nxt = tmp;
        ++done;
    }
    for (size_t i = 0; i < NP; ++i) {
        psi_packed[2 * i] = creal(psi[i]);
        psi_packed[2 * i + 1] = cimag(psi[i]);
    }
    if (steps_done) *steps_done = done;
    free(psi);
    free(nxt);
    free(Y);
    free(K);
    free(acc);
    free(rho);
    free(dl);
    scratch_free(&w);
    ctx_free(&c);
    return status;
}

/* Cylinder model: the latitude shift Phi' - Phi of background angle bin jp
 * seen from angle bin j at radius r, and its coupling weight
 * w_jp (1 - cos(alpha_j - alpha_jp)) (Eq. 3.20); 0, or -1 for a bad index. */
int orc_cyl_pair(const orc_params *p, double r, int j, int jp, double *shift, double *weight)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc || p->geometry != ORC_CYLINDER || j < 0 || jp < 0 || j >= c.nu || jp >= c.nu) {
        ctx_free(&c);
        return rc ? rc : -1;
    }
    scratch_t w;
    scratch_alloc(&c, &w);
    double mu;
    geometry(&c, r, &w.g, &mu);
    double a = w.g.alpha[j * c.nphi], ap = w.g.alpha[jp * c.nphi];
    *shift = c.th[jp] - c.th[j] + a - ap;
    *weight = w.g.wc[jp * c.nphi] * (1.0 - cos(a - ap));
    scratch_free(&w);
    ctx_free(&c);
    return 0;
}

/* Moments of a packed state at radius r (packed Hermitian n*n each). */
/* All four moments of a packed state at radius r (Eq. 3.13 / 3.18): Mp holds
 * M0, M1, M2, M3 packed (n*n each); M2 = M3 = 0 without azimuth bins. */
int orc_moments_ex(const orc_params *p, const double *rho_packed, double r, double *Mp)
{
    orc_ctx c;
    int rc = ctx_init(&c, p);
    if (rc) {
        ctx_free(&c);
        return rc;
    }
    size_t N = (size_t)c.nbins * c.m;
    cplx *rho = malloc(sizeof(cplx) * N);
    for (int b = 0; b < c.nbins; ++b) unpack(c.n, rho_packed + (size_t)b * c.m, rho + (size_t)b * c.m);
    scratch_t w;
    scratch_alloc(&c, &w);
    double mu;
    mom_t M;
    geometry(&c, r, &w.g, &mu);
    moments(&c, rho, &w.g, M, w.Sbuf);
    for (int q = 0; q < 4; ++q) pack(c.n, M[q], Mp + (size_t)q * c.m);
    free(rho);
    scratch_free(&w);
    ctx_free(&c);
    return 0;
}

/* Moments M0 and M1 of a packed state at radius r (packed Hermitian n*n each). */
int orc_moments(const orc_params *p, const double *rho_packed, double r, double *M0p, double *M1p)
{
    double M[4 * NFMAX * NFMAX];
    int rc = orc_moments_ex(p, rho_packed, r, M);
    if (rc) return rc;
    const int m = p->n_f * p->n_f;
    memcpy(M0p, M, sizeof(double) * m);
    memcpy(M1p, M + m, sizeof(double) * m);
    return 0;
}

/* Matter potential and single-angle factor at r, for tests. */
double orc_matter_A(const orc_params *p, double r)
{
    orc_ctx c;
    if (ctx_init(&c, p)) {
        ctx_free(&c);
        return NAN;
    }
    double A = matter_A(&c, r);
    ctx_free(&c);
    return A;
}
