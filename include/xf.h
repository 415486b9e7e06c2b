/*
 * xf.h -- C ABI of the GB300 flavor-evolution library (libxf.so).
 *
 * The library integrates the nonlinear mean-field flavor equations of the
 * neutrino bulb model (XFLAT, arXiv 1907.05560, Sec. 3.1-3.2): for every
 * angle bin u and energy bin E it evolves the neutrino and antineutrino
 * density matrices rho(E,u) (2 or 3 flavors) in radius r,
 *     d rho / dr = -i [H, rho] dl/dr,                     (Eq. 3.2, Eq. 3.4)
 *     H_nu    = H_vac(E) + A(r) P_e + G_u,                 (Eq. 3.5-3.7)
 *     H_nubar = H_vac(E) - A(r) P_e - conj(G_u),           (rule after Eq. 3.4)
 *     G_u     = mu (M0 - cos(theta_u) M1),                 (Eq. 3.13-3.15)
 * where M0 and M1 are reductions over every bin of rho_nu - conj(rho_nubar).
 * Each integrator stage is one fused GPU pass (moment reduction + per-bin
 * update) inside a persistent kernel with a grid-wide barrier.
 *
 * Conventions for every entry point:
 *   - Return value: XF_OK (0) or a negative XF_E_* code.  No function throws,
 *     aborts or exits; xf_last_error(ctx) describes the last failure.
 *   - Handles are opaque and owned by the caller until xf_destroy.
 *   - Every pointer argument is caller-owned; the library copies what it needs
 *     before returning and keeps no pointer after return (except the
 *     allocator callbacks and the stream handle, which must outlive the ctx).
 *   - Host arrays use the packed layout below.  Device memory is allocated by
 *     the library (cudaMalloc, or the allocator given to xf_create_ex).
 *   - Calls on one ctx are not thread-safe; distinct ctxs are independent.
 *
 * Packed host layout of a state (n_doubles = 2 * n_u * n_E * n_f * n_f):
 *   rho[((s * n_u + j) * n_E + e) * n_f*n_f + k], s = 0 neutrino, 1 antineutrino,
 *   j = angle bin, e = energy bin; per bin k runs over the n_f real diagonal
 *   entries, then (Re, Im) of the upper-triangle entries in row order:
 *   2 flavors (rho11, rho22, Re rho12, Im rho12); 3 flavors (rho11, rho22,
 *   rho33, Re/Im rho12, Re/Im rho13, Re/Im rho23).  Flavor order e, x (2 fl)
 *   or e, mu, tau (3 fl).
 * Grids: E_e = E_min + (e + 1/2) dE, dE = (E_max - E_min)/n_E; angle variable
 *   u_j = (j + 1/2)/n_u with u = sin^2(theta_0) at the neutrinosphere (Eq. 3.14).
 */
#ifndef XF_H
#define XF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define XF_OK 0
#define XF_PENDING 1              /* xf_poll: job not finished yet */
#define XF_E_ARG (-1)             /* bad argument: null, size, enum, range */
#define XF_E_STATE (-2)           /* state values not finite / not Hermitian-packable */
#define XF_E_NOMEM (-3)           /* device or host allocation failed */
#define XF_E_CUDA (-4)            /* CUDA runtime error (message in xf_last_error) */
#define XF_E_NONFINITE (-5)       /* integration produced a non-finite moment; state
                                     is left at the last finite step */
#define XF_E_BARRIER_TIMEOUT (-6) /* a grid barrier wait exceeded its time limit */
#define XF_E_UNSTABLE (-7)        /* strict mode: RK4 step outside its stable region */
#define XF_E_BUSY (-8)            /* serving: queue full */
#define XF_E_TOO_BIG (-9)         /* serving: job larger than the memory budget */
#define XF_E_NOTFOUND (-10)       /* serving: unknown job id */
#define XF_E_TIMEOUT (-11)        /* serving: job exceeded its time limit */
#define XF_E_UNSUPPORTED (-12)    /* combination not built */
#define XF_E_STEPSIZE (-13)       /* error-controlled step: step size fell below 1e-12 r */
#define XF_E_BUDGET (-14)         /* error-controlled step: attempt budget spent before r_end */

/* ---- enums -------------------------------------------------------------- */
enum xf_stepper {
    XF_RK4 = 0,  /* classic fixed-step RK4 on d rho/dr = -i[H,rho] dl/dr: 4 fused stages */
    XF_EXPH = 1, /* the paper's coarse predictor-corrector (Sec. 4.2.3, Listing 5.1 S1-S3)
                    with the exact propagator exp(-i H dl) (Eq. 3.10-3.12): 2 stages */
    XF_EXPH_ADAPTIVE = 2 /* the paper's error-controlled step (Sec. 4.2.3, Fig. 4.8-4.9,
                    S1-S5 of Listings 5.1-5.3): per attempt a coarse path (the XF_EXPH step)
                    and a fine path (half step, midpoint half step, full step under the end-
                    point Hamiltonian, averaged) from four Hamiltonians in 3 fused stages;
                    error = max over bins of |rho_c - rho_f| / tr rho; accepted (coarse
                    result kept) when error <= eps0; next step ksi h (eps0/error)^(1/2)
                    trimmed to dr_max.  Driven by xf_evolve / xf_batch_evolve, FP64 and
                    XF_FP32_M64 only */
};
enum xf_precision {
    XF_FP64 = 0,        /* FP64 everywhere */
    XF_FP32_M64 = 1,    /* FP32 per-bin arithmetic and storage; FP64 moments, radius, phase */
    XF_FP32_COMP = 2,   /* as FP32_M64, but each thread's and each warp's moment sums are
                           compensated FP32 (TwoSum, error carried beside the sum) before the
                           FP64 sum over warps and tiles */
    XF_FP32_M64_RENORM = 3 /* FP32_M64 plus, after every step, each bin's traceless part scaled
                              back to its initial tr(T^2) (|P| in 2 flavors, tr rho^2 in 3; both
                              are constants of the exact flow, Eq. 3.10).  The trace is exact in
                              every variant (kept per bin in FP64, never updated) */,
    XF_FP32X2 = 4 /* FP64 state, tables, moments, radius and phase; the predictor-corrector's
                     propagator (Eq. 3.10-3.12: the eigendecomposition and U T U^dagger) in
                     float-float arithmetic (hi + lo of two floats, about 48 bits; Dekker's
                     products and Knuth's sums) on the FP32 pipes.  XF_EXPH only; fixed steps,
                     density matrices, bulb-type geometries, one azimuth bin; batches and the
                     server accept it.  Error per propagation about 1e-14 of |T| (FP32 bins:
                     1.5e-7), so it meets the FP32 target where FP32 rounding is amplified.
                     Float-float numbers keep float's exponent range: Hamiltonian entries
                     and their squares must stay within 1e-38 .. 3e38 (km^-1), else the run
                     stops with XF_E_NONFINITE */
};
enum xf_geometry {
    XF_GEOM_BULB = 0,         /* Eq. 3.13-3.15: w_u = x^2 du/(2 cos_u), x = R/r; dl/dr = 1/cos_u */
    XF_GEOM_MU_R4 = 1,        /* literal mu0 (R/r)^4 with r-independent weights du; dl/dr = 1/cos_u */
    XF_GEOM_SINGLE_ANGLE = 2, /* Eq. 3.16-3.17: G = mu0 D(r/R) dE sum(rho - conj rho_bar), dl = dr */
    XF_GEOM_CONST = 3,        /* isotropic, constant mu0: G = mu0 dE du sum(...), dl = dr */
    XF_GEOM_CYLINDER = 4      /* Sec. 3.2.5, Eq. 3.20: an infinite cylinder of radius R_nu emitting
                                 perpendicular to its axis.  n_u angle bins theta_j = -pi/2 +
                                 (j + 1/2) pi/n_u from the outward normal (clockwise), n_phi
                                 latitude bins Phi_k = (k + 1/2) 2 pi/n_phi; alpha_j =
                                 asin((R/r) sin theta_j), dl/dr = 1/cos(alpha_j);
                                 G_jk = mu0 (R/r) dE sum_j' w_j' (1 - cos(alpha_j - alpha_j'))
                                 D(Phi', j'), w_j' = cos(theta_j')/cos(alpha_j') pi/n_u,
                                 Phi' = Phi_k + theta_j' - theta_j + alpha_j - alpha_j', D the
                                 per-trajectory sum over E of (rho_nu - conj rho_nubar), read at
                                 Phi' by periodic linear interpolation.  Fixed steps, XF_FP64 or
                                 XF_FP32_M64, density-matrix form, n_u <= 2048, one problem per
                                 context, not strict.  The moments (xf_moments_ex) are the
                                 latitude averages of w, w cos(alpha), w sin(alpha) */
};
enum xf_form {
    XF_FORM_RHO = 0, /* density matrices rho(u, E), Eq. 3.1-3.4 */
    XF_FORM_PSI = 1  /* the wavefunction form (Eq. 3.9-3.11): per bin one wavefunction psi_a
                        for each initial flavor a (nu_e and the n_f - 1 others), rho =
                        sum_a phi_a psi_a psi_a^+ with phi_a the flavor's number-flux weight
                        (Eq. 4.1-4.2); each psi_a evolves with the Hamiltonian of rho.  The
                        XF_EXPH step averages the two propagated wavefunctions (no
                        renormalisation).  Fixed steps, XF_FP64 or XF_FP32_M64, one azimuth
                        bin; not served.  State I/O: xf_set_psi / xf_get_psi; every rho-valued
                        output (xf_get_state, xf_outputs, the moments, the energy average) is
                        computed from the wavefunctions */
};
enum xf_matter {
    XF_MATTER_NONE = 0,
    XF_MATTER_POWER = 1, /* n_e = ne_ref (r_ref/r)^ne_power   (Eq. 4.3 shape) */
    XF_MATTER_EXP = 2    /* n_e = Ye nb0 exp(-(r - R)/h_ns)      (Eq. 4.4) */
};

#define XF_PARAMS_VERSION 3u

/* Problem parameters.  Fill with xf_params_default, then set fields.
 * Keyword names of the paper's configuration file (App. A.3) in brackets. */
typedef struct xf_params {
    uint32_t size;      /* = sizeof(xf_params) */
    uint32_t version;   /* = XF_PARAMS_VERSION */
    int32_t stepper;    /* enum xf_stepper */
    int32_t precision;  /* enum xf_precision */
    int32_t geometry;   /* enum xf_geometry */
    int32_t hierarchy;  /* +1 normal, -1 inverted: sign of dm2 (2 fl) / dm2_31 (3 fl) */
    int32_t matter;     /* enum xf_matter */
    int32_t n_phi;      /* azimuth bins of the extended bulb model (Eq. 3.18) [Pbins], or the
                           latitude bins of XF_GEOM_CYLINDER; 1 = the
                           azimuthally symmetric bulb model (default).  > 1 needs XF_GEOM_BULB
                           or XF_GEOM_CYLINDER, a fixed-step stepper and XF_FP64 or XF_FP32_M64.
                           A problem has 2 n_u n_phi n_E bins, ordered [s][u][phi][E] in every
                           host array */
    int32_t form;       /* enum xf_form: what a bin's state is (default XF_FORM_RHO) */
    int32_t strict;     /* 1: xf_step / xf_batch_step with RK4 return XF_E_UNSTABLE, without
                           stepping, when for some angle u
                           h kappa_u sqrt(2) (max_E |H_vac| + A |P_e| + mu |M0 - gamma_u M1|)
                           exceeds RK4's imaginary-axis bound 2 sqrt(2) (Frobenius norms of the
                           traceless parts at the current radius and state, kappa_u = dl/dr) */
    double R_nu_km;     /* neutrinosphere radius [R0 is the start radius; R_nu is Eq. 3.14's R] */
    double mu0_per_km;  /* nu-nu coupling, absorbs the normalisation of Eq. 3.8 */
    double E_min_MeV, E_max_MeV; /* [E0, E1] */
    double dm2_eV2[2];  /* magnitudes; 2 fl: dm2[0] [dm2]; 3 fl: dm2_21, dm2_31 */
    double theta[3];    /* 2 fl: theta[0] [theta]; 3 fl: theta12, theta13, theta23 (delta_CP = 0) */
    double ne_ref_cm3, r_ref_km, ne_power; /* XF_MATTER_POWER */
    double nb0_cm3, h_ns_km, Ye;           /* XF_MATTER_EXP [nb0, hNS, Ye] */
    double T_MeV[4];    /* temperatures nu_e, nubar_e, nu_x, nubar_x [T*] */
    double eta[4];      /* degeneracy parameters [eta*] */
    double L[4];        /* luminosities, any common unit [L*] */
    double eps_perturb; /* seeded off-diagonal amplitude (fraction of sqrt(rho_ii rho_jj)) */
    uint64_t seed;      /* seed of the SplitMix64 phases of the perturbation */
    double eps0;        /* XF_EXPH_ADAPTIVE: error tolerance [eps0], default 1e-6 */
    double ksi;         /* XF_EXPH_ADAPTIVE: safety factor of the step update, (0, 1] [ksi], default 0.9 */
    double dr_max_km;   /* XF_EXPH_ADAPTIVE: largest step [max_dr], default 1 km */
} xf_params;

typedef struct xf_ctx xf_ctx;

/* Device allocator hook: alloc(bytes, user) returns a device pointer or NULL;
 * free(ptr, user) releases it.  Must stay valid until xf_destroy. */
typedef struct xf_allocator {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} xf_allocator;

/* Default parameters: the bulb-model values of Sec. 4.5 (eta = 3,
 * T = 2.76/4.01/6.26 MeV, equal L, R = 10 km, theta = 0.1), RK4, FP64, BULB,
 * no matter, dm2 = 2.4e-3 eV^2 inverted, mu0 = 1e5 km^-1, eps = 1e-6, seed 1.
 * p must be non-null. */
void xf_params_default(xf_params *p);

/* Create a context for one problem of n_u angle bins x n_E energy bins x
 * {nu, nubar}, n_flavor in {2, 3}.  Validates p (XF_E_ARG on bad sizes,
 * enums, non-finite or non-positive physical values), builds the per-energy
 * tables on the host in FP64 and allocates the device state.  On success
 * *out owns the context; on failure *out is NULL.  The state is undefined
 * until xf_set_state or xf_init_state. */
int xf_create(int n_E, int n_u, int n_flavor, const xf_params *p, xf_ctx **out);
/* As xf_create, with device memory taken from `alloc` (NULL: cudaMalloc). */
int xf_create_ex(int n_E, int n_u, int n_flavor, const xf_params *p, const xf_allocator *alloc,
                 xf_ctx **out);
/* Release the context and its device memory.  NULL is accepted (no-op). */
int xf_destroy(xf_ctx *ctx);

/* Use `stream` (a cudaStream_t) for all later work on this ctx; NULL = the
 * legacy default stream.  The stream must outlive its use by the ctx. */
int xf_set_stream(xf_ctx *ctx, void *stream);

/* Copy a packed host state (layout above, n_doubles exact) to the device and
 * set the radius to r_km (>= R_nu).  XF_E_STATE if any value is non-finite.  The trace
 * of every bin is kept in FP64 and never changes (d tr rho/dr = 0). */
int xf_set_state(xf_ctx *ctx, const double *rho, size_t n_doubles, double r_km);

/* Seeded initial state at radius r_km (>= R_nu): rho_nu(u,E) = diag(phi_nue(E),
 * phi_nux(E)[, phi_nux(E)]), rho_nubar likewise with the antineutrino spectra
 * (Eq. 4.1-4.2; phi_a = (L_a/<E_a>) f_a(E) relative to nu_e), and each upper
 * entry (i<j) = eps sqrt(rho_ii rho_jj) exp(2 pi i U), U the SplitMix64 uniform
 * number at counter b * n_f(n_f-1)/2 + k for bin b = (s n_u + j) n_E + e. */
int xf_init_state(xf_ctx *ctx, double r_km);

/* Advance n_steps >= 0 fixed steps of dr_km > 0 from the current radius.
 * Synchronous: returns when the work has finished on the ctx stream.
 * XF_E_NONFINITE: the state is left at the last step whose moments were
 * finite (xf_get_state reports how many steps were taken).
 * XF_E_BARRIER_TIMEOUT: a grid barrier did not complete within its limit; the
 * kernel returned without hanging and the state is undefined. */
int xf_step(xf_ctx *ctx, int64_t n_steps, double dr_km);
/* As xf_step but returns after enqueuing (no host synchronisation); errors
 * from the device are reported by the next synchronous call on the ctx. */
int xf_step_async(xf_ctx *ctx, int64_t n_steps, double dr_km);
/* Wait for enqueued work; returns its device status. */
int xf_sync(xf_ctx *ctx);

/* Copy the current state to a packed host array (n_doubles exact); r_km and
 * steps_done (total steps since the last set/init) may be NULL. */
int xf_get_state(xf_ctx *ctx, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done);

/* The wavefunction form (XF_FORM_PSI).  psi: n_doubles = 2 n_f^2 * bins
 * doubles, [s][u][phi][E][a][i] as (re, im) pairs: bin b's wavefunction of
 * initial flavor a has components i = 0..n_f-1.  xf_set_psi copies it in at
 * radius r_km (>= R_nu), XF_E_STATE if a value is not finite;
 * xf_get_psi copies the current wavefunctions out (r_km, steps_done as
 * xf_get_state, either may be NULL).  xf_init_state seeds
 * psi_a = (e_a + eps sum_{b != a} exp(2 pi i U_ab) e_b) / sqrt(1 + (n_f-1) eps^2),
 * U_ab the SplitMix64 uniform number at counter bin n_f(n_f-1) + k, k running
 * over the pairs (a, b != a) in row order.  XF_E_UNSUPPORTED on a
 * density-matrix ctx, and xf_set_state is XF_E_UNSUPPORTED on a wavefunction
 * ctx (a density matrix does not fix its wavefunctions). */
int xf_set_psi(xf_ctx *ctx, const double *psi, size_t n_doubles, double r_km);
int xf_get_psi(xf_ctx *ctx, double *psi, size_t n_doubles, double *r_km, int64_t *steps_done);
int xf_batch_set_psi(xf_ctx *ctx, int inst, const double *psi, size_t n_doubles, double r_km);
int xf_batch_get_psi(xf_ctx *ctx, int inst, double *psi, size_t n_doubles, double *r_km,
                     int64_t *steps_done);

/* nu-nu moments of the current state at the current radius (Eq. 3.13-3.15
 * for the ctx geometry), packed Hermitian n_f*n_f doubles each (layout of one
 * bin above), trace included, computed on the device in FP64:
 *   M0 = dE sum_{u,E} a_u (rho_nu - conj rho_nubar),  M1 = dE sum b_u (...),
 *   BULB: a_u = x^2 du / (2 cos_u), b_u = a_u cos_u. */
int xf_moments(xf_ctx *ctx, double *M0, double *M1, size_t n_doubles);
/* All four moments of the extended bulb model (Eq. 3.18): M[4][n_f*n_f],
 * M0 and M1 as above, M2 and M3 the sin th cos ph / sin th sin ph weighted
 * ones (zero with one azimuth bin).  inst = 0 for a single problem. */
int xf_moments_ex(xf_ctx *ctx, int inst, double *M, size_t n_doubles);

/* Per-bin outputs of the current state (Sec. 4.5 survival probability), each
 * array n_bins = 2 n_u n_E doubles in [s][u][E] order, any may be NULL:
 *   p_surv: (rho_ee - phi_x)/(phi_e - phi_x) with phi the initial diagonal
 *           weights of that species and energy (NaN where phi_e == phi_x);
 *   trace:  tr rho;   purity: tr(rho0^2), rho0 the traceless part
 *           (= |P|^2/2 in two flavors). */
int xf_outputs(xf_ctx *ctx, double *p_surv, double *trace, double *purity, size_t n_bins);

/* Host copies of the per-energy tables, for inspection: E[n_E] (MeV),
 * phi[4 * n_E] (nu_e, nubar_e, nu_x, nubar_x).  Any pointer may be NULL. */
int xf_tables(xf_ctx *ctx, double *E, double *phi);

/* Number of grid barriers per integrator step of this ctx's stepper
 * (RK4: 4, EXPH: 2) and the device grid size used. */
int xf_launch_info(xf_ctx *ctx, int *ctas, int *threads, int *barriers_per_step);

/* ---- batches: many problems in one persistent launch ----------------------
 * A batch ctx holds several independent problems (sizes, flavors, couplings,
 * hierarchies and spectra may all differ; stepper and precision are shared)
 * and advances them together: one cooperative launch per call tiles every
 * problem into runs of (angle, energy) pairs, and each problem's moments are
 * summed from its own tiles only, so a problem's result does not depend on
 * what it is packed with (bitwise, for equal tile size and precision).
 * The single-problem calls above act on problem 0 of a batch. */
typedef struct xf_problem {
    int32_t n_E, n_u, n_flavor, reserved; /* reserved: set to 0 */
    xf_params params;
} xf_problem;

/* Create a batch of n_problems >= 1 problems (validated as xf_create does;
 * XF_E_ARG if steppers or precisions differ).  All states start undefined. */
int xf_create_batch(int n_problems, const xf_problem *problems, const xf_allocator *alloc, xf_ctx **out);
int xf_batch_size(xf_ctx *ctx, int *n_problems);
/* Per-problem state I/O (layouts and rules as the single-problem calls);
 * xf_batch_init_state with inst = -1 initialises every problem. */
int xf_batch_set_state(xf_ctx *ctx, int inst, const double *rho, size_t n_doubles, double r_km);
int xf_batch_init_state(xf_ctx *ctx, int inst, double r_km);
int xf_batch_get_state(xf_ctx *ctx, int inst, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done);
int xf_batch_outputs(xf_ctx *ctx, int inst, double *p_surv, double *trace, double *purity, size_t n_bins);
/* Advance every problem by n_steps steps; dr_km holds one step size per
 * problem (NULL: each keeps its previous one).  Synchronous.  A problem whose
 * moments turn non-finite stops at its last finite state while the others
 * continue: xf_batch_status tells which (status XF_OK / XF_E_NONFINITE /
 * XF_E_STATE), how many steps each took and its radius. */
int xf_batch_step(xf_ctx *ctx, int64_t n_steps, const double *dr_km);
int xf_batch_status(xf_ctx *ctx, int inst, int *status, int64_t *steps_done, double *r_km);
/* The moments M0, M1 (Eq. 3.13, host arrays of n_f*n_f doubles each, packed
 * like a bin) of problem `inst`'s current state as the integrator's own
 * in-launch reduction summed them, i.e. in the precision variant's
 * arithmetic (FP32 terms and warp sums, compensated for XF_FP32_COMP, FP64
 * above the warp).  Traceless part only: the trace part of nu - conj(nubar)
 * adds a multiple of the identity to H, which the flow ignores, so the
 * integrator never forms it (the diagonal entries sum to zero).  Compare with
 * xf_moments / the batch's FP64 moments of the same state to see the
 * summation error.  Valid after a step call that advanced the problem;
 * XF_E_STATE before that (and after a state reset or a non-finite stop).
 * Also accepts a single-problem context with inst = 0. */
int xf_batch_run_moments(xf_ctx *ctx, int inst, double *M0, double *M1, size_t n_doubles);

/* ---- error-controlled integration (stepper XF_EXPH_ADAPTIVE) -------------
 * Integrate until r_end_km (the last step is shortened to land on it; a
 * radius within 1e-12 r_end counts as arrived), making at most max_iters
 * attempts (accepted + rejected).  dr0_km: the first step to try; <= 0
 * keeps the step size the previous call ended with (dr_max if none).
 * Synchronous.  Returns XF_OK when r_end was reached; XF_E_BUDGET when the
 * attempts ran out first (state and radius are those of the last accepted
 * step, and a further call continues); XF_E_NONFINITE when an attempt was
 * not finite (state kept at the last accepted step); XF_E_STEPSIZE when the
 * step fell below 1e-12 r.  XF_E_ARG on a context of another stepper.
 * xf_step / xf_batch_step are XF_E_ARG on an XF_EXPH_ADAPTIVE context. */
int xf_evolve(xf_ctx *ctx, double r_end_km, int64_t max_iters, double dr0_km);
/* Every problem of a batch to its own r_end_km[i] (dr0_km: NULL, or one
 * value per problem as above).  Returns XF_OK if all arrived, else the first
 * non-OK status in problem order (xf_adapt_status tells each). */
int xf_batch_evolve(xf_ctx *ctx, const double *r_end_km, int64_t max_iters, const double *dr0_km);
/* Outcome of problem `inst`'s last error-controlled call: status (XF_OK,
 * XF_E_BUDGET, XF_E_NONFINITE, XF_E_STEPSIZE), radius, the next step size,
 * accepted and rejected attempts of the call, and the last attempt's error.
 * Any output pointer may be NULL. */
int xf_adapt_status(xf_ctx *ctx, int inst, int *status, double *r_km, double *h_next_km, int64_t *n_accepted,
                    int64_t *n_rejected, double *last_error);

/* ---- snapshots, checkpoints and reduced outputs (the paper's I/O module,
 * Sec. 4.2.4: dump mode 1 = a snapshot of every bin's state from which a run
 * resumes; dump mode 2 = the flavor state of each trajectory averaged over
 * its energy bins) ------------------------------------------------------------
 * A checkpoint is the problem's state in the library's own device layout
 * (traceless components in the working precision, the FP64 trace per bin,
 * the renormalising variant's reference values) plus its position (radius,
 * step size, step counts, error-controlled progress), so loading it and
 * continuing gives bitwise the same result as never having stopped.  The
 * buffer is opaque, versioned and tied to the problem's shape, stepper and
 * precision.  inst = 0 for a single-problem context. */
int xf_checkpoint_bytes(xf_ctx *ctx, int inst, size_t *bytes);
/* Synchronous save into host memory of xf_checkpoint_bytes bytes. */
int xf_checkpoint_save(xf_ctx *ctx, int inst, void *buf, size_t bytes);
/* Asynchronous save: the state is copied on the device in the context's
 * stream order (after the steps already enqueued), then to `buf` on a
 * separate copy stream, so steps enqueued after this call run while the
 * copy to the host is in flight.  `buf` must stay valid until
 * xf_checkpoint_wait; pinned host memory makes the copy truly asynchronous.
 * One save may be in flight per context (XF_E_BUSY otherwise). */
int xf_checkpoint_save_async(xf_ctx *ctx, int inst, void *buf, size_t bytes);
int xf_checkpoint_wait(xf_ctx *ctx);
/* Restore problem `inst` from a checkpoint (XF_E_ARG if the buffer is not a
 * checkpoint of a problem of this shape, stepper and precision). */
int xf_checkpoint_load(xf_ctx *ctx, int inst, const void *buf, size_t bytes);
/* Dump mode 2: out[s][t][n_f*n_f] (packed like a bin) = the mean over the
 * n_E energy bins of trajectory t's density matrices (t = u n_phi + phi),
 * s = 0 nu, 1 nubar; summed in FP64 on the device in energy order.
 * n_doubles = 2 n_u n_phi n_f^2. */
int xf_angle_average(xf_ctx *ctx, int inst, double *out, size_t n_doubles);

/* ---- serving: a continuous-batching job server ---------------------------
 * A server owns one pack of `max_jobs` slots and a device arena of
 * `mem_budget_bytes`, and a scheduler thread that repeats epochs:
 *   1. admit queued jobs (first come, first served) while a slot is free
 *      and their state fits the memory budget;
 *   2. advance every resident job by min(its remaining steps, chunk_steps)
 *      in one persistent launch;
 *   3. retire finished jobs (state copied to host if kept), freeing slots
 *      and memory for the next admissions.
 * Jobs that arrive while others run are thus admitted between launches and
 * share the GPU with them.  The server uses a fixed tile size, so a job's
 * result is the same (bitwise, for equal tile size, stepper and precision)
 * alone and in any mix.  Timestamps are seconds since xf_server_create. */
typedef struct xf_server xf_server;
typedef struct xf_server_cfg {
    uint32_t size;            /* = sizeof(xf_server_cfg) */
    int32_t max_jobs;         /* resident slots, >= 1 */
    int64_t mem_budget_bytes; /* device memory for resident jobs (their blocks) */
    int64_t chunk_steps;      /* radial steps per epoch, >= 1 */
    int32_t queue_cap;        /* queued jobs beyond which xf_submit returns XF_E_BUSY */
    int32_t stepper;          /* shared by all jobs */
    int32_t precision;        /* shared by all jobs */
    int32_t n_flavor;         /* 2 or 3 (every job), or 0 (mixed) */
    int32_t tile_pairs;       /* tile size in pairs (0: 1024) */
    int32_t reserved;         /* set to 0 */
} xf_server_cfg;
typedef struct xf_job {
    xf_problem problem;       /* its params.stepper / precision must match the server's */
    double r0_km, dr_km;      /* start radius (>= R_nu) and step size */
    int64_t n_steps;          /* steps to take, >= 1 */
    const double *rho0;       /* packed host state at r0_km (copied at submit), or NULL
                                 for the seeded initial state of xf_init_state */
    int32_t keep_state;       /* 1: keep the final state for xf_poll */
    int32_t reserved;         /* set to 0 */
} xf_job;
typedef struct xf_job_result {
    int32_t status;           /* XF_OK, or XF_E_NONFINITE (state = last finite step) */
    int32_t reserved;
    int64_t steps_done;
    double r_km;              /* radius of the final state */
    double t_submit, t_start, t_done; /* queued, admitted, finished (s) */
} xf_job_result;
typedef struct xf_server_stats {
    int64_t submitted, completed, queued, resident, max_resident;
    int64_t epochs;
    double bin_steps;         /* sum over launches of bins x steps taken */
    double busy_s;            /* time spent in launches */
    int64_t mem_used_bytes, mem_peak_bytes;
} xf_server_stats;

/* Create a server (XF_E_ARG on bad configuration); the scheduler thread
 * starts at once and uses the device current in the calling thread. */
int xf_server_create(const xf_server_cfg *cfg, xf_server **out);
/* Queue a job; *job_id identifies it.  XF_E_ARG: invalid job; XF_E_TOO_BIG:
 * its block exceeds the memory budget; XF_E_BUSY: the queue is full. */
int xf_submit(xf_server *srv, const xf_job *job, uint64_t *job_id);
/* XF_PENDING while the job is queued or running.  When finished: XF_OK,
 * *res filled, the final state copied to rho_out (n_doubles exact; if the job
 * kept it and rho_out is non-NULL) and the job forgotten.  XF_E_NOTFOUND for
 * an unknown (or already collected) id. */
int xf_poll(xf_server *srv, uint64_t job_id, xf_job_result *res, double *rho_out, size_t n_doubles);
/* Wait until every submitted job has finished, at most timeout_s seconds
 * (XF_E_TIMEOUT when it runs out). */
int xf_server_drain(xf_server *srv, double timeout_s);
int xf_server_get_stats(xf_server *srv, xf_server_stats *st);
/* Stop the scheduler, drop queued and resident jobs, free everything. */
int xf_server_destroy(xf_server *srv);

/* Options (xf_set_option), for tuning and testing:
 *   XF_OPT_GRID: persistent grid size in CTAs; 0 = automatic (default).  The
 *     value is clamped to the co-resident maximum and to the tile count.
 *   XF_OPT_TILE_PAIRS: tile size in (angle, energy) pairs, rounded up to a
 *     multiple of 32; 0 = automatic (one problem: one tile per co-resident
 *     CTA slot; several problems: about 8 tiles per slot).  Each problem's
 *     reduction tree follows its tiles, so a different tile size can change
 *     results by rounding; equal tile sizes give bitwise equal results.
 *   XF_OPT_GRAPH: 1 = capture the launch sequence of a step call into a CUDA
 *     graph on first use and replay it afterwards (re-captured when the
 *     step count per launch or the tiling changes); 0 = plain launches.
 *   XF_OPT_BARRIER_TIMEOUT_NS: time limit of one grid-barrier wait
 *     (default 2e9 ns).  On expiry every CTA leaves and the call returns
 *     XF_E_BARRIER_TIMEOUT.
 *   XF_OPT_DYNAMIC_TILES: 1 = when a pack has more tiles than CTAs, every
 *     stage's tiles are claimed from a device counter instead of each CTA
 *     taking its own run of them (fixed-step steppers); 0 (default) = own
 *     runs.  The results do not depend on it (a tile's arithmetic is the
 *     same wherever it runs, and the moments add in tile order).  Claiming
 *     pays on packs of unequal problems whose cost the static split
 *     misjudges, and costs two CTA barriers and an atomic per tile;
 *     xf_autotune measures both.
 *   XF_OPT_TEST_SKIP_ARRIVAL: test hook; CTA `value` (>= 0) leaves the kernel
 *     at its first grid barrier without arriving, so the other CTAs' bounded
 *     wait runs out.  -1 (default) disables it.  Exercises the timeout path
 *     without faulting or hanging the GPU. */
enum xf_option {
    XF_OPT_GRID = 1,
    XF_OPT_BARRIER_TIMEOUT_NS = 2,
    XF_OPT_TEST_SKIP_ARRIVAL = 3,
    XF_OPT_TILE_PAIRS = 4,
    XF_OPT_GRAPH = 5,
    XF_OPT_DYNAMIC_TILES = 6
};
int xf_set_option(xf_ctx *ctx, int option, int64_t value);
/* Current value of an option (for XF_OPT_GRID and XF_OPT_TILE_PAIRS the
 * request, 0 = automatic; after xf_autotune the settings it chose).
 * XF_E_ARG for an unknown option or a NULL pointer. */
int xf_get_option(xf_ctx *ctx, int option, int64_t *value);

/* Measured search of the tile size of a fixed-step context or batch: for
 * each candidate (pairs per tile; 0 = the automatic rule; candidates = NULL
 * takes 0, 128, 256, 512, 1024, 2048, 3072, 4096, 5120, 6144, 8192, 12288
 * and 16384), time n_probe steps of size dr_km (<= 0:
 * each problem's current step size) after one untimed launch, and keep the
 * fastest, which stays set as XF_OPT_TILE_PAIRS.  On a batch mixing two-
 * and three-flavor problems each candidate also runs with 0.7 and 1.4 times
 * the default cost weight of a three-flavor pair in the split of tiles over
 * CTAs, and the fastest weight stays set.  Every plan with more tiles than
 * CTAs also runs with XF_OPT_DYNAMIC_TILES on and off, and the faster
 * setting stays.  Every problem's state,
 * radius and step count are restored afterwards (device copies of the state
 * planes), so the search does not advance the problems.  Needs a valid
 * state in every problem.  *best_tile (may be NULL) receives the chosen
 * size, *best_ms (may be NULL) its time per step in milliseconds.  Results
 * depend on the tile size only by rounding (see XF_OPT_TILE_PAIRS). */
int xf_autotune(xf_ctx *ctx, int64_t n_probe, double dr_km, const int *candidates, int n_candidates,
                int *best_tile, double *best_ms);

/* Measured ALU peaks of the current device, for roofline denominators:
 * XF_PEAK_FP64_FMA / XF_PEAK_FP32_FMA write the FMA throughput in FLOP/s
 * (an FMA counts 2) of a register-resident FMA loop over 8 CTAs per SM,
 * best of 5 timed launches (CUDA events).  XF_PEAK_FP64_RSQRT and
 * XF_PEAK_FP64_SINCOS write calls per second of the FP64 reciprocal square
 * root and sine-cosine pair in the same kind of loop (each call with one FMA
 * that feeds the next), the two functions the 3x3 propagator (Eq. 3.11)
 * calls besides its counted arithmetic.  Not part of the integration. */
enum xf_peak_kind { XF_PEAK_FP64_FMA = 0, XF_PEAK_FP32_FMA = 1, XF_PEAK_FP64_RSQRT = 2, XF_PEAK_FP64_SINCOS = 3 };
int xf_peak(int which, double *value);

/* ---- stepping without allocation -----------------------------------------
 * Some callers cannot allocate device memory when they want to step a
 * problem: code that runs inside a memory pool owning the whole device
 * budget, plug-ins whose host application forbids allocation on its hot
 * path, and latency-bound loops where cudaMalloc's implicit synchronisation
 * is not acceptable.  xf_step_noalloc serves them.  It has no counterpart in
 * the paper: it is the xf_step integration (same kernels, same equations),
 * packaged so that the call allocates nothing.
 *
 * The caller passes the state in its own device memory: rho_dev holds
 * 2 * n_u * n_E * n_flavor^2 doubles in the packed layout above, is read as
 * the state at radius r_km (>= R_nu) and overwritten with the state after
 * n_steps steps of dr_km (on XF_E_NONFINITE: the last finite state).  All
 * working memory (component-major state buffers, the per-energy table, the
 * CTA partial moments, the barrier, error and step words) lives in one
 * file-scope device array of XF_NOALLOC_SCRATCH_BYTES that every GPU loading
 * libxf.so holds until the process exits.  The call makes no cudaMalloc,
 * cudaFree or other allocating call.  Steppers XF_RK4 and XF_EXPH, every
 * precision (XF_FP64, XF_FP32_M64, XF_FP32_COMP, XF_FP32_M64_RENORM),
 * geometries bulb, literal mu0 (R/r)^4, single-angle and constant, no azimuth
 * bins, the rho form (other choices: XF_E_UNSUPPORTED).
 *
 *   - n_steps == 0 returns XF_OK at once and leaves rho_dev untouched.
 *   - XF_E_STATE: rho_dev holds a non-finite value; refused before any step
 *     is taken, rho_dev untouched.
 *   - XF_E_TOO_BIG: the problem's working set (about 2(n_f^2-1) x 3 x
 *     sizeof(Real) + 16 bytes per (angle, energy) pair, plus small tables)
 *     exceeds XF_NOALLOC_SCRATCH_BYTES; nothing was run.
 *   - The call is synchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream): it synchronises the stream and reads status words back
 *     to the host, so it must never be called while `stream` is being
 *     captured into a CUDA graph.
 *   - Every failure's message is left where xf_last_error(NULL) reads it (per
 *     host thread, the same slot as a failed xf_create); a successful call
 *     clears it.
 *   - Every call shares the array and it keeps the previous call's contents;
 *     each call clears the words that must start at zero and rewrites the
 *     state buffers from rho_dev.  Calls whose GPU work overlaps (several
 *     host threads or streams at once) race on the array: serialise them.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current. */
#define XF_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int xf_step_noalloc(int n_E, int n_u, int n_flavor, const xf_params *p, double *rho_dev, double r_km,
                    int64_t n_steps, double dr_km, void *stream);

/* Human-readable name of a status code (static storage). */
const char *xf_status_str(int status);
/* Message of the last failure on ctx (static per-ctx storage; "" if none).
 * With ctx == NULL: the last failure of xf_create (or of the create calls of
 * batches and servers) or of xf_step_noalloc in this thread. */
const char *xf_last_error(const xf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* XF_H */
