// xf_api.cu -- host side of the C ABI declared in include/xf.h: argument
// validation, per-energy tables (FP64, on the host), device memory, layout
// conversion and the launches of the persistent integrator.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/xf.h"
#include "xf_aux.cuh"
#include "xf_kernels.h"

using namespace xf;

namespace {

// ---- physical constants (CODATA 2018 / PDG), stated for this library -----
constexpr double kHbarcEvKm = 1.973269804e-10; // hbar c, eV km
constexpr double kHbarcEvCm = 1.973269804e-5;  // hbar c, eV cm
constexpr double kFermiEv2 = 1.1663787e-23;    // G_F, eV^-2

// dm^2/(2E) in km^-1 for dm^2 in eV^2 and E in MeV (Eq. 3.6)
double vac_coefficient() { return 1.0 / (2.0e6 * kHbarcEvKm); }
// sqrt(2) G_F n_e in km^-1 per cm^-3 (Eq. 3.7)
double matter_coefficient() { return std::sqrt(2.0) * kFermiEv2 * std::pow(kHbarcEvCm, 3) / kHbarcEvKm; }

// Complete Fermi-Dirac integral F_k(eta) = int_0^inf x^k / (exp(x - eta) + 1) dx
// (Eq. 4.2) by composite 5-point Gauss-Legendre on [0, max(eta,0) + 60].
double fermi_dirac(int k, double eta)
{
    const double r1 = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
    const double r2 = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
    const double w0 = 128.0 / 225.0;
    const double w1 = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0;
    const double w2 = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
    const double xs[5] = {-r2, -r1, 0.0, r1, r2};
    const double ws[5] = {w2, w1, w0, w1, w2};
    const double top = std::max(eta, 0.0) + 60.0;
    const int panels = 4000;
    const double hw = 0.5 * top / panels;
    double sum = 0.0;
    for (int i = 0; i < panels; ++i) {
        const double mid = (2 * i + 1) * hw;
        double ps = 0.0;
        for (int q = 0; q < 5; ++q) {
            const double x = mid + hw * xs[q];
            ps += ws[q] * std::pow(x, k) / (std::exp(x - eta) + 1.0);
        }
        sum += ps * hw;
    }
    return sum;
}

thread_local std::string g_create_error;

// One enqueued launch: steps k0 .. k0 + n - 1 of the run r0 + k h.
struct Pending {
    double r0, h;
    long long k0, n;
};

} // namespace

struct xf_ctx {
    int n_E = 0, n_u = 0, nf = 0, S = 0, n_pairs = 0, npad = 0;
    long long n_bins = 0;
    xf_params p{};
    int real_bytes = 8;
    cudaStream_t stream = nullptr;
    xf_allocator alloc{};
    bool has_alloc = false;
    int device = 0, num_sms = 0;

    std::vector<double> E, phi, hvac; // host tables (phi [4][n_E], hvac [n_E][S])

    // device memory
    void *rho[2] = {nullptr, nullptr};
    void *aux = nullptr;
    void *hvac_d = nullptr;
    double *trace = nullptr, *phi_d = nullptr, *staging = nullptr;
    double *partials = nullptr, *mom_out = nullptr, *mom_part = nullptr, *mom_full = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr, *bad = nullptr;
    unsigned long long *steps = nullptr;
    std::vector<void *> owned;

    // launch shape
    RunKernel kern{nullptr, 0};
    int G = 1, pairs_per_cta = 0, span_max = 1;
    size_t smem = 0;
    int mom_G = 1, mom_chunk = 0;

    // run state.  Radii follow r = r_base + k h with k counted from the last
    // change of h, so a run split into several calls takes the same radii as
    // one call.  The "pred" fields anticipate the enqueued launches.
    bool state_valid = false;
    int cur = 0;                   // buffer of the current state (after sync)
    double r = 0.0;                // radius of the current state (after sync)
    long long steps_total = 0;
    double r_base = 0.0, h_base = 0.0;
    long long k_base = 0;
    int pred_cur = 0;
    double pred_r_base = 0.0, pred_h = 0.0;
    long long pred_k_base = 0;
    std::vector<Pending> pending;
    unsigned long long timeout_ns = 2000000000ull;
    int grid_request = 0, skip_cta = -1;

    std::string last_error;
};

namespace {

int fail(xf_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->last_error = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(xf_ctx *c, cudaError_t e, const char *what)
{
    cudaGetLastError(); // clear the sticky-free error state
    if (e == cudaErrorMemoryAllocation) return fail(c, XF_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(c, XF_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define XF_CUDA(ctx, call, what)                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);                                     \
    } while (0)

void *dev_alloc(xf_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (c->has_alloc) p = c->alloc.alloc(bytes, c->alloc.user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->owned.push_back(p);
    return p;
}

void free_all(xf_ctx *c)
{
    for (void *p : c->owned) {
        if (c->has_alloc) c->alloc.free(p, c->alloc.user);
        else cudaFree(p);
    }
    c->owned.clear();
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int validate(const xf_params *p, int n_E, int n_u, int nf)
{
    if (!p) return fail(nullptr, XF_E_ARG, "params is NULL");
    if (p->size != sizeof(xf_params)) return fail(nullptr, XF_E_ARG, "params.size %u != %zu", p->size, sizeof(xf_params));
    if (p->version != XF_PARAMS_VERSION) return fail(nullptr, XF_E_ARG, "params.version %u unsupported", p->version);
    if (n_E <= 0 || n_u <= 0) return fail(nullptr, XF_E_ARG, "n_E and n_u must be positive (got %d, %d)", n_E, n_u);
    if (nf != 2 && nf != 3) return fail(nullptr, XF_E_ARG, "n_flavor must be 2 or 3 (got %d)", nf);
    if ((long long)n_E * n_u > (long long)(INT_MAX / 16)) return fail(nullptr, XF_E_ARG, "n_E * n_u too large");
    if (p->stepper != XF_RK4 && p->stepper != XF_EXPH) return fail(nullptr, XF_E_ARG, "bad stepper %d", p->stepper);
    if (p->precision < XF_FP64 || p->precision > XF_FP32_M64_RENORM)
        return fail(nullptr, XF_E_ARG, "bad precision %d", p->precision);
    if (p->precision == XF_FP32_COMP || p->precision == XF_FP32_M64_RENORM)
        return fail(nullptr, XF_E_UNSUPPORTED, "precision %d not built", p->precision);
    if (p->geometry < XF_GEOM_BULB || p->geometry > XF_GEOM_CONST)
        return fail(nullptr, XF_E_ARG, "bad geometry %d", p->geometry);
    if (p->geometry == XF_GEOM_SINGLE_ANGLE && n_u != 1)
        return fail(nullptr, XF_E_ARG, "single-angle geometry needs n_u == 1");
    if (p->hierarchy != 1 && p->hierarchy != -1) return fail(nullptr, XF_E_ARG, "hierarchy must be +1 or -1");
    if (p->matter < XF_MATTER_NONE || p->matter > XF_MATTER_EXP) return fail(nullptr, XF_E_ARG, "bad matter %d", p->matter);
    if (!finite_pos(p->R_nu_km)) return fail(nullptr, XF_E_ARG, "R_nu_km must be finite and > 0");
    if (!std::isfinite(p->mu0_per_km) || p->mu0_per_km < 0) return fail(nullptr, XF_E_ARG, "mu0 must be finite and >= 0");
    if (!std::isfinite(p->E_min_MeV) || p->E_min_MeV < 0 || !std::isfinite(p->E_max_MeV) || p->E_max_MeV <= p->E_min_MeV)
        return fail(nullptr, XF_E_ARG, "need 0 <= E_min < E_max, finite");
    for (int i = 0; i < 2; ++i)
        if (!std::isfinite(p->dm2_eV2[i])) return fail(nullptr, XF_E_ARG, "dm2 not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(p->theta[i])) return fail(nullptr, XF_E_ARG, "theta not finite");
    for (int a = 0; a < 4; ++a)
        if (!finite_pos(p->T_MeV[a]) || !std::isfinite(p->eta[a]) || !finite_pos(p->L[a]))
            return fail(nullptr, XF_E_ARG, "spectrum parameters of species %d invalid", a);
    if (!std::isfinite(p->eps_perturb) || p->eps_perturb < 0) return fail(nullptr, XF_E_ARG, "eps must be finite and >= 0");
    if (p->matter == XF_MATTER_POWER &&
        (!std::isfinite(p->ne_ref_cm3) || p->ne_ref_cm3 < 0 || !finite_pos(p->r_ref_km) || !std::isfinite(p->ne_power)))
        return fail(nullptr, XF_E_ARG, "power-law matter parameters invalid");
    if (p->matter == XF_MATTER_EXP &&
        (!std::isfinite(p->nb0_cm3) || p->nb0_cm3 < 0 || !finite_pos(p->h_ns_km) || !std::isfinite(p->Ye)))
        return fail(nullptr, XF_E_ARG, "exponential matter parameters invalid");
    return XF_OK;
}

// Host tables: energy grid, number-flux weights phi_a(E) (Eq. 4.1-4.2),
// traceless vacuum Hamiltonian per energy bin (Eq. 3.5-3.6; 3 flavors in the
// mass basis with the standard mixing matrix, delta_CP = 0).
void build_tables(xf_ctx *c)
{
    const xf_params &p = c->p;
    const double dE = (p.E_max_MeV - p.E_min_MeV) / c->n_E;
    c->E.resize(c->n_E);
    for (int e = 0; e < c->n_E; ++e) c->E[e] = p.E_min_MeV + (e + 0.5) * dE;
    c->phi.assign(4 * (size_t)c->n_E, 0.0);
    double flux_ref = 0.0;
    for (int a = 0; a < 4; ++a) {
        const double F2 = fermi_dirac(2, p.eta[a]), F3 = fermi_dirac(3, p.eta[a]);
        const double T = p.T_MeV[a];
        const double flux = p.L[a] / (T * F3 / F2); // L / <E>
        if (a == 0) flux_ref = flux;
        for (int e = 0; e < c->n_E; ++e) {
            const double E = c->E[e];
            const double f = E * E / (F2 * T * T * T * (std::exp(E / T - p.eta[a]) + 1.0));
            c->phi[(size_t)a * c->n_E + e] = flux / flux_ref * f;
        }
    }
    const double K = vac_coefficient();
    c->hvac.assign((size_t)c->n_E * c->S, 0.0);
    for (int e = 0; e < c->n_E; ++e) {
        double *h = &c->hvac[(size_t)e * c->S];
        if (c->nf == 2) {
            const double Delta = K * p.hierarchy * p.dm2_eV2[0] / c->E[e];
            h[0] = -0.5 * Delta * std::cos(2.0 * p.theta[0]);
            h[1] = 0.5 * Delta * std::sin(2.0 * p.theta[0]);
            h[2] = 0.0;
        } else {
            const double s12 = std::sin(p.theta[0]), c12 = std::cos(p.theta[0]);
            const double s13 = std::sin(p.theta[1]), c13 = std::cos(p.theta[1]);
            const double s23 = std::sin(p.theta[2]), c23 = std::cos(p.theta[2]);
            const double U[3][3] = {{c12 * c13, s12 * c13, s13},
                                    {-s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13},
                                    {s12 * s23 - c12 * c23 * s13, -c12 * s23 - s12 * c23 * s13, c23 * c13}};
            const double m2[3] = {0.0, p.dm2_eV2[0], p.hierarchy * p.dm2_eV2[1]};
            double H[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += U[i][k] * m2[k] * U[j][k];
                    H[i][j] = K / c->E[e] * s;
                }
            const double tau = (H[0][0] + H[1][1] + H[2][2]) / 3.0;
            h[0] = H[0][0] - tau;
            h[1] = H[1][1] - tau;
            h[2] = H[0][1];
            h[3] = 0.0;
            h[4] = H[0][2];
            h[5] = 0.0;
            h[6] = H[1][2];
            h[7] = 0.0;
        }
    }
}

LayoutArgs layout_args(xf_ctx *c)
{
    LayoutArgs a;
    a.n_E = c->n_E;
    a.n_u = c->n_u;
    a.n_pairs = c->n_pairs;
    a.npad = c->npad;
    a.phi = c->phi_d;
    a.eps = c->p.eps_perturb;
    a.seed = c->p.seed;
    a.bad = c->bad;
    return a;
}

int elementwise_grid(xf_ctx *c)
{
    long long nb = c->n_bins;
    long long g = (nb + 255) / 256;
    return (int)std::min<long long>(g, (long long)c->num_sms * 16);
}

// Choose the persistent launch shape: CTAs co-resident (cooperative launch),
// contiguous pair chunks per CTA, angle-table span for the dynamic smem.
int plan_launch(xf_ctx *c)
{
    const int nt = c->kern.nt;
    auto span_for = [&](int chunk) {
        // a chunk of `chunk` consecutive pairs touches at most this many angles
        return std::min(c->n_u, (chunk + c->n_E - 1) / c->n_E + 1);
    };
    int occ = 0;
    int G = 1;
    for (int iter = 0; iter < 4; ++iter) {
        int chunk = (c->n_pairs + G - 1) / G;
        int span = span_for(chunk);
        size_t smem = 5 * sizeof(double) * (size_t)std::max(span, 1);
        if (smem > 48 * 1024) {
            if (cudaFuncSetAttribute(c->kern.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, XF_E_UNSUPPORTED, "angle table needs %zu bytes of shared memory", smem);
            }
        }
        XF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->kern.fn, nt, smem), "occupancy");
        if (occ < 1) return fail(c, XF_E_UNSUPPORTED, "kernel cannot be resident (smem %zu)", smem);
        int gmax = occ * c->num_sms;
        int want = (c->n_pairs + nt - 1) / nt;
        if (c->n_pairs <= 8 * nt) want = 1; // small problems: one CTA, no grid barrier
        if (c->grid_request > 0) want = std::min(c->grid_request, c->n_pairs);
        int newG = std::max(1, std::min(gmax, want));
        c->G = newG;
        c->pairs_per_cta = (c->n_pairs + newG - 1) / newG;
        c->span_max = span_for(c->pairs_per_cta);
        c->smem = 5 * sizeof(double) * (size_t)std::max(c->span_max, 1);
        if (newG == G && iter > 0) break;
        G = newG;
    }
    // recheck residency with the final smem
    XF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->kern.fn, nt, c->smem), "occupancy");
    if (occ * c->num_sms < c->G) return fail(c, XF_E_UNSUPPORTED, "grid of %d CTAs not co-resident", c->G);
    return XF_OK;
}

double radius_of(double r_base, long long k, double h) { return h != 0.0 ? r_base + (double)k * h : r_base; }

void reset_position(xf_ctx *c, double r_km)
{
    c->cur = c->pred_cur = 0;
    c->r = r_km;
    c->steps_total = 0;
    c->r_base = c->pred_r_base = r_km;
    c->h_base = c->pred_h = 0.0;
    c->k_base = c->pred_k_base = 0;
    c->pending.clear();
}

int sync_status(xf_ctx *c)
{
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    int err = 0;
    unsigned long long done = 0;
    XF_CUDA(c, cudaMemcpy(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    XF_CUDA(c, cudaMemcpy(&done, c->steps, sizeof(done), cudaMemcpyDeviceToHost), "read step count");
    // walk the enqueued launches with the number of steps actually taken
    long long left = (long long)done;
    for (const Pending &q : c->pending) {
        long long n = std::min(left, q.n);
        c->r_base = q.r0;
        c->h_base = q.h;
        c->k_base = q.k0 + n;
        left -= n;
        if (n < q.n) break;
    }
    c->pending.clear();
    c->steps_total += (long long)done;
    c->cur = (c->cur + (int)(done & 1ull)) & 1;
    c->r = radius_of(c->r_base, c->k_base, c->h_base);
    c->pred_cur = c->cur;
    c->pred_r_base = c->r_base;
    c->pred_h = c->h_base;
    c->pred_k_base = c->k_base;
    XF_CUDA(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "reset error word");
    XF_CUDA(c, cudaMemsetAsync(c->steps, 0, sizeof(unsigned long long), c->stream), "reset step count");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    if (err & ERR_BARRIER) return fail(c, XF_E_BARRIER_TIMEOUT, "grid barrier timed out; state undefined");
    if (err & ERR_NONFINITE)
        return fail(c, XF_E_NONFINITE, "non-finite moments; state kept at step %lld", c->steps_total);
    return XF_OK;
}

int launch_steps(xf_ctx *c, long long n, double dr)
{
    const long long kChunk = 1ll << 16;
    if (dr != c->pred_h) { // new step size: restart the step count at the current radius
        c->pred_r_base = radius_of(c->pred_r_base, c->pred_k_base, c->pred_h);
        c->pred_k_base = 0;
        c->pred_h = dr;
    }
    while (n > 0) {
        long long m = std::min(n, kChunk);
        RunArgs a;
        std::memset(&a, 0, sizeof a);
        a.n_E = c->n_E;
        a.n_u = c->n_u;
        a.n_pairs = c->n_pairs;
        a.npad = c->npad;
        a.geometry = c->p.geometry;
        a.matter = c->p.matter;
        a.pairs_per_cta = c->pairs_per_cta;
        a.span_max = c->span_max;
        a.R = c->p.R_nu_km;
        a.mu0 = c->p.mu0_per_km;
        a.du = 1.0 / c->n_u;
        a.dE = (c->p.E_max_MeV - c->p.E_min_MeV) / c->n_E;
        a.ne_ref = c->p.ne_ref_cm3;
        a.r_ref = c->p.r_ref_km;
        a.ne_power = c->p.ne_power;
        a.nb0 = c->p.nb0_cm3;
        a.h_ns = c->p.h_ns_km;
        a.Ye = c->p.Ye;
        a.gf = matter_coefficient();
        a.r0 = c->pred_r_base;
        a.h = dr;
        a.k0 = c->pred_k_base;
        a.n_steps = m;
        a.cur = c->pred_cur;
        a.hvac = c->hvac_d;
        a.rho0 = c->rho[0];
        a.rho1 = c->rho[1];
        a.aux = c->aux;
        a.partials = c->partials;
        a.mom_out = c->mom_out;
        a.bar = c->bar;
        a.err = c->err;
        a.steps_done = c->steps;
        a.timeout_ns = c->timeout_ns;
        a.skip_cta = c->skip_cta;
        XF_CUDA(c, cudaMemsetAsync(c->bar, 0, sizeof(unsigned), c->stream), "reset barrier");
        void *args[] = {&a};
        cudaError_t e;
        if (c->G > 1)
            e = cudaLaunchCooperativeKernel(c->kern.fn, dim3(c->G), dim3(c->kern.nt), args, c->smem, c->stream);
        else
            e = cudaLaunchKernel(c->kern.fn, dim3(1), dim3(c->kern.nt), args, c->smem, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "launch of the integrator kernel");
        c->pending.push_back({c->pred_r_base, dr, c->pred_k_base, m});
        c->pred_k_base += m;
        c->pred_cur = (c->pred_cur + (int)(m & 1)) & 1;
        n -= m;
    }
    return XF_OK;
}

template <typename F>
int dispatch_layout(xf_ctx *c, F &&f)
{
    if (c->nf == 2) {
        if (c->real_bytes == 8) return f(std::integral_constant<int, 2>(), (double *)nullptr);
        return f(std::integral_constant<int, 2>(), (float *)nullptr);
    }
    if (c->real_bytes == 8) return f(std::integral_constant<int, 3>(), (double *)nullptr);
    return f(std::integral_constant<int, 3>(), (float *)nullptr);
}

} // namespace

// ============================================================== C ABI
extern "C" {

void xf_params_default(xf_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->size = sizeof(xf_params);
    p->version = XF_PARAMS_VERSION;
    p->stepper = XF_RK4;
    p->precision = XF_FP64;
    p->geometry = XF_GEOM_BULB;
    p->hierarchy = -1;
    p->matter = XF_MATTER_NONE;
    p->R_nu_km = 10.0;
    p->mu0_per_km = 1.0e5;
    p->E_min_MeV = 1.0;
    p->E_max_MeV = 60.0;
    p->dm2_eV2[0] = 2.4e-3;
    p->theta[0] = 0.1;
    p->r_ref_km = 10.0;
    p->ne_power = 3.0;
    p->h_ns_km = 1.0;
    p->Ye = 0.5;
    const double T[4] = {2.76, 4.01, 6.26, 6.26};
    for (int a = 0; a < 4; ++a) {
        p->T_MeV[a] = T[a];
        p->eta[a] = 3.0;
        p->L[a] = 1.0;
    }
    p->eps_perturb = 1e-6;
    p->seed = 1;
}

int xf_create(int n_E, int n_u, int n_flavor, const xf_params *p, xf_ctx **out)
{
    return xf_create_ex(n_E, n_u, n_flavor, p, nullptr, out);
}

int xf_create_ex(int n_E, int n_u, int n_flavor, const xf_params *p, const xf_allocator *alloc, xf_ctx **out)
{
    g_create_error.clear();
    if (!out) return fail(nullptr, XF_E_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate(p, n_E, n_u, n_flavor);
    if (rc) return rc;
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, XF_E_ARG, "allocator callbacks missing");

    xf_ctx *c = new (std::nothrow) xf_ctx();
    if (!c) return fail(nullptr, XF_E_NOMEM, "host allocation failed");
    c->n_E = n_E;
    c->n_u = n_u;
    c->nf = n_flavor;
    c->S = n_flavor * n_flavor - 1;
    c->n_pairs = n_E * n_u;
    c->npad = (c->n_pairs + 63) & ~63;
    c->n_bins = 2ll * c->n_pairs;
    c->p = *p;
    c->real_bytes = (p->precision == XF_FP64) ? 8 : 4;
    if (alloc) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    auto bail = [&](int code) {
        free_all(c);
        g_create_error = c->last_error;
        delete c;
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "no usable CUDA device"));

    build_tables(c);
    const int st = (p->stepper == XF_RK4) ? STEP_RK4 : STEP_EXPH;
    c->kern = (c->real_bytes == 8) ? run_kernel_fp64(c->nf, st) : run_kernel_fp32(c->nf, st);
    if (!c->kern.fn) return bail(fail(c, XF_E_UNSUPPORTED, "kernel variant not built"));
    rc = plan_launch(c);
    if (rc) return bail(rc);

    const size_t plane = (size_t)2 * c->S * c->npad * c->real_bytes;
    const int NV = 2 * c->S;
    c->mom_chunk = std::max(256, (c->n_pairs + c->num_sms * 4 - 1) / (c->num_sms * 4));
    c->mom_G = (c->n_pairs + c->mom_chunk - 1) / c->mom_chunk;
    c->rho[0] = dev_alloc(c, plane);
    c->rho[1] = dev_alloc(c, plane);
    c->aux = dev_alloc(c, plane);
    c->trace = (double *)dev_alloc(c, sizeof(double) * 2 * (size_t)c->npad);
    c->hvac_d = dev_alloc(c, (size_t)c->n_E * c->S * c->real_bytes);
    c->phi_d = (double *)dev_alloc(c, sizeof(double) * 4 * (size_t)c->n_E);
    c->staging = (double *)dev_alloc(c, sizeof(double) * (size_t)c->n_bins * c->nf * c->nf);
    int occ_max = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_max, c->kern.fn, c->kern.nt, 0) != cudaSuccess) {
        cudaGetLastError();
        occ_max = 32;
    }
    c->partials = (double *)dev_alloc(c, sizeof(double) * 2 * (size_t)std::max(c->G, occ_max * c->num_sms) * NV);
    c->mom_out = (double *)dev_alloc(c, sizeof(double) * NV);
    c->mom_part = (double *)dev_alloc(c, sizeof(double) * (size_t)c->mom_G * (NV + 2));
    c->mom_full = (double *)dev_alloc(c, sizeof(double) * 2 * c->nf * c->nf);
    c->bar = (unsigned *)dev_alloc(c, 64);
    c->err = (int *)dev_alloc(c, 64);
    c->bad = (int *)dev_alloc(c, 64);
    c->steps = (unsigned long long *)dev_alloc(c, 64);
    for (void *q : {c->rho[0], c->rho[1], c->aux, (void *)c->trace, c->hvac_d, (void *)c->phi_d,
                    (void *)c->staging, (void *)c->partials, (void *)c->mom_out, (void *)c->mom_part,
                    (void *)c->mom_full, (void *)c->bar, (void *)c->err, (void *)c->bad, (void *)c->steps})
        if (!q) return bail(fail(c, XF_E_NOMEM, "device allocation failed"));

    // tables to the device (Real copy of H_vac)
    if (c->real_bytes == 8) {
        e = cudaMemcpy(c->hvac_d, c->hvac.data(), sizeof(double) * c->hvac.size(), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> hf(c->hvac.begin(), c->hvac.end());
        e = cudaMemcpy(c->hvac_d, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(c->phi_d, c->phi.data(), sizeof(double) * c->phi.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, 64);
    if (e == cudaSuccess) e = cudaMemset(c->steps, 0, 64);
    if (e == cudaSuccess) e = cudaMemset(c->bar, 0, 64);
    if (e == cudaSuccess) e = cudaMemset(c->rho[0], 0, plane);
    if (e == cudaSuccess) e = cudaMemset(c->rho[1], 0, plane);
    if (e == cudaSuccess) e = cudaMemset(c->aux, 0, plane);
    if (e == cudaSuccess) e = cudaMemset(c->trace, 0, sizeof(double) * 2 * (size_t)c->npad);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "device set-up"));
    *out = c;
    return XF_OK;
}

int xf_destroy(xf_ctx *c)
{
    if (!c) return XF_OK;
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    free_all(c);
    delete c;
    return XF_OK;
}

int xf_set_stream(xf_ctx *c, void *stream)
{
    if (!c) return XF_E_ARG;
    if (!c->pending.empty()) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    c->stream = (cudaStream_t)stream;
    return XF_OK;
}

int xf_set_state(xf_ctx *c, const double *rho, size_t n_doubles, double r_km)
{
    if (!c) return XF_E_ARG;
    if (!rho) return fail(c, XF_E_ARG, "rho is NULL");
    if (n_doubles != (size_t)c->n_bins * c->nf * c->nf)
        return fail(c, XF_E_ARG, "n_doubles %zu != %lld", n_doubles, c->n_bins * c->nf * c->nf);
    if (!std::isfinite(r_km) || r_km < c->p.R_nu_km) return fail(c, XF_E_ARG, "r_km must be finite and >= R_nu");
    if (!c->pending.empty()) sync_status(c);
    XF_CUDA(c, cudaMemcpyAsync(c->staging, rho, sizeof(double) * n_doubles, cudaMemcpyHostToDevice, c->stream),
            "copy state to device");
    XF_CUDA(c, cudaMemsetAsync(c->bad, 0, sizeof(int), c->stream), "reset flag");
    LayoutArgs la = layout_args(c);
    const int grid = elementwise_grid(c);
    int rc = dispatch_layout(c, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        pack_to_state_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, c->staging, (Real *)c->rho[0], c->trace);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "layout kernel");
    int bad = 0;
    XF_CUDA(c, cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    reset_position(c, r_km);
    c->state_valid = !bad;
    if (bad) return fail(c, XF_E_STATE, "state contains non-finite values");
    return XF_OK;
}

int xf_init_state(xf_ctx *c, double r_km)
{
    if (!c) return XF_E_ARG;
    if (!std::isfinite(r_km) || r_km < c->p.R_nu_km) return fail(c, XF_E_ARG, "r_km must be finite and >= R_nu");
    if (!c->pending.empty()) sync_status(c);
    LayoutArgs la = layout_args(c);
    const int grid = elementwise_grid(c);
    int rc = dispatch_layout(c, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        init_state_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (Real *)c->rho[0], c->trace);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "init kernel");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    reset_position(c, r_km);
    c->state_valid = true;
    return XF_OK;
}

int xf_step_async(xf_ctx *c, int64_t n_steps, double dr_km)
{
    if (!c) return XF_E_ARG;
    if (n_steps < 0) return fail(c, XF_E_ARG, "n_steps must be >= 0");
    if (!std::isfinite(dr_km) || dr_km <= 0) return fail(c, XF_E_ARG, "dr_km must be finite and > 0");
    if (!c->state_valid) return fail(c, XF_E_STATE, "no valid state (call xf_set_state or xf_init_state)");
    if (n_steps == 0) return XF_OK;
    return launch_steps(c, n_steps, dr_km);
}

int xf_sync(xf_ctx *c)
{
    if (!c) return XF_E_ARG;
    int rc = sync_status(c);
    if (rc == XF_E_BARRIER_TIMEOUT) c->state_valid = false;
    return rc;
}

int xf_step(xf_ctx *c, int64_t n_steps, double dr_km)
{
    int rc = xf_step_async(c, n_steps, dr_km);
    if (rc) return rc;
    return xf_sync(c);
}

int xf_get_state(xf_ctx *c, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    if (!c) return XF_E_ARG;
    if (!rho) return fail(c, XF_E_ARG, "rho is NULL");
    if (n_doubles != (size_t)c->n_bins * c->nf * c->nf)
        return fail(c, XF_E_ARG, "n_doubles %zu != %lld", n_doubles, c->n_bins * c->nf * c->nf);
    if (!c->pending.empty()) sync_status(c);
    if (!c->state_valid) return fail(c, XF_E_STATE, "no valid state");
    LayoutArgs la = layout_args(c);
    const int grid = elementwise_grid(c);
    int rc = dispatch_layout(c, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        state_to_pack_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (const Real *)c->rho[c->cur], c->trace,
                                                                    c->staging);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "layout kernel");
    XF_CUDA(c, cudaMemcpyAsync(rho, c->staging, sizeof(double) * n_doubles, cudaMemcpyDeviceToHost, c->stream),
            "copy state to host");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    if (r_km) *r_km = c->r;
    if (steps_done) *steps_done = c->steps_total;
    return XF_OK;
}

int xf_moments(xf_ctx *c, double *M0, double *M1, size_t n_doubles)
{
    if (!c) return XF_E_ARG;
    if (!M0 || !M1) return fail(c, XF_E_ARG, "M0/M1 NULL");
    if (n_doubles != (size_t)c->nf * c->nf) return fail(c, XF_E_ARG, "n_doubles must be n_f*n_f");
    if (!c->pending.empty()) sync_status(c);
    if (!c->state_valid) return fail(c, XF_E_STATE, "no valid state");
    MomArgs m;
    m.n_E = c->n_E;
    m.n_u = c->n_u;
    m.n_pairs = c->n_pairs;
    m.npad = c->npad;
    m.geometry = c->p.geometry;
    m.chunk = c->mom_chunk;
    m.R = c->p.R_nu_km;
    m.du = 1.0 / c->n_u;
    m.dE = (c->p.E_max_MeV - c->p.E_min_MeV) / c->n_E;
    m.r = c->r;
    const double dE = m.dE;
    int rc = dispatch_layout(c, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        moments_partial_kernel<NF, Real, 256><<<c->mom_G, 256, 0, c->stream>>>(m, (const Real *)c->rho[c->cur],
                                                                             c->trace, c->mom_part);
        moments_final_kernel<NF><<<1, 32, 0, c->stream>>>(c->mom_part, c->mom_G, dE, c->mom_full,
                                                        c->mom_full + NF * NF);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "moments kernel");
    double host[18];
    XF_CUDA(c, cudaMemcpyAsync(host, c->mom_full, sizeof(double) * 2 * n_doubles, cudaMemcpyDeviceToHost, c->stream),
            "copy moments");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    std::memcpy(M0, host, sizeof(double) * n_doubles);
    std::memcpy(M1, host + n_doubles, sizeof(double) * n_doubles);
    return XF_OK;
}

int xf_outputs(xf_ctx *c, double *p_surv, double *trace, double *purity, size_t n_bins)
{
    if (!c) return XF_E_ARG;
    if (n_bins != (size_t)c->n_bins) return fail(c, XF_E_ARG, "n_bins %zu != %lld", n_bins, c->n_bins);
    if (!c->pending.empty()) sync_status(c);
    if (!c->state_valid) return fail(c, XF_E_STATE, "no valid state");
    double *outs[3] = {p_surv, trace, purity};
    double *dev[3] = {nullptr, nullptr, nullptr};
    // staging holds n_bins * n_f^2 >= 4 n_bins doubles: room for three outputs
    for (int i = 0; i < 3; ++i)
        if (outs[i]) dev[i] = c->staging + (size_t)i * c->n_bins;
    LayoutArgs la = layout_args(c);
    const int grid = elementwise_grid(c);
    int rc = dispatch_layout(c, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        outputs_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (const Real *)c->rho[c->cur], c->trace, dev[0],
                                                              dev[1], dev[2]);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "outputs kernel");
    for (int i = 0; i < 3; ++i)
        if (outs[i])
            XF_CUDA(c, cudaMemcpyAsync(outs[i], dev[i], sizeof(double) * n_bins, cudaMemcpyDeviceToHost, c->stream),
                    "copy outputs");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    return XF_OK;
}

int xf_set_option(xf_ctx *c, int option, int64_t value)
{
    if (!c) return XF_E_ARG;
    if (!c->pending.empty()) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    switch (option) {
    case XF_OPT_GRID: {
        if (value < 0 || value > INT_MAX) return fail(c, XF_E_ARG, "grid must be >= 0");
        int old = c->grid_request;
        c->grid_request = (int)value;
        int rc = plan_launch(c);
        if (rc) {
            c->grid_request = old;
            plan_launch(c);
        }
        return rc;
    }
    case XF_OPT_BARRIER_TIMEOUT_NS:
        if (value <= 0) return fail(c, XF_E_ARG, "timeout must be > 0");
        c->timeout_ns = (unsigned long long)value;
        return XF_OK;
    case XF_OPT_TEST_SKIP_ARRIVAL:
        if (value < -1 || value > INT_MAX) return fail(c, XF_E_ARG, "bad CTA index");
        c->skip_cta = (int)value;
        return XF_OK;
    default: return fail(c, XF_E_ARG, "unknown option %d", option);
    }
}

int xf_tables(xf_ctx *c, double *E, double *phi)
{
    if (!c) return XF_E_ARG;
    if (E) std::memcpy(E, c->E.data(), sizeof(double) * c->E.size());
    if (phi) std::memcpy(phi, c->phi.data(), sizeof(double) * c->phi.size());
    return XF_OK;
}

int xf_launch_info(xf_ctx *c, int *ctas, int *threads, int *barriers_per_step)
{
    if (!c) return XF_E_ARG;
    if (ctas) *ctas = c->G;
    if (threads) *threads = c->kern.nt;
    if (barriers_per_step) *barriers_per_step = (c->p.stepper == XF_RK4) ? 4 : 2;
    return XF_OK;
}

const char *xf_status_str(int s)
{
    switch (s) {
    case XF_OK: return "XF_OK";
    case XF_PENDING: return "XF_PENDING";
    case XF_E_ARG: return "XF_E_ARG";
    case XF_E_STATE: return "XF_E_STATE";
    case XF_E_NOMEM: return "XF_E_NOMEM";
    case XF_E_CUDA: return "XF_E_CUDA";
    case XF_E_NONFINITE: return "XF_E_NONFINITE";
    case XF_E_BARRIER_TIMEOUT: return "XF_E_BARRIER_TIMEOUT";
    case XF_E_UNSTABLE: return "XF_E_UNSTABLE";
    case XF_E_BUSY: return "XF_E_BUSY";
    case XF_E_TOO_BIG: return "XF_E_TOO_BIG";
    case XF_E_NOTFOUND: return "XF_E_NOTFOUND";
    case XF_E_TIMEOUT: return "XF_E_TIMEOUT";
    case XF_E_UNSUPPORTED: return "XF_E_UNSUPPORTED";
    default: return "XF_E_UNKNOWN";
    }
}

const char *xf_last_error(const xf_ctx *c)
{
    if (!c) return g_create_error.c_str();
    return c->last_error.c_str();
}

} // extern "C"
