// xf_api.cu -- host side of the C ABI declared in include/xf.h: argument
// validation, per-energy tables (FP64, on the host), device memory, layout
// conversion, tiling of one or many problems onto the persistent grid, and
// the launches of the integrator (optionally replayed from a CUDA graph).
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
#include "xf_adapt.cuh"
#include "xf_aux.cuh"
#include "xf_kernels.h"
#include "xf_cyl.cuh"
#include "xf_pack.h"

using namespace xf;

namespace xfp {

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

} // namespace xfp


namespace xfp {

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
    cudaGetLastError(); // clear the non-sticky error state
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

void dev_free(xf_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->owned.begin(), c->owned.end(), p);
    if (it == c->owned.end()) return;
    c->owned.erase(it);
    if (c->has_alloc) c->alloc.free(p, c->alloc.user);
    else cudaFree(p);
}

void free_all(xf_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    c->gstream = nullptr;
    c->ev_in = c->ev_out = nullptr;
    if (c->ck_stream) {
        cudaStreamSynchronize(c->ck_stream);
        cudaStreamDestroy(c->ck_stream);
    }
    if (c->ck_event) cudaEventDestroy(c->ck_event);
    c->ck_stream = nullptr;
    c->ck_event = nullptr;
    c->ck_buf = nullptr;
    c->ck_bytes = 0;
    c->ck_pending = false;
    for (void *p : c->owned) {
        if (c->has_alloc) c->alloc.free(p, c->alloc.user);
        else cudaFree(p);
    }
    c->owned.clear();
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int validate(xf_ctx *c, const xf_params *p, int n_E, int n_u, int nf)
{
    if (!p) return fail(c, XF_E_ARG, "params is NULL");
    if (p->size != sizeof(xf_params)) return fail(c, XF_E_ARG, "params.size %u != %zu", p->size, sizeof(xf_params));
    if (p->version != XF_PARAMS_VERSION) return fail(c, XF_E_ARG, "params.version %u unsupported", p->version);
    if (n_E <= 0 || n_u <= 0) return fail(c, XF_E_ARG, "n_E and n_u must be positive (got %d, %d)", n_E, n_u);
    if (nf != 2 && nf != 3) return fail(c, XF_E_ARG, "n_flavor must be 2 or 3 (got %d)", nf);
    if ((long long)n_E * n_u > (long long)(INT_MAX / 16)) return fail(c, XF_E_ARG, "n_E * n_u too large");
    if (p->stepper != XF_RK4 && p->stepper != XF_EXPH && p->stepper != XF_EXPH_ADAPTIVE)
        return fail(c, XF_E_ARG, "bad stepper %d", p->stepper);
    if (p->stepper == XF_EXPH_ADAPTIVE) {
        if (p->precision != XF_FP64 && p->precision != XF_FP32_M64)
            return fail(c, XF_E_UNSUPPORTED, "the error-controlled step runs in FP64 or FP32_M64 only");
        if (!(p->eps0 > 0) || !std::isfinite(p->eps0)) return fail(c, XF_E_ARG, "eps0 must be finite and > 0");
        if (!(p->ksi > 0) || !(p->ksi <= 1)) return fail(c, XF_E_ARG, "ksi must be in (0, 1]");
        if (!(p->dr_max_km > 0) || !std::isfinite(p->dr_max_km)) return fail(c, XF_E_ARG, "dr_max must be finite and > 0");
    }
    if (p->precision < XF_FP64 || p->precision > XF_FP32X2)
        return fail(c, XF_E_ARG, "bad precision %d", p->precision);
    if (p->precision == XF_FP32X2 && p->stepper != XF_EXPH)
        return fail(c, XF_E_UNSUPPORTED, "XF_FP32X2 runs the predictor-corrector (XF_EXPH) only");
    if (p->geometry < XF_GEOM_BULB || p->geometry > XF_GEOM_CYLINDER)
        return fail(c, XF_E_ARG, "bad geometry %d", p->geometry);
    if (p->geometry == XF_GEOM_CYLINDER) {
        if (p->stepper == XF_EXPH_ADAPTIVE || (p->precision != XF_FP64 && p->precision != XF_FP32_M64) ||
            p->form != XF_FORM_RHO || p->strict)
            return fail(c, XF_E_UNSUPPORTED,
                        "the cylinder model runs fixed steps in FP64 or FP32_M64, density matrices, not strict");
        if (n_u > xf::CYL_MAX_U) return fail(c, XF_E_UNSUPPORTED, "the cylinder model takes n_u <= %d", xf::CYL_MAX_U);
    }
    if (p->geometry == XF_GEOM_SINGLE_ANGLE && n_u != 1) return fail(c, XF_E_ARG, "single-angle geometry needs n_u == 1");
    if (p->n_phi < 1) return fail(c, XF_E_ARG, "n_phi must be >= 1");
    if ((long long)n_E * n_u * p->n_phi > (long long)(INT_MAX / 16)) return fail(c, XF_E_ARG, "n_E * n_u * n_phi too large");
    if (p->n_phi > 1) {
        if (p->geometry != XF_GEOM_BULB && p->geometry != XF_GEOM_CYLINDER)
            return fail(c, XF_E_ARG, "azimuth (latitude) bins extend the bulb (cylinder) geometry only");
        if (p->stepper == XF_EXPH_ADAPTIVE || (p->precision != XF_FP64 && p->precision != XF_FP32_M64))
            return fail(c, XF_E_UNSUPPORTED, "azimuth bins run with fixed steps in FP64 or FP32_M64");
    }
    if (p->form != XF_FORM_RHO && p->form != XF_FORM_PSI) return fail(c, XF_E_ARG, "bad form %d", p->form);
    if (p->form == XF_FORM_PSI &&
        (p->stepper == XF_EXPH_ADAPTIVE || (p->precision != XF_FP64 && p->precision != XF_FP32_M64) || p->n_phi != 1))
        return fail(c, XF_E_UNSUPPORTED, "the wavefunction form runs fixed steps in FP64 or FP32_M64, one azimuth bin");
    if (p->hierarchy != 1 && p->hierarchy != -1) return fail(c, XF_E_ARG, "hierarchy must be +1 or -1");
    if (p->matter < XF_MATTER_NONE || p->matter > XF_MATTER_EXP) return fail(c, XF_E_ARG, "bad matter %d", p->matter);
    if (!finite_pos(p->R_nu_km)) return fail(c, XF_E_ARG, "R_nu_km must be finite and > 0");
    if (!std::isfinite(p->mu0_per_km) || p->mu0_per_km < 0) return fail(c, XF_E_ARG, "mu0 must be finite and >= 0");
    if (!std::isfinite(p->E_min_MeV) || p->E_min_MeV < 0 || !std::isfinite(p->E_max_MeV) || p->E_max_MeV <= p->E_min_MeV)
        return fail(c, XF_E_ARG, "need 0 <= E_min < E_max, finite");
    for (int i = 0; i < 2; ++i)
        if (!std::isfinite(p->dm2_eV2[i])) return fail(c, XF_E_ARG, "dm2 not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(p->theta[i])) return fail(c, XF_E_ARG, "theta not finite");
    for (int a = 0; a < 4; ++a)
        if (!finite_pos(p->T_MeV[a]) || !std::isfinite(p->eta[a]) || !finite_pos(p->L[a]))
            return fail(c, XF_E_ARG, "spectrum parameters of species %d invalid", a);
    if (!std::isfinite(p->eps_perturb) || p->eps_perturb < 0) return fail(c, XF_E_ARG, "eps must be finite and >= 0");
    if (p->matter == XF_MATTER_POWER &&
        (!std::isfinite(p->ne_ref_cm3) || p->ne_ref_cm3 < 0 || !finite_pos(p->r_ref_km) || !std::isfinite(p->ne_power)))
        return fail(c, XF_E_ARG, "power-law matter parameters invalid");
    if (p->matter == XF_MATTER_EXP &&
        (!std::isfinite(p->nb0_cm3) || p->nb0_cm3 < 0 || !finite_pos(p->h_ns_km) || !std::isfinite(p->Ye)))
        return fail(c, XF_E_ARG, "exponential matter parameters invalid");
    return XF_OK;
}

// Host tables: energy grid, number-flux weights phi_a(E) (Eq. 4.1-4.2),
// traceless vacuum Hamiltonian per energy bin (Eq. 3.5-3.6; 3 flavors in the
// mass basis with the standard mixing matrix, delta_CP = 0).
void build_tables(InstHost &c)
{
    const xf_params &p = c.p;
    const double dE = (p.E_max_MeV - p.E_min_MeV) / c.n_E;
    c.E.resize(c.n_E);
    for (int e = 0; e < c.n_E; ++e) c.E[e] = p.E_min_MeV + (e + 0.5) * dE;
    c.phi.assign(4 * (size_t)c.n_E, 0.0);
    double flux_ref = 0.0;
    for (int a = 0; a < 4; ++a) {
        const double F2 = fermi_dirac(2, p.eta[a]), F3 = fermi_dirac(3, p.eta[a]);
        const double T = p.T_MeV[a];
        const double flux = p.L[a] / (T * F3 / F2); // L / <E>
        if (a == 0) flux_ref = flux;
        for (int e = 0; e < c.n_E; ++e) {
            const double E = c.E[e];
            const double f = E * E / (F2 * T * T * T * (std::exp(E / T - p.eta[a]) + 1.0));
            c.phi[(size_t)a * c.n_E + e] = flux / flux_ref * f;
        }
    }
    const double K = vac_coefficient();
    c.hvac.assign((size_t)c.n_E * c.S, 0.0);
    for (int e = 0; e < c.n_E; ++e) {
        double *h = &c.hvac[(size_t)e * c.S];
        if (c.nf == 2) {
            const double Delta = K * p.hierarchy * p.dm2_eV2[0] / c.E[e];
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
                    H[i][j] = K / c.E[e] * s;
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

LayoutArgs layout_args(xf_ctx *c, const InstHost &in)
{
    LayoutArgs a;
    a.n_E = in.n_E;
    a.n_u = in.n_u * in.n_phi; // trajectories
    a.n_pairs = in.n_pairs;
    a.npad = in.npad;
    a.phi = (const double *)c->arena + in.phi_off;
    a.eps = in.p.eps_perturb;
    a.seed = in.p.seed;
    a.bad = c->bad;
    return a;
}

int elementwise_grid(xf_ctx *c, const InstHost &in)
{
    long long g = (in.n_bins + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, (long long)c->num_sms * 16));
}

// Cost weight of a three-flavor pair against a two-flavor one (relative work
// per step).  FP64 bins are bound by the FP64 ALUs: the per-bin operation
// counts give 2097 / 122 ~ 17 for the predictor-corrector (a 3x3
// eigendecomposition against a Bloch rotation; the error-controlled attempt
// alike), the 256-problem ensemble ran fastest at 12 (4.45e8 bin-steps/s
// against 4.25e8 at 17 and 3.9e8 at 24), a two-flavor pair carrying some
// fixed per-pair work; 684 / 172 ~ 4 for RK4.  FP32 bins run at 64x the ALU
// rate and a pair costs about its state bytes (8 against 3 components): 3
// measured best on the ensemble (1.33e10 bin-steps/s against 1.0e10 at 1 or
// 5 and 6.0e9 at 10).  xf_autotune also tries 0.7 and 1.4 times the value
// on packs of mixed flavors.
double default_cost3(int stepper, int precision)
{
    const bool fp64 = precision == XF_FP64 || precision == XF_FP32X2;
    if (stepper == XF_RK4) return fp64 ? 4.0 : 3.0;
    return fp64 ? 12.0 : 3.0;
}
double pair_cost(const xf_ctx *c, const InstHost &in) { return in.nf == 3 ? c->cost3 : 1.0; }

// Tile every instance into runs of at most TP pairs, then give
// each CTA a contiguous run of tiles of about equal cost.
int plan_launch_cyl(xf_ctx *c);

int plan_launch(xf_ctx *c)
{
    if (c->cyl) return plan_launch_cyl(c);
    const int nt = c->kern.nt;
    int occ_free = 0;
    XF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_free, c->kern.fn, nt, 0), "occupancy");
    if (occ_free < 1) return fail(c, XF_E_UNSUPPORTED, "integrator kernel cannot be resident");
    long long total_pairs = 0;
    double total_cost = 0.0;
    int n_active = 0;
    for (const InstHost &in : c->in) {
        if (!in.active) continue;
        total_pairs += in.n_pairs;
        total_cost += pair_cost(c, in) * in.n_pairs;
        ++n_active;
    }
    // tile size: one problem -> one tile per co-resident CTA slot (every CTA
    // gets the same work); several problems -> about 8 tiles per slot, so that
    // runs of unequal tiles balance.  A multiple of 32 (whole warps).
    const long long slots = (long long)occ_free * c->num_sms;
    long long tp = c->tile_request;
    if (tp <= 0) {
        const long long per = (n_active <= 1) ? slots : 8 * slots;
        tp = (total_pairs + per - 1) / per;
    }
    tp = std::min<long long>(std::max<long long>((tp + 31) / 32 * 32, 32), 1 << 20);
    const int TP = (int)tp;
    // problems in descending order of the cost of a pair (three-flavor ones
    // first, stable otherwise): CTAs working at the same time then mostly
    // run one flavor's code, which keeps the instruction cache warm on packs
    // of mixed flavors, and dynamic claiming hands out the dearer tiles
    // first.  Each problem's tiles stay contiguous and in order, so its
    // moment sums do not change.
    std::vector<int> order(c->in.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return pair_cost(c, c->in[x]) > pair_cost(c, c->in[y]);
    });
    c->tiles.clear();
    for (const int i : order) {
        InstHost &in = c->in[i];
        in.tile_begin = (int)c->tiles.size();
        if (in.active)
            for (int p0 = 0; p0 < in.n_pairs; p0 += TP)
                c->tiles.push_back({i, p0, std::min(TP, in.n_pairs - p0), 0});
        in.tile_end = (int)c->tiles.size();
    }
    const int T = (int)c->tiles.size();
    c->dirty = false;
    if (T == 0) { // nothing to run
        c->G = 0;
        c->tile_pairs = TP;
        c->cta_tiles.assign(1, 0);
        return XF_OK;
    }
    int span = 1;
    for (const Tile &t : c->tiles) {
        const InstHost &in = c->in[t.inst];
        span = std::max(span, (t.p0 + t.np - 1) / in.n_E - t.p0 / in.n_E + 1);
    }
    // per-angle tables: 5 FP64 slots, or 6 FP32 slots (step length as hi + lo);
    // the error-controlled step: 8 FP64 or 10 FP32 slots
    const bool ad = c->stepper == XF_EXPH_ADAPTIVE;
    const size_t per_angle = ad ? (c->real_bytes == 8 ? xf::ASlots<double>::n * sizeof(double)
                                                      : xf::ASlots<float>::n * sizeof(float))
                                : (size_t)((c->real_bytes == 8 ? 5 : 6) + (c->nmom == 4 ? 4 : 0)) * c->real_bytes;
    int stage_off = 0;
    size_t smem = ad ? ((per_angle * (size_t)span + 15) & ~size_t(15))
                     : xf::run_smem(per_angle * (size_t)span, c->real_bytes, c->stepper == XF_EXPH, c->nmom, c->form,
                                    c->nfm, nt, &stage_off);
    if (!allow_dynamic_smem(c->kern.fn, smem)) { // static plus dynamic shared memory may pass 48 KB
        cudaGetLastError();
        return fail(c, XF_E_UNSUPPORTED, "angle table needs %zu bytes of shared memory", smem);
    }
    int occ = 0;
    XF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->kern.fn, nt, smem), "occupancy");
    if (occ < 1) return fail(c, XF_E_UNSUPPORTED, "kernel cannot be resident (smem %zu)", smem);
    int G = std::min(T, occ * c->num_sms);
    if (c->grid_request > 0) G = std::min(G, c->grid_request);
    G = std::max(G, 1);
    // contiguous runs of tiles with about total_cost / G each, at least one
    // tile per CTA
    std::vector<int> ct(G + 1, T);
    ct[0] = 0;
    double acc = 0.0;
    int cta = 1;
    for (int t = 0; t < T && cta < G; ++t) {
        const InstHost &in = c->in[c->tiles[t].inst];
        acc += pair_cost(c, in) * c->tiles[t].np;
        const bool must_cut = (T - (t + 1)) == (G - cta); // one tile left per remaining CTA
        if ((acc >= total_cost * cta / G || must_cut) && T - (t + 1) >= G - cta) ct[cta++] = t + 1;
    }
    for (; cta < G; ++cta) ct[cta] = std::max(ct[cta - 1] + 1, T - (G - cta));
    c->G = G;
    c->tile_pairs = TP;
    c->span_max = span;
    c->smem = smem;
    c->stage_off = stage_off;
    c->cta_tiles = ct;
    // device copies (the tile buffers are sized for the most tiles seen)
    if (T > c->max_tiles) {
        c->partials = (double *)dev_alloc(c, ad ? sizeof(double) * 4 * (size_t)T * xf::APS
                                                : sizeof(double) * 2 * (size_t)T * NVMAX);
        if (ad) {
            c->tstate_d = (AdaptPos *)dev_alloc(c, sizeof(AdaptPos) * (size_t)T);
            if (!c->tstate_d) return fail(c, XF_E_NOMEM, "device allocation of the tile tables failed");
        }
        c->tiles_d = (Tile *)dev_alloc(c, sizeof(Tile) * (size_t)T);
        c->cta_tiles_d = (int *)dev_alloc(c, sizeof(int) * (size_t)(T + 1));
        if (!c->partials || !c->tiles_d || !c->cta_tiles_d)
            return fail(c, XF_E_NOMEM, "device allocation of the tile tables failed");
        c->max_tiles = T;
    }
    XF_CUDA(c, cudaMemcpy(c->tiles_d, c->tiles.data(), sizeof(Tile) * T, cudaMemcpyHostToDevice), "copy tiles");
    XF_CUDA(c, cudaMemcpy(c->cta_tiles_d, ct.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice), "copy tiling");
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return XF_OK;
}

// Cylinder model: one problem; CTA c owns tile c, a run of whole trajectories
// (about T / G each), and tables of 8 doubles and 2 ints per angle bin; the
// partials buffer holds two slots of per-trajectory sums (8 doubles each).
int plan_launch_cyl(xf_ctx *c)
{
    InstHost &in = c->in[0];
    c->tiles.clear();
    c->dirty = false;
    if (!in.active) {
        c->G = 0;
        c->cta_tiles.assign(1, 0);
        return XF_OK;
    }
    const int T = in.n_u * in.n_phi, nw = c->kern.nt / 32;
    const size_t smem = (size_t)(4 + 2 * xf::CYL_ROWS) * in.n_u * sizeof(double) + (size_t)xf::CYL_ROWS * in.n_u * sizeof(int);
    if (!allow_dynamic_smem(c->kern.fn, smem)) { // static plus dynamic shared memory may pass 48 KB
        cudaGetLastError();
        return fail(c, XF_E_UNSUPPORTED, "angle table needs %zu bytes of shared memory", smem);
    }
    int occ = 0;
    XF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->kern.fn, c->kern.nt, smem), "occupancy");
    if (occ < 1) return fail(c, XF_E_UNSUPPORTED, "kernel cannot be resident (smem %zu)", smem);
    int G = std::min((T + nw - 1) / nw, occ * c->num_sms);
    if (c->grid_request > 0) G = std::min(G, c->grid_request);
    G = std::max(G, 1);
    for (int g = 0; g < G; ++g) {
        const int ta = (int)((long long)T * g / G), tb = (int)((long long)T * (g + 1) / G);
        c->tiles.push_back({0, ta * in.n_E, (tb - ta) * in.n_E, 0});
    }
    in.tile_begin = 0;
    in.tile_end = G;
    std::vector<int> ct(G + 1);
    for (int g = 0; g <= G; ++g) ct[g] = g;
    c->G = G;
    c->tile_pairs = 0;
    c->span_max = in.n_u;
    c->smem = smem;
    c->cta_tiles = ct;
    const size_t need = std::max((size_t)2 * G * NVMAX, (size_t)2 * T * xf::CYL_DS);
    if (G > c->max_tiles || need > c->partials_doubles) {
        if (c->partials) dev_free(c, c->partials);
        c->partials = (double *)dev_alloc(c, sizeof(double) * need);
        c->partials_doubles = c->partials ? need : 0;
        c->tiles_d = (Tile *)dev_alloc(c, sizeof(Tile) * (size_t)G);
        c->cta_tiles_d = (int *)dev_alloc(c, sizeof(int) * (size_t)(G + 1));
        if (!c->partials || !c->tiles_d || !c->cta_tiles_d)
            return fail(c, XF_E_NOMEM, "device allocation of the tile tables failed");
        c->max_tiles = G;
    }
    XF_CUDA(c, cudaMemcpy(c->tiles_d, c->tiles.data(), sizeof(Tile) * G, cudaMemcpyHostToDevice), "copy tiles");
    XF_CUDA(c, cudaMemcpy(c->cta_tiles_d, ct.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice), "copy tiling");
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return XF_OK;
}

// The device descriptor of one problem (static fields and the current r0, h).
Inst make_inst(const InstHost &h)
{
    const double gf = matter_coefficient();
    Inst d;
    std::memset(&d, 0, sizeof d);
    d.n_E = h.n_E;
    d.n_u = h.n_u;
    d.nf = h.nf;
    d.geometry = h.p.geometry;
    d.matter = h.p.matter;
    d.n_pairs = h.n_pairs;
    d.npad = h.npad;
    d.n_phi = h.n_phi;
    d.hvac_off = h.hvac_off;
    d.ref_off = h.ref_off;
    d.trace_off = h.trace_off;
    d.phi_off = h.phi_off;
    d.form = h.p.form;
    for (int b = 0; b < 3; ++b) d.off[b] = h.off[b];
    d.R = h.p.R_nu_km;
    d.mu0 = h.p.mu0_per_km;
    d.du = 1.0 / h.n_u;
    d.dE = (h.p.E_max_MeV - h.p.E_min_MeV) / h.n_E;
    d.ne_ref = h.p.ne_ref_cm3;
    d.r_ref = h.p.r_ref_km;
    d.ne_power = h.p.ne_power;
    d.nb0 = h.p.nb0_cm3;
    d.h_ns = h.p.h_ns_km;
    d.Ye = h.p.Ye;
    d.gf = gf;
    d.r0 = h.r0;
    d.h = h.h;
    d.eps0 = h.p.eps0;
    d.ksi = h.p.ksi;
    d.dr_max = h.p.dr_max_km;
    d.tile_begin = h.tile_begin;
    d.tile_end = h.tile_end;
    return d;
}

// Device copy of the instance table.
int upload_instances(xf_ctx *c)
{
    std::vector<Inst> v(c->in.size());
    for (size_t i = 0; i < c->in.size(); ++i) v[i] = make_inst(c->in[i]);
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    XF_CUDA(c, cudaMemcpy(c->inst_d, v.data(), sizeof(Inst) * v.size(), cudaMemcpyHostToDevice), "copy instances");
    return XF_OK;
}

__global__ void set_requests_kernel(InstPos *pos, int n, long long steps, int only)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (only < 0 || i == only) && pos[i].err == 0) pos[i].remaining = steps;
}
// Restart instance i's step count at k0 (keeping its step total when `keep`).
__global__ void reset_pos_kernel(InstPos *pos, int i, int cur, int keep)
{
    pos[i].k0 = 0;
    pos[i].remaining = 0;
    if (!keep) {
        pos[i].steps = 0;
        pos[i].cur = cur;
        pos[i].err = 0;
    }
}

__global__ void set_apos_kernel(AdaptPos *apos, int i, AdaptPos v) { apos[i] = v; }
__global__ void set_pos_kernel(InstPos *pos, int i, InstPos v) { pos[i] = v; }

// Read the device progress of every instance into the host view.
int sync_status(xf_ctx *c)
{
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    std::vector<InstPos> ps(c->in.size());
    int err = 0;
    XF_CUDA(c, cudaMemcpy(ps.data(), c->pos_d, sizeof(InstPos) * ps.size(), cudaMemcpyDeviceToHost), "read progress");
    XF_CUDA(c, cudaMemcpy(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (c->stepper == XF_EXPH_ADAPTIVE) {
        std::vector<AdaptPos> ap(c->in.size());
        XF_CUDA(c, cudaMemcpy(ap.data(), c->apos_d, sizeof(AdaptPos) * ap.size(), cudaMemcpyDeviceToHost),
                "read progress");
        for (size_t i = 0; i < c->in.size(); ++i) {
            InstHost &h = c->in[i];
            h.cur = ap[i].cur;
            h.r_ad = ap[i].r;
            h.h_ad = ap[i].h;
            h.err_ad = ap[i].err;
            h.n_acc = ap[i].n_acc;
            h.n_rej = ap[i].n_rej;
            h.ad_status = ap[i].status;
            h.steps = ap[i].n_acc;
        }
    } else {
        for (size_t i = 0; i < c->in.size(); ++i) {
            InstHost &h = c->in[i];
            h.k0 = ps[i].k0;
            h.cur = ps[i].cur;
            h.steps = (long long)ps[i].steps;
            h.err = ps[i].err;
        }
    }
    c->pending = 0;
    if (err == ERR_LAUNCH) { // the kernel left before touching anything
        XF_CUDA(c, cudaMemset(c->err, 0, sizeof(int)), "reset error word");
        return fail(c, XF_E_CUDA, "integrator launched without its shared-memory staging area");
    }
    if (err) {
        XF_CUDA(c, cudaMemset(c->err, 0, sizeof(int)), "reset error word");
        for (InstHost &h : c->in) h.state_valid = false;
        return fail(c, XF_E_BARRIER_TIMEOUT, "grid barrier timed out; state undefined");
    }
    return XF_OK;
}

double radius(const InstHost &h)
{
    if (h.adaptive) return h.r_ad;
    return h.h != 0.0 ? h.r0 + (double)h.k0 * h.h : h.r0;
}

// Enqueue one integrator launch of n steps (every instance with remaining > 0).
int enqueue_run(xf_ctx *c, long long n, cudaStream_t stream)
{
    RunArgs a;
    std::memset(&a, 0, sizeof a);
    a.inst = c->inst_d;
    a.tiles = c->tiles_d;
    a.cta_tiles = c->cta_tiles_d;
    a.n_inst = (int)c->in.size();
    a.n_tiles = (int)c->tiles.size();
    a.span_max = c->span_max;
    a.n_steps = n;
    a.arena = c->arena;
    a.partials = c->partials;
    a.mom_out = c->mom_out;
    a.pos = c->pos_d;
    a.bar = c->bar;
    a.err = c->err;
    a.timeout_ns = c->timeout_ns;
    a.skip_cta = c->skip_cta;
    a.apos = c->apos_d;
    a.tstate = c->tstate_d;
    a.first_bad = c->bar + 1;
    a.ticket = (unsigned long long *)(c->bar + 2);
    a.dynamic = (!c->cyl && c->stepper != XF_EXPH_ADAPTIVE && c->dynamic_tiles && (int)c->tiles.size() > c->G) ? 1 : 0;
    a.stage_off = c->stage_off;
    if (c->G == 0) return XF_OK;
    XF_CUDA(c, cudaMemsetAsync(c->bar, 0, sizeof(unsigned), stream), "reset barrier");
    if (a.dynamic) XF_CUDA(c, cudaMemsetAsync(c->bar + 2, 0, sizeof(unsigned long long), stream), "reset tickets");
    if (c->cyl) XF_CUDA(c, cudaMemsetAsync(c->bar + 1, 0xff, sizeof(unsigned), stream), "reset flag");
    void *args[] = {&a};
    cudaError_t e;
    if (c->G > 1)
        e = cudaLaunchCooperativeKernel(c->kern.fn, dim3(c->G), dim3(c->kern.nt), args, c->smem, stream);
    else
        e = cudaLaunchKernel(c->kern.fn, dim3(1), dim3(c->kern.nt), args, c->smem, stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "launch of the integrator kernel");
    return XF_OK;
}

// Enqueue n steps for instance `only` (or all with only < 0): request, launch.
// With the graph option the (request, reset, launch) sequence of a given n is
// captured once and replayed.
int enqueue_steps(xf_ctx *c, long long n, int only)
{
    const long long kChunk = 1ll << 16;
    const int ni = (int)c->in.size();
    while (n > 0) {
        const long long m = std::min(n, kChunk);
        if (c->use_graph && only < 0) {
            if (!c->gstream) {
                XF_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking), "graph stream");
                XF_CUDA(c, cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming), "graph event");
                XF_CUDA(c, cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming), "graph event");
            }
            if (!c->graph || c->graph_steps != m) {
                if (c->graph) cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
                cudaGraph_t g = nullptr;
                XF_CUDA(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal), "begin capture");
                set_requests_kernel<<<(ni + 127) / 128, 128, 0, c->gstream>>>(c->pos_d, ni, m, -1);
                int rc = enqueue_run(c, m, c->gstream);
                cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
                if (rc) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
                e = cudaGraphInstantiate(&c->graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
                c->graph_steps = m;
            }
            XF_CUDA(c, cudaEventRecord(c->ev_in, c->stream), "order graph after stream");
            XF_CUDA(c, cudaStreamWaitEvent(c->gstream, c->ev_in, 0), "order graph after stream");
            XF_CUDA(c, cudaGraphLaunch(c->graph, c->gstream), "graph launch");
            XF_CUDA(c, cudaEventRecord(c->ev_out, c->gstream), "order stream after graph");
            XF_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_out, 0), "order stream after graph");
        } else {
            set_requests_kernel<<<(ni + 127) / 128, 128, 0, c->stream>>>(c->pos_d, ni, m, only);
            XF_CUDA(c, cudaGetLastError(), "request kernel");
            int rc = enqueue_run(c, m, c->stream);
            if (rc) return rc;
        }
        ++c->pending;
        n -= m;
    }
    return XF_OK;
}

__global__ void set_request_array_kernel(InstPos *pos, int n, const long long *req)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pos[i].err == 0) pos[i].remaining = req[i];
}

// One launch of up to n steps in which problem i takes req[i] <= n steps
// (0: idle); re-tiles first if problems were added or removed.
int enqueue_requests(xf_ctx *c, long long n, const std::vector<long long> &req)
{
    if (c->dirty) {
        int rc = plan_launch(c);
        if (!rc) rc = upload_instances(c);
        if (rc) return rc;
    }
    const int ni = (int)c->in.size();
    if ((int)req.size() != ni || n <= 0) return fail(c, XF_E_ARG, "request vector size mismatch");
    XF_CUDA(c, cudaMemcpy(c->staging, req.data(), sizeof(long long) * ni, cudaMemcpyHostToDevice), "copy requests");
    set_request_array_kernel<<<(ni + 127) / 128, 128, 0, c->stream>>>(c->pos_d, ni, (const long long *)c->staging);
    XF_CUDA(c, cudaGetLastError(), "request kernel");
    int rc = enqueue_run(c, n, c->stream);
    if (rc) return rc;
    ++c->pending;
    return XF_OK;
}

int adapt_code(int status)
{
    switch (status) {
    case xf::AD_DONE: return XF_OK;
    case xf::AD_BUDGET: return XF_E_BUDGET;
    case xf::AD_NONFINITE: return XF_E_NONFINITE;
    case xf::AD_STEPSIZE: return XF_E_STEPSIZE;
    default: return XF_E_STATE;
    }
}

// Error-controlled integration of every active problem (or only `only`) to
// its r_end: set the device progress records, then launch chunks of
// attempts until no problem is running.  Each chunk is sized from the
// largest number of steps left at the current step sizes.
int evolve_impl(xf_ctx *c, const double *r_end, long long max_iters, const double *dr0, int only)
{
    if (c->stepper != XF_EXPH_ADAPTIVE) return fail(c, XF_E_ARG, "xf_evolve needs the XF_EXPH_ADAPTIVE stepper");
    if (max_iters < 0) return fail(c, XF_E_ARG, "max_iters must be >= 0");
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    if (c->dirty) {
        int rc = plan_launch(c);
        if (!rc) rc = upload_instances(c);
        if (rc) return rc;
    }
    const int ni = (int)c->in.size();
    std::vector<AdaptPos> ap(ni);
    for (int i = 0; i < ni; ++i) {
        InstHost &h = c->in[i];
        AdaptPos &a = ap[i];
        std::memset(&a, 0, sizeof a);
        a.r = a.r_end = h.r_ad;
        a.h = h.h_ad;
        a.cur = h.cur;
        a.err = h.err_ad;
        a.n_acc = h.n_acc;
        a.n_rej = h.n_rej;
        a.status = h.ad_status == xf::AD_RUN ? xf::AD_DONE : h.ad_status;
        if (!h.active || (only >= 0 && i != only)) continue;
        if (!h.state_valid) return fail(c, XF_E_STATE, "problem %d has no valid state", i);
        const double re = r_end[only >= 0 ? 0 : i];
        if (!std::isfinite(re) || re < h.r_ad) return fail(c, XF_E_ARG, "r_end of problem %d is behind its radius", i);
        const double d0 = dr0 ? dr0[only >= 0 ? 0 : i] : 0.0;
        if (!std::isfinite(d0)) return fail(c, XF_E_ARG, "dr0 of problem %d not finite", i);
        double h0 = d0 > 0 ? d0 : (h.h_ad > 0 ? h.h_ad : h.p.dr_max_km);
        h0 = h0 < h.p.dr_max_km ? h0 : h.p.dr_max_km;
        a.h = h0;
        a.r_end = re;
        a.iters_left = max_iters;
        a.n_acc = a.n_rej = 0;
        a.err = 0.0;
        if (!(re - a.r > 1e-12 * re)) {
            a.status = xf::AD_DONE;
            a.r = re;
        } else if (max_iters == 0) {
            a.status = xf::AD_BUDGET;
        } else if (h0 < 1e-12 * a.r) {
            a.status = xf::AD_STEPSIZE;
        } else {
            a.status = xf::AD_RUN;
        }
    }
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    XF_CUDA(c, cudaMemcpy(c->apos_d, ap.data(), sizeof(AdaptPos) * ni, cudaMemcpyHostToDevice), "copy progress");
    for (int i = 0; i < ni; ++i) c->in[i].ad_status = ap[i].status;
    long long left = max_iters;
    for (;;) {
        long long want = 0;
        for (int i = 0; i < ni; ++i) {
            const InstHost &h = c->in[i];
            if (h.ad_status != xf::AD_RUN) continue;
            const double hh = h.h_ad > 0 ? h.h_ad : ap[i].h;
            const double est = std::ceil((ap[i].r_end - h.r_ad) / hh) + 1.0;
            want = std::max(want, (long long)std::min(est, 4096.0));
        }
        if (want == 0) break;
        const long long K = std::max(1ll, std::min(want, left));
        int rc = enqueue_run(c, K, c->stream);
        if (rc) return rc;
        ++c->pending;
        rc = sync_status(c);
        if (rc) return rc;
        left -= K;
        if (left <= 0) break; // every running problem has spent its budget (the kernel set AD_BUDGET)
    }
    for (int i = 0; i < ni; ++i) {
        if (!c->in[i].active || (only >= 0 && i != only)) continue;
        const int code = adapt_code(c->in[i].ad_status);
        if (code) return fail(c, code, "problem %d: error-controlled run stopped at r = %.9g km (%s)", i,
                              c->in[i].r_ad, xf_status_str(code));
    }
    return XF_OK;
}

InstHost *instance(xf_ctx *c, int i)
{
    if (!c || i < 0 || i >= (int)c->in.size()) return nullptr;
    return &c->in[i];
}

// Set instance i's step size: a new h restarts the step count at the current
// radius (the caller uploads the instance table afterwards).
int set_step_size(xf_ctx *c, int i, double dr)
{
    InstHost &h = c->in[i];
    if (dr == h.h) return XF_OK;
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    h.r0 = radius(h);
    h.k0 = 0;
    h.h = dr;
    reset_pos_kernel<<<1, 1, 0, c->stream>>>(c->pos_d, i, h.cur, 1);
    XF_CUDA(c, cudaGetLastError(), "position kernel");
    return XF_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of a problem's block: three state buffers (S or, in the psi form,
// 2 n_f^2 planes each), trace, vacuum table,
// weights, and for the renormalising variant the initial tr(T^2) per bin.
long long block_bytes(int n_E, int n_u, int nf, int precision, int form)
{
    const long long rb = (precision == XF_FP64 || precision == XF_FP32X2) ? 8 : 4;
    const long long S = nf * nf - 1, n_pairs = (long long)n_E * n_u, npad = (n_pairs + 63) & ~63ll;
    const long long SS = form == XF_FORM_PSI ? 2 * nf * nf : S;
    const long long ref = precision == XF_FP32_M64_RENORM ? (long long)align256(2 * npad * rb) : 0;
    return 3 * (long long)align256(2 * SS * npad * rb) + (long long)align256(2 * npad * 8) +
           (long long)align256((size_t)n_E * S * rb) + (long long)align256((size_t)4 * n_E * 8) + ref;
}

// Fill slot i with a problem: tables on the host, a block of the arena, the
// tables copied into it, state buffers zeroed.  The slot becomes active; the
// launch is re-tiled before the next step.
int setup_problem(xf_ctx *c, int i, const xf_problem &prob)
{
    InstHost &h = c->in[i];
    h = InstHost();
    h.n_E = prob.n_E;
    h.n_u = prob.n_u;
    h.n_phi = prob.params.n_phi;
    h.nf = prob.n_flavor;
    h.S = h.nf * h.nf - 1;
    h.SS = prob.params.form == XF_FORM_PSI ? 2 * h.nf * h.nf : h.S;
    h.n_pairs = h.n_E * h.n_u * h.n_phi;
    h.npad = (h.n_pairs + 63) & ~63;
    h.n_bins = 2ll * h.n_pairs;
    h.p = prob.params;
    h.adaptive = c->stepper == XF_EXPH_ADAPTIVE;
    const int rb = c->real_bytes;
    h.block_bytes = block_bytes(h.n_E, h.n_u * h.n_phi, h.nf, c->precision, prob.params.form);
    h.block = c->blocks.alloc(h.block_bytes);
    if (h.block < 0) return fail(c, XF_E_NOMEM, "no room for the problem in the arena");
    const long long plane = (long long)align256((size_t)2 * h.SS * h.npad * rb);
    const long long tr = (long long)align256((size_t)2 * h.npad * 8);
    const long long hv = (long long)align256((size_t)h.n_E * h.S * rb);
    for (int b = 0; b < 3; ++b) h.off[b] = (h.block + b * plane) / rb;
    h.trace_off = (h.block + 3 * plane) / 8;
    h.hvac_off = (h.block + 3 * plane + tr) / rb;
    h.phi_off = (h.block + 3 * plane + tr + hv) / 8;
    h.ref_off = c->precision == XF_FP32_M64_RENORM
                    ? (h.block + 3 * plane + tr + hv + (long long)align256((size_t)4 * h.n_E * 8)) / rb
                    : 0;
    build_tables(h);
    const size_t need = (size_t)h.n_bins * h.nf * h.nf * (h.SS > h.S ? 2 : 1); // a packed state
    if (need > c->staging_doubles) {
        double *st = (double *)dev_alloc(c, sizeof(double) * std::max(need, (size_t)c->in.size()));
        if (!st) return fail(c, XF_E_NOMEM, "device allocation of the staging buffer failed");
        c->staging = st;
        c->staging_doubles = std::max(need, (size_t)c->in.size());
    }
    cudaError_t e;
    if (rb == 8) {
        e = cudaMemcpy((double *)c->arena + h.hvac_off, h.hvac.data(), sizeof(double) * h.hvac.size(),
                       cudaMemcpyHostToDevice);
    } else {
        std::vector<float> hf(h.hvac.begin(), h.hvac.end());
        e = cudaMemcpy((float *)c->arena + h.hvac_off, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy((double *)c->arena + h.phi_off, h.phi.data(), sizeof(double) * h.phi.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->arena + h.block, 0, 3 * plane + tr, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "problem set-up");
    h.active = true;
    c->dirty = true;
    return XF_OK;
}

// A ctx with its control buffers and an arena of arena_bytes, no problem yet.
int create_ctx(int n_slots, long long arena_bytes, int stepper, int precision, int nfm, const xf_allocator *alloc,
               xf_ctx **out, int nmom = 2, int form = XF_FORM_RHO, bool cyl = false)
{
    xf_ctx *c = new (std::nothrow) xf_ctx();
    if (!c) return fail(nullptr, XF_E_NOMEM, "host allocation failed");
    if (alloc) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    c->real_bytes = (precision == XF_FP64 || precision == XF_FP32X2) ? 8 : 4;
    c->precision = precision;
    c->stepper = stepper;
    c->cost3 = default_cost3(stepper, precision);
    c->nfm = nfm;
    auto bail = [&](int code) {
        free_all(c);
        g_create_error = c->last_error;
        delete c;
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "no usable CUDA device"));
    const int st = (stepper == XF_RK4) ? STEP_RK4 : STEP_EXPH;
    c->nmom = nmom;
    c->form = form;
    c->cyl = cyl;
    if (cyl)
        c->kern = run_kernel_cyl(nfm, st, c->real_bytes == 8);
    else if (form == XF_FORM_PSI)
        c->kern = run_kernel_psi(nfm, st, c->real_bytes == 8);
    else if (stepper == XF_EXPH_ADAPTIVE)
        c->kern = run_kernel_adapt(nfm, c->real_bytes == 8);
    else if (nmom == 4)
        c->kern = run_kernel_azimuth(nfm, st, c->real_bytes == 8);
    else
        c->kern = precision == XF_FP32X2 ? run_kernel_ff(nfm, st)
                  : (c->real_bytes == 8) ? run_kernel_fp64(nfm, st)
                  : precision == XF_FP32_COMP ? run_kernel_fp32(nfm, st, VAR_COMP)
                  : precision == XF_FP32_M64_RENORM ? run_kernel_fp32(nfm, st, VAR_RENORM)
                                                     : run_kernel_fp32(nfm, st, VAR_PLAIN);
    if (!c->kern.fn) return bail(fail(c, XF_E_UNSUPPORTED, "kernel variant not built"));
    c->in.resize(n_slots);
    c->arena = (unsigned char *)dev_alloc(c, (size_t)std::max(arena_bytes, 256ll));
    c->blocks.reset(arena_bytes);
    c->staging_doubles = (size_t)n_slots;
    c->staging = (double *)dev_alloc(c, sizeof(double) * c->staging_doubles);
    c->inst_d = (Inst *)dev_alloc(c, sizeof(Inst) * n_slots);
    c->pos_d = (InstPos *)dev_alloc(c, sizeof(InstPos) * n_slots);
    if (stepper == XF_EXPH_ADAPTIVE) {
        c->apos_d = (AdaptPos *)dev_alloc(c, sizeof(AdaptPos) * n_slots);
        if (!c->apos_d) return bail(fail(c, XF_E_NOMEM, "device allocation failed"));
    }
    c->mom_out = (double *)dev_alloc(c, sizeof(double) * NVMAX * n_slots);
    c->mom_full = (double *)dev_alloc(c, sizeof(double) * 36);
    c->bar = (unsigned *)dev_alloc(c, 64);
    c->err = (int *)dev_alloc(c, 64);
    c->bad = (int *)dev_alloc(c, 64);
    for (void *q : {(void *)c->arena, (void *)c->staging, (void *)c->inst_d, (void *)c->pos_d, (void *)c->mom_out,
                    (void *)c->mom_full, (void *)c->bar, (void *)c->err, (void *)c->bad})
        if (!q) return bail(fail(c, XF_E_NOMEM, "device allocation failed"));
    e = cudaMemset(c->err, 0, 64);
    if (e == cudaSuccess) e = cudaMemset(c->bar, 0, 64);
    if (e == cudaSuccess) e = cudaMemset(c->pos_d, 0, sizeof(InstPos) * n_slots);
    if (e == cudaSuccess) e = cudaMemset(c->inst_d, 0, sizeof(Inst) * n_slots);
    if (e == cudaSuccess && c->apos_d) e = cudaMemset(c->apos_d, 0, sizeof(AdaptPos) * n_slots);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "device set-up"));
    *out = c;
    return XF_OK;
}

void destroy_pack(xf_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    free_all(c);
    delete c;
}

int create_pack(int n, const xf_problem *probs, const xf_allocator *alloc, xf_ctx **out)
{
    g_create_error.clear();
    if (!out) return fail(nullptr, XF_E_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !probs) return fail(nullptr, XF_E_ARG, "need at least one problem");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, XF_E_ARG, "allocator callbacks missing");
    bool has2 = false, has3 = false, has_phi = false, has_cyl = false;
    for (int i = 0; i < n; ++i) {
        has_phi = has_phi || probs[i].params.n_phi > 1;
        has_cyl = has_cyl || probs[i].params.geometry == XF_GEOM_CYLINDER;
        int rc = validate(nullptr, &probs[i].params, probs[i].n_E, probs[i].n_u, probs[i].n_flavor);
        if (rc) {
            if (n > 1) g_create_error = "problem " + std::to_string(i) + ": " + g_create_error;
            return rc;
        }
        if (probs[i].params.stepper != probs[0].params.stepper || probs[i].params.precision != probs[0].params.precision ||
            probs[i].params.form != probs[0].params.form)
            return fail(nullptr, XF_E_ARG, "all problems of a pack need the same stepper, precision and form");
        (probs[i].n_flavor == 2 ? has2 : has3) = true;
    }
    if (has_cyl && n > 1) return fail(nullptr, XF_E_UNSUPPORTED, "a cylinder-model problem runs alone in its context");
    long long bytes = 0;
    for (int i = 0; i < n; ++i)
        bytes += block_bytes(probs[i].n_E, probs[i].n_u * probs[i].params.n_phi, probs[i].n_flavor,
                             probs[0].params.precision, probs[0].params.form);
    xf_ctx *c = nullptr;
    int rc = create_ctx(n, bytes, probs[0].params.stepper, probs[0].params.precision,
                        (has2 && has3) ? 0 : (has3 ? 3 : 2), alloc, &c, has_phi ? 4 : 2, probs[0].params.form,
                        has_cyl);
    if (rc) return rc;
    for (int i = 0; i < n && !rc; ++i) rc = setup_problem(c, i, probs[i]);
    if (!rc) rc = plan_launch(c);
    if (!rc) rc = upload_instances(c);
    if (!rc) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(c, e, "device set-up");
    }
    if (rc) {
        g_create_error = c->last_error;
        destroy_pack(c);
        return rc;
    }
    *out = c;
    return XF_OK;
}

// A pack of n_slots empty slots sharing an arena of arena_bytes (serving).
int create_slots(int n_slots, long long arena_bytes, int stepper, int precision, int nfm, xf_ctx **out)
{
    return create_ctx(n_slots, arena_bytes, stepper, precision, nfm, nullptr, out);
}

int add_problem(xf_ctx *c, const xf_problem &prob, const double *rho, double r_km, double dr_km, int *slot)
{
    int rc = validate(c, &prob.params, prob.n_E, prob.n_u, prob.n_flavor);
    if (rc) return rc;
    if (prob.params.stepper != c->stepper || prob.params.precision != c->precision || prob.params.form != c->form)
        return fail(c, XF_E_ARG, "stepper, precision or form differs from the pack's");
    if (c->nfm && prob.n_flavor != c->nfm) return fail(c, XF_E_ARG, "flavor count differs from the pack's");
    if (prob.params.n_phi > 1 && c->nmom != 4) return fail(c, XF_E_UNSUPPORTED, "azimuth bins need a 4-moment pack");
    if (prob.params.geometry == XF_GEOM_CYLINDER || c->cyl)
        return fail(c, XF_E_UNSUPPORTED, "a cylinder-model problem runs alone in its context");
    if (!std::isfinite(dr_km) || dr_km <= 0) return fail(c, XF_E_ARG, "dr_km must be finite and > 0");
    int i = -1;
    for (int k = 0; k < (int)c->in.size(); ++k)
        if (!c->in[k].active) {
            i = k;
            break;
        }
    if (i < 0) return fail(c, XF_E_BUSY, "no free slot");
    if (c->pending) {
        rc = sync_status(c);
        if (rc) return rc;
    }
    rc = setup_problem(c, i, prob);
    if (rc) {
        c->in[i].active = false;
        return rc == XF_E_NOMEM ? XF_E_BUSY : rc;
    }
    const size_t n = (size_t)c->in[i].n_bins * prob.n_flavor * prob.n_flavor;
    rc = rho ? set_state_impl(c, i, rho, n, r_km) : init_state_impl(c, i, r_km);
    if (rc) {
        remove_problem(c, i);
        return rc;
    }
    c->in[i].h = dr_km; // start the step count at r_km with this step size
    c->dirty = true;
    *slot = i;
    return XF_OK;
}

int remove_problem(xf_ctx *c, int slot)
{
    if (!c || slot < 0 || slot >= (int)c->in.size() || !c->in[slot].active) return XF_E_ARG;
    InstHost &h = c->in[slot];
    c->blocks.release(h.block);
    h.active = false;
    h.state_valid = false;
    h.block = -1;
    c->dirty = true;
    return XF_OK;
}

int check_r(xf_ctx *c, const InstHost &h, double r_km)
{
    if (!std::isfinite(r_km) || r_km < h.p.R_nu_km) return fail(c, XF_E_ARG, "r_km must be finite and >= R_nu");
    return XF_OK;
}

// Instance i now holds a fresh state in buffer 0 at radius r_km.
int reset_instance(xf_ctx *c, int i, double r_km, bool valid)
{
    InstHost &h = c->in[i];
    h.r0 = r_km;
    h.h = 0.0;
    h.k0 = 0;
    h.steps = 0;
    h.cur = 0;
    h.err = 0;
    h.state_valid = valid;
    reset_pos_kernel<<<1, 1, 0, c->stream>>>(c->pos_d, i, 0, 0);
    XF_CUDA(c, cudaGetLastError(), "position kernel");
    if (c->stepper == XF_EXPH_ADAPTIVE) {
        h.adaptive = true;
        h.r_ad = r_km;
        h.h_ad = 0.0;
        h.err_ad = 0.0;
        h.n_acc = h.n_rej = 0;
        h.ad_status = xf::AD_DONE;
        AdaptPos a;
        std::memset(&a, 0, sizeof a);
        a.r = a.r_end = r_km;
        a.status = xf::AD_DONE;
        set_apos_kernel<<<1, 1, 0, c->stream>>>(c->apos_d, i, a);
        XF_CUDA(c, cudaGetLastError(), "position kernel");
    }
    return upload_instances(c);
}

// Where the layout kernels store each bin's initial tr(T^2) (renormalising
// variant), else NULL.
template <typename Real>
Real *ref_ptr(xf_ctx *c, const InstHost &h)
{
    return c->precision == XF_FP32_M64_RENORM ? (Real *)c->arena + h.ref_off : nullptr;
}

int set_state_impl(xf_ctx *c, int i, const double *rho, size_t n_doubles, double r_km)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    if (c->form == XF_FORM_PSI)
        return fail(c, XF_E_UNSUPPORTED, "a wavefunction-form problem takes its state from xf_set_psi");
    if (!rho) return fail(c, XF_E_ARG, "rho is NULL");
    if (n_doubles != (size_t)h.n_bins * h.nf * h.nf)
        return fail(c, XF_E_ARG, "n_doubles %zu != %lld", n_doubles, h.n_bins * h.nf * h.nf);
    int rc = check_r(c, h, r_km);
    if (rc) return rc;
    if (c->pending) sync_status(c);
    XF_CUDA(c, cudaMemcpyAsync(c->staging, rho, sizeof(double) * n_doubles, cudaMemcpyHostToDevice, c->stream),
            "copy state to device");
    XF_CUDA(c, cudaMemsetAsync(c->bad, 0, sizeof(int), c->stream), "reset flag");
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        pack_to_state_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, c->staging, (Real *)c->arena + h.off[0],
                                                                    (double *)c->arena + h.trace_off, ref_ptr<Real>(c, h));
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "layout kernel");
    int bad = 0;
    XF_CUDA(c, cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    rc = reset_instance(c, i, r_km, !bad);
    if (rc) return rc;
    if (bad) return fail(c, XF_E_STATE, "state contains non-finite values");
    return XF_OK;
}

int init_state_impl(xf_ctx *c, int i, double r_km)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    int rc = check_r(c, h, r_km);
    if (rc) return rc;
    if (c->pending) sync_status(c);
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        if (c->form == XF_FORM_PSI)
            psi_init_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (Real *)c->arena + h.off[0]);
        else
            init_state_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (Real *)c->arena + h.off[0],
                                                                     (double *)c->arena + h.trace_off,
                                                                     ref_ptr<Real>(c, h));
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "init kernel");
    return reset_instance(c, i, r_km, true);
}

int get_state_impl(xf_ctx *c, int i, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    if (!rho) return fail(c, XF_E_ARG, "rho is NULL");
    if (n_doubles != (size_t)h.n_bins * h.nf * h.nf)
        return fail(c, XF_E_ARG, "n_doubles %zu != %lld", n_doubles, h.n_bins * h.nf * h.nf);
    if (c->pending) sync_status(c);
    if (!h.state_valid) return fail(c, XF_E_STATE, "no valid state");
    int rc = XF_OK;
    const long long plane = rho_plane(c, h, &rc);
    if (rc) return rc;
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        state_to_pack_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(
            la, (const Real *)c->arena + plane, (const double *)c->arena + h.trace_off, c->staging);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "layout kernel");
    XF_CUDA(c, cudaMemcpyAsync(rho, c->staging, sizeof(double) * n_doubles, cudaMemcpyDeviceToHost, c->stream),
            "copy state to host");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    if (r_km) *r_km = radius(h);
    if (steps_done) *steps_done = h.steps;
    return XF_OK;
}

long long rho_plane(xf_ctx *c, InstHost &h, int *rc)
{
    *rc = XF_OK;
    if (c->form != XF_FORM_PSI) return h.off[h.cur];
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    *rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        psi_to_rho_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (const Real *)c->arena + h.off[h.cur],
                                                                 (Real *)c->arena + h.off[2],
                                                                 (double *)c->arena + h.trace_off);
        return (int)cudaGetLastError();
    });
    if (*rc) *rc = cuda_fail(c, (cudaError_t)*rc, "wavefunction conversion kernel");
    return h.off[2];
}

int set_psi_impl(xf_ctx *c, int i, const double *psi, size_t n_doubles, double r_km)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    if (c->form != XF_FORM_PSI) return fail(c, XF_E_UNSUPPORTED, "not a wavefunction-form problem");
    if (!psi) return fail(c, XF_E_ARG, "psi is NULL");
    if (n_doubles != (size_t)h.n_bins * h.SS)
        return fail(c, XF_E_ARG, "n_doubles %zu != %lld", n_doubles, h.n_bins * h.SS);
    int rc = check_r(c, h, r_km);
    if (rc) return rc;
    if (c->pending) sync_status(c);
    XF_CUDA(c, cudaMemcpyAsync(c->staging, psi, sizeof(double) * n_doubles, cudaMemcpyHostToDevice, c->stream),
            "copy state to device");
    XF_CUDA(c, cudaMemsetAsync(c->bad, 0, sizeof(int), c->stream), "reset flag");
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        psi_pack_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, c->staging, (Real *)c->arena + h.off[0], 1);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "layout kernel");
    int bad = 0;
    XF_CUDA(c, cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    rc = reset_instance(c, i, r_km, !bad);
    if (rc) return rc;
    if (bad) return fail(c, XF_E_STATE, "state contains non-finite values");
    return XF_OK;
}

int get_psi_impl(xf_ctx *c, int i, double *psi, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    if (c->form != XF_FORM_PSI) return fail(c, XF_E_UNSUPPORTED, "not a wavefunction-form problem");
    if (!psi) return fail(c, XF_E_ARG, "psi is NULL");
    if (n_doubles != (size_t)h.n_bins * h.SS)
        return fail(c, XF_E_ARG, "n_doubles %zu != %lld", n_doubles, h.n_bins * h.SS);
    if (c->pending) sync_status(c);
    if (!h.state_valid) return fail(c, XF_E_STATE, "no valid state");
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    int rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        psi_pack_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, c->staging, (Real *)c->arena + h.off[h.cur], 0);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "layout kernel");
    XF_CUDA(c, cudaMemcpyAsync(psi, c->staging, sizeof(double) * n_doubles, cudaMemcpyDeviceToHost, c->stream),
            "copy state to host");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    if (r_km) *r_km = radius(h);
    if (steps_done) *steps_done = h.steps;
    return XF_OK;
}

int outputs_impl(xf_ctx *c, int i, double *p_surv, double *trace, double *purity, size_t n_bins)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    if (n_bins != (size_t)h.n_bins) return fail(c, XF_E_ARG, "n_bins %zu != %lld", n_bins, h.n_bins);
    if (c->pending) sync_status(c);
    if (!h.state_valid) return fail(c, XF_E_STATE, "no valid state");
    double *outs[3] = {p_surv, trace, purity};
    double *dev[3] = {nullptr, nullptr, nullptr};
    // staging holds n_bins * n_f^2 >= 4 n_bins doubles: room for three outputs
    for (int k = 0; k < 3; ++k)
        if (outs[k]) dev[k] = c->staging + (size_t)k * h.n_bins;
    int rc = XF_OK;
    const long long plane = rho_plane(c, h, &rc);
    if (rc) return rc;
    LayoutArgs la = layout_args(c, h);
    const int grid = elementwise_grid(c, h);
    rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        outputs_kernel<NF, Real><<<grid, 256, 0, c->stream>>>(la, (const Real *)c->arena + plane,
                                                              (const double *)c->arena + h.trace_off, dev[0],
                                                              dev[1], dev[2]);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "outputs kernel");
    for (int k = 0; k < 3; ++k)
        if (outs[k])
            XF_CUDA(c, cudaMemcpyAsync(outs[k], dev[k], sizeof(double) * n_bins, cudaMemcpyDeviceToHost, c->stream),
                    "copy outputs");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    return XF_OK;
}

// All four moments M0..M3 of problem i's current state (FP64 sums on the
// device), packed n_f^2 each into M[4 n_f^2]; M2 = M3 = 0 without azimuth bins.
int moments_all(xf_ctx *c, int i, double *M)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    InstHost &h = *hp;
    if (c->pending) sync_status(c);
    if (!h.state_valid) return fail(c, XF_E_STATE, "no valid state");
    MomArgs m;
    std::memset(&m, 0, sizeof m);
    m.n_E = h.n_E;
    m.n_u = h.n_u;
    m.n_phi = h.n_phi;
    m.n_pairs = h.n_pairs;
    m.npad = h.npad;
    m.geometry = h.p.geometry;
    m.chunk = std::max(256, (h.n_pairs + c->num_sms * 4 - 1) / (c->num_sms * 4));
    m.R = h.p.R_nu_km;
    m.du = 1.0 / h.n_u;
    m.dE = (h.p.E_max_MeV - h.p.E_min_MeV) / h.n_E;
    m.r = radius(h);
    const int G = (h.n_pairs + m.chunk - 1) / m.chunk;
    if (G > c->mom_part_slots) {
        c->mom_part = (double *)dev_alloc(c, sizeof(double) * (size_t)G * 36);
        if (!c->mom_part) return fail(c, XF_E_NOMEM, "device allocation failed");
        c->mom_part_slots = G;
    }
    const double dE = m.dE;
    int rc = XF_OK;
    const long long plane = rho_plane(c, h, &rc);
    if (rc) return rc;
    rc = dispatch_layout(c, h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        moments_partial_kernel<NF, Real, 256><<<G, 256, 0, c->stream>>>(
            m, (const Real *)c->arena + plane, (const double *)c->arena + h.trace_off, c->mom_part);
        moments_final_kernel<NF><<<1, 32, 0, c->stream>>>(c->mom_part, G, dE, c->mom_full);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "moments kernel");
    XF_CUDA(c, cudaMemcpyAsync(M, c->mom_full, sizeof(double) * 4 * h.nf * h.nf, cudaMemcpyDeviceToHost, c->stream),
            "copy moments");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    return XF_OK;
}

int moments_impl(xf_ctx *c, int i, double *M0, double *M1, size_t n_doubles)
{
    InstHost *hp = instance(c, i);
    if (!hp) return c ? fail(c, XF_E_ARG, "bad instance index %d", i) : XF_E_ARG;
    if (!M0 || !M1) return fail(c, XF_E_ARG, "M0/M1 NULL");
    if (n_doubles != (size_t)hp->nf * hp->nf) return fail(c, XF_E_ARG, "n_doubles must be n_f*n_f");
    double M[36];
    int rc = moments_all(c, i, M);
    if (rc) return rc;
    std::memcpy(M0, M, sizeof(double) * n_doubles);
    std::memcpy(M1, M + n_doubles, sizeof(double) * n_doubles);
    return XF_OK;
}

} // namespace xfp

using namespace xfp;

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
    p->eps0 = 1e-6;
    p->ksi = 0.9;
    p->dr_max_km = 1.0;
    p->n_phi = 1;
}

int xf_create(int n_E, int n_u, int n_flavor, const xf_params *p, xf_ctx **out)
{
    return xf_create_ex(n_E, n_u, n_flavor, p, nullptr, out);
}

int xf_create_ex(int n_E, int n_u, int n_flavor, const xf_params *p, const xf_allocator *alloc, xf_ctx **out)
{
    if (!out) return fail(nullptr, XF_E_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, XF_E_ARG, "params is NULL");
    xf_problem prob;
    std::memset(&prob, 0, sizeof prob);
    prob.n_E = n_E;
    prob.n_u = n_u;
    prob.n_flavor = n_flavor;
    prob.params = *p;
    return create_pack(1, &prob, alloc, out);
}

int xf_create_batch(int n_problems, const xf_problem *problems, const xf_allocator *alloc, xf_ctx **out)
{
    return create_pack(n_problems, problems, alloc, out);
}

int xf_destroy(xf_ctx *c)
{
    destroy_pack(c);
    return XF_OK;
}

int xf_set_stream(xf_ctx *c, void *stream)
{
    if (!c) return XF_E_ARG;
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    c->stream = (cudaStream_t)stream;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return XF_OK;
}

int xf_set_state(xf_ctx *c, const double *rho, size_t n_doubles, double r_km)
{
    if (!c) return XF_E_ARG;
    return set_state_impl(c, 0, rho, n_doubles, r_km);
}
int xf_batch_set_state(xf_ctx *c, int inst, const double *rho, size_t n_doubles, double r_km)
{
    if (!c) return XF_E_ARG;
    return set_state_impl(c, inst, rho, n_doubles, r_km);
}

int xf_set_psi(xf_ctx *c, const double *psi, size_t n_doubles, double r_km)
{
    if (!c) return XF_E_ARG;
    return set_psi_impl(c, 0, psi, n_doubles, r_km);
}
int xf_batch_set_psi(xf_ctx *c, int inst, const double *psi, size_t n_doubles, double r_km)
{
    if (!c) return XF_E_ARG;
    return set_psi_impl(c, inst, psi, n_doubles, r_km);
}
int xf_get_psi(xf_ctx *c, double *psi, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    if (!c) return XF_E_ARG;
    return get_psi_impl(c, 0, psi, n_doubles, r_km, steps_done);
}
int xf_batch_get_psi(xf_ctx *c, int inst, double *psi, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    if (!c) return XF_E_ARG;
    return get_psi_impl(c, inst, psi, n_doubles, r_km, steps_done);
}

int xf_init_state(xf_ctx *c, double r_km)
{
    if (!c) return XF_E_ARG;
    return init_state_impl(c, 0, r_km);
}
int xf_batch_init_state(xf_ctx *c, int inst, double r_km)
{
    if (!c) return XF_E_ARG;
    if (inst >= 0) return init_state_impl(c, inst, r_km);
    for (int i = 0; i < (int)c->in.size(); ++i) {
        int rc = init_state_impl(c, i, r_km);
        if (rc) return rc;
    }
    return XF_OK;
}

namespace xfp {

// Frobenius norm of the traceless part of a packed n x n Hermitian matrix.
double traceless_norm(const double *x, int nf)
{
    double tr = 0.0, q = 0.0;
    for (int i = 0; i < nf; ++i) tr += x[i];
    for (int i = 0; i < nf; ++i) q += (x[i] - tr / nf) * (x[i] - tr / nf);
    for (int k = nf; k < nf * nf; ++k) q += 2.0 * x[k] * x[k];
    return std::sqrt(q);
}

// Strict mode, RK4 only: refuse a step size outside RK4's stable region.
// d(rho)/dr = -i kappa_u [H, rho] has eigenvalues -i kappa_u (l_a - l_b), and
// for a traceless Hermitian H the spread l_max - l_min is at most
// sqrt(2) ||H||_F.  Classic RK4 is stable on the imaginary axis for
// |z| <= 2 sqrt(2), so the step is refused when, for some angle u,
//   h kappa_u sqrt(2) (max_E ||H_vac|| + A ||P_e|| + mu ||M0 - gamma_u M1||) > 2 sqrt(2)
// (Frobenius norms of traceless parts; the nu-nu term is taken per angle, so
// the near cancellation of M0 and gamma_u M1 far from the neutrinosphere is
// kept).  Every term is taken at the current radius and state: the matter
// density, the coupling and the bulb weights all fall with r, so the start
// of a call is the worst point.
int check_rk4_stable(xf_ctx *c, int i, double h_km)
{
    InstHost &h = c->in[i];
    if (!h.p.strict || c->stepper != XF_RK4) return XF_OK;
    const int nf = h.nf, m = nf * nf;
    double M[36];
    int rc = moments_all(c, i, M);
    if (rc) return rc;
    const double r = radius(h);
    const Inst d = make_inst(h);
    double hv = 0.0;
    for (int e = 0; e < h.n_E; ++e) {
        const double *t = &h.hvac[(size_t)e * h.S];
        hv = std::max(hv, std::sqrt(nf == 2 ? purity<2, double>(t) : purity<3, double>(t)));
    }
    const double pe = std::sqrt((nf - 1.0) / nf); // ||diag(1, 0[, 0]) - I/n||_F
    const double base = hv + matter_A(d, r) * pe, mu = mu_eff(d, r);
    const bool bulb = h.p.geometry == XF_GEOM_BULB || h.p.geometry == XF_GEOM_MU_R4;
    const double x = h.p.R_nu_km / r;
    double z = 0.0;
    for (int t = 0; t < h.n_u * h.n_phi; ++t) {
        const int j = t / h.n_phi, k = t % h.n_phi;
        const double u = (j + 0.5) / h.n_u;
        const double cu = bulb ? std::sqrt(1.0 - x * x * u) : 1.0;
        const double gam = bulb ? cu : 0.0, kappa = bulb ? 1.0 / cu : 1.0;
        double g2 = 0.0, g3 = 0.0;
        if (h.n_phi > 1) {
            const double sn = std::sqrt(x * x * u), ph = (k + 0.5) * 2.0 * 3.14159265358979323846 / h.n_phi;
            g2 = sn * std::cos(ph);
            g3 = sn * std::sin(ph);
        }
        double G[9];
        for (int q = 0; q < m; ++q) G[q] = M[q] - gam * M[m + q] - g2 * M[2 * m + q] - g3 * M[3 * m + q];
        z = std::max(z, h_km * kappa * std::sqrt(2.0) * (base + mu * traceless_norm(G, nf)));
    }
    if (!(z <= 2.0 * std::sqrt(2.0)))
        return fail(c, XF_E_UNSTABLE, "RK4 step %.6g km at r = %.6g km is outside the stable region (|z| = %.3g > 2.83)",
                    h_km, r, z);
    return XF_OK;
}

} // namespace xfp

int xf_step_async(xf_ctx *c, int64_t n_steps, double dr_km)
{
    if (!c) return XF_E_ARG;
    if (c->stepper == XF_EXPH_ADAPTIVE) return fail(c, XF_E_ARG, "an XF_EXPH_ADAPTIVE context steps with xf_evolve");
    if (n_steps < 0) return fail(c, XF_E_ARG, "n_steps must be >= 0");
    if (!std::isfinite(dr_km) || dr_km <= 0) return fail(c, XF_E_ARG, "dr_km must be finite and > 0");
    InstHost &h = c->in[0];
    if (!h.state_valid) return fail(c, XF_E_STATE, "no valid state (call xf_set_state or xf_init_state)");
    if (n_steps == 0) return XF_OK;
    int rs = check_rk4_stable(c, 0, dr_km);
    if (rs) return rs;
    if (dr_km != h.h) {
        int rc = set_step_size(c, 0, dr_km);
        if (rc) return rc;
        rc = upload_instances(c);
        if (rc) return rc;
    }
    return enqueue_steps(c, n_steps, c->in.size() == 1 ? -1 : 0);
}

int xf_sync(xf_ctx *c)
{
    if (!c) return XF_E_ARG;
    int rc = sync_status(c);
    if (rc) return rc;
    if (c->in[0].err & ERR_NONFINITE)
        return fail(c, XF_E_NONFINITE, "non-finite moments; state kept at step %lld", c->in[0].steps);
    return XF_OK;
}

int xf_step(xf_ctx *c, int64_t n_steps, double dr_km)
{
    int rc = xf_step_async(c, n_steps, dr_km);
    if (rc) return rc;
    return xf_sync(c);
}

int xf_batch_step(xf_ctx *c, int64_t n_steps, const double *dr_km)
{
    if (!c) return XF_E_ARG;
    if (c->stepper == XF_EXPH_ADAPTIVE) return fail(c, XF_E_ARG, "an XF_EXPH_ADAPTIVE context steps with xf_batch_evolve");
    if (n_steps < 0) return fail(c, XF_E_ARG, "n_steps must be >= 0");
    bool changed = false;
    for (size_t i = 0; i < c->in.size(); ++i) {
        InstHost &h = c->in[i];
        if (!h.state_valid) return fail(c, XF_E_STATE, "problem %zu has no valid state", i);
        const double dr = dr_km ? dr_km[i] : h.h;
        if (!std::isfinite(dr) || dr <= 0) return fail(c, XF_E_ARG, "step size of problem %zu invalid", i);
        if (n_steps > 0) {
            int rs = check_rk4_stable(c, (int)i, dr);
            if (rs) return rs;
        }
        if (dr != h.h) {
            int rc = set_step_size(c, (int)i, dr);
            if (rc) return rc;
            changed = true;
        }
    }
    if (changed) {
        int rc = upload_instances(c);
        if (rc) return rc;
    }
    if (n_steps == 0) return XF_OK;
    int rc = enqueue_steps(c, n_steps, -1);
    if (rc) return rc;
    return sync_status(c);
}

int xf_batch_get_state(xf_ctx *c, int inst, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    if (!c) return XF_E_ARG;
    return get_state_impl(c, inst, rho, n_doubles, r_km, steps_done);
}

int xf_batch_status(xf_ctx *c, int inst, int *status, int64_t *steps_done, double *r_km)
{
    InstHost *h = instance(c, inst);
    if (!h) return c ? fail(c, XF_E_ARG, "bad instance index %d", inst) : XF_E_ARG;
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    if (status) *status = !h->state_valid ? XF_E_STATE : (h->err & ERR_NONFINITE) ? XF_E_NONFINITE : XF_OK;
    if (steps_done) *steps_done = h->steps;
    if (r_km) *r_km = radius(*h);
    return XF_OK;
}

int xf_moments_ex(xf_ctx *c, int inst, double *M, size_t n_doubles)
{
    InstHost *h = instance(c, inst);
    if (!h) return c ? fail(c, XF_E_ARG, "bad instance index %d", inst) : XF_E_ARG;
    if (!M || n_doubles != (size_t)4 * h->nf * h->nf) return fail(c, XF_E_ARG, "M must hold 4 n_f^2 doubles");
    return moments_all(c, inst, M);
}

int xf_evolve(xf_ctx *c, double r_end_km, int64_t max_iters, double dr0_km)
{
    if (!c) return XF_E_ARG;
    return evolve_impl(c, &r_end_km, max_iters, &dr0_km, 0);
}

int xf_batch_evolve(xf_ctx *c, const double *r_end_km, int64_t max_iters, const double *dr0_km)
{
    if (!c) return XF_E_ARG;
    if (!r_end_km) return fail(c, XF_E_ARG, "r_end_km is NULL");
    return evolve_impl(c, r_end_km, max_iters, dr0_km, -1);
}

int xf_adapt_status(xf_ctx *c, int inst, int *status, double *r_km, double *h_next_km, int64_t *n_accepted,
                    int64_t *n_rejected, double *last_error)
{
    InstHost *h = instance(c, inst);
    if (!h) return c ? fail(c, XF_E_ARG, "bad instance index %d", inst) : XF_E_ARG;
    if (c->stepper != XF_EXPH_ADAPTIVE) return fail(c, XF_E_ARG, "not an XF_EXPH_ADAPTIVE context");
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    if (status) *status = h->state_valid ? adapt_code(h->ad_status) : XF_E_STATE;
    if (r_km) *r_km = h->r_ad;
    if (h_next_km) *h_next_km = h->h_ad;
    if (n_accepted) *n_accepted = h->n_acc;
    if (n_rejected) *n_rejected = h->n_rej;
    if (last_error) *last_error = h->err_ad;
    return XF_OK;
}

int xf_batch_run_moments(xf_ctx *c, int inst, double *M0, double *M1, size_t n_doubles)
{
    InstHost *h = instance(c, inst);
    if (!h) return c ? fail(c, XF_E_ARG, "bad instance index %d", inst) : XF_E_ARG;
    if (!M0 || !M1) return fail(c, XF_E_ARG, "M0/M1 NULL");
    if (n_doubles != (size_t)h->nf * h->nf) return fail(c, XF_E_ARG, "n_doubles must be n_f*n_f");
    if (c->cyl) return fail(c, XF_E_UNSUPPORTED, "the cylinder model's G is not a sum of two moments");
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    if (!h->state_valid || h->steps == 0 || (h->err & ERR_NONFINITE))
        return fail(c, XF_E_STATE, "no finite step taken since the state was set");
    double t[NVMAX];
    XF_CUDA(c, cudaMemcpyAsync(t, c->mom_out + (size_t)inst * NVMAX, sizeof t, cudaMemcpyDeviceToHost, c->stream),
            "copy moments");
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    const int S = h->S;
    for (int w = 0; w < 2; ++w) {
        const double *m = t + w * S;
        double *x = (w == 0) ? M0 : M1;
        if (h->nf == 2) {
            x[0] = m[0];
            x[1] = -m[0];
            x[2] = m[1];
            x[3] = m[2];
        } else {
            x[0] = m[0];
            x[1] = m[1];
            x[2] = -(m[0] + m[1]);
            for (int k = 0; k < 6; ++k) x[3 + k] = m[2 + k];
        }
    }
    return XF_OK;
}

int xf_batch_outputs(xf_ctx *c, int inst, double *p_surv, double *trace, double *purity, size_t n_bins)
{
    if (!c) return XF_E_ARG;
    return outputs_impl(c, inst, p_surv, trace, purity, n_bins);
}

int xf_batch_size(xf_ctx *c, int *n_problems)
{
    if (!c || !n_problems) return XF_E_ARG;
    *n_problems = (int)c->in.size();
    return XF_OK;
}

int xf_get_state(xf_ctx *c, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done)
{
    if (!c) return XF_E_ARG;
    return get_state_impl(c, 0, rho, n_doubles, r_km, steps_done);
}

int xf_moments(xf_ctx *c, double *M0, double *M1, size_t n_doubles)
{
    if (!c) return XF_E_ARG;
    return moments_impl(c, 0, M0, M1, n_doubles);
}

int xf_outputs(xf_ctx *c, double *p_surv, double *trace, double *purity, size_t n_bins)
{
    if (!c) return XF_E_ARG;
    return outputs_impl(c, 0, p_surv, trace, purity, n_bins);
}

int xf_autotune(xf_ctx *c, int64_t n_probe, double dr_km, const int *cand_in, int n_cand, int *best_tile,
                double *best_ms)
{
    if (!c) return XF_E_ARG;
    if (c->stepper == XF_EXPH_ADAPTIVE) return fail(c, XF_E_ARG, "tile search runs fixed steps");
    if (n_probe < 1 || (cand_in && n_cand < 1) || !std::isfinite(dr_km)) return fail(c, XF_E_ARG, "bad arguments");
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    std::vector<int> cands;
    if (cand_in) {
        for (int k = 0; k < n_cand; ++k) {
            if (cand_in[k] < 0 || cand_in[k] > (1 << 20)) return fail(c, XF_E_ARG, "candidate %d out of range", k);
            cands.push_back(cand_in[k]);
        }
    } else {
        // 0, powers of two from 128 to 16384, and 1.25x / 1.5x steps above 2048
        // (the batched ensemble's optimum lies between 4096 and 8192)
        for (int t : {0, 128, 256, 512, 1024, 2048, 3072, 4096, 5120, 6144, 8192, 12288, 16384}) cands.push_back(t);
    }
    // snapshot: the state planes of every active problem, the progress
    // records and the host views
    std::vector<size_t> offs;
    size_t total = 0;
    for (const InstHost &h : c->in) {
        if (!h.active) continue;
        if (!h.state_valid) return fail(c, XF_E_STATE, "every problem needs a valid state");
        offs.push_back(total);
        total += 3 * align256((size_t)2 * h.SS * h.npad * c->real_bytes);
    }
    unsigned char *snap = (unsigned char *)dev_alloc(c, std::max<size_t>(total, 256));
    if (!snap) return fail(c, XF_E_NOMEM, "device allocation of the state snapshot failed");
    const std::vector<InstHost> views = c->in;
    const int ni = (int)c->in.size();
    std::vector<InstPos> pos(ni);
    XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    XF_CUDA(c, cudaMemcpy(pos.data(), c->pos_d, sizeof(InstPos) * ni, cudaMemcpyDeviceToHost), "read progress");
    auto planes = [&](bool save) -> int {
        size_t k = 0;
        for (const InstHost &h : views) {
            if (!h.active) continue;
            const size_t bytes = 3 * align256((size_t)2 * h.SS * h.npad * c->real_bytes);
            unsigned char *src = c->arena + h.block, *dst = snap + offs[k++];
            XF_CUDA(c, cudaMemcpyAsync(save ? dst : src, save ? src : dst, bytes, cudaMemcpyDeviceToDevice, c->stream),
                    "state snapshot");
        }
        return XF_OK;
    };
    int rc = planes(true);
    const int tile0 = c->tile_request;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = cuda_fail(c, cudaErrorUnknown, "event");
    // cost weights of a three-flavor pair to try: the default, and on packs of
    // mixed flavors also 0.7 and 1.4 times it
    bool has2 = false, has3 = false;
    for (const InstHost &h : c->in)
        if (h.active) (h.nf == 3 ? has3 : has2) = true;
    const double cost0 = c->cost3;
    std::vector<double> costs = {cost0};
    if (has2 && has3) costs = {cost0, 0.7 * cost0, 1.4 * cost0};
    std::vector<std::pair<int, double>> trials;
    for (double w : costs)
        for (int t : cands) trials.push_back({t, w});
    // each plan runs with static runs of tiles and, where it has more tiles
    // than CTAs, with dynamic claiming too
    const int dyn0 = c->dynamic_tiles;
    int best = -1, best_dyn = dyn0;
    double best_t = 0.0, best_cost = cost0;
    for (size_t k = 0; k < trials.size() && !rc; ++k) {
        c->tile_request = trials[k].first;
        c->cost3 = trials[k].second;
        rc = plan_launch(c);
        if (!rc) rc = upload_instances(c);
        for (int i = 0; i < ni && !rc; ++i)
            if (c->in[i].active && dr_km > 0) rc = set_step_size(c, i, dr_km);
        if (!rc) rc = upload_instances(c);
        for (int dyn = 0; dyn < 2 && !rc; ++dyn) {
            if (dyn && (int)c->tiles.size() <= c->G) break;
            c->dynamic_tiles = dyn;
            if (c->graph) { // a captured launch holds the previous setting
                cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
            }
            rc = enqueue_steps(c, n_probe, -1); // untimed
            if (!rc && cudaEventRecord(e0, c->stream) != cudaSuccess) rc = cuda_fail(c, cudaErrorUnknown, "event");
            if (!rc) rc = enqueue_steps(c, n_probe, -1);
            if (!rc && cudaEventRecord(e1, c->stream) != cudaSuccess) rc = cuda_fail(c, cudaErrorUnknown, "event");
            if (!rc) rc = sync_status(c);
            float ms = 0.0f;
            if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = cuda_fail(c, cudaErrorUnknown, "event");
            if (!rc && (best < 0 || ms < best_t)) {
                best = trials[k].first;
                best_cost = trials[k].second;
                best_dyn = dyn;
                best_t = ms;
            }
        }
    }
    // restore states, progress and host views whatever happened
    int rr = planes(false);
    if (!rr) {
        XF_CUDA(c, cudaMemcpyAsync(c->pos_d, pos.data(), sizeof(InstPos) * ni, cudaMemcpyHostToDevice, c->stream),
                "restore progress");
        XF_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    }
    for (int i = 0; i < ni; ++i) {
        InstHost &h = c->in[i];
        const int tb = h.tile_begin, te = h.tile_end;
        h = views[i];
        h.tile_begin = tb;
        h.tile_end = te;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(c, snap);
    c->tile_request = rc ? tile0 : best;
    c->cost3 = rc ? cost0 : best_cost;
    c->dynamic_tiles = rc ? dyn0 : best_dyn;
    int rp = plan_launch(c);
    if (!rp) rp = upload_instances(c);
    if (rc) return rc;
    if (rr) return rr;
    if (rp) return rp;
    if (best_tile) *best_tile = best;
    if (best_ms) *best_ms = best_t / (double)n_probe;
    return XF_OK;
}

int xf_set_option(xf_ctx *c, int option, int64_t value)
{
    if (!c) return XF_E_ARG;
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    switch (option) {
    case XF_OPT_GRID:
    case XF_OPT_TILE_PAIRS: {
        if (value < 0 || value > (1 << 20)) return fail(c, XF_E_ARG, "value must be in [0, 2^20]");
        int &slot = (option == XF_OPT_GRID) ? c->grid_request : c->tile_request;
        int old = slot;
        slot = (int)value;
        int rc = plan_launch(c);
        if (!rc) rc = upload_instances(c);
        if (rc) {
            slot = old;
            plan_launch(c);
            upload_instances(c);
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
    case XF_OPT_GRAPH:
        if (value != 0 && value != 1) return fail(c, XF_E_ARG, "graph option is 0 or 1");
        c->use_graph = (int)value;
        return XF_OK;
    case XF_OPT_DYNAMIC_TILES:
        if (value != 0 && value != 1) return fail(c, XF_E_ARG, "dynamic-tile option is 0 or 1");
        if (c->pending) {
            int rc = sync_status(c);
            if (rc) return rc;
        }
        c->dynamic_tiles = (int)value;
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        return XF_OK;
    default: return fail(c, XF_E_ARG, "unknown option %d", option);
    }
}

int xf_tables(xf_ctx *c, double *E, double *phi)
{
    if (!c) return XF_E_ARG;
    if (E) std::memcpy(E, c->in[0].E.data(), sizeof(double) * c->in[0].E.size());
    if (phi) std::memcpy(phi, c->in[0].phi.data(), sizeof(double) * c->in[0].phi.size());
    return XF_OK;
}

int xf_get_option(xf_ctx *c, int option, int64_t *value)
{
    if (!c || !value) return XF_E_ARG;
    switch (option) {
    case XF_OPT_GRID: *value = c->grid_request; break;
    case XF_OPT_BARRIER_TIMEOUT_NS: *value = (int64_t)c->timeout_ns; break;
    case XF_OPT_TEST_SKIP_ARRIVAL: *value = c->skip_cta; break;
    case XF_OPT_TILE_PAIRS: *value = c->tile_request; break;
    case XF_OPT_GRAPH: *value = c->use_graph; break;
    case XF_OPT_DYNAMIC_TILES: *value = c->dynamic_tiles; break;
    default: return fail(c, XF_E_ARG, "unknown option %d", option);
    }
    return XF_OK;
}

int xf_launch_info(xf_ctx *c, int *ctas, int *threads, int *barriers_per_step)
{
    if (!c) return XF_E_ARG;
    if (ctas) *ctas = c->G;
    if (threads) *threads = c->kern.nt;
    if (barriers_per_step) *barriers_per_step = (c->stepper == XF_RK4) ? 4 : (c->stepper == XF_EXPH) ? 2 : 3;
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
    case XF_E_STEPSIZE: return "XF_E_STEPSIZE";
    case XF_E_BUDGET: return "XF_E_BUDGET";
    default: return "XF_E_UNKNOWN";
    }
}

const char *xf_last_error(const xf_ctx *c)
{
    if (!c) return g_create_error.c_str();
    return c->last_error.c_str();
}

} // extern "C"
