// xf_noalloc.cu -- xf_step_noalloc: advance a state held in the caller's
// device memory without allocating anything.
//
// Who needs this: callers that cannot call cudaMalloc at the moment they want
// to step a problem.  Examples are code running inside a memory pool that
// owns the whole device budget, a plug-in loaded into a host application that
// forbids allocations on its hot path, and real-time loops where an allocation
// (and its implicit synchronisation) would break the latency budget.  They pass
// device buffers they already own for the input and the output; every other
// byte of working memory (the component-major state buffers, the per-energy
// table, the CTA partial moments and the barrier / error / step words of the
// persistent kernel) comes from one file-scope device array.
//
// Limits and behaviour (also stated in include/xf.h):
//   - the array holds XF_NOALLOC_SCRATCH_BYTES (32 MiB) on every GPU that
//     loads libxf.so, for the life of the process;
//   - problems whose working set exceeds it are rejected with XF_E_TOO_BIG;
//   - every call shares the array: the control words are cleared at the start
//     of each call, the state buffers are fully rewritten from the input, and
//     two calls whose work overlaps on the GPU (different streams or host
//     threads) race on the array;
//   - the call synchronises on its stream and reads status words back to the
//     host, so it must never be called while that stream is being captured;
//     the first call on a device also looks up the device address of the
//     array (cudaGetSymbolAddress);
//   - n_steps == 0 returns at once and leaves the caller's buffer untouched;
//     a non-finite input is refused (XF_E_STATE) before any step is taken;
//   - every failure leaves its message where xf_last_error(NULL) reads it
//     (per host thread, shared with xf_create).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "../../include/xf.h"
#include "xf_aux.cuh"
#include "xf_kernels.h"
#include "xf_pack.h"

using namespace xf;

static __device__ __align__(256) unsigned char g_noalloc_scratch[XF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
// Failures return their status code and leave `why` in this host thread's
// last-error message (xf_last_error(NULL)), as a failed xf_create does.
int noalloc_fail(int code, const char *why)
{
    return xfp::fail(nullptr, code, "xf_step_noalloc: %s", why);
}

// Device address of the scratch array for the current device, looked up once
// per device with that device current.
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(XF_E_CUDA, "no usable CUDA device");
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return noalloc_fail(XF_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return XF_OK;
}

// Traceless vacuum Hamiltonian per energy bin (Eq. 3.5-3.6; 3 flavors in the
// mass basis), computed on the device so that no host table is needed.
template <int NF, typename Real>
__global__ void vacuum_table_kernel(Real *hv, int n_E, double E_min, double dE, double K, double dm2a,
                                    double dm2b, double c2, double s2, double u00, double u01, double u02,
                                    double u10, double u11, double u12, double u20, double u21, double u22)
{
    constexpr int S = Comp<NF>::S;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_E; e += gridDim.x * blockDim.x) {
        const double E = E_min + (e + 0.5) * dE;
        double h[S];
        if constexpr (NF == 2) {
            const double Delta = K * dm2a / E;
            h[0] = -0.5 * Delta * c2;
            h[1] = 0.5 * Delta * s2;
            h[2] = 0.0;
        } else {
            const double U[3][3] = {{u00, u01, u02}, {u10, u11, u12}, {u20, u21, u22}};
            const double m2[3] = {0.0, dm2a, dm2b};
            double H[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += U[i][k] * m2[k] * U[j][k];
                    H[i][j] = K / E * s;
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
        for (int c = 0; c < S; ++c) hv[(size_t)e * S + c] = (Real)h[c];
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Tiles of TP pairs over one problem, and contiguous runs of tiles per CTA
// (computed on the device so that no host array is needed).
__global__ void noalloc_plan_kernel(Tile *tiles, int *cta_tiles, int T, int TP, int n_pairs, int G)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int p0 = t * TP;
        tiles[t] = Tile{0, p0, min(TP, n_pairs - p0), 0};
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= G; c += gridDim.x * blockDim.x)
        cta_tiles[c] = (int)(((long long)c * T) / G);
}

__global__ void noalloc_pos_kernel(InstPos *pos, long long n_steps)
{
    pos->k0 = 0;
    pos->remaining = n_steps;
    pos->steps = 0;
    pos->cur = 0;
    pos->err = 0;
}

template <int NF, typename Real>
int run_noalloc(int n_E, int n_u, const xf_params *p, double *rho_dev, double r_km, int64_t n_steps,
                double dr_km, cudaStream_t stream, unsigned char *base)
{
    constexpr int S = Comp<NF>::S;
    const int n_pairs = n_E * n_u;
    const int npad = (n_pairs + 63) & ~63;
    const int st = (p->stepper == XF_RK4) ? STEP_RK4 : STEP_EXPH;
    const int var = p->precision == XF_FP32_COMP ? VAR_COMP : p->precision == XF_FP32_M64_RENORM ? VAR_RENORM : VAR_PLAIN;
    const bool renorm = var == VAR_RENORM;
    const RunKernel kern = std::is_same<Real, double>::value ? run_kernel_fp64(NF, st) : run_kernel_fp32(NF, st, var);
    if (!kern.fn) return noalloc_fail(XF_E_UNSUPPORTED, "kernel variant not built");

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(XF_E_CUDA, "device query failed");
    }
    // launch shape: at most one tile per co-resident CTA
    int occ0 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, kern.fn, kern.nt, 0) != cudaSuccess || occ0 < 1) {
        cudaGetLastError();
        return noalloc_fail(XF_E_UNSUPPORTED, "integrator kernel cannot be resident");
    }
    // one tile per co-resident CTA slot, a multiple of 32 pairs
    const long long slots = (long long)occ0 * sms;
    const int TP = (int)std::min<long long>(
        1 << 20, std::max<long long>(32, ((n_pairs + slots - 1) / slots + 31) / 32 * 32));
    const int T = (n_pairs + TP - 1) / TP;
    const int span = std::min(n_u, (TP + n_E - 1) / n_E + 1);
    int stage_off = 0;
    const size_t smem = run_smem((sizeof(Real) == 8 ? 5 * sizeof(double) : 6 * sizeof(float)) * (size_t)std::max(span, 1),
                                 (int)sizeof(Real), st == STEP_EXPH, 2, FORM_RHO, NF, kern.nt, &stage_off);
    if (!allow_dynamic_smem(kern.fn, smem)) { // static plus dynamic shared memory may pass 48 KB
        cudaGetLastError();
        return noalloc_fail(XF_E_UNSUPPORTED, "angle table too large for shared memory");
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern.fn, kern.nt, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return noalloc_fail(XF_E_UNSUPPORTED, "integrator kernel cannot be resident");
    }
    const int G = std::max(1, std::min(T, occ * sms));

    // carve the scratch array
    const size_t plane = align256((size_t)2 * S * npad * sizeof(Real));
    size_t off = 0;
    Real *rho0 = (Real *)(base + off);
    off += plane;
    Real *rho1 = (Real *)(base + off);
    off += plane;
    Real *aux = (Real *)(base + off);
    off += plane;
    double *trace = (double *)(base + off);
    off += align256(sizeof(double) * 2 * (size_t)npad);
    Real *hvac = (Real *)(base + off);
    off += align256(sizeof(Real) * (size_t)n_E * S);
    Real *ref = renorm ? (Real *)(base + off) : nullptr;
    if (renorm) off += align256(sizeof(Real) * 2 * (size_t)npad);
    double *partials = (double *)(base + off);
    off += align256(sizeof(double) * 2 * (size_t)T * NVMAX);
    Tile *tiles = (Tile *)(base + off);
    off += align256(sizeof(Tile) * (size_t)T);
    int *cta_tiles = (int *)(base + off);
    off += align256(sizeof(int) * (size_t)(G + 1));
    Inst *inst = (Inst *)(base + off);
    off += align256(sizeof(Inst));
    InstPos *pos = (InstPos *)(base + off);
    off += align256(sizeof(InstPos));
    double *mom_out = (double *)(base + off);
    off += align256(sizeof(double) * NVMAX);
    unsigned char *ctrl = base + off; // bar | err | bad
    off += 256;
    if (off > (size_t)XF_NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(XF_E_TOO_BIG, "working set larger than XF_NOALLOC_SCRATCH_BYTES");
    unsigned *bar = (unsigned *)ctrl;
    int *err = (int *)(ctrl + 64);
    int *bad = (int *)(ctrl + 128);

#define NA_CUDA(call, what)                                                                         \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            cudaGetLastError();                                                                     \
            return noalloc_fail(e_ == cudaErrorMemoryAllocation ? XF_E_NOMEM : XF_E_CUDA, what);    \
        }                                                                                           \
    } while (0)

    // the array keeps the previous call's contents: clear what must start at zero
    NA_CUDA(cudaMemsetAsync(ctrl, 0, 256, stream), "clear control words");

    // per-energy table (mixing scalars from the host, the table on the device)
    const double K = 1.0 / (2.0e6 * 1.973269804e-10); // dm^2/(2E) in km^-1 (Eq. 3.6)
    const double dE = (p->E_max_MeV - p->E_min_MeV) / n_E;
    double u[9] = {0};
    if (NF == 3) {
        const double s12 = std::sin(p->theta[0]), c12 = std::cos(p->theta[0]);
        const double s13 = std::sin(p->theta[1]), c13 = std::cos(p->theta[1]);
        const double s23 = std::sin(p->theta[2]), c23 = std::cos(p->theta[2]);
        const double U[9] = {c12 * c13, s12 * c13, s13,
                             -s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13,
                             s12 * s23 - c12 * c23 * s13, -c12 * s23 - s12 * c23 * s13, c23 * c13};
        std::memcpy(u, U, sizeof u);
    }
    const double dm2a = (NF == 2) ? p->hierarchy * p->dm2_eV2[0] : p->dm2_eV2[0];
    const double dm2b = (NF == 2) ? 0.0 : p->hierarchy * p->dm2_eV2[1];
    vacuum_table_kernel<NF, Real><<<(n_E + 127) / 128, 128, 0, stream>>>(
        hvac, n_E, p->E_min_MeV, dE, K, dm2a, dm2b, std::cos(2.0 * p->theta[0]), std::sin(2.0 * p->theta[0]),
        u[0], u[1], u[2], u[3], u[4], u[5], u[6], u[7], u[8]);
    NA_CUDA(cudaGetLastError(), "table kernel");
    noalloc_plan_kernel<<<(std::max(T, G + 1) + 127) / 128, 128, 0, stream>>>(tiles, cta_tiles, T, TP, n_pairs, G);
    NA_CUDA(cudaGetLastError(), "plan kernel");
    noalloc_pos_kernel<<<1, 1, 0, stream>>>(pos, n_steps);
    NA_CUDA(cudaGetLastError(), "position kernel");

    // the problem's descriptor (a stack value; the copy is staged before return)
    Inst d;
    std::memset(&d, 0, sizeof d);
    d.n_E = n_E;
    d.n_u = n_u;
    d.nf = NF;
    d.geometry = p->geometry;
    d.matter = p->matter;
    d.n_pairs = n_pairs;
    d.npad = npad;
    d.n_phi = 1;
    d.off[0] = rho0 - (Real *)base;
    d.off[1] = rho1 - (Real *)base;
    d.off[2] = aux - (Real *)base;
    d.hvac_off = hvac - (Real *)base;
    d.ref_off = renorm ? ref - (Real *)base : 0;
    d.R = p->R_nu_km;
    d.mu0 = p->mu0_per_km;
    d.du = 1.0 / n_u;
    d.dE = dE;
    d.ne_ref = p->ne_ref_cm3;
    d.r_ref = p->r_ref_km;
    d.ne_power = p->ne_power;
    d.nb0 = p->nb0_cm3;
    d.h_ns = p->h_ns_km;
    d.Ye = p->Ye;
    d.gf = std::sqrt(2.0) * 1.1663787e-23 * std::pow(1.973269804e-5, 3) / 1.973269804e-10; // Eq. 3.7
    d.r0 = r_km;
    d.h = dr_km;
    d.tile_begin = 0;
    d.tile_end = T;
    NA_CUDA(cudaMemcpyAsync(inst, &d, sizeof d, cudaMemcpyHostToDevice, stream), "copy descriptor");

    // caller's packed state -> component-major working buffers
    LayoutArgs la;
    std::memset(&la, 0, sizeof la);
    la.n_E = n_E;
    la.n_u = n_u;
    la.n_pairs = n_pairs;
    la.npad = npad;
    la.bad = bad;
    const int egrid = (int)std::min<long long>((2ll * n_pairs + 255) / 256, (long long)sms * 16);
    pack_to_state_kernel<NF, Real><<<egrid, 256, 0, stream>>>(la, rho_dev, rho0, trace, ref);
    NA_CUDA(cudaGetLastError(), "layout kernel");
    // refuse a non-finite input before spending any step on it
    int h_bad = 0;
    NA_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, stream), "read flag");
    NA_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    if (h_bad) return noalloc_fail(XF_E_STATE, "input state contains non-finite values; nothing was run");

    // the persistent integrator, in launches of at most 65536 steps
    const long long kChunk = 1ll << 16;
    for (long long done = 0; done < n_steps;) {
        const long long m = std::min<long long>(n_steps - done, kChunk);
        RunArgs a;
        std::memset(&a, 0, sizeof a);
        a.inst = inst;
        a.tiles = tiles;
        a.cta_tiles = cta_tiles;
        a.n_inst = 1;
        a.n_tiles = T;
        a.span_max = span;
        a.n_steps = m;
        a.arena = base;
        a.partials = partials;
        a.mom_out = mom_out;
        a.pos = pos;
        a.bar = bar;
        a.err = err;
        a.timeout_ns = 2000000000ull;
        a.skip_cta = -1;
        a.stage_off = stage_off;
        NA_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), stream), "clear barrier");
        void *args[] = {&a};
        cudaError_t e = (G > 1) ? cudaLaunchCooperativeKernel(kern.fn, dim3(G), dim3(kern.nt), args, smem, stream)
                                : cudaLaunchKernel(kern.fn, dim3(1), dim3(kern.nt), args, smem, stream);
        NA_CUDA(e, "launch of the integrator kernel");
        done += m;
    }

    int h_err = 0;
    InstPos h_pos;
    NA_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream), "read error word");
    NA_CUDA(cudaMemcpyAsync(&h_pos, pos, sizeof(InstPos), cudaMemcpyDeviceToHost, stream), "read progress");
    NA_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    if (h_err & ERR_LAUNCH) return noalloc_fail(XF_E_CUDA, "integrator launched without its staging area");
    if (h_err & ERR_BARRIER) return noalloc_fail(XF_E_BARRIER_TIMEOUT, "grid barrier timed out; output not written");

    // working buffers -> caller's packed state (the buffer of the last step taken)
    Real *last = h_pos.cur ? rho1 : rho0;
    state_to_pack_kernel<NF, Real><<<egrid, 256, 0, stream>>>(la, last, trace, rho_dev);
    NA_CUDA(cudaGetLastError(), "layout kernel");
    NA_CUDA(cudaStreamSynchronize(stream), "stream synchronize");
    if (h_pos.err & ERR_NONFINITE)
        return noalloc_fail(XF_E_NONFINITE, "non-finite moments; output holds the last finite state");
#undef NA_CUDA
    return XF_OK;
}

} // namespace

extern "C" int xf_step_noalloc(int n_E, int n_u, int n_flavor, const xf_params *p, double *rho_dev, double r_km,
                               int64_t n_steps, double dr_km, void *stream)
{
    if (!p || !rho_dev) return noalloc_fail(XF_E_ARG, "params and rho_dev must be non-NULL");
    if (p->size != sizeof(xf_params) || p->version != XF_PARAMS_VERSION)
        return noalloc_fail(XF_E_ARG, "params.size / params.version mismatch");
    if (n_E <= 0 || n_u <= 0 || (n_flavor != 2 && n_flavor != 3))
        return noalloc_fail(XF_E_ARG, "need n_E, n_u > 0 and n_flavor in {2, 3}");
    if ((long long)n_E * n_u > (long long)(INT_MAX / 16)) return noalloc_fail(XF_E_ARG, "n_E * n_u too large");
    if (p->stepper == XF_EXPH_ADAPTIVE)
        return noalloc_fail(XF_E_UNSUPPORTED, "the error-controlled step is not built for this entry point");
    if (p->n_phi != 1) return noalloc_fail(XF_E_UNSUPPORTED, "azimuth bins are not built for this entry point");
    if (p->form != XF_FORM_RHO)
        return noalloc_fail(XF_E_UNSUPPORTED, "the wavefunction form is not built for this entry point");
    if (p->geometry == XF_GEOM_CYLINDER)
        return noalloc_fail(XF_E_UNSUPPORTED, "the cylinder model is not built for this entry point");
    if (p->stepper != XF_RK4 && p->stepper != XF_EXPH) return noalloc_fail(XF_E_ARG, "bad stepper");
    if (p->precision < XF_FP64 || p->precision > XF_FP32_M64_RENORM) return noalloc_fail(XF_E_ARG, "bad precision");
    if (p->geometry < XF_GEOM_BULB || p->geometry > XF_GEOM_CONST) return noalloc_fail(XF_E_ARG, "bad geometry");
    if (p->geometry == XF_GEOM_SINGLE_ANGLE && n_u != 1)
        return noalloc_fail(XF_E_ARG, "single-angle geometry needs n_u == 1");
    if (p->hierarchy != 1 && p->hierarchy != -1) return noalloc_fail(XF_E_ARG, "hierarchy must be +1 or -1");
    if (p->matter < XF_MATTER_NONE || p->matter > XF_MATTER_EXP) return noalloc_fail(XF_E_ARG, "bad matter profile");
    if (!(p->R_nu_km > 0) || !std::isfinite(p->R_nu_km) || !std::isfinite(p->mu0_per_km) || p->mu0_per_km < 0 ||
        !(p->E_max_MeV > p->E_min_MeV) || p->E_min_MeV < 0 || !std::isfinite(p->E_max_MeV))
        return noalloc_fail(XF_E_ARG, "physical parameters invalid");
    if (!std::isfinite(r_km) || r_km < p->R_nu_km) return noalloc_fail(XF_E_ARG, "r_km must be finite and >= R_nu");
    if (n_steps < 0) return noalloc_fail(XF_E_ARG, "n_steps must be >= 0");
    if (!std::isfinite(dr_km) || dr_km <= 0) return noalloc_fail(XF_E_ARG, "dr_km must be finite and > 0");
    xfp::fail(nullptr, XF_OK, "%s", ""); // no failure so far in this call
    if (n_steps == 0) return XF_OK;     // nothing to do: rho_dev is left as it is
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool fp64 = (p->precision == XF_FP64);
    unsigned char *base = (unsigned char *)scratch;
    if (n_flavor == 2)
        return fp64 ? run_noalloc<2, double>(n_E, n_u, p, rho_dev, r_km, n_steps, dr_km, s, base)
                    : run_noalloc<2, float>(n_E, n_u, p, rho_dev, r_km, n_steps, dr_km, s, base);
    return fp64 ? run_noalloc<3, double>(n_E, n_u, p, rho_dev, r_km, n_steps, dr_km, s, base)
                : run_noalloc<3, float>(n_E, n_u, p, rho_dev, r_km, n_steps, dr_km, s, base);
}
