// xf_run.cuh -- the persistent fused integrator kernel (one or many problems).
//
// One cooperative launch advances every active problem ("instance") of a
// pack by up to n_steps fixed radial steps.  Each instance is cut into tiles
// of at most TP (angle, energy) pairs (a multiple of 32); the CTAs of the grid take
// contiguous runs of tiles.  Every integrator stage is one pass over the tiles:
//
//   1. for each of its tiles a CTA sums the partials of all tiles of the
//      tile's instance in tile order (the moments M0, M1 of the stage input,
//      Eq. 3.13), builds the per-angle tables of the tile (weights, cos theta,
//      dl/dr, path length) and updates every pair (both species); each thread
//      accumulates the weighted nu-nu sums of the stage output
//   2. the tile's sums are reduced in fixed order (thread, warp shuffle tree,
//      warps in order) into one partial per tile in global memory
//   3. grid barrier (bounded spin; times out with an error flag, never hangs)
//
// An instance's moments depend only on its own tiles: not on the grid size and
// not on the other instances packed with it, so a problem gives bitwise the
// same result alone and inside a batch (same tile size, threads and precision).
// RK4 needs 4 stages per step, the predictor-corrector (Sec. 4.2.3, Listing
// 5.1 S1-S3) needs 2.  FP32 variants accumulate a warp's sums in FP32 and
// everything above the warp in FP64 (a warp-wide FP64 instruction occupies the
// SM's FP64 pipe for 16 cycles on this GPU).
#pragma once

#include <mutex>

#include <cuda_runtime.h>
#include <stdint.h>

#include "xf_math.cuh"
#include "xf_psi.cuh"

namespace xf {

enum { GEOM_BULB = 0, GEOM_MU_R4 = 1, GEOM_SA = 2, GEOM_CONST = 3, GEOM_CYL = 4 };
enum { MAT_NONE = 0, MAT_POWER = 1, MAT_EXP = 2 };
enum { STEP_RK4 = 0, STEP_EXPH = 1, STEP_ADAPT = 2 };
enum { ERR_NONFINITE = 1, ERR_BARRIER = 2, ERR_LAUNCH = 4 };
// variants of the per-bin arithmetic: plain; moments summed in compensated
// FP32 (TwoSum) up to the warp; plain with the per-step restoration of each
// bin's tr(rho0^2) (|P|^2 / 2 in two flavors) to its initial value
enum { VAR_PLAIN = 0, VAR_COMP = 1, VAR_RENORM = 2, VAR_FF = 3 };

// what the state planes hold: traceless density matrices, or one wavefunction
// per initial flavor (2 n_f^2 reals per bin)
enum { FORM_RHO = 0, FORM_PSI = 1 };
constexpr int NVMAX = 32; // 4 moments x (n_f^2 - 1) for three flavors (extended bulb model)

// One problem of a pack.  Its three state buffers (the two ping-pong copies
// of rho and the auxiliary stage buffer) are component-major planes at Real
// offsets off[0..2] from the arena base: element (c, s, p) at
// off[b] + (c * 2 + s) * npad + p.  Its vacuum table is at Real offset hvac_off.
struct Inst {
    int n_E, n_u, nf, geometry;
    int matter, n_pairs, npad, n_phi; // n_phi: azimuth bins (1: the bulb model); pairs = n_u n_phi n_E
    long long off[3], hvac_off;
    long long ref_off;      // Real: per-bin tr(rho0^2) of the initial state (renormalising variant)
    long long trace_off;    // double: trace per bin [2][npad]
    long long phi_off;      // double: number-flux weights [4][n_E] (nu_e, nubar_e, nu_x, nubar_x)
    int form, pad1_;        // FORM_RHO or FORM_PSI (state planes hold wavefunctions)
    double R, mu0, du, dE;
    double ne_ref, r_ref, ne_power, nb0, h_ns, Ye, gf;
    double r0, h;           // step k of the run starts at r0 + k h
    double eps0, ksi, dr_max; // error-controlled step: tolerance, safety factor, largest step
    int tile_begin, tile_end;
};

// Progress of an instance, kept on the device and advanced by the kernel, so
// that a launch can be replayed (CUDA graph) without host updates.
struct InstPos {
    long long k0;           // steps taken since (r0, h) were set
    long long remaining;    // steps still requested
    unsigned long long steps; // steps taken in total (reported to the host)
    int cur;                // buffer (0/1) holding the current state
    int err;                // ERR_NONFINITE once the instance stopped
};

// Progress of an instance under the error-controlled step.  The device
// keeps one copy per instance between launches and one per tile within a
// launch; every tile of an instance makes the same accept / reject decision
// from the same sums, so the copies stay equal without a further barrier.
enum { AD_RUN = 0, AD_DONE = 1, AD_BUDGET = 2, AD_NONFINITE = 3, AD_STEPSIZE = 4 };
struct AdaptPos {
    double r, h, ht, r_end, err; // radius, next step, step of the attempt in flight, end, last error
    long long iters_left, n_acc, n_rej;
    int cur, in_slot, status, last; // state buffer 0..2; partial slot of its moments; AD_*; attempt ends on r_end
    int ran, pad_;                  // attempted in this launch
};

struct Tile {
    int inst, p0, np, pad_;
};

struct RunArgs {
    const Inst *inst;
    const Tile *tiles;
    const int *cta_tiles;   // [grid + 1]: CTA c processes tiles [cta_tiles[c], cta_tiles[c+1])
    int n_inst, n_tiles, span_max, pad_;
    long long n_steps;      // max over instances
    void *arena;            // base of the problems' state buffers and tables
    double *partials;       // [2][n_tiles][NVMAX]
    double *mom_out;        // [n_inst][NVMAX] M0 | M1 of each instance's final state (dE applied)
    InstPos *pos;           // [n_inst] progress (read and advanced by the kernel)
    unsigned *bar;          // barrier counter, zero at launch
    int *err;               // launch-wide error bits (barrier)
    unsigned long long timeout_ns;
    int skip_cta;           // test hook: this CTA leaves at its first barrier (-1: none)
    AdaptPos *apos;         // error-controlled step: [n_inst] progress (else unused)
    AdaptPos *tstate;       // error-controlled step: [n_tiles] per-tile copies of it
    unsigned *first_bad;    // cylinder model: lowest barrier number after which a non-finite
                            // trajectory sum is read (all ones at launch)
    unsigned long long *ticket; // dynamic tile claiming: ticket counter (zero at launch)
    int dynamic;            // 1: CTAs claim a stage's tiles from the counter; 0: own runs
    int stage_off;          // byte offset of the state staging columns in dynamic shared
                            // memory (FP32 predictor-corrector kernels; 0: none)
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

__host__ __device__ __forceinline__ double matter_A(const Inst &a, double r)
{
    if (a.matter == MAT_POWER) return a.gf * a.ne_ref * pow(a.r_ref / r, a.ne_power);
    if (a.matter == MAT_EXP) return a.gf * a.Ye * a.nb0 * exp(-(r - a.R) / a.h_ns);
    return 0.0;
}

__host__ __device__ __forceinline__ double mu_eff(const Inst &a, double r)
{
    double x = a.R / r, x2 = x * x;
    if (a.geometry == GEOM_MU_R4) return a.mu0 * x2 * x2;
    if (a.geometry == GEOM_CYL) return a.mu0 * x; // a line source thins as 1/r
    if (a.geometry == GEOM_SA) {
        double t = 1.0 - sqrt(1.0 - x2); // Eq. 3.17
        return a.mu0 * 0.5 * t * t;
    }
    return a.mu0;
}

// cos(theta) of trajectory j at radius r (Eq. 3.14), u_j = (j + 1/2) du.
__device__ __forceinline__ double cos_u(const Inst &a, int j, double r)
{
    double x = a.R / r;
    return sqrt(1.0 - x * x * ((j + 0.5) * a.du));
}

// Per-tile tables in shared memory, each slot span_max entries of Real,
// computed in FP64 and stored in the kernel's precision: 0 gamma
// (G = mu (M0 - gamma M1)), 1 kappa = dl/dr, 2 weight a (M0), 3 weight b (M1),
// 4 dl (path length of the step; FP32 kernels keep dl as hi in slot 4 and lo
// in slot 5, see StepLen).
template <typename Real> struct TabSlots;
template <> struct TabSlots<double> { static constexpr int n = 5; };
template <> struct TabSlots<float> { static constexpr int n = 6; };

__device__ __forceinline__ void store_dl(double *tb, int smax, int q, double dl) { tb[4 * smax + q] = dl; }
__device__ __forceinline__ void store_dl(float *tb, int smax, int q, double dl)
{
    const StepLen<float> d = make_step_len(dl, (float *)nullptr);
    tb[4 * smax + q] = d.hi;
    tb[5 * smax + q] = d.lo;
}
__device__ __forceinline__ StepLen<double> load_dl(const double *tb, int smax, int q) { return {tb[4 * smax + q]}; }
__device__ __forceinline__ StepLen<float> load_dl(const float *tb, int smax, int q)
{
    return {tb[4 * smax + q], tb[5 * smax + q]};
}

// Trajectory t = j n_phi + k: zenith bin j, azimuth bin k (n_phi = 1: the
// bulb model's trajectory j).

// Angle factor gamma of G = mu (M0 - gamma M1 - ...) and kappa = dl/dr of
// trajectory t at radius r.
__device__ __forceinline__ void gamma_kappa(const Inst &a, int t, double r, double *g, double *k)
{
    *g = 0.0;
    *k = 1.0;
    if (a.geometry == GEOM_BULB || a.geometry == GEOM_MU_R4) {
        double c = cos_u(a, t / a.n_phi, r);
        *g = c;
        *k = 1.0 / c;
    }
}
// Weights of the nu-nu sums M0, M1 at radius r (Eq. 3.13-3.15; with azimuth
// bins each carries 1/n_phi of its zenith bin's weight).
__device__ __forceinline__ void nu_weights(const Inst &a, int t, double r, double *wa, double *wb)
{
    const int j = t / a.n_phi;
    *wa = a.du;
    *wb = 0.0;
    if (a.geometry == GEOM_BULB) {
        double x = a.R / r, x2 = x * x;
        double c = sqrt(1.0 - x2 * ((j + 0.5) * a.du));
        double w = x2 * a.du / (2.0 * c);
        *wa = w / a.n_phi;
        *wb = w * c / a.n_phi;
    } else if (a.geometry == GEOM_MU_R4) {
        *wb = a.du * cos_u(a, j, r);
    }
}
// Extended bulb model (Eq. 3.18): with cos(gamma) = cos th cos th'
// + sin th sin th' cos(ph - ph'), the azimuthal moments M2, M3 carry the
// weights w sin th' (cos ph', sin ph') / n_phi and enter G with the factors
// sin th (cos ph, sin ph); sin th = x sqrt(u), azimuth midpoints
// ph_k = (k + 1/2) 2 pi / n_phi; a problem with one azimuth bin has none.
__device__ __forceinline__ void azimuth_terms(const Inst &a, int t, double r, double *g2, double *g3, double *wc,
                                              double *wd)
{
    if (a.n_phi == 1) { // one azimuth bin: the azimuthally symmetric bulb model, M2 = M3 = 0
        *g2 = *g3 = *wc = *wd = 0.0;
        return;
    }
    const int j = t / a.n_phi, k = t - j * a.n_phi;
    double x = a.R / r, x2 = x * x, u = (j + 0.5) * a.du;
    double c = sqrt(1.0 - x2 * u), sn = sqrt(x2 * u);
    double sp, cp;
    sincos((k + 0.5) * 2.0 * 3.14159265358979323846 / a.n_phi, &sp, &cp);
    double w = x2 * a.du / (2.0 * c);
    *g2 = sn * cp;
    *g3 = sn * sp;
    *wc = w * sn * cp / a.n_phi;
    *wd = w * sn * sp / a.n_phi;
}
// Exact path length from r to r + h along trajectory t (Eq. 3.3, l = r cos):
// l(r+h) - l(r) = h (2r + h) / (l(r) + l(r+h)), free of cancellation.
__device__ __forceinline__ double path_length(const Inst &a, int t, double r, double h)
{
    if (a.geometry == GEOM_BULB || a.geometry == GEOM_MU_R4) {
        const int j = t / a.n_phi;
        double l0 = r * cos_u(a, j, r), l1 = (r + h) * cos_u(a, j, r + h);
        return h * (2.0 * r + h) / (l0 + l1);
    }
    return h;
}

template <typename Real>
__device__ inline void build_rhs_table(const Inst &a, Real *tb, int smax, int j_lo, int span, double r)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        double g, k;
        gamma_kappa(a, j_lo + q, r, &g, &k);
        tb[0 * smax + q] = (Real)g;
        tb[1 * smax + q] = (Real)k;
    }
}
template <typename Real>
__device__ inline void build_weight_table(const Inst &a, Real *tb, int smax, int j_lo, int span, double r)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        double wa, wb;
        nu_weights(a, j_lo + q, r, &wa, &wb);
        tb[2 * smax + q] = (Real)wa;
        tb[3 * smax + q] = (Real)wb;
    }
}
template <typename Real>
__device__ inline void build_dl_table(const Inst &a, Real *tb, int smax, int j_lo, int span, double r, double h)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) store_dl(tb, smax, q, path_length(a, j_lo + q, r, h));
}
// Extended bulb model: slots base + 0, 1 = the G factors of M2, M3 at r_rhs;
// base + 2, 3 = the weights of M2, M3 at r_out.
template <typename Real>
__device__ inline void build_azimuth_table(const Inst &a, Real *tb, int smax, int base, int j_lo, int span,
                                           double r_rhs, double r_out)
{
    for (int q = threadIdx.x; q < span; q += blockDim.x) {
        double g2, g3, wc, wd;
        azimuth_terms(a, j_lo + q, r_rhs, &g2, &g3, &wc, &wd);
        tb[(base + 0) * smax + q] = (Real)g2;
        tb[(base + 1) * smax + q] = (Real)g3;
        if (r_out != r_rhs) azimuth_terms(a, j_lo + q, r_out, &g2, &g3, &wc, &wd);
        tb[(base + 2) * smax + q] = (Real)wc;
        tb[(base + 3) * smax + q] = (Real)wd;
    }
}

// Shared per-CTA scratch of the kernel.
template <int NT>
struct Shared {
    double M[NVMAX];        // moments (dE applied) of the current tile's instance
    union {                 // never live at once: a barrier separates their uses
        double scr[NT];     // instance totals' scratch
        double w[NT / 32][NVMAX]; // per-warp sums of a tile's partial
    };
    double A, mu;           // stage scalars of the current tile's instance
    int flag, m_inst;       // barrier flag; instance whose moments sit in M
    int ticket, pad_;       // the tile this CTA claimed (-1: none left; dynamic claiming)
    InstPos ps;             // progress record of the current tile's instance
};

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e)
{
    s = a + b;
    T bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Compensated version of cta_partial: the per-thread sums carry their
// rounding errors mc; the warp tree adds pairs with TwoSum; the warp leaders
// hand s + e to the FP64 sum over warps.
template <int NV, int NT, typename Acc, typename SH>
__device__ __forceinline__ void cta_partial_comp(Acc *m, Acc *mc, SH &sh, double *part)
{
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        Acc v = m[c], e = mc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Acc v2 = __shfl_down_sync(0xffffffffu, v, off), e2 = __shfl_down_sync(0xffffffffu, e, off);
            Acc s, er;
            two_sum(v, v2, s, er);
            v = s;
            e = e + e2 + er;
        }
        m[c] = v;
        mc[c] = e;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) sh.w[w][c] = (double)m[c] + (double)mc[c];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) s += sh.w[q][threadIdx.x];
        __stcg(part + threadIdx.x, s);
    }
    __syncthreads();
}

// Reduce per-thread partial sums over the CTA in fixed order: warp shuffle
// tree in Acc precision, warps in order in FP64; writes NV doubles to part.
template <int NV, int NT, typename Acc, typename SH>
__device__ __forceinline__ void cta_partial(Acc *m, SH &sh, double *part)
{
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        Acc v = m[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        m[c] = v;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) sh.w[w][c] = (double)m[c];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) s += sh.w[q][threadIdx.x];
        __stcg(part + threadIdx.x, s);
    }
    __syncthreads();
}

// Moments of an instance: the partials of its tiles [t0, t1) summed (times
// dE), written to sh.M.  Component c of tile g is read by thread
// (g - t0) mod lg * nvp + c, nvp = nv rounded up to a power of two and
// lg = NT / nvp, so that neighbouring threads read one tile's slot; each
// thread keeps two running sums (alternate tiles) to have more loads in
// flight, and the lg sums of a component are added in thread order: a fixed
// order, so results are reproducible.
template <int NT>
__device__ __forceinline__ void instance_total(const double *part, int t0, int t1, int nv, double dE, Shared<NT> &sh)
{
    const int nvp = nv <= 8 ? 8 : (nv <= 16 ? 16 : 32);
    const int lg = NT / nvp;
    const int t = threadIdx.x, c = t & (nvp - 1), k = t / nvp;
    double a0 = 0.0, a1 = 0.0;
    if (c < nv) {
        int g = t0 + k;
        for (; g + lg < t1; g += 2 * lg) {
            a0 += __ldcg(part + (size_t)g * NVMAX + c);
            a1 += __ldcg(part + (size_t)(g + lg) * NVMAX + c);
        }
        if (g < t1) a0 += __ldcg(part + (size_t)g * NVMAX + c);
    }
    sh.scr[t] = a0 + a1;
    __syncthreads();
    if (t < nv) {
        double s = 0.0;
        for (int q = 0; q < lg; ++q) s += sh.scr[q * nvp + t];
        sh.M[t] = s * dE;
    }
    __syncthreads();
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
template <int NF, typename Real, typename Acc>
__device__ __forceinline__ void accum(const Real *tn, const Real *tb, Acc wa, Acc wb, Acc *m)
{
    constexpr int S = Comp<NF>::S;
    Real d[S];
    nu_minus_conj_nubar<NF, Real>(tn, tb, d);
#pragma unroll
    for (int c = 0; c < S; ++c) {
        Acc dc = (Acc)d[c];
        m[c] += wa * dc;
        m[S + c] += wb * dc;
    }
}

// The extended bulb model's four weighted sums (M0..M3).
template <int NF, typename Real, typename Acc>
__device__ __forceinline__ void accum4(const Real *tn, const Real *tb, Acc wa, Acc wb, Acc wc, Acc wd, Acc *m)
{
    constexpr int S = Comp<NF>::S;
    Real d[S];
    nu_minus_conj_nubar<NF, Real>(tn, tb, d);
#pragma unroll
    for (int c = 0; c < S; ++c) {
        Acc dc = (Acc)d[c];
        m[c] += wa * dc;
        m[S + c] += wb * dc;
        m[2 * S + c] += wc * dc;
        m[3 * S + c] += wd * dc;
    }
}

// As accum, with each running sum's rounding error carried in mc (TwoSum).
template <int NF, typename Real, typename Acc>
__device__ __forceinline__ void accum_comp(const Real *tn, const Real *tb, Acc wa, Acc wb, Acc *m, Acc *mc)
{
    constexpr int S = Comp<NF>::S;
    Real d[S];
    nu_minus_conj_nubar<NF, Real>(tn, tb, d);
#pragma unroll
    for (int c = 0; c < S; ++c) {
        Acc dc = (Acc)d[c], s, e;
        two_sum(m[c], wa * dc, s, e);
        m[c] = s;
        mc[c] += e;
        two_sum(m[S + c], wb * dc, s, e);
        m[S + c] = s;
        mc[S + c] += e;
    }
}

// The fields of an instance a tile's inner loop needs, held in registers.
template <typename Real>
struct TileView {
    const Real *cur, *hvac, *ref;
    const double *phi;      // number-flux weights (wavefunction form)
    Real *nxt, *aux;
    int n_E, npad, p0, p1, j_lo;
    double h;
};

// Asynchronous 4-byte copies global -> shared (cp.async, completion tracked
// per thread in commit groups).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// State staging of the FP32 predictor-corrector: while a thread updates one
// pair, the planes of its next pair (rho_n, and in the corrector the
// predictor's output) are already on their way into shared memory.  Each
// thread copies and reads only its own column, two buffers of
// stage_planes(NF) words ([plane][thread], stride NT), so no CTA barrier
// is involved.
// Kernels of one flavor count only: in the kernel for mixed packs, which
// issues on most cycles, the extra copy and shared-load instructions cost
// more than the hidden latency gives (the 256-problem ensemble: 1.73e10
// against 1.77e10 bin-steps/s), while the one-flavor kernels gain 2-3 %.
template <int NFM, int STEP, typename Real, int NMOM>
struct Staging { static constexpr bool on = NFM != 0 && STEP == STEP_EXPH && sizeof(Real) == 4 && NMOM == 2; };
__host__ __device__ constexpr int stage_planes(int nf) { return 4 * (nf == 2 ? 3 : 8); }
// Bytes of staging columns of a kernel of nfm (2 or 3) flavors.
__host__ __device__ constexpr size_t stage_bytes(int nfm, int nt) { return (size_t)2 * stage_planes(nfm) * nt * 4; }
// Dynamic shared memory of a fixed-step run kernel: the per-angle tables
// (table_bytes), then, for the kernels that stage (FP32 predictor-corrector,
// density-matrix form, two moments), the staging columns at *stage_off
// (0 for the others).
inline size_t run_smem(size_t table_bytes, int real_bytes, bool exph, int nmom, int form, int nfm, int nt,
                       int *stage_off)
{
    size_t smem = (table_bytes + 15) & ~(size_t)15;
    *stage_off = 0;
    if (nfm != 0 && real_bytes == 4 && exph && nmom == 2 && form == FORM_RHO) {
        *stage_off = (int)smem;
        smem += stage_bytes(nfm, nt);
    }
    return smem;
}
// Let a kernel launch with `bytes` of dynamic shared memory.  The limit is a
// property of the kernel shared by every context of the process, so it only
// ever grows.  Returns false when the device cannot grant it.
inline bool allow_dynamic_smem(const void *fn, size_t bytes)
{
    static std::mutex mu; // read-and-raise is one step for the whole process
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, fn) != cudaSuccess) return false;
    if ((size_t)at.maxDynamicSharedSizeBytes >= bytes) return true;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}
__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

template <int S, typename Real, int NT>
__device__ __forceinline__ void stage_issue(Real *col, const TileView<Real> &v, int p, bool with_aux)
{
#pragma unroll
    for (int k = 0; k < 2 * S; ++k) cp_async4(col + k * NT, v.cur + (size_t)k * v.npad + p);
    if (with_aux)
#pragma unroll
        for (int k = 0; k < 2 * S; ++k) cp_async4(col + (2 * S + k) * NT, v.aux + (size_t)k * v.npad + p);
}

// One bin's propagation T' = U T U^dagger of the predictor-corrector.  With
// VAR_FF the state, Hamiltonian, tables and sums stay FP64 and only the
// propagator (the eigendecomposition and U T U^dagger, nearly all of a
// bin-step's arithmetic) runs in float-float on the FP32 pipes; its inputs
// are rounded to float-float and its output read back as a double.
template <int NF, typename Real, int VAR>
__device__ __forceinline__ void propagate(const Real *h, StepLen<Real> dl, const Real *t, Real *out)
{
    if constexpr (VAR == VAR_FF) {
        static_assert(sizeof(Real) == 8, "float-float propagation of FP64 state");
        constexpr int S = Comp<NF>::S;
        ff hf[S], tf[S], of[S];
#pragma unroll
        for (int c = 0; c < S; ++c) {
            hf[c] = ff(h[c]);
            tf[c] = ff(t[c]);
        }
        prop<NF, ff>(hf, make_step_len(step_len_value(dl), (ff *)nullptr), tf, of);
#pragma unroll
        for (int c = 0; c < S; ++c) out[c] = to_double(of[c]);
    } else {
        prop<NF, Real>(h, dl, t, out);
    }
}

// One stage of one tile: update every pair, accumulate and reduce the sums.
template <int NF, int STEP, typename Real, int NT, int VAR, int NMOM, bool PF>
__device__ __forceinline__ void stage_tile(const TileView<Real> v, int smax, int st, const Real *tb, Shared<NT> &sh,
                                           double *part_out, Real *stg)
{
    constexpr int NPL = stage_planes(NF);
    static_assert(NMOM == 2 || (NMOM == 4 && VAR == VAR_PLAIN), "azimuth moments: plain arithmetic only");
    constexpr int S = Comp<NF>::S, NV = NMOM * S, AB = TabSlots<Real>::n;
    using Acc = Real; // warp-level accumulation precision
    constexpr int NC = (VAR == VAR_COMP) ? NV : 1;
    Acc mc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) mc[c] = Acc(0);
    const bool last_stage = (STEP == STEP_RK4) ? (st == 3) : (st == 1);
    const double h = v.h;
    const double mu = sh.mu;
    const Real A = (Real)sh.A;
    Real Mq[NMOM][S];
#pragma unroll
    for (int k = 0; k < NMOM; ++k)
#pragma unroll
        for (int c = 0; c < S; ++c) Mq[k][c] = (Real)(mu * sh.M[k * S + c]);
    Acc m[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) m[c] = Acc(0);

    Real *const col0 = PF ? stg + threadIdx.x : nullptr;
    if constexpr (PF) {
        if (v.p0 + (int)threadIdx.x < v.p1) stage_issue<S, Real, NT>(col0, v, v.p0 + threadIdx.x, st == 1);
        cp_async_commit();
    }
    int buf = 0;
    // the pair's angle and energy, (j, e) = divmod(p, n_E), advanced by the
    // stride NT = dj n_E + de without a division per pair
    const int dj = NT / v.n_E, de = NT - dj * v.n_E;
    int j = (v.p0 + (int)threadIdx.x) / v.n_E, e = v.p0 + (int)threadIdx.x - j * v.n_E;
    for (int p = v.p0 + threadIdx.x; p < v.p1; p += NT, buf ^= 1) {
        Real *const col = PF ? col0 + buf * NPL * NT : nullptr;
        if constexpr (PF) {
            if (p + NT < v.p1) stage_issue<S, Real, NT>(col0 + (buf ^ 1) * NPL * NT, v, p + NT, st == 1);
            cp_async_commit();
            cp_async_wait<1>(); // this pair's copies have landed
        }
        const int q = j - v.j_lo;
        const Real gam = tb[q];
        Real g[S], hv[S], hn[S], hb[S];
#pragma unroll
        for (int c = 0; c < S; ++c) {
            g[c] = Mq[0][c] - gam * Mq[1][c];
            hv[c] = v.hvac[(size_t)e * S + c];
        }
        if constexpr (NMOM == 4) {
            const Real g2 = tb[AB * smax + q], g3 = tb[(AB + 1) * smax + q];
#pragma unroll
            for (int c = 0; c < S; ++c) g[c] = g[c] - g2 * Mq[2][c] - g3 * Mq[3][c];
        }
        hamiltonians<NF, Real>(hv, A, g, hn, hb);
        Real on[S], ob[S]; // stage outputs (nu, nubar)
        if constexpr (STEP == STEP_RK4) {
            const Real kap = tb[smax + q];
            const Real cy = (Real)((st == 2) ? h : 0.5 * h);
            const Real cb = (Real)((st == 0 || st == 3) ? h / 6.0 : h / 3.0);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
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
                if (VAR == VAR_RENORM && last_stage) renormalise<NF, Real>(bb, v.ref[(size_t)s * v.npad + p]);
                store_state<Real, S>(v.nxt, v.npad, s, p, bb);
                Real *o = (s == 0) ? on : ob;
                if (st < 3) {
#pragma unroll
                    for (int c = 0; c < S; ++c) o[c] = rn[c] + cy * kk[c];
                    store_state<Real, S>(v.aux, v.npad, s, p, o);
                } else {
#pragma unroll
                    for (int c = 0; c < S; ++c) o[c] = bb[c];
                }
            }
        } else if constexpr (VAR == VAR_FF) {
            // one copy of the float-float propagator in the code, run once per
            // species (unrolled, the two copies overflow the instruction cache:
            // the three-flavor workload ran 18 % and the ensemble 53 % slower)
            const StepLen<Real> dl = load_dl(tb, smax, q);
#pragma unroll 1
            for (int s = 0; s < 2; ++s) {
                Real hs[S], rn[S], pr[S], o[S];
#pragma unroll
                for (int c = 0; c < S; ++c) hs[c] = s == 0 ? hn[c] : hb[c];
                load_state<Real, S>(v.cur, v.npad, s, p, rn);
                propagate<NF, Real, VAR>(hs, dl, rn, pr);
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
                // the weighted sums of the stage output, as the prologue forms them
                // from stored states (so that chunked launches equal one launch)
                if (s == 0) {
#pragma unroll
                    for (int c = 0; c < S; ++c) on[c] = o[c];
                } else {
                    accum<NF, Real, Acc>(on, o, tb[2 * smax + q], tb[3 * smax + q], m);
                }
            }
        } else {
            const StepLen<Real> dl = load_dl(tb, smax, q);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                Real rn[S], pr[S];
                if constexpr (PF) {
#pragma unroll
                    for (int c = 0; c < S; ++c) rn[c] = col[(c * 2 + s) * NT];
                } else {
                    load_state<Real, S>(v.cur, v.npad, s, p, rn);
                }
                propagate<NF, Real, VAR>(s == 0 ? hn : hb, dl, rn, pr);
                Real *o = (s == 0) ? on : ob;
                if (st == 0) {
#pragma unroll
                    for (int c = 0; c < S; ++c) o[c] = pr[c];
                    store_state<Real, S>(v.aux, v.npad, s, p, o);
                } else {
                    Real pp[S];
                    if constexpr (PF) {
#pragma unroll
                        for (int c = 0; c < S; ++c) pp[c] = col[(2 * S + c * 2 + s) * NT];
                    } else {
                        load_state<Real, S>(v.aux, v.npad, s, p, pp);
                    }
#pragma unroll
                    for (int c = 0; c < S; ++c) o[c] = Real(0.5) * (pp[c] + pr[c]);
                    if (VAR == VAR_RENORM && last_stage) renormalise<NF, Real>(o, v.ref[(size_t)s * v.npad + p]);
                    store_state<Real, S>(v.nxt, v.npad, s, p, o);
                }
            }
        }
        if constexpr (VAR == VAR_FF && STEP == STEP_EXPH) {
            // accumulated per species above
        } else if constexpr (NMOM == 4)
            accum4<NF, Real, Acc>(on, ob, tb[2 * smax + q], tb[3 * smax + q], tb[(AB + 2) * smax + q],
                                  tb[(AB + 3) * smax + q], m);
        else if constexpr (VAR == VAR_COMP)
            accum_comp<NF, Real, Acc>(on, ob, tb[2 * smax + q], tb[3 * smax + q], m, mc);
        else accum<NF, Real, Acc>(on, ob, tb[2 * smax + q], tb[3 * smax + q], m);
        e += de;
        j += dj;
        if (e >= v.n_E) {
            e -= v.n_E;
            ++j;
        }
    }
    if constexpr (PF) cp_async_wait<0>();
    if constexpr (VAR == VAR_COMP) cta_partial_comp<NV, NT, Acc>(m, mc, sh, part_out);
    else cta_partial<NV, NT, Acc>(m, sh, part_out);
}

// Number-flux weights of the e flavor and the others for species s at energy e.
template <typename Real>
__device__ __forceinline__ void psi_weights(const TileView<Real> &v, int s, int e, Real *w0, Real *w1)
{
    *w0 = (Real)v.phi[(s == 0 ? 0 : 1) * v.n_E + e];
    *w1 = (Real)v.phi[(s == 0 ? 2 : 3) * v.n_E + e];
}

// One stage of one tile in the wavefunction form: the same stage structure as
// stage_tile (RK4 on d(psi)/dr = -i H psi dl/dr, or the predictor-corrector
// averaging wavefunctions), moments of rho = sum_a phi_a psi_a psi_a^+.
template <int NF, int STEP, typename Real, int NT>
__device__ __forceinline__ void psi_stage_tile(const TileView<Real> v, int smax, int st, const Real *tb, Shared<NT> &sh,
                                               double *part_out)
{
    constexpr int S = Comp<NF>::S, SS = PsiComp<NF>::SS, NV = 2 * S;
    const double h = v.h;
    const double mu = sh.mu;
    const Real A = (Real)sh.A;
    Real M0[S], M1[S];
#pragma unroll
    for (int c = 0; c < S; ++c) {
        M0[c] = (Real)(mu * sh.M[c]);
        M1[c] = (Real)(mu * sh.M[S + c]);
    }
    Real m[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) m[c] = Real(0);
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
        Real tr_[2][S]; // traceless rho of the stage outputs (nu, nubar)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Real w0, w1, o[SS], tr;
            psi_weights(v, s, e, &w0, &w1);
            if constexpr (STEP == STEP_RK4) {
                const Real kap = tb[smax + q];
                const Real cy = (Real)((st == 2) ? h : 0.5 * h);
                const Real cb = (Real)((st == 0 || st == 3) ? h / 6.0 : h / 3.0);
                Real y[SS], k[SS], bb[SS];
                if (st == 0) load_state<Real, SS>(v.cur, v.npad, s, p, y);
                else load_state<Real, SS>(v.aux, v.npad, s, p, y);
                rhs_psi<NF, Real>(s == 0 ? hn : hb, kap, y, k);
                if (st == 0) {
#pragma unroll
                    for (int c = 0; c < SS; ++c) bb[c] = y[c] + cb * k[c];
                } else {
                    load_state<Real, SS>(v.nxt, v.npad, s, p, bb);
#pragma unroll
                    for (int c = 0; c < SS; ++c) bb[c] += cb * k[c];
                }
                store_state<Real, SS>(v.nxt, v.npad, s, p, bb);
                if (st < 3) {
                    Real rn[SS];
                    if (st == 0) {
#pragma unroll
                        for (int c = 0; c < SS; ++c) rn[c] = y[c];
                    } else {
                        load_state<Real, SS>(v.cur, v.npad, s, p, rn);
                    }
#pragma unroll
                    for (int c = 0; c < SS; ++c) o[c] = rn[c] + cy * k[c];
                    store_state<Real, SS>(v.aux, v.npad, s, p, o);
                } else {
#pragma unroll
                    for (int c = 0; c < SS; ++c) o[c] = bb[c];
                }
            } else {
                const StepLen<Real> dl = load_dl(tb, smax, q);
                Real x[SS], u[SS];
                load_state<Real, SS>(v.cur, v.npad, s, p, x);
                prop_psi<NF, Real>(s == 0 ? hn : hb, dl, x, u);
                if (st == 0) {
#pragma unroll
                    for (int c = 0; c < SS; ++c) o[c] = u[c];
                    store_state<Real, SS>(v.aux, v.npad, s, p, o);
                } else {
                    Real pp[SS];
                    load_state<Real, SS>(v.aux, v.npad, s, p, pp);
#pragma unroll
                    for (int c = 0; c < SS; ++c) o[c] = Real(0.5) * (pp[c] + u[c]);
                    store_state<Real, SS>(v.nxt, v.npad, s, p, o);
                }
            }
            psi_rho<NF, Real>(o, w0, w1, tr_[s], &tr);
        }
        accum<NF, Real, Real>(tr_[0], tr_[1], tb[2 * smax + q], tb[3 * smax + q], m);
    }
    cta_partial<NV, NT, Real>(m, sh, part_out);
}

// Prologue for one tile in the wavefunction form: moments of the input state.
template <int NF, typename Real, int NT>
__device__ __forceinline__ void psi_prologue_tile(const TileView<Real> v, int smax, const Real *tb, Shared<NT> &sh,
                                                  double *part_out)
{
    constexpr int S = Comp<NF>::S, SS = PsiComp<NF>::SS, NV = 2 * S;
    Real m[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) m[c] = Real(0);
    for (int p = v.p0 + threadIdx.x; p < v.p1; p += NT) {
        const int j = p / v.n_E, e = p - j * v.n_E, q = j - v.j_lo;
        Real t[2][S];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Real x[SS], w0, w1, tr;
            load_state<Real, SS>(v.cur, v.npad, s, p, x);
            psi_weights(v, s, e, &w0, &w1);
            psi_rho<NF, Real>(x, w0, w1, t[s], &tr);
        }
        accum<NF, Real, Real>(t[0], t[1], tb[2 * smax + q], tb[3 * smax + q], m);
    }
    cta_partial<NV, NT, Real>(m, sh, part_out);
}

// Prologue for one tile: weighted sums of the input state.
template <int NF, typename Real, int NT, int VAR, typename SH, int NMOM = 2>
__device__ __forceinline__ void prologue_tile(const TileView<Real> v, int smax, const Real *tb, SH &sh,
                                              double *part_out)
{
    constexpr int S = Comp<NF>::S, NV = NMOM * S, AB = TabSlots<Real>::n;
    using Acc = Real;
    constexpr int NC = (VAR == VAR_COMP) ? NV : 1;
    Acc m[NV], mc[NC];
#pragma unroll
    for (int c = 0; c < NV; ++c) m[c] = Acc(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) mc[c] = Acc(0);
    for (int p = v.p0 + threadIdx.x; p < v.p1; p += NT) {
        const int q = p / v.n_E - v.j_lo;
        Real tn[S], tb_[S];
        load_state<Real, S>(v.cur, v.npad, 0, p, tn);
        load_state<Real, S>(v.cur, v.npad, 1, p, tb_);
        if constexpr (NMOM == 4)
            accum4<NF, Real, Acc>(tn, tb_, tb[2 * smax + q], tb[3 * smax + q], tb[(AB + 2) * smax + q],
                                  tb[(AB + 3) * smax + q], m);
        else if constexpr (VAR == VAR_COMP)
            accum_comp<NF, Real, Acc>(tn, tb_, tb[2 * smax + q], tb[3 * smax + q], m, mc);
        else accum<NF, Real, Acc>(tn, tb_, tb[2 * smax + q], tb[3 * smax + q], m);
    }
    if constexpr (VAR == VAR_COMP) cta_partial_comp<NV, NT, Acc>(m, mc, sh, part_out);
    else cta_partial<NV, NT, Acc>(m, sh, part_out);
}

__device__ __forceinline__ bool moments_finite(const double *M, int nv)
{
    bool ok = true;
    for (int c = 0; c < nv; ++c) ok = ok && isfinite(M[c]);
    return ok;
}

// Steps instance i takes in this launch (read at each visit; once the owner
// of its first tile advances the record, later visits see 0 and skip it).
__device__ __forceinline__ long long launch_steps(const RunArgs &a, const InstPos &ps)
{
    if (ps.err) return 0;
    return ps.remaining < a.n_steps ? ps.remaining : a.n_steps;
}

template <typename Real>
__device__ __forceinline__ TileView<Real> make_view(const RunArgs &a, const Inst &in, const InstPos &ps,
                                                    const Tile &tl, long long k)
{
    TileView<Real> v;
    Real *const base = (Real *)a.arena;
    Real *const b0 = base + in.off[0], *const b1 = base + in.off[1];
    const bool odd = ((ps.cur + (int)(k & 1)) & 1) != 0;
    v.cur = odd ? b1 : b0;
    v.nxt = odd ? b0 : b1;
    v.aux = base + in.off[2];
    v.hvac = base + in.hvac_off;
    v.ref = base + in.ref_off;
    v.phi = (const double *)a.arena + in.phi_off;
    v.n_E = in.n_E;
    v.npad = in.npad;
    v.p0 = tl.p0;
    v.p1 = tl.p0 + tl.np;
    v.j_lo = tl.p0 / in.n_E;
    v.h = in.h;
    return v;
}

// Record the step count and final moments of an instance whose last step
// has just completed (part_in holds the partials of its final state).
// Advance an instance's progress record by `done` steps (called once per
// instance and launch, by the CTA that owns its first tile).
__device__ __forceinline__ void advance(InstPos *pp, long long done, int err)
{
    pp->k0 += done;
    pp->remaining -= done;
    pp->steps += (unsigned long long)done;
    pp->cur ^= (int)(done & 1);
    if (err) {
        pp->err = err;
        pp->remaining = 0;
    }
}

template <int NT>
__device__ __forceinline__ void finish_instance(const RunArgs &a, const Inst &in, int inst, long long n,
                                                const double *part_in, int nv, Shared<NT> &sh)
{
    __syncthreads();
    instance_total<NT>(part_in, in.tile_begin, in.tile_end, nv, in.dE, sh);
    if (threadIdx.x == 0) {
        sh.m_inst = -1;
        if (moments_finite(sh.M, nv)) {
            for (int c = 0; c < nv; ++c) a.mom_out[(size_t)inst * NVMAX + c] = sh.M[c];
            advance(a.pos + inst, n, 0);
        } else {
            // the last step's output is not finite: its input is the last finite state
            advance(a.pos + inst, n - 1, ERR_NONFINITE);
        }
    }
    __syncthreads();
}

// Resident CTAs per SM the register allocation is fitted to (occupancy for
// latency hiding; no kernel here is limited by shared memory):
//   FP64, 128 threads (three flavors / mixed): 3 (168 registers, a few words
//     spilled); 2 at 244-252 registers measured no faster (the FP64 pipe
//     bounds it);
//   FP32, 128 threads, three flavors: 4 (128 registers, no spills); 5 and 6
//     ran the L2-resident 400,000-bin problem 16 % and 32 % slower;
//   FP32, 128 threads, mixed packs (nfm 0): 6 (80 registers, 56 bytes
//     spilled): their state streams from HBM and more warps hide it (the
//     256-problem ensemble ran 14 % faster than at 4);
//   FP64, 256 threads (two flavors): 2 (~120 registers, no spills);
//   FP32, 256 threads (two flavors): 6 (40 registers, 68 bytes spilled): a
//     stream of served jobs finished 11 % sooner than at 4 (64 registers),
//     a 150-job pack ran 4 % faster.
__host__ __device__ constexpr int min_blocks(int nt, int real_bytes, int nfm = 3, int var = 0)
{
    // float-float: 4 CTAs of 128 threads (128 registers; despite the spills the
    // three-flavor workload ran 4 % and the ensemble 1 % faster than at 3, and
    // 3 ran 14 % and 2 % faster than 2: the kernel wants warps)
    return var == VAR_FF ? (nt == 128 ? 4 : 2)
                         : nt == 128 ? (real_bytes == 8 ? 3 : (nfm == 0 ? 6 : 4)) : (real_bytes == 8 ? 2 : 6);
}

// NFM: 2 or 3 (every instance has that many flavors) or 0 (mixed pack);
// VAR: VAR_PLAIN, VAR_COMP or VAR_RENORM.
// NMOM: 2 moments (the bulb model) or 4 (the extended bulb model, Eq. 3.18;
// its problems may also have a single azimuth bin).  FORM: FORM_RHO, or
// FORM_PSI (wavefunctions; plain arithmetic, two moments).
template <int NFM, int STEP, typename Real, int NT, int VAR, int NMOM = 2, int FORM = FORM_RHO>
__global__ void __launch_bounds__(NT, min_blocks(NT, sizeof(Real), NFM, VAR)) xf_run_kernel(RunArgs a)
{
    extern __shared__ double s_dyn[];
    Real *const s_tab = (Real *)s_dyn;
    Real *const s_stg = (Real *)((char *)s_dyn + a.stage_off);
    __shared__ Shared<NT> sh;
    const int t_begin = a.cta_tiles[blockIdx.x], t_end = a.cta_tiles[blockIdx.x + 1];
    const int smax = a.span_max;
    unsigned nbar = 0;

    // an earlier launch on these buffers failed at a barrier: touch nothing
    if (threadIdx.x == 0) sh.flag = *(volatile int *)a.err;
    __syncthreads();
    if (sh.flag) return;
    constexpr bool STG = FORM == FORM_RHO && Staging<NFM, STEP, Real, NMOM>::on;
    if constexpr (STG) {
        // a launch without room for the staging columns leaves at once, with
        // every CTA, before any barrier
        if (a.stage_off <= 0 || dynamic_smem_bytes() < (unsigned)a.stage_off + stage_bytes(NFM, NT)) {
            if (threadIdx.x == 0) atomicOr(a.err, ERR_LAUNCH);
            return;
        }
    }

    // ---- prologue: weighted sums of every tile's input state at its start radius
    for (int t = t_begin; t < t_end; ++t) {
        const Tile tl = a.tiles[t];
        const Inst &in = a.inst[tl.inst];
        const InstPos ps = a.pos[tl.inst];
        if (launch_steps(a, ps) <= 0) continue;
        const int nf = NFM ? NFM : in.nf;
        const TileView<Real> v = make_view<Real>(a, in, ps, tl, 0);
        const int span = (v.p1 - 1) / in.n_E - v.j_lo + 1;
        __syncthreads();
        const double r_in = in.r0 + (double)ps.k0 * in.h;
        build_weight_table(in, s_tab, smax, v.j_lo, span, r_in);
        if constexpr (NMOM == 4) build_azimuth_table(in, s_tab, smax, TabSlots<Real>::n, v.j_lo, span, r_in, r_in);
        __syncthreads();
        double *out = a.partials + (size_t)t * NVMAX;
        if constexpr (FORM == FORM_PSI) {
            if (nf == 2) {
                if constexpr (NFM != 3) psi_prologue_tile<2, Real, NT>(v, smax, s_tab, sh, out);
            } else {
                if constexpr (NFM != 2) psi_prologue_tile<3, Real, NT>(v, smax, s_tab, sh, out);
            }
        } else if (nf == 2) {
            if constexpr (NFM != 3) prologue_tile<2, Real, NT, VAR, Shared<NT>, NMOM>(v, smax, s_tab, sh, out);
        } else {
            if constexpr (NFM != 2) prologue_tile<3, Real, NT, VAR, Shared<NT>, NMOM>(v, smax, s_tab, sh, out);
        }
    }
    if (!grid_barrier(a, ++nbar, &sh.flag)) return;

    constexpr int NSTAGE = (STEP == STEP_RK4) ? 4 : 2;
    for (long long k = 0; k < a.n_steps; ++k) {
#pragma unroll 1
        for (int st = 0; st < NSTAGE; ++st) {
            const double *part_in = a.partials + (size_t)((nbar - 1) & 1) * a.n_tiles * NVMAX;
            double *part_out = a.partials + (size_t)(nbar & 1) * a.n_tiles * NVMAX;
            if (threadIdx.x == 0) sh.m_inst = -1;
            auto tile_stage = [&](const int t) {
                const Tile tl = a.tiles[t];
                const Inst &in = a.inst[tl.inst];
                const InstPos &ps = sh.ps;
                const long long n_i = launch_steps(a, ps);
                if (n_i <= 0 || k > n_i) return;
                const int nf = NFM ? NFM : in.nf, nv = NMOM * (nf * nf - 1);
                if (k == n_i) { // the instance's last step of this launch just completed
                    if (st == 0 && t == in.tile_begin) finish_instance<NT>(a, in, tl.inst, n_i, part_in, nv, sh);
                    return;
                }
                double *out = part_out + (size_t)t * NVMAX;
                // moments of the stage input of this tile's instance (once per instance)
                __syncthreads();
                if (sh.m_inst != tl.inst) {
                    instance_total<NT>(part_in, in.tile_begin, in.tile_end, nv, in.dE, sh);
                    if (threadIdx.x == 0) sh.m_inst = tl.inst;
                }
                __syncthreads();
                if (!moments_finite(sh.M, nv)) {
                    // The instance stops.  Stage 0 checks the output of the
                    // previous step: the last finite state is then step k-1's
                    // input; later stages check intermediates of step k.
                    // Non-finite partials keep every later stage skipping it.
                    if (threadIdx.x < NVMAX) __stcg(out + threadIdx.x, (double)NAN);
                    if (threadIdx.x == 0 && t == in.tile_begin) {
                        const long long done = (st == 0) ? (k > 0 ? k - 1 : 0) : k;
                        advance(a.pos + tl.inst, done, ERR_NONFINITE);
                    }
                    return;
                }
                const double kk = (double)(ps.k0 + k), h = in.h;
                const double r = in.r0 + kk * h, r_half = in.r0 + (kk + 0.5) * h, r_next = in.r0 + (kk + 1.0) * h;
                double r_rhs, r_out;
                if constexpr (STEP == STEP_RK4) {
                    r_rhs = (st == 0) ? r : (st == 3 ? r_next : r_half);
                    r_out = (st <= 1) ? r_half : r_next;
                } else {
                    r_rhs = (st == 0) ? r : r_next;
                    r_out = r_next;
                }
                const TileView<Real> v = make_view<Real>(a, in, ps, tl, k);
                const int span = (v.p1 - 1) / in.n_E - v.j_lo + 1;
                build_rhs_table(in, s_tab, smax, v.j_lo, span, r_rhs);
                build_weight_table(in, s_tab, smax, v.j_lo, span, r_out);
                // the step's path lengths serve both stages; a CTA holding several
                // tiles rebuilds them for every tile
                if (STEP == STEP_EXPH) build_dl_table(in, s_tab, smax, v.j_lo, span, r, h);
                if constexpr (NMOM == 4)
                    build_azimuth_table(in, s_tab, smax, TabSlots<Real>::n, v.j_lo, span, r_rhs, r_out);
                if (threadIdx.x == 0) {
                    sh.mu = mu_eff(in, r_rhs);
                    sh.A = matter_A(in, r_rhs);
                }
                __syncthreads();
                if constexpr (FORM == FORM_PSI) {
                    if (nf == 2) {
                        if constexpr (NFM != 3) psi_stage_tile<2, STEP, Real, NT>(v, smax, st, s_tab, sh, out);
                    } else {
                        if constexpr (NFM != 2) psi_stage_tile<3, STEP, Real, NT>(v, smax, st, s_tab, sh, out);
                    }
                } else if (nf == 2) {
                    if constexpr (NFM != 3) stage_tile<2, STEP, Real, NT, VAR, NMOM, STG>(v, smax, st, s_tab, sh, out, s_stg);
                } else {
                    if constexpr (NFM != 2) stage_tile<3, STEP, Real, NT, VAR, NMOM, STG>(v, smax, st, s_tab, sh, out, s_stg);
                }
            };
            // Thread 0 takes the next tile (the next of the CTA's own run, or
            // a ticket) and reads its instance's progress record; both reach
            // the CTA through shared memory.  One call site of tile_stage
            // serves both ways of taking tiles, so a tile runs the same
            // instructions whichever CTA takes it.  Dynamic claiming: stage s
            // owns the tickets [s (T + G), (s + 1) (T + G)); each CTA draws
            // until one lands past the T tiles, so exactly G tickets beyond
            // them go.  The progress record is read once per tile and CTA:
            // another CTA may advance it meanwhile (an instance that ends or
            // stops), and every thread must take the same branches.
            int next = t_begin;
            for (;;) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    int t = -1;
                    if (a.dynamic) {
                        const unsigned long long base =
                            (unsigned long long)(k * NSTAGE + st) * (unsigned long long)(a.n_tiles + gridDim.x);
                        const long long d = (long long)(atomicAdd(a.ticket, 1ull) - base);
                        if (d < a.n_tiles) t = (int)d;
                    } else if (next < t_end) {
                        t = next++;
                    }
                    sh.ticket = t;
                    if (t >= 0) sh.ps = a.pos[a.tiles[t].inst];
                }
                __syncthreads();
                const int t = sh.ticket;
                if (t < 0) break;
                tile_stage(t);
            }
            if (!grid_barrier(a, ++nbar, &sh.flag)) return;
        }
    }
    // instances that ran to the end of the launch
    const double *part_in = a.partials + (size_t)((nbar - 1) & 1) * a.n_tiles * NVMAX;
    for (int t = t_begin; t < t_end; ++t) {
        const Tile tl = a.tiles[t];
        const Inst &in = a.inst[tl.inst];
        if (t != in.tile_begin) continue;
        const long long n_i = launch_steps(a, a.pos[tl.inst]);
        if (n_i != a.n_steps || n_i <= 0) continue;
        const int nf = NFM ? NFM : in.nf;
        finish_instance<NT>(a, in, tl.inst, n_i, part_in, NMOM * (nf * nf - 1), sh);
    }
}

} // namespace xf
