// xf_pack.h -- host-side state of a pack of problems (an xf_ctx) and the
// internal operations on it, shared by the C ABI (xf_api.cu) and the
// serving loop (xf_server.cu).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/xf.h"
#include "xf_aux.cuh"
#include "xf_kernels.h"

namespace xfp {

using xf::AdaptPos;
using xf::Inst;
using xf::InstPos;
using xf::RunKernel;
using xf::Tile;

// First-fit allocator of byte ranges inside one preallocated device arena.
class Arena {
  public:
    void reset(long long capacity)
    {
        free_.clear();
        cap_ = capacity;
        used_ = 0;
        if (capacity > 0) free_[0] = capacity;
    }
    // offset of a free range of n bytes (n > 0), 256-byte aligned, or -1
    long long alloc(long long n)
    {
        n = (n + 255) & ~255ll;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                long long off = it->first, rest = it->second - n;
                free_.erase(it);
                if (rest > 0) free_[off + n] = rest;
                sizes_[off] = n;
                used_ += n;
                return off;
            }
        }
        return -1;
    }
    void release(long long off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        long long n = s->second;
        sizes_.erase(s);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    long long used() const { return used_; }
    long long capacity() const { return cap_; }

  private:
    std::map<long long, long long> free_, sizes_;
    long long cap_ = 0, used_ = 0;
};

// Host record of one problem of a pack.
struct InstHost {
    bool active = false;              // slot holds a problem
    int n_E = 0, n_u = 0, n_phi = 1, nf = 0, S = 0, n_pairs = 0, npad = 0; // pairs = n_u n_phi n_E
    int SS = 0;                       // state components per bin: S (rho form) or 2 n_f^2 (psi form)
    long long n_bins = 0;
    xf_params p{};
    std::vector<double> E, phi, hvac; // tables: E[n_E], phi[4][n_E], hvac[n_E][S]
    // the problem's block in the pack arena (bytes) and its parts (element
    // offsets from the arena base in the part's own type)
    long long block = -1, block_bytes = 0;
    long long off[3] = {0, 0, 0};     // Real: the state (two copies) and the stage buffer, SS planes each
    long long trace_off = 0;          // double: trace per bin (2 npad)
    long long hvac_off = 0;           // Real: vacuum table (n_E x S)
    long long ref_off = 0;            // Real: initial tr(T^2) per bin (2 npad), renormalising variant only
    long long phi_off = 0;            // double: number-flux weights (4 n_E)
    int tile_begin = 0, tile_end = 0;
    // position (host view, valid after a sync): r = r0 + k0 h
    bool state_valid = false;
    double r0 = 0.0, h = 0.0;
    long long k0 = 0, steps = 0;
    int cur = 0, err = 0;
    // error-controlled step (host view of the device AdaptPos)
    bool adaptive = false;
    double r_ad = 0.0, h_ad = 0.0, err_ad = 0.0;
    long long n_acc = 0, n_rej = 0;
    int ad_status = 1; // AD_DONE
};


} // namespace xfp

struct xf_ctx {
    std::vector<xfp::InstHost> in;
    int real_bytes = 8, precision = XF_FP64, stepper = XF_RK4, nfm = 2;
    int nmom = 2; // moments per stage: 2, or 4 when a problem has azimuth bins (extended bulb model)
    int form = XF_FORM_RHO; // what the state planes hold (one form per pack)
    bool cyl = false;       // the cylinder model's kernel (one problem)
    double cost3 = 17.0;    // cost weight of a three-flavor pair against a two-flavor one
    cudaStream_t stream = nullptr;
    xf_allocator alloc{};
    bool has_alloc = false;
    int device = 0, num_sms = 0;

    // one device arena; every problem owns a block of it (first-fit)
    unsigned char *arena = nullptr;
    xfp::Arena blocks;
    double *staging = nullptr;
    size_t staging_doubles = 0;
    bool dirty = false; // problems were added or removed since the last tiling
    std::vector<void *> owned;

    // tiling and launch shape
    xfp::RunKernel kern{nullptr, 0};
    std::vector<xfp::Tile> tiles;
    std::vector<int> cta_tiles;
    int G = 1, tile_pairs = 0, span_max = 1, max_tiles = 0;
    size_t smem = 0;
    xfp::Tile *tiles_d = nullptr;
    int *cta_tiles_d = nullptr;
    xfp::Inst *inst_d = nullptr;
    xfp::InstPos *pos_d = nullptr;
    xfp::AdaptPos *apos_d = nullptr, *tstate_d = nullptr; // error-controlled step only
    double *partials = nullptr, *mom_out = nullptr, *mom_part = nullptr, *mom_full = nullptr;
    int mom_part_slots = 0;
    size_t partials_doubles = 0; // cylinder model: size of the partials buffer
    unsigned *bar = nullptr;
    int *err = nullptr, *bad = nullptr;

    // options
    int grid_request = 0, tile_request = 0, skip_cta = -1, use_graph = 0;
    int stage_off = 0; // byte offset of the run kernel's staging columns in dynamic shared memory
    int dynamic_tiles = 0; // CTAs claim tiles per stage from a counter (when tiles outnumber CTAs)
    unsigned long long timeout_ns = 2000000000ull;

    // launches since the last sync; graph of one step launch, captured and
    // replayed on a private stream ordered after / before the ctx stream
    int pending = 0;
    cudaGraphExec_t graph = nullptr;
    long long graph_steps = 0;
    cudaStream_t gstream = nullptr;
    // asynchronous checkpoint: device copy, then a copy stream to the host
    cudaStream_t ck_stream = nullptr;
    cudaEvent_t ck_event = nullptr;
    unsigned char *ck_buf = nullptr;
    size_t ck_bytes = 0;
    bool ck_pending = false;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;

    std::string last_error;
};

namespace xfp {

int fail(xf_ctx *c, int code, const char *fmt, ...);
int cuda_fail(xf_ctx *c, cudaError_t e, const char *what);
int validate(xf_ctx *c, const xf_params *p, int n_E, int n_u, int nf);
int plan_launch(xf_ctx *c);
int upload_instances(xf_ctx *c);
int sync_status(xf_ctx *c);
double radius(const InstHost &h);
int enqueue_requests(xf_ctx *c, long long n, const std::vector<long long> &req);
int create_pack(int n, const xf_problem *probs, const xf_allocator *alloc, xf_ctx **out);
int create_slots(int n_slots, long long arena_bytes, int stepper, int precision, int nfm, xf_ctx **out);
long long block_bytes(int n_E, int n_u, int nf, int precision, int form = XF_FORM_RHO);
// The density matrices of problem i's current state: its state plane (rho
// form), or (psi form) rho = sum_a phi_a psi_a psi_a^+ written into its stage
// plane and trace array on the ctx stream.  Element offset from the arena base.
long long rho_plane(xf_ctx *c, InstHost &h, int *rc);
int add_problem(xf_ctx *c, const xf_problem &prob, const double *rho, double r_km, double dr_km, int *slot);
int remove_problem(xf_ctx *c, int slot);
int set_state_impl(xf_ctx *c, int i, const double *rho, size_t n_doubles, double r_km);
int init_state_impl(xf_ctx *c, int i, double r_km);
int get_state_impl(xf_ctx *c, int i, double *rho, size_t n_doubles, double *r_km, int64_t *steps_done);
void destroy_pack(xf_ctx *c);
int moments_impl(xf_ctx *c, int i, double *M0, double *M1, size_t n_doubles);
int moments_all(xf_ctx *c, int i, double *M);
InstHost *instance(xf_ctx *c, int i);
xf::LayoutArgs layout_args(xf_ctx *c, const InstHost &in);
int elementwise_grid(xf_ctx *c, const InstHost &in);
void *dev_alloc(xf_ctx *c, size_t bytes);
void dev_free(xf_ctx *c, void *p);
int upload_instances(xf_ctx *c);
__global__ void set_apos_kernel(AdaptPos *apos, int i, AdaptPos v);
__global__ void set_pos_kernel(InstPos *pos, int i, InstPos v);

// Run f(std::integral_constant<int, NF>, (Real *)nullptr) for the problem's
// flavor count and the context's working precision.
template <typename F>
int dispatch_layout(xf_ctx *c, const InstHost &in, F &&f)
{
    if (in.nf == 2) {
        if (c->real_bytes == 8) return f(std::integral_constant<int, 2>(), (double *)nullptr);
        return f(std::integral_constant<int, 2>(), (float *)nullptr);
    }
    if (c->real_bytes == 8) return f(std::integral_constant<int, 3>(), (double *)nullptr);
    return f(std::integral_constant<int, 3>(), (float *)nullptr);
}

} // namespace xfp
