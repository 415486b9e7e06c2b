// xf_ckpt.cu -- checkpoints (the paper's dump mode 1 and resume, Sec. 4.2.4)
// and the per-trajectory energy average (dump mode 2).
//
// A checkpoint holds the problem's current state planes in the working
// precision (density matrices, or the wavefunctions of the psi form), its
// FP64 trace per bin, the renormalising variant's reference
// values, and the position (radius, step size, step counts, error-controlled
// progress), behind a header that ties it to the problem's shape, stepper and
// precision.  Loading it puts the state into plane 0 and restores the
// position, so the next step is bitwise the one that would have followed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "../../include/xf.h"
#include "xf_pack.h"

using namespace xfp;

namespace {

constexpr uint32_t kMagic = 0x4b434658u; // "XFCK"
constexpr uint32_t kVersion = 1u;

struct CkptHeader {
    uint32_t magic, version;
    int32_t n_E, n_u, n_f, real_bytes, stepper, precision;
    int64_t npad, plane_bytes, trace_bytes, ref_bytes;
    double r0, h;
    int64_t k0, steps;
    int32_t err, adaptive;
    double r_ad, h_ad, err_ad;
    int64_t n_acc, n_rej;
    int32_t ad_status, form;
};

struct Layout {
    size_t plane, trace, ref, total;
};

Layout layout_of(const xf_ctx *c, const InstHost &h)
{
    Layout L;
    L.plane = (size_t)2 * h.SS * h.npad * c->real_bytes;
    L.trace = (size_t)2 * h.npad * sizeof(double);
    L.ref = c->precision == XF_FP32_M64_RENORM ? (size_t)2 * h.npad * c->real_bytes : 0;
    L.total = sizeof(CkptHeader) + L.plane + L.trace + L.ref;
    return L;
}

CkptHeader header_of(const xf_ctx *c, const InstHost &h, const Layout &L)
{
    CkptHeader H;
    std::memset(&H, 0, sizeof H);
    H.magic = kMagic;
    H.version = kVersion;
    H.n_E = h.n_E;
    H.n_u = h.n_u;
    H.n_f = h.nf;
    H.real_bytes = c->real_bytes;
    H.stepper = c->stepper;
    H.precision = c->precision;
    H.npad = h.npad;
    H.plane_bytes = (int64_t)L.plane;
    H.trace_bytes = (int64_t)L.trace;
    H.ref_bytes = (int64_t)L.ref;
    H.r0 = h.r0;
    H.h = h.h;
    H.k0 = h.k0;
    H.steps = h.steps;
    H.err = h.err;
    H.adaptive = h.adaptive ? 1 : 0;
    H.r_ad = h.r_ad;
    H.h_ad = h.h_ad;
    H.err_ad = h.err_ad;
    H.n_acc = h.n_acc;
    H.n_rej = h.n_rej;
    H.ad_status = h.ad_status;
    H.form = c->form;
    return H;
}

// The problem, synchronised and with a valid state; its layout.
int prepare(xf_ctx *c, int inst, InstHost **hp, Layout *L)
{
    InstHost *h = instance(c, inst);
    if (!h) return c ? fail(c, XF_E_ARG, "bad instance index %d", inst) : XF_E_ARG;
    if (!h->active) return fail(c, XF_E_ARG, "slot %d holds no problem", inst);
    if (c->pending) {
        int rc = sync_status(c);
        if (rc) return rc;
    }
    *hp = h;
    *L = layout_of(c, *h);
    return XF_OK;
}

// Enqueue the device-to-`dst` copies of the payload (dst: host or device).
int copy_payload(xf_ctx *c, const InstHost &h, const Layout &L, unsigned char *dst, cudaStream_t stream,
                 cudaMemcpyKind kind)
{
    const unsigned char *plane = c->arena + (size_t)h.off[h.cur] * c->real_bytes;
    const unsigned char *trace = c->arena + (size_t)h.trace_off * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(dst, plane, L.plane, kind, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + L.plane, trace, L.trace, kind, stream);
    if (e == cudaSuccess && L.ref)
        e = cudaMemcpyAsync(dst + L.plane + L.trace, c->arena + (size_t)h.ref_off * c->real_bytes, L.ref, kind,
                            stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
    return XF_OK;
}

} // namespace

extern "C" {

int xf_checkpoint_bytes(xf_ctx *c, int inst, size_t *bytes)
{
    if (!c || !bytes) return XF_E_ARG;
    InstHost *h = instance(c, inst);
    if (!h || !h->active) return fail(c, XF_E_ARG, "bad instance index %d", inst);
    *bytes = layout_of(c, *h).total;
    return XF_OK;
}

int xf_checkpoint_save(xf_ctx *c, int inst, void *buf, size_t bytes)
{
    if (!c || !buf) return XF_E_ARG;
    InstHost *h;
    Layout L;
    int rc = prepare(c, inst, &h, &L);
    if (rc) return rc;
    if (bytes != L.total) return fail(c, XF_E_ARG, "checkpoint needs %zu bytes (got %zu)", L.total, bytes);
    if (!h->state_valid) return fail(c, XF_E_STATE, "no valid state");
    const CkptHeader H = header_of(c, *h, L);
    std::memcpy(buf, &H, sizeof H);
    rc = copy_payload(c, *h, L, (unsigned char *)buf + sizeof H, c->stream, cudaMemcpyDeviceToHost);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    return XF_OK;
}

int xf_checkpoint_save_async(xf_ctx *c, int inst, void *buf, size_t bytes)
{
    if (!c || !buf) return XF_E_ARG;
    if (c->ck_pending) return fail(c, XF_E_BUSY, "a checkpoint copy is in flight (xf_checkpoint_wait)");
    InstHost *h;
    Layout L;
    int rc = prepare(c, inst, &h, &L);
    if (rc) return rc;
    if (bytes != L.total) return fail(c, XF_E_ARG, "checkpoint needs %zu bytes (got %zu)", L.total, bytes);
    if (!h->state_valid) return fail(c, XF_E_STATE, "no valid state");
    if (!c->ck_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->ck_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ck_event, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint stream");
    }
    const size_t payload = L.total - sizeof(CkptHeader);
    if (payload > c->ck_bytes) {
        if (c->ck_buf) dev_free(c, c->ck_buf);
        c->ck_buf = (unsigned char *)dev_alloc(c, payload);
        c->ck_bytes = c->ck_buf ? payload : 0;
        if (!c->ck_buf) return fail(c, XF_E_NOMEM, "device allocation of the checkpoint buffer failed");
    }
    const CkptHeader H = header_of(c, *h, L);
    std::memcpy(buf, &H, sizeof H);
    // device copy in stream order (steps enqueued later overwrite other planes
    // only after it), then the host copy on the copy stream
    rc = copy_payload(c, *h, L, c->ck_buf, c->stream, cudaMemcpyDeviceToDevice);
    if (rc) return rc;
    cudaError_t e = cudaEventRecord(c->ck_event, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->ck_stream, c->ck_event, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((unsigned char *)buf + sizeof H, c->ck_buf, payload, cudaMemcpyDeviceToHost, c->ck_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
    c->ck_pending = true;
    return XF_OK;
}

int xf_checkpoint_wait(xf_ctx *c)
{
    if (!c) return XF_E_ARG;
    if (!c->ck_pending) return XF_OK;
    c->ck_pending = false;
    cudaError_t e = cudaStreamSynchronize(c->ck_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
    return XF_OK;
}

int xf_checkpoint_load(xf_ctx *c, int inst, const void *buf, size_t bytes)
{
    if (!c || !buf) return XF_E_ARG;
    InstHost *h;
    Layout L;
    int rc = prepare(c, inst, &h, &L);
    if (rc) return rc;
    if (bytes != L.total) return fail(c, XF_E_ARG, "checkpoint of %zu bytes, this problem needs %zu", bytes, L.total);
    CkptHeader H;
    std::memcpy(&H, buf, sizeof H);
    if (H.magic != kMagic || H.version != kVersion) return fail(c, XF_E_ARG, "not a checkpoint of this library");
    if (H.n_E != h->n_E || H.n_u != h->n_u || H.n_f != h->nf || H.real_bytes != c->real_bytes ||
        H.stepper != c->stepper || H.precision != c->precision || H.form != c->form || H.npad != h->npad ||
        H.plane_bytes != (int64_t)L.plane || H.trace_bytes != (int64_t)L.trace || H.ref_bytes != (int64_t)L.ref)
        return fail(c, XF_E_ARG, "checkpoint of another problem shape, stepper, precision or form");
    const unsigned char *src = (const unsigned char *)buf + sizeof H;
    // the state goes to plane 0
    cudaError_t e = cudaMemcpyAsync(c->arena + (size_t)h->off[0] * c->real_bytes, src, L.plane,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->arena + (size_t)h->trace_off * sizeof(double), src + L.plane, L.trace,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && L.ref)
        e = cudaMemcpyAsync(c->arena + (size_t)h->ref_off * c->real_bytes, src + L.plane + L.trace, L.ref,
                            cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
    h->r0 = H.r0;
    h->h = H.h;
    h->k0 = H.k0;
    h->steps = H.steps;
    h->err = H.err;
    h->cur = 0;
    h->state_valid = true;
    InstPos ps;
    std::memset(&ps, 0, sizeof ps);
    ps.k0 = H.k0;
    ps.steps = (unsigned long long)H.steps;
    ps.cur = 0;
    ps.err = H.err;
    set_pos_kernel<<<1, 1, 0, c->stream>>>(c->pos_d, inst, ps);
    if (c->stepper == XF_EXPH_ADAPTIVE) {
        h->adaptive = true;
        h->r_ad = H.r_ad;
        h->h_ad = H.h_ad;
        h->err_ad = H.err_ad;
        h->n_acc = H.n_acc;
        h->n_rej = H.n_rej;
        h->ad_status = H.ad_status == xf::AD_RUN ? xf::AD_DONE : H.ad_status;
        AdaptPos a;
        std::memset(&a, 0, sizeof a);
        a.r = a.r_end = h->r_ad;
        a.h = h->h_ad;
        a.err = h->err_ad;
        a.n_acc = h->n_acc;
        a.n_rej = h->n_rej;
        a.status = h->ad_status;
        set_apos_kernel<<<1, 1, 0, c->stream>>>(c->apos_d, inst, a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "position kernel");
    rc = upload_instances(c);
    if (rc) return rc;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    return XF_OK;
}

int xf_angle_average(xf_ctx *c, int inst, double *out, size_t n_doubles)
{
    if (!c || !out) return XF_E_ARG;
    InstHost *h;
    Layout L;
    int rc = prepare(c, inst, &h, &L);
    if (rc) return rc;
    if (!h->state_valid) return fail(c, XF_E_STATE, "no valid state");
    const size_t n_traj = (size_t)h->n_u * h->n_phi;
    const size_t need = 2 * n_traj * h->nf * h->nf;
    if (n_doubles != need) return fail(c, XF_E_ARG, "n_doubles %zu != %zu", n_doubles, need);
    const long long plane = rho_plane(c, *h, &rc);
    if (rc) return rc;
    xf::LayoutArgs la = layout_args(c, *h);
    rc = dispatch_layout(c, *h, [&](auto nfc, auto *realp) {
        constexpr int NF = decltype(nfc)::value;
        using Real = std::remove_pointer_t<decltype(realp)>;
        xf::angle_average_kernel<NF, Real, 128><<<(unsigned)(2 * n_traj), 128, 0, c->stream>>>(
            la, (const Real *)c->arena + plane, (const double *)c->arena + h->trace_off, c->staging);
        return (int)cudaGetLastError();
    });
    if (rc) return cuda_fail(c, (cudaError_t)rc, "average kernel");
    cudaError_t e = cudaMemcpyAsync(out, c->staging, sizeof(double) * need, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy average");
    return XF_OK;
}

} // extern "C"
