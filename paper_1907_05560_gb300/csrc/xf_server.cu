// xf_server.cu -- continuous-batching job server over a pack of slots.
//
// A scheduler thread repeats epochs: admit queued jobs into free slots while
// their blocks fit the memory budget, advance all resident jobs together in
// one persistent launch of up to chunk_steps radial steps (each job takes
// min(remaining, chunk_steps)), then retire the finished ones.  Submission
// and polling only touch the host-side queue and result records.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/xf.h"
#include "xf_pack.h"

using namespace xfp;
using xf::ERR_NONFINITE;

namespace {

struct Job {
    xf_job spec{};
    std::vector<double> rho0, result;
    long long bytes = 0;
    int slot = -1;
    bool done = false;
    xf_job_result res{};
};

} // namespace

struct xf_server {
    xf_server_cfg cfg{};
    int device = 0;
    xf_ctx *pack = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Job> jobs;
    std::vector<uint64_t> slot_job; // slot -> job id (0: free)
    uint64_t next_id = 1;
    bool stop = false;
    xf_server_stats st{};
    std::chrono::steady_clock::time_point t0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Admit queued jobs while a slot is free and the budget allows (called with
// the lock held; drops it around device work).
void admit(xf_server *s, std::unique_lock<std::mutex> &lk)
{
    while (!s->queue.empty() && s->st.resident < s->cfg.max_jobs) {
        const uint64_t id = s->queue.front();
        Job &j = s->jobs[id];
        if (s->st.mem_used_bytes + j.bytes > s->cfg.mem_budget_bytes) break;
        s->queue.pop_front();
        s->st.queued = (int64_t)s->queue.size();
        const xf_job spec = j.spec;
        const std::vector<double> rho0 = j.rho0;
        lk.unlock();
        int slot = -1;
        int rc = add_problem(s->pack, spec.problem, rho0.empty() ? nullptr : rho0.data(), spec.r0_km, spec.dr_km,
                             &slot);
        lk.lock();
        Job &jj = s->jobs[id];
        if (rc == XF_E_BUSY) { // arena fragmentation: retry after a retirement
            s->queue.push_front(id);
            s->st.queued = (int64_t)s->queue.size();
            break;
        }
        jj.res.t_start = s->now();
        if (rc) {
            jj.done = true;
            jj.res.status = rc;
            jj.res.t_done = jj.res.t_start;
            ++s->st.completed;
            s->cv_done.notify_all();
            continue;
        }
        jj.slot = slot;
        s->slot_job[slot] = id;
        ++s->st.resident;
        s->st.max_resident = std::max(s->st.max_resident, s->st.resident);
        s->st.mem_used_bytes += jj.bytes;
        s->st.mem_peak_bytes = std::max(s->st.mem_peak_bytes, s->st.mem_used_bytes);
    }
}

void scheduler(xf_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    const long long K = s->cfg.chunk_steps;
    while (!s->stop) {
        s->cv.wait(lk, [&] { return s->stop || !s->queue.empty() || s->st.resident > 0; });
        if (s->stop) break;
        admit(s, lk);
        if (s->st.resident == 0) continue;

        // one launch: every resident job takes min(remaining, K) steps
        xf_ctx *c = s->pack;
        std::vector<long long> req(c->in.size(), 0), before(c->in.size(), 0);
        long long n_launch = 0;
        double bins_steps = 0.0;
        for (size_t i = 0; i < c->in.size(); ++i) before[i] = c->in[i].steps;
        for (size_t i = 0; i < c->in.size(); ++i) {
            const uint64_t id = s->slot_job[i];
            if (!id) continue;
            const Job &j = s->jobs[id];
            const long long left = j.spec.n_steps - c->in[i].steps;
            req[i] = std::max(0ll, std::min(left, K));
            n_launch = std::max(n_launch, req[i]);
        }
        lk.unlock();
        const double t_start = s->now();
        int rc = XF_OK;
        if (n_launch > 0) {
            rc = enqueue_requests(c, n_launch, req);
            if (!rc) rc = sync_status(c);
        }
        const double t_end = s->now();
        lk.lock();
        s->st.busy_s += t_end - t_start;
        ++s->st.epochs;

        // retire finished (or failed) jobs
        for (size_t i = 0; i < c->in.size(); ++i) {
            const uint64_t id = s->slot_job[i];
            if (!id) continue;
            Job &j = s->jobs[id];
            InstHost &h = c->in[i];
            bins_steps += (double)h.n_bins * (double)(h.steps - before[i]);
            const bool failed = rc != XF_OK || (h.err & ERR_NONFINITE);
            if (h.steps < j.spec.n_steps && !failed) continue;
            j.res.status = rc != XF_OK ? rc : (h.err & ERR_NONFINITE) ? XF_E_NONFINITE : XF_OK;
            j.res.steps_done = h.steps;
            j.res.r_km = radius(h);
            if (j.spec.keep_state && rc == XF_OK) {
                j.result.resize((size_t)h.n_bins * h.nf * h.nf);
                lk.unlock();
                int64_t n = 0;
                double r = 0;
                get_state_impl(c, (int)i, j.result.data(), j.result.size(), &r, &n);
                lk.lock();
            }
            remove_problem(c, (int)i);
            s->slot_job[i] = 0;
            s->st.mem_used_bytes -= j.bytes;
            --s->st.resident;
            ++s->st.completed;
            j.res.t_done = s->now();
            j.done = true;
        }
        s->st.bin_steps += bins_steps;
        s->cv_done.notify_all();
    }
}

} // namespace

extern "C" {

int xf_server_create(const xf_server_cfg *cfg, xf_server **out)
{
    if (!out) return XF_E_ARG;
    *out = nullptr;
    if (!cfg || cfg->size != sizeof(xf_server_cfg)) return XF_E_ARG;
    if (cfg->max_jobs < 1 || cfg->mem_budget_bytes <= 0 || cfg->chunk_steps < 1 || cfg->queue_cap < 1)
        return XF_E_ARG;
    if (cfg->stepper == XF_EXPH_ADAPTIVE) return XF_E_UNSUPPORTED; // jobs advance in fixed chunks of steps
    if (cfg->stepper != XF_RK4 && cfg->stepper != XF_EXPH) return XF_E_ARG;
    if (cfg->precision < XF_FP64 || cfg->precision > XF_FP32X2) return XF_E_ARG;
    if (cfg->n_flavor != 0 && cfg->n_flavor != 2 && cfg->n_flavor != 3) return XF_E_ARG;
    if (cfg->tile_pairs < 0) return XF_E_ARG;
    xf_server *s = new (std::nothrow) xf_server();
    if (!s) return XF_E_NOMEM;
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return XF_E_CUDA;
    }
    int rc = create_slots(cfg->max_jobs, cfg->mem_budget_bytes, cfg->stepper, cfg->precision, cfg->n_flavor, &s->pack);
    if (rc) {
        delete s;
        return rc;
    }
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess) s->pack->stream = stream;
    s->pack->tile_request = cfg->tile_pairs > 0 ? cfg->tile_pairs : 1024;
    s->slot_job.assign(cfg->max_jobs, 0);
    s->th = std::thread(scheduler, s);
    *out = s;
    return XF_OK;
}

int xf_submit(xf_server *s, const xf_job *job, uint64_t *job_id)
{
    if (!s || !job || !job_id) return XF_E_ARG;
    const xf_problem &p = job->problem;
    if (validate(nullptr, &p.params, p.n_E, p.n_u, p.n_flavor)) return XF_E_ARG;
    if (p.params.n_phi != 1) return XF_E_UNSUPPORTED; // the server's packs run the bulb model's two moments
    if (p.params.form != XF_FORM_RHO) return XF_E_UNSUPPORTED; // the server's packs hold density matrices
    if (p.params.geometry == XF_GEOM_CYLINDER) return XF_E_UNSUPPORTED; // runs alone in its context
    if (p.params.stepper != s->cfg.stepper || p.params.precision != s->cfg.precision) return XF_E_ARG;
    if (s->cfg.n_flavor && p.n_flavor != s->cfg.n_flavor) return XF_E_ARG;
    if (!std::isfinite(job->r0_km) || job->r0_km < p.params.R_nu_km || !std::isfinite(job->dr_km) ||
        job->dr_km <= 0 || job->n_steps < 1)
        return XF_E_ARG;
    Job j;
    j.spec = *job;
    j.bytes = block_bytes(p.n_E, p.n_u, p.n_flavor, s->cfg.precision);
    if (j.bytes > s->cfg.mem_budget_bytes) return XF_E_TOO_BIG;
    if (job->rho0) {
        const size_t n = (size_t)2 * p.n_u * p.n_E * p.n_flavor * p.n_flavor;
        j.rho0.assign(job->rho0, job->rho0 + n);
    }
    j.spec.rho0 = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->queue.size() >= s->cfg.queue_cap) return XF_E_BUSY;
    const uint64_t id = s->next_id++;
    j.res.t_submit = s->now();
    s->jobs.emplace(id, std::move(j));
    s->queue.push_back(id);
    ++s->st.submitted;
    s->st.queued = (int64_t)s->queue.size();
    *job_id = id;
    s->cv.notify_all();
    return XF_OK;
}

int xf_poll(xf_server *s, uint64_t job_id, xf_job_result *res, double *rho_out, size_t n_doubles)
{
    if (!s) return XF_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return XF_E_NOTFOUND;
    Job &j = it->second;
    if (!j.done) return XF_PENDING;
    if (rho_out) {
        if (j.result.empty()) return XF_E_STATE;
        if (n_doubles != j.result.size()) return XF_E_ARG;
        std::memcpy(rho_out, j.result.data(), sizeof(double) * n_doubles);
    }
    if (res) *res = j.res;
    s->jobs.erase(it);
    return XF_OK;
}

int xf_server_drain(xf_server *s, double timeout_s)
{
    if (!s) return XF_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    // every submitted job finished (a job being admitted is neither queued nor
    // resident for a moment, so the counters are what tells)
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->st.completed == s->st.submitted; });
    return ok ? XF_OK : XF_E_TIMEOUT;
}

int xf_server_get_stats(xf_server *s, xf_server_stats *st)
{
    if (!s || !st) return XF_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    return XF_OK;
}

int xf_server_destroy(xf_server *s)
{
    if (!s) return XF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaStream_t stream = s->pack ? s->pack->stream : nullptr;
    destroy_pack(s->pack);
    if (stream) cudaStreamDestroy(stream);
    delete s;
    return XF_OK;
}

} // extern "C"
