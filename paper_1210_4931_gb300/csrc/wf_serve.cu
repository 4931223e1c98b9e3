// Serving engine: many HEALPix Wiener-filter, fluctuation and constrained-
// realization solves of mixed size on one GPU (the request loop declared at
// the end of wf.h).
//
// Design:
//   * `slots` worker threads, each with its own non-blocking CUDA stream; a
//     worker runs one solve at a time through the host-buffer entry points,
//     so the solves of different workers overlap on the device;
//   * a pool of plans keyed by (nside, lmax, precision, ncomp): a plan holds the
//     geometry's Legendre and ring tables and the workspace, and is reused by
//     later requests of the same key (a key's tables are built once for each
//     of its solves that run at the same time, not once per request);
//   * admission by device memory: the device bytes of all pooled plans stay
//     within the budget (a new plan is counted at its estimate, then at its
//     measured size); the queue head may evict idle plans, least recently used
//     first; requests behind the head are admitted only into free memory, so
//     a large request at the head is never overtaken into memory it needs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "wf_internal.cuh"

namespace {

struct PooledPlan {
    wf_plan p = nullptr;
    int nside = 0, lmax = 0, ncomp = 1;
    wf_precision prec = WF_PREC_FP64;
    long long bytes = 0;
    bool busy = false;
    double last_used = 0;
};

struct Pending {
    wf_request r;
    double t_submit;
};

struct Admit {
    bool ok = false;
    size_t idx = 0;
    PooledPlan *pp = nullptr;          // idle plan of the request's key, or
    long long reserve = 0;             // bytes reserved for a new plan
    std::vector<PooledPlan *> evict;   // idle plans to destroy first
};

int ncomp_of(const wf_request &r) { return r.ncomp == 3 ? 3 : 1; }

long long request_bytes(const wf_request &r)
{
    wf_geometry g{};
    g.kind = WF_GEOM_HEALPIX;
    g.nside = r.nside;
    g.ncomp = ncomp_of(r);
    long long b = wf_plan_estimate_bytes(&g, r.lmax, r.precision, 1);
    if (b < 0) return b;
    // FP64 sub-plan of the correction sweeps and of the correction form's FP64 step
    if (r.precision != WF_PREC_FP64 && (r.opt.refine_sweeps > 0 || r.opt.mixed_correction > 0.0))
        b += wf_plan_estimate_bytes(&g, r.lmax, WF_PREC_FP64, 0);
    // the correction form's buffers: x0, d0 and delta - d0 (a_lm, FP64) and a zero FP32 source map
    if (r.precision != WF_PREC_FP64 && r.opt.mixed_correction > 0.0 && g.ncomp == 1) {
        const long long nalm = (long long)(r.lmax + 1) * (r.lmax + 2) / 2;
        b += 3 * nalm * 16 + 12LL * r.nside * r.nside * 4;
    }
    return b;
}

// An idle pooled plan has no queued work (the host-buffer entry points wait
// for their stream before returning), so it can be rebound to another stream
// without waiting on the stream of the worker that used it last.
void bind_stream(wf_plan p, cudaStream_t st)
{
    for (; p; p = p->sub) p->stream = st;
}

const char *request_error(const wf_request &r)
{
    if (r.kind < WF_REQ_WF || r.kind > WF_REQ_CR) return "unknown request kind";
    if (r.nside < 1 || r.lmax < 2 || r.lmax > 2 * r.nside) return "need 2 <= lmax <= 2 nside";
    if (r.precision != WF_PREC_FP64 && r.precision != WF_PREC_MIXED_FP32 && !wf::tc_prec(r.precision))
        return "unknown precision";
    if (r.ncomp != 0 && r.ncomp != 1 && r.ncomp != 3) return "ncomp must be 0, 1 or 3";
    if (!(r.tol > 0)) return "tol must be > 0";
    if (!r.noise_var || !r.C_ell || !r.s_out) return "noise_var, C_ell and s_out are required";
    if (r.kind != WF_REQ_FLUCT && !r.d) return "d is required";
    if (r.kind != WF_REQ_WF && (!r.g1 || !r.g2)) return "g1 and g2 are required";
    return nullptr;
}

}  // namespace

struct wf_server_s {
    int device = 0;
    long long budget = 0;
    int nslots = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> pending;
    std::vector<PooledPlan *> pool;
    std::deque<wf_result> done;
    std::vector<std::thread> workers;
    bool stop = false;
    long long bytes_in_use = 0, peak = 0, completed = 0, rejected = 0, created = 0, evicted = 0;
    int active = 0, max_active = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // under mu
    Admit try_admit()
    {
        Admit a;
        const size_t look = std::min<size_t>(pending.size(), 32);
        for (size_t i = 0; i < look; ++i) {
            const wf_request &r = pending[i].r;
            for (PooledPlan *pp : pool)
                if (!pp->busy && pp->nside == r.nside && pp->lmax == r.lmax && pp->prec == r.precision &&
                    pp->ncomp == ncomp_of(r)) {
                    a.ok = true;
                    a.idx = i;
                    a.pp = pp;
                    return a;
                }
            const long long est = request_bytes(r);
            if (bytes_in_use + est <= budget) {
                a.ok = true;
                a.idx = i;
                a.reserve = est;
                return a;
            }
            if (i == 0) {  // the head may evict idle plans, least recently used first
                std::vector<PooledPlan *> idle;
                for (PooledPlan *pp : pool)
                    if (!pp->busy) idle.push_back(pp);
                std::sort(idle.begin(), idle.end(),
                          [](const PooledPlan *x, const PooledPlan *y) { return x->last_used < y->last_used; });
                long long freed = 0;
                std::vector<PooledPlan *> ev;
                for (PooledPlan *pp : idle) {
                    if (bytes_in_use - freed + est <= budget) break;
                    ev.push_back(pp);
                    freed += pp->bytes;
                }
                if (bytes_in_use - freed + est <= budget) {
                    a.ok = true;
                    a.idx = 0;
                    a.reserve = est;
                    a.evict = std::move(ev);
                    return a;
                }
            }
        }
        return a;
    }

    void finish(const wf_result &res)  // under mu
    {
        done.push_back(res);
        ++completed;
        cv_done.notify_all();
    }

    void worker(int slot);
};

namespace {

// one request on a plan that is bound to this worker's stream
void run_request(wf_plan p, const wf_request &r, wf_result &res)
{
    wf_set_options(p, &r.opt);
    wf_info info{};
    const long long nmap = wf_npix(p) * ncomp_of(r);  // values per map argument
    if (r.kind == WF_REQ_WF) {
        res.status = wf_solve_host(p, r.d, r.noise_var, r.mask, r.C_ell, r.tol, r.s_out, nullptr, &info);
        res.iters = info.iters;
        res.converged = info.converged;
        res.final_residual = info.final_residual;
        res.chi2_over_ndof = info.chi2_over_ndof;
        return;
    }
    if (r.kind == WF_REQ_FLUCT) {
        res.status = wf_fluct_host(p, r.noise_var, r.mask, r.C_ell, r.g1, r.g2, r.tol, r.s_out, nullptr, &info);
        res.iters = info.iters;
        res.converged = info.converged;
        res.final_residual = info.final_residual;
        res.chi2_over_ndof = NAN;
        return;
    }
    // constrained realization (Sect. 2.3): s_WF + f
    wf_status s1 = wf_solve_host(p, r.d, r.noise_var, r.mask, r.C_ell, r.tol, r.s_out, nullptr, &info);
    res.iters = info.iters;
    res.converged = info.converged;
    res.final_residual = info.final_residual;
    res.chi2_over_ndof = info.chi2_over_ndof;
    if (s1 != WF_OK && s1 != WF_ENOCONV) {
        res.status = s1;
        return;
    }
    std::vector<double> tmp;
    double *f = r.f_out;
    if (!f) {
        tmp.resize((size_t)nmap);
        f = tmp.data();
    }
    wf_info fi{};
    wf_status s2 = wf_fluct_host(p, r.noise_var, r.mask, r.C_ell, r.g1, r.g2, r.tol, f, nullptr, &fi);
    res.iters += fi.iters;
    res.converged = res.converged && fi.converged;
    res.final_residual = std::max(res.final_residual, fi.final_residual);
    if (s2 != WF_OK && s2 != WF_ENOCONV) {
        res.status = s2;
        return;
    }
    for (long long i = 0; i < nmap; ++i) r.s_out[i] += f[i];
    res.status = (s1 == WF_OK && s2 == WF_OK) ? WF_OK : WF_ENOCONV;
}

}  // namespace

void wf_server_s::worker(int slot)
{
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        Admit ad;
        cv_work.wait(lk, [&] {
            if (stop) return true;
            ad = try_admit();
            return ad.ok;
        });
        if (stop) break;
        const Pending job = pending[ad.idx];
        pending.erase(pending.begin() + (long)ad.idx);
        PooledPlan *pp = ad.pp;
        const bool reused = pp != nullptr;
        if (pp) {
            pp->busy = true;
        } else {
            for (PooledPlan *e : ad.evict) {
                pool.erase(std::find(pool.begin(), pool.end(), e));
                bytes_in_use -= e->bytes;
                ++evicted;
            }
            bytes_in_use += ad.reserve;
            peak = std::max(peak, bytes_in_use);
        }
        ++active;
        max_active = std::max(max_active, active);
        wf_result res{};
        res.tag = job.r.tag;
        res.t_submit = job.t_submit;
        res.t_start = now();
        res.slot = slot;
        res.plan_reused = reused ? 1 : 0;
        lk.unlock();

        for (PooledPlan *e : ad.evict) {
            bind_stream(e->p, st);
            wf_plan_destroy(e->p);
            delete e;
        }
        wf_status cs = WF_OK;
        if (!pp) {
            wf_geometry g{};
            g.kind = WF_GEOM_HEALPIX;
            g.nside = job.r.nside;
            g.ncomp = ncomp_of(job.r);
            wf_plan p = nullptr;
            cs = wf_plan_create(&g, job.r.lmax, job.r.precision, (void *)st, &p);
            if (cs == WF_OK) {
                pp = new PooledPlan();
                pp->p = p;
                pp->nside = job.r.nside;
                pp->lmax = job.r.lmax;
                pp->ncomp = ncomp_of(job.r);
                pp->prec = job.r.precision;
                pp->bytes = ad.reserve;
                pp->busy = true;
            }
        } else {
            bind_stream(pp->p, st);
        }
        if (cs == WF_OK) run_request(pp->p, job.r, res);
        else res.status = cs;
        const long long nb = pp ? wf_plan_device_bytes(pp->p) : 0;
        res.t_done = now();

        lk.lock();
        if (pp) {
            if (!reused) {
                pool.push_back(pp);
                ++created;
            }
            bytes_in_use += nb - pp->bytes;  // measured size replaces the estimate
            pp->bytes = nb;
            peak = std::max(peak, bytes_in_use);
            pp->busy = false;
            pp->last_used = now();
        } else {
            bytes_in_use -= ad.reserve;
        }
        --active;
        finish(res);
        cv_work.notify_all();
    }
    lk.unlock();
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

extern "C" {

wf_status wf_server_create(int device, long long mem_budget, int slots, wf_server *out)
{
    if (!out) return wf::set_error(WF_EINVAL, "null argument");
    *out = nullptr;
    if (slots < 1 || slots > 64) return wf::set_error(WF_EINVAL, "slots must be in [1, 64]");
    if (mem_budget <= 0) return wf::set_error(WF_EINVAL, "mem_budget must be > 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return wf::set_error(WF_EINVAL, "no CUDA device %d", device);
    wf_server s = new (std::nothrow) wf_server_s();
    if (!s) return wf::set_error(WF_ENOMEM, "host allocation");
    s->device = device;
    s->budget = mem_budget;
    s->nslots = slots;
    for (int i = 0; i < slots; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
    *out = s;
    return WF_OK;
}

wf_status wf_server_submit(wf_server s, const wf_request *req)
{
    if (!s || !req) return wf::set_error(WF_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = s->now();
    const char *why = request_error(*req);
    wf_status bad = WF_OK;
    if (why) bad = wf::set_error(WF_EINVAL, "request %llu: %s", (unsigned long long)req->tag, why);
    else if (request_bytes(*req) > s->budget)
        bad = wf::set_error(WF_ENOMEM, "request %llu needs ~%lld device bytes, over the budget", (unsigned long long)req->tag,
                            request_bytes(*req));
    if (bad != WF_OK) {
        wf_result res{};
        res.tag = req->tag;
        res.status = bad;
        res.t_submit = res.t_start = res.t_done = t;
        res.slot = -1;
        ++s->rejected;
        s->finish(res);
        return WF_OK;
    }
    s->pending.push_back(Pending{*req, t});
    s->cv_work.notify_one();
    return WF_OK;
}

int wf_server_poll(wf_server s, wf_result *out, int cap)
{
    if (!s || !out || cap <= 0) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < cap && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

int wf_server_wait(wf_server s, wf_result *out, int cap, double timeout_s)
{
    if (!s || !out || cap <= 0) return 0;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)), [&] { return !s->done.empty(); });
    int n = 0;
    while (n < cap && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

wf_status wf_server_get_stats(wf_server s, wf_server_stats *st)
{
    if (!s || !st) return wf::set_error(WF_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    st->pending = (long long)s->pending.size();
    st->active = s->active;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->bytes_in_use = s->bytes_in_use;
    st->peak_bytes = s->peak;
    st->budget = s->budget;
    st->plans = (int)s->pool.size();
    st->max_active = s->max_active;
    st->plans_created = s->created;
    st->plans_evicted = s->evicted;
    return WF_OK;
}

void wf_server_destroy(wf_server s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->pending.clear();
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    cudaSetDevice(s->device);
    for (PooledPlan *pp : s->pool) {
        bind_stream(pp->p, nullptr);  // the workers' streams are gone
        wf_plan_destroy(pp->p);
        delete pp;
    }
    delete s;
}

}  // extern "C"
