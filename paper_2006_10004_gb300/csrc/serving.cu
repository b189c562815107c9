// Serving: continuous batching of single-image decompositions at ROF-step boundaries.
//
// A scheduler thread owns the device work of served requests. Each tick it
//   1. retires cancelled requests,
//   2. admits waiting requests (FIFO) while their workspace fits the memory budget and the
//      number of resident requests stays below max_batch, uploads their images and starts
//      them (u_0 = f) at the current global step,
//   3. runs one ROF step (all dual iterations + the epilogue) for every resident request in
//      one set of launches over the tiles of all of them,
//   4. copies out the requests that just finished their K-th step and frees their workspace.
// Requests therefore join and leave while others are mid-flight; each request's arithmetic
// is the same as when it runs alone (tiling-invariant dual iterations, per-image reductions
// in a fixed order), so its results are bit-identical.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "runtime.h"

namespace tvspec {

using Clock = std::chrono::steady_clock;

struct ServeReq {
    uint64_t ticket = 0;
    Job job;
    int state = 0;  // 0 queued, 1 running, 2 finished (result below)
    bool cancel = false;
    tvspec_status result = TVSPEC_ENOTREADY;
    Clock::time_point t_submit, t_done;
    Slot slot;
    int s0 = 0;
    size_t bytes = 0;
};

struct Server {
    tvspec_plan *plan = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<ServeReq>> waiting;
    std::vector<std::shared_ptr<ServeReq>> active;  // scheduler thread only
    std::map<uint64_t, std::shared_ptr<ServeReq>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t used = 0;
    std::vector<double> lat_ms;
    cudaStream_t st = nullptr;
    LaunchSet ls, init_ls;
    int gstep = 0;
    int shape = -2, depth = 1;
    void loop();
};

static void finish(Server *S, const std::shared_ptr<ServeReq> &r, tvspec_status result) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->result = result;
    r->state = 2;
    r->t_done = Clock::now();
    if (result == TVSPEC_OK)
        S->lat_ms.push_back(
            std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    S->cv_done.notify_all();
}

// Copies the outputs of a request that finished on the device to its host buffers.
static tvspec_status copy_out(Server *S, ServeReq &r) {
    const tvspec_request &q = r.job.r;
    const size_t N = (size_t)q.H * q.W;
    TV_CK(cudaMemcpyAsync(q.bands, r.slot.bands, (size_t)r.slot.n_bands * N * 4, cudaMemcpyDeviceToHost, S->st));
    TV_CK(cudaMemcpyAsync(q.residual, r.slot.residual, N * 4, cudaMemcpyDeviceToHost, S->st));
    TV_CK(cudaMemcpyAsync(q.S, r.slot.S, (size_t)(q.K - 1) * 8, cudaMemcpyDeviceToHost, S->st));
    if (q.u_trace)
        TV_CK(cudaMemcpyAsync(q.u_trace, r.slot.utrace, (size_t)(q.K + 1) * N * 8, cudaMemcpyDeviceToHost, S->st));
    unsigned status = 0;
    TV_CK(cudaMemcpyAsync(&status, r.slot.status, sizeof(unsigned), cudaMemcpyDeviceToHost, S->st));
    TV_CK(cudaStreamSynchronize(S->st));
    if (status & kStatusNonFinite) return fail(TVSPEC_ECUDA, "non-finite value in the flow");
    return TVSPEC_OK;
}

static void fail_all_active(Server *S, tvspec_status s) {
    for (auto &r : S->active) {
        slot_free(&r->slot, S->st);
        S->used -= r->bytes;
        finish(S, r, s);
    }
    S->active.clear();
    cudaStreamSynchronize(S->st);
}

void Server::loop() {
    cudaSetDevice(plan->device);
    const tvspec_config &c = plan->cfg;
    const int max_batch = c.max_batch > 0 ? c.max_batch : 256;
    const size_t budget = plan_budget(plan);
    bool changed = true;
    for (;;) {
        std::vector<std::shared_ptr<ServeReq>> admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !waiting.empty() || !active.empty(); });
            if (stop) break;
            // cancelled requests still waiting
            for (auto it = waiting.begin(); it != waiting.end();) {
                if ((*it)->cancel) {
                    (*it)->result = TVSPEC_ECANCELLED;
                    (*it)->state = 2;
                    (*it)->t_done = Clock::now();
                    it = waiting.erase(it);
                    cv_done.notify_all();
                } else {
                    ++it;
                }
            }
            while (!waiting.empty() && (int)(active.size() + admitted.size()) < max_batch) {
                auto &r = waiting.front();
                if (used + r->bytes > budget) {
                    if (active.empty() && admitted.empty()) {
                        // can never fit: reject rather than wait forever
                        r->result = fail(TVSPEC_ENOMEM, "request exceeds the serving memory budget");
                        r->state = 2;
                        r->t_done = Clock::now();
                        waiting.pop_front();
                        cv_done.notify_all();
                        continue;
                    }
                    break;
                }
                used += r->bytes;
                r->state = 1;
                admitted.push_back(r);
                waiting.pop_front();
            }
        }
        // running requests cancelled since the last tick
        for (size_t i = 0; i < active.size();) {
            bool cancel;
            {
                std::lock_guard<std::mutex> lk(mu);
                cancel = active[i]->cancel;
            }
            if (cancel) {
                auto r = active[i];
                cudaStreamSynchronize(st);
                slot_free(&r->slot, st);
                used -= r->bytes;
                active.erase(active.begin() + i);
                finish(this, r, TVSPEC_ECANCELLED);
                changed = true;
            } else {
                ++i;
            }
        }
        // admission: workspace, image upload, u_0 = f
        std::vector<std::shared_ptr<ServeReq>> started;
        for (auto &r : admitted) {
            tvspec_status s = slot_alloc(&r->slot, r->job, c.p_storage, false, st, true);
            if (s == TVSPEC_OK) {
                cudaError_t e = cudaMemsetAsync(r->slot.base + r->slot.zero_off, 0, r->slot.zero_bytes, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(r->slot.f, r->job.r.f, (size_t)r->job.r.H * r->job.r.W * 4,
                                        cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) {
                    slot_free(&r->slot, st);
                    s = fail_cuda(e, "request upload");
                }
            }
            if (s != TVSPEC_OK) {
                used -= r->bytes;
                finish(this, r, s);
                continue;
            }
            r->s0 = gstep;
            started.push_back(r);
        }
        if (!started.empty()) {
            std::vector<ImgDesc> nd;
            for (auto &r : started) nd.push_back(slot_desc(r->slot, r->s0));
            if (cudaStreamSynchronize(st) != cudaSuccess ||
                launchset_build(&init_ls, nd, -1, 1) != TVSPEC_OK ||
                launch_init(init_ls.d_descs, init_ls.d_ep_img, init_ls.d_ep_base,
                            init_ls.ep_prefix[init_ls.n], st) != cudaSuccess) {
                for (auto &r : started) {
                    slot_free(&r->slot, st);
                    used -= r->bytes;
                    finish(this, r, fail(TVSPEC_ECUDA, "request start"));
                }
                started.clear();
            } else {
                plan->kernel_launches++;
            }
            for (auto &r : started) active.push_back(r);
            changed = changed || !started.empty();
        }
        if (active.empty()) continue;
        std::vector<Slot *> sp;
        for (auto &r : active) sp.push_back(&r->slot);
        if (changed) {
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                fail_all_active(this, fail(TVSPEC_ECUDA, "stream error"));
                continue;
            }
            if (shape == -2) {
                // tile choice once, on the first request's shape; every shape gives the same bits
                std::vector<Slot *> one{sp[0]};
                if (choose_tiles(plan, one, st, &shape, &depth) != TVSPEC_OK) {
                    fail_all_active(this, TVSPEC_ECUDA);
                    shape = -2;
                    continue;
                }
                // the tuner used the first request's buffers: restart it cleanly
                Slot &s0 = active[0]->slot;
                cudaMemsetAsync(s0.base + s0.zero_off, 0, s0.zero_bytes, st);
                std::vector<ImgDesc> d0{slot_desc(s0, active[0]->s0)};
                launchset_build(&init_ls, d0, -1, 1);
                launch_init(init_ls.d_descs, init_ls.d_ep_img, init_ls.d_ep_base,
                            init_ls.ep_prefix[1], st);
            }
            std::vector<ImgDesc> descs;
            for (auto &r : active) descs.push_back(slot_desc(r->slot, r->s0));
            if (cudaStreamSynchronize(st) != cudaSuccess ||
                launchset_build(&ls, descs, shape, depth) != TVSPEC_OK) {
                fail_all_active(this, TVSPEC_ECUDA);
                continue;
            }
            changed = false;
        }
        uint64_t nk = 0;
        tvspec_status s = enqueue_step(plan, ls, sp, (int)active.size(), gstep, st, &nk);
        plan->kernel_launches += nk;
        if (s != TVSPEC_OK) {
            fail_all_active(this, s);
            changed = true;
            continue;
        }
        // retire the requests whose last step just ran
        for (size_t i = 0; i < active.size();) {
            auto r = active[i];
            if (gstep - r->s0 == r->job.r.K - 1) {
                tvspec_status cs = copy_out(this, *r);
                slot_free(&r->slot, st);
                used -= r->bytes;
                active.erase(active.begin() + i);
                plan->decompositions++;
                finish(this, r, cs);
                changed = true;
            } else {
                ++i;
            }
        }
        ++gstep;
    }
    // shutdown: cancel everything still resident or queued
    cudaStreamSynchronize(st);
    for (auto &r : active) {
        slot_free(&r->slot, st);
        finish(this, r, TVSPEC_ECANCELLED);
    }
    active.clear();
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &r : waiting) {
            r->result = TVSPEC_ECANCELLED;
            r->state = 2;
        }
        waiting.clear();
        cv_done.notify_all();
    }
    cudaStreamSynchronize(st);
    ls.release();
    init_ls.release();
}

}  // namespace tvspec

using namespace tvspec;

extern "C" {

void tvspec_server_stop(tvspec_plan *plan) {
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(plan->server_mu);
        S = plan->server;
        plan->server = nullptr;
    }
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(plan->device);
    cudaStreamDestroy(S->st);
    delete S;
}

static tvspec_status get_server(tvspec_plan *plan, Server **out) {
    std::lock_guard<std::mutex> lk(plan->server_mu);
    if (!plan->server) {
        TV_CK(cudaSetDevice(plan->device));
        auto *S = new (std::nothrow) Server();
        if (!S) return fail(TVSPEC_ENOMEM, "server allocation");
        S->plan = plan;
        cudaError_t e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete S;
            return fail_cuda(e, "serving stream");
        }
        S->th = std::thread([S] { S->loop(); });
        plan->server = S;
    }
    *out = plan->server;
    return TVSPEC_OK;
}

tvspec_status tvspec_submit(tvspec_plan *plan, const tvspec_request *req, uint64_t *ticket) {
    if (!plan || !req || !ticket) return fail(TVSPEC_EINVAL, "NULL argument");
    if (req->mem_kind != TVSPEC_MEM_HOST)
        return fail(TVSPEC_EINVAL, "serving accepts host-memory requests only");
    if (plan->cfg.kernel == TVSPEC_KERNEL_NAIVE)
        return fail(TVSPEC_ENOTSUP, "serving runs the tiled kernel only");
    auto r = std::make_shared<ServeReq>();
    tvspec_status s = make_job(*req, &r->job);
    if (s != TVSPEC_OK) return s;
    r->bytes = slot_bytes_for(r->job, plan->cfg.p_storage, false);
    Server *S = nullptr;
    s = get_server(plan, &S);
    if (s != TVSPEC_OK) return s;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        r->t_submit = Clock::now();
        S->all[r->ticket] = r;
        S->waiting.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();
    return TVSPEC_OK;
}

static std::shared_ptr<ServeReq> find(Server *S, uint64_t t) {
    auto it = S->all.find(t);
    return it == S->all.end() ? nullptr : it->second;
}

tvspec_status tvspec_poll(tvspec_plan *plan, uint64_t ticket) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(plan->server_mu);
        S = plan->server;
    }
    if (!S) return fail(TVSPEC_EINVAL, "unknown ticket");
    std::lock_guard<std::mutex> lk(S->mu);
    auto r = find(S, ticket);
    if (!r) return fail(TVSPEC_EINVAL, "unknown ticket");
    return r->state == 2 ? r->result : TVSPEC_ENOTREADY;
}

tvspec_status tvspec_wait(tvspec_plan *plan, uint64_t ticket, int timeout_ms) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(plan->server_mu);
        S = plan->server;
    }
    if (!S) return fail(TVSPEC_EINVAL, "unknown ticket");
    std::unique_lock<std::mutex> lk(S->mu);
    auto r = find(S, ticket);
    if (!r) return fail(TVSPEC_EINVAL, "unknown ticket");
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, [&] { return r->state == 2; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                    [&] { return r->state == 2; })) {
        return fail(TVSPEC_ETIMEOUT, "request not finished within the timeout");
    }
    return r->result;
}

tvspec_status tvspec_cancel(tvspec_plan *plan, uint64_t ticket) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(plan->server_mu);
        S = plan->server;
    }
    if (!S) return fail(TVSPEC_EINVAL, "unknown ticket");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto r = find(S, ticket);
        if (!r || r->state == 2) return fail(TVSPEC_EINVAL, "unknown or finished ticket");
        r->cancel = true;
    }
    S->cv_work.notify_all();
    return TVSPEC_OK;
}

tvspec_status tvspec_serving_stats(tvspec_plan *plan, int reset, uint64_t *count, double *p50_ms,
                                   double *p99_ms) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(plan->server_mu);
        S = plan->server;
    }
    std::vector<double> v;
    if (S) {
        std::lock_guard<std::mutex> lk(S->mu);
        v = S->lat_ms;
        if (reset) S->lat_ms.clear();
    }
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(q * v.size()) - 1);
        return v[i];
    };
    if (count) *count = v.size();
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    return TVSPEC_OK;
}

}  // extern "C"
