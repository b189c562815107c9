// Serving: continuous batching of single-image decompositions at ROF-step boundaries.
//
// A scheduler thread owns the device work of served requests. Each tick it
//   1. takes cancelled requests out of the resident set,
//   2. admits waiting requests (FIFO) while their workspace fits the memory budget and the
//      number of resident requests stays below max_batch, allocates their workspace
//      (stream-ordered), uploads their images and starts them (u_0 = f) at the current
//      global step,
//   3. runs one ROF step (all dual iterations + the epilogue) for every resident request in
//      one set of launches over the tiles of all of them,
//   4. hands the requests whose K-th step was just enqueued to a retire thread.
// The retire thread waits for a request's last step on its own stream, copies the outputs
// to the caller's buffers, frees the workspace and signals completion, while the scheduler
// keeps the compute stream busy with the next ticks. Launch tables are double-buffered:
// a table is rebuilt only after the event recorded behind its last use has completed.
//
// Requests therefore join and leave while others are mid-flight; each request's arithmetic
// is the same as when it runs alone (tiling-invariant dual iterations, per-image reductions
// in a fixed order), so its results are bit-identical. The tile shape is the configured one,
// or tuned once on a 2048 x 2048 image under the plan lock.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "runtime.h"

namespace tvspec {

using Clock = std::chrono::steady_clock;

struct ServeReq {
    uint64_t ticket = 0;
    Job job;
    int state = 0;  // 0 queued, 1 resident or retiring, 2 finished (result below)
    bool cancel = false;
    tvspec_status result = TVSPEC_ENOTREADY;
    tvspec_status pending = TVSPEC_OK;  // result to report once retired
    Clock::time_point t_submit, t_done;
    Slot slot;
    int s0 = 0;
    size_t bytes = 0;
    cudaEvent_t done_ev = nullptr;
};

struct Server {
    tvspec_plan *plan = nullptr;
    std::thread th, retire_th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_retire;
    std::deque<std::shared_ptr<ServeReq>> waiting;
    std::vector<std::shared_ptr<ServeReq>> active;  // scheduler thread only
    std::deque<std::shared_ptr<ServeReq>> retire_q;
    std::map<uint64_t, std::shared_ptr<ServeReq>> all;
    uint64_t next_ticket = 1;
    bool stop = false, retire_stop = false;
    size_t used = 0;
    std::vector<double> lat_ms;
    cudaStream_t st = nullptr;   // compute
    cudaStream_t cst = nullptr;  // copies out
    LaunchSet ls[2];
    cudaEvent_t ls_ev[2] = {nullptr, nullptr};
    bool ls_used[2] = {false, false};
    int cur = 0;
    int gstep = 0;
    int shape = -2, depth = 1;
    bool pdl = false;
    void loop();
    void retire_loop();
    void hand_to_retire(const std::shared_ptr<ServeReq> &r, tvspec_status pending);
    void fail_all_active(tvspec_status s);
};

static void finish(Server *S, const std::shared_ptr<ServeReq> &r, tvspec_status result) {
    // a finished ticket stays queryable; it keeps its status, not its request's tables
    std::vector<double>().swap(r->job.edges);
    std::vector<signed char>().swap(r->job.band_of_k);
    std::vector<double>().swap(r->job.filt_H);
    std::vector<double>().swap(r->job.filt_res);
    std::lock_guard<std::mutex> lk(S->mu);
    r->result = result;
    r->state = 2;
    r->t_done = Clock::now();
    if (result == TVSPEC_OK)
        S->lat_ms.push_back(
            std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    S->cv_done.notify_all();
}

// The request's work is enqueued on the compute stream; record its completion and queue it
// for the retire thread.
void Server::hand_to_retire(const std::shared_ptr<ServeReq> &r, tvspec_status pending) {
    r->pending = pending;
    if (cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r->done_ev, st) != cudaSuccess) {
        cudaGetLastError();
        if (r->done_ev) cudaEventDestroy(r->done_ev);
        r->done_ev = nullptr;
        cudaStreamSynchronize(st);  // fall back to waiting here
        if (r->pending == TVSPEC_OK) r->pending = TVSPEC_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        retire_q.push_back(r);
    }
    cv_retire.notify_one();
}

void Server::fail_all_active(tvspec_status s) {
    for (auto &r : active) hand_to_retire(r, s);
    active.clear();
}

// Copies the outputs of a finished request to its host buffers on the copy stream.
static tvspec_status copy_out(cudaStream_t cst, ServeReq &r) {
    const tvspec_request &q = r.job.r;
    const size_t N = (size_t)q.H * q.W;
    TV_CK(cudaMemcpyAsync(q.bands, r.slot.bands, (size_t)r.slot.n_bands * N * 4, cudaMemcpyDeviceToHost, cst));
    TV_CK(cudaMemcpyAsync(q.residual, r.slot.residual, N * 4, cudaMemcpyDeviceToHost, cst));
    TV_CK(cudaMemcpyAsync(q.S, r.slot.S, (size_t)(q.K - 1) * 8, cudaMemcpyDeviceToHost, cst));
    if (q.u_trace)
        TV_CK(cudaMemcpyAsync(q.u_trace, r.slot.utrace, (size_t)(q.K + 1) * N * 8, cudaMemcpyDeviceToHost, cst));
    if (q.n_filters > 0)
        TV_CK(cudaMemcpyAsync(q.filtered, r.slot.filtered, (size_t)q.n_filters * N * 4, cudaMemcpyDeviceToHost, cst));
    if (q.S_parseval)
        TV_CK(cudaMemcpyAsync(q.S_parseval, r.slot.S_par, (size_t)(q.K - 1) * 8, cudaMemcpyDeviceToHost, cst));
    unsigned status = 0;
    TV_CK(cudaMemcpyAsync(&status, r.slot.status, sizeof(unsigned), cudaMemcpyDeviceToHost, cst));
    TV_CK(cudaStreamSynchronize(cst));
    if (!r.slot.guards.empty()) {
        tvspec_status g = slot_check_guards(r.slot, cst);
        if (g != TVSPEC_OK) return g;
    }
    if (status & kStatusBarrierTimeout)
        return fail(TVSPEC_ETIMEOUT, "a grid barrier wait ran out (a CTA did not arrive)");
    if (status & kStatusCopyTimeout) return fail(TVSPEC_ETIMEOUT, "a wait for a tile's TMA copies ran out");
    if (status & kStatusNonFinite) return fail(TVSPEC_ECUDA, "non-finite value in the flow");
    return TVSPEC_OK;
}

void Server::retire_loop() {
    cudaSetDevice(plan->device);
    for (;;) {
        std::shared_ptr<ServeReq> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_retire.wait(lk, [&] { return retire_stop || !retire_q.empty(); });
            if (retire_q.empty()) break;  // retire_stop and nothing left
            r = retire_q.front();
            retire_q.pop_front();
        }
        if (r->done_ev) cudaStreamWaitEvent(cst, r->done_ev, 0);
        tvspec_status res = r->pending;
        if (res == TVSPEC_OK) res = copy_out(cst, *r);
        slot_free(&r->slot, cst);  // stream-ordered after the copies and the last step
        if (r->done_ev) cudaEventDestroy(r->done_ev);
        r->done_ev = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            used -= r->bytes;
        }
        if (res == TVSPEC_OK) plan->decompositions++;
        finish(this, r, res);
        cv_work.notify_all();  // memory came free: waiting requests may fit now
    }
    cudaStreamSynchronize(cst);
}

void Server::loop() {
    cudaSetDevice(plan->device);
    const tvspec_config &c = plan->cfg;
    const int max_batch = c.max_batch > 0 ? c.max_batch : 256;
    const size_t budget = plan_budget(plan);
    for (int i = 0; i < 2; ++i) cudaEventCreateWithFlags(&ls_ev[i], cudaEventDisableTiming);
    bool changed = true;
    for (;;) {
        std::vector<std::shared_ptr<ServeReq>> admitted;
        std::vector<std::shared_ptr<ServeReq>> cancelled;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !waiting.empty() || !active.empty(); });
            if (stop) break;
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
                    if (active.empty() && admitted.empty() && used == 0) {
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
            for (auto &r : active)
                if (r->cancel) cancelled.push_back(r);
        }
        for (auto &r : cancelled) {
            active.erase(std::find(active.begin(), active.end(), r));
            hand_to_retire(r, TVSPEC_ECANCELLED);
            changed = true;
        }
        // admission: workspace, image upload
        std::vector<std::shared_ptr<ServeReq>> started;
        for (auto &r : admitted) {
            tvspec_status s = slot_alloc(&r->slot, r->job, c.p_storage, false, st, true, c.acc_mode,
                                         c.test_guard_bytes);
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
                {
                    std::lock_guard<std::mutex> lk(mu);
                    used -= r->bytes;
                }
                finish(this, r, s);
                continue;
            }
            r->s0 = gstep;
            started.push_back(r);
        }
        for (auto &r : started) active.push_back(r);
        if (!started.empty()) changed = true;
        if (active.empty()) {
            // nothing resident: the queue head waits for memory a retiring request holds;
            // sleep until the retire thread (or a submit / stop) signals
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        if (shape == -2) {
            // one tile choice for all mixes: tuned on a 2048 x 2048 image, the size class
            // that carries most of the served pixels (every shape gives the same bits)
            if (c.tile >= 0) {
                std::vector<Slot *> none;
                if (choose_tiles(plan, none, st, &shape, &depth, true, &pdl) != TVSPEC_OK) shape = -2;
            } else if (tune_for_size(plan, 2048, 2048, &shape, &depth, &pdl) != TVSPEC_OK) {
                shape = -2;
            }
            if (shape == -2) {
                fail_all_active(TVSPEC_ECUDA);
                continue;
            }
        }
        if (changed) {
            const int nb = cur ^ 1;
            if (ls_used[nb]) cudaEventSynchronize(ls_ev[nb]);  // its last tick is done
            std::vector<ImgDesc> descs;
            for (auto &r : active) descs.push_back(slot_desc(r->slot, r->s0));
            ls[nb].pdl = pdl;
            if (launchset_build(&ls[nb], descs, shape, depth) != TVSPEC_OK) {
                fail_all_active(TVSPEC_ECUDA);
                continue;
            }
            cur = nb;
            if (!started.empty()) {
                // the newly started images are the last ones of the set
                const int first = (int)(active.size() - started.size());
                const int n = (int)active.size();
                const int b0 = ls[cur].ep_prefix[first];
                if (launch_init(ls[cur].d_descs, ls[cur].d_ep_img, ls[cur].d_ep_base,
                                ls[cur].ep_prefix[n] - b0, st, b0) != cudaSuccess) {
                    fail_all_active(fail(TVSPEC_ECUDA, "request start"));
                    continue;
                }
                plan->kernel_launches++;
            }
            changed = false;
        }
        NvtxRange tick("tvspec serving step");
        std::vector<Slot *> sp;
        for (auto &r : active) sp.push_back(&r->slot);
        uint64_t nk = 0;
        tvspec_status s = enqueue_step(plan, ls[cur], sp, (int)active.size(), gstep, st, &nk);
        plan->kernel_launches += nk;
        cudaEventRecord(ls_ev[cur], st);
        ls_used[cur] = true;
        if (s != TVSPEC_OK) {
            fail_all_active(s);
            changed = true;
            continue;
        }
        // requests whose last step was just enqueued leave the resident set
        for (size_t i = 0; i < active.size();) {
            auto r = active[i];
            if (gstep - r->s0 == r->job.r.K - 1) {
                hand_to_retire(r, TVSPEC_OK);
                active.erase(active.begin() + i);
                changed = true;
            } else {
                ++i;
            }
        }
        ++gstep;
    }
    // shutdown: everything resident is cancelled, everything queued too
    fail_all_active(TVSPEC_ECANCELLED);
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &r : waiting) {
            r->result = TVSPEC_ECANCELLED;
            r->state = 2;
        }
        waiting.clear();
        retire_stop = true;
        cv_done.notify_all();
    }
    cv_retire.notify_all();
    if (retire_th.joinable()) retire_th.join();
    cudaStreamSynchronize(st);
    for (int i = 0; i < 2; ++i) {
        ls[i].release();
        if (ls_ev[i]) cudaEventDestroy(ls_ev[i]);
    }
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
    cudaStreamDestroy(S->cst);
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
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cst, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (S->st) cudaStreamDestroy(S->st);
            delete S;
            return fail_cuda(e, "serving streams");
        }
        // keep memory freed by retired requests in the stream-ordered pool for the next ones
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, plan->device) == cudaSuccess) {
            uint64_t keep = plan_budget(plan);
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
        S->retire_th = std::thread([S] { S->retire_loop(); });
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
    r->bytes = slot_bytes_for(r->job, plan->cfg.p_storage, false, plan->cfg.test_guard_bytes);
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

static Server *server_of(tvspec_plan *plan) {
    std::lock_guard<std::mutex> lk(plan->server_mu);
    return plan->server;
}

tvspec_status tvspec_poll(tvspec_plan *plan, uint64_t ticket) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    Server *S = server_of(plan);
    if (!S) return fail(TVSPEC_EINVAL, "unknown ticket");
    std::lock_guard<std::mutex> lk(S->mu);
    auto r = find(S, ticket);
    if (!r) return fail(TVSPEC_EINVAL, "unknown ticket");
    return r->state == 2 ? r->result : TVSPEC_ENOTREADY;
}

tvspec_status tvspec_wait(tvspec_plan *plan, uint64_t ticket, int timeout_ms) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    Server *S = server_of(plan);
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
    Server *S = server_of(plan);
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
    Server *S = server_of(plan);
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
