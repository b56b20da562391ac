// Spectrum server: continuous batching of KPM requests on one GPU.
//
// Two threads own the GPU side.  Requests wait in a FIFO queue; the admission
// thread takes one when a slot is free and its estimated device memory fits in
// the configured budget, and sets it up (context: tables, integrals, tensor-core
// operands and autotuning; the dipole and first step) on the request's own
// non-blocking stream, so that set-up overlaps the rounds of the requests
// already resident instead of stalling them.  The round thread then adds the
// set-up request to its resident set.  Each round, it queues `steps_per_round`
// Chebyshev steps for every resident request before it waits on any of them,
// so the kernels of different requests overlap on the device; a request
// admitted while others are mid-recursion joins the next round.  A finished
// request's moments are combined (doubling identities), its spectrum is
// reconstructed on its stream, and its context is released, which frees budget
// for the queue.  A request whose set-up or advance fails is finished with that
// status at once and its slot and budget are released; the others go on.
//
// Every request's arithmetic is what it would be alone: its own context, the
// same kernels, launch shapes and reduction grids (on the FP64 / FP32 gather
// path, requests that advance by the same number of steps in a round share
// batched launches whose per-request work is that of the single launches), so
// its result does not depend on what else is resident.  All waits are bounded (kpm_server_wait's timeout; the worker's
// condition-variable waits).
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "common.cuh"

using namespace kpm;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

struct Req {
    uint64_t id = 0;
    int norb = 0, na = 0, nb = 0;
    std::vector<double> h1, eri, dip, psi0;
    unsigned mask = 0;
    int ncol = 0;
    double a = 1.0, b = 0.0;
    int nmoments = 0, npoints = 0, kernel = 1;
    bool deflate = false;
    double e0 = 0.0;
    size_t mem = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    bool done = false;
    std::atomic<bool> cancelled{false};
    std::atomic<int> inject{KPM_OK};   // testing aid: next advance "returns" this status
    kpm_status status = KPM_OK;
    std::string err;
    std::vector<double> moments, omega, intensity;
};

struct Slot {
    std::shared_ptr<Req> req;
    kpm_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    DevBuf psi, mom, dmp, om, in;
    int steps = 0, total = 0;
    kpm_status failed = KPM_OK;   // an advance of this request failed
    std::string fail_msg;
};

// Device bytes a request keeps resident (vectors, workspaces, tables).
size_t estimate_bytes(int n, int na, int nb, int ncol, kpm_precision prec) {
    int64_t sa = binom(n, na), sb = binom(n, nb), dim = sa * sb;
    size_t esz = prec == KPM_FP64 ? 8 : 4;
    size_t v = (size_t)dim * esz * 3 * ncol + (size_t)dim * 8;
    v += prec == KPM_FP64 ? 0 : (size_t)dim * 8;   // exact diagonal (hi, lo floats)
    if (prec == KPM_MIXED || prec == KPM_MIXED_BF16) {
        // split FP16 copies of x and x^T, dense split string Hamiltonians
        v += (size_t)dim * 8 + (size_t)4 * sa * ((sa + 7) / 8 * 8);
        if (na != nb) v += (size_t)4 * sb * ((sb + 7) / 8 * 8);
    }
    auto tables = [&](int m, int64_t ns) {
        int64_t nexc = m * (n - m + 1);
        int64_t nnbr = 1 + (int64_t)m * (n - m) + binom(m, 2) * binom(n - m, 2);
        int P = ((n * (n + 1) / 2 + 1 + 15) / 16) * 16;
        return (size_t)ns * (4 + 14 * nexc + 16 * nnbr + 4 * P);
    };
    v += tables(na, sa) + (na == nb ? 0 : tables(nb, sb));
    v += (size_t)n * n * n * n * 12 + (64 << 20);
    return v;
}

}  // namespace

struct kpm_server {
    kpm_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work;    // admission thread: queue or budget changed
    std::condition_variable cv_round;   // round thread: a request is ready
    std::condition_variable cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    std::vector<std::unique_ptr<Slot>> ready;   // set up, not yet resident (guarded by mu)
    size_t mem_used = 0;
    int in_setup = 0;                           // being set up (guarded by mu)
    int n_active = 0;                           // resident (guarded by mu)
    uint64_t next_id = 1;
    bool stop = false;
    std::thread admitter, worker;
    std::vector<std::unique_ptr<Slot>> active;  // round thread only
    std::atomic<int> resident{0};

    void admit_loop();
    void run();
    void setup(Slot& s);
    void finish(Slot& s);
    void fail(Slot& s, kpm_status st, const std::string& msg);
    void release(Slot& s);
    void complete(Slot& s, bool resident_slot);
};

// Admission thread: FIFO, a free slot and room in the budget (a request larger
// than the whole budget was refused at submit; one is always admitted when
// nothing else is held), then set-up on the request's own stream.
void kpm_server::admit_loop() {
    cudaSetDevice(device);
    for (;;) {
        std::shared_ptr<Req> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop) return;
                while (!queue.empty() && queue.front()->cancelled) queue.pop_front();
                const int held = n_active + (int)ready.size() + in_setup;
                if (!queue.empty() && held < cfg.max_slots &&
                    (mem_used + queue.front()->mem <= cfg.mem_budget_bytes || held == 0)) {
                    r = queue.front();
                    queue.pop_front();
                    mem_used += r->mem;
                    ++in_setup;
                    r->t_admit = now_s();
                    break;
                }
                cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
        }
        auto s = std::make_unique<Slot>();
        s->req = r;
        try {
            setup(*s);
        } catch (const Error& e) {
            fail(*s, e.status, e.msg);
            complete(*s, false);
            continue;
        }
        std::lock_guard<std::mutex> lk(mu);
        --in_setup;
        ready.push_back(std::move(s));
        cv_round.notify_one();
    }
}

// Frees a slot's device resources (its context and buffers, then its stream).
void kpm_server::release(Slot& s) {
    if (s.ctx) kpm_destroy(s.ctx);
    s.ctx = nullptr;
    s.psi.release();
    s.mom.release();
    s.dmp.release();
    s.om.release();
    s.in.release();
    if (s.st) cudaStreamDestroy(s.st);
    s.st = nullptr;
}

// Records a request's failure status; complete() makes it visible.
void kpm_server::fail(Slot& s, kpm_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(mu);
    s.req->status = st;
    s.req->err = msg;
}

// Releases the slot's device resources and budget, then marks the request done
// (so that a waiter that returns sees the server's accounting already updated).
void kpm_server::complete(Slot& s, bool resident_slot) {
    release(s);
    std::lock_guard<std::mutex> lk(mu);
    mem_used -= s.req->mem;
    if (resident_slot) {
        --n_active;
        resident.store(n_active);
    } else {
        --in_setup;
    }
    s.req->done = true;
    s.req->t_done = now_s();
    cv_done.notify_all();
    cv_work.notify_one();
}

void kpm_server::setup(Slot& s) {
    Req& r = *s.req;
    KPM_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
    kpm_status st = kpm_create(r.h1.data(), r.eri.data(), r.dip.data(), r.norb, r.na, r.nb,
                               cfg.precision, s.st, &s.ctx);
    if (st != KPM_OK) KPM_THROW(st, "%s", kpm_last_error(nullptr));
    int64_t dim = kpm_dim(s.ctx);
    s.psi.alloc((size_t)dim * 8);
    KPM_CUDA(cudaMemcpyAsync(s.psi.p, r.psi0.data(), (size_t)dim * 8, cudaMemcpyHostToDevice, s.st));
    st = r.deflate ? kpm_recursion_begin_deflated(s.ctx, s.psi.as<double>(), r.e0, r.mask, r.a,
                                                  r.b, r.nmoments)
                   : kpm_recursion_begin(s.ctx, s.psi.as<double>(), r.mask, r.a, r.b, r.nmoments);
    if (st != KPM_OK) KPM_THROW(st, "%s", kpm_last_error(s.ctx));
    s.steps = 1;
    s.total = r.nmoments / 2;
}

void kpm_server::finish(Slot& s) {
    Req& r = *s.req;
    std::vector<double> m((size_t)r.ncol * r.nmoments);
    int nm = 0;
    kpm_status st = kpm_recursion_moments(s.ctx, m.data(), &nm);
    if (st != KPM_OK && st != KPM_EBOUNDS) KPM_THROW(st, "%s", kpm_last_error(s.ctx));
    // total spectrum: moments summed over the requested components
    std::vector<double> tot(r.nmoments, 0.0);
    for (int c = 0; c < r.ncol; ++c)
        for (int i = 0; i < r.nmoments; ++i) tot[i] += m[(size_t)c * r.nmoments + i];
    s.mom.alloc(sizeof(double) * r.nmoments);
    s.dmp.alloc(sizeof(double) * r.nmoments);
    s.om.alloc(sizeof(double) * r.npoints);
    s.in.alloc(sizeof(double) * r.npoints);
    KPM_CUDA(cudaMemcpyAsync(s.mom.p, tot.data(), sizeof(double) * r.nmoments,
                             cudaMemcpyHostToDevice, s.st));
    spectrum_dev(s.mom.as<double>(), r.nmoments, r.a, r.b, r.npoints, r.kernel,
                 s.dmp.as<double>(), s.om.as<double>(), s.in.as<double>(), s.st);
    std::vector<double> om(r.npoints), in(r.npoints);
    KPM_CUDA(cudaMemcpyAsync(om.data(), s.om.p, sizeof(double) * r.npoints,
                             cudaMemcpyDeviceToHost, s.st));
    KPM_CUDA(cudaMemcpyAsync(in.data(), s.in.p, sizeof(double) * r.npoints,
                             cudaMemcpyDeviceToHost, s.st));
    KPM_CUDA(cudaStreamSynchronize(s.st));
    std::lock_guard<std::mutex> lk(mu);
    r.moments = std::move(m);
    r.omega = std::move(om);
    r.intensity = std::move(in);
    r.status = st;
    if (st == KPM_EBOUNDS) r.err = "moments exceed Omega_0: [b-a, b+a] misses the spectrum";
}

// Round thread: resident requests advance by steps_per_round Chebyshev steps
// per round, queued for all of them before any result is waited for.
void kpm_server::run() {
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            for (auto& s : ready) active.push_back(std::move(s));
            ready.clear();
            n_active = (int)active.size();
            resident.store(n_active);

            if (active.empty()) {
                if (stop && in_setup == 0) break;
                cv_round.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
        }
        // On the gather path (FP64, FP32) the requests that advance by the same
        // number of steps share one sigma and one update launch per step
        // (kpm_recursion_advance_batch); each result is identical either way.
        // A failed advance (or an injected failure) finishes that request with
        // its status; a failed batch finishes every request of the batch.
        const bool gather = cfg.precision == KPM_FP64 || cfg.precision == KPM_FP32;
        std::map<int, std::vector<Slot*>> by_k;
        for (auto& s : active) {
            if (s->req->cancelled) continue;
            int k = std::min(cfg.steps_per_round, s->total - s->steps);
            if (k <= 0) continue;
            const int inj = s->req->inject.exchange(KPM_OK);
            if (inj != KPM_OK) {
                s->failed = (kpm_status)inj;
                s->fail_msg = "injected advance failure (testing aid)";
                continue;
            }
            if (gather) {
                by_k[k].push_back(s.get());
                continue;
            }
            kpm_status st = kpm_recursion_advance(s->ctx, k);
            if (st == KPM_OK) {
                s->steps += k;
            } else {
                s->failed = st;
                s->fail_msg = kpm_last_error(s->ctx);
            }
        }
        for (auto& kv : by_k) {
            const int k = kv.first;
            std::vector<Slot*>& group = kv.second;
            std::vector<kpm_ctx*> ctxs;
            for (Slot* s : group) ctxs.push_back(s->ctx);
            kpm_status st = group.size() == 1
                                ? kpm_recursion_advance(ctxs[0], k)
                                : kpm_recursion_advance_batch(ctxs.data(), (int)ctxs.size(), k);
            for (Slot* s : group) {
                if (st == KPM_OK) {
                    s->steps += k;
                } else {
                    s->failed = st;
                    s->fail_msg = kpm_last_error(ctxs[0]);
                }
            }
        }
        std::vector<std::unique_ptr<Slot>> keep;
        for (auto& s : active) {
            const bool cancelled = s->req->cancelled;
            if (s->failed == KPM_OK && s->steps < s->total && !cancelled) {
                keep.push_back(std::move(s));
                continue;
            }
            try {
                if (s->failed != KPM_OK) fail(*s, s->failed, s->fail_msg);
                else if (cancelled) fail(*s, KPM_ECANCELLED, "cancelled");
                else finish(*s);
            } catch (const Error& e) {
                fail(*s, e.status, e.msg);
            }
            complete(*s, true);
        }
        active.swap(keep);
    }
}

extern "C" {

kpm_status kpm_server_create(const kpm_server_config* cfg, kpm_server** out) {
    if (out) *out = nullptr;
    if (!cfg || !out || cfg->max_slots < 1 || cfg->steps_per_round < 1 || cfg->mem_budget_bytes == 0) {
        set_thread_error("bad server configuration");
        return KPM_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_thread_error("no CUDA device available");
        return KPM_ECUDA;
    }
    auto* s = new kpm_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->worker = std::thread([s] { s->run(); });
    s->admitter = std::thread([s] { s->admit_loop(); });
    *out = s;
    return KPM_OK;
}

kpm_status kpm_server_submit(kpm_server* s, const kpm_request* q, uint64_t* id) {
    if (!s || !q || !id || !q->h1 || !q->eri || !q->dipole || !q->psi0) {
        set_thread_error("NULL argument");
        return KPM_EINVAL;
    }
    if (q->norb < 1 || q->norb > KPM_MAX_ORB || q->nalpha < 0 || q->nbeta < 0 ||
        q->nalpha > q->norb || q->nbeta > q->norb || q->nmoments < 2 || (q->nmoments & 1) ||
        q->npoints < 1 || !(q->comp_mask & 7u) || (q->comp_mask & ~7u) || !(q->a > 0.0) ||
        q->kernel < 0 || q->kernel > 2) {
        set_thread_error("bad request");
        return KPM_EINVAL;
    }
    auto r = std::make_shared<Req>();
    int n = q->norb;
    r->norb = n;
    r->na = q->nalpha;
    r->nb = q->nbeta;
    r->h1.assign(q->h1, q->h1 + (size_t)n * n);
    r->eri.assign(q->eri, q->eri + (size_t)n * n * n * n);
    r->dip.assign(q->dipole, q->dipole + (size_t)3 * n * n);
    int64_t dim = binom(n, q->nalpha) * binom(n, q->nbeta);
    r->psi0.assign(q->psi0, q->psi0 + dim);
    r->mask = q->comp_mask;
    r->ncol = __builtin_popcount(q->comp_mask);
    r->a = q->a;
    r->b = q->b;
    r->nmoments = q->nmoments;
    r->npoints = q->npoints;
    r->kernel = q->kernel;
    r->deflate = q->deflate != 0;
    r->e0 = q->e0;
    r->mem = estimate_bytes(n, q->nalpha, q->nbeta, r->ncol, s->cfg.precision);
    if (r->mem > s->cfg.mem_budget_bytes) {
        set_thread_error("request needs more device memory than the server budget");
        return KPM_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->t_submit = now_s();
        s->reqs[r->id] = r;
        s->queue.push_back(r);
    }
    s->cv_work.notify_all();
    *id = r->id;
    return KPM_OK;
}

kpm_status kpm_server_wait(kpm_server* s, uint64_t id, int timeout_ms, kpm_result* out) {
    if (!s) {
        set_thread_error("NULL server");
        return KPM_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_thread_error("unknown request id");
        return KPM_EINVAL;
    }
    std::shared_ptr<Req> r = it->second;
    bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                  [&] { return r->done; });
    if (!ok) {
        set_thread_error("request not finished within the timeout");
        return KPM_ETIMEOUT;
    }
    if (out) {
        if (out->moments && !r->moments.empty())
            std::memcpy(out->moments, r->moments.data(), sizeof(double) * r->moments.size());
        if (out->omega && !r->omega.empty())
            std::memcpy(out->omega, r->omega.data(), sizeof(double) * r->omega.size());
        if (out->intensity && !r->intensity.empty())
            std::memcpy(out->intensity, r->intensity.data(), sizeof(double) * r->intensity.size());
        out->t_queue_s = r->t_admit > 0 ? r->t_admit - r->t_submit : 0.0;
        out->t_run_s = r->t_admit > 0 ? r->t_done - r->t_admit : 0.0;
        out->t_total_s = r->t_done - r->t_submit;
    }
    kpm_status st = r->status;
    if (st != KPM_OK) set_thread_error(r->err);
    s->reqs.erase(id);
    return st;
}

kpm_status kpm_server_cancel(kpm_server* s, uint64_t id) {
    if (!s) return KPM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_thread_error("unknown request id");
        return KPM_EINVAL;
    }
    std::shared_ptr<Req> r = it->second;
    r->cancelled = true;
    // still queued: finish it here
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if ((*q)->id == id) {
            s->queue.erase(q);
            r->status = KPM_ECANCELLED;
            r->err = "cancelled";
            r->done = true;
            r->t_done = now_s();
            s->cv_done.notify_all();
            break;
        }
    return KPM_OK;
}

kpm_status kpm_server_stats(kpm_server* s, size_t* mem_used, int* resident, int* queued) {
    if (!s) return KPM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (mem_used) *mem_used = s->mem_used;
    if (queued) *queued = (int)s->queue.size();
    if (resident) *resident = s->resident.load();
    return KPM_OK;
}

void kpm_server_destroy(kpm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& q : s->queue) {
            q->cancelled = true;
            q->status = KPM_ECANCELLED;
            q->done = true;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_round.notify_all();
    s->cv_done.notify_all();
    // the admission thread finishes the set-up it is in, then stops; the round
    // thread then runs every resident request to its end
    if (s->admitter.joinable()) s->admitter.join();
    s->cv_round.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

kpm_status kpm_server_inject_failure(kpm_server* s, uint64_t id, kpm_status status) {
    if (!s || status == KPM_OK) {
        set_thread_error("NULL server or KPM_OK status");
        return KPM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_thread_error("unknown request id");
        return KPM_EINVAL;
    }
    it->second->inject.store((int)status);
    return KPM_OK;
}

}  // extern "C"
