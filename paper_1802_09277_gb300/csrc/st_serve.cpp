// Serving loop with continuous batching (see st_serve_* in include/st_iga.h).
//
// Host-side scheduler only: every solve goes through st_setup / st_solve of
// this library on the worker's own CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/st_iga.h"
#include "st_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Key {
    int geometry, degree, spans[3], slabs;
    double tol;
    int coeffs;
    bool operator<(const Key &o) const {
        return std::memcmp(this, &o, sizeof(Key)) < 0;
    }
    bool same_problem(const Key &o) const {
        return geometry == o.geometry && degree == o.degree && spans[0] == o.spans[0] &&
               spans[1] == o.spans[1] && spans[2] == o.spans[2] && slabs == o.slabs;
    }
};

struct Pending {
    uint64_t ticket;
    Key key;
    std::vector<double> rhs;
    Clock::time_point submitted;
};

struct Done {
    bool done = false;
    st_result res{};
    std::vector<double> u;
    Clock::time_point submitted;
};

struct Entry {  // a cached setup for one configuration and batch size
    Key key;
    int nrhs = 1;
    st_handle h = nullptr;
    double *f = nullptr, *u = nullptr;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_used = 0;
};

void zero_key(Key &k) { std::memset(&k, 0, sizeof k); }

}  // namespace

struct st_server_s {
    st_server_opts o{};
    int device = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    std::map<uint64_t, Done> results;
    std::vector<std::unique_ptr<Entry>> cache;
    std::vector<std::thread> threads;
    uint64_t next_ticket = 1, clock = 0;
    int busy_workers = 0;
    bool stop = false;
};

namespace {

void destroy_entry(st_server_s *s, Entry *e) {
    if (e->h) st_destroy(e->h);
    if (e->f) cudaFree(e->f);
    if (e->u) cudaFree(e->u);
    s->used -= e->bytes;
}

// Create a setup for (key, nrhs) within the remaining budget (lock held).
int make_entry(st_server_s *s, const Key &key, int nrhs, Entry **out) {
    st_options opt = s->o.opt;
    opt.nrhs = nrhs;
    opt.hbm_budget = s->budget > s->used ? s->budget - s->used : 1;
    st_handle h = nullptr;
    int rc = st_setup(&h, key.geometry, key.degree, key.spans, key.slabs, &opt, nullptr);
    if (rc != ST_OK) return rc;
    rc = st::prepare_solve(h);
    size_t hb = 0;
    int64_t n = 0;
    st_sizes(h, &n, nullptr, nullptr, nullptr, &hb);
    const size_t vb = (size_t)n * sizeof(double);
    if (rc == ST_OK && s->used + hb + 2 * vb > s->budget) rc = ST_ERR_OVER_BUDGET;
    std::unique_ptr<Entry> e(new Entry());
    e->key = key;
    e->nrhs = nrhs;
    e->h = h;
    if (rc == ST_OK && (cudaMalloc(&e->f, vb) != cudaSuccess || cudaMalloc(&e->u, vb) != cudaSuccess)) {
        cudaGetLastError();
        rc = ST_ERR_OOM;
    }
    if (rc != ST_OK) {
        e->bytes = 0;
        destroy_entry(s, e.get());
        return rc;
    }
    e->bytes = hb + 2 * vb;
    s->used += e->bytes;
    *out = e.get();
    s->cache.push_back(std::move(e));
    return ST_OK;
}

bool evict_one(st_server_s *s) {
    int best = -1;
    for (int i = 0; i < (int)s->cache.size(); ++i)
        if (!s->cache[i]->busy && (best < 0 || s->cache[i]->last_used < s->cache[best]->last_used))
            best = i;
    if (best < 0) return false;
    destroy_entry(s, s->cache[best].get());
    s->cache.erase(s->cache.begin() + best);
    return true;
}

void finish(st_server_s *s, const std::vector<Pending> &batch, int status, const st_solve_info *info,
            Entry *e, Clock::time_point admitted, const std::vector<std::vector<double>> *u,
            const std::string &msg = std::string()) {
    const auto now = Clock::now();
    for (size_t i = 0; i < batch.size(); ++i) {
        Done &d = s->results[batch[i].ticket];
        d.done = true;
        d.res.status = status;
        d.res.iterations = info ? info->iterations : 0;
        d.res.refinements = info ? info->refinements : 0;
        d.res.rel_residual = info ? info->rel_residual : 0.0;
        d.res.queue_seconds = std::chrono::duration<double>(admitted - batch[i].submitted).count();
        d.res.solve_seconds = std::chrono::duration<double>(now - admitted).count();
        d.res.latency_seconds = std::chrono::duration<double>(now - batch[i].submitted).count();
        d.res.batch_size = (int)batch.size();
        d.res.n_dofs = (int64_t)batch[i].rhs.size();
        std::snprintf(d.res.error, sizeof d.res.error, "%s", status == ST_OK ? "" : msg.c_str());
        if (u) d.u = (*u)[i];
    }
    (void)e;
}

void worker(st_server_s *s) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv.wait(lock, [s] { return s->stop || !s->pending.empty(); });
        if (s->pending.empty()) {
            if (s->stop) break;
            continue;
        }
        // the oldest request and up to max_batch - 1 more of the same configuration
        const Key key = s->pending.front().key;
        std::vector<Pending> batch;
        for (auto it = s->pending.begin(); it != s->pending.end() && (int)batch.size() < s->o.max_batch;) {
            if (std::memcmp(&it->key, &key, sizeof(Key)) == 0) {
                batch.push_back(std::move(*it));
                it = s->pending.erase(it);
            } else {
                ++it;
            }
        }
        const int R = (int)batch.size();
        // find or create a setup
        Entry *e = nullptr;
        int rc = ST_OK;
        std::string why;
        for (;;) {
            e = nullptr;
            for (auto &c : s->cache)
                if (!c->busy && c->nrhs == R && c->key.same_problem(key)) {
                    e = c.get();
                    break;
                }
            if (e) {  // a cached setup (possibly freed while this worker waited)
                rc = ST_OK;
                break;
            }
            rc = make_entry(s, key, R, &e);
            if (rc == ST_OK) break;
            why = std::string("setup: ") + st_last_error();
            if (rc != ST_ERR_OVER_BUDGET && rc != ST_ERR_OOM) break;
            if (evict_one(s)) continue;
            if (s->busy_workers > 0) {  // wait for running solves to release memory
                s->cv.wait(lock);
                continue;
            }
            rc = ST_ERR_OVER_BUDGET;
            char buf[200];
            std::snprintf(buf, sizeof buf, "does not fit the HBM budget (%zu of %zu bytes held; %s)",
                          s->used, s->budget, why.c_str());
            why = buf;
            break;
        }
        if (rc != ST_OK) {
            finish(s, batch, rc, nullptr, nullptr, Clock::now(), nullptr, why);
            s->cv.notify_all();
            continue;
        }
        e->busy = true;
        e->last_used = ++s->clock;
        ++s->busy_workers;
        const auto admitted = Clock::now();
        lock.unlock();

        // ---- solve (no lock held) ----
        const int64_t n1 = (int64_t)batch[0].rhs.size();
        st_solve_info info{};
        std::vector<std::vector<double>> u(R, std::vector<double>(n1));
        int st = st_set_stream(e->h, stream);
        double *in = key.coeffs ? e->u : e->f;
        for (int r = 0; r < R && st == ST_OK; ++r)
            if (cudaMemcpyAsync(in + r * n1, batch[r].rhs.data(), n1 * sizeof(double),
                                cudaMemcpyHostToDevice, stream) != cudaSuccess)
                st = ST_ERR_CUDA;
        if (st == ST_OK && key.coeffs) st = st_load_coeffs(e->h, e->u, e->f);
        if (st == ST_OK) st = st_solve(e->h, e->f, key.tol, e->u, 0, &info);
        if (st == ST_OK || st == ST_ERR_NO_CONVERGENCE) {
            for (int r = 0; r < R; ++r)
                if (cudaMemcpyAsync(u[r].data(), e->u + r * n1, n1 * sizeof(double),
                                    cudaMemcpyDeviceToHost, stream) != cudaSuccess)
                    st = ST_ERR_CUDA;
            if (cudaStreamSynchronize(stream) != cudaSuccess) st = ST_ERR_CUDA;
        }
        if (st == ST_ERR_CUDA) cudaGetLastError();

        const std::string solve_msg = (st == ST_OK) ? std::string() : std::string(st_last_error());
        lock.lock();
        finish(s, batch, st, &info, e, admitted, &u, solve_msg);
        e->busy = false;
        --s->busy_workers;
        s->cv.notify_all();
    }
    lock.unlock();
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void st_serve_opts_default(st_server_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->workers = 4;
    o->max_batch = 8;
    st_options_default(&o->opt);
}

int st_serve_start(st_server *out, const st_server_opts *o) {
    if (!out) return ST_ERR_INVALID_ARG;
    *out = nullptr;
    st_server_opts oo;
    if (o) oo = *o; else st_serve_opts_default(&oo);
    if (oo.workers < 1 || oo.workers > 64 || oo.max_batch < 1 || oo.max_batch > 32)
        return ST_ERR_INVALID_ARG;
    st_server_s *s = new st_server_s();
    s->o = oo;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return ST_ERR_CUDA;
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return ST_ERR_CUDA;
    }
    s->budget = oo.hbm_budget ? oo.hbm_budget : (size_t)(0.9 * (double)fr);
    for (int i = 0; i < oo.workers; ++i) s->threads.emplace_back(worker, s);
    *out = s;
    return ST_OK;
}

int st_serve_submit(st_server s, const st_request *req, uint64_t *ticket) {
    if (!s || !req || !req->rhs || !ticket) return ST_ERR_INVALID_ARG;
    if (req->geometry < 1 || req->geometry > 3 || req->degree < 1 || req->slabs < 1 ||
        !(req->tol > 0))
        return ST_ERR_INVALID_ARG;
    if (req->degree > 3) return ST_ERR_UNSUPPORTED;
    Key k;
    zero_key(k);
    k.geometry = req->geometry;
    k.degree = req->degree;
    int64_t nx = 1;
    for (int a = 0; a < 3; ++a) {
        k.spans[a] = a < req->geometry ? req->spans[a] : 1;
        if (a < req->geometry) {
            if (req->spans[a] < 2) return ST_ERR_INVALID_ARG;
            nx *= req->spans[a] + req->degree - 2;
        }
    }
    k.slabs = req->slabs;
    k.tol = req->tol;
    k.coeffs = req->rhs_is_coeffs ? 1 : 0;
    const int64_t n = (int64_t)req->slabs * (s->o.opt.ne_per_slab + req->degree) * nx;
    Pending p;
    p.key = k;
    p.rhs.assign(req->rhs, req->rhs + n);
    p.submitted = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return ST_ERR_INVALID_ARG;
        p.ticket = s->next_ticket++;
        *ticket = p.ticket;
        s->results[p.ticket].submitted = p.submitted;
        s->pending.push_back(std::move(p));
    }
    s->cv.notify_all();
    return ST_OK;
}

static int take_result(st_server s, uint64_t ticket, st_result *res, double *u_host) {
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return ST_ERR_INVALID_ARG;
    if (!it->second.done) return ST_ERR_NOT_READY;
    if (res) *res = it->second.res;
    if (u_host && !it->second.u.empty())
        std::memcpy(u_host, it->second.u.data(), it->second.u.size() * sizeof(double));
    s->results.erase(it);
    return ST_OK;
}

int st_serve_poll(st_server s, uint64_t ticket, st_result *res, double *u_host) {
    if (!s) return ST_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    return take_result(s, ticket, res, u_host);
}

int st_serve_wait(st_server s, uint64_t ticket, double timeout_s, st_result *res, double *u_host) {
    if (!s) return ST_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto ready = [&] {
        auto it = s->results.find(ticket);
        return it == s->results.end() || it->second.done;
    };
    if (timeout_s < 0)
        s->cv.wait(lock, ready);
    else
        s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), ready);
    return take_result(s, ticket, res, u_host);
}

int st_serve_stop(st_server s) {
    if (!s) return ST_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto &t : s->threads) t.join();
    for (auto &e : s->cache) destroy_entry(s, e.get());
    s->cache.clear();
    delete s;
    return ST_OK;
}

}  // extern "C"
