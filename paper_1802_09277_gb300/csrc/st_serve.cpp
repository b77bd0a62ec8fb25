// Serving loop with continuous batching (see st_serve_* in include/st_iga.h).
//
// Host-side scheduler only: every solve goes through st_setup / st_solve of
// this library on the worker's own CUDA stream.  The server mutex guards the
// queue, the result table, the setup cache and the budget accounting; it is
// never held across a host factorisation, a device allocation or free, or a
// solve, so submit / poll / wait and the other workers' admissions never wait
// for one worker's setup.
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
#include <utility>
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

// a setup is shared by every request of the same problem (the tolerance and
// the kind of right-hand side only matter to the solve)
struct ShapeKey {
    int geometry, degree, spans[3], slabs, nrhs;
    bool operator<(const ShapeKey &o) const {
        return std::memcmp(this, &o, sizeof(ShapeKey)) < 0;
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
    bool running = false;
    st_result res{};
    std::vector<double> u;
    Clock::time_point submitted;
};

struct Entry {  // a cached setup for one configuration and batch-size class
    Key key;
    int nrhs = 1;  // a power of two: batches of nrhs/2 + 1 .. nrhs requests share it
    st_handle h = nullptr;
    double *f = nullptr, *u = nullptr;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_used = 0;
};

void zero_key(Key &k) { std::memset(&k, 0, sizeof k); }

ShapeKey shape_of(const Key &k, int nrhs) {
    ShapeKey s;
    std::memset(&s, 0, sizeof s);
    s.geometry = k.geometry;
    s.degree = k.degree;
    for (int a = 0; a < 3; ++a) s.spans[a] = k.spans[a];
    s.slabs = k.slabs;
    s.nrhs = nrhs;
    return s;
}

}  // namespace

struct st_server_s {
    st_server_opts o{};
    int device = 0;
    // every setup's device memory comes from this stream-ordered pool, so that
    // releasing a setup never synchronises the whole device (cudaFree would)
    cudaMemPool_t pool = nullptr;
    size_t budget = 0;
    size_t used = 0;      // bytes held by cached setups plus reservations of setups being built
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    std::map<uint64_t, Done> results;
    std::vector<std::unique_ptr<Entry>> cache;
    std::map<ShapeKey, size_t> footprint;  // measured device bytes of a setup + its two vectors
    std::vector<std::thread> threads;
    uint64_t next_ticket = 1, clock = 0;
    int busy_workers = 0;  // solving, building a setup or freeing one
    bool paused = false;
    bool stop = false;
};

namespace {

// Returns an idle entry's device memory to the pool, stream-ordered on
// `stream` (its last solve has completed: the worker synchronised its stream).
void free_entry(Entry *e, cudaStream_t stream) {
    if (e->h) {
        st_set_stream(e->h, stream);
        st_destroy(e->h);
    }
    if (e->f) cudaFreeAsync(e->f, stream);
    if (e->u) cudaFreeAsync(e->u, stream);
    e->h = nullptr;
    e->f = e->u = nullptr;
}

// the batch-size class: the next power of two (setups are shared by the
// batch sizes of one class; the unused right-hand sides are zero)
int size_class(int R) {
    int c = 1;
    while (c < R) c *= 2;
    return c;
}

// First guess of a setup's device bytes before one of its shape was built:
// the Krylov space and the level vectors dominate.  Deliberately generous; the
// reservation is trimmed to the measured size once the setup exists.
size_t guess_bytes(const st_server_s *s, const Key &k, int nrhs) {
    int64_t nx = 1;
    for (int a = 0; a < k.geometry; ++a) nx *= k.spans[a] + k.degree - 2;
    const double n = (double)k.slabs * (s->o.opt.ne_per_slab + k.degree) * nx * nrhs;
    const int m = s->o.opt.gmres_restart > 0 ? s->o.opt.gmres_restart : 20;
    // 2m+1 Krylov vectors (counted as FP64), level vectors and work space
    // (about 8 more), the request's two FP64 vectors, factors and tables
    return (size_t)(8.0 * n * (2.0 * m + 1.0 + 8.0 + 2.0)) + ((size_t)32 << 20);
}

// Builds a setup for (key, nrhs) whose device memory stays within `limit`
// bytes (setup, Krylov space and the two request vectors).  No lock held.
int build_entry(st_server_s *s, const Key &key, int nrhs, size_t limit, cudaStream_t stream,
                Entry **out, std::string *why) {
    st_options opt = s->o.opt;
    opt.nrhs = nrhs;
    int64_t nx = 1;
    for (int a = 0; a < key.geometry; ++a) nx *= key.spans[a] + key.degree - 2;
    const size_t vb = (size_t)key.slabs * (opt.ne_per_slab + key.degree) * nx * nrhs * sizeof(double);
    if (limit <= 2 * vb) {
        *why = "the request's vectors alone exceed the reservation";
        return ST_ERR_OVER_BUDGET;
    }
    opt.hbm_budget = limit - 2 * vb;
    cudaSetDevice(s->device);
    std::unique_ptr<Entry> e(new Entry());
    e->key = key;
    e->nrhs = nrhs;
    int rc = st::setup_pooled(&e->h, key.geometry, key.degree, key.spans, key.slabs, &opt, stream,
                              s->pool);
    if (rc == ST_OK) rc = st::prepare_solve(e->h);
    if (rc == ST_OK) {
        void *pf = nullptr, *pu = nullptr;
        if (cudaMallocFromPoolAsync(&pf, vb, s->pool, stream) != cudaSuccess ||
            cudaMallocFromPoolAsync(&pu, vb, s->pool, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            cudaGetLastError();
            rc = ST_ERR_OOM;
        }
        e->f = static_cast<double *>(pf);
        e->u = static_cast<double *>(pu);
    }
    if (rc != ST_OK) {
        *why = std::string("setup: ") + st_last_error();
        free_entry(e.get(), stream);
        cudaStreamSynchronize(stream);
        return rc;
    }
    size_t hb = 0;
    st_sizes(e->h, nullptr, nullptr, nullptr, nullptr, &hb);
    e->bytes = hb + 2 * vb;
    *out = e.release();
    return ST_OK;
}

void finish(st_server_s *s, const std::vector<Pending> &batch, int status, const st_solve_info *info,
            Clock::time_point admitted, const std::vector<std::vector<double>> *u,
            const std::string &msg = std::string(), int group_requests = 0) {
    const auto now = Clock::now();
    for (size_t i = 0; i < batch.size(); ++i) {
        Done &d = s->results[batch[i].ticket];
        d.done = true;
        d.running = false;
        d.res.status = status;
        d.res.iterations = info ? info->iterations : 0;
        d.res.refinements = info ? info->refinements : 0;
        d.res.rel_residual = info ? info->rel_residual : 0.0;
        d.res.queue_seconds = std::chrono::duration<double>(admitted - batch[i].submitted).count();
        d.res.solve_seconds = std::chrono::duration<double>(now - admitted).count();
        d.res.latency_seconds = std::chrono::duration<double>(now - batch[i].submitted).count();
        d.res.batch_size = (int)batch.size();
        d.res.n_dofs = (int64_t)batch[i].rhs.size();
        d.res.group_requests = group_requests > 0 ? group_requests : (int)batch.size();
        d.res.host_syncs = info ? info->host_syncs : 0;
        d.res.vector_launches = info ? info->vector_launches : 0;
        std::snprintf(d.res.error, sizeof d.res.error, "%s", status == ST_OK ? "" : msg.c_str());
        if (u) d.u = (*u)[i];
    }
}

// Finds or builds a setup for the batch (lock held on entry and on return; it
// is released while a setup is built or an evicted one is freed).  On success
// the entry is marked busy.
int acquire_entry(st_server_s *s, std::unique_lock<std::mutex> &lock, const Key &key, int R,
                  cudaStream_t stream, Entry **out, std::string *why, bool may_wait = true) {
    const ShapeKey sk = shape_of(key, R);
    for (;;) {
        for (auto &c : s->cache)
            if (!c->busy && c->nrhs == R && c->key.same_problem(key)) {
                c->busy = true;
                *out = c.get();
                return ST_OK;
            }
        auto fp = s->footprint.find(sk);
        size_t want = fp != s->footprint.end() ? fp->second : guess_bytes(s, key, R);
        const size_t avail = s->budget > s->used ? s->budget - s->used : 0;
        const bool idle = s->busy_workers == 0;
        const bool any_free = std::any_of(s->cache.begin(), s->cache.end(),
                                          [](const std::unique_ptr<Entry> &c) { return !c->busy; });
        // an idle server with nothing to evict tries whatever is left (the
        // guess may be too generous)
        if (want > avail && idle && !any_free) want = avail;
        if (want <= avail && want > 0) {
            s->used += want;  // reserve, then build without the lock
            ++s->busy_workers;
            lock.unlock();
            Entry *e = nullptr;
            std::string msg;
            const int rc = build_entry(s, key, R, want, stream, &e, &msg);
            lock.lock();
            --s->busy_workers;
            s->used -= want;
            if (rc == ST_OK) {
                s->used += e->bytes;
                s->footprint[sk] = e->bytes;
                e->busy = true;
                s->cache.emplace_back(e);
                *out = e;
                s->cv.notify_all();
                return ST_OK;
            }
            s->cv.notify_all();
            if (rc != ST_ERR_OVER_BUDGET && rc != ST_ERR_OOM) {
                *why = msg;
                return rc;
            }
            if (want >= s->budget || (want == avail && idle && !any_free)) {
                char buf[200];
                std::snprintf(buf, sizeof buf, "does not fit the HBM budget (%zu bytes; %s)",
                              s->budget, msg.c_str());
                *why = buf;
                return ST_ERR_OVER_BUDGET;
            }
            // the setup needed more than reserved: reserve more next time
            s->footprint[sk] = std::min(s->budget, 2 * want);
            continue;
        }
        // make room: evict the least recently used idle setup, freeing it
        // without the lock (its bytes stay counted until they are freed)
        int best = -1;
        for (int i = 0; i < (int)s->cache.size(); ++i)
            if (!s->cache[i]->busy &&
                (best < 0 || s->cache[i]->last_used < s->cache[best]->last_used))
                best = i;
        if (best >= 0) {
            std::unique_ptr<Entry> victim = std::move(s->cache[best]);
            s->cache.erase(s->cache.begin() + best);
            ++s->busy_workers;
            lock.unlock();
            free_entry(victim.get(), stream);
            lock.lock();
            --s->busy_workers;
            s->used -= victim->bytes;
            s->cv.notify_all();
            continue;
        }
        if (s->busy_workers > 0) {  // wait for running work to release memory
            if (!may_wait) {
                *why = "no room now";
                return ST_ERR_NOT_READY;
            }
            s->cv.wait(lock);
            continue;
        }
        char buf[200];
        std::snprintf(buf, sizeof buf, "does not fit the HBM budget (%zu of %zu bytes held)", s->used,
                      s->budget);
        *why = buf;
        return ST_ERR_OVER_BUDGET;
    }
}

// one configuration's share of a solve call: its requests and its setup
struct Member {
    Key key;
    std::vector<Pending> batch;
    int R = 0, RC = 0;
    Entry *e = nullptr;
};

// back into the queue in submission order (lock held)
void requeue(st_server_s *s, std::vector<Pending> &batch) {
    for (Pending &p : batch) {
        s->results[p.ticket].running = false;
        auto at = std::upper_bound(s->pending.begin(), s->pending.end(), p.ticket,
                                   [](uint64_t t, const Pending &q) { return t < q.ticket; });
        s->pending.insert(at, std::move(p));
    }
    batch.clear();
}

// configurations are solved together (st_solve_group) when the server's
// solver is the mixed-precision refinement
bool grouping(const st_server_s *s) {
    return s->o.group_members > 1 && s->o.opt.precision != ST_FP64 &&
           s->o.opt.outer == ST_OUTER_IR;
}

void worker(st_server_s *s) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv.wait(lock, [s] { return s->stop || (!s->paused && !s->pending.empty()); });
        if (s->pending.empty()) {
            if (s->stop) break;
            continue;
        }
        // the oldest request and up to max_batch - 1 more of the same
        // configuration; for a group solve, then the same for further
        // configurations (oldest first) while the group stays within its
        // right-hand-side and dofs limits
        std::vector<Member> mem;
        std::vector<Key> tried;
        const int gmax = grouping(s) ? std::min(s->o.group_members, st::GH) : 1;
        const double tol0 = s->pending.front().key.tol;
        const long long n0 = (long long)s->pending.front().rhs.size();
        long long gdofs = 0;
        int gsys = 0;
        // takes the requests of the oldest configuration not yet tried into
        // m (false: none left)
        auto form = [&](Member &m) {
            for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
                const Key key = it->key;
                // a group never waits for a larger problem than its oldest
                // request's (it runs at the pace of its slowest member)
                bool skip = !mem.empty() && (key.tol != tol0 || (long long)it->rhs.size() > n0);
                for (const Member &o : mem) skip = skip || o.key.same_problem(key);
                for (const Key &k : tried) skip = skip || std::memcmp(&k, &key, sizeof(Key)) == 0;
                if (skip) continue;
                tried.push_back(key);
                m = Member();
                m.key = key;
                long long dofs = 0;
                for (auto jt = s->pending.begin();
                     jt != s->pending.end() && (int)m.batch.size() < s->o.max_batch;) {
                    const long long n = (long long)jt->rhs.size();
                    bool take = std::memcmp(&jt->key, &key, sizeof(Key)) == 0;
                    if (take && !(mem.empty() && m.batch.empty()))  // the oldest always runs
                        take = (s->o.batch_dofs <= 0 || gdofs + dofs + n <= s->o.batch_dofs) &&
                               gsys + size_class((int)m.batch.size() + 1) <= st::NSYS_MAX;
                    if (take) {
                        dofs += n;
                        s->results[jt->ticket].running = true;
                        m.batch.push_back(std::move(*jt));
                        jt = s->pending.erase(jt);
                    } else {
                        ++jt;
                    }
                }
                if (m.batch.empty()) continue;  // its oldest request does not fit
                m.R = (int)m.batch.size();
                m.RC = size_class(m.R);
                return true;
            }
            return false;
        };
        // the first configuration may wait for memory; the others join only
        // if their setup is at hand now, else they go back to the queue
        bool failed0 = false;
        for (;;) {
            if ((int)mem.size() >= gmax) break;
            Member m;
            if (!form(m)) break;
            std::string why;
            const bool first = mem.empty();
            const int rc = acquire_entry(s, lock, m.key, m.RC, stream, &m.e, &why, first);
            if (rc != ST_OK) {
                if (first) {
                    finish(s, m.batch, rc, nullptr, Clock::now(), nullptr, why);
                    failed0 = true;
                    break;
                }
                requeue(s, m.batch);
                continue;
            }
            m.e->last_used = ++s->clock;
            for (const Pending &p : m.batch) gdofs += (long long)p.rhs.size();
            gsys += m.RC;
            mem.push_back(std::move(m));
        }
        if (failed0 || mem.empty()) {
            s->cv.notify_all();
            continue;
        }
        ++s->busy_workers;
        const auto admitted = Clock::now();
        lock.unlock();

        // ---- solve (no lock held) ----
        const int nm = (int)mem.size();
        std::vector<st_solve_info> infos(nm);
        std::vector<std::vector<std::vector<double>>> us(nm);
        int st = ST_OK;
        for (int i = 0; i < nm && st == ST_OK; ++i) {
            Member &m = mem[i];
            Entry *e = m.e;
            const int64_t n1 = (int64_t)m.batch[0].rhs.size();
            us[i].assign(m.R, std::vector<double>(n1));
            st = st_set_stream(e->h, stream);
            double *in = m.key.coeffs ? e->u : e->f;
            for (int r = 0; r < m.R && st == ST_OK; ++r)
                if (cudaMemcpyAsync(in + r * n1, m.batch[r].rhs.data(), n1 * sizeof(double),
                                    cudaMemcpyHostToDevice, stream) != cudaSuccess)
                    st = ST_ERR_CUDA;
            if (st == ST_OK && m.RC > m.R &&
                cudaMemsetAsync(in + m.R * n1, 0, (size_t)(m.RC - m.R) * n1 * sizeof(double),
                                stream) != cudaSuccess)
                st = ST_ERR_CUDA;
            if (st == ST_OK && m.key.coeffs) st = st_load_coeffs(e->h, e->u, e->f);
        }
        if (st == ST_OK) {
            if (nm == 1) {
                st = st_solve(mem[0].e->h, mem[0].e->f, tol0, mem[0].e->u, 0, &infos[0]);
            } else {
                std::vector<st_handle> hs(nm);
                std::vector<const double *> fs(nm);
                std::vector<double *> uu(nm);
                for (int i = 0; i < nm; ++i) {
                    hs[i] = mem[i].e->h;
                    fs[i] = mem[i].e->f;
                    uu[i] = mem[i].e->u;
                }
                st = st_solve_group(nm, hs.data(), fs.data(), tol0, uu.data(), 0, infos.data());
            }
        }
        if (st == ST_OK || st == ST_ERR_NO_CONVERGENCE) {
            for (int i = 0; i < nm; ++i) {
                const int64_t n1 = (int64_t)mem[i].batch[0].rhs.size();
                for (int r = 0; r < mem[i].R; ++r)
                    if (cudaMemcpyAsync(us[i][r].data(), mem[i].e->u + r * n1, n1 * sizeof(double),
                                        cudaMemcpyDeviceToHost, stream) != cudaSuccess)
                        st = ST_ERR_CUDA;
            }
            if (cudaStreamSynchronize(stream) != cudaSuccess) st = ST_ERR_CUDA;
        }
        if (st == ST_ERR_CUDA) cudaGetLastError();

        const std::string solve_msg = (st == ST_OK) ? std::string() : std::string(st_last_error());
        int greq = 0;
        for (const Member &m : mem) greq += m.R;
        lock.lock();
        for (int i = 0; i < nm; ++i) {
            const bool ran = st == ST_OK || st == ST_ERR_NO_CONVERGENCE;
            const int status = ran ? infos[i].status : st;
            finish(s, mem[i].batch, status, &infos[i], admitted, &us[i],
                   status == ST_OK ? std::string() : solve_msg, greq);
            mem[i].e->busy = false;
        }
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
    o->start_paused = 0;
    o->batch_dofs = 8388608;
    o->group_members = 8;
    st_options_default(&o->opt);
    // per-setup kernel tuning would time candidate kernels for every new
    // configuration on the serving path
    o->opt.autotune = 0;
}

int st_serve_start(st_server *out, const st_server_opts *o) {
    if (!out) return ST_ERR_INVALID_ARG;
    *out = nullptr;
    st_server_opts oo;
    if (o) oo = *o; else st_serve_opts_default(&oo);
    if (oo.workers < 1 || oo.workers > 64 || oo.max_batch < 1 || oo.max_batch > 32 ||
        oo.group_members < 0)
        return ST_ERR_INVALID_ARG;
    st_server_s *s = new st_server_s();
    s->o = oo;
    s->paused = oo.start_paused != 0;
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
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return ST_ERR_CUDA;
    }
    // keep released memory in the pool (no return to the driver between setups)
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int i = 0; i < oo.workers; ++i) s->threads.emplace_back(worker, s);
    *out = s;
    return ST_OK;
}

int st_serve_pause(st_server s) {
    if (!s) return ST_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->paused = true;  // batches already taken run to the end
    return ST_OK;
}

int st_serve_resume(st_server s) {
    if (!s) return ST_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->paused = false;
    }
    s->cv.notify_all();
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

int st_serve_cancel(st_server s, uint64_t ticket) {
    if (!s) return ST_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto r = s->results.find(ticket);
    if (r == s->results.end() || r->second.done) return ST_ERR_INVALID_ARG;
    if (r->second.running) return ST_ERR_NOT_READY;
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
        if (it->ticket == ticket) {
            std::vector<Pending> one;
            one.push_back(std::move(*it));
            s->pending.erase(it);
            finish(s, one, ST_ERR_CANCELLED, nullptr, Clock::now(), nullptr, "cancelled");
            s->cv.notify_all();
            return ST_OK;
        }
    return ST_ERR_INVALID_ARG;
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
        s->paused = false;  // queued work is finished before the workers exit
    }
    s->cv.notify_all();
    for (auto &t : s->threads) t.join();
    for (auto &e : s->cache) free_entry(e.get(), nullptr);
    s->cache.clear();
    cudaStreamSynchronize(nullptr);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return ST_OK;
}

}  // extern "C"
