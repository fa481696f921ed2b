// serve.cu -- npb_submit / npb_poll: continuous batching of RE+V solves.
//
// One scheduler thread per context owns a serving stream and loops:
//   1. admit   queued requests in arrival order while their device footprint fits the
//              context's budget (a request whose footprint alone exceeds it fails with
//              NPB_ENOMEM); each admitted request gets a grid built on a separate set-up
//              stream, and the serving stream waits on an event before it first touches it;
//   2. step    every active leg of every admitted request advances one LOD step; legs of
//              equal grid size, precision, scheme and eps reading share the same launches,
//              so requests that arrive while others run join the running batch;
//   3. retire  a request whose legs are done gets its energy reduction and an event; when the
//              event completes its result is posted and its grid freed, returning memory to
//              admission.
// At most kLookahead iterations are in flight on the device, so a new arrival waits for a
// bounded amount of queued work before it joins.  Each leg's arithmetic is independent of
// which other legs share its launches (the solver shape depends only on precision,
// direction and line length), so a result is bit-identical alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "runtime.h"

using namespace npb;

namespace npb {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    std::vector<double> xyz, q, radius;
    npb_problem prob{};
    npb_opts opts{};
    Clock::time_point t_submit, t_admit;
};

struct Active {
    Request *r = nullptr;
    npb_grid *g = nullptr;
    int iter = 0;         // LOD steps taken by the dt/2 legs
    int total = 0;        // 2n with Richardson, else n
    bool finishing = false;
    cudaEvent_t done{};
};

struct Table {  // device LegDev table of one launch group
    LegDev *d = nullptr;
    size_t cap = 0;
    std::vector<LegDev> host;
};

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::map<uint64_t, npb_result> done;
    std::map<uint64_t, bool> known;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;  // steps and energies
    cudaStream_t setup = nullptr;   // grid set-up of admitted requests
    std::map<std::tuple<int, int, int, int, int, int>, Table> tables;
};

static constexpr int kLookahead = 4;

static double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

static void post(ServeState *s, Request *r, int status, double dG) {
    npb_result res{};
    const auto now = Clock::now();
    res.dG_kcal_mol = dG;
    res.status = status;
    res.wall_ms = ms_between(r->t_submit, now);
    res.queue_ms = ms_between(r->t_submit, r->t_admit.time_since_epoch().count() ? r->t_admit : now);
    for (int d = 0; d < 3; ++d) res.n[d] = r->prob.n[d];
    const int64_t inner = (int64_t)(r->prob.n[0] - 2) * (r->prob.n[1] - 2) * (r->prob.n[2] - 2);
    res.point_steps = status == NPB_OK ? inner * (int64_t)r->opts.n_steps * (r->opts.richardson ? 6 : 2) : 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->done[r->ticket] = res;
    }
    s->cv_done.notify_all();
}

static int table_for(npb_ctx *ctx, Table &t, const std::vector<LegDev> &legs, cudaStream_t st) {
    if (t.cap < legs.size()) {
        if (t.d) {
            cudaStreamSynchronize(st);
            ctx->release(t.d, t.cap * sizeof(LegDev));
            t.d = nullptr;
        }
        const size_t cap = std::max<size_t>(16, legs.size() * 2);
        void *p = nullptr;
        int rc = ctx->alloc(&p, cap * sizeof(LegDev));
        if (rc) return rc;
        t.d = static_cast<LegDev *>(p);
        t.cap = cap;
        t.host.clear();
    }
    const bool same = t.host.size() == legs.size() &&
                      std::memcmp(t.host.data(), legs.data(), legs.size() * sizeof(LegDev)) == 0;
    if (!same) {
        t.host = legs;  // pageable source: the copy has consumed it when the call returns
        cudaError_t e = cudaMemcpyAsync(t.d, t.host.data(), legs.size() * sizeof(LegDev), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(NPB_ECUDA, "leg table upload failed: %s", cudaGetErrorString(e));
    }
    return 0;
}

// Admit one request: build and prepare its grid on the set-up stream, start its legs.
static int admit(npb_ctx *ctx, ServeState *s, Request *r, Active &a) {
    npb_grid *g = nullptr;
    int rc = grid_build(ctx, &r->prob, s->setup, &g);
    if (rc) return rc;
    if ((rc = grid_prepare(g, &r->opts, s->setup)) == 0) {
        const int re = r->opts.richardson ? 1 : 0;
        const int legs_re[4] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_SOLVENT_HALF, NPB_LEG_VACUUM_TAU, NPB_LEG_VACUUM_HALF};
        const int legs_plain[2] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_VACUUM_TAU};
        rc = init_legs(g, r->opts.precision, re ? legs_re : legs_plain, re ? 4 : 2, s->setup);
    }
    cudaEvent_t ready;
    if (rc == 0 && cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ready, s->setup);
        cudaStreamWaitEvent(s->stream, ready, 0);
        cudaEventDestroy(ready);
    } else if (rc == 0) {
        rc = fail(NPB_ECUDA, "cannot create an event");
    }
    if (rc) {
        cudaStreamSynchronize(s->setup);
        grid_free(g);
        return rc;
    }
    a.r = r;
    a.g = g;
    a.iter = 0;
    a.total = r->opts.richardson ? 2 * r->opts.n_steps : r->opts.n_steps;
    return 0;
}

static void serve_loop(npb_ctx *ctx, ServeState *s) {
    cudaSetDevice(ctx->device);
    std::vector<Active> active;
    std::deque<cudaEvent_t> inflight;
    for (;;) {
        // ---- 1. admission
        std::vector<Request *> fresh;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (active.empty() && s->queue.empty())
                s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop && s->queue.empty() && active.empty()) break;
            size_t planned = 0;  // footprints admitted in this pass, not yet allocated
            while (!s->queue.empty()) {
                Request *r = s->queue.front();
                const size_t fp = npb_grid_footprint(&r->prob, r->opts.precision);
                if (ctx->in_use.load() + planned + fp > ctx->budget) {
                    if (!active.empty() || planned > 0) break;  // wait for memory to come back
                    if (fp > ctx->budget) {      // can never fit
                        s->queue.pop_front();
                        r->t_admit = Clock::now();
                        lk.unlock();
                        fail(NPB_ENOMEM, "request needs %zu bytes, budget is %zu", fp, ctx->budget);
                        post(s, r, NPB_ENOMEM, 0.0);
                        delete r;
                        lk.lock();
                        continue;
                    }
                }
                s->queue.pop_front();
                fresh.push_back(r);
                planned += fp;
            }
        }
        for (Request *r : fresh) {
            r->t_admit = Clock::now();
            Active a;
            const int rc = admit(ctx, s, r, a);
            if (rc) {
                post(s, r, rc, 0.0);
                delete r;
                continue;
            }
            active.push_back(a);
        }

        // ---- 2. one LOD step for every running leg, grouped into shared launches
        std::map<std::tuple<int, int, int, int, int, int>, std::vector<LegRef>> groups;
        for (Active &a : active) {
            if (a.finishing) continue;
            const npb_opts &o = a.r->opts;
            auto key = std::make_tuple(a.g->geo.nx, a.g->geo.ny, a.g->geo.nz, o.precision, o.scheme, o.eps_mode);
            auto &refs = groups[key];
            // dt/2 legs run 2n steps, dt legs n (slots: s_half 0, v_half 1, s_tau 2, v_tau 3)
            if (o.richardson) {
                refs.push_back({a.g, 0});
                refs.push_back({a.g, 1});
                if (a.iter < o.n_steps) {
                    refs.push_back({a.g, 2});
                    refs.push_back({a.g, 3});
                }
            } else {
                refs.push_back({a.g, 2});
                refs.push_back({a.g, 3});
            }
        }
        int err = 0;
        for (auto &kv : groups) {
            const int prec = std::get<3>(kv.first), scheme = std::get<4>(kv.first);
            std::vector<LegDev> legs;
            legs.reserve(kv.second.size());
            for (const LegRef &r : kv.second) legs.push_back(r.g->h_legs[prec][r.slot]);
            Table &t = s->tables[kv.first];
            err = table_for(ctx, t, legs, s->stream);
            if (!err) err = step_legs(ctx, kv.second.data(), (int)kv.second.size(), t.d, prec, scheme, s->stream);
            if (err) break;
        }
        for (Active &a : active) {
            if (a.finishing) continue;
            if (err) {  // a launch failed: fail the running requests
                a.finishing = true;
                a.iter = -1;
                continue;
            }
            if (++a.iter >= a.total) {
                a.finishing = true;
                int rc = enqueue_energy_reduce(a.g, a.r->opts.precision, a.r->opts.richardson, s->stream);
                if (rc == 0 && cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming) == cudaSuccess)
                    cudaEventRecord(a.done, s->stream);
                else
                    a.iter = -1;
            }
        }
        // bound the work queued on the device
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, s->stream);
            inflight.push_back(ev);
        }
        while ((int)inflight.size() > kLookahead) {
            cudaEventSynchronize(inflight.front());
            cudaEventDestroy(inflight.front());
            inflight.pop_front();
        }

        // ---- 3. retire finished requests
        const bool idle = groups.empty();
        for (size_t i = 0; i < active.size();) {
            Active &a = active[i];
            bool ready = false;
            if (a.finishing) {
                if (a.iter < 0) {
                    cudaStreamSynchronize(s->stream);
                    ready = true;
                } else {
                    cudaError_t q = idle ? cudaEventSynchronize(a.done) : cudaEventQuery(a.done);
                    ready = q == cudaSuccess || (q != cudaErrorNotReady);
                }
            }
            if (!ready) {
                ++i;
                continue;
            }
            int status = NPB_OK;
            double dG = 0.0;
            if (a.iter < 0) {
                status = NPB_ECUDA;
            } else {
                cudaEventDestroy(a.done);
                if (*reinterpret_cast<int32_t *>(a.g->h_result + 1)) status = NPB_ETIMEOUT;
                dG = a.g->h_result[0];
            }
            post(s, a.r, status, dG);
            grid_free(a.g);
            delete a.r;
            active.erase(active.begin() + i);
        }
    }
    for (cudaEvent_t e : inflight) cudaEventDestroy(e);
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->tables)
        if (kv.second.d) ctx->release(kv.second.d, kv.second.cap * sizeof(LegDev));
    s->tables.clear();
}

void serve_shutdown(npb_ctx *ctx) {
    ServeState *s = ctx->serve;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Request *r : s->queue) delete r;
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->setup) cudaStreamDestroy(s->setup);
    delete s;
    ctx->serve = nullptr;
}

static std::mutex g_serve_init;

static int serve_start(npb_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_serve_init);
    if (ctx->serve) return 0;
    auto *s = new ServeState();
    cudaSetDevice(ctx->device);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return fail(NPB_ECUDA, "cannot create the serving streams");
    }
    ctx->serve = s;
    s->worker = std::thread(serve_loop, ctx, s);
    return 0;
}

}  // namespace npb

extern "C" int npb_submit(npb_ctx *ctx, const npb_problem *p, const npb_opts *o, uint64_t *ticket) {
    if (!ctx || !p || !o || !ticket) return fail(NPB_EINVAL, "NULL argument");
    if (p->n_atoms < 0 || (p->n_atoms > 0 && (!p->xyz || !p->q || !p->radius)))
        return fail(NPB_EINVAL, "bad atom arrays");
    if (!(o->dt > 0) || !(o->alpha > 0) || o->n_steps < 0 || !o->vacuum_recovery ||
        (o->scheme < NPB_LODIE1 || o->scheme > NPB_LODCN2) ||
        (o->precision != NPB_FP64 && o->precision != NPB_FP32_SWEEP) ||
        (o->eps_mode != NPB_EPS_HARMONIC && o->eps_mode != NPB_EPS_MIDPOINT))
        return fail(NPB_EINVAL, "invalid options");
    int rc = serve_start(ctx);
    if (rc) return rc;
    auto *r = new Request();
    const int na = p->n_atoms;
    r->xyz.assign(p->xyz, p->xyz + 3 * na);
    r->q.assign(p->q, p->q + na);
    r->radius.assign(p->radius, p->radius + na);
    r->prob = *p;
    r->prob.xyz = r->xyz.data();
    r->prob.q = r->q.data();
    r->prob.radius = r->radius.data();
    r->opts = *o;
    r->t_submit = Clock::now();
    ServeState *s = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return fail(NPB_ESHUTDOWN, "context is shutting down");
        }
        r->ticket = s->next_ticket++;
        s->known[r->ticket] = true;
        *ticket = r->ticket;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    return NPB_OK;
}

extern "C" int npb_poll(npb_ctx *ctx, uint64_t ticket, int32_t timeout_ms, npb_result *out) {
    if (!ctx || !out) return fail(NPB_EINVAL, "NULL argument");
    ServeState *s = ctx->serve;
    if (!s) return fail(NPB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->known.count(ticket)) return fail(NPB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_ms == 0) return NPB_PENDING;
        if (timeout_ms < 0) s->cv_done.wait(lk, ready);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return NPB_PENDING;
    }
    *out = s->done[ticket];
    s->done.erase(ticket);
    s->known.erase(ticket);
    return NPB_OK;
}
