// serve.cu -- npb_submit / npb_poll: a request queue in front of the RE+V solve.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace npb;

namespace npb {

struct Request {
    uint64_t ticket = 0;
    std::vector<double> xyz, q, radius;
    npb_problem prob{};
    npb_opts opts{};
    std::chrono::steady_clock::time_point t_submit;
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
    cudaStream_t stream = nullptr;
};

static double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

static void serve_loop(npb_ctx *ctx, ServeState *s) {
    cudaSetDevice(ctx->device);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop && s->queue.empty()) return;
            r = s->queue.front();
            s->queue.pop_front();
        }
        npb_result res{};
        res.queue_ms = ms_since(r->t_submit);
        for (int d = 0; d < 3; ++d) res.n[d] = r->prob.n[d];
        npb_grid *g = nullptr;
        int rc = grid_build(ctx, &r->prob, s->stream, &g);
        if (rc == 0) {
            cudaStream_t saved = ctx->stream;
            (void)saved;
            rc = grid_prepare(g, &r->opts, s->stream);
            if (rc == 0) rc = enqueue_energy(g, &r->opts, s->stream);
            if (rc == 0 && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = NPB_ECUDA;
            if (rc == 0) res.dG_kcal_mol = g->h_result[0];
            grid_free(g);
        }
        const int64_t inner = (int64_t)(r->prob.n[0] - 2) * (r->prob.n[1] - 2) * (r->prob.n[2] - 2);
        res.point_steps = inner * (int64_t)r->opts.n_steps * (r->opts.richardson ? 6 : 2);
        res.status = rc;
        res.wall_ms = ms_since(r->t_submit);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->done[r->ticket] = res;
        }
        s->cv_done.notify_all();
        delete r;
    }
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
    delete s;
    ctx->serve = nullptr;
}

static std::mutex g_serve_init;

static int serve_start(npb_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_serve_init);
    if (ctx->serve) return 0;
    auto *s = new ServeState();
    cudaSetDevice(ctx->device);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return fail(NPB_ECUDA, "cannot create the serving stream");
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
    r->t_submit = std::chrono::steady_clock::now();
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
