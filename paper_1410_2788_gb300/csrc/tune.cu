// tune.cu -- autotuner for the line-solver shape (lines per block TX, segments per line SEG,
// rows per segment L).  SEG = 1 would be a plain Thomas sweep per line, large SEG with short
// L is mostly parallel cyclic reduction; the tuner times every instantiated shape that fits
// the line on a live grid (all four legs batched, as a solve launches them) and keeps the
// fastest per (precision, direction, line length).
#include <cstdio>
#include <string>

#include "runtime.h"

using namespace npb;

extern "C" int npb_autotune(npb_grid *g, const npb_opts *o, int32_t reps, char *report, size_t report_len) {
    if (!g || !o) return fail(NPB_EINVAL, "NULL argument");
    if (reps <= 0) reps = 5;
    npb_ctx *ctx = g->ctx;
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    int rc = grid_prepare(g, o, st);
    if (rc) return rc;
    const int prec = o->precision;
    const int legs[4] = {0, 1, 2, 3};
    if ((rc = init_legs(g, prec, legs, 4, st))) return rc;
    const int n_dir[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    SweepShape shapes[96];
    const int nc = sweep_shapes(prec, shapes, 48);
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    std::string rep = "[";
    for (int d = 0; d < 3; ++d) {
        int ns = nc;
        if (prec == NPB_FP32_SWEEP && g->tma_ok[d]) {
            ns += tma_shapes(d, shapes + ns, 96 - ns);
            ns += inner_shapes(d, shapes + ns, 96 - ns);
        }
        SweepShape best{0, 0, 0, 0};
        float best_ms = 1e30f;
        for (int i = 0; i < ns; ++i) {
            const SweepShape s = shapes[i];
            const int need = s.kind == 2 ? n_dir[d] - 2 : n_dir[d];  // interior-row shapes cover n-2 rows
            if (s.seg * s.len < need) continue;
            if (s.seg * s.len > 2 * need + 32) continue;  // mostly padding: never faster
            cudaError_t e = launch_dir(g, prec, d, s, 0, 4, 0, st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            CU(cudaEventRecord(a, st));
            for (int r = 0; r < reps; ++r)
                CU(launch_dir(g, prec, d, s, 0, 4, 0, st));
            CU(cudaEventRecord(b, st));
            CU(cudaEventSynchronize(b));
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, a, b));
            ms /= reps;
            char buf[160];
            snprintf(buf, sizeof buf,
                     "%s{\"dir\":%d,\"n\":%d,\"tx\":%d,\"seg\":%d,\"len\":%d,\"kind\":%d,\"ms\":%.5f}",
                     rep.size() > 1 ? "," : "", d, n_dir[d], s.tx, s.seg, s.len, s.kind, ms);
            rep += buf;
            if (ms < best_ms) {
                best_ms = ms;
                best = s;
            }
        }
        if (best.tx) {
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            ctx->tuned[tune_key(prec, d, n_dir[d])] = best;
        }
    }
    rep += "]";
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    for (auto &c : g->graphs)
        if (c.exec) cudaGraphExecDestroy(c.exec);
    g->graphs.clear();  // captured graphs hold the old shapes
    if (report && report_len) {
        snprintf(report, report_len, "%s", rep.c_str());
    }
    return NPB_OK;
}

extern "C" int npb_tune_set(npb_ctx *ctx, int32_t precision, int32_t dir, int32_t n, int32_t kind, int32_t tx,
                            int32_t seg, int32_t len) {
    if (!ctx || dir < 0 || dir > 2 || kind < 0 || kind > 2) return fail(NPB_EINVAL, "bad argument");
    SweepShape s{tx, seg, len, kind}, t[32];
    bool found = false;
    if (kind == 0) {
        found = sweep_shape_available(precision, s);
    } else if (precision == NPB_FP32_SWEEP) {
        const int k = kind == 1 ? tma_shapes(dir, t, 32) : inner_shapes(dir, t, 32);
        for (int i = 0; i < k && !found; ++i) found = t[i].tx == tx && t[i].seg == seg && t[i].len == len;
    }
    if (!found) return fail(NPB_EINVAL, "shape kind %d %d/%d/%d not instantiated", kind, tx, seg, len);
    const int need = kind == 2 ? n - 2 : n;
    if (seg * len < need) return fail(NPB_EINVAL, "shape covers %d rows, too few for n = %d", seg * len, n);
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tuned[tune_key(precision, dir, n)] = s;
    return NPB_OK;
}

extern "C" int npb_tune_get(npb_ctx *ctx, int32_t precision, int32_t dir, int32_t n, int32_t *kind, int32_t *tx,
                            int32_t *seg, int32_t *len) {
    if (!ctx || !kind || !tx || !seg || !len) return fail(NPB_EINVAL, "bad argument");
    const SweepShape s = shape_for(ctx, precision, dir, n);
    *kind = s.kind;
    *tx = s.tx;
    *seg = s.seg;
    *len = s.len;
    return s.tx ? NPB_OK : fail(NPB_EINVAL, "no shape covers n = %d", n);
}
