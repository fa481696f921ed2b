// tune.cu -- autotuner for the line-solver shape (lines per block TX, segments per line SEG,
// rows per segment L).  SEG = 1 would be a plain Thomas sweep per line, large SEG with short
// L is mostly parallel cyclic reduction; the tuner times every instantiated shape that fits
// the line on a live grid (all four legs batched, as a solve launches them) and keeps the
// fastest per (precision, direction, line length).
#include <cstdio>
#include <cstdlib>
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
            ns += line_shapes(d, shapes + ns, 96 - ns);
        }
        if (prec == NPB_FP64 && ns < 96) shapes[ns++] = SweepShape{32, 2, 1, 3};  // Thomas per line
        SweepShape best{0, 0, 0, 0};
        float best_ms = 1e30f;
        for (int i = 0; i < ns; ++i) {
            const SweepShape s = shapes[i];
            const int need = s.kind == 2 ? n_dir[d] - 2 : n_dir[d];  // interior-row shapes cover n-2 rows
            if (s.kind != 3 && s.seg * s.len < need) continue;          // (kind 3: any line length)
            if (s.kind != 3 && s.seg * s.len > 2 * need + 32) continue;  // mostly padding: never faster
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
    if (!ctx || dir < 0 || dir > 2 || kind < 0 || kind > 3) return fail(NPB_EINVAL, "bad argument");
    SweepShape s{tx, seg, len, kind}, t[64];
    bool found = false;
    if (kind == 0) {
        found = sweep_shape_available(precision, s);
    } else if (precision == NPB_FP64) {
        found = kind == 3 && tx == 32 && seg == 2 && len == 1;  // Thomas per line, multipliers once per leg
    } else if (precision == NPB_FP32_SWEEP) {
        const int k = kind == 1 ? tma_shapes(dir, t, 64) : (kind == 2 ? inner_shapes(dir, t, 64) : line_shapes(dir, t, 64));
        for (int i = 0; i < k && !found; ++i) found = t[i].tx == tx && t[i].seg == seg && t[i].len == len;
    }
    if (!found) return fail(NPB_EINVAL, "shape kind %d %d/%d/%d not instantiated", kind, tx, seg, len);
    const int need = kind == 2 ? n - 2 : n;
    if (kind != 3 && seg * len < need) return fail(NPB_EINVAL, "shape covers %d rows, too few for n = %d", seg * len, n);
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

// Device time of one sweep launch as a solve makes it: direction dir over the legs in slots
// [0, n_legs) (n_legs 4 or 2: the four legs of steps 1..n, or the two dt/2 legs after step n),
// with the solve's fused stages (LODIE2: the source stage in the x sweep, the nonlinear stage in
// the z sweep).  `reps` launches are captured in one CUDA graph; the graph is replayed once untimed
// and `rounds` times between two events on the context stream.  The legs' states are overwritten.
extern "C" int npb_sweep_time(npb_grid *g, const npb_opts *o, int32_t dir, int32_t n_legs, int32_t reps,
                              int32_t rounds, double *ms_per_launch) {
    if (!g || !o || !ms_per_launch) return fail(NPB_EINVAL, "NULL argument");
    if (dir < 0 || dir > 2 || (n_legs != 2 && n_legs != 4) || reps <= 0 || rounds <= 0)
        return fail(NPB_EINVAL, "dir in 0..2, n_legs 2 or 4, reps and rounds > 0");
    if (scheme_additive(o->scheme) || scheme_cn(o->scheme))
        return fail(NPB_EINVAL, "npb_sweep_time times the implicit-Euler LOD schemes");
    npb_ctx *ctx = g->ctx;
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    if (!st) return fail(NPB_EINVAL, "npb_sweep_time needs a non-default stream");
    int rc = grid_prepare(g, o, st);
    if (rc) return rc;
    const int legs[4] = {0, 1, 2, 3};
    if ((rc = init_legs(g, o->precision, legs, 4, st))) return rc;
    const int n_dir[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    const SweepShape s = shape_for(ctx, o->precision, dir, n_dir[dir]);
    // the stages fused as a solve fuses them: S leaves the x sweep where the solve gives it a
    // launch of its own (kind-1 TMA sweeps, large charge lists)
    const bool src_apart = o->precision == NPB_FP32_SWEEP && s.kind >= 1 && g->tma_ok[0] &&
                           (s.kind == 1 || 8 * g->n_atoms >= kSourceApartEntries);
    int flags = 0;
    if (o->scheme == NPB_LODIE2) flags = dir == 0 ? (src_apart ? 0 : FUSE_PRE_SRC) : (dir == 2 ? FUSE_POST_NL : 0);
    else if (dir == 0) flags = FUSE_PRE_NL;
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_dir(g, o->precision, dir, s, 0, n_legs, flags, st);
    cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess) {
        if (ec == cudaSuccess) cudaGraphDestroy(graph);
        return fail(NPB_ECUDA, "sweep launch failed: %s", cudaGetErrorString(e));
    }
    CU(ec);
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CU(e);
    cudaEvent_t a, b;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int r = 0; r < rounds && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return fail(NPB_ECUDA, "sweep timing failed: %s", cudaGetErrorString(e));
    *ms_per_launch = (double)ms / ((double)reps * rounds);
    return grid_check_err(g, st, 0);
}

// ---- the tuning cache: the context's pinned shapes as a JSON list on disk
extern "C" int npb_tune_save(npb_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(NPB_EINVAL, "NULL argument");
    std::string out = "[\n";
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        bool first = true;
        for (const auto &kv : ctx->tuned) {
            const int prec = (int)(kv.first >> 40), dir = (int)((kv.first >> 32) & 0xff), n = (int)(kv.first & 0xffffffff);
            const SweepShape &s = kv.second;
            char buf[200];
            snprintf(buf, sizeof buf,
                     "%s {\"precision\": %d, \"dir\": %d, \"n\": %d, \"kind\": %d, \"tx\": %d, \"seg\": %d, \"len\": %d}",
                     first ? "" : ",\n", prec, dir, n, s.kind, s.tx, s.seg, s.len);
            out += buf;
            first = false;
        }
    }
    out += "\n]\n";
    FILE *f = fopen(path, "w");
    if (!f) return fail(NPB_EINVAL, "cannot write %s", path);
    const size_t w = fwrite(out.data(), 1, out.size(), f);
    const int c = fclose(f);
    if (w != out.size() || c != 0) return fail(NPB_EINVAL, "short write to %s", path);
    return NPB_OK;
}

// Reads the integer value of "key" inside one {...} entry.
static bool json_int(const std::string &obj, const char *key, int *out) {
    const std::string k = std::string("\"") + key + "\"";
    const size_t at = obj.find(k);
    if (at == std::string::npos) return false;
    size_t i = obj.find(':', at + k.size());
    if (i == std::string::npos) return false;
    ++i;
    while (i < obj.size() && (obj[i] == ' ' || obj[i] == '\t' || obj[i] == '\n' || obj[i] == '\r')) ++i;
    char *end = nullptr;
    const long v = strtol(obj.c_str() + i, &end, 10);
    if (end == obj.c_str() + i) return false;
    *out = (int)v;
    return true;
}

extern "C" int npb_tune_load(npb_ctx *ctx, const char *path, int32_t *n_loaded) {
    if (!ctx || !path) return fail(NPB_EINVAL, "NULL argument");
    FILE *f = fopen(path, "r");
    if (!f) return fail(NPB_EINVAL, "cannot read %s", path);
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, r);
    fclose(f);
    int loaded = 0;
    size_t pos = 0;
    while ((pos = text.find('{', pos)) != std::string::npos) {
        const size_t end = text.find('}', pos);
        if (end == std::string::npos) return fail(NPB_EINVAL, "%s: unterminated entry", path);
        const std::string obj = text.substr(pos, end - pos + 1);
        int prec, dir, n, kind, tx, seg, len;
        if (!json_int(obj, "precision", &prec) || !json_int(obj, "dir", &dir) || !json_int(obj, "n", &n) ||
            !json_int(obj, "kind", &kind) || !json_int(obj, "tx", &tx) || !json_int(obj, "seg", &seg) ||
            !json_int(obj, "len", &len))
            return fail(NPB_EINVAL, "%s: an entry lacks one of precision, dir, n, kind, tx, seg, len", path);
        // entries this build does not instantiate are skipped (npb_tune_set validates them)
        if (npb_tune_set(ctx, prec, dir, n, kind, tx, seg, len) == NPB_OK) ++loaded;
        pos = end + 1;
    }
    if (n_loaded) *n_loaded = loaded;
    return NPB_OK;
}
