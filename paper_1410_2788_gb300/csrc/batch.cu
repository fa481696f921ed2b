// batch.cu -- RE+V energies of many molecules as one stream of launches (npb_energy_batch).
//
// The grids of a batch may differ in size.  Grids of equal size form a group; at every LOD step
// (Sec. 3.1, LODIE2 or LODIE1) each group advances all its legs (4 per molecule with Richardson
// extrapolation, Sec. 5.3) in one persistent launch per sweep direction, the legs' tensor maps and
// constants read from a device-memory table.  The whole batch -- leg starts, steps, the FP64
// energies of Eqs. (rich) and (deltaG3) and their read-back -- is captured once as a CUDA graph and
// replayed while the same grids, options and solver shapes come back.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "runtime.h"
#include "sweep_tma.cuh"

namespace npb {

cudaError_t launch_sweep_inner_table(int dir, const LegTma *table, int n_legs, int nx, int ny, int nz,
                                    int32_t *err, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                    cudaStream_t st);
cudaError_t launch_source(int prec, const LegDev *legs, int n_legs, int ny, int nz, cudaStream_t st);

struct BatchGroup {
    std::vector<Grid *> grids;
    bool table = false;           // every leg in table launches (else per-grid steps)
    SweepShape shape[3]{};
    LegTma *d_tab[3] = {};        // per direction: [slot-major][grid] legs
    LegDev *d_dev = nullptr;      // the same legs' constants (stand-alone source stage)
};

struct BatchPlan {
    std::string key;
    std::vector<Grid *> grids;
    std::vector<BatchGroup> groups;
    void *d_mem = nullptr;
    size_t bytes = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
};

static void plan_free(Ctx *ctx, BatchPlan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->d_mem) ctx->release(p->d_mem, p->bytes);
    delete p;
}

// Plans that name grid g (or every plan, g == nullptr) are dropped: their tables hold its maps.
void batch_forget(Ctx *ctx, Grid *g) {
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    auto &v = ctx->batches;
    for (size_t i = 0; i < v.size();) {
        BatchPlan *p = v[i];
        if (!g || std::find(p->grids.begin(), p->grids.end(), g) != p->grids.end()) {
            plan_free(ctx, p);
            v.erase(v.begin() + i);
        } else {
            ++i;
        }
    }
}

// The slots a solve runs: Richardson runs all four ([s_half, v_half, s_tau, v_tau]; the dt/2 legs
// first, so that the legs still running after step n are a prefix), plain runs slots 2..3.
static int slot_of(int richardson, int j) { return richardson ? j : 2 + j; }

static int plan_build(Ctx *ctx, Grid *const *grids, int n, const npb_opts *o, BatchPlan *plan) {
    const int prec = o->precision;
    const int re = o->richardson ? 1 : 0;
    const int nslot = re ? 4 : 2;
    for (int i = 0; i < n; ++i) {
        Grid *g = grids[i];
        BatchGroup *grp = nullptr;
        for (auto &q : plan->groups)
            if (q.grids[0]->geo.nx == g->geo.nx && q.grids[0]->geo.ny == g->geo.ny &&
                q.grids[0]->geo.nz == g->geo.nz)
                grp = &q;
        if (!grp) {
            plan->groups.emplace_back();
            grp = &plan->groups.back();
        }
        grp->grids.push_back(g);
    }
    size_t bytes = 0;
    for (auto &q : plan->groups) {
        const Grid *g0 = q.grids[0];
        const int dims[3] = {g0->geo.nx, g0->geo.ny, g0->geo.nz};
        bool ok = prec == NPB_FP32_SWEEP && o->eps_mode == NPB_EPS_HARMONIC && o->scheme <= NPB_LODIE2;
        for (int d = 0; d < 3; ++d) {
            bool tables = true;
            for (Grid *g : q.grids)
                for (int j = 0; j < nslot; ++j) tables = tables && g->h_legs[prec][slot_of(re, j)].line_tab[d];
            q.shape[d] = usable_shape(shape_for(ctx, prec, d, dims[d]), d, dims[d], tables,
                                      scheme_cn(o->scheme) ? FUSE_PRE_CN : 0);
            ok = ok && (q.shape[d].kind == 2 || q.shape[d].kind == 3) && tma_variant(d, q.shape[d].tx) >= 0;
            for (Grid *g : q.grids) ok = ok && g->tma_ok[d];
        }
        q.table = ok;
        if (ok) bytes += 3 * ((q.grids.size() * nslot * sizeof(LegTma) + 255) & ~(size_t)255);
        bytes += (q.grids.size() * nslot * sizeof(LegDev) + 255) & ~(size_t)255;
    }
    if (bytes) {
        int rc = ctx->alloc(&plan->d_mem, bytes);
        if (rc) return rc;
        plan->bytes = bytes;
    }
    // host copies of the tables, then one upload
    struct Free {
        void operator()(void *p) const { free(p); }
    };
    std::unique_ptr<unsigned char, Free> hbuf(static_cast<unsigned char *>(aligned_alloc(256, (bytes + 255) & ~(size_t)255)));
    if (bytes && !hbuf) return fail(NPB_ENOMEM, "host staging for the batch tables");
    unsigned char *hostp = hbuf.get();
    size_t off = 0;
    for (auto &q : plan->groups) {
        const size_t m = q.grids.size();
        if (q.table) {
            for (int d = 0; d < 3; ++d) {
                const int v = tma_variant(d, q.shape[d].tx);
                LegTma *h = reinterpret_cast<LegTma *>(hostp + off);
                for (int j = 0; j < nslot; ++j)
                    for (size_t i = 0; i < m; ++i) {
                        const Grid *g = q.grids[i];
                        const int slot = slot_of(re, j);
                        LegTma &e = h[j * m + i];
                        memcpy(&e.umap, &g->tma_u[d][v][slot], sizeof(CUtensorMap));
                        memcpy(&e.mmap, &g->tma_m[d][v], sizeof(CUtensorMap));
                        e.dev = g->h_legs[prec][slot];
                    }
                q.d_tab[d] = reinterpret_cast<LegTma *>(static_cast<unsigned char *>(plan->d_mem) + off);
                off += (m * nslot * sizeof(LegTma) + 255) & ~(size_t)255;
            }
        }
        LegDev *h = reinterpret_cast<LegDev *>(hostp + off);
        for (int j = 0; j < nslot; ++j)
            for (size_t i = 0; i < m; ++i) h[j * m + i] = q.grids[i]->h_legs[prec][slot_of(re, j)];
        q.d_dev = reinterpret_cast<LegDev *>(static_cast<unsigned char *>(plan->d_mem) + off);
        off += (m * nslot * sizeof(LegDev) + 255) & ~(size_t)255;
    }
    if (bytes) {
        CU(cudaMemcpy(plan->d_mem, hostp, bytes, cudaMemcpyHostToDevice));
    }
    return 0;
}

// One LOD step of a group: its first n_legs table entries (all legs, or the dt/2 prefix).
static int group_step(Ctx *ctx, const BatchGroup &q, int n_legs, int prec, int scheme, int richardson,
                      int slot0, cudaStream_t st) {
    if (!q.table) {  // per-grid steps on the fallback kernels
        for (Grid *g : q.grids) {
            int rc = run_step(g, prec, scheme, slot0, n_legs / (int)q.grids.size(), st);
            if (rc) return rc;
        }
        return 0;
    }
    (void)richardson;
    Profiler &pr = ctx->prof;
    const Grid *g0 = q.grids[0];
    const int dims[3] = {g0->geo.nx, g0->geo.ny, g0->geo.nz};
    cudaEvent_t ev{};
    int rc;
    for (int d = 0; d < 3; ++d) {
        int flags = 0;
        if (d == 0) flags = scheme == NPB_LODIE2 ? FUSE_PRE_SRC : FUSE_PRE_NL;
        if (d == 2 && scheme == NPB_LODIE2) flags = FUSE_POST_NL;
        if ((rc = pr.begin(st, &ev))) return rc;
        if (q.shape[d].kind == 3)
            CU(launch_sweep_line_table(d, q.d_tab[d], n_legs, dims[0], dims[1], dims[2], g0->d_err, g0->tma_g[d],
                                       flags, q.shape[d], ctx->sm_count, st));
        else
            CU(launch_sweep_inner_table(d, q.d_tab[d], n_legs, dims[0], dims[1], dims[2], g0->d_err, g0->tma_g[d],
                                        flags, q.shape[d], ctx->sm_count, st));
        if ((rc = pr.end(st, ev, K_SWEEP_X + d))) return rc;
    }
    if (scheme == NPB_LODIE1) {
        if ((rc = pr.begin(st, &ev))) return rc;
        CU(launch_source(prec, q.d_dev, n_legs, dims[1], dims[2], st));
        if ((rc = pr.end(st, ev, K_SOURCE))) return rc;
    }
    return 0;
}

static int enqueue_batch(Ctx *ctx, const BatchPlan &plan, const npb_opts *o, cudaStream_t st) {
    const int prec = o->precision;
    const int re = o->richardson ? 1 : 0;
    const int n = o->n_steps;
    const int legs_re[4] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_SOLVENT_HALF, NPB_LEG_VACUUM_TAU, NPB_LEG_VACUUM_HALF};
    const int legs_plain[2] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_VACUUM_TAU};
    int rc;
    for (Grid *g : plan.grids)
        if ((rc = init_legs(g, prec, re ? legs_re : legs_plain, re ? 4 : 2, st))) return rc;
    for (int s = 0; s < n; ++s)
        for (const auto &q : plan.groups) {
            const int m = (int)q.grids.size();
            if ((rc = group_step(ctx, q, (re ? 4 : 2) * m, prec, o->scheme, re, re ? 0 : 2, st))) return rc;
        }
    if (re)
        for (int s = 0; s < n; ++s)
            for (const auto &q : plan.groups) {
                const int m = (int)q.grids.size();
                if ((rc = group_step(ctx, q, 2 * m, prec, o->scheme, re, 0, st))) return rc;
            }
    for (Grid *g : plan.grids)
        if ((rc = enqueue_energy_reduce(g, prec, re, st))) return rc;
    return 0;
}

}  // namespace npb

using namespace npb;

extern "C" int npb_energy_batch(npb_grid *const *grids, int32_t n_grids, const npb_opts *o, double *dG) {
    if (!grids || n_grids <= 0 || !dG) return fail(NPB_EINVAL, "grids/dG is NULL or n_grids <= 0");
    if (!o) return fail(NPB_EINVAL, "opts is NULL");
    if (!(o->dt > 0) || !(o->alpha > 0) || o->n_steps < 0) return fail(NPB_EINVAL, "dt, alpha > 0, n_steps >= 0");
    if (o->scheme < NPB_LODIE1 || o->scheme > NPB_LODCN2)
        return fail(NPB_EINVAL, "npb_energy_batch runs the LOD schemes (1-4), not scheme %d", o->scheme);
    if (o->precision != NPB_FP64 && o->precision != NPB_FP32_SWEEP)
        return fail(NPB_EINVAL, "unknown precision %d", o->precision);
    if (!o->vacuum_recovery)
        return fail(NPB_EINVAL, "npb_energy_batch runs the LOD vacuum legs (vacuum_recovery = 1); use npb_energy");
    npb_ctx *ctx = grids[0] ? grids[0]->ctx : nullptr;
    for (int i = 0; i < n_grids; ++i) {
        if (!grids[i]) return fail(NPB_EINVAL, "grids[%d] is NULL", i);
        if (grids[i]->ctx != ctx) return fail(NPB_EINVAL, "grids[%d] belongs to another context", i);
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return fail(NPB_EINVAL, "grid %d appears twice", i);
    }
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    int rc;
    std::string key;
    {
        char buf[160];
        snprintf(buf, sizeof buf, "%.17g/%.17g/%d/%d/%d/%d/%d|", o->dt, o->alpha, o->n_steps, o->scheme,
                 o->richardson, o->precision, o->eps_mode);
        key = buf;
    }
    for (int i = 0; i < n_grids; ++i) {
        Grid *g = grids[i];
        if ((rc = grid_prepare(g, o, st))) return rc;
        for (int m = 0; m < 2; ++m) {  // face data on first use, outside any capture
            const double *bc;
            if ((rc = grid_boundary(g, m, o->precision, st, &bc))) return rc;
        }
        char buf[64];
        snprintf(buf, sizeof buf, "%p;", (void *)g);
        key += buf;
        key += g->legs_key[o->precision];
    }
    for (int d = 0; d < 3; ++d)  // the solver shapes in force
        for (int i = 0; i < n_grids; ++i) {
            const SweepShape s = shape_for(ctx, o->precision, d, d == 0 ? grids[i]->geo.nx
                                                                        : (d == 1 ? grids[i]->geo.ny : grids[i]->geo.nz));
            char buf[48];
            snprintf(buf, sizeof buf, "|%d,%d,%d,%d", s.kind, s.tx, s.seg, s.len);
            key += buf;
        }
    BatchPlan *plan = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->batch_mu);
        for (BatchPlan *p : ctx->batches)
            if (p->key == key && p->stream == st) plan = p;
    }
    const bool use_graph = !ctx->prof.enabled && st != nullptr && ctx->use_graphs;
    if (!plan) {
        plan = new BatchPlan;
        plan->key = key;
        plan->stream = st;
        plan->grids.assign(grids, grids + n_grids);
        if ((rc = plan_build(ctx, grids, n_grids, o, plan))) {
            plan_free(ctx, plan);
            return rc;
        }
        if (use_graph) {
            cudaGraph_t graph;
            cudaError_t eb = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (eb != cudaSuccess) {
                plan_free(ctx, plan);
                CU(eb);
            }
            rc = enqueue_batch(ctx, *plan, o, st);
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (rc || ec != cudaSuccess) {
                if (ec == cudaSuccess) cudaGraphDestroy(graph);
                plan_free(ctx, plan);
                if (rc) return rc;
                CU(ec);
            }
            cudaError_t ei = cudaGraphInstantiate(&plan->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                plan_free(ctx, plan);
                CU(ei);
            }
        }
        std::lock_guard<std::mutex> lk(ctx->batch_mu);
        ctx->batches.push_back(plan);
    }
    if (plan->exec && use_graph) {
        CU(cudaGraphLaunch(plan->exec, st));
    } else if ((rc = enqueue_batch(ctx, *plan, o, st))) {
        return rc;
    }
    CU(cudaStreamSynchronize(st));
    int first_err = 0;
    for (int i = 0; i < n_grids; ++i) {
        rc = grid_check_err(grids[i], st, 1);
        if (rc && !first_err) first_err = rc;
        dG[i] = grids[i]->h_result[0];
    }
    return first_err ? first_err : NPB_OK;
}
