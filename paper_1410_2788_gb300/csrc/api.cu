// api.cu -- host runtime behind include/npb.h: contexts, grids, leg scheduling, CUDA-graph
// replay of whole RE+V solves, per-kernel profiling, and the serving scheduler.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/npb.h"
#include "npb_internal.cuh"
#include "runtime.h"
#include "setup_kernels.cuh"
#include "sweep_tma.cuh"

using namespace npb;

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

int npb::fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

extern "C" const char *npb_last_error(void) { return t_err.c_str(); }
extern "C" const char *npb_version(void) { return "npb-lod-gb300 1.0 (sm_103a)"; }

namespace npb {
cudaError_t launch_sweep_f32(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, int flags,
                             SweepShape s, cudaStream_t st);
cudaError_t launch_sweep_f64(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, int flags,
                             SweepShape s, cudaStream_t st);
cudaError_t prepare_sweep_f32();
cudaError_t prepare_sweep_f64();
cudaError_t launch_energy(int prec, const void *s_tau, const void *s_half, const void *v_tau,
                          const void *v_half, const int64_t *off, const double *qt, const int32_t *n_ent,
                          int richardson, const double *vac, double *part, double *out, cudaStream_t st);

// Shapes the line solver is instantiated for (kept in sync with NPB_SWEEP_SHAPES).
static const SweepShape kShapes[] = {{16, 2, 17}, {16, 4, 9},   {16, 4, 17}, {16, 8, 9},
                                     {16, 8, 13}, {16, 8, 17},  {16, 16, 9}, {16, 16, 11},
                                     {16, 16, 17}, {16, 32, 9}, {32, 8, 17}, {32, 16, 9}};

int sweep_shapes(int, SweepShape *out, int max) {
    int n = 0;
    for (const auto &s : kShapes)
        if (n < max) out[n++] = s;
    return n;
}

bool sweep_shape_available(int, SweepShape s) {
    for (const auto &k : kShapes)
        if (k.tx == s.tx && k.seg == s.seg && k.len == s.len) return true;
    return false;
}

// Smallest SEG*L >= n among the TX = 16 shapes; ties go to the longer segment.
SweepShape default_sweep_shape(int, int, int n) {
    SweepShape best{0, 0, 0};
    for (const auto &s : kShapes) {
        if (s.tx != 16 || s.seg * s.len < n) continue;
        if (best.tx == 0 || s.seg * s.len < best.seg * best.len ||
            (s.seg * s.len == best.seg * best.len && s.len > best.len))
            best = s;
    }
    return best;
}

cudaError_t launch_sweep(int prec, int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, int flags,
                         SweepShape s, cudaStream_t st) {
    if (prec == NPB_FP64) return launch_sweep_f64(dir, legs, n_legs, nx, ny, nz, flags, s, st);
    return launch_sweep_f32(dir, legs, n_legs, nx, ny, nz, flags, s, st);
}

const char *kKernelNames[K_COUNT] = {"sweep_x", "sweep_y", "sweep_z", "nonlinear", "source", "init_leg",
                                     "energy", "setup_mask", "setup_charges", "setup_boundary", "pad", "cn_explicit",
                                     "additive_combine"};
}  // namespace npb

// ------------------------------------------------------------------ context
Profiler::~Profiler() {
    for (auto &p : pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
}

int Profiler::begin(cudaStream_t st, cudaEvent_t *a) {
    if (!enabled) return 0;
    CU(cudaEventCreate(a));
    CU(cudaEventRecord(*a, st));
    return 0;
}

int Profiler::end(cudaStream_t st, cudaEvent_t a, int kind, int kernels) {
    if (!enabled) return 0;
    cudaEvent_t b;
    CU(cudaEventCreate(&b));
    CU(cudaEventRecord(b, st));
    std::lock_guard<std::mutex> lk(mu);
    pending.push_back({a, b, kind, kernels});
    return 0;
}

int Profiler::collect() {
    std::lock_guard<std::mutex> lk(mu);
    for (auto &p : pending) {
        CU(cudaEventSynchronize(p.b));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, p.a, p.b));
        launches[p.kind] += p.kernels;
        total_ms[p.kind] += ms;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    pending.clear();
    return 0;
}

int Ctx::alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return 0;
    const size_t sz = (bytes + 511) / 512 * 512;
    std::lock_guard<std::mutex> lk(mem_mu);
    const size_t cur = in_use.load();
    if (cur + sz > budget)
        return fail(NPB_ENOMEM, "HBM budget exceeded: %zu in use + %zu requested > %zu budget", cur, sz, budget);
    auto it = cached.find(sz);
    if (it != cached.end()) {
        *p = it->second;
        cached.erase(it);
        cached_bytes -= sz;
    } else {
        if (cur + cached_bytes + sz > budget) trim();
        cudaError_t e = cudaMalloc(p, sz);
        if (e != cudaSuccess && cached_bytes) {  // the driver may be short of what the cache holds
            cudaGetLastError();
            trim();
            e = cudaMalloc(p, sz);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return fail(NPB_ENOMEM, "cudaMalloc(%zu) failed: %s", sz, cudaGetErrorString(e));
        }
    }
    live[*p] = sz;
    in_use += sz;
    return 0;
}

// The block goes back to the cache.  Every caller has synchronised the streams that used it (the
// same point at which cudaFree would have synchronised the device).
void Ctx::release(void *p, size_t) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mem_mu);
    auto it = live.find(p);
    if (it == live.end()) return;
    const size_t sz = it->second;
    live.erase(it);
    in_use -= sz;
    cached.emplace(sz, p);
    cached_bytes += sz;
}

void Ctx::trim() {
    for (auto &c : cached) cudaFree(c.second);
    cached.clear();
    cached_bytes = 0;
}

int Ctx::pinned_slot(double **out) {
    std::lock_guard<std::mutex> lk(mem_mu);
    if (pinned_free.empty()) {
        constexpr int kSlots = 64;
        void *slab = nullptr;
        if (cudaMallocHost(&slab, kSlots * 8 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NPB_ENOMEM, "cudaMallocHost failed");
        }
        pinned_slabs.push_back(slab);
        for (int i = kSlots - 1; i >= 0; --i) pinned_free.push_back(static_cast<double *>(slab) + 8 * i);
    }
    *out = pinned_free.back();
    pinned_free.pop_back();
    return 0;
}

void Ctx::pinned_release(double *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mem_mu);
    pinned_free.push_back(p);
}

extern "C" int npb_ctx_create(int device, size_t budget, npb_ctx **out) {
    if (!out) return fail(NPB_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(NPB_EINVAL, "device %d out of range (%d devices)", device, ndev);
    CU(cudaSetDevice(device));
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, device));
    auto ctx = std::make_unique<npb_ctx>();
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    ctx->budget = budget ? budget : (size_t)(0.9 * (double)free_b);
    CU(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
    ctx->stream = ctx->own_stream;
    CU(prepare_sweep_f32());
    CU(prepare_sweep_f64());
    CU(prepare_sweep_tma());
    CU(prepare_sweep_inner());
    CU(prepare_sweep_line());
    *out = ctx.release();
    return NPB_OK;
}

extern "C" void npb_ctx_destroy(npb_ctx *ctx) {
    if (!ctx) return;
    serve_shutdown(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    batch_forget(ctx, nullptr);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    {
        std::lock_guard<std::mutex> lk(ctx->mem_mu);
        ctx->trim();
        for (auto &l : ctx->live) cudaFree(l.first);  // blocks a caller never released
        for (void *s : ctx->pinned_slabs) cudaFreeHost(s);
    }
    delete ctx;
}

extern "C" int npb_ctx_set_stream(npb_ctx *ctx, void *stream) {
    if (!ctx) return fail(NPB_EINVAL, "ctx is NULL");
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return NPB_OK;
}

extern "C" int npb_ctx_profile(npb_ctx *ctx, int32_t enable) {
    if (!ctx) return fail(NPB_EINVAL, "ctx is NULL");
    int rc = ctx->prof.collect();
    if (rc) return rc;
    ctx->prof.enabled = enable != 0;
    if (enable) {
        for (int i = 0; i < K_COUNT; ++i) {
            ctx->prof.launches[i] = 0;
            ctx->prof.total_ms[i] = 0.0;
        }
    }
    return NPB_OK;
}

extern "C" int npb_ctx_kernel_stats(npb_ctx *ctx, int32_t max_kernels, const char **names, int64_t *launches,
                                    double *ms) {
    if (!ctx) return fail(NPB_EINVAL, "ctx is NULL");
    int rc = ctx->prof.collect();
    if (rc) return rc;
    int n = 0;
    for (int i = 0; i < K_COUNT && n < max_kernels; ++i, ++n) {
        if (names) names[n] = kKernelNames[i];
        if (launches) launches[n] = ctx->prof.launches[i];
        if (ms) ms[n] = ctx->prof.total_ms[i];
    }
    return n;
}

extern "C" int npb_ctx_probe_wait_expiry(npb_ctx *ctx, int64_t cycles) {
    if (!ctx) return fail(NPB_EINVAL, "ctx is NULL");
    if (cycles < 0) return fail(NPB_EINVAL, "cycles must be >= 0");
    ctx->probe_cycles = cycles;
    return NPB_OK;
}

extern "C" int npb_ctx_memory(npb_ctx *ctx, size_t *in_use, size_t *budget) {
    if (!ctx) return fail(NPB_EINVAL, "ctx is NULL");
    if (in_use) *in_use = ctx->in_use.load();
    if (budget) *budget = ctx->budget;
    return NPB_OK;
}

// ------------------------------------------------------------------ grid set-up
static int validate(const npb_problem *p, double origin[3]) {
    if (!p) return fail(NPB_EINVAL, "problem is NULL");
    for (int d = 0; d < 3; ++d)
        if (p->n[d] < 3 || p->n[d] > kMaxLine)
            return fail(NPB_EINVAL, "n[%d] = %d outside [3, %d]", d, p->n[d], kMaxLine);
    if (!(p->h > 0)) return fail(NPB_EINVAL, "h must be > 0");
    if (!(p->eps_in > 0) || !(p->eps_out > 0)) return fail(NPB_EINVAL, "eps_in and eps_out must be > 0");
    if (!(p->kappa2 >= 0)) return fail(NPB_EINVAL, "kappa2 must be >= 0");
    if (p->n_atoms < 0) return fail(NPB_EINVAL, "n_atoms < 0");
    if (p->n_atoms > 0 && (!p->xyz || !p->q || !p->radius)) return fail(NPB_EINVAL, "atom arrays are NULL");
    // origin: NaN means centre the atoms' bounding box
    for (int d = 0; d < 3; ++d) {
        origin[d] = p->origin[d];
        if (std::isnan(origin[d])) {
            double lo = 0, hi = 0;
            for (int a = 0; a < p->n_atoms; ++a) {
                const double x = p->xyz[3 * a + d];
                if (a == 0 || x < lo) lo = x;
                if (a == 0 || x > hi) hi = x;
            }
            origin[d] = 0.5 * (lo + hi) - 0.5 * (p->n[d] - 1) * p->h;
        }
    }
    for (int a = 0; a < p->n_atoms; ++a) {
        if (!(p->radius[a] > 0)) return fail(NPB_EINVAL, "atom %d: radius must be > 0", a);
        for (int d = 0; d < 3; ++d) {
            const double s = (p->xyz[3 * a + d] - origin[d]) / p->h;
            if (!std::isfinite(s)) return fail(NPB_EINVAL, "atom %d: non-finite position", a);
            const double i0 = std::floor(s);
            if (i0 < 1 || i0 + 1 > p->n[d] - 2)
                return fail(NPB_EINVAL, "atom %d: charge stencil leaves the interior along axis %d", a, d);
        }
    }
    return 0;
}


extern "C" size_t npb_grid_footprint(const npb_problem *p, int32_t precision) {
    if (!p) return 0;
    const size_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
    const size_t pitch = (nx + 31) / 32 * 32;
    const size_t lines = ny * nz;
    const size_t na = p->n_atoms > 0 ? p->n_atoms : 0;
    const size_t raw = std::max<size_t>(1, 8 * na);
    size_t b = 0;
    b += 4 * state_bytes(p->n, precision);                                   // four leg states
    if (precision == NPB_FP64) b += 12 * state_bytes(p->n, precision);       // their multipliers
    b += (size_t)mask_words_per_row((int)pitch) * lines * 4;                 // node mask
    b += nz * nx * line_words((int)ny) * 4 + ny * nx * line_words((int)nz) * 4;  // line-major masks
    b += 2 * lines * 4 + raw * (4 + 8 + 8 + 8);                              // charge list
    b += 3 * lines * 4 + 2 * raw * sizeof(RawEntry) + 64;                    // its build scratch
    b += 2 * (size_t)face_count(p->n[0], p->n[1], p->n[2]) * 8;              // face data, 2 media
    b += na * 5 * 8 + 4 * sizeof(LegDev) + kEnergyScratch * 8 + 4096;        // atoms, legs, energy, result
    return b;
}


void npb::grid_free(npb_grid *g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    batch_forget(g->ctx, g);
    for (auto &c : g->graphs) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
    }
    for (auto &a : g->allocs) g->ctx->release(a.p, a.bytes);
    g->ctx->pinned_release(g->h_result);
    delete g;
}

int npb::grid_build(npb_ctx *ctx, const npb_problem *p, cudaStream_t st, npb_grid **out) {
    *out = nullptr;
    double origin[3];
    int rc = validate(p, origin);
    if (rc) return rc;
    CU(cudaSetDevice(ctx->device));
    auto g = new npb_grid();
    g->ctx = ctx;
    g->geo.nx = p->n[0];
    g->geo.ny = p->n[1];
    g->geo.nz = p->n[2];
    g->geo.pitch = (p->n[0] + 31) / 32 * 32;
    g->geo.h = p->h;
    g->geo.ox = origin[0];
    g->geo.oy = origin[1];
    g->geo.oz = origin[2];
    g->eps_in = p->eps_in;
    g->eps_out = p->eps_out;
    g->kappa2 = p->kappa2;
    g->n_atoms = p->n_atoms;
    const int na = p->n_atoms;
    const int n_lines = g->geo.ny * g->geo.nz;
    const size_t words = (size_t)mask_words_per_row(g->geo.pitch) * n_lines;
    auto guard = [&](int r) {
        if (r) grid_free(g);
        return r;
    };
    if ((rc = galloc(g, &g->d_xyz, std::max(1, 3 * na)))) return guard(rc);
    if ((rc = galloc(g, &g->d_q, std::max(1, na)))) return guard(rc);
    if ((rc = galloc(g, &g->d_rad, std::max(1, na)))) return guard(rc);
    if ((rc = galloc(g, &g->d_mask, words))) return guard(rc);
    if ((rc = galloc(g, &g->d_mask_y, (size_t)g->geo.nz * g->geo.nx * line_words(g->geo.ny)))) return guard(rc);
    if ((rc = galloc(g, &g->d_mask_z, (size_t)g->geo.ny * g->geo.nx * line_words(g->geo.nz)))) return guard(rc);
    if ((rc = galloc(g, &g->d_line_begin, n_lines))) return guard(rc);
    if ((rc = galloc(g, &g->d_line_count, n_lines))) return guard(rc);
    const int n_raw = std::max(1, 8 * na);
    if ((rc = galloc(g, &g->d_ent_x, n_raw))) return guard(rc);
    if ((rc = galloc(g, &g->d_ent_qt, n_raw))) return guard(rc);
    if ((rc = galloc(g, &g->d_ent_off, n_raw))) return guard(rc);
    if ((rc = galloc(g, &g->d_ent_xq, n_raw))) return guard(rc);
    if ((rc = galloc(g, &g->d_result, 8))) return guard(rc);
    if ((rc = galloc(g, &g->d_epart, kEnergyScratch))) return guard(rc);
    CU(cudaMemsetAsync(g->d_epart, 0, kEnergyScratch * sizeof(double), st));
    if ((rc = galloc(g, &g->d_err, 4))) return guard(rc);
    CU(cudaMemsetAsync(g->d_err, 0, 4 * sizeof(int32_t), st));
    if ((rc = ctx->pinned_slot(&g->h_result))) return guard(rc);
    if (na > 0) {
        CU(cudaMemcpyAsync(g->d_xyz, p->xyz, sizeof(double) * 3 * na, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(g->d_q, p->q, sizeof(double) * na, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(g->d_rad, p->radius, sizeof(double) * na, cudaMemcpyHostToDevice, st));
    }
    (void)words;
    // charge list, with scratch released at the end of set-up
    // charge-list scratch stays with the grid so that set-up can be re-run without allocating
    const size_t ints = 3 * (size_t)n_lines + 4;
    g->scratch_bytes = ints * sizeof(int32_t) + 2 * sizeof(RawEntry) * n_raw + 64;
    if ((rc = ctx->alloc(&g->d_scratch, g->scratch_bytes))) return guard(rc);
    g->allocs.push_back({g->d_scratch, g->scratch_bytes});
    ChargeScratch &sc = g->sc;
    sc.count = (int32_t *)g->d_scratch;
    sc.fill = sc.count + n_lines;
    sc.raw_begin = sc.fill + n_lines;
    sc.total = sc.raw_begin + n_lines;
    uintptr_t rp = ((uintptr_t)(sc.total + 4) + 15) & ~(uintptr_t)15;
    sc.raw = (RawEntry *)rp;
    sc.bucket = sc.raw + n_raw;
    if ((rc = grid_setup(g, st))) return guard(rc);
    int32_t total = 0;
    CU(cudaMemcpyAsync(&total, sc.total, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    g->n_ent = total;
    *out = g;
    return 0;
}

// Set-up kernels from the grid's resident atoms: node mask (and half-point masks when
// they exist), charge list, and every face array already in use.  No allocation, no sync.
int npb::grid_setup(npb_grid *g, cudaStream_t st) {
    Profiler &pr = g->ctx->prof;
    const int na = g->n_atoms;
    const size_t words = (size_t)mask_words_per_row(g->geo.pitch) * g->geo.ny * g->geo.nz;
    int rc;
    cudaEvent_t ev{};
    CU(cudaMemsetAsync(g->d_mask, 0, words * 4, st));
    CU(cudaMemsetAsync(g->d_mask_y, 0, sizeof(uint32_t) * g->geo.nz * g->geo.nx * line_words(g->geo.ny), st));
    CU(cudaMemsetAsync(g->d_mask_z, 0, sizeof(uint32_t) * g->geo.ny * g->geo.nx * line_words(g->geo.nz), st));
    for (int d = 0; d < 3; ++d)
        if (g->d_half[d]) CU(cudaMemsetAsync(g->d_half[d], 0, words * 4, st));
    if ((rc = pr.begin(st, &ev))) return rc;
    CU(setup_mask(g->geo, g->d_xyz, g->d_rad, na, g->d_mask, g->d_half[0], g->d_half[1], g->d_half[2], g->d_mask_y,
                  g->d_mask_z, st));
    if ((rc = pr.end(st, ev, K_SETUP_MASK, na > 0 ? 2 : 1))) return rc;  // atoms' bits, transposes
    if ((rc = pr.begin(st, &ev))) return rc;
    CU(setup_charges(g->geo, g->d_xyz, g->d_q, na, g->sc, g->d_line_begin, g->d_line_count, g->d_ent_x,
                     g->d_ent_qt, g->d_ent_off, g->d_ent_xq, st));
    if ((rc = pr.end(st, ev, K_SETUP_CHARGES, na > 0 ? 6 : 4))) return rc;  // the charge-list build
    // face data are recomputed on their next use, only for the precision that uses them
    for (int m = 0; m < 2; ++m)
        for (int k = 0; k < 2; ++k) g->bc_valid[m][k] = false;
    g->vac_fft_valid = false;
    g->fac_valid = false;  // the mask may have changed
    return 0;
}

extern "C" int npb_grid_refresh(npb_grid *g) {
    if (!g) return fail(NPB_EINVAL, "grid is NULL");
    CU(cudaSetDevice(g->ctx->device));
    return grid_setup(g, g->ctx->stream);
}

extern "C" int npb_grid_create(npb_ctx *ctx, const npb_problem *p, npb_grid **out) {
    if (!ctx || !out) return fail(NPB_EINVAL, "ctx/out is NULL");
    return grid_build(ctx, p, ctx->stream, out);
}

extern "C" void npb_grid_destroy(npb_grid *g) { grid_free(g); }

// Face data of a medium, computed on first use -- both media in one pass, with FP64 pair terms
// (parity path) or FP32 pair terms (mixed path) -- then cached.
int npb::grid_boundary(npb_grid *g, int medium, int prec, cudaStream_t st, const double **out) {
    const int kind = prec == NPB_FP64 ? 0 : 1;
    double *&bc = g->d_bc[medium][kind];
    if (!bc || !g->bc_valid[medium][kind]) {
        const int64_t nf = face_count(g->geo.nx, g->geo.ny, g->geo.nz);
        int rc;
        for (int m = 0; m < 2; ++m)
            if (!g->d_bc[m][kind] && (rc = galloc(g, &g->d_bc[m][kind], (size_t)nf))) return rc;
        g->bc_valid[NPB_SOLVENT][kind] = g->bc_valid[NPB_VACUUM][kind] = true;
        cudaEvent_t ev{};
        if ((rc = g->ctx->prof.begin(st, &ev))) return rc;
        CU(setup_boundary_pair(g->geo, g->d_xyz, g->d_q, g->n_atoms, g->eps_out, std::sqrt(g->kappa2), g->eps_in,
                               g->d_bc[NPB_SOLVENT][kind], g->d_bc[NPB_VACUUM][kind], st, kind == 0));
        if ((rc = g->ctx->prof.end(st, ev, K_SETUP_BOUNDARY))) return rc;
    }
    *out = bc;
    return 0;
}

int npb::grid_half_masks(npb_grid *g, cudaStream_t st) {
    if (g->d_half[0]) return 0;
    const size_t words = (size_t)mask_words_per_row(g->geo.pitch) * g->geo.ny * g->geo.nz;
    for (int d = 0; d < 3; ++d) {
        int rc = galloc(g, &g->d_half[d], words);
        if (rc) return rc;
        CU(cudaMemsetAsync(g->d_half[d], 0, words * 4, st));
    }
    // the node mask is rebuilt alongside (atomicOr keeps it identical)
    CU(setup_mask(g->geo, g->d_xyz, g->d_rad, g->n_atoms, g->d_mask, g->d_half[0], g->d_half[1], g->d_half[2],
                  nullptr, nullptr, st));
    return 0;
}

// ------------------------------------------------------------------ legs
// Device leg table order: [s_half, v_half, s_tau, v_tau], so that the legs still running
// after step n (the dt/2 legs) form a prefix.
const int npb::kLegSlot[4] = {2, 0, 3, 1};  // NPB_LEG_* -> slot

int npb::grid_states(npb_grid *g, int prec, cudaStream_t st) {
    if (g->d_u[prec][0]) return 0;
    int n[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    const size_t bytes = state_bytes(n, prec);
    for (int s = 0; s < 4; ++s) {
        unsigned char *p = nullptr;
        int rc = galloc(g, &p, bytes);
        if (rc) return rc;
        CU(cudaMemsetAsync(p, 0, bytes, st));
        g->d_u[prec][s] = p;
    }
    int rc = galloc(g, &g->d_legs[prec], 4);
    if (rc) return rc;
    if (prec == NPB_FP32_SWEEP && (rc = galloc(g, &g->d_line_tab, (size_t)4 * 3 * kLineTabMax))) return rc;
    if (prec == NPB_FP64)
        for (int s = 0; s < 4; ++s)
            for (int d = 0; d < 3; ++d)
                if ((rc = galloc(g, &g->d_fac[s][d], bytes / sizeof(double)))) return rc;
    g->legs_key[prec] = "";
    return 0;
}

LegDev npb::make_leg(const npb_grid *g, int leg, const npb_opts *o) {
    LegDev L{};
    const int prec = o->precision;
    const bool solvent = leg == NPB_LEG_SOLVENT_TAU || leg == NPB_LEG_SOLVENT_HALF;
    const bool half = leg == NPB_LEG_SOLVENT_HALF || leg == NPB_LEG_VACUUM_HALF;
    const double tau = (half ? 0.5 : 1.0) * o->dt / o->alpha;
    const double h = g->geo.h;
    // the Crank-Nicolson sweeps split r between their explicit and implicit halves (Eq. LODCN1_2)
    const double r = tau / (h * h) * (scheme_cn(o->scheme) ? 0.5 : 1.0);
    L.u = g->d_u[prec][kLegSlot[leg]];
    L.nx = g->geo.nx;
    L.ny = g->geo.ny;
    L.nz = g->geo.nz;
    L.pitch = g->geo.pitch;
    L.line_begin = g->d_line_begin;
    L.line_count = g->d_line_count;
    L.ent_x = g->d_ent_x;
    L.ent_qt = g->d_ent_qt;
    L.ent_xq = g->d_ent_xq;
    L.ent_off = g->d_ent_off;
    L.n_ent = g->sc.total;
    L.src = tau * 4.0 * kPi * kBjerrum / (h * h * h);
    L.eps_mode = o->eps_mode == NPB_EPS_MIDPOINT ? 1 : 0;
    for (int d = 0; d < 3; ++d) L.fac[d] = prec == NPB_FP64 ? g->d_fac[kLegSlot[leg]][d] : nullptr;
    if (solvent) {
        const double ei = g->eps_in, eo = g->eps_out;
        L.mask = g->d_mask;
        L.lmask[0] = g->d_mask;
        L.lmask[1] = g->d_mask_y;
        L.lmask[2] = g->d_mask_z;
        L.rE[0] = r * eo;
        L.rE[1] = r * (2.0 * ei * eo / (ei + eo));
        L.rE[2] = r * ei;
        for (int d = 0; d < 3; ++d) L.half[d] = L.eps_mode ? g->d_half[d] : nullptr;
        L.nl_on = g->kappa2 > 0 ? 1 : 0;
        L.nl_q = std::exp(-g->kappa2 * tau);
        L.nl_omq = -std::expm1(-g->kappa2 * tau);
    } else {
        L.mask = nullptr;
        for (int d = 0; d < 3; ++d) L.lmask[d] = nullptr;
        L.rE[0] = L.rE[1] = L.rE[2] = r * g->eps_in;
        for (int d = 0; d < 3; ++d) L.half[d] = nullptr;
        L.nl_on = 0;
        L.nl_q = 1.0;
        L.nl_omq = 0.0;
    }
    for (int i = 0; i < 3; ++i) L.rEf[i] = (float)L.rE[i];
    L.nl_qf = (float)L.nl_q;
    L.nl_omqf = (float)L.nl_omq;
    L.srcf = (float)L.src;
    return L;
}

static int check_opts(const npb_opts *o) {
    if (!o) return fail(NPB_EINVAL, "opts is NULL");
    if (!(o->dt > 0) || !(o->alpha > 0)) return fail(NPB_EINVAL, "dt and alpha must be > 0");
    if (o->n_steps < 0) return fail(NPB_EINVAL, "n_steps < 0");
    if (o->scheme < NPB_LODIE1 || o->scheme > NPB_MAOSCN) return fail(NPB_EINVAL, "unknown scheme %d", o->scheme);
    if (o->precision != NPB_FP64 && o->precision != NPB_FP32_SWEEP)
        return fail(NPB_EINVAL, "unknown precision %d", o->precision);
    if (o->eps_mode != NPB_EPS_HARMONIC && o->eps_mode != NPB_EPS_MIDPOINT)
        return fail(NPB_EINVAL, "unknown eps_mode %d", o->eps_mode);
    return 0;
}

// Upload the leg table (as the solve's opts say) once per change.
int npb::grid_prepare(npb_grid *g, const npb_opts *o, cudaStream_t st) {
    int rc = grid_states(g, o->precision, st);
    if (rc) return rc;
    if (o->eps_mode == NPB_EPS_MIDPOINT && (rc = grid_half_masks(g, st))) return rc;
    if (o->precision == NPB_FP32_SWEEP && (rc = grid_tma(g))) return rc;
    const int prec = o->precision;
    g->u_prec = prec;
    char key[256];
    snprintf(key, sizeof key, "%.17g/%.17g/%d/%d", o->dt, o->alpha, o->eps_mode, scheme_cn(o->scheme) ? 1 : 0);
    if (g->legs_key[prec] != key) {
        for (int leg = 0; leg < 4; ++leg) g->h_legs[prec][kLegSlot[leg]] = make_leg(g, leg, o);
        std::vector<float2> tab;
        if (prec == NPB_FP32_SWEEP && g->d_line_tab) {
            // per slot and direction: the multipliers of a constant-coefficient line (the leg's r*eps
            // outside the molecule; vacuum legs carry r*eps_in everywhere)
            tab.assign((size_t)4 * 3 * kLineTabMax, make_float2(0.f, 0.f));
            const int n3[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
            for (int s = 0; s < 4; ++s) {
                LegDev &L = g->h_legs[prec][s];
                const double e = L.mask ? L.rE[0] : L.rE[2];
                for (int d = 0; d < 3; ++d) {
                    const size_t at = ((size_t)s * 3 + d) * kLineTabMax;
                    line_table(e, n3[d], tab.data() + at);
                    L.line_tab[d] = g->d_line_tab + at;
                }
            }
            CU(cudaMemcpyAsync(g->d_line_tab, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        }
        CU(cudaMemcpyAsync(g->d_legs[prec], g->h_legs[prec], sizeof(LegDev) * 4, cudaMemcpyHostToDevice, st));
        CU(cudaStreamSynchronize(st));
        g->legs_key[prec] = key;
        if (prec == NPB_FP64) g->fac_valid = false;
    }
    if (prec == NPB_FP64 && !g->fac_valid && o->eps_mode == NPB_EPS_HARMONIC) {
        // the FP64 line solver's multipliers: once per legs and mask, before any graph capture
        for (int d = 0; d < 3; ++d)
            CU(launch_line64_factors(d, g->d_legs[prec], 4, g->geo.nx, g->geo.ny, g->geo.nz, st));
        g->fac_valid = true;
    }
    return scheme_additive(o->scheme) ? additive_prepare(g, o, st) : 0;
}

SweepShape npb::shape_for(npb_ctx *ctx, int prec, int dir, int n) {
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tuned.find(tune_key(prec, dir, n));
        if (it != ctx->tuned.end()) return it->second;
    }
    if (prec == NPB_FP32_SWEEP) {
        // the interior-row segments (the line-per-thread-pair kernel, the paper's plain Thomas,
        // measured 3x slower on 257^3: latency-bound at the few warps its shared tiles leave room for)
        const SweepShape best = inner_default_shape(dir, n);
        if (best.tx) return best;
    }
    // FP64: Thomas per line with the multipliers computed once per leg (FP64-unit bound: the fewest
    // FP64 operations per node)
    if (prec == NPB_FP64) return SweepShape{32, 2, 1, 3};
    return default_sweep_shape(prec, dir, n);
}

// The shape a launch can take for legs that cannot use `s`: the line-per-thread-pair kernel needs
// every leg's multiplier table and runs the implicit-Euler sweeps only (no fused Crank-Nicolson
// half step); those legs take the interior-row segments instead.
SweepShape npb::usable_shape(SweepShape s, int dir, int n, bool tables, int flags, int prec) {
    if (s.kind == 3 && prec == NPB_FP64 && !tables) return default_sweep_shape(prec, dir, n);
    if (s.kind == 3 && prec != NPB_FP64 && (!tables || (flags & FUSE_PRE_CN))) return inner_default_shape(dir, n);
    return s;
}

// Tensor maps of the FP32 leg states and of the mask, built once per grid.
int npb::grid_tma(npb_grid *g) {
    if (g->tma_built) return 0;
    g->tma_built = true;
    const int nx = g->geo.nx, ny = g->geo.ny, nz = g->geo.nz, pitch = g->geo.pitch;
    for (int d = 0; d < 3; ++d) {
        g->tma_g[d] = tma_geometry(d, nx, ny, nz, pitch);
        bool ok = g->tma_g[d].ok && g->d_u[NPB_FP32_SWEEP][0] != nullptr;
        const uint32_t *lm = d == 0 ? g->d_mask : (d == 1 ? g->d_mask_y : g->d_mask_z);
        for (int v = 0; v < tma_variant_count(d) && ok; ++v) {  // x: 8 lines per tile; y/z: 32, 16 or 8
            for (int s = 0; s < 4 && ok; ++s)
                ok = tma_encode_state(&g->tma_u[d][v][s], g->d_u[NPB_FP32_SWEEP][s], d, g->tma_g[d], nx, ny, nz,
                                      pitch, tma_variant_tx(d, v));
            if (ok) ok = tma_encode_mask(&g->tma_m[d][v], lm, d, g->tma_g[d], nx, ny, nz, tma_variant_tx(d, v));
        }
        g->tma_ok[d] = ok;
    }
    return 0;
}

// One sweep direction over legs [slot0, slot0 + n_legs): the TMA pipeline for FP32 when
// the shape asks for it and the grid's geometry allows it, else the one-tile-per-block kernel.
cudaError_t npb::launch_dir(npb_grid *g, int prec, int d, SweepShape shape, int slot0, int n_legs, int flags,
                            cudaStream_t st) {
    const int nx = g->geo.nx, ny = g->geo.ny, nz = g->geo.nz;
    const int n_dir[3] = {nx, ny, nz};
    // the TMA kernels take eps at half points from the node mask (harmonic reading only)
    if (shape.kind >= 1 && prec == NPB_FP32_SWEEP && g->tma_ok[d] && n_legs <= kTmaMaxLegs &&
        g->h_legs[prec][slot0].eps_mode == 0) {
        TmaLaunch P;
        memset(&P, 0, sizeof P);
        bool tables = true;
        for (int i = 0; i < n_legs; ++i) tables = tables && g->h_legs[prec][slot0 + i].line_tab[d] != nullptr;
        shape = usable_shape(shape, d, n_dir[d], tables, flags);
        const int v = tma_variant(d, shape.tx);
        if (v < 0) return cudaErrorInvalidValue;
        for (int i = 0; i < n_legs; ++i) {
            P.umap[i] = g->tma_u[d][v][slot0 + i];
            P.mmap[i] = g->tma_m[d][v];
            P.legs[i] = g->h_legs[prec][slot0 + i];
        }
        P.n_legs = n_legs;
        P.err = g->d_err;
        if (g->ctx->probe_cycles > 0) {
            const cudaError_t ep = launch_wait_probe(g->d_err, g->ctx->probe_cycles, g->ctx->sm_count, st);
            if (ep != cudaSuccess) return ep;
        }
        if (shape.kind == 3) return launch_sweep_line(d, P, g->tma_g[d], flags, shape, g->ctx->sm_count, st);
        if (shape.kind == 2) return launch_sweep_inner(d, P, g->tma_g[d], flags, shape, g->ctx->sm_count, st);
        return launch_sweep_tma(d, P, g->tma_g[d], flags, shape, g->ctx->sm_count, st);
    }
    if (shape.kind == 3 && prec == NPB_FP64 && g->fac_valid && g->h_legs[prec][slot0].eps_mode == 0 &&
        !(flags & FUSE_PRE_CN))
        return launch_sweep_line64(d, g->d_legs[prec] + slot0, n_legs, nx, ny, nz, flags, st);
    if (shape.kind >= 1) shape = default_sweep_shape(prec, d, n_dir[d]);
    return launch_sweep(prec, d, g->d_legs[prec] + slot0, n_legs, nx, ny, nz, flags, shape, st);
}

// One LOD step for an arbitrary list of legs of equal grid size, precision, scheme and eps
// reading (possibly from different grids).  d_table holds their LegDev entries in the same order
// (the one-tile-per-block kernels and the source stage read it).  FP32 legs use the
// TMA-pipelined sweeps, in launches of up to kTmaMaxLegs legs, where every grid's geometry
// allows it; otherwise the one-tile-per-block sweeps.  The source stage is fused into the x
// sweep, except with the kind-1 TMA kernel and for large charge lists, where it is a launch of
// its own over the charge entries.
int npb::step_legs(npb_ctx *ctx, const LegRef *refs, int n, const LegDev *d_table, int prec, int scheme,
                   cudaStream_t st) {
    if (n <= 0) return 0;
    Profiler &pr = ctx->prof;
    const GridGeom &geo = refs[0].g->geo;
    const int nx = geo.nx, ny = geo.ny, nz = geo.nz;
    const int n_dir[3] = {nx, ny, nz};
    SweepShape shape[3];
    bool tma[3];
    const bool cn_scheme = scheme_cn(scheme);
    for (int d = 0; d < 3; ++d) {
        shape[d] = shape_for(ctx, prec, d, n_dir[d]);
        bool tables = true;
        for (int i = 0; i < n; ++i) tables = tables && refs[i].g->h_legs[prec][refs[i].slot].line_tab[d] != nullptr;
        if (prec == NPB_FP64) {  // the multipliers exist for harmonic-eps legs of prepared grids
            tables = true;
            for (int i = 0; i < n; ++i)
                tables = tables && refs[i].g->fac_valid && refs[i].g->h_legs[prec][refs[i].slot].eps_mode == 0;
        }
        shape[d] = usable_shape(shape[d], d, n_dir[d], tables, cn_scheme ? FUSE_PRE_CN : 0, prec);
        bool ok = shape[d].kind >= 1 && prec == NPB_FP32_SWEEP;
        for (int i = 0; i < n && ok; ++i)
            ok = refs[i].g->tma_ok[d] && refs[i].g->h_legs[prec][refs[i].slot].eps_mode == 0;
        tma[d] = ok && tma_variant(d, shape[d].tx) >= 0;
        const bool line64 = prec == NPB_FP64 && shape[d].kind == 3;  // no TMA: direct global access
        if (shape[d].kind >= 1 && !tma[d] && !line64) shape[d] = default_sweep_shape(prec, d, n_dir[d]);
    }
    cudaEvent_t ev{};
    int rc;
    // Crank-Nicolson schemes: each direction is the explicit half step followed by the implicit
    // sweep; the first stage (S or N) comes before the x half step (fused into its load, or a launch
    // of its own where the half step is a launch of its own)
    const bool cn = scheme_cn(scheme);
    const bool first_n = scheme == NPB_LODIE1 || scheme == NPB_LODCN1;
    // Crank-Nicolson: the interior-row kernels take the explicit half step on their loaded lines
    // (after a fused S); elsewhere it is its own launch before each sweep
    bool cn_fused = cn;
    for (int d = 0; d < 3; ++d) cn_fused = cn_fused && tma[d] && shape[d].kind == 2;
    // LODIE2's source stage: fused into the x sweep's load except by the kind-1 TMA kernel, before
    // an explicit half step of its own launch, and for charge lists of kSourceApartEntries or more
    int ent_max = 1;  // bound on the legs' charge entries (8 trilinear nodes per atom)
    for (int i = 0; i < n; ++i) ent_max = std::max(ent_max, 8 * refs[i].g->n_atoms);
    const bool src_apart =
        !first_n && ((cn && !cn_fused) || (tma[0] && (shape[0].kind == 1 || ent_max >= kSourceApartEntries)));
    if (src_apart) {
        bool one_grid = n <= 4;  // legs of one grid: everything by value, no table reads
        for (int i = 1; i < n && one_grid; ++i) one_grid = refs[i].g == refs[0].g;
        if ((rc = pr.begin(st, &ev))) return rc;
        if (one_grid) {
            SourceLegs S{};
            const npb_grid *g0 = refs[0].g;
            for (int i = 0; i < n; ++i) {
                const LegDev &L = g0->h_legs[prec][refs[i].slot];
                S.u[i] = L.u;
                S.srcf[i] = L.srcf;
                S.src[i] = L.src;
            }
            S.ent_off = g0->d_ent_off;
            S.ent_xq = g0->d_ent_xq;
            S.ent_qt = g0->d_ent_qt;
            S.n_ent = g0->sc.total;
            S.n_slots = 8 * g0->n_atoms;
            S.n_legs = n;
            CU(launch_source_legs(prec, S, st));
        } else {
            CU(launch_source_entries(prec, d_table, n, ent_max, st));
        }
        if ((rc = pr.end(st, ev, K_SOURCE))) return rc;
    }
    if (cn && first_n && !cn_fused) {
        if ((rc = pr.begin(st, &ev))) return rc;
        CU(launch_nonlinear(prec, d_table, n, nx, ny, nz, st));
        if ((rc = pr.end(st, ev, K_NONLINEAR))) return rc;
    }
    for (int d = 0; d < 3; ++d) {
        int flags = 0;
        if (d == 0 && (!cn || cn_fused)) flags = !first_n ? (src_apart ? 0 : FUSE_PRE_SRC) : FUSE_PRE_NL;
        if (d == 2 && !first_n) flags = FUSE_POST_NL;
        if (cn_fused) flags |= FUSE_PRE_CN;
        if (cn && !cn_fused) {
            if ((rc = pr.begin(st, &ev))) return rc;
            CU(launch_cn_explicit(prec, d_table, n, d, st));
            if ((rc = pr.end(st, ev, K_CN_EXPLICIT))) return rc;
        }
        if ((rc = pr.begin(st, &ev))) return rc;
        if (tma[d]) {
            const int v = tma_variant(d, shape[d].tx);
            for (int c0 = 0; c0 < n; c0 += kTmaMaxLegs) {
                const int m = std::min(kTmaMaxLegs, n - c0);
                TmaLaunch P;
                memset(&P, 0, sizeof P);
                for (int i = 0; i < m; ++i) {
                    const LegRef &r = refs[c0 + i];
                    P.umap[i] = r.g->tma_u[d][v][r.slot];
                    P.mmap[i] = r.g->tma_m[d][v];
                    P.legs[i] = r.g->h_legs[prec][r.slot];
                }
                P.n_legs = m;
                P.err = refs[c0].g->d_err;
                if (ctx->probe_cycles > 0)
                    for (int i = 0; i < m; ++i)
                        CU(launch_wait_probe(refs[c0 + i].g->d_err, ctx->probe_cycles, ctx->sm_count, st));
                if (shape[d].kind == 3) CU(launch_sweep_line(d, P, refs[c0].g->tma_g[d], flags, shape[d], ctx->sm_count, st));
                else if (shape[d].kind == 2) CU(launch_sweep_inner(d, P, refs[c0].g->tma_g[d], flags, shape[d], ctx->sm_count, st));
                else CU(launch_sweep_tma(d, P, refs[c0].g->tma_g[d], flags, shape[d], ctx->sm_count, st));
            }
        } else if (prec == NPB_FP64 && shape[d].kind == 3) {
            CU(launch_sweep_line64(d, d_table, n, nx, ny, nz, flags, st));
        } else {
            CU(launch_sweep(prec, d, d_table, n, nx, ny, nz, flags, shape[d], st));
        }
        if ((rc = pr.end(st, ev, K_SWEEP_X + d))) return rc;
    }
    if (first_n) {
        if ((rc = pr.begin(st, &ev))) return rc;
        CU(launch_source(prec, d_table, n, ny, nz, st));
        if ((rc = pr.end(st, ev, K_SOURCE))) return rc;
    }
    return 0;
}

// One step of `scheme` for legs [slot0, slot0 + n_legs) of one grid's leg table.
int npb::run_step(npb_grid *g, int prec, int scheme, int slot0, int n_legs, cudaStream_t st) {
    if (scheme_additive(scheme)) return additive_step(g, prec, scheme, slot0, n_legs, nullptr, st);
    LegRef refs[4];
    for (int i = 0; i < n_legs; ++i) refs[i] = {g, slot0 + i};
    return step_legs(g->ctx, refs, n_legs, g->d_legs[prec] + slot0, prec, scheme, st);
}

int npb::init_legs(npb_grid *g, int prec, const int *legs, int n, cudaStream_t st) {
    for (int i = 0; i < n; ++i) {
        const int leg = legs[i];
        const int medium = (leg == NPB_LEG_SOLVENT_TAU || leg == NPB_LEG_SOLVENT_HALF) ? NPB_SOLVENT : NPB_VACUUM;
        const double *bc = nullptr;
        int rc = grid_boundary(g, medium, prec, st, &bc);
        if (rc) return rc;
        cudaEvent_t ev{};
        if ((rc = g->ctx->prof.begin(st, &ev))) return rc;
        CU(init_leg(prec, g->geo, bc, g->d_u[prec][kLegSlot[leg]], st));
        if ((rc = g->ctx->prof.end(st, ev, K_INIT))) return rc;
    }
    return 0;
}

// The whole RE+V solve as a stream of launches: init, steps, energy, result read-back.
int npb::enqueue_energy(npb_grid *g, const npb_opts *o, cudaStream_t st) {
    const int prec = o->precision;
    const int re = o->richardson ? 1 : 0;
    const int n = o->n_steps;
    const int legs_re[4] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_SOLVENT_HALF, NPB_LEG_VACUUM_TAU, NPB_LEG_VACUUM_HALF};
    const int legs_plain[2] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_VACUUM_TAU};
    int rc;
    if (!o->vacuum_recovery) {  // Eq. (deltaG2): solvent legs only, phi_0^FFT for the vacuum
        const int legs_s[2] = {NPB_LEG_SOLVENT_TAU, NPB_LEG_SOLVENT_HALF};
        if ((rc = init_legs(g, prec, legs_s, re ? 2 : 1, st))) return rc;
        const int s_tau = kLegSlot[NPB_LEG_SOLVENT_TAU], s_half = kLegSlot[NPB_LEG_SOLVENT_HALF];
        for (int s = 0; s < n; ++s) {
            if ((rc = run_step(g, prec, o->scheme, s_tau, 1, st))) return rc;
            if (re && (rc = run_step(g, prec, o->scheme, s_half, 1, st))) return rc;
        }
        if (re)
            for (int s = 0; s < n; ++s)
                if ((rc = run_step(g, prec, o->scheme, s_half, 1, st))) return rc;
    } else {
    rc = init_legs(g, prec, re ? legs_re : legs_plain, re ? 4 : 2, st);
    if (rc) return rc;
    if (re) {
        // steps 1..n: all four legs (slots 0..3); steps n+1..2n: the dt/2 legs (slots 0..1)
        for (int s = 0; s < n; ++s)
            if ((rc = run_step(g, prec, o->scheme, 0, 4, st))) return rc;
        for (int s = 0; s < n; ++s)
            if ((rc = run_step(g, prec, o->scheme, 0, 2, st))) return rc;
    } else {
        // slots 2..3 hold the dt legs
        for (int s = 0; s < n; ++s)
            if ((rc = run_step(g, prec, o->scheme, 2, 2, st))) return rc;
    }
    }
    cudaEvent_t ev{};
    if ((rc = g->ctx->prof.begin(st, &ev))) return rc;
    void *const *U = g->d_u[prec];
    CU(launch_energy(prec, U[kLegSlot[0]], U[kLegSlot[1]], U[kLegSlot[2]], U[kLegSlot[3]],
                     g->d_ent_off, g->d_ent_qt, g->sc.total, re, o->vacuum_recovery ? nullptr : g->d_vac_fft,
                     g->d_epart, g->d_result, st));
    if ((rc = g->ctx->prof.end(st, ev, K_ENERGY))) return rc;
    CU(cudaMemcpyAsync(g->h_result, g->d_result, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(reinterpret_cast<int32_t *>(g->h_result + 1), g->d_err, sizeof(int32_t),
                       cudaMemcpyDeviceToHost, st));
    return 0;
}

// The RE+V energy of a grid whose legs have run, into its pinned result slot (no sync).
int npb::enqueue_energy_reduce(npb_grid *g, int prec, int richardson, cudaStream_t st) {
    void *const *U = g->d_u[prec];
    CU(launch_energy(prec, U[kLegSlot[0]], U[kLegSlot[1]], U[kLegSlot[2]], U[kLegSlot[3]], g->d_ent_off,
                     g->d_ent_qt, g->sc.total, richardson, nullptr, g->d_epart, g->d_result, st));
    CU(cudaMemcpyAsync(g->h_result, g->d_result, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(reinterpret_cast<int32_t *>(g->h_result + 1), g->d_err, sizeof(int32_t),
                       cudaMemcpyDeviceToHost, st));
    return 0;
}

// A device wait that expired leaves its flag set: report it, then clear it.
int npb::grid_check_err(npb_grid *g, cudaStream_t st, int host_copy) {
    int32_t e = 0;
    if (host_copy) {
        e = *reinterpret_cast<int32_t *>(g->h_result + 1);
    } else {
        CU(cudaMemcpyAsync(&e, g->d_err, sizeof e, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
    }
    if (e) {
        CU(cudaMemsetAsync(g->d_err, 0, sizeof(int32_t), st));
        CU(cudaStreamSynchronize(st));
        return fail(NPB_ETIMEOUT, "a bounded device wait expired in a sweep (tile copies did not complete)");
    }
    return 0;
}

extern "C" int npb_energy(npb_grid *g, const npb_opts *o, double *dG) {
    if (!g || !dG) return fail(NPB_EINVAL, "grid/dG is NULL");
    int rc = check_opts(o);
    if (rc) return rc;
    npb_ctx *ctx = g->ctx;
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    if ((rc = grid_prepare(g, o, st))) return rc;
    // boundary data (and phi_0^FFT) are computed on first use, outside any graph capture
    const int legs[4] = {0, 1, 2, 3};
    for (int i = 0; i < 4; ++i) {
        const double *bc;
        if ((rc = grid_boundary(g, legs[i] < 2 ? NPB_SOLVENT : NPB_VACUUM, o->precision, st, &bc))) return rc;
    }
    if (!o->vacuum_recovery && (rc = grid_vacuum_fft(g, o->precision, st))) return rc;
    g->last_richardson = o->richardson ? 1 : 0;
    g->last_vacuum_lod = o->vacuum_recovery ? 1 : 0;
    const bool use_graph = !ctx->prof.enabled && st != nullptr && ctx->use_graphs && ctx->probe_cycles == 0;
    if (use_graph) {
        // the line-solver shapes are part of the key: a shape pinned after a capture takes effect
        const int nd[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
        SweepShape sh[3];
        for (int d = 0; d < 3; ++d) sh[d] = shape_for(ctx, o->precision, d, nd[d]);
        char key[384];
        snprintf(key, sizeof key, "%d/%d/%d/%d/%d/%d/%d.%d.%d.%d/%d.%d.%d.%d/%d.%d.%d.%d/%s", o->precision, o->scheme,
                 o->richardson, o->n_steps, o->eps_mode, o->vacuum_recovery, sh[0].kind, sh[0].tx, sh[0].seg,
                 sh[0].len, sh[1].kind, sh[1].tx, sh[1].seg, sh[1].len, sh[2].kind, sh[2].tx, sh[2].seg, sh[2].len,
                 g->legs_key[o->precision].c_str());
        GraphCache *hit = nullptr;
        for (auto &c : g->graphs)
            if (c.key == key && c.stream == st) hit = &c;
        // A solve seen for the first time runs as direct launches (the launches overlap the GPU
        // work); the graph is captured when the same solve comes back, where replay pays off.
        const std::string seen = std::string(key) + "@" + std::to_string((uintptr_t)st);
        if (!hit && g->seen.insert(seen).second) {
            if ((rc = enqueue_energy(g, o, st))) return rc;
        } else if (!hit) {
            cudaGraph_t graph;
            CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            rc = enqueue_energy(g, o, st);
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (rc) {
                if (ec == cudaSuccess) cudaGraphDestroy(graph);
                return rc;
            }
            CU(ec);
            GraphCache c;
            c.key = key;
            c.stream = st;
            cudaError_t ei = cudaGraphInstantiate(&c.exec, graph, 0);
            cudaGraphDestroy(graph);
            CU(ei);
            g->graphs.push_back(c);
            hit = &g->graphs.back();
        }
        if (hit) CU(cudaGraphLaunch(hit->exec, st));
    } else {
        if ((rc = enqueue_energy(g, o, st))) return rc;
    }
    CU(cudaStreamSynchronize(st));
    if ((rc = grid_check_err(g, st, 1))) return rc;
    *dG = g->h_result[0];
    return NPB_OK;
}

extern "C" int npb_lod_solve(npb_grid *g, const npb_opts *o, int32_t medium, double dt_scale) {
    if (!g) return fail(NPB_EINVAL, "grid is NULL");
    int rc = check_opts(o);
    if (rc) return rc;
    if (medium != NPB_SOLVENT && medium != NPB_VACUUM) return fail(NPB_EINVAL, "unknown medium %d", medium);
    if (dt_scale != 1.0 && dt_scale != 0.5) return fail(NPB_EINVAL, "dt_scale must be 1 or 0.5");
    CU(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    if ((rc = grid_prepare(g, o, st))) return rc;
    const int leg = medium == NPB_SOLVENT ? (dt_scale == 1.0 ? NPB_LEG_SOLVENT_TAU : NPB_LEG_SOLVENT_HALF)
                                          : (dt_scale == 1.0 ? NPB_LEG_VACUUM_TAU : NPB_LEG_VACUUM_HALF);
    if ((rc = init_legs(g, o->precision, &leg, 1, st))) return rc;
    const int steps = dt_scale == 1.0 ? o->n_steps : 2 * o->n_steps;
    for (int s = 0; s < steps; ++s)
        if ((rc = run_step(g, o->precision, o->scheme, kLegSlot[leg], 1, st))) return rc;
    CU(cudaStreamSynchronize(st));
    return grid_check_err(g, st, 0);
}

extern "C" int npb_potential(npb_grid *g, int32_t leg, double *host_out, size_t n_elems) {
    if (!g || !host_out) return fail(NPB_EINVAL, "grid/host_out is NULL");
    if (leg < 0 || leg > NPB_LEG_RECOVERED) return fail(NPB_EINVAL, "unknown leg %d", leg);
    const size_t total = (size_t)g->geo.nx * g->geo.ny * g->geo.nz;
    if (n_elems != total) return fail(NPB_EINVAL, "n_elems %zu != nx*ny*nz %zu", n_elems, total);
    if (g->u_prec < 0 || !g->d_u[g->u_prec][0]) return fail(NPB_EINVAL, "no solve has run on this grid");
    if (leg == NPB_LEG_RECOVERED && !g->last_vacuum_lod)
        return fail(NPB_EINVAL, "the recovered potential needs a solve with the LOD vacuum legs");
    CU(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    int rc;
    if (leg >= NPB_LEG_VACUUM_FFT && (rc = grid_vacuum_fft(g, g->u_prec, st))) return rc;
    void *tmp = nullptr;
    if ((rc = g->ctx->alloc(&tmp, total * sizeof(double)))) return rc;
    void *const *U = g->d_u[g->u_prec];
    cudaError_t e;
    if (leg == NPB_LEG_VACUUM_FFT)
        e = unpad_state(NPB_FP64, g->geo, g->d_vac_fft, (double *)tmp, st);
    else if (leg == NPB_LEG_RECOVERED)
        e = launch_recover(g->u_prec, g->geo, U[kLegSlot[0]], U[kLegSlot[1]], U[kLegSlot[2]], U[kLegSlot[3]],
                           g->d_vac_fft, g->last_richardson, (double *)tmp, st);
    else
        e = unpad_state(g->u_prec, g->geo, U[kLegSlot[leg]], (double *)tmp, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, total * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    g->ctx->release(tmp, total * sizeof(double));
    if (e != cudaSuccess) return fail(NPB_ECUDA, "potential read-back failed: %s", cudaGetErrorString(e));
    return NPB_OK;
}

extern "C" int npb_apply(npb_grid *g, const npb_opts *o, int32_t leg, int32_t op, double *u_inout,
                         size_t n_elems) {
    if (!g || !u_inout) return fail(NPB_EINVAL, "grid/u_inout is NULL");
    int rc = check_opts(o);
    if (rc) return rc;
    if (leg < 0 || leg > 3) return fail(NPB_EINVAL, "unknown leg %d", leg);
    if (op < NPB_OP_SOURCE || op > NPB_OP_STEP) return fail(NPB_EINVAL, "unknown op %d", op);
    const size_t total = (size_t)g->geo.nx * g->geo.ny * g->geo.nz;
    if (n_elems != total) return fail(NPB_EINVAL, "n_elems %zu != nx*ny*nz %zu", n_elems, total);
    CU(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    if ((rc = grid_prepare(g, o, st))) return rc;
    void *tmp = nullptr;
    if ((rc = g->ctx->alloc(&tmp, total * sizeof(double)))) return rc;
    const int slot = kLegSlot[leg];
    const int prec = o->precision;
    void *u = g->d_u[prec][slot];
    const LegDev *legs = g->d_legs[prec] + slot;
    const int nx = g->geo.nx, ny = g->geo.ny, nz = g->geo.nz;
    cudaError_t e = cudaMemcpyAsync(tmp, u_inout, total * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(u, 0, state_bytes(&g->geo.nx, prec), st);
    if (e == cudaSuccess) e = pad_state(prec, g->geo, (const double *)tmp, u, st);
    if (e == cudaSuccess) {
        const int n_dir[3] = {nx, ny, nz};
        switch (op) {
        case NPB_OP_SOURCE: e = launch_source(prec, legs, 1, ny, nz, st); break;
        case NPB_OP_NONLINEAR: e = launch_nonlinear(prec, legs, 1, nx, ny, nz, st); break;
        case NPB_OP_SWEEP_X:
        case NPB_OP_SWEEP_Y:
        case NPB_OP_SWEEP_Z: {
            const int d = op - NPB_OP_SWEEP_X;
            e = launch_dir(g, prec, d, shape_for(g->ctx, prec, d, n_dir[d]), slot, 1, 0, st);
            break;
        }
        case NPB_OP_STEP: {
            int r2 = run_step(g, prec, o->scheme, slot, 1, st);
            if (r2) {
                cudaStreamSynchronize(st);
                g->ctx->release(tmp, total * sizeof(double));
                return r2;
            }
            break;
        }
        }
    }
    if (e == cudaSuccess) e = unpad_state(prec, g->geo, u, (double *)tmp, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u_inout, tmp, total * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    g->ctx->release(tmp, total * sizeof(double));
    if (e != cudaSuccess) return fail(NPB_ECUDA, "npb_apply failed: %s", cudaGetErrorString(e));
    return grid_check_err(g, st, 0);
}

// n LOD steps of one leg from a caller-given state, optionally with a dense source in place of the
// molecule's charges (the manufactured-solution benchmark of Sec. 4.1).
extern "C" int npb_lod_run(npb_grid *g, const npb_opts *o, int32_t leg, int32_t n_steps, double *u_inout,
                           const double *source, size_t n_elems) {
    if (!g || !u_inout) return fail(NPB_EINVAL, "grid/u_inout is NULL");
    int rc = check_opts(o);
    if (rc) return rc;
    if (leg < 0 || leg > 3) return fail(NPB_EINVAL, "unknown leg %d", leg);
    if (n_steps < 0) return fail(NPB_EINVAL, "n_steps < 0");
    const size_t total = (size_t)g->geo.nx * g->geo.ny * g->geo.nz;
    if (n_elems != total) return fail(NPB_EINVAL, "n_elems %zu != nx*ny*nz %zu", n_elems, total);
    CU(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    if ((rc = grid_prepare(g, o, st))) return rc;
    const int slot = kLegSlot[leg];
    const int prec = o->precision;
    void *u = g->d_u[prec][slot];
    const size_t sbytes = state_bytes(&g->geo.nx, prec);
    void *tmp = nullptr, *src = nullptr;
    if ((rc = g->ctx->alloc(&tmp, total * sizeof(double)))) return rc;
    if (source && (rc = g->ctx->alloc(&src, sbytes))) {
        g->ctx->release(tmp, total * sizeof(double));
        return rc;
    }
    auto done = [&](int r) {
        cudaStreamSynchronize(st);
        g->ctx->release(tmp, total * sizeof(double));
        if (src) g->ctx->release(src, sbytes);
        return r;
    };
    cudaError_t e = cudaSuccess;
    if (source) {  // tau * rho in the state's precision and layout
        const bool half = leg == NPB_LEG_SOLVENT_HALF || leg == NPB_LEG_VACUUM_HALF;
        const double tau = (half ? 0.5 : 1.0) * o->dt / o->alpha;
        std::vector<double> scaled(source, source + total);
        for (double &v : scaled) v *= tau;
        e = cudaMemcpyAsync(tmp, scaled.data(), total * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(src, 0, sbytes, st);
        if (e == cudaSuccess) e = pad_state(prec, g->geo, (const double *)tmp, src, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `scaled` goes out of scope
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, u_inout, total * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(u, 0, sbytes, st);
    if (e == cudaSuccess) e = pad_state(prec, g->geo, (const double *)tmp, u, st);
    if (e != cudaSuccess) return done(fail(NPB_ECUDA, "npb_lod_run failed: %s", cudaGetErrorString(e)));
    const int n_dir[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    for (int s = 0; s < n_steps; ++s) {
        if (!source) {
            if ((rc = run_step(g, prec, o->scheme, slot, 1, st))) return done(rc);
            continue;
        }
        if (scheme_additive(o->scheme)) {  // each directional part adds its share of tau rho
            if ((rc = additive_step(g, prec, o->scheme, slot, 1, src, st))) return done(rc);
            continue;
        }
        // the stages of Sec. 3.1 with S = u + tau rho: LODIE2/LODCN2 S, X, Y, Z, N;
        // LODIE1/LODCN1 N, X, Y, Z, S (Crank-Nicolson: each sweep after its explicit half step)
        const bool cn = scheme_cn(o->scheme);
        const bool first_n = o->scheme == NPB_LODIE1 || o->scheme == NPB_LODCN1;
        const LegDev *legs = g->d_legs[prec] + slot;
        if (!first_n) e = launch_add_interior(prec, g->geo, src, u, 1.0, st);
        else if (cn) e = launch_nonlinear(prec, legs, 1, n_dir[0], n_dir[1], n_dir[2], st);
        for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
            int flags = 0;
            if (d == 0 && first_n && !cn) flags = FUSE_PRE_NL;
            if (d == 2 && !first_n) flags = FUSE_POST_NL;
            if (cn) e = launch_cn_explicit(prec, legs, 1, d, st);
            if (e == cudaSuccess) e = launch_dir(g, prec, d, shape_for(g->ctx, prec, d, n_dir[d]), slot, 1, flags, st);
        }
        if (e == cudaSuccess && first_n) e = launch_add_interior(prec, g->geo, src, u, 1.0, st);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = unpad_state(prec, g->geo, u, (double *)tmp, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u_inout, tmp, total * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(fail(NPB_ECUDA, "npb_lod_run failed: %s", cudaGetErrorString(e)));
    done(0);
    return grid_check_err(g, st, 0);
}

// n explicit Euler steps of one leg from a caller-given state (the steady-state reference).
extern "C" int npb_euler_run(npb_grid *g, const npb_opts *opts, int32_t leg, int32_t n_steps, double *u_inout,
                             size_t n_elems) {
    if (!g || !u_inout) return fail(NPB_EINVAL, "grid/u_inout is NULL");
    int rc = check_opts(opts);
    if (rc) return rc;
    if (leg < 0 || leg > 3) return fail(NPB_EINVAL, "unknown leg %d", leg);
    if (n_steps < 0) return fail(NPB_EINVAL, "n_steps < 0");
    const size_t total = (size_t)g->geo.nx * g->geo.ny * g->geo.nz;
    if (n_elems != total) return fail(NPB_EINVAL, "n_elems %zu != nx*ny*nz %zu", n_elems, total);
    npb_opts o = *opts;
    o.scheme = NPB_LODIE2;  // the leg constants with the full r = tau/h^2
    CU(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    if ((rc = grid_prepare(g, &o, st))) return rc;
    const int slot = kLegSlot[leg];
    const int prec = o.precision;
    void *u = g->d_u[prec][slot];
    const size_t sbytes = state_bytes(&g->geo.nx, prec);
    const bool solvent = leg == NPB_LEG_SOLVENT_TAU || leg == NPB_LEG_SOLVENT_HALF;
    const bool half = leg == NPB_LEG_SOLVENT_HALF || leg == NPB_LEG_VACUUM_HALF;
    const double tau = (half ? 0.5 : 1.0) * o.dt / o.alpha;
    void *tmp = nullptr, *work = nullptr;
    if ((rc = g->ctx->alloc(&tmp, total * sizeof(double)))) return rc;
    if ((rc = g->ctx->alloc(&work, sbytes))) {
        g->ctx->release(tmp, total * sizeof(double));
        return rc;
    }
    const LegDev *legs = g->d_legs[prec] + slot;
    cudaError_t e = cudaMemcpyAsync(tmp, u_inout, total * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(u, 0, sbytes, st);
    if (e == cudaSuccess) e = pad_state(prec, g->geo, (const double *)tmp, u, st);
    for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
        e = launch_euler_step(prec, legs, u, work, g->geo, solvent ? tau * g->kappa2 : 0.0, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, work, sbytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = launch_source(prec, legs, 1, g->geo.ny, g->geo.nz, st);
    }
    if (e == cudaSuccess) e = unpad_state(prec, g->geo, u, (double *)tmp, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u_inout, tmp, total * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamSynchronize(st);
    g->ctx->release(tmp, total * sizeof(double));
    g->ctx->release(work, sbytes);
    if (e != cudaSuccess) return fail(NPB_ECUDA, "npb_euler_run failed: %s", cudaGetErrorString(e));
    return NPB_OK;
}

extern "C" int npb_grid_export(npb_grid *g, int32_t what, void *host_out, size_t n_elems) {
    if (!g || !host_out) return fail(NPB_EINVAL, "grid/host_out is NULL");
    const size_t total = (size_t)g->geo.nx * g->geo.ny * g->geo.nz;
    if (n_elems != total) return fail(NPB_EINVAL, "n_elems %zu != nx*ny*nz %zu", n_elems, total);
    CU(cudaSetDevice(g->ctx->device));
    cudaStream_t st = g->ctx->stream;
    void *tmp = nullptr;
    int rc = g->ctx->alloc(&tmp, total * sizeof(double));
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    size_t out_bytes = total * sizeof(double);
    switch (what) {
    case NPB_EXPORT_MASK:
        e = mask_dense(g->geo, g->d_mask, (uint8_t *)tmp, st);
        out_bytes = total;
        break;
    case NPB_EXPORT_QTILDE:
        e = cudaMemsetAsync(tmp, 0, total * sizeof(double), st);
        if (e == cudaSuccess)
            e = qt_dense(g->geo, g->d_line_begin, g->d_line_count, g->d_ent_x, g->d_ent_qt, (double *)tmp, st);
        break;
    case NPB_EXPORT_U0_SOLVENT:
    case NPB_EXPORT_U0_VACUUM: {
        const double *bc = nullptr;
        rc = grid_boundary(g, what == NPB_EXPORT_U0_SOLVENT ? NPB_SOLVENT : NPB_VACUUM, NPB_FP64, st, &bc);
        if (rc) {
            g->ctx->release(tmp, total * sizeof(double));
            return rc;
        }
        void *pad = nullptr;
        int n3[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
        const size_t pb = state_bytes(n3, NPB_FP64);
        if ((rc = g->ctx->alloc(&pad, pb))) {
            g->ctx->release(tmp, total * sizeof(double));
            return rc;
        }
        e = init_leg(NPB_FP64, g->geo, bc, pad, st);
        if (e == cudaSuccess) e = unpad_state(NPB_FP64, g->geo, pad, (double *)tmp, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        g->ctx->release(pad, pb);
        break;
    }
    default:
        g->ctx->release(tmp, total * sizeof(double));
        return fail(NPB_EINVAL, "unknown export %d", what);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    g->ctx->release(tmp, total * sizeof(double));
    if (e != cudaSuccess) return fail(NPB_ECUDA, "export failed: %s", cudaGetErrorString(e));
    return NPB_OK;
}
