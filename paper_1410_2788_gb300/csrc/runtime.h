// runtime.h -- host-side state behind the opaque handles of include/npb.h.
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/npb.h"
#include "npb_internal.cuh"
#include "setup_kernels.cuh"
#include "tma.h"

namespace npb {

constexpr int kMaxLine = 288;  // longest line the instantiated solver shapes cover

enum KernelKind {
    K_SWEEP_X = 0, K_SWEEP_Y, K_SWEEP_Z, K_NONLINEAR, K_SOURCE, K_INIT, K_ENERGY,
    K_SETUP_MASK, K_SETUP_CHARGES, K_SETUP_BOUNDARY, K_PAD, K_CN_EXPLICIT, K_COMBINE, K_COUNT
};
extern const char *kKernelNames[K_COUNT];

int fail(int code, const char *fmt, ...);

// Return NPB_ECUDA with the failing call's text when a CUDA call fails.
#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(NPB_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)


// Per-kernel CUDA-event timing (only while enabled; graphs are bypassed then).
struct Profiler {
    struct Pending {
        cudaEvent_t a, b;
        int kind;
        int kernels;  // kernel launches inside the region
    };
    bool enabled = false;
    std::mutex mu;
    std::vector<Pending> pending;
    int64_t launches[K_COUNT] = {};
    double total_ms[K_COUNT] = {};
    ~Profiler();
    int begin(cudaStream_t st, cudaEvent_t *a);
    int end(cudaStream_t st, cudaEvent_t a, int kind, int kernels = 1);
    int collect();
};

struct ServeState;  // serving scheduler (serve.cu)
struct BatchPlan;   // npb_energy_batch plan (batch.cu)

inline int64_t tune_key(int prec, int dir, int n) { return ((int64_t)prec << 40) | ((int64_t)dir << 32) | n; }

// Schemes whose directional solves are Crank-Nicolson (legs carry r/2 per half step).
inline bool scheme_cn(int s) {
    return s == NPB_LODCN1 || s == NPB_LODCN2 || s == NPB_AOSCN1 || s == NPB_AOSCN2 || s == NPB_MAOSCN;
}
// The additive schemes of Sec. 3.2-3.3 (additive.cu).
inline bool scheme_additive(int s) { return s >= NPB_AOSIE1 && s <= NPB_MAOSCN; }

}  // namespace npb

struct npb_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    std::atomic<size_t> in_use{0};
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    bool use_graphs = true;
    long long probe_cycles = 0;     // > 0: failure-detection probe before every TMA sweep launch
    npb::Profiler prof;
    std::mutex tune_mu;
    std::map<int64_t, npb::SweepShape> tuned;  // autotuned line-solver shapes
    npb::ServeState *serve = nullptr;
    std::mutex batch_mu;
    std::vector<npb::BatchPlan *> batches;  // npb_energy_batch plans: leg tables and graphs
    // Device memory: released blocks are kept by size and handed to later requests of the same
    // size (grids of one shape come and go in serving and one-shot use); they count against the
    // budget and are returned to the driver when a request would not fit otherwise.
    std::mutex mem_mu;
    std::multimap<size_t, void *> cached;
    std::map<void *, size_t> live;
    size_t cached_bytes = 0;
    int alloc(void **p, size_t bytes);
    void release(void *p, size_t bytes);
    void trim();  // caller holds mem_mu
    // Pinned host slots of 8 doubles for result read-backs, carved from shared slabs.
    std::vector<double *> pinned_free;
    std::vector<void *> pinned_slabs;
    int pinned_slot(double **out);
    void pinned_release(double *p);
};

namespace npb {
using Ctx = ::npb_ctx;

struct GraphCache {
    std::string key;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct Alloc {
    void *p;
    size_t bytes;
};

}  // namespace npb

struct npb_grid {
    npb_ctx *ctx = nullptr;
    npb::GridGeom geo{};
    double eps_in = 1, eps_out = 80, kappa2 = 0;
    int n_atoms = 0;
    double *d_xyz = nullptr, *d_q = nullptr, *d_rad = nullptr;
    uint32_t *d_mask = nullptr;
    uint32_t *d_mask_y = nullptr;  // line-major copies of the node mask for the y and z sweeps
    uint32_t *d_mask_z = nullptr;
    uint32_t *d_half[3] = {nullptr, nullptr, nullptr};
    int32_t *d_line_begin = nullptr, *d_line_count = nullptr, *d_ent_x = nullptr;
    double *d_ent_qt = nullptr;
    int2 *d_ent_xq = nullptr;  // (x | y << 16, FP32 qtilde) of each entry: the FP32 sweeps' fused source
    int64_t *d_ent_off = nullptr;
    int n_ent = 0;
    double *d_bc[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [medium][0 fp64 | 1 fp32 pairs]
    bool bc_valid[2][2] = {{false, false}, {false, false}};
    void *d_u[2][4] = {};              // leg states by [precision][slot]
    int u_prec = -1;                   // precision of the last solve (for npb_potential)
    npb::LegDev *d_legs[2] = {};       // device leg tables by precision
    float2 *d_line_tab = nullptr;      // FP32 legs: multiplier tables [slot][direction][kLineTabMax]
    npb::LegDev h_legs[2][4];
    std::string legs_key[2];
    // additive schemes (additive.cu): per slot the saved U^n, the x part and the y part; the
    // directional solves' legs [direction][slot]; the combine stage's legs; x/y tensor maps
    void *d_aux[2][4][3] = {};
    npb::LegDev h_sub[2][3][4];
    npb::LegDev *d_sub[2] = {};
    npb::AddLeg h_add[2][4];
    npb::AddLeg *d_add[2] = {};
    std::string add_key[2];
    CUtensorMap tma_aux[2][3][4];  // [x | y][variant][slot]
    bool tma_aux_built = false;
    double *d_vac_fft = nullptr;  // phi_0^FFT of Eq. (deltaG2), padded FP64 (fft_vacuum.cu)
    double *d_fac[4][3] = {};     // FP64 legs: Thomas multipliers per slot and direction (sweep_line64.cu)
    bool fac_valid = false;       // they match the current legs and mask
    bool vac_fft_valid = false;
    int vac_fft_kind = -1;         // face flavour it was built from (0 FP64 pairs, 1 FP32 pairs)
    int last_richardson = 1;       // flags of the last npb_energy (for the recovered potential)
    int last_vacuum_lod = 1;
    double *d_result = nullptr;
    double *d_epart = nullptr;   // energy reduction scratch: block partials and a counter
    double *h_result = nullptr;  // pinned
    int32_t *d_err = nullptr;    // set by a device wait that expired
    CUtensorMap tma_u[3][3][4];  // FP32 leg states by [direction][lines-per-tile variant][slot]
    CUtensorMap tma_m[3][3];     // line-major mask by [direction][variant]
    npb::TmaGeom tma_g[3] = {};
    bool tma_ok[3] = {false, false, false};
    bool tma_built = false;
    void *d_scratch = nullptr;   // charge-list scratch (kept for re-running set-up)
    size_t scratch_bytes = 0;
    npb::ChargeScratch sc{};
    std::vector<npb::Alloc> allocs;
    std::vector<npb::GraphCache> graphs;
    std::set<std::string> seen;  // solves run once already (captured as a graph the next time)
};

namespace npb {
using Grid = ::npb_grid;

// Bytes of one padded state of n nodes (x-rows padded to 32 elements).
inline size_t state_bytes(const int n[3], int prec) {
    const size_t pitch = (size_t)(n[0] + 31) / 32 * 32;
    return pitch * n[1] * n[2] * (prec == NPB_FP64 ? 8 : 4);
}

// count elements of T on the device, owned by the grid (freed with it).
template <typename T>
int galloc(Grid *g, T **p, size_t count) {
    void *v = nullptr;
    int rc = g->ctx->alloc(&v, count * sizeof(T));
    if (rc) return rc;
    g->allocs.push_back({v, count * sizeof(T)});
    *p = static_cast<T *>(v);
    return 0;
}

extern const int kLegSlot[4];

int grid_build(Ctx *ctx, const npb_problem *p, cudaStream_t st, Grid **out);
void grid_free(Grid *g);
int grid_setup(Grid *g, cudaStream_t st);
int grid_boundary(Grid *g, int medium, int prec, cudaStream_t st, const double **out);
int grid_half_masks(Grid *g, cudaStream_t st);
int grid_states(Grid *g, int prec, cudaStream_t st);
int grid_prepare(Grid *g, const npb_opts *o, cudaStream_t st);
LegDev make_leg(const Grid *g, int leg, const npb_opts *o);
SweepShape shape_for(Ctx *ctx, int prec, int dir, int n);
SweepShape usable_shape(SweepShape s, int dir, int n, bool tables, int flags, int prec = NPB_FP32_SWEEP);
cudaError_t launch_line64_factors(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, cudaStream_t st);
cudaError_t launch_sweep_line64(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, int flags,
                                cudaStream_t st);
struct LegRef {
    Grid *g;
    int slot;
};
int step_legs(Ctx *ctx, const LegRef *refs, int n, const LegDev *d_table, int prec, int scheme, cudaStream_t st);
int run_step(Grid *g, int prec, int scheme, int slot0, int n_legs, cudaStream_t st);
int enqueue_energy_reduce(Grid *g, int prec, int richardson, cudaStream_t st);
int grid_tma(Grid *g);
cudaError_t launch_dir(Grid *g, int prec, int d, SweepShape shape, int slot0, int n_legs, int flags, cudaStream_t st);
int grid_check_err(Grid *g, cudaStream_t st, int host_copy);
int init_legs(Grid *g, int prec, const int *legs, int n, cudaStream_t st);
int enqueue_energy(Grid *g, const npb_opts *o, cudaStream_t st);
void serve_shutdown(Ctx *ctx);
void batch_forget(Ctx *ctx, Grid *g);  // drop batch plans naming g (all plans when g is null)
int grid_vacuum_fft(Grid *g, int prec, cudaStream_t st);  // phi_0^FFT into g->d_vac_fft
// Additive schemes: the extra states and leg tables for opts (once per change), and one step of
// legs [slot0, slot0 + n) (dense: a padded tau*rho in place of the charges, or null).
int additive_prepare(Grid *g, const npb_opts *o, cudaStream_t st);
int additive_step(Grid *g, int prec, int scheme, int slot0, int n, const void *dense, cudaStream_t st);

}  // namespace npb

