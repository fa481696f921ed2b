// additive.cu -- the additive splittings of Sec. 3.2 (AOSIE1/2, AOSCN1/2) and Sec. 3.3 (MAOSIE,
// MAOSCN) on the LOD scheme's kernels.
//
// One step of a leg U, with c = 4 (AOS) or 3 (MAOS):
//   MAOS only  the nonlinear stage on U in place (alpha w_t = -kbar^2 sinh w, Eq. MAOS1_1);
//   copies     AOS: U -> A (U^n, kept for the nonlinear part), U -> B, U -> C; MAOS: U -> B, U -> C;
//   x, y, z    B, C and U itself are the x, y and z parts: each gets [the explicit half of a
//              Crank-Nicolson solve with c r/2,] its share of the source, then the line solves
//              with c r (CN: c r/2) -- the sweep kernels of the LOD scheme on legs whose
//              constants carry the factor c (the directional legs);
//   combine    U = (W(A) + B + C + U)/4, W the exact flow of alpha w_t = -4 kbar^2 sinh w over tau
//              (Eqs. AOS1_5, AOS2_5), or U = (B + C + U)/3 (Eq. MAOS1_5).
// The source shares: AOS1 4 tau Q on x alone, AOS2 4/3 tau Q on each direction, MAOS tau Q on each.
// The three directional parts are independent of one another (the paper's point about parallel
// hardware); on one GPU each sweep already fills the machine, so they run one after another on
// the solver's stream and the graph of a solve holds them as a chain.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "runtime.h"
#include "sweep_tma.cuh"

namespace npb {

static void additive_shares(int scheme, double share[3]) {
    share[0] = share[1] = share[2] = 1.0;  // MAOS
    if (scheme == NPB_AOSIE1 || scheme == NPB_AOSCN1) share[0] = 4.0, share[1] = share[2] = 0.0;
    if (scheme == NPB_AOSIE2 || scheme == NPB_AOSCN2) share[0] = share[1] = share[2] = 4.0 / 3.0;
}

static bool scheme_aos(int s) { return s >= NPB_AOSIE1 && s <= NPB_AOSCN2; }

// The extra states (three per slot), their x/y tensor maps (FP32), and the directional and
// combine leg tables; grid_prepare has made the LOD legs for the same opts.
int additive_prepare(Grid *g, const npb_opts *o, cudaStream_t st) {
    const int prec = o->precision;
    const int n3[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    const size_t bytes = state_bytes(n3, prec);
    int rc;
    if (!g->d_aux[prec][0][0]) {
        for (int s = 0; s < 4; ++s)
            for (int k = 0; k < 3; ++k) {
                unsigned char *p = nullptr;
                if ((rc = galloc(g, &p, bytes))) return rc;
                CU(cudaMemsetAsync(p, 0, bytes, st));  // padding stays zero (copies keep it so)
                g->d_aux[prec][s][k] = p;
            }
        if ((rc = galloc(g, &g->d_sub[prec], 12))) return rc;
        if ((rc = galloc(g, &g->d_add[prec], 4))) return rc;
        g->add_key[prec] = "";
    }
    if (prec == NPB_FP32_SWEEP && !g->tma_aux_built) {
        g->tma_aux_built = true;
        for (int d = 0; d < 2; ++d) {  // the x parts (slot's B) in the x view, the y parts (C) in the y view
            if (!g->tma_ok[d]) continue;
            bool ok = true;
            for (int v = 0; v < tma_variant_count(d) && ok; ++v)
                for (int s = 0; s < 4 && ok; ++s)
                    ok = tma_encode_state(&g->tma_aux[d][v][s], g->d_aux[prec][s][1 + d], d, g->tma_g[d], n3[0],
                                          n3[1], n3[2], g->geo.pitch, tma_variant_tx(d, v));
            if (!ok) return fail(NPB_ECUDA, "tensor maps of the additive scheme's states could not be encoded");
        }
    }
    char key[256];
    snprintf(key, sizeof key, "%s/%d", g->legs_key[prec].c_str(), o->scheme);
    if (g->add_key[prec] == key) return 0;
    const bool aos = scheme_aos(o->scheme);
    const double c = aos ? 4.0 : 3.0;
    double share[3];
    additive_shares(o->scheme, share);
    for (int leg = 0; leg < 4; ++leg) {
        const int s = kLegSlot[leg];
        const LegDev &L = g->h_legs[prec][s];
        for (int d = 0; d < 3; ++d) {
            LegDev D = L;
            D.u = d == 2 ? L.u : g->d_aux[prec][s][1 + d];
            for (int i = 0; i < 3; ++i) {
                D.rE[i] = c * L.rE[i];
                D.rEf[i] = (float)D.rE[i];
            }
            D.src = share[d] * L.src;
            D.srcf = (float)D.src;
            D.nl_on = 0;
            for (int i = 0; i < 3; ++i) {  // tables and multipliers of the unscaled r*eps
                D.line_tab[i] = nullptr;
                D.fac[i] = nullptr;
            }
            g->h_sub[prec][d][s] = D;
        }
        const bool half = leg == NPB_LEG_SOLVENT_HALF || leg == NPB_LEG_VACUUM_HALF;
        const double tau = (half ? 0.5 : 1.0) * o->dt / o->alpha;
        AddLeg A{};
        A.u = L.u;
        A.a = g->d_aux[prec][s][0];
        A.b = g->d_aux[prec][s][1];
        A.c = g->d_aux[prec][s][2];
        A.mask = L.mask;
        A.nx = L.nx;
        A.ny = L.ny;
        A.nz = L.nz;
        A.pitch = L.pitch;
        A.nl_on = L.nl_on;
        A.q = std::exp(-4.0 * g->kappa2 * tau);
        A.omq = -std::expm1(-4.0 * g->kappa2 * tau);
        g->h_add[prec][s] = A;
    }
    LegDev flat[12];
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 4; ++s) flat[d * 4 + s] = g->h_sub[prec][d][s];
    CU(cudaMemcpyAsync(g->d_sub[prec], flat, sizeof flat, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(g->d_add[prec], g->h_add[prec], sizeof(AddLeg) * 4, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
    g->add_key[prec] = key;
    return 0;
}

// The line solves of direction d on the directional legs of slots [slot0, slot0 + n): the FP32
// TMA kernels where the grid allows them (as for the LOD legs), else the one-tile-per-block kernel.
static cudaError_t directional_sweep(Grid *g, int prec, int d, int slot0, int n, cudaStream_t st) {
    const int n3[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    // the directional legs carry scaled r*eps and no multiplier tables
    SweepShape shape = usable_shape(shape_for(g->ctx, prec, d, n3[d]), d, n3[d], false, 0, prec);
    const int v = tma_variant(d, shape.tx);
    if (shape.kind >= 1 && prec == NPB_FP32_SWEEP && g->tma_ok[d] && v >= 0 && n <= kTmaMaxLegs &&
        g->h_sub[prec][d][slot0].eps_mode == 0) {
        TmaLaunch P;
        memset(&P, 0, sizeof P);
        for (int i = 0; i < n; ++i) {
            const int s = slot0 + i;
            P.umap[i] = d == 2 ? g->tma_u[d][v][s] : g->tma_aux[d][v][s];
            P.mmap[i] = g->tma_m[d][v];
            P.legs[i] = g->h_sub[prec][d][s];
        }
        P.n_legs = n;
        P.err = g->d_err;
        if (shape.kind == 2) return launch_sweep_inner(d, P, g->tma_g[d], 0, shape, g->ctx->sm_count, st);
        return launch_sweep_tma(d, P, g->tma_g[d], 0, shape, g->ctx->sm_count, st);
    }
    if (shape.kind >= 1) shape = default_sweep_shape(prec, d, n3[d]);
    return launch_sweep(prec, d, g->d_sub[prec] + d * 4 + slot0, n, n3[0], n3[1], n3[2], 0, shape, st);
}

int additive_step(Grid *g, int prec, int scheme, int slot0, int n, const void *dense, cudaStream_t st) {
    if (n <= 0) return 0;
    Profiler &pr = g->ctx->prof;
    const bool aos = scheme_aos(scheme), cn = scheme_cn(scheme);
    double share[3];
    additive_shares(scheme, share);
    const int n3[3] = {g->geo.nx, g->geo.ny, g->geo.nz};
    const size_t bytes = state_bytes(n3, prec);
    cudaEvent_t ev{};
    int rc;
    if (!aos) {  // MAOS: the nonlinear stage first; the directional parts start from its result
        if ((rc = pr.begin(st, &ev))) return rc;
        CU(launch_nonlinear(prec, g->d_legs[prec] + slot0, n, n3[0], n3[1], n3[2], st));
        if ((rc = pr.end(st, ev, K_NONLINEAR))) return rc;
    }
    for (int i = 0; i < n; ++i) {
        const int s = slot0 + i;
        const void *u = g->d_u[prec][s];
        for (int k = aos ? 0 : 1; k < 3; ++k)
            CU(cudaMemcpyAsync(g->d_aux[prec][s][k], u, bytes, cudaMemcpyDeviceToDevice, st));
    }
    for (int d = 0; d < 3; ++d) {
        const LegDev *tab = g->d_sub[prec] + d * 4 + slot0;
        if (cn) {
            if ((rc = pr.begin(st, &ev))) return rc;
            CU(launch_cn_explicit(prec, tab, n, d, st));
            if ((rc = pr.end(st, ev, K_CN_EXPLICIT))) return rc;
        }
        if (share[d] != 0.0) {
            if ((rc = pr.begin(st, &ev))) return rc;
            if (dense) {
                for (int i = 0; i < n; ++i)
                    CU(launch_add_interior(prec, g->geo, dense, g->h_sub[prec][d][slot0 + i].u, share[d], st));
            } else {
                CU(launch_source(prec, tab, n, n3[1], n3[2], st));
            }
            if ((rc = pr.end(st, ev, K_SOURCE))) return rc;
        }
        if ((rc = pr.begin(st, &ev))) return rc;
        CU(directional_sweep(g, prec, d, slot0, n, st));
        if ((rc = pr.end(st, ev, K_SWEEP_X + d))) return rc;
    }
    if ((rc = pr.begin(st, &ev))) return rc;
    CU(launch_additive_combine(prec, g->d_add[prec] + slot0, n, aos ? 1 : 0, st));
    if ((rc = pr.end(st, ev, K_COMBINE))) return rc;
    return 0;
}

}  // namespace npb
