/*
 * npb.h -- C ABI of the GB300 LOD solver for the time-dependent nonlinear
 * Poisson-Boltzmann (NPB) equation (Wilson & Zhao, arXiv 1410.2788).
 *
 * The solver integrates the pseudo-time NPB equation of Sec. 2.2,
 *     alpha u_t = div(eps grad u) - kbar^2 sinh(u) + rho_m,            Eq. (TimeDepNPB)
 * with the locally-one-dimensional implicit-Euler splitting LODIE2 of Sec. 3.1:
 *     S:  u += tau Q                                                   Eq. (LODIE1_5)
 *     X, Y, Z:  (1 - tau delta_d^2) v = w, one tridiagonal system per grid line,
 *               eps taken at half points                              Eqs. (LODIE1_2)-(LODIE1_4),
 *                                                                      (SpatialOperators)
 *     N:  analytic flow of alpha w_t = -kbar^2 sinh w                  Eq. (ana3)
 * with tau = dt/alpha, and computes the electrostatic solvation energy with
 * the Richardson extrapolation of Eq. (rich) and the LOD vacuum recovery of
 * Eq. (deltaG3) (Sec. 5.3, "LODIE2 RE+V").
 *
 * Units follow Sec. 2.1: lengths in Angstrom, charges in e_c, the potential u
 * dimensionless (e_c phi / k_B T at 298 K); energies in kcal/mol.
 *
 * Conventions (every call):
 *   - Return codes: NPB_OK (0), NPB_PENDING (1), or a negative NPB_E* code.  On a
 *     negative code npb_last_error() gives a message (thread-local) and no output
 *     argument has been written.
 *   - Ownership: every input pointer is read during the call only; the library
 *     copies what it keeps.  Handles are freed by their destroy call.  Host
 *     buffers are plain CPU memory (pinned or pageable).
 *   - Threads: npb_submit / npb_poll are thread-safe.  All other calls on one
 *     grid must not run concurrently with each other.
 *   - Device: the library allocates its own device memory on the context's
 *     device and launches on the context's stream; there is no CPU fallback.
 */
#ifndef NPB_H
#define NPB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------- */
#define NPB_OK 0
#define NPB_PENDING 1       /* npb_poll: the request has not finished yet            */
#define NPB_EINVAL (-1)     /* invalid argument (sizes, signs, atoms off the grid)    */
#define NPB_ENOMEM (-2)     /* over the context's HBM budget or cudaMalloc failed     */
#define NPB_ECUDA (-3)      /* a CUDA call failed                                     */
#define NPB_ETIMEOUT (-4)   /* a bounded wait expired (poll timeout, device wait)      */
#define NPB_ENOTFOUND (-5)  /* unknown ticket                                         */
#define NPB_ESHUTDOWN (-6)  /* the context is shutting down                           */

/* ---- enums ------------------------------------------------------------------------- */
#define NPB_SOLVENT 0       /* eps_out outside the molecule, kbar^2 in solvent          */
#define NPB_VACUUM 1        /* eps_in everywhere, kbar = 0 (the vacuum leg of Eq. deltaG3) */

#define NPB_LODIE2 2        /* S, X, Y, Z, N  (Sec. 3.1; the paper's chosen scheme)     */
#define NPB_LODIE1 1        /* N, X, Y, Z, S                                            */
#define NPB_LODCN1 3        /* LODIE1's order with the Crank-Nicolson sweeps (Eqs. LODCN1_2-4) */
#define NPB_LODCN2 4        /* LODIE2's order with the Crank-Nicolson sweeps            */
/* Additive splittings (Sec. 3.2, 3.3): the parts advance side by side from one state and are
 * averaged.  AOS: the nonlinear part (4 kbar^2, integrated exactly) and one line solve per
 * direction from U^n with 4 tau (Crank-Nicolson: 2 tau on each side), mean of the four; the
 * source goes to x alone (AOS*1) or a third to each direction (AOS*2).  MAOS: the nonlinear stage
 * first, then three line solves from its result with 3 tau (CN: 3 tau/2 each side) and tau Q
 * each, mean of the three.  Each leg uses three extra device states, allocated on first use
 * (not counted by npb_grid_footprint).  npb_energy, npb_lod_solve, npb_lod_run and npb_apply
 * (NPB_OP_STEP) run them; npb_energy_batch and npb_submit take the LOD schemes only. */
#define NPB_AOSIE1 5        /* Eqs. AOSIE1_1-5                                          */
#define NPB_AOSIE2 6        /* Eqs. AOSIE2_2-4 in place of AOSIE1_2-4                   */
#define NPB_AOSCN1 7        /* Eqs. AOSCN1_2-4                                          */
#define NPB_AOSCN2 8        /* Eqs. AOSCN2_2-4                                          */
#define NPB_MAOSIE 9        /* Eqs. MAOS1_1-5, implicit Euler                          */
#define NPB_MAOSCN 10       /* Eqs. MAOS1_1-5, Crank-Nicolson                          */

#define NPB_FP64 0          /* every stage in FP64                                      */
#define NPB_FP32_SWEEP 1    /* potential stored and swept in FP32; energy in FP64       */

#define NPB_EPS_HARMONIC 0  /* eps at a half point = harmonic mean of its two nodes     */
#define NPB_EPS_MIDPOINT 1  /* eps at a half point decided by the half point's location */

/* Legs of one RE+V solve, in the order npb_potential() and npb_apply() name them. */
#define NPB_LEG_SOLVENT_TAU 0
#define NPB_LEG_SOLVENT_HALF 1
#define NPB_LEG_VACUUM_TAU 2
#define NPB_LEG_VACUUM_HALF 3
/* npb_potential() only: phi_0^FFT of Eq. (deltaG2), the vacuum potential by the direct (sine
 * transform) Poisson solve; and the recovered potential phi_m^LOD + phi_0^LOD - phi_0^FFT of
 * Sec. 5.3 (each LOD potential Richardson-combined when the last solve used Richardson). */
#define NPB_LEG_VACUUM_FFT 4
#define NPB_LEG_RECOVERED 5

/* Single stages for npb_apply() (row-level checks of one LOD stage). */
#define NPB_OP_SOURCE 0     /* u += tau Q at interior charge nodes        Eq. (LODIE1_5) */
#define NPB_OP_SWEEP_X 1    /* x line solves                               Eq. (LODIE1_2) */
#define NPB_OP_SWEEP_Y 2    /* y line solves                               Eq. (LODIE1_3) */
#define NPB_OP_SWEEP_Z 3    /* z line solves                               Eq. (LODIE1_4) */
#define NPB_OP_NONLINEAR 4  /* analytic sinh stage at solvent nodes        Eq. (ana3)     */
#define NPB_OP_STEP 5       /* one full step of opts->scheme                             */

/* What npb_grid_export() copies out (dense nz*ny*nx arrays, x fastest). */
#define NPB_EXPORT_MASK 0        /* uint8: 1 on/inside the molecular surface            */
#define NPB_EXPORT_QTILDE 1      /* double: trilinear node charges, e_c                 */
#define NPB_EXPORT_U0_SOLVENT 2  /* double: Eq. (BoundaryCond) faces, zero interior     */
#define NPB_EXPORT_U0_VACUUM 3   /* double: Coulomb faces with eps_in, zero interior    */

/* ---- types ------------------------------------------------------------------------- */
typedef struct npb_ctx npb_ctx;    /* device, stream, HBM budget, serving scheduler   */
typedef struct npb_grid npb_grid;  /* one molecule's device arrays and leg states      */

/* The problem statement of Sec. 2.1 on the uniform grid of Sec. 3:
 * atoms r_j (xyz, 3*n_atoms doubles, A), partial charges q_j (e_c), radii (A; the
 * molecule Omega_m is the union of the closed balls, standing in for an MSMS
 * surface), eps_in = eps_m and eps_out = eps_s, kappa2 = kbar^2 in A^-2 (solvent
 * only), grid spacing h (A) and node counts n = (nx, ny, nz), each >= 3.
 * Node (i, j, k) sits at origin + h (i, j, k).  Every atom's 8-node charge stencil
 * must lie in the interior (indices 1 .. n-2), else NPB_EINVAL. */
typedef struct {
    int32_t n_atoms;
    const double *xyz;
    const double *q;
    const double *radius;
    double eps_in, eps_out, kappa2, h;
    int32_t n[3];
    double origin[3];
} npb_problem;

/* Pseudo-time options: tau = dt/alpha; the Richardson leg uses dt/2 and 2 n_steps
 * (Sec. 5.3).  richardson and vacuum_recovery are 0/1 flags.  vacuum_recovery = 1: the
 * vacuum potential is the LOD vacuum legs' (Eq. deltaG3, the paper's RE+V); 0: it is the
 * direct Poisson solution phi_0^FFT (Eq. deltaG2), and only the solvent legs run
 * (npb_energy only; npb_energy_batch and npb_submit need 1). */
typedef struct {
    double dt, alpha;
    int32_t n_steps;
    int32_t scheme;           /* NPB_LODIE2 (default), NPB_LODIE1, NPB_LODCN1/2, or an
                                 additive scheme NPB_AOSIE1 ... NPB_MAOSCN               */
    int32_t richardson;       /* 1: RE of Eq. (rich)                                   */
    int32_t vacuum_recovery;  /* 1: LOD vacuum legs of Eq. (deltaG3); 0: Eq. (deltaG2) */
    int32_t precision;        /* NPB_FP64 or NPB_FP32_SWEEP                            */
    int32_t eps_mode;         /* NPB_EPS_HARMONIC (default) or NPB_EPS_MIDPOINT        */
} npb_opts;

typedef struct {
    double dG_kcal_mol;   /* solvation energy, Eq. (deltaG3)                          */
    double wall_ms;       /* submit -> completion                                     */
    double queue_ms;      /* submit -> admission                                      */
    int64_t point_steps;  /* interior nodes x steps, summed over legs                 */
    int32_t status;       /* NPB_OK or a negative code                                */
    int32_t n[3];         /* grid of the request                                      */
} npb_result;

/* ---- context ------------------------------------------------------------------------ */
/* Create a context on CUDA device `device` whose solves may hold at most
 * hbm_budget_bytes of device memory (0: 90% of the free memory).  *out owns it. */
int npb_ctx_create(int device, size_t hbm_budget_bytes, npb_ctx **out);
void npb_ctx_destroy(npb_ctx *ctx);
/* Launch on `stream` (a cudaStream_t) from now on; NULL returns to the context's own
 * non-blocking stream.  Whole solves are replayed as CUDA graphs captured on this stream. */
int npb_ctx_set_stream(npb_ctx *ctx, void *stream);
/* 1: bracket every kernel launch with CUDA events and keep per-kernel totals. */
int npb_ctx_profile(npb_ctx *ctx, int32_t enable);
/* Per-kernel totals since profiling was enabled: for kernel class i < max_kernels,
 * names[i] (static strings), launches[i] (kernel launches: a set-up class counts each kernel
 * of its stage) and total device ms[i].  Returns the number of classes written.  Synchronises
 * the stream. */
int npb_ctx_kernel_stats(npb_ctx *ctx, int32_t max_kernels, const char **names,
                         int64_t *launches, double *ms);
/* Failure-detection probe, to test the error path of the bounded device waits without a GPU
 * fault.  Every wait of the TMA-pipelined sweeps on their tile copies gives up after about 4e9 SM
 * cycles (two seconds), sets the grid's error flag and returns; the call reports NPB_ETIMEOUT once
 * the stream has synchronised, and the context stays usable.  While `cycles` > 0, a probe kernel
 * runs before every TMA sweep launch: each of its blocks waits, with the same bounded-wait helper
 * and a bound of `cycles`, on a barrier that nothing arrives at (no copy is in flight), so the wait
 * expires and sets the same flag.  0 turns the probe off.  Solves run as direct launches (no graph)
 * while it is on. */
int npb_ctx_probe_wait_expiry(npb_ctx *ctx, int64_t cycles);
/* Bytes of device memory the context's grids hold right now. */
int npb_ctx_memory(npb_ctx *ctx, size_t *in_use, size_t *budget);

/* ---- one molecule --------------------------------------------------------------------- */
/* Copy the problem to the device and run the set-up kernels on the context stream:
 * the vdW-union node mask (Sec. 3.1), the trilinear charges Q grouped by x-line
 * (Sec. 3.1, Eq. RhoEq), and the Dirichlet face data for solvent (Eq. BoundaryCond)
 * and vacuum (the same formula with eps_in and kbar = 0).  NPB_ENOMEM when the
 * grid would push the context over its budget. */
int npb_grid_create(npb_ctx *ctx, const npb_problem *problem, npb_grid **out);
void npb_grid_destroy(npb_grid *grid);
/* Re-run every set-up kernel (mask, charge list, face data in use) from the atoms the grid
 * already holds on the device; enqueued on the context stream, no host copy, no allocation.
 * The results are identical to those of npb_grid_create. */
int npb_grid_refresh(npb_grid *grid);
/* Device bytes the grid needs for one RE+V solve at `precision`. */
size_t npb_grid_footprint(const npb_problem *problem, int32_t precision);

/* One pseudo-time leg from the trivial initial solution u = 0 (Sec. 2.2):
 * tau = dt_scale * dt / alpha, n_steps / dt_scale steps.  dt_scale is 1 or 0.5.
 * The result stays on the device as leg (medium, dt_scale) for npb_potential(). */
int npb_lod_solve(npb_grid *grid, const npb_opts *opts, int32_t medium, double dt_scale);

/* The RE+V solvation energy in kcal/mol: the solvent and vacuum legs at dt and (with
 * richardson) dt/2 run batched on the device, then the FP64 charge-weighted sum
 *   dG = 1/2 * 0.592183 * sum_p Q_p [(2 u_s^{dt/2} - u_s^{dt}) - (2 u_v^{dt/2} - u_v^{dt})]_p
 * of Eqs. (rich) and (deltaG3).  Blocks until the value is on the host. */
int npb_energy(npb_grid *grid, const npb_opts *opts, double *dG_kcal_mol);

/* npb_energy for n_grids molecules at once (the batched workload of many uneven grids): every
 * grid runs the same opts; grids of equal size share one persistent sweep launch per direction
 * at each LOD step (Sec. 3.1) over all their legs, and the whole batch -- leg starts, steps and
 * the FP64 energies of Eqs. (rich) and (deltaG3) -- runs as one CUDA graph, kept for repeat
 * calls with the same grids, opts and solver shapes.  dG_kcal_mol[i] receives grid i's energy;
 * each equals npb_energy(grids[i], opts) bit for bit.  The grids must belong to one context and
 * appear once each; the call blocks until every value is on the host.  NPB_ETIMEOUT when a
 * bounded device wait expired (all values are then unreliable). */
int npb_energy_batch(npb_grid *const *grids, int32_t n_grids, const npb_opts *opts, double *dG_kcal_mol);

/* Copy leg `leg` (NPB_LEG_*) of the last solve -- or phi_0^FFT (NPB_LEG_VACUUM_FFT), or the
 * recovered potential (NPB_LEG_RECOVERED, after a solve with vacuum_recovery = 1) -- to host_out
 * as dense FP64 values of u
 * (dimensionless), nz*ny*nx of them, x fastest.  n_elems must equal nx*ny*nz. */
int npb_potential(npb_grid *grid, int32_t leg, double *host_out, size_t n_elems);

/* n_steps steps of opts->scheme (Sec. 3.1-3.3) of leg `leg` from a caller-given state, the
 * pseudo-time run of Eq. (TimeDepNPB) with that leg's medium, eps at half points (opts->eps_mode)
 * and tau = dt/alpha (halved for the *_HALF legs).  u_inout: nz*ny*nx FP64 values of u, x
 * fastest; its interior is the initial value and its faces the Dirichlet data, which no stage
 * changes; the final state is copied back into it.  source (same layout, may be NULL) is a dense
 * source density rho: stage S then adds tau*rho at the interior nodes in place of the molecule's
 * point charges (an additive scheme: each direction's share of it), the manufactured-solution
 * benchmark of Sec. 4.1 (Eqs. NPB_analytical_1/2);
 * with NULL the step is the usual one with the charges.  n_elems must equal nx*ny*nz. */
int npb_lod_run(npb_grid *grid, const npb_opts *opts, int32_t leg, int32_t n_steps, double *u_inout,
                const double *source, size_t n_elems);

/* n_steps explicit Euler steps of Eq. (TimeDepNPB) for leg `leg` from a caller-given state
 * (layout and faces as npb_lod_run; tau = dt/alpha, halved for the *_HALF legs; the molecule's
 * charges as the source): u += tau (div(eps grad u) - kbar^2 sinh u + rho) with the same
 * half-point eps as the LOD sweeps.  The conditionally stable reference the paper compares its
 * splitting schemes with (Sec. 5.2); tau must respect h^2/(6 eps_max) for stability. */
int npb_euler_run(npb_grid *grid, const npb_opts *opts, int32_t leg, int32_t n_steps, double *u_inout,
                  size_t n_elems);

/* Row-level access to single LOD stages: load the dense FP64 field u_inout (nz*ny*nx)
 * into leg `leg`'s state (rounded to opts->precision), apply stage `op` (NPB_OP_*)
 * with that leg's medium and tau = dt/alpha (halved for the *_HALF legs), and copy the
 * result back.  Faces are never changed by any stage. */
int npb_apply(npb_grid *grid, const npb_opts *opts, int32_t leg, int32_t op, double *u_inout,
              size_t n_elems);

/* Copy set-up arrays out (NPB_EXPORT_*); host_out must hold n_elems elements of the
 * stated type and n_elems must equal nx*ny*nz. */
int npb_grid_export(npb_grid *grid, int32_t what, void *host_out, size_t n_elems);

/* ---- charge list without allocation --------------------------------------------------- */
/* The paper has no counterpart: this is a service for callers that cannot allocate device
 * memory when they need a charge list -- applications whose own memory pool owns the device and
 * forbids library allocations, and latency-critical paths that cannot pay for the implicit
 * device synchronisation of cudaMalloc/cudaFree.
 *
 * It builds the same x-line-grouped trilinear charge list as npb_grid_create, on the calling
 * thread's current device and on `stream` (a cudaStream_t; NULL = the legacy default
 * stream), and calls no cudaMalloc, cudaFree or allocating routine.  Its temporaries live in
 * one fixed device array compiled into the library (about 9.3 MB on every GPU that loads it,
 * kept until the process exits), which bounds the problem: n_atoms <= NPB_STATIC_MAX_ATOMS
 * and ny*nz <= NPB_STATIC_MAX_LINES; larger inputs return NPB_EINVAL.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current.
 * Every call reuses the same array and clears what it accumulates into: calls that overlap on
 * the GPU race, so serialise them.
 *
 * Inputs (host memory, read during the call): xyz (3*n_atoms doubles), q (n_atoms), grid n, h,
 * origin as in npb_problem; every atom's 8-node stencil must lie in the interior.  Outputs
 * (device memory the caller owns): d_line_begin and d_line_count (ny*nz each; entries of x-line
 * z*ny + y), d_ent_x, d_ent_qt and d_ent_off (room for 8*n_atoms each: node x index, charge in
 * e_c, element offset (z*ny + y)*pitch + x with pitch = nx rounded up to 32), and d_n_entries
 * (one int32: the number of entries).  The work is enqueued; synchronise `stream` before
 * reading the outputs.  NPB_ECUDA when a copy, clear or launch is refused. */
#define NPB_STATIC_MAX_ATOMS 20000
#define NPB_STATIC_MAX_LINES (288 * 288)
int npb_charge_list_static(const double *xyz, const double *q, int32_t n_atoms, const int32_t n[3], double h,
                           const double origin[3], int32_t *d_line_begin, int32_t *d_line_count,
                           int32_t *d_ent_x, double *d_ent_qt, int64_t *d_ent_off, int32_t *d_n_entries,
                           void *stream);

/* ---- serving: continuous batching ---------------------------------------------------- */
/* Queue one RE+V energy request; the library copies the problem.  A scheduler thread
 * admits queued requests while their device footprint fits the budget, runs the legs
 * of every admitted request in shared batched launches, and retires requests as they
 * finish, so requests that arrive while others run join the running batch. */
int npb_submit(npb_ctx *ctx, const npb_problem *problem, const npb_opts *opts,
               uint64_t *ticket);
/* Wait up to timeout_ms (0: do not wait, <0: wait forever) for `ticket`.  NPB_OK with
 * *out filled (the ticket is then consumed), NPB_PENDING, or a negative code. */
int npb_poll(npb_ctx *ctx, uint64_t ticket, int32_t timeout_ms, npb_result *out);

/* ---- line-solver autotuning ------------------------------------------------------------ */
/* Each line of a sweep (the implicit-Euler tridiagonal solve of one LOD direction, Eqs. LODIE1_2-4)
 * is solved by one of four kernel families, the solver kind:
 *   NPB_KIND_TILE      0: one tile per block, FP64 or FP32: SEG threads per line holding L
 *                         consecutive rows each (a segmented Thomas elimination), the segment ends
 *                         reduced by parallel cyclic reduction; TX lines per block.  SEG = 2 is
 *                         close to Thomas per line, many short segments close to pure PCR;
 *   NPB_KIND_TMA       1: FP32 only, persistent blocks fed by bulk tensor copies, the same
 *                         segmentation as kind 0;
 *   NPB_KIND_TMA_INNER 2: FP32 only, persistent TMA blocks, SEG segments of L rows over the n-2
 *                         interior rows, segment ends reduced by parallel cyclic reduction in
 *                         shared memory (x: 8 lines per tile; y/z: 16 or 8);
 *   NPB_KIND_LINE      3: FP32 only, y and z: the Thomas algorithm of the paper (Sec. 3.1), one
 *                         line per pair of threads (each eliminates from one end of the line, the
 *                         two meet in the middle), 32 lines per tile, TMA-pipelined; tx = 32,
 *                         seg = 2, len = pipeline stages (1 or 2).  Tiles of constant coefficients
 *                         take the leg's precomputed multipliers.  The FP32 default for y and z.
 * npb_autotune times every instantiated (kind, TX, SEG, L) that covers the grid's lines, on
 * all four legs of `grid` at opts->precision, `reps` launches each, and keeps the fastest
 * per (precision, direction, line length) in the context.  report (may be NULL) receives a
 * JSON list of the timings, truncated to report_len bytes.  The legs' states are
 * overwritten.  Kinds 1-3 fall back to kind 0's default shape where the grid's geometry does
 * not suit bulk tensor copies or eps at half points is the midpoint reading; kind 3 falls back
 * to kind 2 for the Crank-Nicolson and additive schemes. */
enum { NPB_KIND_TILE = 0, NPB_KIND_TMA = 1, NPB_KIND_TMA_INNER = 2, NPB_KIND_LINE = 3 };
int npb_autotune(npb_grid *grid, const npb_opts *opts, int32_t reps, char *report, size_t report_len);
/* Pin / read the shape used for lines of n nodes along dir (0 = x, 1 = y, 2 = z).
 * npb_tune_set fails with NPB_EINVAL when (kind, tx, seg, len) is not instantiated for that
 * precision and direction or covers fewer rows than the kind needs (n, or n - 2 for
 * kind 2; kind 3 covers any line).  npb_tune_get returns the pinned shape, else the default for n. */
int npb_tune_set(npb_ctx *ctx, int32_t precision, int32_t dir, int32_t n, int32_t kind, int32_t tx,
                 int32_t seg, int32_t len);
int npb_tune_get(npb_ctx *ctx, int32_t precision, int32_t dir, int32_t n, int32_t *kind, int32_t *tx,
                 int32_t *seg, int32_t *len);
/* The tuning cache: npb_tune_save writes every shape pinned in the context (by npb_autotune or
 * npb_tune_set) to the file `path` as a JSON list of {"precision", "dir", "n", "kind", "tx",
 * "seg", "len"} entries, one per (precision, direction, line length).  npb_tune_load reads such a
 * file and pins each entry that this build instantiates (others are skipped); *n_loaded (may be
 * NULL) receives the number pinned.  NPB_EINVAL when the file cannot be written, read or parsed. */
int npb_tune_save(npb_ctx *ctx, const char *path);
int npb_tune_load(npb_ctx *ctx, const char *path, int32_t *n_loaded);

/* Average device time (ms) of one sweep launch as npb_energy issues it (measurement aid, not a
 * stage of the method): direction dir (0 = x, 1 = y, 2 = z) over the legs of slots [0, n_legs)
 * -- n_legs = 4 is the launch of LOD steps 1 .. n (all four legs of Eq. deltaG3's RE+V solve),
 * n_legs = 2 the launch of steps n+1 .. 2n (the dt/2 legs) -- with the solve's shape for that
 * direction and its fused stages (LODIE2: S in the x sweep, N in the z sweep, except that S is a
 * launch of its own, left out of the timing, where a solve gives it one: FP32 grids of 8,192 atoms
 * or more, and the kind-1 sweeps; LODIE1: N in the x sweep).  reps launches are captured in one CUDA graph on the context stream (which must not be
 * the legacy default stream), replayed once untimed, then `rounds` times between two CUDA events;
 * *ms_per_launch = elapsed / (reps * rounds).  The legs' states are overwritten.  Implicit-Euler
 * LOD schemes only (NPB_EINVAL otherwise). */
int npb_sweep_time(npb_grid *grid, const npb_opts *opts, int32_t dir, int32_t n_legs, int32_t reps, int32_t rounds,
                   double *ms_per_launch);

/* Rates of the device's FP64 units (measurement aid for the plain FP64 path's roofline, not a stage
 * of the method): fused multiply-adds per second and IEEE divisions per second, each from a
 * kernel of eight independent dependency chains per thread over all SMs, timed with CUDA events on
 * the context stream after one untimed pass.  Uses 64 bytes of the context's device memory. */
int npb_measure_fp64(npb_ctx *ctx, double *dfma_per_s, double *ddiv_per_s);

/* ---- errors --------------------------------------------------------------------------- */
const char *npb_last_error(void);
const char *npb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NPB_H */
