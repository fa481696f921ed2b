// npb_internal.cuh -- device-side types shared by the GB300 LOD-NPB kernels.
//
// Data layout in HBM (one grid, one leg):
//   u     : T[nz][ny][pitch], x fastest; pitch = nx rounded up to 32 elements, so
//           every x-row starts on a 128-byte boundary.  Faces (an index 0 or n-1)
//           hold the Dirichlet data and are never written by a sweep; padding
//           columns x >= nx are zero.
//   mask  : uint32[nz][ny][mwpr], mwpr = pitch/32 rounded up to 4 words (16-byte rows, so
//           the mask can be a TMA tensor); bit x of row (y, z) is 1 on/inside the
//           molecule (Omega_m).  Vacuum legs pass no mask (every node "inside").
//   half  : for NPB_EPS_MIDPOINT, one such bit array per direction d, whose bit at
//           node p says that the half point p + e_d/2 is inside.
//   charges: entries grouped by x-line (z*ny + y): line_begin/line_count index
//           ent_x (node x) and ent_qt (trilinear charge, e_c), and ent_off (element
//           offset of the node in u) for gathers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace npb {

constexpr double kCoulomb = 332.0637;            // kcal A / (mol e^2)
constexpr double kKT = 0.592183;                 // kcal/mol at 298 K (Sec. 2.1)
constexpr double kBjerrum = kCoulomb / kKT;      // e_c^2 / (k_B T) in A
constexpr double kPi = 3.14159265358979323846;

enum Dir { DIR_X = 0, DIR_Y = 1, DIR_Z = 2 };

// uint32 words per x-row of a bit array: pitch/32 rounded up to a multiple of 4.
__host__ __device__ __forceinline__ int mask_words_per_row(int pitch) { return ((pitch >> 5) + 3) & ~3; }

// uint32 words per line of a line-major bit array along a line of n nodes: ceil(n/32)
// rounded up to a multiple of 4 (16-byte lines).  The y-major mask is [nz][nx][words(ny)]
// (bit y of line (x, z)), the z-major mask [ny][nx][words(nz)] (bit z of line (x, y)).
__host__ __device__ __forceinline__ int line_words(int n) { return (((n + 31) >> 5) + 3) & ~3; }

// Everything a sweep / stage kernel needs for one leg.  Lives in device memory as an
// array indexed by blockIdx.z, so one launch can advance several legs of equal size.
struct LegDev {
    void *u;
    const uint32_t *mask;      // node bits, nullptr = all inside
    const uint32_t *half[3];   // half-point bits (midpoint eps mode), nullptr otherwise
    const int32_t *line_begin;
    const int32_t *line_count;
    const int32_t *ent_x;
    const double *ent_qt;
    int32_t nx, ny, nz, pitch;
    double rE[3];              // r*eps for a half point with 0, 1, 2 inside nodes
    double src;                // tau * 4 pi C / h^3: S adds src * qtilde
    double nl_q;               // exp(-kbar^2 tau)
    double nl_omq;             // 1 - nl_q, as -expm1(-kbar^2 tau)
    int32_t nl_on;             // 1: solvent nodes get the nonlinear stage
    int32_t eps_mode;          // 0 harmonic, 1 midpoint
    float rEf[3], nl_qf, nl_omqf, srcf;  // the same constants rounded once to FP32 (FP32 sweeps)
    const int2 *ent_xq;                  // charge entries as (x | y << 16, FP32 qtilde), ent_x's order
    const int64_t *ent_off;              // element offset of each entry's node in the state
    const int32_t *n_ent;                // number of entries (device)
    // FP32 legs, per direction: the Thomas multipliers (m_j, cp_j) of a line whose half points all
    // carry the leg's r*eps outside the molecule (r*eps_in for vacuum legs), j = 1 .. ceil((n-2)/2);
    // the line-per-thread-pair sweeps use them on tiles of constant coefficients (null: no table)
    const float2 *line_tab[3];
    // FP64 legs, per direction: the line-per-thread-pair solver's multipliers m of every node (the
    // state's layout), computed once per leg from eps and r (null: not in use); and the node mask
    // line-major along each direction ([0]: the x rows of `mask`; null with `mask`)
    double *fac[3];
    const uint32_t *lmask[3];
};

// Entries of one direction's multiplier table (n <= 288 nodes per line).
constexpr int kLineTabMax = 144;
// Lines per tile of the line-per-thread-pair sweeps.
constexpr int kLineTX = 32;

// One leg of an additive step (AOS/MAOS, Sec. 3.2-3.3): the states its combine stage reads.
struct AddLeg {
    void *u;                   // the leg's state: on entry the z part, on exit U^{n+1}
    const void *a, *b, *c;     // U^n (AOS: the nonlinear part's start), the x part, the y part
    const uint32_t *mask;      // node bits (the nonlinear part runs at solvent nodes outside)
    int32_t nx, ny, nz, pitch;
    int32_t nl_on;             // AOS: the nonlinear part runs (solvent legs with kbar > 0)
    double q, omq;             // AOS: exp(-4 kbar^2 tau) and 1 - that
};

// The energy reduction: blocks of a launch, threads per block.  Its scratch is kEnergyBlocks
// doubles of block partials followed by a 32-bit counter (zero between launches).
constexpr int kEnergyBlocks = 256, kEnergyThreads = 256;
constexpr int kEnergyScratch = kEnergyBlocks + 1;  // doubles

// Stage flags for the sweep kernels.
enum : int {
    FUSE_PRE_SRC = 1,   // X sweep: add tau Q to the loaded line (LODIE2 stage S)
    FUSE_PRE_NL = 2,    // X sweep: nonlinear stage on the loaded line (LODIE1 stage N)
    FUSE_POST_NL = 4,   // Z sweep: nonlinear stage before the store (LODIE2 stage N)
    FUSE_PRE_CN = 8,    // interior-row sweeps: the explicit half of a Crank-Nicolson sweep on the
                        // loaded lines (after a fused S), the leg's r*eps already halved
};

struct SweepShape {     // one instantiated line-solver shape
    int tx, seg, len;
    int kind;           // 0: one tile per block, direct loads; 1: persistent TMA pipeline (FP32);
                        // 2: interior-row TMA segments (FP32); 3: a line per thread pair (FP32, y/z)
};

// Launchers (defined in sweep_*.cu).  Return cudaError of the launch.
cudaError_t launch_sweep(int prec, int dir, const LegDev *legs_dev, int n_legs, int nx, int ny,
                         int nz, int flags, SweepShape shape, cudaStream_t st);
bool sweep_shape_available(int prec, SweepShape shape);
SweepShape default_sweep_shape(int prec, int dir, int n_dir);
int sweep_shapes(int prec, SweepShape *out, int max);

cudaError_t launch_nonlinear(int prec, const LegDev *legs_dev, int n_legs, int nx, int ny, int nz,
                             cudaStream_t st);
// Charge lists of at least this many entries (bound: 8 per atom) take LODIE2's S as a launch of its
// own before the x sweep; the fused form costs the x sweep's tiles with charges a block barrier
// and a dependent load chain each, which outweighs the extra launch on large molecules only.
constexpr int kSourceApartEntries = 65536;
// LODIE2's S for up to four legs of one grid, everything a thread needs passed by value (no leg
// table to read first): the legs' states and source factors, the grid's charge entries and the
// device count of them.
struct SourceLegs {
    void *u[4];
    float srcf[4];
    double src[4];
    const int64_t *ent_off;
    const int2 *ent_xq;
    const double *ent_qt;
    const int32_t *n_ent;
    int n_slots;  // allocated entry slots (8 per atom), a bound on *n_ent
    int n_legs;
};
cudaError_t launch_source_legs(int prec, const SourceLegs &S, cudaStream_t st);
// LODIE2's S over the charge entries, one thread per entry for all n_legs legs; n_ent_max bounds
// every leg's entry count.
cudaError_t launch_source_entries(int prec, const LegDev *legs_dev, int n_legs, int n_ent_max, cudaStream_t st);
cudaError_t launch_source(int prec, const LegDev *legs_dev, int n_legs, int ny, int nz,
                          cudaStream_t st);
struct GridGeom;
// One explicit Euler step of Eq. (TimeDepNPB) for one leg (*leg in device memory), in -> out.
cudaError_t launch_euler_step(int prec, const LegDev *leg, const void *in, void *out, const GridGeom &g,
                              double tau_kappa2, cudaStream_t st);
// The explicit half step of the Crank-Nicolson sweeps along dir, in place, for n_legs legs.
cudaError_t launch_cn_explicit(int prec, const LegDev *legs_dev, int n_legs, int dir, cudaStream_t st);
// phi_m^LOD + phi_0^LOD - phi_0^FFT as dense FP64 (the recovered potential of Sec. 5.3).
cudaError_t launch_recover(int prec, const GridGeom &g, const void *s_tau, const void *s_half, const void *v_tau,
                           const void *v_half, const double *vac, int richardson, double *out, cudaStream_t st);
// u += scale * src at the interior nodes of a padded state (dense source stage).
cudaError_t launch_add_interior(int prec, const GridGeom &g, const void *src, void *u, double scale,
                                cudaStream_t st);
// The last stage of an additive step for n_legs legs: U^{n+1} = (W + x + y + z)/4 (aos = 1, W the
// nonlinear part from U^n) or (x + y + z)/3 (aos = 0), at interior nodes.
cudaError_t launch_additive_combine(int prec, const AddLeg *legs_dev, int n_legs, int aos, cudaStream_t st);

}  // namespace npb
