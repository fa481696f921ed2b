// tma.h -- host interface of the TMA-pipelined FP32 sweeps (sweep_tma_f32.cu).
#pragma once
#include <cuda.h>

#include "npb_internal.cuh"

namespace npb {

struct TmaLaunch;
struct LegTma;

struct TmaGeom {
    bool ok;
    int rows, nload;      // y/z: rows per box, boxes per tile
    int sx, xc, nchunk;   // x: shared row stride = xc * nchunk
    int mwpr;             // words per line of the line-major mask of this direction
};

TmaGeom tma_geometry(int dir, int nx, int ny, int nz, int pitch);
bool tma_encode_state(CUtensorMap *m, void *u, int dir, const TmaGeom &g, int nx, int ny, int nz, int pitch,
                      int tx);
bool tma_encode_mask(CUtensorMap *m, const uint32_t *mask, int dir, const TmaGeom &g, int nx, int ny, int nz, int tx);
cudaError_t launch_sweep_tma(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                             cudaStream_t st);
cudaError_t prepare_sweep_tma();

// Lines per tile of the tensor-map variants: x sweeps 8 (variant 0 only); y/z sweeps 32, 16 or 8.
constexpr int kTmaVariants = 3;
inline int tma_variant_count(int dir) { return dir == DIR_X ? 1 : kTmaVariants; }
inline int tma_variant_tx(int dir, int v) { return dir == DIR_X ? 8 : (v == 0 ? 32 : (v == 1 ? 16 : 8)); }
inline int tma_variant(int dir, int tx) {
    if (dir == DIR_X) return tx == 8 ? 0 : -1;
    return tx == 32 ? 0 : (tx == 16 ? 1 : (tx == 8 ? 2 : -1));
}
int tma_shapes(int dir, SweepShape *out, int max);

// Interior-row sweeps (kind 2): x tiles of 8 lines, y/z tiles of 16 or 8.
cudaError_t launch_sweep_inner(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                            cudaStream_t st);
cudaError_t prepare_sweep_inner();
int inner_shapes(int dir, SweepShape *out, int max);
// The cheapest interior-row shape covering the n-2 unknowns of a line along dir.
SweepShape inner_default_shape(int dir, int n);

// Line-per-thread-pair sweeps (kind 3): y/z tiles of 32 lines; `len` of the shape is the number of
// pipeline stages (1 or 2).  Every leg needs its multiplier table (LegDev::line_tab).
cudaError_t launch_sweep_line(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                              cudaStream_t st);
cudaError_t launch_sweep_line_table(int dir, const LegTma *table, int n_legs, int nx, int ny, int nz,
                                    int32_t *err, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                    cudaStream_t st);
cudaError_t prepare_sweep_line();
// Failure-detection probe: waits, with the sweeps' bounded-wait helper and a bound of `limit` SM
// cycles, on a barrier that nothing arrives at, and sets *err as an expired sweep wait does.
cudaError_t launch_wait_probe(int32_t *err, long long limit, int sm_count, cudaStream_t st);
int line_shapes(int dir, SweepShape *out, int max);
void line_table(double e, int n, float2 *out);

}  // namespace npb
