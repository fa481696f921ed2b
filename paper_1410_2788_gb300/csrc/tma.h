// tma.h -- host interface of the TMA-pipelined FP32 sweeps (sweep_tma_f32.cu).
#pragma once
#include <cuda.h>

#include "npb_internal.cuh"

namespace npb {

struct TmaLaunch;

struct TmaGeom {
    bool ok;
    int rows, nload;      // y/z: rows per box, boxes per tile
    int sx, xc, nchunk;   // x: shared row stride = xc * nchunk
    int mwpr;             // mask words per row
};

TmaGeom tma_geometry(int dir, int nx, int ny, int nz, int pitch);
bool tma_encode_state(CUtensorMap *m, void *u, int dir, const TmaGeom &g, int nx, int ny, int nz, int pitch);
bool tma_encode_mask(CUtensorMap *m, const uint32_t *mask, int dir, const TmaGeom &g, int ny, int nz);
cudaError_t launch_sweep_tma(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                             cudaStream_t st);
cudaError_t prepare_sweep_tma();
int tma_shapes(int dir, SweepShape *out, int max);

}  // namespace npb
