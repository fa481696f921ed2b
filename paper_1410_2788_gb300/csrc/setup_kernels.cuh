// setup_kernels.cuh -- declarations of the per-grid set-up kernels and state helpers.
#pragma once
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

namespace npb {

struct GridGeom {
    int nx, ny, nz, pitch;
    double h, ox, oy, oz;
};

struct RawEntry {       // one (atom, corner) contribution of the trilinear spread
    int32_t x, line, key, pad;
    double val;
};

struct ChargeScratch {  // device scratch used while building the charge list
    int32_t *count;      // [ny*nz] raw entries per x-line
    int32_t *fill;       // [ny*nz] bucket fill counters
    int32_t *raw_begin;  // [ny*nz] bucket offsets
    int32_t *total;      // [1] number of merged entries
    RawEntry *raw;       // [8*n_atoms]
    RawEntry *bucket;    // [8*n_atoms]
};

__host__ __device__ int64_t face_count(int nx, int ny, int nz);

cudaError_t setup_mask(const GridGeom &g, const double *xyz, const double *radius, int n_atoms,
                       uint32_t *mask, uint32_t *hx, uint32_t *hy, uint32_t *hz, uint32_t *my, uint32_t *mz,
                       cudaStream_t st);
cudaError_t setup_charges(const GridGeom &g, const double *xyz, const double *q, int n_atoms,
                          ChargeScratch &s, int32_t *line_begin, int32_t *line_count, int32_t *ent_x,
                          double *ent_qt, int64_t *ent_off, int2 *ent_xq, cudaStream_t st);
// Both media's faces in one pass with FP32 pair terms: solvent (eps_out, kbar) into out_s,
// vacuum (eps_in, Coulomb) into out_v.
cudaError_t setup_boundary_pair(const GridGeom &g, const double *xyz, const double *q, int n_atoms, double eps_out,
                                double kbar, double eps_in, double *out_s, double *out_v, cudaStream_t st,
                                bool fp64 = false);
cudaError_t init_leg(int prec, const GridGeom &g, const double *bc, void *u, cudaStream_t st);
cudaError_t unpad_state(int prec, const GridGeom &g, const void *u, double *out, cudaStream_t st);
cudaError_t pad_state(int prec, const GridGeom &g, const double *in, void *u, cudaStream_t st);
cudaError_t mask_dense(const GridGeom &g, const uint32_t *mask, uint8_t *out, cudaStream_t st);
cudaError_t qt_dense(const GridGeom &g, const int32_t *line_begin, const int32_t *line_count,
                     const int32_t *ent_x, const double *ent_qt, double *out, cudaStream_t st);

}  // namespace npb
