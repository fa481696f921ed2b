// sweep_launch.cuh -- instantiates the line solver for one element type and dispatches
// a (TX, SEG, L) shape to its kernel.  Included once per element type.
#pragma once
#include "sweep_kernel.cuh"

namespace npb {

// The instantiated shapes: TX lines per block, SEG segments per line, L rows per segment.
// A line of n nodes needs SEG * L >= n; the largest supported line is 32 * 9 = 288 nodes.
#define NPB_SWEEP_SHAPES(X) \
    X(16, 2, 17)            \
    X(16, 4, 9)             \
    X(16, 4, 17)            \
    X(16, 8, 9)             \
    X(16, 8, 13)            \
    X(16, 8, 17)            \
    X(16, 16, 9)            \
    X(16, 16, 11)           \
    X(16, 16, 17)           \
    X(16, 32, 9)            \
    X(32, 8, 17)            \
    X(32, 16, 9)

template <typename T, int DIR, int TX, int SEG, int L>
static cudaError_t launch_shape(const LegDev *legs, int n_legs, int nx, int ny, int nz, int flags,
                                cudaStream_t st) {
    dim3 block(TX, SEG);
    dim3 grid;
    if (DIR == DIR_X) grid = dim3((ny - 2 + TX - 1) / TX, nz - 2, n_legs);
    else if (DIR == DIR_Y) grid = dim3((nx - 1 + TX - 1) / TX, nz - 2, n_legs);
    else grid = dim3((nx - 1 + TX - 1) / TX, ny - 2, n_legs);
    const int pitch = (nx + 31) / 32 * 32;
    const size_t smem = sweep_smem_bytes<T, DIR, TX, SEG>(nx, pitch);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    sweep_kernel<T, DIR, TX, SEG, L><<<grid, block, smem, st>>>(legs, flags);
    return cudaGetLastError();
}

template <typename T, int TX, int SEG, int L>
static cudaError_t prepare_shape() {
    cudaError_t e = cudaSuccess;
    const int big = 200 * 1024;
    const int carve = cudaSharedmemCarveoutMaxShared;
    e = cudaFuncSetAttribute(sweep_kernel<T, DIR_X, TX, SEG, L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             carve);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_kernel<T, DIR_Y, TX, SEG, L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 carve);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_kernel<T, DIR_Z, TX, SEG, L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 carve);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<T, DIR_X, TX, SEG, L>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_kernel<T, DIR_Y, TX, SEG, L>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_kernel<T, DIR_Z, TX, SEG, L>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    return e;
}

template <typename T>
static cudaError_t launch_typed(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz,
                                int flags, SweepShape s, cudaStream_t st) {
#define NPB_CASE(TX_, SEG_, L_)                                                                  \
    if (s.tx == TX_ && s.seg == SEG_ && s.len == L_) {                                           \
        if (dir == DIR_X) return launch_shape<T, DIR_X, TX_, SEG_, L_>(legs, n_legs, nx, ny, nz, flags, st); \
        if (dir == DIR_Y) return launch_shape<T, DIR_Y, TX_, SEG_, L_>(legs, n_legs, nx, ny, nz, flags, st); \
        return launch_shape<T, DIR_Z, TX_, SEG_, L_>(legs, n_legs, nx, ny, nz, flags, st);       \
    }
    NPB_SWEEP_SHAPES(NPB_CASE)
#undef NPB_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t prepare_typed() {
    cudaError_t e = cudaSuccess;
#define NPB_PREP(TX_, SEG_, L_) \
    if (e == cudaSuccess) e = prepare_shape<T, TX_, SEG_, L_>();
    NPB_SWEEP_SHAPES(NPB_PREP)
#undef NPB_PREP
    return e;
}

}  // namespace npb
