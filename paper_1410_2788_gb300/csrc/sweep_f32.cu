// FP32 instantiations of the LOD line solver (the mixed-precision path).
#include "sweep_launch.cuh"

namespace npb {
cudaError_t launch_sweep_f32(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz,
                             int flags, SweepShape s, cudaStream_t st) {
    return launch_typed<float>(dir, legs, n_legs, nx, ny, nz, flags, s, st);
}
cudaError_t prepare_sweep_f32() { return prepare_typed<float>(); }
}  // namespace npb
