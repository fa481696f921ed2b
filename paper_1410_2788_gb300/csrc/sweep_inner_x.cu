// Interior-row TMA sweeps along x (8 lines per tile).
#include "sweep_inner_launch.cuh"

namespace npb {
cudaError_t launch_sweep_inner_x(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                  cudaStream_t st) {
    if (s.tx != 8) return cudaErrorInvalidValue;
    return launch_inner_dir<DIR_X, 8>(P, g, flags, s, sm_count, st);
}
cudaError_t prepare_sweep_inner_x() { return prepare_inner_dir<DIR_X, 8>(); }
}  // namespace npb
