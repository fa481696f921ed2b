// Interior-row TMA sweeps along z (16 lines per tile).
#include "sweep_inner_launch.cuh"

namespace npb {
cudaError_t launch_sweep_inner_z(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                  cudaStream_t st) {
    if (s.tx != 16) return cudaErrorInvalidValue;
    return launch_inner_dir<DIR_Z, 16>(P, g, flags, s, sm_count, st);
}
cudaError_t prepare_sweep_inner_z() { return prepare_inner_dir<DIR_Z, 16>(); }
}  // namespace npb
