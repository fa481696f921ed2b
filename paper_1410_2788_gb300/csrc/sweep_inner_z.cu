// Interior-row TMA sweeps along z (16 or 8 lines per tile).
#include "sweep_inner_launch.cuh"

namespace npb {
cudaError_t launch_sweep_inner_z(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                  cudaStream_t st) {
    if (s.tx == 16) return launch_inner_dir<DIR_Z, 16>(P, g, flags, s, sm_count, st);
    if (s.tx == 8) return launch_inner_dir<DIR_Z, 8>(P, g, flags, s, sm_count, st);
    return cudaErrorInvalidValue;
}
cudaError_t prepare_sweep_inner_z() {
    cudaError_t e = prepare_inner_dir<DIR_Z, 16>();
    return e == cudaSuccess ? prepare_inner_dir<DIR_Z, 8>() : e;
}
}  // namespace npb
