// sweep_inner_launch.cuh -- instantiates the interior-row TMA sweeps (kind 2) for one direction.
#pragma once
#include <algorithm>
#include <map>
#include <utility>
#include <mutex>

#include "sweep_inner.cuh"
#include "tma.h"

namespace npb {

// (SEG, L) pairs for tiles of 8 lines (SEG a multiple of 4 fills whole warps) and of 16 lines
// (SEG even).  L is odd, which keeps the shared-memory rows conflict-free.  (96, 3) is the
// parallel-cyclic-reduction end of the range: three rows per thread, seven PCR rounds.  (8, 13),
// (10, 17), (12, 15) and (16, 15) cover lines of 97, 161 and 225 nodes with less than 10% padding.
#define NPB_INNER_SEGS_X(X) X(4, 17) X(8, 9) X(8, 17) X(12, 11) X(12, 17) X(16, 9) X(16, 17) X(20, 13) X(24, 11) X(24, 17) X(32, 9) \
    X(8, 13) X(12, 15) X(16, 15) X(96, 3)
#define NPB_INNER_SEGS_YZ(X) X(4, 17) X(8, 9) X(8, 17) X(10, 13) X(12, 17) X(16, 9) X(16, 17) X(20, 13) X(24, 11) X(24, 17) X(32, 9) \
    X(8, 13) X(10, 17) X(12, 15) X(16, 15)

template <int DIR, int TX, int SEG, int L>
static cudaError_t launch_inner_shape(const TmaLaunch &P, const TmaGeom &g, int flags, int sm_count, cudaStream_t st) {
    const size_t smem = inner_smem_bytes<TX, SEG>(DIR, g.rows, g.nload, g.sx, g.mwpr);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (DIR != DIR_X && g.nload > 1 && tma_data_box_bytes(g.rows, TX) % 128) return cudaErrorInvalidValue;
    const bool table = P.table != nullptr;
    const bool cn = (flags & FUSE_PRE_CN) != 0;
    if (table && cn) return cudaErrorInvalidValue;  // table launches run the implicit-Euler schemes
    const int variant = table ? 1 : (cn ? 2 : 0);
    auto kern = table ? sweep_inner_kernel<DIR, TX, SEG, L, true>
                      : (cn ? sweep_inner_kernel<DIR, TX, SEG, L, false, true> : sweep_inner_kernel<DIR, TX, SEG, L, false>);
    static std::mutex mu;
    static std::map<std::pair<size_t, int>, int> occ;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = occ.find({smem, variant});
        if (it == occ.end()) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * SEG, smem);
            if (e != cudaSuccess) return e;
            occ[{smem, variant}] = per_sm;
        } else {
            per_sm = it->second;
        }
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int total = P.n_legs * P.tiles_a * P.tiles_b;
    const int grid = std::max(1, std::min(total, per_sm * sm_count));
    kern<<<grid, dim3(TX, SEG), smem, st>>>(P, flags);
    return cudaGetLastError();
}

template <int DIR, int TX>
static cudaError_t launch_inner_dir(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                 cudaStream_t st) {
#define NPB_INNER_CASE(SEG_, L_) \
    if (s.seg == SEG_ && s.len == L_) return launch_inner_shape<DIR, TX, SEG_, L_>(P, g, flags, sm_count, st);
    if constexpr (TX == 8) { NPB_INNER_SEGS_X(NPB_INNER_CASE) } else { NPB_INNER_SEGS_YZ(NPB_INNER_CASE) }
#undef NPB_INNER_CASE
    return cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t prepare_inner_kernel(K kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int DIR, int TX>
static cudaError_t prepare_inner_dir() {
    cudaError_t e = cudaSuccess;
#define NPB_INNER_PREP(SEG_, L_)                                                                                  \
    if (e == cudaSuccess)                                                                                      \
        e = prepare_inner_kernel(sweep_inner_kernel<DIR, TX, SEG_, L_, false>);                                \
    if (e == cudaSuccess) e = prepare_inner_kernel(sweep_inner_kernel<DIR, TX, SEG_, L_, true>);              \
    if (e == cudaSuccess) e = prepare_inner_kernel(sweep_inner_kernel<DIR, TX, SEG_, L_, false, true>);
    if constexpr (TX == 8) { NPB_INNER_SEGS_X(NPB_INNER_PREP) } else { NPB_INNER_SEGS_YZ(NPB_INNER_PREP) }
#undef NPB_INNER_PREP
    return e;
}

}  // namespace npb
