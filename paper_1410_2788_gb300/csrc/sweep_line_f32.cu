// sweep_line_f32.cu -- host side of the FP32 line-per-thread-pair sweeps (solver kind 3, y and z):
// tile geometry, occupancy-sized persistent launches, the instantiated pipeline depths.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "sweep_line.cuh"
#include "tma.h"

namespace npb {

template <int DIR, bool TABLE, int NS>
static cudaError_t launch_line_ns(const TmaLaunch &P, const TmaGeom &g, int flags, int sm_count, cudaStream_t st) {
    const size_t smem = line_smem_bytes(NS, g.rows, g.nload, g.mwpr);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    // every shared-memory destination of a bulk tensor copy sits on a 128-byte boundary
    if (g.nload > 1 && tma_data_box_bytes(g.rows, kLineTX) % 128) return cudaErrorInvalidValue;
    auto kern = sweep_line_kernel<DIR, TABLE, NS>;
    static std::mutex mu;
    static std::map<std::pair<size_t, int>, int> occ;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto key = std::make_pair(smem, (int)TABLE * 2 + NS);
        auto it = occ.find(key);
        if (it == occ.end()) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLineThreads, smem);
            if (e != cudaSuccess) return e;
            occ[key] = per_sm;
        } else {
            per_sm = it->second;
        }
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int total = P.n_legs * P.tiles_a * P.tiles_b;
    const int grid = std::max(1, std::min(total, per_sm * sm_count));
    kern<<<grid, kLineThreads, smem, st>>>(P, flags);
    return cudaGetLastError();
}

template <bool TABLE>
static cudaError_t launch_line(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                               cudaStream_t st) {
    if (dir == DIR_X || s.tx != kLineTX || s.seg != 2) return cudaErrorInvalidValue;
    const int nx = TABLE ? P.tiles_a : P.legs[0].nx;  // (table launches pass the extents in tiles_a/b)
    const int nplane = TABLE ? P.tiles_b : (dir == DIR_Y ? P.legs[0].nz : P.legs[0].ny);
    P.mwpr = g.mwpr;
    P.rows = g.rows;
    P.nload = g.nload;
    P.sx = 0;
    P.tiles_a = (nx - 1 + kLineTX - 1) / kLineTX;
    P.tiles_b = nplane - 2;
    P.tx_u = (uint32_t)(g.nload * g.rows * kLineTX * 4);
    P.tx_m = (uint32_t)(kLineTX * g.mwpr * 4);
    if (s.len == 1) {
        if (dir == DIR_Y) return launch_line_ns<DIR_Y, TABLE, 1>(P, g, flags, sm_count, st);
        return launch_line_ns<DIR_Z, TABLE, 1>(P, g, flags, sm_count, st);
    }
    if (s.len == 2) {
        if (dir == DIR_Y) return launch_line_ns<DIR_Y, TABLE, 2>(P, g, flags, sm_count, st);
        return launch_line_ns<DIR_Z, TABLE, 2>(P, g, flags, sm_count, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_line(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                              cudaStream_t st) {
    if (P.table) return cudaErrorInvalidValue;
    for (int i = 0; i < P.n_legs; ++i)
        if (!P.legs[i].line_tab[dir]) return cudaErrorInvalidValue;
    return launch_line<false>(dir, P, g, flags, s, sm_count, st);
}

cudaError_t launch_sweep_line_table(int dir, const LegTma *table, int n_legs, int nx, int ny, int nz, int32_t *err,
                                    const TmaGeom &g, int flags, SweepShape s, int sm_count, cudaStream_t st) {
    TmaLaunch P;
    memset(&P, 0, sizeof P);
    P.table = table;
    P.n_legs = n_legs;
    P.err = err;
    P.tiles_a = nx;
    P.tiles_b = dir == DIR_Y ? nz : ny;
    return launch_line<true>(dir, P, g, flags, s, sm_count, st);
}

template <int DIR, bool TABLE, int NS>
static cudaError_t prepare_line_ns() {
    auto kern = sweep_line_kernel<DIR, TABLE, NS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t prepare_sweep_line() {
    cudaError_t e = cudaSuccess;
#define NPB_LINE_PREP(D_, T_, NS_) \
    if (e == cudaSuccess) e = prepare_line_ns<D_, T_, NS_>();
    NPB_LINE_PREP(DIR_Y, false, 1)
    NPB_LINE_PREP(DIR_Y, false, 2)
    NPB_LINE_PREP(DIR_Y, true, 1)
    NPB_LINE_PREP(DIR_Y, true, 2)
    NPB_LINE_PREP(DIR_Z, false, 1)
    NPB_LINE_PREP(DIR_Z, false, 2)
    NPB_LINE_PREP(DIR_Z, true, 1)
    NPB_LINE_PREP(DIR_Z, true, 2)
#undef NPB_LINE_PREP
    return e;
}

// One block per SM waits on an mbarrier that no copy and no thread ever arrives at, bounded to
// `limit` SM cycles by the helper every sweep wait uses; the wait expires and the block sets the
// error flag an expired sweep wait sets.  No copy is in flight anywhere in the probe.
__global__ void k_wait_probe(int32_t *err, long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit)) atomicExch(err, 1);
}

cudaError_t launch_wait_probe(int32_t *err, long long limit, int sm_count, cudaStream_t st) {
    k_wait_probe<<<sm_count, 32, 0, st>>>(err, limit);
    return cudaGetLastError();
}

// Kind-3 shapes: 32 lines per tile, two threads per line, 1 or 2 pipeline stages (in `len`).
int line_shapes(int dir, SweepShape *out, int max) {
    int n = 0;
    if (dir == DIR_X) return 0;
    const SweepShape s[2] = {{kLineTX, 2, 2, 3}, {kLineTX, 2, 1, 3}};
    for (const auto &x : s)
        if (n < max) out[n++] = x;
    return n;
}

// (m_j, cp_j), j = 1 .. ceil((n-2)/2): the Thomas multipliers of a line of n nodes whose half
// points all carry r*eps = e, eliminated from either end (the two halves mirror each other).
void line_table(double e, int n, float2 *out) {
    const int N = n - 2, p = (N + 1) / 2;
    double cp = 0.0;
    for (int j = 1; j <= p; ++j) {
        const double m = 1.0 / (1.0 + 2.0 * e - e * cp);
        cp = e * m;
        out[j - 1] = make_float2((float)m, (float)cp);
    }
}

}  // namespace npb
