// sweep_tma_f32.cu -- host side of the TMA-pipelined FP32 sweeps: tensor-map geometry and
// encoding, occupancy-sized persistent launches, and the instantiated shapes.
#include <cudaTypedefs.h>

#include <map>
#include <mutex>

#include "sweep_tma.cuh"
#include "tma.h"

namespace npb {

// Instantiated TMA shapes: x sweeps use 8 lines per tile, y/z sweeps 32.
#define NPB_TMA_X_SHAPES(X) X(8, 2, 17) X(8, 4, 9) X(8, 4, 17) X(8, 8, 13) X(8, 8, 17) X(8, 16, 11) X(8, 16, 17) X(8, 32, 9)
#define NPB_TMA_YZ_SHAPES(X) X(32, 2, 17) X(32, 4, 9) X(32, 4, 17) X(32, 8, 13) X(32, 8, 17) X(32, 16, 11) X(32, 16, 17) \
    X(16, 4, 17) X(16, 8, 13) X(16, 8, 17) X(16, 16, 11) X(16, 16, 17) X(16, 32, 9)

static const SweepShape kTmaX[] = {{8, 2, 17, 1}, {8, 4, 9, 1}, {8, 4, 17, 1}, {8, 8, 13, 1},
                                   {8, 8, 17, 1}, {8, 16, 11, 1}, {8, 16, 17, 1}, {8, 32, 9, 1}};
static const SweepShape kTmaYZ[] = {{32, 2, 17, 1}, {32, 4, 9, 1},  {32, 4, 17, 1},  {32, 8, 13, 1},
                                    {32, 8, 17, 1}, {32, 16, 11, 1}, {32, 16, 17, 1}, {16, 4, 17, 1},
                                    {16, 8, 13, 1}, {16, 8, 17, 1},  {16, 16, 11, 1}, {16, 16, 17, 1},
                                    {16, 32, 9, 1}};

int tma_shapes(int dir, SweepShape *out, int max) {
    int n = 0;
    if (dir == DIR_X) {
        for (const auto &s : kTmaX)
            if (n < max) out[n++] = s;
    } else {
        for (const auto &s : kTmaYZ)
            if (n < max) out[n++] = s;
    }
    return n;
}

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// x: the row is viewed as {xc, nchunk} with sx = xc * nchunk, nx <= sx <= pitch, sx = 4 (mod 8),
// xc a multiple of 4 and at most 256 (a TMA box dimension).  y/z: rows per box <= 256.
TmaGeom tma_geometry(int dir, int nx, int ny, int nz, int pitch) {
    TmaGeom g{};
    g.mwpr = dir == DIR_X ? mask_words_per_row(pitch) : line_words(dir == DIR_Y ? ny : nz);
    if (dir == DIR_X) {
        for (int sx = (nx + 3) / 4 * 4; sx <= pitch && !g.ok; sx += 4) {
            if (sx % 8 != 4) continue;
            for (int nc = (sx + 255) / 256; nc <= 8; ++nc) {
                if (sx % nc || (sx / nc) % 4 || sx / nc > 256) continue;
                g.sx = sx;
                g.xc = sx / nc;
                g.nchunk = nc;
                g.ok = true;
                break;
            }
        }
        if (g.mwpr > 256) g.ok = false;
    } else {
        const int n = dir == DIR_Y ? ny : nz;
        g.nload = (n + 255) / 256;
        g.rows = (n + g.nload - 1) / g.nload;
        if (g.nload > 1) g.rows = (g.rows + 3) & ~3;  // boxes of 8 or more lines stay 128-byte multiples
        g.ok = g.nload <= 2 && g.rows <= 256;
    }
    return g;
}

bool tma_encode_state(CUtensorMap *m, void *u, int dir, const TmaGeom &g, int nx, int ny, int nz, int pitch,
                      int tx) {
    auto enc = encoder();
    if (!enc || !g.ok) return false;
    (void)nx;
    CUresult r;
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (dir == DIR_X) {
        const cuuint64_t dims[4] = {(cuuint64_t)g.xc, (cuuint64_t)g.nchunk, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[3] = {(cuuint64_t)g.xc * 4, (cuuint64_t)pitch * 4, (cuuint64_t)ny * pitch * 4};
        const cuuint32_t box[4] = {(cuuint32_t)g.xc, (cuuint32_t)g.nchunk, (cuuint32_t)tx, 1};
        r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, u, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)ny * pitch * 4};
        const cuuint32_t box[3] = {(cuuint32_t)tx, dir == DIR_Y ? (cuuint32_t)g.rows : 1u,
                                   dir == DIR_Z ? (cuuint32_t)g.rows : 1u};
        r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, u, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

// The mask of direction d as a line-major bit array: x -> the node mask [nz][ny][words(pitch)],
// y -> [nz][nx][words(ny)], z -> [ny][nx][words(nz)].  One box holds all the bits of the tile's
// lines: {words, tx lines, 1}.
bool tma_encode_mask(CUtensorMap *m, const uint32_t *mask, int dir, const TmaGeom &g, int nx, int ny, int nz, int tx) {
    auto enc = encoder();
    if (!enc || !g.ok) return false;
    const cuuint32_t one[3] = {1, 1, 1};
    const cuuint64_t lines = dir == DIR_X ? (cuuint64_t)ny : (cuuint64_t)nx;
    const cuuint64_t planes = dir == DIR_Z ? (cuuint64_t)ny : (cuuint64_t)nz;
    const cuuint64_t dims[3] = {(cuuint64_t)g.mwpr, lines, planes};
    const cuuint64_t strides[2] = {(cuuint64_t)g.mwpr * 4, lines * g.mwpr * 4};
    const cuuint32_t box[3] = {(cuuint32_t)g.mwpr, (cuuint32_t)tx, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint32_t *>(mask), dims, strides, box, one,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int DIR, int TX, int SEG, int L>
static cudaError_t launch_tma_shape(const TmaLaunch &P, const TmaGeom &g, int flags, int sm_count, cudaStream_t st) {
    const size_t smem = tma_smem_bytes<DIR, TX, SEG>(g.rows, g.nload, g.sx, g.mwpr);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    // every shared-memory destination of a bulk tensor copy must sit on a 128-byte boundary
    if (DIR != DIR_X && g.nload > 1 && tma_data_box_bytes(g.rows, TX) % 128) return cudaErrorInvalidValue;
    auto kern = sweep_tma_kernel<DIR, TX, SEG, L>;
    static std::mutex mu;
    static std::map<size_t, int> occ;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = occ.find(smem);
        if (it == occ.end()) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * SEG, smem);
            if (e != cudaSuccess) return e;
            occ[smem] = per_sm;
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

cudaError_t launch_sweep_inner_x(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count, cudaStream_t st);
cudaError_t launch_sweep_inner_y(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count, cudaStream_t st);
cudaError_t launch_sweep_inner_z(TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count, cudaStream_t st);
cudaError_t prepare_sweep_inner_x();
cudaError_t prepare_sweep_inner_y();
cudaError_t prepare_sweep_inner_z();

static const int kInnerSegsX[][2] = {{4, 17},  {8, 9},   {8, 17},  {12, 11}, {12, 17}, {16, 9},  {16, 17}, {20, 13},
                                     {24, 11}, {24, 17}, {32, 9},  {8, 13},  {12, 15}, {16, 15}, {96, 3}};
static const int kInnerSegsYZ[][2] = {{4, 17},  {8, 9},   {8, 17}, {10, 13}, {12, 17}, {16, 9},  {16, 17}, {20, 13},
                                      {24, 11}, {24, 17}, {32, 9}, {8, 13},  {10, 17}, {12, 15}, {16, 15}};

int inner_shapes(int dir, SweepShape *out, int max) {
    int n = 0;
    if (dir != DIR_X) {
        for (const auto &p : kInnerSegsYZ)
            if (n < max) out[n++] = SweepShape{16, p[0], p[1], 2};
    }
    for (const auto &p : kInnerSegsX)  // 8 lines per tile: x, and y/z in 32-byte boxes
        if (n < max) out[n++] = SweepShape{8, p[0], p[1], 2};
    return n;
}

SweepShape inner_default_shape(int dir, int n) {
    // rows solved (padding included) plus about eight rows' worth of work per segment for the
    // reduced system; the cheapest shape covering the n-2 unknowns
    SweepShape t[64], best{0, 0, 0, 0};
    const int k = inner_shapes(dir, t, 64);
    auto cost = [](const SweepShape &s) { return s.seg * s.len + 8 * s.seg; };
    for (int i = 0; i < k; ++i) {
        if (t[i].seg * t[i].len < n - 2) continue;
        if (best.tx == 0 || cost(t[i]) < cost(best)) best = t[i];
    }
    return best;
}

cudaError_t prepare_sweep_inner() {
    cudaError_t e = prepare_sweep_inner_x();
    if (e == cudaSuccess) e = prepare_sweep_inner_y();
    if (e == cudaSuccess) e = prepare_sweep_inner_z();
    return e;
}

static void tma_tiles(int dir, TmaLaunch &P, const TmaGeom &g, SweepShape s, int nx, int ny, int nz) {
    P.mwpr = g.mwpr;
    P.rows = g.rows;
    P.nload = g.nload;
    P.sx = g.sx;
    if (dir == DIR_X) {
        P.tiles_a = (ny - 2 + s.tx - 1) / s.tx;
        P.tiles_b = nz - 2;
        P.tx_u = (uint32_t)(s.tx * g.sx * 4);
        P.tx_m = (uint32_t)(s.tx * g.mwpr * 4);
    } else {
        P.tiles_a = (nx - 1 + s.tx - 1) / s.tx;
        P.tiles_b = dir == DIR_Y ? nz - 2 : ny - 2;
        P.tx_u = (uint32_t)(g.nload * g.rows * s.tx * 4);
        P.tx_m = (uint32_t)(s.tx * g.mwpr * 4);
    }
}

cudaError_t launch_sweep_inner(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                            cudaStream_t st) {
    if (P.table) return cudaErrorInvalidValue;
    tma_tiles(dir, P, g, s, P.legs[0].nx, P.legs[0].ny, P.legs[0].nz);
    if (dir == DIR_X) return launch_sweep_inner_x(P, g, flags, s, sm_count, st);
    if (dir == DIR_Y) return launch_sweep_inner_y(P, g, flags, s, sm_count, st);
    return launch_sweep_inner_z(P, g, flags, s, sm_count, st);
}

cudaError_t launch_sweep_inner_table(int dir, const LegTma *table, int n_legs, int nx, int ny, int nz,
                                    int32_t *err, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                                    cudaStream_t st) {
    TmaLaunch P;
    memset(&P, 0, sizeof P);
    P.table = table;
    P.n_legs = n_legs;
    P.err = err;
    tma_tiles(dir, P, g, s, nx, ny, nz);
    if (dir == DIR_X) return launch_sweep_inner_x(P, g, flags, s, sm_count, st);
    if (dir == DIR_Y) return launch_sweep_inner_y(P, g, flags, s, sm_count, st);
    return launch_sweep_inner_z(P, g, flags, s, sm_count, st);
}

cudaError_t launch_sweep_tma(int dir, TmaLaunch &P, const TmaGeom &g, int flags, SweepShape s, int sm_count,
                             cudaStream_t st) {
    const int nx = P.legs[0].nx, ny = P.legs[0].ny, nz = P.legs[0].nz;
    P.mwpr = g.mwpr;
    P.rows = g.rows;
    P.nload = g.nload;
    P.sx = g.sx;
    if (dir == DIR_X) {
        P.tiles_a = (ny - 2 + s.tx - 1) / s.tx;
        P.tiles_b = nz - 2;
        P.tx_u = (uint32_t)(s.tx * g.sx * 4);
        P.tx_m = (uint32_t)(s.tx * g.mwpr * 4);
    } else {
        P.tiles_a = (nx - 1 + s.tx - 1) / s.tx;
        P.tiles_b = dir == DIR_Y ? nz - 2 : ny - 2;
        P.tx_u = (uint32_t)(g.nload * g.rows * s.tx * 4);
        P.tx_m = (uint32_t)(s.tx * g.mwpr * 4);
    }
#define NPB_TMA_CASE_X(TX_, SEG_, L_)                                                        \
    if (dir == DIR_X && s.tx == TX_ && s.seg == SEG_ && s.len == L_)                         \
        return launch_tma_shape<DIR_X, TX_, SEG_, L_>(P, g, flags, sm_count, st);
#define NPB_TMA_CASE_YZ(TX_, SEG_, L_)                                                       \
    if (dir != DIR_X && s.tx == TX_ && s.seg == SEG_ && s.len == L_) {                       \
        if (dir == DIR_Y) return launch_tma_shape<DIR_Y, TX_, SEG_, L_>(P, g, flags, sm_count, st); \
        return launch_tma_shape<DIR_Z, TX_, SEG_, L_>(P, g, flags, sm_count, st);            \
    }
    NPB_TMA_X_SHAPES(NPB_TMA_CASE_X)
    NPB_TMA_YZ_SHAPES(NPB_TMA_CASE_YZ)
#undef NPB_TMA_CASE_X
#undef NPB_TMA_CASE_YZ
    return cudaErrorInvalidValue;
}

template <int DIR, int TX, int SEG, int L>
static cudaError_t prepare_tma_shape() {
    cudaError_t e = cudaFuncSetAttribute(sweep_tma_kernel<DIR, TX, SEG, L>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_tma_kernel<DIR, TX, SEG, L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t prepare_sweep_tma() {
    cudaError_t e = cudaSuccess;
#define NPB_TMA_PREP_X(TX_, SEG_, L_) \
    if (e == cudaSuccess) e = prepare_tma_shape<DIR_X, TX_, SEG_, L_>();
#define NPB_TMA_PREP_YZ(TX_, SEG_, L_)                                      \
    if (e == cudaSuccess) e = prepare_tma_shape<DIR_Y, TX_, SEG_, L_>(); \
    if (e == cudaSuccess) e = prepare_tma_shape<DIR_Z, TX_, SEG_, L_>();
    NPB_TMA_X_SHAPES(NPB_TMA_PREP_X)
    NPB_TMA_YZ_SHAPES(NPB_TMA_PREP_YZ)
#undef NPB_TMA_PREP_X
#undef NPB_TMA_PREP_YZ
    return e;
}

}  // namespace npb
