// sweep_tma.cuh -- the FP32 LOD line solves as a persistent, TMA-pipelined kernel.
//
// Same arithmetic as sweep_kernel (segment_reduce + segment_ends per line), different
// data movement: every CTA walks a list of tiles (TX lines each, all their rows); one
// elected thread brings the next tile into the other of two shared-memory stages with
// tensor-memory-accelerator bulk copies (cp.async.bulk.tensor, completion counted on an
// mbarrier) while the block solves the current tile, and sends each solved tile back to
// HBM with a bulk tensor store.  So global traffic is two bulk copies per tile and the
// next tile is always in flight.
//
//   y, z sweeps: a tile is TX = 32 x-adjacent lines; the box is {32 x, rows, 1} (y) or
//     {32 x, 1, rows} (z) of the state, plus the 4-word mask column holding their bits.
//   x sweep: a tile is TX = 8 consecutive y-lines of one z-plane; the row is viewed as
//     {xc, nchunk} so that one box covers sx = xc*nchunk >= nx columns with
//     sx = 4 (mod 8): a warp (8 lines x 4 segments, odd L) then reads its rows from shared
//     memory without bank conflicts.
// Faces, padding rows/columns and inactive lines stay untouched in shared memory, so the
// store writes their loaded values back unchanged.
//
// Every wait on an mbarrier is bounded (about two seconds of SM clock); on expiry the block
// records an error flag that the host reads, waits (again bounded) for its own copies,
// and returns.
#pragma once
#include <cuda.h>

#include "sweep_kernel.cuh"

namespace npb {

constexpr int kTmaMaxLegs = 8;

// One leg of a launch whose legs live in device memory (any number of legs of one grid size).
struct alignas(128) LegTma {
    CUtensorMap umap;  // the leg's state, box of this launch's direction and tile width
    CUtensorMap mmap;  // its line-major node mask (unused when dev.mask is null)
    LegDev dev;
};

struct TmaLaunch {
    CUtensorMap umap[kTmaMaxLegs];  // state of each leg (box per direction)
    CUtensorMap mmap[kTmaMaxLegs];  // node mask of each leg (unused when legs[i].mask is null)
    LegDev legs[kTmaMaxLegs];
    const LegTma *table;            // when set: the legs are table[0 .. n_legs), the arrays above unused
    int32_t *err;                   // set to 1 when a bounded wait expires
    int32_t n_legs, tiles_a, tiles_b;
    int32_t rows, nload;            // y/z: rows per box and boxes per tile
    int32_t sx, mwpr;               // x: shared row stride; mask words per row
    uint32_t tx_u, tx_m;            // bytes per stage: state boxes, mask boxes
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` SM cycles (the launch's bound; by default ~4e9 cycles, about
// two seconds).
constexpr long long kWaitCycles = 4000000000LL;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
                 "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int c0, int c1, int c2,
                                             int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(map),
                 "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__host__ __device__ __forceinline__ size_t tma_align(size_t b) { return (b + 127) & ~(size_t)127; }

// Every bulk tensor copy into shared memory starts on a 128-byte boundary: the stage buffers
// are 128-aligned, and the y/z state boxes of a tile follow each other contiguously, each
// rows*tx*4 bytes long -- a multiple of 128 (tx = 32, or tx = 16 with an even row count), so
// row g of the tile is element g*tx + line whichever box holds it.
__host__ __device__ __forceinline__ size_t tma_data_box_bytes(int rows, int tx) { return (size_t)rows * tx * 4; }

template <int DIR, int TX, int SEG>
__host__ __device__ __forceinline__ size_t tma_smem_bytes(int rows, int nload, int sx, int mwpr) {
    const size_t data = DIR == DIR_X ? (size_t)TX * sx * 4 : (size_t)nload * tma_data_box_bytes(rows, TX);
    const size_t mask = (size_t)TX * mwpr * 4;
    return 128 + 2 * (tma_align(data) + tma_align(mask)) + tma_align((size_t)13 * TX * SEG * 4) + 64;
}

// Bits of rows g0-1 .. g0+L of one line (bit k+1 <-> row g0+k) from its line-major words.
// Row -1 does not exist; its bit never matters because row 0 is a face row.
__device__ __forceinline__ uint32_t segment_bits(const uint32_t *W, int nwords, int g0) {
    const int s = g0 - 1;
    const int s0 = s < 0 ? 0 : s;
    const int w = s0 >> 5;
    const uint32_t lo = w < nwords ? W[w] : 0u;
    const uint32_t hi = w + 1 < nwords ? W[w + 1] : 0u;
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    if (s < 0) return ((uint32_t)v << 1) | 1u;
    return (uint32_t)(v >> (s & 31));
}

template <int DIR, int TX, int SEG, int L>
__global__ void __launch_bounds__(TX *SEG) sweep_tma_kernel(const __grid_constant__ TmaLaunch P, int flags) {
    using T = float;
    static_assert(L >= 3 && L <= 30 && (L & 1), "odd segment length (conflict-free x rows)");
    static_assert((SEG & (SEG - 1)) == 0, "SEG must be a power of two");
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int tid = threadIdx.y * TX + threadIdx.x;
    const int line = threadIdx.x, seg = threadIdx.y, g0 = seg * L;
    const size_t dbox = DIR == DIR_X ? 0 : tma_data_box_bytes(P.rows, TX);  // bytes between state boxes
    const size_t data_b = DIR == DIR_X ? (size_t)TX * P.sx * 4 : (size_t)P.nload * dbox;
    const size_t mask_b = (size_t)TX * P.mwpr * 4;
    T *data[2];
    uint32_t *msk[2];
    // round the dynamic shared base up to 128 bytes (128 spare bytes are requested for this)
    size_t off = (128 - (smem_addr(smem_raw) & 127u)) & 127u;
    for (int s = 0; s < 2; ++s) {
        data[s] = reinterpret_cast<T *>(smem_raw + off);
        off += tma_align(data_b);
        msk[s] = reinterpret_cast<uint32_t *>(smem_raw + off);
        off += tma_align(mask_b);
    }
    T *red = reinterpret_cast<T *>(smem_raw + off);
    off += tma_align((size_t)13 * TX * SEG * 4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + off);
    T *fbuf = red, *pbuf = red + 4 * TX * SEG, *ebuf = red + 12 * TX * SEG;
    const int dboxf = (int)(dbox / 4);
    // shared-memory element of row g of this thread's line
    auto at = [&](int g) -> int { return DIR == DIR_X ? line * P.sx + g : g * TX + line; };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int tpl = P.tiles_a * P.tiles_b;
    const int total = P.n_legs * tpl;

    auto issue = [&](int t, int s) {  // thread 0 only
        const int leg = t / tpl, r = t - leg * tpl, a = r % P.tiles_a, b = r / P.tiles_a;
        const bool has_mask = P.legs[leg].mask != nullptr;
        mbar_expect_tx(&bar[s], P.tx_u + (has_mask ? P.tx_m : 0u));
        if (DIR == DIR_X) {
            const int y0 = 1 + a * TX, z = 1 + b;
            tma_load_4d(data[s], &P.umap[leg], &bar[s], 0, 0, y0, z);
            if (has_mask) tma_load_3d(msk[s], &P.mmap[leg], &bar[s], 0, y0, z);
        } else {
            const int x0 = a * TX, c = 1 + b;
            for (int q = 0; q < P.nload; ++q) {
                const int r0 = q * P.rows;
                T *dst = data[s] + (size_t)q * dboxf;
                if (DIR == DIR_Y) tma_load_3d(dst, &P.umap[leg], &bar[s], x0, r0, c);
                else tma_load_3d(dst, &P.umap[leg], &bar[s], x0, c, r0);
            }
            if (has_mask) tma_load_3d(msk[s], &P.mmap[leg], &bar[s], 0, x0, c);
        }
    };

    int t = blockIdx.x, it = 0;
    if (tid == 0 && t < total) issue(t, 0);
    for (; t < total; t += gridDim.x, ++it) {
        const int s = it & 1;
        const int tn = t + gridDim.x;
        if (tid == 0 && tn < total) {
            bulk_wait_read_all();  // the store from stage s^1 has finished reading it
            issue(tn, s ^ 1);
        }
        const bool got = __syncthreads_and(mbar_wait_bounded(&bar[s], (it >> 1) & 1));
        if (!got) {
            if (tid == 0) {
                atomicExch(P.err, 1);
                if (tn < total) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1);
                bulk_wait_all();
            }
            return;
        }

        // ---- this tile
        const int leg = t / tpl, rr = t - leg * tpl, a = rr % P.tiles_a, bb = rr / P.tiles_a;
        const LegDev &lg = P.legs[leg];
        const int nx = lg.nx, ny = lg.ny, nz = lg.nz;
        const int ndir = DIR == DIR_X ? nx : (DIR == DIR_Y ? ny : nz);
        const T rE0 = (T)lg.rE[0], rE1 = (T)lg.rE[1], rE2 = (T)lg.rE[2];
        const T nlq = (T)lg.nl_q, nlomq = (T)lg.nl_omq;
        const bool nl_on = lg.nl_on != 0;
        const bool has_mask = lg.mask != nullptr;
        T *D = data[s];
        const bool active = DIR == DIR_X ? (1 + a * TX + line <= ny - 2)
                                         : (a * TX + line >= 1 && a * TX + line <= nx - 2);

        const uint32_t nb = !active ? 0u : (has_mask ? segment_bits(msk[s] + line * P.mwpr, P.mwpr, g0) : 0xffffffffu);
        constexpr uint32_t kHalfMask = (1u << (L + 1)) - 1u;
        constexpr uint32_t kNodeMask = (1u << (L + 2)) - 1u;
        const uint32_t both = nb & (nb >> 1), any = nb | (nb >> 1);
        const bool interior_seg = g0 >= 1 && g0 + L - 1 <= ndir - 2;
        const bool all_in = (both & kHalfMask) == kHalfMask && (nb & kNodeMask) == kNodeMask;
        const bool all_out = (any & kHalfMask) == 0u && (nb & kNodeMask) == 0u;
        const bool uniform = active && interior_seg && (all_in || all_out);
        const bool pre_nl = (flags & FUSE_PRE_NL) && nl_on;
        const bool post_nl = (flags & FUSE_POST_NL) && nl_on;

        T al[L], be[L], ga[L];
        T fa, fb, fc, fd, ea, eb, ec, ed;
        if (uniform) {
            // every row is an interior row with the same coefficients
            const bool nl_rows = pre_nl && all_out;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const T v = D[at(g0 + k)];
                al[k] = nl_rows ? nl_flow(v, nlq, nlomq) : v;
            }
            const T e = all_in ? rE2 : rE0;
            const T ca = -e, cb = T(1) + e + e;
            auto coef = [&](int, T &ca_, T &cb_, T &cc_) {
                ca_ = ca;
                cb_ = cb;
                cc_ = ca;
            };
            segment_reduce<T, L>(al, be, ga, coef, fa, fb, fc, fd, ea, eb, ec, ed);
        } else {
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const int g = g0 + k;
                T v = T(0);
                if (active && g < ndir) {
                    v = D[at(g)];
                    if (pre_nl && g >= 1 && g <= ndir - 2 && ((nb >> (k + 1)) & 1u) == 0u) v = nl_flow(v, nlq, nlomq);
                }
                al[k] = v;
            }
            auto eh = [&](int k) -> T {
                return ((both >> k) & 1u) ? rE2 : (((any >> k) & 1u) ? rE1 : rE0);
            };
            auto coef = [&](int k, T &ca_, T &cb_, T &cc_) {
                const int g = g0 + k;
                if (g < 1 || g > ndir - 2) {
                    ca_ = T(0);
                    cb_ = T(1);
                    cc_ = T(0);
                    return;
                }
                const T em = eh(k), ep = eh(k + 1);
                ca_ = -em;
                cc_ = -ep;
                cb_ = T(1) + em + ep;
            };
            segment_reduce<T, L>(al, be, ga, coef, fa, fb, fc, fd, ea, eb, ec, ed);
        }
        T F, E;
        segment_ends<T, TX, SEG>(fa, fb, fc, fd, ea, eb, ec, ed, seg, line, fbuf, pbuf, ebuf, F, E);

        if (uniform) {
            const bool nl_rows = post_nl && all_out;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                T x = k == 0 ? F : (k == L - 1 ? E : al[k] + be[k] * F + ga[k] * E);
                if (nl_rows) x = nl_flow(x, nlq, nlomq);
                D[at(g0 + k)] = x;
            }
        } else if (active) {
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const int g = g0 + k;
                if (g >= 1 && g <= ndir - 2) {
                    T x = k == 0 ? F : (k == L - 1 ? E : al[k] + be[k] * F + ga[k] * E);
                    if (post_nl && ((nb >> (k + 1)) & 1u) == 0u) x = nl_flow(x, nlq, nlomq);
                    D[at(g)] = x;
                }
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (DIR == DIR_X) {
                tma_store_4d(&P.umap[leg], D, 0, 0, 1 + a * TX, 1 + bb);
            } else {
                const int x0 = a * TX, c = 1 + bb;
                for (int q = 0; q < P.nload; ++q) {
                    const int r0 = q * P.rows;
                    const T *src = D + (size_t)q * dboxf;
                    if (DIR == DIR_Y) tma_store_3d(&P.umap[leg], src, x0, r0, c);
                    else tma_store_3d(&P.umap[leg], src, x0, c, r0);
                }
            }
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace npb
