// sweep_inner.cuh -- FP32 LOD line solves over the interior rows, TMA-pipelined, one code path.
//
// The implicit-Euler line system of one LOD direction (Eq. 12 with the harmonic half-point
// eps of Eq. 14) has n-2 unknowns per line, rows 1 .. n-2; the face values u_0 and u_{n-1} are
// Dirichlet data.  A tile of TX lines sits in shared memory (bulk tensor copies, two stages,
// persistent blocks, exactly as sweep_tma.cuh).  Thread (line, seg) holds the L unknowns
// seg*L+1 .. seg*L+L of its line in registers and runs the modified Thomas elimination on them,
// writing every row as alpha + beta F + gamma E in its segment's first (F) and last (E)
// unknown; the segment ends of a line then form a tridiagonal system in the E's that the SEG
// threads of the line solve by parallel cyclic reduction through shared memory.
//
// Every segment runs the same instruction stream (no divergence between segments inside and
// outside the molecule, or at the ends of the line):
//   * eps at the half points comes from the node-mask bits (both nodes inside: eps_in; one:
//     the harmonic mean; none: eps_out), decoded as the elimination walks the rows;
//   * rows past the last unknown (the segment grid is rounded up to SEG*L) read as zero and are
//     decoupled from the unknowns below them by dropping the upward coupling of row n-2, whose
//     face term eps u_{n-1} is moved to its right-hand side before the solve;
//   * u_0 enters through the first row of segment 0 in the reduced system.
#pragma once
#include <type_traits>

#include "f32x2.cuh"
#include "sweep_tma.cuh"

namespace npb {

// Charge entries of the next x tile held in registers per thread (the fused source stage); a
// tile with more than kSrcRegs * threads entries reads the rest when they are applied.
constexpr int kSrcRegs = 2;

// Shared-memory stages of the tile pipeline: tile t+k*grid is in flight while tile t is solved,
// k < kInnerStages.
constexpr int kInnerStages = 2;

// Largest PCR stride for SEG segments (the highest power of two below SEG).
template <int SEG>
__host__ __device__ constexpr int pcr_top() {
    int s = 1;
    while (2 * s < SEG) s *= 2;
    return SEG > 1 ? s : 0;
}

// PCR buffer of one round: SEG*TX rows with pcr_top*TX identity rows on either side, so that the
// reads at +-stride need no bounds checks.
template <int TX, int SEG>
__host__ __device__ constexpr int pcr_rows() {
    return (SEG + 2 * pcr_top<SEG>()) * TX;
}

template <int TX, int SEG>
__host__ __device__ __forceinline__ size_t inner_smem_bytes(int dir, int rows, int nload, int sx, int mwpr) {
    const size_t data = dir == DIR_X ? (size_t)TX * sx * 4 : (size_t)nload * tma_data_box_bytes(rows, TX);
    const size_t mask = (size_t)TX * mwpr * 4;
    const size_t red = (size_t)(TX * SEG + 2 * pcr_rows<TX, SEG>()) * 16 + (size_t)TX * SEG * 4;
    return 128 + kInnerStages * (tma_align(data) + tma_align(mask)) + tma_align(red) + 128;  // + barriers, tile indices
}

// The segment ends of one line: segment s contributes its F row (fa E_{s-1} + fb F_s + fc E_s = fd)
// and its E row (ea F_s + eb E_s + ec F_{s+1} = ed).  Eliminating the F's with the neighbour's
// F row leaves one tridiagonal row per segment in the E's, reduced by PCR in ceil(log2 SEG)
// rounds.  pbuf points at the first real row of two margined buffers (pcr_rows apart).  Every
// thread of the block calls it (it synchronises the block).
template <int TX, int SEG>
__device__ __forceinline__ void inner_ends(float fa, float fb, float fc, float fd, float ea, float eb, float ec,
                                           float ed, int seg, int line, float4 *fbuf, float4 *pbuf, float *ebuf,
                                           float &F, float &E) {
    const int me = seg * TX + line;
    fbuf[me] = make_float4(fa, fb, fc, fd);
    __syncthreads();
    const float ifb = fast_rcp(fb);
    float A = -ea * fa * ifb;
    float B = eb - ea * fc * ifb;
    float C = 0.f;
    float D = ed - ea * fd * ifb;
    if (seg + 1 < SEG) {
        const float4 n = fbuf[me + TX];
        const float inb = ec * fast_rcp(n.y);
        B -= n.x * inb;
        C = -n.z * inb;
        D -= n.w * inb;
    }
#pragma unroll
    for (int st = 1, r = 0; st < SEG; st <<= 1, ++r) {
        float4 *buf = pbuf + (r & 1) * pcr_rows<TX, SEG>();
        buf[me] = make_float4(A, B, C, D);
        __syncthreads();
        const float4 lo = buf[me - st * TX], hi = buf[me + st * TX];
        const float k1 = A * fast_rcp(lo.y), k2 = C * fast_rcp(hi.y);
        B = B - k1 * lo.z - k2 * hi.x;
        D = D - k1 * lo.w - k2 * hi.w;
        A = -k1 * lo.x;
        C = -k2 * hi.z;
    }
    E = D * fast_rcp(B);
    ebuf[me] = E;
    __syncthreads();
    const float Ep = seg > 0 ? ebuf[me - TX] : 0.f;
    F = (fd - fa * Ep - fc * E) * ifb;
}

// TABLE: the legs' tensor maps and constants come from the device-memory table P.table (any number
// of legs of one grid size) instead of the launch's inline arrays (up to kTmaMaxLegs legs).
// Resident blocks asked of the register allocator: 24 warps per SM for blocks below 256 threads;
// 32 warps (64 registers) for 256 threads and more, where it measured faster despite a few spills.
template <int NT>
constexpr int inner_min_blocks() {
    return NT >= 256 ? (1024 / NT > 0 ? 1024 / NT : 1) : (768 / NT > 0 ? 768 / NT : 1);
}

// CN: the explicit half of a Crank-Nicolson sweep on the loaded lines (flag FUSE_PRE_CN), compiled
// as its own variant so that the implicit-Euler sweeps carry none of its code.
template <int DIR, int TX, int SEG, int L, bool TABLE, bool CN = false>
__global__ void __launch_bounds__(TX *SEG, inner_min_blocks<TX * SEG>())
    sweep_inner_kernel(const __grid_constant__ TmaLaunch P, int flags) {
    using T = float;
    static_assert(L >= 3 && L <= 29 && (L & 1), "odd segment length (conflict-free rows); L+2 node bits fit a word");
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int tid = threadIdx.y * TX + threadIdx.x;
    const int line = threadIdx.x, seg = threadIdx.y;
    const size_t dbox = DIR == DIR_X ? 0 : tma_data_box_bytes(P.rows, TX);
    const size_t data_b = DIR == DIR_X ? (size_t)TX * P.sx * 4 : (size_t)P.nload * dbox;
    const size_t mask_b = (size_t)TX * P.mwpr * 4;
    // stage s: data at base + s * stage, mask after it (selected, not indexed: no local memory)
    const size_t base = (128 - (smem_addr(smem_raw) & 127u)) & 127u;
    const size_t stage = tma_align(data_b) + tma_align(mask_b);
    constexpr int NS = kInnerStages;
    auto data = [&](int s) { return reinterpret_cast<T *>(smem_raw + base + (size_t)s * stage); };
    auto msk = [&](int s) {
        return reinterpret_cast<uint32_t *>(smem_raw + base + (size_t)s * stage + tma_align(data_b));
    };
    size_t off = base + NS * stage;
    constexpr int kPad = pcr_top<SEG>() * TX, kRows = pcr_rows<TX, SEG>();
    float4 *fbuf = reinterpret_cast<float4 *>(smem_raw + off);
    float4 *pbuf = fbuf + TX * SEG + kPad;  // first real row of PCR buffer 0
    float *ebuf = reinterpret_cast<float *>(fbuf + TX * SEG + 2 * kRows);
    off += tma_align((size_t)(TX * SEG + 2 * kRows) * 16 + (size_t)TX * SEG * 4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + off);
    int4 *tinfo = reinterpret_cast<int4 *>(bar + 4);  // (leg, a, b) of the tile in each stage
    auto legp = [&](int leg) -> const LegDev & {
        if constexpr (TABLE) return P.table[leg].dev;
        else return P.legs[leg];
    };
    auto umap = [&](int leg) -> const CUtensorMap * {
        if constexpr (TABLE) return &P.table[leg].umap;
        else return &P.umap[leg];
    };
    auto mmap = [&](int leg) -> const CUtensorMap * {
        if constexpr (TABLE) return &P.table[leg].mmap;
        else return &P.mmap[leg];
    };
    for (int i = tid; i < 2 * kRows; i += TX * SEG) {  // identity rows; the margins are never written again
        fbuf[TX * SEG + i] = make_float4(0.f, 1.f, 0.f, 0.f);
    }
    auto at = [&](int g) -> int { return DIR == DIR_X ? line * P.sx + g : g * TX + line; };

    const int tpl = P.tiles_a * P.tiles_b;
    const int total = P.n_legs * tpl;

    auto issue = [&](int t, int s) {  // thread 0 only; the other threads read the tile's indices
        const int leg = t / tpl, r = t - leg * tpl, b = r / P.tiles_a, a = r - b * P.tiles_a;
        tinfo[s] = make_int4(leg, a, b, 0);
        const bool has_mask = legp(leg).mask != nullptr;
        mbar_expect_tx(&bar[s], P.tx_u + (has_mask ? P.tx_m : 0u));
        if (DIR == DIR_X) {
            const int y0 = 1 + a * TX, z = 1 + b;
            tma_load_4d(data(s), umap(leg), &bar[s], 0, 0, y0, z);
            if (has_mask) tma_load_3d(msk(s), mmap(leg), &bar[s], 0, y0, z);
        } else {
            const int x0 = a * TX, c = 1 + b;
            for (int q = 0; q < P.nload; ++q) {
                T *dst = data(s) + (size_t)q * (dbox / 4);
                if (DIR == DIR_Y) tma_load_3d(dst, umap(leg), &bar[s], x0, q * P.rows, c);
                else tma_load_3d(dst, umap(leg), &bar[s], x0, c, q * P.rows);
            }
            if (has_mask) tma_load_3d(msk(s), mmap(leg), &bar[s], 0, x0, c);
        }
    };

    int t = blockIdx.x, it = 0;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
        for (int k = 0; k + 1 < NS; ++k)
            if (t + k * (int)gridDim.x < total) issue(t + k * gridDim.x, k);
    }
    __syncthreads();  // barriers initialised, the first tile's indices visible

    // Fused source stage (x sweep).  The charge entries of an x tile are contiguous in the charge
    // list (lines ordered by z, then y), each a node (x | y << 16, FP32 qtilde).  They are read one
    // tile ahead, one or two per thread, and added to the tile's staged rows right after its copy
    // has landed, followed by one block barrier (tiles without charges skip both); the first tile
    // of a block is handled before the loop.
    constexpr int NT = TX * SEG;
    const bool fuse_src = DIR == DIR_X && (flags & FUSE_PRE_SRC) != 0;
    auto src_range = [&](int q, int &tb, int &te) {  // entry range of stage q's tile
        const int4 ti = tinfo[q];
        const LegDev &lg = legp(ti.x);
        const int y0 = 1 + ti.y * TX, y1 = min(y0 + TX, lg.ny - 1);  // lines y0 .. y1-1
        const int ln = (1 + ti.z) * lg.ny;
        tb = lg.line_begin[ln + y0];
        te = lg.line_begin[ln + y1 - 1] + lg.line_count[ln + y1 - 1];
    };
    auto src_apply = [&](int q, int2 v) {  // one entry into stage q's rows
        const int4 ti = tinfo[q];
        const int l = (v.x >> 16) - (1 + ti.y * TX), x = v.x & 0xffff;
        float &d = data(q)[l * P.sx + x];
        d = fmaf(legp(ti.x).srcf, __int_as_float(v.y), d);
    };
    if (fuse_src && t < total) {
        int tb, te;
        src_range(0, tb, te);
        const int2 *ent = legp(tinfo[0].x).ent_xq;
        const bool ok = mbar_wait_bounded(&bar[0], 0);
        if (ok)
            for (int e = tb + tid; e < te; e += NT) src_apply(0, ent[e]);
        else if (tid == 0)
            atomicExch(P.err, 1);
    }
    int2 sv[kSrcRegs];
    int cur_tb = 0, cur_te = 0;  // entries held in sv for the tile solved next (none for the first)
    for (; t < total; t += gridDim.x, ++it) {
        const int s = it % NS, sn = (it + 1) % NS;
        const int tn = t + gridDim.x;
        const int tq = t + (NS - 1) * gridDim.x;  // issued now into the stage stored last iteration
        if (tid == 0 && tq < total) {
            bulk_wait_read_all();
            issue(tq, (it + NS - 1) % NS);
        }
        const bool got = __syncthreads_and(mbar_wait_bounded(&bar[s], (it / NS) & 1));
        if (!got) {
            if (tid == 0) {
                atomicExch(P.err, 1);
                for (int k = 1; k < NS; ++k)  // the copies still in flight
                    if (t + k * (int)gridDim.x < total) mbar_wait_bounded(&bar[(it + k) % NS], ((it + k) / NS) & 1);
                bulk_wait_all();
            }
            return;
        }
        if (cur_te > cur_tb) {  // block-uniform: tau Q into this tile's rows, then a barrier
#pragma unroll
            for (int r = 0; r < kSrcRegs; ++r)
                if (cur_tb + tid + r * NT < cur_te) src_apply(s, sv[r]);
            const int2 *ent = legp(tinfo[s].x).ent_xq;
            for (int e = cur_tb + tid + kSrcRegs * NT; e < cur_te; e += NT) src_apply(s, ent[e]);
            __syncthreads();
        }

        const int4 ti = tinfo[s];
        const int leg = ti.x, a = ti.y, bb = ti.z;
        const LegDev &lg = legp(leg);
        const int ndir = DIR == DIR_X ? lg.nx : (DIR == DIR_Y ? lg.ny : lg.nz);
        const T rE0 = lg.rEf[0], rE1 = lg.rEf[1], rE2 = lg.rEf[2];
        const T nlq = lg.nl_qf, nlomq = lg.nl_omqf;
        const bool nl_on = lg.nl_on != 0;
        const bool pre_nl = (flags & FUSE_PRE_NL) && nl_on;
        const bool post_nl = (flags & FUSE_POST_NL) && nl_on;
        constexpr bool pre_cn = CN;
        T *D = data(s);
        const bool active = DIR == DIR_X ? (1 + a * TX + line <= lg.ny - 2)
                                         : (a * TX + line >= 1 && a * TX + line <= lg.nx - 2);
        const int r0 = seg * L;  // unknown index of the segment's first row (grid row r0 + 1)
        const int g0 = r0 + 1;
        // rows k < nrem are unknowns of this line; nrem <= 0 for an inactive line
        const int nrem = active ? ndir - 2 - r0 : 0;

        // node bits g0-1 .. g0+L of the line (bit j = node g0-1+j); no mask: all inside
        const uint32_t nb =
            lg.mask != nullptr ? segment_bits(msk(s) + line * P.mwpr, P.mwpr, g0) : 0xffffffffu;
        const uint32_t both = nb & (nb >> 1), any = nb | (nb >> 1);
        auto eh = [&](int j) -> T { return ((both >> j) & 1u) ? rE2 : (((any >> j) & 1u) ? rE1 : rE0); };
        // nodes that take the nonlinear flow: unknowns outside the molecule
        uint32_t flow = ~(nb >> 1) & (nrem >= 32 ? 0xffffffffu : (nrem > 0 ? (1u << nrem) - 1u : 0u));

        // LODIE2 stage S fused into the x sweep: tau Q at this thread's own charge nodes (each
        // thread scans its line's charge list, so no other thread's rows are touched)
        // the next tile's charge entries: range now, entries after the local elimination
        const bool src_next = fuse_src && tn < total;
        int ntb = 0, nte = 0;
        if (src_next) src_range(sn, ntb, nte);
        // row n-2 of the line: move its face coupling eps u_{n-1} to the right-hand side (after
        // the inflowing nonlinear stage, so the flow sees the bare node value)
        if (!pre_cn && nrem >= 1 && nrem <= L) {  // (Crank-Nicolson: in registers after the explicit half)
            const int k = nrem - 1;
            T v = D[at(g0 + k)];
            if (pre_nl && ((flow >> k) & 1u)) v = nl_flow_leg(v, nlq, nlomq);
            const T etop = ((both >> nrem) & 1u) ? rE2 : (((any >> nrem) & 1u) ? rE1 : rE0);
            D[at(g0 + k)] = v + etop * D[at(g0 + k + 1)];
            flow &= ~(1u << k);
        }

        T al[L], be[L], ga[L];
        T fa, fb, fc, fd, ea, eb, ec, ed;
        // The local elimination; FULL: every row of the segment is an unknown (no padding rows, no
        // cut coupling below the E row), so the per-row guards drop out.
        auto local = [&](auto full_tag) {
            constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
            for (int k = 0; k < L; ++k) al[k] = (FULL || k < nrem) ? D[at(g0 + k)] : T(0);
            if (pre_nl) {  // uniform over the tile: the flow code is not issued for other sweeps
#pragma unroll
                for (int k = 0; k < L; ++k)
                    if ((flow >> k) & 1u) al[k] = nl_flow_leg(al[k], nlq, nlomq);
            }
            if constexpr (pre_cn) {
                // the explicit half w_k + e_{k+1/2} (w_{k+1} - w_k) - e_{k-1/2} (w_k - w_{k-1}) from the
                // staged values (no thread writes the tile before the elimination's first barrier);
                // the neighbours beyond the segment and the top face come from shared memory
                T wprev = nrem > 0 ? D[at(g0 - 1)] : T(0);
                T wtop = nrem >= L ? D[at(g0 + L)] : T(0);
                if (pre_nl) {  // LODCN1: the neighbours take the inflowing nonlinear stage too
                    if (seg > 0 && nrem > 0 && !(nb & 1u)) wprev = nl_flow_leg(wprev, nlq, nlomq);
                    if (nrem > L && !((nb >> (L + 1)) & 1u)) wtop = nl_flow_leg(wtop, nlq, nlomq);
                }
                if (!FULL) {
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        if (k == nrem) al[k] = D[at(g0 + k)];  // the face u_{n-1} above the last unknown
                }
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const T w = al[k];
                    const T wn = k + 1 < L ? al[k + 1] : wtop;
                    const T v = w + eh(k + 1) * (wn - w) - eh(k) * (w - wprev);
                    wprev = w;
                    al[k] = (FULL || k < nrem) ? v : T(0);
                }
                if (nrem >= 1 && nrem <= L) {  // row n-2: its face coupling eps u_{n-1} to the right-hand side
                    const T etop = ((both >> nrem) & 1u) ? rE2 : (((any >> nrem) & 1u) ? rE1 : rE0);
                    const T face = D[at(g0 + nrem)];
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        if (k == nrem - 1) al[k] = fmaf(etop, face, al[k]);
                }
            }
            // row 0 (F) coefficients, then the forward elimination over rows 1 .. L-2 with x_0 = F
            const T em0 = eh(0), ep0 = eh(1);
            const T epc0 = (FULL || 1 < nrem) ? ep0 : T(0);
            // (alpha, beta) of a row travel as one packed pair: (ap, bp) = ((al_k, 0) + em (ap, bp)) m
            T em = ep0, h = T(1);
            unsigned long long ab[L];
            ab[0] = f2_pack(T(0), T(1));
#pragma unroll
            for (int k = 1; k <= L - 2; ++k) {
                const T ep = eh(k + 1);
                const T epc = (FULL || k + 1 < nrem) ? ep : T(0);  // row n-2, padding rows: no upward coupling
                const T m = fast_rcp(fmaf(em, h, T(1) + ep));
                const T g = epc * m;
                h = T(1) - g;
                ab[k] = f2_mul(f2_fma(f2_pack(em, em), ab[k - 1], f2_pack(al[k], T(0))), f2_pack(m, m));
                ga[k] = g;
                em = ep;
            }
            // back substitution of the x_k = al + be F + ga E representation
#pragma unroll
            for (int k = L - 3; k >= 1; --k) {
                const T g = ga[k];
                ab[k] = f2_fma(f2_pack(g, g), ab[k + 1], ab[k]);
                ga[k] = g * ga[k + 1];
            }
#pragma unroll
            for (int k = 1; k <= L - 2; ++k) f2_unpack(ab[k], al[k], be[k]);
            const T emL = em, epL = eh(L);
            const T epcL = L < nrem ? epL : T(0);
            fa = -em0;
            fb = T(1) + em0 + ep0 - epc0 * be[1];
            fc = -epc0 * ga[1];
            fd = fmaf(epc0, al[1], al[0]);
            ea = -emL * be[L - 2];
            eb = T(1) + emL + epL - emL * ga[L - 2];
            ec = -epcL;
            ed = fmaf(emL, al[L - 2], al[L - 1]);
        };
        const bool warp_full = __all_sync(0xffffffffu, nrem >= L);
        if (warp_full) local(std::true_type{});
        else local(std::false_type{});
        if (seg == 0) {  // row 1 couples to the face value u_0
            fd -= fa * D[at(0)];
            fa = T(0);
        }
        if (src_next) {
            const int2 *ent = legp(tinfo[sn].x).ent_xq;
#pragma unroll
            for (int r = 0; r < kSrcRegs; ++r) {
                const int e = ntb + tid + r * NT;
                sv[r] = e < nte ? ent[e] : make_int2(0, 0);
            }
        }
        T F_, E_;
        inner_ends<TX, SEG>(fa, fb, fc, fd, ea, eb, ec, ed, seg, line, fbuf, pbuf, ebuf, F_, E_);

#pragma unroll
        for (int k = 1; k < L - 1; ++k) al[k] = fmaf(ga[k], E_, fmaf(be[k], F_, al[k]));
        al[0] = F_;
        al[L - 1] = E_;
        if (post_nl) {  // the outflowing nonlinear stage on the unknowns outside the molecule
            const uint32_t post = ~(nb >> 1) & (nrem >= 32 ? 0xffffffffu : (nrem > 0 ? (1u << nrem) - 1u : 0u));
            if (nlq <= kNlSeriesMaxQ) {  // the leg's form chosen once, outside the row loop
#pragma unroll
                for (int k = 0; k < L; ++k)
                    if ((post >> k) & 1u) al[k] = nl_flow_tanh(al[k], 2.0f * nlq);
            } else {
#pragma unroll
                for (int k = 0; k < L; ++k)
                    if ((post >> k) & 1u) al[k] = nl_flow(al[k], nlq, nlomq);
            }
        }
        if (warp_full) {
#pragma unroll
            for (int k = 0; k < L; ++k) D[at(g0 + k)] = al[k];
        } else {
#pragma unroll
            for (int k = 0; k < L; ++k)
                if (k < nrem) D[at(g0 + k)] = al[k];
        }
        cur_tb = ntb;
        cur_te = nte;
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (DIR == DIR_X) {
                tma_store_4d(umap(leg), D, 0, 0, 1 + a * TX, 1 + bb);
            } else {
                const int x0 = a * TX, c = 1 + bb;
                for (int q = 0; q < P.nload; ++q) {
                    const T *src = D + (size_t)q * (dbox / 4);
                    if (DIR == DIR_Y) tma_store_3d(umap(leg), src, x0, q * P.rows, c);
                    else tma_store_3d(umap(leg), src, x0, c, q * P.rows);
                }
            }
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace npb
