// sweep_line.cuh -- FP32 LOD line solves, one grid line per pair of threads (solver kind 3).
//
// The implicit-Euler system of one LOD direction (Eqs. LODIE1_2-LODIE1_4, eps at half points by
// Eq. SpatialOperators) has n-2 unknowns per line, rows 1 .. N = n-2; the face values u_0 and
// u_{n-1} are Dirichlet data.  The paper solves each such line with the Thomas algorithm
// (Sec. 3.1).  Here the Thomas recurrence runs from both ends of the line at once: a tile of 32
// x-adjacent y or z lines sits in shared memory (bulk tensor copies, persistent blocks), and the
// block's two warps hold one thread per line each.
//   * lower thread: forward elimination of rows 1 .. p (p = ceil(N/2)), giving
//     v_k = dp_k + cp_k v_{k+1};
//   * upper thread: the same elimination from row N down to p + 1, giving
//     v_k = dq_k + aq_k v_{k-1};
//   * the two middle rows meet: v_p = (dp_p + cp_p dq_{p+1}) / (1 - cp_p aq_{p+1}), then
//     v_{p+1} = dq_{p+1} + aq_{p+1} v_p, and each thread back-substitutes its half.
// dp/dq overwrite the right-hand side in the tile, cp/aq go to a second shared array, so a line
// costs one read and one write of each row per pass and no block-wide reduction at all.  Every
// row matrix is strictly diagonally dominant, so neither direction needs pivoting.
//
// eps at a half point comes from the two node bits of the line-major mask (both inside: eps_in;
// one: the harmonic mean; none: eps_out).  A tile whose lines carry no inside node (every vacuum
// leg, and solvent tiles clear of the molecule) has constant coefficients; its multipliers
// m_j = 1/(1 + 2e - e cp_{j-1}) and cp_j = e m_j are the leg's table (computed once in FP64 on
// the host and rounded), and only the right-hand-side recurrence runs per row.
//
// Fused stage: LODIE2's nonlinear stage N (Eq. ana3) on the z sweep's results before the store.
#pragma once
#include "sweep_tma.cuh"

namespace npb {

constexpr int kLineThreads = 2 * kLineTX;  // two threads per line

// Shared bytes of one block: NS stages of (state boxes, mask box), the multiplier array, the meet
// exchange, barriers and tile indices.
__host__ __device__ __forceinline__ size_t line_smem_bytes(int ns, int rows, int nload, int mwpr) {
    const size_t data = (size_t)nload * tma_data_box_bytes(rows, kLineTX);
    const size_t mask = (size_t)kLineTX * mwpr * 4;
    return 128 + ns * (tma_align(data) + tma_align(mask)) + tma_align(data) + tma_align(2 * kLineTX * 8) + 128;
}

template <int DIR, bool TABLE, int NS>
__global__ void __launch_bounds__(kLineThreads) sweep_line_kernel(const __grid_constant__ TmaLaunch P, int flags) {
    static_assert(DIR == DIR_Y || DIR == DIR_Z, "lines along y or z");
    constexpr int TX = kLineTX;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool upper = tid >= 32;

    const size_t dbox = tma_data_box_bytes(P.rows, TX);
    const size_t data_b = (size_t)P.nload * dbox;
    const size_t mask_b = (size_t)TX * P.mwpr * 4;
    const size_t base = (128 - (smem_addr(smem_raw) & 127u)) & 127u;
    const size_t stage = tma_align(data_b) + tma_align(mask_b);
    auto data = [&](int s) { return reinterpret_cast<float *>(smem_raw + base + (size_t)s * stage); };
    auto msk = [&](int s) {
        return reinterpret_cast<const uint32_t *>(smem_raw + base + (size_t)s * stage + tma_align(data_b));
    };
    size_t off = base + NS * stage;
    float *C = reinterpret_cast<float *>(smem_raw + off);  // cp (lower rows) and aq (upper rows)
    off += tma_align(data_b);
    float2 *xbuf = reinterpret_cast<float2 *>(smem_raw + off);  // [lower | upper][line]
    off += tma_align(2 * TX * 8);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + off);
    int4 *tinfo = reinterpret_cast<int4 *>(bar + 4);

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

    const int tpl = P.tiles_a * P.tiles_b;
    const int total = P.n_legs * tpl;
    auto issue = [&](int t, int s) {  // thread 0 only
        const int leg = t / tpl, r = t - leg * tpl, b = r / P.tiles_a, a = r - b * P.tiles_a;
        tinfo[s] = make_int4(leg, a, b, 0);
        const bool has_mask = legp(leg).mask != nullptr;
        mbar_expect_tx(&bar[s], P.tx_u + (has_mask ? P.tx_m : 0u));
        const int x0 = a * TX, c = 1 + b;
        for (int q = 0; q < P.nload; ++q) {
            float *dst = data(s) + (size_t)q * (dbox / 4);
            if (DIR == DIR_Y) tma_load_3d(dst, umap(leg), &bar[s], x0, q * P.rows, c);
            else tma_load_3d(dst, umap(leg), &bar[s], x0, c, q * P.rows);
        }
        if (has_mask) tma_load_3d(const_cast<uint32_t *>(msk(s)), mmap(leg), &bar[s], 0, x0, c);
    };

    int t = blockIdx.x, it = 0;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
        for (int k = 0; k + 1 < NS; ++k)
            if (t + k * (int)gridDim.x < total) issue(t + k * gridDim.x, k);
    }
    __syncthreads();

    for (; t < total; t += gridDim.x, ++it) {
        const int s = it % NS;
        const int tq = t + (NS - 1) * gridDim.x;  // into the stage stored last iteration
        if (tid == 0 && tq < total) {
            bulk_wait_read_all();
            issue(tq, (it + NS - 1) % NS);
        }
        const bool got = __syncthreads_and(mbar_wait_bounded(&bar[s], (it / NS) & 1));
        if (!got) {
            if (tid == 0) {
                atomicExch(P.err, 1);
                for (int k = 1; k < NS; ++k)
                    if (t + k * (int)gridDim.x < total) mbar_wait_bounded(&bar[(it + k) % NS], ((it + k) / NS) & 1);
                bulk_wait_all();
            }
            return;
        }
        const int4 ti = tinfo[s];
        const int leg = ti.x, a = ti.y, bb = ti.z;
        const LegDev &lg = legp(leg);
        const int n = DIR == DIR_Y ? lg.ny : lg.nz;
        const int N = n - 2, p = (N + 1) >> 1;
        const int x = a * TX + lane;
        const bool active = x >= 1 && x <= lg.nx - 2;
        float *D = data(s) + lane;  // row g of this thread's line at D[g * TX]
        float *Cl = C + lane;
        const uint32_t *M = msk(s) + lane * P.mwpr;
        const bool has_mask = lg.mask != nullptr;
        // constant coefficients: no mask (vacuum), or no inside node on any line of the tile
        bool uni = !has_mask;
        if (has_mask) {
            uint32_t any = 0;
            if (active)
                for (int w = 0; w < P.mwpr; ++w) any |= M[w];
            uni = __reduce_or_sync(0xffffffffu, any) == 0u;  // the same lines in both warps
        }
        const float rE0 = lg.rEf[0], rE1 = lg.rEf[1], rE2 = lg.rEf[2];
        const bool post_nl = (flags & FUSE_POST_NL) && lg.nl_on;
        const float nlq = lg.nl_qf, nlomq = lg.nl_omqf;
        auto flow = [&](float v) { return nl_flow_leg(v, nlq, nlomq); };
        auto bit = [&](int g) -> uint32_t { return (M[g >> 5] >> (g & 31)) & 1u; };
        auto eh = [&](uint32_t b0, uint32_t b1) -> float { return (b0 & b1) ? rE2 : ((b0 | b1) ? rE1 : rE0); };
        const float2 *tab = lg.line_tab[DIR];  // (m_j, cp_j), j = 1 .. p, constant-coefficient lines
        const float ec = uni ? (has_mask ? rE0 : rE2) : 0.f;  // the constant r*eps of such a tile

        // ---- elimination towards the middle
        float dv = 0.f, cv = 0.f;  // (dp_p, cp_p) for the lower thread, (dq_{p+1}, aq_{p+1}) for the upper
        if (active) {
            if (!upper) {
                dv = D[0];  // u_0: the face term of row 1 enters as e_{1/2} dp_0
                if (uni) {
#pragma unroll 4
                    for (int k = 1; k <= p; ++k) {
                        const float2 f = __ldg(tab + k - 1);
                        dv = fmaf(ec, dv, D[k * TX]) * f.x;
                        D[k * TX] = dv;
                        cv = f.y;
                    }
                } else {
                    uint32_t w = M[0], b0 = w & 1u;
                    float el = 0.f;
                    {
                        const uint32_t b1 = (w >> 1) & 1u;
                        el = eh(b0, b1);
                        b0 = b1;
                    }
#pragma unroll 4
                    for (int k = 1; k <= p; ++k) {
                        const int g = k + 1;
                        if ((g & 31) == 0) w = M[g >> 5];
                        const uint32_t b1 = (w >> (g & 31)) & 1u;
                        const float er = eh(b0, b1);
                        b0 = b1;
                        const float m = fast_rcp(fmaf(-el, cv, 1.f + el + er));
                        dv = fmaf(el, dv, D[k * TX]) * m;
                        cv = er * m;
                        D[k * TX] = dv;
                        Cl[k * TX] = cv;
                        el = er;
                    }
                }
            } else {
                dv = D[(N + 1) * TX];  // u_{n-1}
                if (uni) {
#pragma unroll 4
                    for (int k = N; k > p; --k) {
                        const float2 f = __ldg(tab + (N - k));
                        dv = fmaf(ec, dv, D[k * TX]) * f.x;
                        D[k * TX] = dv;
                        cv = f.y;
                    }
                } else {
                    uint32_t b1 = bit(N + 1), b0 = bit(N);
                    float er = eh(b0, b1);
                    b1 = b0;
                    uint32_t w = M[(N - 1) >> 5];
#pragma unroll 4
                    for (int k = N; k > p; --k) {
                        const int g = k - 1;
                        if ((g & 31) == 31) w = M[g >> 5];
                        const uint32_t bl = (w >> (g & 31)) & 1u;
                        const float el = eh(bl, b1);
                        b1 = bl;
                        const float m = fast_rcp(fmaf(-er, cv, 1.f + el + er));
                        dv = fmaf(er, dv, D[k * TX]) * m;
                        cv = el * m;
                        D[k * TX] = dv;
                        Cl[k * TX] = cv;
                        er = el;
                    }
                }
            }
        }
        // ---- the two middle rows
        xbuf[tid] = make_float2(dv, cv);
        __syncthreads();
        const float2 lo = xbuf[lane], hi = xbuf[TX + lane];
        const float vp = (lo.x + lo.y * hi.x) / (1.f - lo.y * hi.y);
        // ---- back substitution (and the outflowing nonlinear stage)
        if (active) {
            if (!upper) {
                float v = vp;
                if (post_nl && (uni || !bit(p))) v = flow(v);
                D[p * TX] = v;
                v = vp;
                if (uni) {
#pragma unroll 4
                    for (int k = p - 1; k >= 1; --k) {
                        v = fmaf(__ldg(tab + k - 1).y, v, D[k * TX]);
                        D[k * TX] = post_nl ? flow(v) : v;
                    }
                } else if (!post_nl) {
#pragma unroll 4
                    for (int k = p - 1; k >= 1; --k) {
                        v = fmaf(Cl[k * TX], v, D[k * TX]);
                        D[k * TX] = v;
                    }
                } else {
                    uint32_t w = M[(p - 1) >> 5];
#pragma unroll 4
                    for (int k = p - 1; k >= 1; --k) {
                        if ((k & 31) == 31) w = M[k >> 5];
                        v = fmaf(Cl[k * TX], v, D[k * TX]);
                        D[k * TX] = ((w >> (k & 31)) & 1u) ? v : flow(v);
                    }
                }
            } else if (p < N) {
                float v = fmaf(hi.y, vp, hi.x);
                const float v1 = v;
                if (post_nl && (uni || !bit(p + 1))) v = flow(v);
                D[(p + 1) * TX] = v;
                v = v1;
                if (uni) {
#pragma unroll 4
                    for (int k = p + 2; k <= N; ++k) {
                        v = fmaf(__ldg(tab + (N - k)).y, v, D[k * TX]);
                        D[k * TX] = post_nl ? flow(v) : v;
                    }
                } else if (!post_nl) {
#pragma unroll 4
                    for (int k = p + 2; k <= N; ++k) {
                        v = fmaf(Cl[k * TX], v, D[k * TX]);
                        D[k * TX] = v;
                    }
                } else {
                    uint32_t w = M[(p + 2) >> 5];
#pragma unroll 4
                    for (int k = p + 2; k <= N; ++k) {
                        if ((k & 31) == 0) w = M[k >> 5];
                        v = fmaf(Cl[k * TX], v, D[k * TX]);
                        D[k * TX] = ((w >> (k & 31)) & 1u) ? v : flow(v);
                    }
                }
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const float *Ds = data(s);
            const int x0 = a * TX, c = 1 + bb;
            for (int q = 0; q < P.nload; ++q) {
                const float *src = Ds + (size_t)q * (dbox / 4);
                if (DIR == DIR_Y) tma_store_3d(umap(leg), src, x0, q * P.rows, c);
                else tma_store_3d(umap(leg), src, x0, c, q * P.rows);
            }
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace npb
