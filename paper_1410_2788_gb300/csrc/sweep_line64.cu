// sweep_line64.cu -- FP64 LOD line solves, one grid line per pair of threads, with the Thomas
// multipliers computed once per leg (solver kind 3 for the plain FP64 path).
//
// The implicit-Euler system of one LOD direction (Eqs. LODIE1_2-LODIE1_4, eps at half points) is
// solved by the Thomas recurrence of Sec. 3.1, from both ends of the line at once: the lower thread
// eliminates rows 1 .. p downwards (p = ceil(N/2), N = n-2), the upper thread rows N .. p+1 upwards,
// the two middle rows are solved together, and each thread back-substitutes its half.  The
// multipliers m_k = 1/(1 + e_lo + e_hi - e_lo cp_{k-1}) (downwards; mirrored upwards) depend only on
// eps and r = tau/h^2, not on u, so they are computed once per leg and direction (k_line64_factors)
// and read back at every step: a row then costs two FP64 multiply-adds on the way down and two on the
// way up, instead of a division and the segmented elimination's bookkeeping.  GB300's FP64 units run
// at about 1/64 of its FP32 rate, so the plain FP64 path is bound by them; fewer FP64 operations per
// node is what speeds it up.  u is read and written in place in global memory: for y and z the 32
// lines of a warp are x-adjacent (coalesced rows); for x, whose lanes each walk their own row, the
// rows go through shared memory in chunks copied by whole warps (k_line64_sweep_x).
//
// Fused stages (flags): S (LODIE2) and N (LODIE1) on the x sweep's loaded rows, N (LODIE2) on the z
// sweep's results.
#include <algorithm>
#include <type_traits>

#include "exp_table.cuh"
#include "npb_internal.cuh"
#include "sweep_kernel.cuh"

namespace npb {

constexpr int kL64Lines = 32;
constexpr int kL64Chunk = 8;  // rows whose loads are issued together

struct L64Line {
    int64_t base, step;    // element of row g: base + g * step
    int64_t mbase;         // first mask word of the line
    bool active;
};

template <int DIR>
__device__ __forceinline__ L64Line l64_line(const LegDev &lg, int a, int c, int lane) {
    L64Line L;
    const int64_t pitch = lg.pitch, ny = lg.ny;
    if (DIR == DIR_X) {  // line (y, z), y = 1 + a*32 + lane, z = c
        const int y = 1 + a * kL64Lines + lane;
        L.active = y <= lg.ny - 2;
        L.base = ((int64_t)c * ny + y) * pitch;
        L.step = 1;
        L.mbase = ((int64_t)c * ny + y) * mask_words_per_row(lg.pitch);
    } else {  // line (x, c): x = a*32 + lane; c = z (y sweep) or y (z sweep)
        const int x = a * kL64Lines + lane;
        L.active = x >= 1 && x <= lg.nx - 2;
        if (DIR == DIR_Y) {
            L.base = (int64_t)c * ny * pitch + x;
            L.step = pitch;
            L.mbase = ((int64_t)c * lg.nx + x) * line_words(lg.ny);
        } else {
            L.base = (int64_t)c * pitch + x;
            L.step = ny * pitch;
            L.mbase = ((int64_t)c * lg.nx + x) * line_words(lg.nz);
        }
    }
    return L;
}

// r*eps at the half point g + 1/2 from the node bits of g and g + 1.
__device__ __forceinline__ double l64_e(const double *rE, uint32_t b0, uint32_t b1) {
    return (b0 & b1) ? rE[2] : ((b0 | b1) ? rE[1] : rE[0]);
}

// Node bit g of a line (1 = inside); no mask: every node inside (the vacuum legs' constant eps_in).
struct L64Bits {
    const uint32_t *w;
    int cur;
    uint32_t word;
    __device__ __forceinline__ uint32_t operator()(int g) {
        if (!w) return 1u;
        if ((g >> 5) != cur) {
            cur = g >> 5;
            word = w[cur];
        }
        return (word >> (g & 31)) & 1u;
    }
};

// Multipliers of every line of leg blockIdx.z along DIR into lg.fac[DIR].
template <int DIR>
__global__ void __launch_bounds__(2 * kL64Lines) k_line64_factors(const LegDev *__restrict__ legs, int tiles_a) {
    const LegDev &lg = legs[blockIdx.z];
    const int lane = threadIdx.x & 31;
    const bool upper = threadIdx.x >= 32;
    const L64Line L = l64_line<DIR>(lg, blockIdx.x, 1 + blockIdx.y, lane);
    if (!L.active) return;
    const int n = DIR == DIR_X ? lg.nx : (DIR == DIR_Y ? lg.ny : lg.nz);
    const int N = n - 2, p = (N + 1) >> 1;
    double *f = lg.fac[DIR] + L.base;
    L64Bits bit{lg.lmask[DIR] ? lg.lmask[DIR] + L.mbase : nullptr, -1, 0u};
    if (!upper) {
        double cp = 0.0, el = l64_e(lg.rE, bit(0), bit(1));
        for (int k = 1; k <= p; ++k) {
            const double er = l64_e(lg.rE, bit(k), bit(k + 1));
            const double m = 1.0 / (1.0 + el + er - el * cp);
            f[k * L.step] = m;
            cp = er * m;
            el = er;
        }
    } else {
        double aq = 0.0, er = l64_e(lg.rE, bit(N), bit(N + 1));
        for (int k = N; k > p; --k) {
            const double el = l64_e(lg.rE, bit(k - 1), bit(k));
            const double m = 1.0 / (1.0 + el + er - er * aq);
            f[k * L.step] = m;
            aq = el * m;
            er = el;
        }
    }
}

// The FP64 series flow of Eq. (ana3) (nl_flow_series) with exp(-|w|) - 1 from the block's exp table:
// t = -expm1(-|w|) / (2 + expm1(-|w|)), x = q t, |w'| = 2 atanh(x) to x^15/15.  The table's rounding
// moves t by at most 2e-14 of itself, and |w'| <= 2q, so w' is off by less than 1e-15 absolute.
__device__ __forceinline__ double nl_flow_series_tab(double w, double q, const double *T) {
    const double em = expm1_nonpos(-fabs(w), T);
    const double x = q * (-em / (2.0 + em)), x2 = x * x;
    double s = 1.0 / 15.0;
    s = fma(s, x2, 1.0 / 13.0);
    s = fma(s, x2, 1.0 / 11.0);
    s = fma(s, x2, 1.0 / 9.0);
    s = fma(s, x2, 1.0 / 7.0);
    s = fma(s, x2, 1.0 / 5.0);
    s = fma(s, x2, 1.0 / 3.0);
    s = fma(s, x2, 1.0);
    return copysign(2.0 * x * s, w);
}

// The y and z sweeps (x: k_line64_sweep_x below), reading and writing u in global memory; the 32
// lines of a warp are x-adjacent, so every row access is coalesced.
template <int DIR>
__global__ void __launch_bounds__(2 * kL64Lines) k_line64_sweep(const LegDev *__restrict__ legs, int flags) {
    static_assert(DIR == DIR_Y || DIR == DIR_Z, "the x sweep is k_line64_sweep_x");
    __shared__ double2 xbuf[2 * kL64Lines];
    __shared__ double T[32];  // exp table of the z sweep's nonlinear stage (visible after the xbuf barrier)
    if (DIR == DIR_Z) exp_table_init(T);
    const LegDev &lg = legs[blockIdx.z];
    const int lane = threadIdx.x & 31;
    const bool upper = threadIdx.x >= 32;
    const int c = 1 + blockIdx.y;
    const L64Line L = l64_line<DIR>(lg, blockIdx.x, c, lane);
    const int n = DIR == DIR_Y ? lg.ny : lg.nz;
    const int N = n - 2, p = (N + 1) >> 1;
    double *u = static_cast<double *>(lg.u) + L.base;
    const double *f = lg.fac[DIR] + L.base;
    const int64_t st = L.step;
    L64Bits bit{lg.lmask[DIR] ? lg.lmask[DIR] + L.mbase : nullptr, -1, 0u};
    const bool post_nl = DIR == DIR_Z && (flags & FUSE_POST_NL) && lg.nl_on != 0;

    double dv = 0.0, cv = 0.0;  // (dp_p, cp_p) of the lower thread, (dq_{p+1}, aq_{p+1}) of the upper
    if (L.active) {
        // the rows this thread owns: 1 .. p (lower) or p+1 .. N (upper), in chunks of kL64Chunk:
        // every chunk's loads are issued before its dependent recurrence, so the latency overlaps
        if (!upper) {
            dv = u[0];  // the face u_0 enters as e_{1/2} dp_0
            double el = l64_e(lg.rE, bit(0), bit(1));
            for (int k0 = 1; k0 <= p; k0 += kL64Chunk) {
                const int nk = min(kL64Chunk, p - k0 + 1);
                double w[kL64Chunk], m[kL64Chunk];
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        w[j] = u[(k0 + j) * st];
                        m[j] = f[(k0 + j) * st];
                    }
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 + j;
                        const double er = l64_e(lg.rE, bit(k), bit(k + 1));
                        dv = fma(el, dv, w[j]) * m[j];
                        u[k * st] = dv;
                        cv = er * m[j];
                        el = er;
                    }
            }
        } else {
            dv = u[(N + 1) * st];  // u_{n-1}
            double er = l64_e(lg.rE, bit(N), bit(N + 1));
            for (int k0 = N; k0 > p; k0 -= kL64Chunk) {
                const int nk = min(kL64Chunk, k0 - p);
                double w[kL64Chunk], m[kL64Chunk];
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        w[j] = u[(k0 - j) * st];
                        m[j] = f[(k0 - j) * st];
                    }
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 - j;
                        const double el = l64_e(lg.rE, bit(k - 1), bit(k));
                        dv = fma(er, dv, w[j]) * m[j];
                        u[k * st] = dv;
                        cv = el * m[j];
                        er = el;
                    }
            }
        }
    }
    xbuf[threadIdx.x] = make_double2(dv, cv);
    __syncthreads();
    if (!L.active) return;
    const double2 lo = xbuf[lane], hi = xbuf[kL64Lines + lane];
    const double vp = (lo.x + lo.y * hi.x) / (1.0 - lo.y * hi.y);
    // back substitution; the leg's flow form (series or closed) is chosen once, outside the rows
    auto back = [&](auto series_tag) {
        constexpr bool SERIES = decltype(series_tag)::value;
        auto flow_out = [&](double x) {
            return SERIES ? nl_flow_series_tab(x, lg.nl_q, T) : nl_flow(x, lg.nl_q, lg.nl_omq);
        };
        if (!upper) {
            double v = vp;
            u[p * st] = (post_nl && !bit(p)) ? flow_out(v) : v;
            for (int k0 = p - 1; k0 >= 1; k0 -= kL64Chunk) {
                const int nk = min(kL64Chunk, k0);
                double w[kL64Chunk], m[kL64Chunk];
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        w[j] = u[(k0 - j) * st];
                        m[j] = f[(k0 - j) * st];
                    }
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 - j;
                        const double er = l64_e(lg.rE, bit(k), bit(k + 1));
                        v = fma(er * m[j], v, w[j]);
                        u[k * st] = (post_nl && !bit(k)) ? flow_out(v) : v;
                    }
            }
        } else if (p < N) {
            double v = fma(hi.y, vp, hi.x);
            u[(p + 1) * st] = (post_nl && !bit(p + 1)) ? flow_out(v) : v;
            for (int k0 = p + 2; k0 <= N; k0 += kL64Chunk) {
                const int nk = min(kL64Chunk, N - k0 + 1);
                double w[kL64Chunk], m[kL64Chunk];
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        w[j] = u[(k0 + j) * st];
                        m[j] = f[(k0 + j) * st];
                    }
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 + j;
                        const double el = l64_e(lg.rE, bit(k - 1), bit(k));
                        v = fma(el * m[j], v, w[j]);
                        u[k * st] = (post_nl && !bit(k)) ? flow_out(v) : v;
                    }
            }
        }
    };
    if (post_nl && lg.nl_q <= (double)kNlSeriesMaxQ) back(std::true_type{});
    else back(std::false_type{});
}

// The x sweep with its rows staged through shared memory: each lane of an x sweep walks its own
// row, so the generic kernel's loads touch 32 rows per warp instruction (latency-bound, ncu: FP64
// pipe 34%, 46 long-scoreboard stalls per issue).  Here a warp copies a chunk of kL64Chunk rows of
// all its 32 lines with four 64-byte row pieces per load instruction, the lanes run the recurrence
// on the staged values, and the warp copies the results back the same way.  Same arithmetic in the
// same order as the generic kernel (bit-identical results).  Every lane of the block takes part in
// the copies (lines past the grid's last y line are skipped); only active lanes compute.
__global__ void __launch_bounds__(2 * kL64Lines) k_line64_sweep_x(const LegDev *__restrict__ legs, int flags) {
    __shared__ double2 xbuf[2 * kL64Lines];
    __shared__ double sw[2][kL64Lines][kL64Chunk + 1], sm[2][kL64Lines][kL64Chunk + 1];
    const LegDev &lg = legs[blockIdx.z];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const bool upper = wp == 1;
    const int c = 1 + blockIdx.y;
    const L64Line L = l64_line<DIR_X>(lg, blockIdx.x, c, lane);
    const int N = lg.nx - 2, p = (N + 1) >> 1;
    double *const ul = static_cast<double *>(lg.u) + L.base;  // this lane's row (active lanes only)
    L64Bits bit{lg.lmask[DIR_X] ? lg.lmask[DIR_X] + L.mbase : nullptr, -1, 0u};
    const bool nl_on = lg.nl_on != 0;
    const bool pre_nl = (flags & FUSE_PRE_NL) && nl_on;
    const bool pre_src = (flags & FUSE_PRE_SRC) != 0;

    // rows [lo, lo + nk) of the warp's 32 lines: lane (e, lsub) copies element e of line 4 it + lsub
    double *const ug = static_cast<double *>(lg.u);
    const double *const fg = lg.fac[DIR_X];
    const int y0 = 1 + blockIdx.x * kL64Lines, e = lane & 7, lsub = lane >> 3;
    auto at = [&](int li, int row) { return ((int64_t)c * lg.ny + (y0 + li)) * lg.pitch + row; };
    auto stage = [&](int lo, int nk) {
#pragma unroll
        for (int it = 0; it < kL64Lines / 4; ++it) {
            const int li = 4 * it + lsub;
            if (e < nk && y0 + li <= lg.ny - 2) {
                const int64_t a = at(li, lo + e);
                sw[wp][li][e] = ug[a];
                sm[wp][li][e] = fg[a];
            }
        }
        __syncwarp();
    };
    auto flush = [&](int lo, int nk) {
        __syncwarp();
#pragma unroll
        for (int it = 0; it < kL64Lines / 4; ++it) {
            const int li = 4 * it + lsub;
            if (e < nk && y0 + li <= lg.ny - 2) ug[at(li, lo + e)] = sw[wp][li][e];
        }
        __syncwarp();
    };
    double *const w = sw[wp][lane], *const m = sm[wp][lane];

    double dv = 0.0, cv = 0.0;  // (dp_p, cp_p) of the lower lane, (dq_{p+1}, aq_{p+1}) of the upper
    if (L.active) {
        const int r0 = upper ? p + 1 : 1, r1 = upper ? N : p;
        if (pre_nl)  // LODIE1's N at the solvent nodes outside the molecule, before the solve
            for (int k = r0; k <= r1; ++k)
                if (!bit(k)) ul[k] = nl_flow_leg(ul[k], lg.nl_q, lg.nl_omq);
        if (pre_src) {  // LODIE2's S: tau Q at this half's charge nodes of the line (y, z = c)
            const int ln = c * lg.ny + (1 + blockIdx.x * kL64Lines + lane);
            const int b = lg.line_begin[ln], en = b + lg.line_count[ln];
            for (int q = b; q < en; ++q) {
                const int x = lg.ent_x[q];
                if (x >= r0 && x <= r1) ul[x] += lg.src * lg.ent_qt[q];
            }
        }
    }
    __syncwarp();  // the stages' writes before the copies read the rows
    if (!upper) {
        double el = 0.0;
        if (L.active) {
            dv = ul[0];  // the face u_0 enters as e_{1/2} dp_0
            el = l64_e(lg.rE, bit(0), bit(1));
        }
        for (int k0 = 1; k0 <= p; k0 += kL64Chunk) {
            const int nk = min(kL64Chunk, p - k0 + 1);
            stage(k0, nk);
            if (L.active) {
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 + j;
                        const double er = l64_e(lg.rE, bit(k), bit(k + 1));
                        dv = fma(el, dv, w[j]) * m[j];
                        w[j] = dv;
                        cv = er * m[j];
                        el = er;
                    }
            }
            flush(k0, nk);
        }
    } else {
        double er = 0.0;
        if (L.active) {
            dv = ul[N + 1];  // u_{n-1}
            er = l64_e(lg.rE, bit(N), bit(N + 1));
        }
        for (int k0 = N; k0 > p; k0 -= kL64Chunk) {
            const int nk = min(kL64Chunk, k0 - p), lo = k0 - nk + 1;
            stage(lo, nk);
            if (L.active) {
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 - j;
                        const double el = l64_e(lg.rE, bit(k - 1), bit(k));
                        dv = fma(er, dv, w[k - lo]) * m[k - lo];
                        w[k - lo] = dv;
                        cv = el * m[k - lo];
                        er = el;
                    }
            }
            flush(lo, nk);
        }
    }
    xbuf[threadIdx.x] = make_double2(dv, cv);
    __syncthreads();
    const double2 lo2 = xbuf[lane], hi2 = xbuf[kL64Lines + lane];
    const double vp = (lo2.x + lo2.y * hi2.x) / (1.0 - lo2.y * hi2.y);
    if (!upper) {
        double v = vp;
        if (L.active) ul[p] = v;
        for (int k0 = p - 1; k0 >= 1; k0 -= kL64Chunk) {
            const int nk = min(kL64Chunk, k0), lo = k0 - nk + 1;
            stage(lo, nk);
            if (L.active) {
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 - j;
                        const double er = l64_e(lg.rE, bit(k), bit(k + 1));
                        v = fma(er * m[k - lo], v, w[k - lo]);
                        w[k - lo] = v;
                    }
            }
            flush(lo, nk);
        }
    } else if (p < N) {
        double v = fma(hi2.y, vp, hi2.x);
        if (L.active) ul[p + 1] = v;
        for (int k0 = p + 2; k0 <= N; k0 += kL64Chunk) {
            const int nk = min(kL64Chunk, N - k0 + 1);
            stage(k0, nk);
            if (L.active) {
#pragma unroll
                for (int j = 0; j < kL64Chunk; ++j)
                    if (j < nk) {
                        const int k = k0 + j;
                        const double el = l64_e(lg.rE, bit(k - 1), bit(k));
                        v = fma(el * m[j], v, w[j]);
                        w[j] = v;
                    }
            }
            flush(k0, nk);
        }
    }
}

static dim3 l64_grid(int dir, int n_legs, int nx, int ny, int nz) {
    if (dir == DIR_X) return dim3((ny - 2 + kL64Lines - 1) / kL64Lines, nz - 2, n_legs);
    return dim3((nx - 1 + kL64Lines - 1) / kL64Lines, dir == DIR_Y ? nz - 2 : ny - 2, n_legs);
}

cudaError_t launch_line64_factors(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, cudaStream_t st) {
    const dim3 g = l64_grid(dir, n_legs, nx, ny, nz);
    if (dir == DIR_X) k_line64_factors<DIR_X><<<g, 2 * kL64Lines, 0, st>>>(legs, g.x);
    else if (dir == DIR_Y) k_line64_factors<DIR_Y><<<g, 2 * kL64Lines, 0, st>>>(legs, g.x);
    else k_line64_factors<DIR_Z><<<g, 2 * kL64Lines, 0, st>>>(legs, g.x);
    return cudaGetLastError();
}

cudaError_t launch_sweep_line64(int dir, const LegDev *legs, int n_legs, int nx, int ny, int nz, int flags,
                                cudaStream_t st) {
    const dim3 g = l64_grid(dir, n_legs, nx, ny, nz);
    if (dir == DIR_X) k_line64_sweep_x<<<g, 2 * kL64Lines, 0, st>>>(legs, flags);
    else if (dir == DIR_Y) k_line64_sweep<DIR_Y><<<g, 2 * kL64Lines, 0, st>>>(legs, flags);
    else k_line64_sweep<DIR_Z><<<g, 2 * kL64Lines, 0, st>>>(legs, flags);
    return cudaGetLastError();
}

}  // namespace npb
