// sweep_kernel.cuh -- one batch of implicit-Euler LOD line solves (Eqs. LODIE1_2-LODIE1_4).
//
// For direction d every interior grid line carries the tridiagonal system
//     -r e_{-} v_{g-1} + (1 + r(e_{-} + e_{+})) v_g - r e_{+} v_{g+1} = w_g,   r = tau/h^2,
// with eps at the half points (Eq. SpatialOperators).  The two face nodes of the line,
// and the padding rows past its end, enter as identity rows, so they keep their values
// and their coupling to the first/last interior unknown is exact.
//
// Line solver (a Thomas / parallel-cyclic-reduction hybrid): a line of up to SEG*L rows
// is cut into SEG segments of L consecutive rows; one thread owns one segment in
// registers.
//   1. Local modified Thomas: for the rows strictly inside the segment,
//      x_k = alpha_k + beta_k F + gamma_k E, where F and E are the segment's own first
//      and last unknowns.
//   2. Substituting this into the segment's first and last rows gives two rows per
//      segment coupling (E_{s-1}, F_s, E_s) and (F_s, E_s, F_{s+1}).  Eliminating the
//      F's leaves one tridiagonal row per segment in the E's, solved by PCR across the
//      SEG threads of the line (log2 SEG rounds in shared memory).
//   3. F_s follows from E_{s-1}, E_s; every interior row is one fused multiply-add pair.
// The reduced systems are Schur complements of strictly diagonally dominant matrices,
// so no step needs pivoting.
//
// Thread block: TX lines x SEG segments (threadIdx.x = line, threadIdx.y = segment).
//   Y / Z sweeps: the TX lines are x-adjacent, so each row load/store of a warp is one
//   contiguous run of TX elements; no staging.
//   X sweep: the line runs along the unit-stride axis; the block stages its TX x-rows
//   with 16-byte vector loads into a shared tile whose row stride is odd (bank-conflict
//   free column access), and writes them back the same way.
// Fused stages: FUSE_PRE_SRC adds tau Q to the staged x-rows (LODIE2 stage S),
// FUSE_PRE_NL applies the nonlinear stage to the loaded x-rows (LODIE1 stage N),
// FUSE_POST_NL applies it before the z-sweep store (LODIE2 stage N).
#pragma once
#include "npb_internal.cuh"

namespace npb {

template <typename T>
__device__ __forceinline__ T fast_rcp(T x);
template <>
__device__ __forceinline__ float fast_rcp<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double fast_rcp<double>(double x) {
    return 1.0 / x;
}

// The nonlinear stage of Eq. (ana3) in tanh form: tanh(w'/2) = q tanh(w/2), q =
// exp(-kbar^2 tau).  With e = exp(-|w|), tanh(|w|/2) = (1-e)/(1+e) and
// 1 - tanh(|w'|/2) = (1-q) + 2 q e/(1+e); then |w'| = log1p(2 t'/(1 - t')).  No term
// overflows for any w and no step subtracts nearly equal numbers.
__device__ __forceinline__ double nl_flow(double w, double q, double omq) {
    const double aw = fabs(w);
    const double em = expm1(-aw);  // e - 1
    const double e = em + 1.0;
    const double inv = 1.0 / (1.0 + e);
    const double t = -q * em * inv;
    const double omt = omq + 2.0 * q * e * inv;
    return copysign(log1p(2.0 * t / omt), w);
}

// FP32 flavour on the special-function unit, three MUFU operations: with e = exp(-|w|),
// t = tanh(|w|/2) = (1-e)/(1+e) and t' = q t, |w'| = log((1+t')/(1-t')) and
//   (1+t')/(1-t') = ((1+q) + (1-q) e) / ((1-q) + (1+q) e),
// numerator and denominator both positive for every w (q < 1 wherever the flow runs).  The
// absolute error of w' stays at a few 1e-7 for every w (relative error is larger only where
// |w'| itself is below ~1e-3), well inside the mixed path's stated tolerance.
__device__ __forceinline__ float nl_flow(float w, float q, float omq) {
    const float e = __expf(-fabsf(w));
    const float opq = 1.0f + q;
    const float num = fmaf(omq, e, opq);
    const float den = fmaf(opq, e, omq);
    return copysignf(__logf(num * fast_rcp(den)), w);
}

// The nonlinear flow of Eq. (ana3) for small q = exp(-kbar^2 tau): with e = exp(-|w|),
// t = tanh(|w|/2) = (1 - e)/(1 + e), x = q t <= q, and |w'| = 2 atanh(x) = 2x (1 + x^2/3 + x^4/5
// + x^6/7 + ...), truncated after x^6/7 (relative error below x^8/9 <= 2e-11 for q <= 1/16): two
// special-function operations instead of three.
__device__ __forceinline__ float nl_flow_series(float w, float q) {
    const float e = __expf(-fabsf(w));
    const float t = (1.0f - e) * fast_rcp(1.0f + e);
    const float x = q * t, x2 = x * x;
    const float s = fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 7.0f, 0.2f), 1.0f / 3.0f), 1.0f);
    return copysignf(2.0f * x * s, w);
}

// q at or below which the series form is used (a leg-uniform choice).
constexpr float kNlSeriesMaxQ = 0.0625f;

// FP64 flavour of the series: t = -expm1(-|w|) / (2 + expm1(-|w|)) and 2 atanh(x) to x^15/15
// (relative truncation error below x^16/17 < 4e-21 for q <= 1/16), in place of log1p and one of the
// two divisions of nl_flow.
__device__ __forceinline__ double nl_flow_series(double w, double q) {
    const double em = expm1(-fabs(w));
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

__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 flow for small q from the hardware tanh: with t = tanh(w/2) and Q = 2q, x = Q t (|x| <= Q <=
// 1/8) and w' = 2 atanh(x/2) = x (1 + x^2/12 + x^4/80 + ...) = t (Q + (Q^3/12) t^2), truncated after
// x^2/12 (relative error below x^4/80 <= 3e-6).  tanh.approx.f32 carries a relative error near 2^-11,
// so |w'| is off by at most 5e-4 of itself: at most 1e-6 kT/e on a leg with tau = 10 (q = 2.2e-4)
// and 1.5e-5 kT/e with tau = 5 (q = 0.015), far inside the FP32 path's tolerance.  Q and Q^3/12 are
// the leg's (hoisted out of the row loops): one special-function operation and four others.
__device__ __forceinline__ float nl_flow_tanh(float w, float q2) {
    const float t = tanh_approx(0.5f * w);
    const float c3 = q2 * q2 * q2 * (1.0f / 12.0f);
    return t * fmaf(c3, t * t, q2);
}

// The nonlinear stage with the leg's q.  FP64: the series where q is small (it replaces log1p and a
// division), else the closed form.  FP32: the tanh form where q is small, else the closed form.
template <typename T>
__device__ __forceinline__ T nl_flow_leg(T w, T q, T omq);
template <>
__device__ __forceinline__ double nl_flow_leg<double>(double w, double q, double omq) {
    return q <= (double)kNlSeriesMaxQ ? nl_flow_series(w, q) : nl_flow(w, q, omq);
}
template <>
__device__ __forceinline__ float nl_flow_leg<float>(float w, float q, float omq) {
    return q <= kNlSeriesMaxQ ? nl_flow_tanh(w, 2.0f * q) : nl_flow(w, q, omq);
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};

constexpr int kMaxLineWords = 288;  // rows of the longest supported line

__host__ __device__ __forceinline__ int sweep_tile_stride(int nx, int vec) {
    const int nxv = (nx + vec - 1) / vec * vec;
    return nxv | 1;
}

template <typename T, int DIR, int TX, int SEG>
__host__ __device__ __forceinline__ size_t sweep_smem_bytes(int nx, int pitch) {
    size_t b = (size_t)(4 + 8 + 1) * TX * SEG * sizeof(T);
    if (DIR == DIR_X) {
        const int S = sweep_tile_stride(nx, Vec16<T>::n);
        b += (size_t)TX * S * sizeof(T);
        b = (b + 15) & ~(size_t)15;
        b += (size_t)2 * TX * mask_words_per_row(pitch) * sizeof(uint32_t);
    } else {
        b = (b + 15) & ~(size_t)15;
        b += (size_t)2 * kMaxLineWords * sizeof(uint32_t);  // the block's mask column (+ half bits)
    }
    return b;
}

// Local modified Thomas over the rows strictly inside one segment (rows 1 .. L-2), for
// row coefficients given by coef(k, a, b, c).  On return, for 1 <= k <= L-2:
//     x_k = al[k] + be[k] F + ga[k] E,
// and the segment's first and last rows have become (fa, fb, fc | fd) coupling
// (E_prev, F, E) and (ea, eb, ec | ed) coupling (F, E, F_next).
template <typename T, int L, typename Coef>
__device__ __forceinline__ void segment_reduce(T (&al)[L], T (&be)[L], T (&ga)[L], const Coef &coef, T &fa,
                                               T &fb, T &fc, T &fd, T &ea, T &eb, T &ec, T &ed) {
    T a0, b0, c0, aL, bL, cL;
    coef(0, a0, b0, c0);
    coef(L - 1, aL, bL, cL);
    if (L >= 3) {
        T cp = T(0), ap = T(0), bp = T(1);
#pragma unroll
        for (int k = 1; k <= L - 2; ++k) {
            T a, b, c;
            coef(k, a, b, c);
            const T m = fast_rcp(b - a * cp);
            cp = c * m;
            ap = (al[k] - a * ap) * m;
            bp = -a * bp * m;
            al[k] = ap;
            be[k] = bp;
            ga[k] = cp;
        }
        ga[L - 2] = -ga[L - 2];
#pragma unroll
        for (int k = L - 3; k >= 1; --k) {
            const T cpk = ga[k];
            al[k] = al[k] - cpk * al[k + 1];
            be[k] = be[k] - cpk * be[k + 1];
            ga[k] = -cpk * ga[k + 1];
        }
        fa = a0;
        fb = b0 + c0 * be[1];
        fc = c0 * ga[1];
        fd = al[0] - c0 * al[1];
        ea = aL * be[L - 2];
        eb = bL + aL * ga[L - 2];
        ec = cL;
        ed = al[L - 1] - aL * al[L - 2];
    } else {
        fa = a0; fb = b0; fc = c0; fd = al[0];
        ea = aL; eb = bL; ec = cL; ed = al[L - 1];
    }
}

// Reduced system of one line: the first/last rows of every segment (from segment_reduce)
// become one tridiagonal row per segment in the segment-end unknowns E after eliminating
// the F's; PCR across the SEG threads of the line solves it (log2 SEG rounds through
// shared memory), then F follows from E_prev and E.  Every thread of the block calls it
// (it synchronises the block).
template <typename T, int TX, int SEG>
__device__ __forceinline__ void segment_ends(T fa, T fb, T fc, T fd, T ea, T eb, T ec, T ed, int seg, int line,
                                             T *fbuf, T *pbuf, T *ebuf, T &F, T &E) {
    const int me = seg * TX + line;
    fbuf[4 * me + 0] = fa;
    fbuf[4 * me + 1] = fb;
    fbuf[4 * me + 2] = fc;
    fbuf[4 * me + 3] = fd;
    __syncthreads();
    const T ifb = fast_rcp(fb);
    T A = -ea * fa * ifb;
    T B = eb - ea * fc * ifb;
    T C = T(0);
    T D = ed - ea * fd * ifb;
    if (seg + 1 < SEG) {
        const int nx_ = (seg + 1) * TX + line;
        const T nfa = fbuf[4 * nx_ + 0], nfb = fbuf[4 * nx_ + 1], nfc = fbuf[4 * nx_ + 2],
                nfd = fbuf[4 * nx_ + 3];
        const T inb = fast_rcp(nfb);
        B -= ec * nfa * inb;
        C = -ec * nfc * inb;
        D -= ec * nfd * inb;
    }
#pragma unroll
    for (int st = 1, r = 0; st < SEG; st <<= 1, ++r) {
        T *buf = pbuf + (r & 1) * 4 * TX * SEG;
        buf[4 * me + 0] = A;
        buf[4 * me + 1] = B;
        buf[4 * me + 2] = C;
        buf[4 * me + 3] = D;
        __syncthreads();
        T la = T(0), lb = T(1), lc = T(0), ld = T(0), ua = T(0), ub = T(1), uc = T(0), ud = T(0);
        if (seg - st >= 0) {
            const int o = 4 * ((seg - st) * TX + line);
            la = buf[o]; lb = buf[o + 1]; lc = buf[o + 2]; ld = buf[o + 3];
        }
        if (seg + st < SEG) {
            const int o = 4 * ((seg + st) * TX + line);
            ua = buf[o]; ub = buf[o + 1]; uc = buf[o + 2]; ud = buf[o + 3];
        }
        const T k1 = A * fast_rcp(lb), k2 = C * fast_rcp(ub);
        B = B - k1 * lc - k2 * ua;
        D = D - k1 * ld - k2 * ud;
        A = -k1 * la;
        C = -k2 * uc;
    }
    E = D * fast_rcp(B);
    ebuf[me] = E;
    __syncthreads();
    const T Eprev = seg > 0 ? ebuf[(seg - 1) * TX + line] : T(0);
    F = (fd - fa * Eprev - fc * E) * ifb;
}

template <typename T, int DIR, int TX, int SEG, int L>
__global__ void __launch_bounds__(TX *SEG)
    sweep_kernel(const LegDev *__restrict__ legs, int flags) {
    static_assert(L >= 2 && L <= 30, "segment length: the row bits of a segment fit one word");
    static_assert((SEG & (SEG - 1)) == 0, "SEG must be a power of two");
    static_assert(32 % TX == 0, "TX divides a mask word");
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const LegDev *lg = legs + blockIdx.z;
    const int nx = lg->nx, ny = lg->ny, nz = lg->nz, pitch = lg->pitch;
    const int wpr = mask_words_per_row(pitch);
    const int line = threadIdx.x;
    const int seg = threadIdx.y;
    const int g0 = seg * L;
    const int tid = threadIdx.y * TX + threadIdx.x;
    constexpr int NTHR = TX * SEG;
    T *__restrict__ u = static_cast<T *>(lg->u);
    const uint32_t *__restrict__ mask = lg->mask;
    const int mid = lg->eps_mode;
    const uint32_t *__restrict__ half = lg->half[DIR];
    const int ndir = DIR == DIR_X ? nx : (DIR == DIR_Y ? ny : nz);
    const T rE0 = (T)lg->rE[0], rE1 = (T)lg->rE[1], rE2 = (T)lg->rE[2];
    const T nlq = (T)lg->nl_q, nlomq = (T)lg->nl_omq;
    const bool nl_on = lg->nl_on != 0;

    // ---- shared memory carve-up
    T *red = reinterpret_cast<T *>(smem_raw);          // 13 * TX * SEG
    T *fbuf = red;                                      // [SEG][TX][4]
    T *pbuf = red + 4 * TX * SEG;                       // [2][SEG][TX][4]
    T *ebuf = red + 12 * TX * SEG;                      // [SEG][TX]
    T *tile = red + 13 * TX * SEG;                      // DIR_X: [TX][S]
    const int S = sweep_tile_stride(nx, Vec16<T>::n);
    uint32_t *smask, *shalf;
    {
        size_t off = (size_t)13 * TX * SEG * sizeof(T) + (DIR == DIR_X ? (size_t)TX * S * sizeof(T) : 0);
        off = (off + 15) & ~(size_t)15;
        smask = reinterpret_cast<uint32_t *>(smem_raw + off);
        shalf = smask + (DIR == DIR_X ? TX * wpr : kMaxLineWords);
    }

    // ---- this thread's line
    // element offsets within one leg fit 32 bits: at most 288^3 elements per leg
    int lx = 0, ly = 0, lz = 0;
    bool active;
    int32_t base, stride;
    if (DIR == DIR_X) {
        ly = 1 + blockIdx.x * TX + line;
        lz = 1 + blockIdx.y;
        active = ly <= ny - 2;
        base = (lz * ny + ly) * pitch;
        stride = 1;
    } else if (DIR == DIR_Y) {
        lx = blockIdx.x * TX + line;
        lz = 1 + blockIdx.y;
        active = lx >= 1 && lx <= nx - 2;
        base = lz * ny * pitch + lx;
        stride = pitch;
    } else {
        lx = blockIdx.x * TX + line;
        ly = 1 + blockIdx.y;
        active = lx >= 1 && lx <= nx - 2;
        base = ly * pitch + lx;
        stride = ny * pitch;
    }

    // ---- stage what the block shares: X -> its TX x-rows and their mask words;
    //      Y/Z -> the mask word column of its TX x-adjacent lines (one word per row)
    if (DIR == DIR_X) {
        constexpr int VEC = Vec16<T>::n;
        using V = typename Vec16<T>::type;
        const int nvec = (nx + VEC - 1) / VEC;
        const int y0 = 1 + blockIdx.x * TX;
        for (int i = tid; i < TX * nvec; i += NTHR) {
            const int l = i / nvec, v = i - l * nvec;
            const int y = y0 + l;
            T vals[VEC];
            if (y <= ny - 2) {
                const V w = *reinterpret_cast<const V *>(u + (lz * ny + y) * pitch + v * VEC);
                *reinterpret_cast<V *>(vals) = w;
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) vals[e] = T(0);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) tile[l * S + v * VEC + e] = vals[e];
        }
        for (int i = tid; i < TX * wpr; i += NTHR) {
            const int l = i / wpr, w = i - l * wpr;
            const int y = y0 + l;
            const int32_t row = (lz * ny + (y <= ny - 2 ? y : 0)) * wpr + w;
            smask[i] = mask ? __ldg(mask + row) : 0xffffffffu;
            shalf[i] = (mid && half) ? __ldg(half + row) : 0u;
        }
        __syncthreads();
        if (flags & FUSE_PRE_SRC) {
            const double src = lg->src;
            for (int l = tid; l < TX; l += NTHR) {
                const int y = y0 + l;
                if (y > ny - 2) continue;
                const int ln = lz * ny + y;
                const int b = lg->line_begin[ln], c = lg->line_count[ln];
                for (int e = b; e < b + c; ++e)
                    tile[l * S + lg->ent_x[e]] += (T)(src * lg->ent_qt[e]);
            }
            __syncthreads();
        }
    } else {
        const int wcol = (blockIdx.x * TX) >> 5;
        for (int g = tid; g < ndir; g += NTHR) {
            const int32_t row = DIR == DIR_Y ? (lz * ny + g) : (g * ny + ly);
            smask[g] = mask ? __ldg(mask + row * wpr + wcol) : 0xffffffffu;
            shalf[g] = (mid && half) ? __ldg(half + row * wpr + wcol) : 0u;
        }
        __syncthreads();
    }

    // ---- node bits of rows g0-1 .. g0+L (bit k+1 <-> row g0+k) and half-point bits
    //      (bit k <-> the half point between rows g0+k-1 and g0+k)
    uint32_t nb = 0, hb = 0;
    if (active) {
#pragma unroll
        for (int k = -1; k <= L; ++k) {
            const int g = g0 + k;
            uint32_t bit = 1u, hbit = 0u;
            if (g >= 0 && g < ndir) {
                if (DIR == DIR_X) {
                    bit = (smask[line * wpr + (g >> 5)] >> (g & 31)) & 1u;
                    hbit = (shalf[line * wpr + (g >> 5)] >> (g & 31)) & 1u;
                } else {
                    bit = (smask[g] >> (lx & 31)) & 1u;
                    hbit = (shalf[g] >> (lx & 31)) & 1u;
                }
            }
            nb |= bit << (k + 1);
            hb |= hbit << (k + 1);
        }
    }
    // half point k lies between rows k-1 and k (k = 0..L): both ends inside / any end inside;
    // in the midpoint reading the half point's own location decides
    constexpr uint32_t kHalfMask = (L + 1 >= 32) ? 0xffffffffu : ((1u << (L + 1)) - 1u);
    constexpr uint32_t kNodeMask = (L + 2 >= 32) ? 0xffffffffu : ((1u << (L + 2)) - 1u);
    const uint32_t both = mid ? hb : (nb & (nb >> 1));
    const uint32_t any = mid ? hb : (nb | (nb >> 1));
    const bool interior_seg = g0 >= 1 && g0 + L - 1 <= ndir - 2;
    const bool all_in = (both & kHalfMask) == kHalfMask && (nb & kNodeMask) == kNodeMask;
    const bool all_out = (any & kHalfMask) == 0u && (nb & kNodeMask) == 0u;
    const bool uniform = interior_seg && (all_in || all_out);

    // ---- load the segment's right-hand sides
    T al[L], be[L], ga[L];
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int g = g0 + k;
        T v = T(0);
        if (active && g < ndir) {
            if (DIR == DIR_X) v = tile[line * S + g];
            else v = u[base + g * stride];
            if ((flags & FUSE_PRE_NL) && nl_on && g >= 1 && g <= ndir - 2 && ((nb >> (k + 1)) & 1u) == 0u)
                v = nl_flow_leg(v, nlq, nlomq);
        }
        al[k] = v;
    }

    // ---- 1. local modified Thomas (constant coefficients on uniform interior segments)
    T fa, fb, fc, fd, ea, eb, ec, ed;
    if (uniform) {
        const T e = all_in ? rE2 : rE0;
        const T ca = -e, cb = T(1) + e + e;
        auto coef = [&](int, T &a, T &b, T &c) {
            a = ca;
            b = cb;
            c = ca;
        };
        segment_reduce<T, L>(al, be, ga, coef, fa, fb, fc, fd, ea, eb, ec, ed);
    } else {
        auto eh = [&](int k) -> T {
            return ((both >> k) & 1u) ? rE2 : (((any >> k) & 1u) ? rE1 : rE0);
        };
        auto coef = [&](int k, T &a, T &b, T &c) {
            const int g = g0 + k;
            if (g < 1 || g > ndir - 2) {
                a = T(0);
                b = T(1);
                c = T(0);
                return;
            }
            const T em = eh(k), ep = eh(k + 1);
            a = -em;
            c = -ep;
            b = T(1) + em + ep;
        };
        segment_reduce<T, L>(al, be, ga, coef, fa, fb, fc, fd, ea, eb, ec, ed);
    }

    // ---- 2. reduced system in the segment ends
    T F, E;
    segment_ends<T, TX, SEG>(fa, fb, fc, fd, ea, eb, ec, ed, seg, line, fbuf, pbuf, ebuf, F, E);

    // ---- 3. expand and store the interior rows
    if (DIR == DIR_X) {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const int g = g0 + k;
            if (active && g >= 1 && g <= ndir - 2) {
                const T x = k == 0 ? F : (k == L - 1 ? E : al[k] + be[k] * F + ga[k] * E);
                tile[line * S + g] = x;
            }
        }
        __syncthreads();
        constexpr int VEC = Vec16<T>::n;
        using V = typename Vec16<T>::type;
        const int nvec = (nx + VEC - 1) / VEC;
        const int y0 = 1 + blockIdx.x * TX;
        for (int i = tid; i < TX * nvec; i += NTHR) {
            const int l = i / nvec, v = i - l * nvec;
            const int y = y0 + l;
            if (y > ny - 2) continue;
            T vals[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) vals[e] = tile[l * S + v * VEC + e];
            *reinterpret_cast<V *>(u + (lz * ny + y) * pitch + v * VEC) =
                *reinterpret_cast<const V *>(vals);
        }
    } else if (active) {
        const bool post_nl = (flags & FUSE_POST_NL) && nl_on;
        if (uniform) {
            const bool nl_all = post_nl && all_out;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                T x = k == 0 ? F : (k == L - 1 ? E : al[k] + be[k] * F + ga[k] * E);
                if (nl_all) x = nl_flow_leg(x, nlq, nlomq);
                u[base + (g0 + k) * stride] = x;
            }
        } else {
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const int g = g0 + k;
                if (g >= 1 && g <= ndir - 2) {
                    T x = k == 0 ? F : (k == L - 1 ? E : al[k] + be[k] * F + ga[k] * E);
                    if (post_nl && ((nb >> (k + 1)) & 1u) == 0u) x = nl_flow_leg(x, nlq, nlomq);
                    u[base + g * stride] = x;
                }
            }
        }
    }
}

}  // namespace npb
