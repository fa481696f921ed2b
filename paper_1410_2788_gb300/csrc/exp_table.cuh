// exp_table.cuh -- exp and expm1 of non-positive FP64 arguments by Tang's table-driven method
// (P. T. P. Tang, ACM TOMS 15(2), 1989), with a 32-entry table T[j] = 2^(j/32) that the calling block
// fills (exp_table_init, then a block barrier before the first use):
//   x = n ln2/32 + r, |r| <= ln2/64, n = 32 m + j,  exp(x) = 2^m 2^(j/32) exp(r),
// ln2/32 split in two doubles (the second 7.2e-19) so that r carries no error from the reduction, and
// exp(r) - 1 by its Taylor series to r^6/720 (truncation below r^7/5040 < 4e-18).
#pragma once

namespace npb {

__device__ __forceinline__ void exp_table_init(double *T) {
    if (threadIdx.x < 32) T[threadIdx.x] = exp2((double)threadIdx.x / 32.0);
}

// n = round(x 32/ln2) and p = exp(r) - 1 for the reduced argument r.
__device__ __forceinline__ int exp_reduce(double x, double &p) {
    constexpr double kInvL = 46.16624130844683;     // 32 / ln 2
    constexpr double kL1 = 0.02166084939249829;     // ln 2 / 32, leading part
    constexpr double kL2 = 7.247021293269686e-19;   // ln 2 / 32 - kL1
    constexpr double kShift = 6755399441055744.0;   // 1.5 * 2^52: rounds to an integer in the low bits
    const double t = fma(x, kInvL, kShift);
    const int n = __double2loint(t);
    const double nd = t - kShift;
    double r = fma(-nd, kL1, x);
    r = fma(-nd, kL2, r);
    double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    p = r * q;
    return n;
}

// v * 2^m by the exponent field (v normal, the result normal).
__device__ __forceinline__ double exp_scale(double v, int m) {
    return __hiloint2double(__double2hiint(v) + (int)((unsigned)m << 20), __double2loint(v));
}

// exp(x), x <= 0; 0 below -700.  Within about 1.5 ulp.
__device__ __forceinline__ double exp_nonpos(double x, const double *T) {
    if (x < -700.0) return 0.0;
    double p;
    const int n = exp_reduce(x, p);
    const double tj = T[n & 31];
    return exp_scale(fma(tj, p, tj), n >> 5);
}

// exp(x) - 1, x <= 0; -1 below -700.  For m = 0 (n = 0, j = 0) it is p itself; for m = -1 the
// difference 2^(j/32) - 2 is exact, so nothing cancels; below, exp(x) < 1/2.  The table entries'
// rounding (half an ulp of 2^(j/32)) bounds the error by about 1.2e-16 absolute, at most 2e-14 of
// |exp(x) - 1| where |x| >= ln2/64.
__device__ __forceinline__ double expm1_nonpos(double x, const double *T) {
    if (x < -700.0) return -1.0;
    double p;
    const int n = exp_reduce(x, p);
    const int m = n >> 5;
    const double tj = T[n & 31];
    if (m == 0) return p;
    if (m == -1) return 0.5 * fma(tj, p, tj - 2.0);
    return exp_scale(fma(tj, p, tj), m) - 1.0;
}

}  // namespace npb
