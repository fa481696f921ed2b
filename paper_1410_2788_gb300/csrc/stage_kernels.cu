// stage_kernels.cu -- stand-alone LOD stages and the energy reduction.
//
//   nonlinear   Eq. (ana3) at every interior solvent node (used on its own by the
//               row-level interface; inside a step it is fused into a sweep)
//   source      Eq. (LODIE1_5): u += tau Q over the charge entries (LODIE1 ends on it)
//   add         u += tau rho over the interior, for a dense source density (Sec. 4.1)
//   energy      Eqs. (rich) and (deltaG3): the FP64 charge-weighted sum over the
//               charge nodes of the Richardson-combined solvent minus vacuum potential,
//               reduced in a fixed order (each block a fixed chunk of the entries and a fixed
//               tree; the last block to finish sums the block partials in a fixed tree), so the
//               value does not depend on scheduling.
#include <algorithm>
#include <type_traits>

#include "npb_internal.cuh"
#include "setup_kernels.cuh"
#include "sweep_kernel.cuh"

namespace npb {

template <typename T>
__global__ void k_nonlinear(const LegDev *__restrict__ legs) {
    const LegDev *lg = legs + blockIdx.z;
    if (!lg->nl_on) return;
    T *u = static_cast<T *>(lg->u);
    const int nx = lg->nx, ny = lg->ny, nz = lg->nz, pitch = lg->pitch, wpr = mask_words_per_row(pitch);
    const int64_t total = (int64_t)(nz - 2) * (ny - 2) * (nx - 2);
    const T q = (T)lg->nl_q, omq = (T)lg->nl_omq;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(p % (nx - 2));
        const int64_t r = p / (nx - 2);
        const int j = 1 + (int)(r % (ny - 2)), k = 1 + (int)(r / (ny - 2));
        const int64_t row = (int64_t)k * ny + j;
        const bool inside = lg->mask ? ((lg->mask[row * wpr + (i >> 5)] >> (i & 31)) & 1u) : true;
        if (!inside) u[row * pitch + i] = nl_flow(u[row * pitch + i], q, omq);
    }
}

template <typename T>
__global__ void k_source(const LegDev *__restrict__ legs) {
    const LegDev *lg = legs + blockIdx.z;
    T *u = static_cast<T *>(lg->u);
    const int ny = lg->ny, nz = lg->nz;
    const int n_lines = ny * nz;
    for (int ln = blockIdx.x * blockDim.x + threadIdx.x; ln < n_lines; ln += gridDim.x * blockDim.x) {
        const int y = ln % ny, z = ln / ny;
        if (y < 1 || y > ny - 2 || z < 1 || z > nz - 2) continue;
        const int b = lg->line_begin[ln], c = lg->line_count[ln];
        for (int e = b; e < b + c; ++e) {
            const int64_t p = (int64_t)ln * lg->pitch + lg->ent_x[e];
            u[p] += (T)(lg->src * lg->ent_qt[e]);
        }
    }
}

cudaError_t launch_nonlinear(int prec, const LegDev *legs, int n_legs, int nx, int ny, int nz,
                             cudaStream_t st) {
    dim3 grid(152 * 4, 1, n_legs);
    if (prec == 0) k_nonlinear<double><<<grid, 256, 0, st>>>(legs);
    else k_nonlinear<float><<<grid, 256, 0, st>>>(legs);
    return cudaGetLastError();
}

// The explicit half step of the Crank-Nicolson sweeps (Eqs. LODCN1_2-4) along `dir`, in place:
// w_g + e_{g+1/2} (w_{g+1} - w_g) - e_{g-1/2} (w_g - w_{g-1}) at every interior node, one thread per
// line carrying the old w_{g-1}.  e = the leg's r*eps/2 at the half point (the legs of a CN scheme
// carry the halved values): harmonic from the two node bits, midpoint from the half-point bit.
template <typename T>
__global__ void k_cn_explicit(const LegDev *__restrict__ legs, int dir) {
    const LegDev *lg = legs + blockIdx.z;
    T *u = static_cast<T *>(lg->u);
    const int nx = lg->nx, ny = lg->ny, nz = lg->nz, pitch = lg->pitch;
    const int wpr = mask_words_per_row(pitch);
    const int n[3] = {nx, ny, nz};
    const int ndir = n[dir];
    const int a_n = dir == 0 ? ny - 2 : nx - 2, b_n = dir == 2 ? ny - 2 : nz - 2;
    const int64_t step = dir == 0 ? 1 : (dir == 1 ? (int64_t)pitch : (int64_t)pitch * ny);
    const T rE0 = (T)lg->rE[0], rE1 = (T)lg->rE[1], rE2 = (T)lg->rE[2];
    const uint32_t *mask = lg->mask;
    const uint32_t *half = lg->eps_mode ? lg->half[dir] : nullptr;
    const int64_t lines = (int64_t)a_n * b_n;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < lines; l += (int64_t)gridDim.x * blockDim.x) {
        const int a = 1 + (int)(l % a_n), b = 1 + (int)(l / a_n);
        int c[3];
        c[dir] = 0;
        if (dir == 0) { c[1] = a; c[2] = b; }
        else if (dir == 1) { c[0] = a; c[2] = b; }
        else { c[0] = a; c[1] = b; }
        const int64_t base = ((int64_t)c[2] * ny + c[1]) * pitch + c[0];
        auto node_in = [&](int g) -> uint32_t {  // node mask bit of node g of the line
            if (!mask) return 1u;
            int q[3] = {c[0], c[1], c[2]};
            q[dir] = g;
            return (mask[((int64_t)q[2] * ny + q[1]) * wpr + (q[0] >> 5)] >> (q[0] & 31)) & 1u;
        };
        auto e_half = [&](int g, uint32_t in_g, uint32_t in_g1) -> T {  // half point g + 1/2
            if (half) {
                int q[3] = {c[0], c[1], c[2]};
                q[dir] = g;
                return ((half[((int64_t)q[2] * ny + q[1]) * wpr + (q[0] >> 5)] >> (q[0] & 31)) & 1u) ? rE2 : rE0;
            }
            return (in_g & in_g1) ? rE2 : ((in_g | in_g1) ? rE1 : rE0);
        };
        T w_prev = u[base], w = u[base + step];
        uint32_t in_prev = node_in(0), in_cur = node_in(1);
        T em = e_half(0, in_prev, in_cur);
        for (int g = 1; g <= ndir - 2; ++g) {
            const T w_next = u[base + (int64_t)(g + 1) * step];
            const uint32_t in_next = node_in(g + 1);
            const T ep = e_half(g, in_cur, in_next);
            u[base + (int64_t)g * step] = w + ep * (w_next - w) - em * (w - w_prev);
            w_prev = w;
            w = w_next;
            in_cur = in_next;
            em = ep;
        }
    }
}

// One explicit Euler step of Eq. (TimeDepNPB) (the reference the pseudo-time schemes are compared
// with): out = w + sum_d [e_+ (w_+ - w) + e_- (w_- - w)] - tau kbar^2 sinh(w) (solvent nodes outside
// the molecule) at interior nodes, e = r*eps at the half points (the leg's rE, r = tau/h^2, from the
// node or half-point bits); faces copied.  The source tau*rho is added by the source stage after it.
template <typename T>
__global__ void k_euler_step(const LegDev *__restrict__ lgp, const T *__restrict__ in, T *__restrict__ out,
                             double tau_kappa2) {
    const LegDev &lg = *lgp;
    const int nx = lg.nx, ny = lg.ny, nz = lg.nz, pitch = lg.pitch;
    const int wpr = mask_words_per_row(pitch);
    const T rE0 = (T)lg.rE[0], rE1 = (T)lg.rE[1], rE2 = (T)lg.rE[2];
    const int64_t total = (int64_t)nz * ny * pitch;
    auto node_in = [&](int i, int j, int k) -> uint32_t {
        if (!lg.mask) return 1u;
        return (lg.mask[((int64_t)k * ny + j) * wpr + (i >> 5)] >> (i & 31)) & 1u;
    };
    auto e_half = [&](int d, int i, int j, int k) -> T {  // half point (i,j,k) + 1/2 along d
        if (lg.eps_mode && lg.half[d])
            return ((lg.half[d][((int64_t)k * ny + j) * wpr + (i >> 5)] >> (i & 31)) & 1u) ? rE2 : rE0;
        const uint32_t a = node_in(i, j, k);
        const uint32_t b = node_in(i + (d == 0), j + (d == 1), k + (d == 2));
        return (a & b) ? rE2 : ((a | b) ? rE1 : rE0);
    };
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % pitch);
        const int64_t r = p / pitch;
        const int j = (int)(r % ny), k = (int)(r / ny);
        if (i >= nx) continue;
        const T w = in[p];
        if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1) {
            out[p] = w;
            continue;
        }
        const int64_t sy = pitch, sz = (int64_t)pitch * ny;
        T lap = e_half(0, i, j, k) * (in[p + 1] - w) + e_half(0, i - 1, j, k) * (in[p - 1] - w);
        lap += e_half(1, i, j, k) * (in[p + sy] - w) + e_half(1, i, j - 1, k) * (in[p - sy] - w);
        lap += e_half(2, i, j, k) * (in[p + sz] - w) + e_half(2, i, j, k - 1) * (in[p - sz] - w);
        T v = w + lap;
        if (lg.nl_on && !node_in(i, j, k)) v -= (T)tau_kappa2 * sinh(w);
        out[p] = v;
    }
}

cudaError_t launch_euler_step(int prec, const LegDev *leg, const void *in, void *out, const GridGeom &g,
                              double tau_kappa2, cudaStream_t st) {
    const int64_t total = (int64_t)g.nz * g.ny * g.pitch;
    const int b = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (prec == 0) k_euler_step<double><<<b, 256, 0, st>>>(leg, (const double *)in, (double *)out, tau_kappa2);
    else k_euler_step<float><<<b, 256, 0, st>>>(leg, (const float *)in, (float *)out, tau_kappa2);
    return cudaGetLastError();
}

cudaError_t launch_cn_explicit(int prec, const LegDev *legs, int n_legs, int dir, cudaStream_t st) {
    dim3 grid(152 * 4, 1, n_legs);
    if (prec == 0) k_cn_explicit<double><<<grid, 128, 0, st>>>(legs, dir);
    else k_cn_explicit<float><<<grid, 128, 0, st>>>(legs, dir);
    return cudaGetLastError();
}

// u += scale * s at interior nodes, s a padded array in the state's layout (a dense source
// tau*rho; scale = 1, or an additive scheme's share for one direction).
template <typename T>
__global__ void k_add_interior(GridGeom g, const T *__restrict__ src, T *__restrict__ u, T scale) {
    const int64_t total = (int64_t)g.nz * g.ny * g.pitch;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.pitch);
        const int64_t r = p / g.pitch;
        const int j = (int)(r % g.ny), k = (int)(r / g.ny);
        if (i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2 && k >= 1 && k <= g.nz - 2) u[p] += scale * src[p];
    }
}

cudaError_t launch_add_interior(int prec, const GridGeom &g, const void *src, void *u, double scale,
                                cudaStream_t st) {
    const int64_t total = (int64_t)g.nz * g.ny * g.pitch;
    const int t = 256;
    const int b = (int)std::min<int64_t>((total + t - 1) / t, 152 * 16);
    if (prec == 0) k_add_interior<double><<<b, t, 0, st>>>(g, (const double *)src, (double *)u, scale);
    else k_add_interior<float><<<b, t, 0, st>>>(g, (const float *)src, (float *)u, (float)scale);
    return cudaGetLastError();
}

// The combine stage of an additive step (Eqs. AOS1_5 / AOS2_5 and MAOS1_5) at interior nodes, summed
// in the order W, x, y, z.  AOS: W is the exact flow of alpha w_t = -4 kbar^2 sinh w over tau from
// the saved U^n at solvent nodes (tanh(W/2) = exp(-4 kbar^2 tau) tanh(U^n/2)), U^n elsewhere.
template <typename T>
__global__ void k_additive_combine(const AddLeg *__restrict__ legs, int aos) {
    const AddLeg *lg = legs + blockIdx.z;
    T *u = static_cast<T *>(lg->u);
    const T *a = static_cast<const T *>(lg->a), *b = static_cast<const T *>(lg->b),
            *c = static_cast<const T *>(lg->c);
    const int nx = lg->nx, ny = lg->ny, nz = lg->nz, pitch = lg->pitch, wpr = mask_words_per_row(pitch);
    const int64_t total = (int64_t)(nz - 2) * (ny - 2) * (nx - 2);
    const T q = (T)lg->q, omq = (T)lg->omq;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(p % (nx - 2));
        const int64_t r = p / (nx - 2);
        const int j = 1 + (int)(r % (ny - 2)), k = 1 + (int)(r / (ny - 2));
        const int64_t row = (int64_t)k * ny + j, e = row * pitch + i;
        if (aos) {
            T w = a[e];
            const bool inside = lg->mask ? ((lg->mask[row * wpr + (i >> 5)] >> (i & 31)) & 1u) : true;
            if (lg->nl_on && !inside) w = nl_flow(w, q, omq);
            u[e] = (((w + b[e]) + c[e]) + u[e]) * (T)0.25;
        } else {
            u[e] = ((b[e] + c[e]) + u[e]) / (T)3;
        }
    }
}

cudaError_t launch_additive_combine(int prec, const AddLeg *legs, int n_legs, int aos, cudaStream_t st) {
    dim3 grid(152 * 4, 1, n_legs);
    if (prec == 0) k_additive_combine<double><<<grid, 256, 0, st>>>(legs, aos);
    else k_additive_combine<float><<<grid, 256, 0, st>>>(legs, aos);
    return cudaGetLastError();
}

// S at the charge entries: thread e adds tau Q at entry e of every leg (the entries are distinct
// nodes, so the adds do not collide).  Legs go in groups of four, every load of a group issued
// before its stores, so that the four read-modify-writes overlap (the compiler cannot move a load
// of one leg's state above a store to another's).  FP32 legs add srcf * qtilde in FP32, as the x
// sweeps' fused source does.
template <typename T>
__global__ void k_source_entries(const LegDev *__restrict__ legs, int n_legs) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    for (int j0 = 0; j0 < n_legs; j0 += 4) {
        T *u[4], v[4], a[4];
        int64_t p[4];
        bool ok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = j0 + k;
            ok[k] = j < n_legs && e < *legs[j].n_ent;
            if (ok[k]) {
                const LegDev &lg = legs[j];
                u[k] = static_cast<T *>(lg.u);
                p[k] = lg.ent_off[e];
                if constexpr (std::is_same<T, float>::value) a[k] = __int_as_float(lg.ent_xq[e].y);
                else a[k] = lg.src * lg.ent_qt[e];
                v[k] = u[k][p[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (ok[k]) {
                if constexpr (std::is_same<T, float>::value) u[k][p[k]] = fmaf(legs[j0 + k].srcf, a[k], v[k]);
                else u[k][p[k]] = v[k] + a[k];
            }
    }
}

// The same adds for the legs of one grid from kernel parameters: the entry count, the entry's
// offset and charge are independent loads, then the legs' state loads, then their stores, so a
// thread waits on two memory round trips.  Threads past the count (but inside the allocated slots)
// load an entry slot and stop before touching a state.
template <typename T>
__global__ void k_source_legs(const SourceLegs S) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S.n_slots) return;
    const int n = *S.n_ent;
    const int64_t p = S.ent_off[e];
    T a;
    if constexpr (std::is_same<T, float>::value) a = __int_as_float(S.ent_xq[e].y);
    else a = S.ent_qt[e];
    if (e >= n) return;
    T v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < S.n_legs) v[k] = static_cast<T *>(S.u[k])[p];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < S.n_legs) {
            if constexpr (std::is_same<T, float>::value) static_cast<T *>(S.u[k])[p] = fmaf(S.srcf[k], a, v[k]);
            else static_cast<T *>(S.u[k])[p] = v[k] + S.src[k] * a;
        }
}

cudaError_t launch_source_legs(int prec, const SourceLegs &S, cudaStream_t st) {
    if (S.n_legs < 0 || S.n_legs > 4) return cudaErrorInvalidValue;
    if (S.n_legs == 0 || S.n_slots < 1) return cudaSuccess;
    const unsigned blocks = (unsigned)((S.n_slots + 255) / 256);
    if (prec == 0) k_source_legs<double><<<blocks, 256, 0, st>>>(S);
    else k_source_legs<float><<<blocks, 256, 0, st>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_source_entries(int prec, const LegDev *legs, int n_legs, int n_ent_max, cudaStream_t st) {
    if (n_legs < 1 || n_ent_max < 1) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_ent_max + 255) / 256);
    if (prec == 0) k_source_entries<double><<<blocks, 256, 0, st>>>(legs, n_legs);
    else k_source_entries<float><<<blocks, 256, 0, st>>>(legs, n_legs);
    return cudaGetLastError();
}

cudaError_t launch_source(int prec, const LegDev *legs, int n_legs, int ny, int nz, cudaStream_t st) {
    dim3 grid((ny * nz + 255) / 256, 1, n_legs);
    if (prec == 0) k_source<double><<<grid, 256, 0, st>>>(legs);
    else k_source<float><<<grid, 256, 0, st>>>(legs);
    return cudaGetLastError();
}

// dG = 1/2 kT sum_e qt_e * combo_e, combo = (2 s_half - s_tau) - (2 v_half - v_tau) with
// Richardson, else s_tau - v_tau.  legs: s_tau, s_half, v_tau, v_half element pointers.
template <typename T>
__global__ void k_energy(const T *__restrict__ s_tau, const T *__restrict__ s_half,
                         const T *__restrict__ v_tau, const T *__restrict__ v_half,
                         const int64_t *__restrict__ off, const double *__restrict__ qt,
                         const int32_t *__restrict__ n_ent_dev, int richardson, const double *__restrict__ vac,
                         double *__restrict__ part, unsigned int *__restrict__ done, double *__restrict__ out) {
    __shared__ double red[kEnergyThreads];
    __shared__ bool last;
    const int n_ent = *n_ent_dev;
    const int chunk = (n_ent + (int)gridDim.x - 1) / (int)gridDim.x;
    const int e0 = blockIdx.x * chunk, e1 = min(n_ent, e0 + chunk);
    double acc = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t p = off[e];
        double us, uv;
        if (richardson) {
            us = 2.0 * (double)s_half[p] - (double)s_tau[p];
            uv = vac ? 0.0 : 2.0 * (double)v_half[p] - (double)v_tau[p];
        } else {
            us = (double)s_tau[p];
            uv = vac ? 0.0 : (double)v_tau[p];
        }
        if (vac) uv = vac[p];  // Eq. (deltaG2): phi_0^FFT in place of the vacuum legs
        acc += qt[e] * (us - uv);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the block that finished last sums the block partials, in the same tree whichever block it is
    __threadfence();
    red[threadIdx.x] = (int)threadIdx.x < (int)gridDim.x ? reinterpret_cast<volatile double *>(part)[threadIdx.x] : 0.0;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = 0.5 * kKT * red[0];
        *done = 0u;  // ready for the next launch
    }
}

cudaError_t launch_energy(int prec, const void *s_tau, const void *s_half, const void *v_tau,
                          const void *v_half, const int64_t *off, const double *qt, const int32_t *n_ent,
                          int richardson, const double *vac, double *part, double *out, cudaStream_t st) {
    unsigned int *done = reinterpret_cast<unsigned int *>(part + kEnergyBlocks);
    if (prec == 0)
        k_energy<double><<<kEnergyBlocks, kEnergyThreads, 0, st>>>((const double *)s_tau, (const double *)s_half,
                                                                   (const double *)v_tau, (const double *)v_half,
                                                                   off, qt, n_ent, richardson, vac, part, done, out);
    else
        k_energy<float><<<kEnergyBlocks, kEnergyThreads, 0, st>>>((const float *)s_tau, (const float *)s_half,
                                                                  (const float *)v_tau, (const float *)v_half, off,
                                                                  qt, n_ent, richardson, vac, part, done, out);
    return cudaGetLastError();
}

// The recovered potential phi_m^LOD + phi_0^LOD - phi_0^FFT (Sec. 5.3), each LOD potential
// Richardson-combined when `richardson`, as dense FP64 (x fastest).
template <typename T>
__global__ void k_recover(GridGeom g, const T *__restrict__ s_tau, const T *__restrict__ s_half,
                          const T *__restrict__ v_tau, const T *__restrict__ v_half, const double *__restrict__ vac,
                          int richardson, double *__restrict__ out) {
    const int64_t total = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.nx);
        const int64_t r = q / g.nx;
        const int64_t p = r * g.pitch + i;
        const double us = richardson ? 2.0 * (double)s_half[p] - (double)s_tau[p] : (double)s_tau[p];
        const double uv = richardson ? 2.0 * (double)v_half[p] - (double)v_tau[p] : (double)v_tau[p];
        out[q] = us + uv - vac[p];
    }
}

cudaError_t launch_recover(int prec, const GridGeom &g, const void *s_tau, const void *s_half, const void *v_tau,
                           const void *v_half, const double *vac, int richardson, double *out, cudaStream_t st) {
    const int64_t total = (int64_t)g.nx * g.ny * g.nz;
    const int b = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (prec == 0)
        k_recover<double><<<b, 256, 0, st>>>(g, (const double *)s_tau, (const double *)s_half, (const double *)v_tau,
                                             (const double *)v_half, vac, richardson, out);
    else
        k_recover<float><<<b, 256, 0, st>>>(g, (const float *)s_tau, (const float *)s_half, (const float *)v_tau,
                                            (const float *)v_half, vac, richardson, out);
    return cudaGetLastError();
}

}  // namespace npb
