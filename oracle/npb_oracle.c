/*
 * npb_oracle.c -- plain FP64 CPU oracle for the pseudo-transient LOD solver of the
 * time-dependent nonlinear Poisson-Boltzmann (NPB) equation of Wilson & Zhao,
 * "Unconditionally stable time splitting methods for the electrostatic analysis of
 * solvated biomolecules" (arXiv 1410.2788).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference that
 * the CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * Every routine is a direct transcription of one passage of the paper:
 *   or_mask_vdw          Sec. 2.1 / Sec. 3.1 (eps is eps_m on/inside the surface)
 *   or_charge_spread     Eq. (RhoEq) spread by trilinear interpolation (Sec. 3.1)
 *   or_boundary          Eq. (BoundaryCond), Dirichlet data on the cubic box
 *   or_eps_half_*        eps at half points used by Eq. (SpatialOperators)
 *   or_sweep             Eqs. (LODIE1_2)-(LODIE1_4): (1 - dt/alpha delta^2) v = w,
 *                        one tridiagonal system per grid line, Thomas algorithm
 *   or_sweep_cn          Eqs. (LODCN1_2)-(LODCN1_4): (1 - dt/(2 alpha) delta^2) v =
 *                        (1 + dt/(2 alpha) delta^2) w, the same solve on the explicit half step
 *   or_nonlinear         Eq. (ana3), the analytic solution of alpha w_t = -kbar^2 sinh w
 *   or_source            Eq. (LODIE1_5), u += dt/alpha * Q
 *   or_lod_run           LODIE1 (N,X,Y,Z,S), LODIE2 (S,X,Y,Z,N), LODCN1, LODCN2 steps (Sec. 3.1)
 *   or_additive_run      AOSIE1/2, AOSCN1/2 (Sec. 3.2) and MAOSIE/MAOSCN (Sec. 3.3) steps: parts
 *                        advanced side by side from one state and averaged
 *   or_euler_run         explicit Euler steps of Eq. (TimeDepNPB) (Sec. 5.2 reference)
 *
 * Layout: node (i,j,k) of an nx*ny*nz grid is stored at u[(k*ny + j)*nx + i];
 * i runs along x.  Faces (any index 0 or n-1) hold Dirichlet values that no stage
 * changes (Sec. 3.1: the same boundary values for w, v, p, q and u).
 *
 * Compile with -ffp-contract=off so that results do not depend on whether the host
 * compiler fuses multiply-adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int or_get_threads(void) {
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

static inline int64_t idx3(int i, int j, int k, int nx, int ny) {
    return ((int64_t)k * ny + j) * nx + i;
}

/* Node inside the molecule (Omega_m) iff it lies on or inside some atom's ball.
 * The loop visits, for every atom, the nodes of its bounding box only; every node of
 * the ball is in that box. */
void or_mask_vdw(int nx, int ny, int nz, double h, const double *origin, int n_atoms,
                 const double *xyz, const double *radius, uint8_t *in_mol) {
    memset(in_mol, 0, (size_t)nx * ny * nz);
    for (int a = 0; a < n_atoms; ++a) {
        const double rx = xyz[3 * a], ry = xyz[3 * a + 1], rz = xyz[3 * a + 2];
        const double rho = radius[a];
        int lo[3], hi[3];
        const double c[3] = {rx, ry, rz};
        const int n[3] = {nx, ny, nz};
        for (int d = 0; d < 3; ++d) {
            lo[d] = (int)floor((c[d] - rho - origin[d]) / h) - 1;
            hi[d] = (int)ceil((c[d] + rho - origin[d]) / h) + 1;
            if (lo[d] < 0) lo[d] = 0;
            if (hi[d] > n[d] - 1) hi[d] = n[d] - 1;
        }
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    const double dx = (origin[0] + i * h) - rx;
                    const double dy = (origin[1] + j * h) - ry;
                    const double dz = (origin[2] + k * h) - rz;
                    if (dx * dx + dy * dy + dz * dz <= rho * rho)
                        in_mol[idx3(i, j, k, nx, ny)] = 1;
                }
    }
}

/* Trilinear distribution of the point charges onto the 8 surrounding nodes
 * (Sec. 3.1, Q(x_i, y_j, z_k)).  qt receives charge in e_c per node.
 * Returns 0, or -1 if some atom's 8-node stencil touches a face. */
int or_charge_spread(int nx, int ny, int nz, double h, const double *origin, int n_atoms,
                     const double *xyz, const double *q, double *qt) {
    memset(qt, 0, sizeof(double) * (size_t)nx * ny * nz);
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < n_atoms; ++a) {
        int i0[3];
        double f[3];
        for (int d = 0; d < 3; ++d) {
            const double s = (xyz[3 * a + d] - origin[d]) / h;
            i0[d] = (int)floor(s);
            f[d] = s - i0[d];
            if (i0[d] < 1 || i0[d] + 1 > n[d] - 2) return -1;
        }
        for (int c = 0; c < 8; ++c) {
            const int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
            const double w = (ox ? f[0] : 1.0 - f[0]) * (oy ? f[1] : 1.0 - f[1]) *
                             (oz ? f[2] : 1.0 - f[2]);
            qt[idx3(i0[0] + ox, i0[1] + oy, i0[2] + oz, nx, ny)] += q[a] * w;
        }
    }
    return 0;
}

/* Eq. (BoundaryCond): u = C sum_i q_i exp(-kbar |r - r_i| / sqrt(eps)) / (eps |r - r_i|)
 * on every face node; C = e_c^2/(k_B T) in A.  Interior values are left untouched. */
void or_boundary(int nx, int ny, int nz, double h, const double *origin, int n_atoms,
                 const double *xyz, const double *q, double eps, double kbar, double C,
                 double *u) {
    const double sq = sqrt(eps);
#pragma omp parallel for collapse(2) schedule(dynamic, 4) num_threads(g_threads)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (!(i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1))
                    continue;
                const double x = origin[0] + i * h, y = origin[1] + j * h, z = origin[2] + k * h;
                double s = 0.0;
                for (int a = 0; a < n_atoms; ++a) {
                    const double dx = x - xyz[3 * a], dy = y - xyz[3 * a + 1], dz = z - xyz[3 * a + 2];
                    const double d = sqrt(dx * dx + dy * dy + dz * dz);
                    s += q[a] * exp(-kbar * d / sq) / (eps * d);
                }
                u[idx3(i, j, k, nx, ny)] = C * s;
            }
}

/* eps at the half points (i+1/2, j, k), (i, j+1/2, k), (i, j, k+1/2) as the harmonic
 * mean of the two node values.  e?[p] refers to the half point just above node p. */
void or_eps_half_harmonic(int nx, int ny, int nz, const double *eps_node, double *ex,
                          double *ey, double *ez) {
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t p = idx3(i, j, k, nx, ny);
                const double e0 = eps_node[p];
                ex[p] = (i + 1 < nx) ? 2.0 * e0 * eps_node[p + 1] / (e0 + eps_node[p + 1]) : 0.0;
                ey[p] = (j + 1 < ny) ? 2.0 * e0 * eps_node[p + nx] / (e0 + eps_node[p + nx]) : 0.0;
                ez[p] = (k + 1 < nz)
                            ? 2.0 * e0 * eps_node[p + (int64_t)nx * ny] /
                                  (e0 + eps_node[p + (int64_t)nx * ny])
                            : 0.0;
            }
}

/* One batch of implicit-Euler line solves along direction dir (0=x, 1=y, 2=z):
 *   -r e_{-} v_{i-1} + (1 + r (e_{-} + e_{+})) v_i - r e_{+} v_{i+1} = w_i,  r = tau/h^2,
 * for the interior unknowns of every interior line; face values enter the right-hand
 * side.  Thomas algorithm (forward elimination, back substitution), no pivoting: every
 * line matrix is strictly diagonally dominant. */
void or_sweep(int nx, int ny, int nz, double *u, const double *e_half, int dir, double r) {
    const int n[3] = {nx, ny, nz};
    const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
    const int len = n[dir];
    const int o1 = dir == 0 ? 1 : 0, o2 = dir == 2 ? 1 : 2; /* the two other axes */
    const int m = len - 2;                                  /* unknowns per line */
    if (m <= 0) return;
    const int64_t s = stride[dir];
    const int n1 = n[o1], n2 = n[o2];
#pragma omp parallel num_threads(g_threads)
    {
        double *cp = (double *)malloc(sizeof(double) * (size_t)m);
        double *dp = (double *)malloc(sizeof(double) * (size_t)m);
#pragma omp for collapse(2) schedule(static)
        for (int b = 1; b < n2 - 1; ++b)
            for (int a = 1; a < n1 - 1; ++a) {
                int ijk[3];
                ijk[dir] = 0;
                ijk[o1] = a;
                ijk[o2] = b;
                const int64_t base = idx3(ijk[0], ijk[1], ijk[2], nx, ny);
                /* forward elimination over unknowns t = 0..m-1 (node index t+1) */
                for (int t = 0; t < m; ++t) {
                    const int64_t p = base + (int64_t)(t + 1) * s;
                    const double em = e_half[p - s]; /* eps at node-1/2 */
                    const double ep = e_half[p];     /* eps at node+1/2 */
                    const double av = -r * em, cv = -r * ep, bv = 1.0 + r * (em + ep);
                    double dv = u[p];
                    if (t == 0) dv -= av * u[p - s];      /* face value at node 0 */
                    if (t == m - 1) dv -= cv * u[p + s];  /* face value at node len-1 */
                    const double c_use = (t == m - 1) ? 0.0 : cv;
                    if (t == 0) {
                        cp[t] = c_use / bv;
                        dp[t] = dv / bv;
                    } else {
                        const double den = bv - av * cp[t - 1];
                        cp[t] = c_use / den;
                        dp[t] = (dv - av * dp[t - 1]) / den;
                    }
                }
                /* back substitution */
                double next = 0.0;
                for (int t = m - 1; t >= 0; --t) {
                    const double v = (t == m - 1) ? dp[t] : dp[t] - cp[t] * next;
                    u[base + (int64_t)(t + 1) * s] = v;
                    next = v;
                }
            }
        free(cp);
        free(dp);
    }
}

/* The explicit half of a Crank-Nicolson sweep along dir, in place at the interior nodes of every
 * interior line: w_t + hr [e_{t+1/2} (w_{t+1} - w_t) - e_{t-1/2} (w_t - w_{t-1})], from the line's
 * old values (faces included). */
static void cn_explicit(int nx, int ny, int nz, double *u, const double *e_half, int dir, double hr) {
    const int n[3] = {nx, ny, nz};
    const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
    const int len = n[dir];
    const int o1 = dir == 0 ? 1 : 0, o2 = dir == 2 ? 1 : 2;
    if (len - 2 <= 0) return;
    const int64_t s = stride[dir];
    const int n1 = n[o1], n2 = n[o2];
#pragma omp parallel num_threads(g_threads)
    {
        double *w = (double *)malloc(sizeof(double) * (size_t)len);
#pragma omp for collapse(2) schedule(static)
        for (int b = 1; b < n2 - 1; ++b)
            for (int a = 1; a < n1 - 1; ++a) {
                int ijk[3];
                ijk[dir] = 0;
                ijk[o1] = a;
                ijk[o2] = b;
                const int64_t base = idx3(ijk[0], ijk[1], ijk[2], nx, ny);
                for (int t = 0; t < len; ++t) w[t] = u[base + (int64_t)t * s];
                for (int t = 1; t < len - 1; ++t) {
                    const int64_t p = base + (int64_t)t * s;
                    const double em = e_half[p - s], ep = e_half[p];
                    u[p] = w[t] + hr * (ep * (w[t + 1] - w[t]) - em * (w[t] - w[t - 1]));
                }
            }
        free(w);
    }
}

/* Eqs. (LODCN1_2)-(LODCN1_4): per line, the right-hand side is the explicit half step with r/2,
 * then the implicit half step is the or_sweep solve with r/2. */
void or_sweep_cn(int nx, int ny, int nz, double *u, const double *e_half, int dir, double r) {
    cn_explicit(nx, ny, nz, u, e_half, dir, 0.5 * r);
    or_sweep(nx, ny, nz, u, e_half, dir, 0.5 * r);
}

/* Eq. (ana3) with a = kbar^2 dt / (2 alpha) = kbar^2 tau / 2:
 *   W' = ln[(cosh a + e^{-W} sinh a) / (e^{-W} cosh a + sinh a)].
 * The map is odd in W, so it is evaluated at |W|, where e^{-|W|} <= 1 cannot overflow.
 * Valid for a < ~700 (cosh a finite). */
double or_ana3(double w, double a) {
    const double sgn = w < 0.0 ? -1.0 : 1.0;
    const double e = exp(-fabs(w));
    const double ch = cosh(a), sh = sinh(a);
    return sgn * log((ch + e * sh) / (e * ch + sh));
}

/* The nonlinear stage at every interior node where kbar^2 > 0 (Eq. LODIE1_1).
 * Where kbar^2 = 0 the stage is alpha w_t = 0 and leaves w unchanged. */
void or_nonlinear(int nx, int ny, int nz, double *u, const double *kappa2_node, double tau) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(g_threads)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                const int64_t p = idx3(i, j, k, nx, ny);
                if (kappa2_node[p] > 0.0) u[p] = or_ana3(u[p], 0.5 * kappa2_node[p] * tau);
            }
}

/* Eq. (LODIE1_5): u += tau * rho at interior nodes (rho is the discrete source Q). */
void or_source(int nx, int ny, int nz, double *u, const double *rho, double tau) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(g_threads)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                const int64_t p = idx3(i, j, k, nx, ny);
                u[p] += tau * rho[p];
            }
}

/* n_steps LOD steps with tau = dt/alpha and r = tau/h^2.
 * scheme 2 (LODIE2, Sec. 3.1): source, x, y, z, nonlinear.
 * scheme 1 (LODIE1):           nonlinear, x, y, z, source.
 * schemes 3, 4 (LODCN1, LODCN2): the orders of 1 and 2 with the Crank-Nicolson sweeps. */
void or_lod_run(int nx, int ny, int nz, double *u, const double *rho, const double *kappa2_node,
                const double *ex, const double *ey, const double *ez, double tau, double h,
                int n_steps, int scheme) {
    const double r = tau / (h * h);
    const int first_n = scheme == 1 || scheme == 3;
    const int cn = scheme == 3 || scheme == 4;
    for (int s = 0; s < n_steps; ++s) {
        if (first_n) or_nonlinear(nx, ny, nz, u, kappa2_node, tau);
        else or_source(nx, ny, nz, u, rho, tau);
        if (cn) {
            or_sweep_cn(nx, ny, nz, u, ex, 0, r);
            or_sweep_cn(nx, ny, nz, u, ey, 1, r);
            or_sweep_cn(nx, ny, nz, u, ez, 2, r);
        } else {
            or_sweep(nx, ny, nz, u, ex, 0, r);
            or_sweep(nx, ny, nz, u, ey, 1, r);
            or_sweep(nx, ny, nz, u, ez, 2, r);
        }
        if (first_n) or_source(nx, ny, nz, u, rho, tau);
        else or_nonlinear(nx, ny, nz, u, kappa2_node, tau);
    }
}

/* n_steps of an additive splitting with tau = dt/alpha and r = tau/h^2 (Sec. 3.2, 3.3).
 * AOS (schemes 5-8; Eqs. AOS1_1-5, AOS2_1-5): four parts advanced from U^n side by side -- the
 *   nonlinear part alpha w_t = -4 kbar^2 sinh w integrated exactly (or_ana3 with a = 2 kbar^2 tau),
 *   and one line solve per direction with 4r (implicit Euler, Eqs. AOSIE1_2-4 / AOSIE2_2-4) or with
 *   2r on each side (Crank-Nicolson, Eqs. AOSCN1_2-4 / AOSCN2_2-4), its right-hand side carrying the
 *   direction's share of the source: AOS1 4 tau Q on x alone, AOS2 4/3 tau Q on each direction;
 *   U^{n+1} is the mean of the four.
 * MAOS (schemes 9, 10; Eqs. MAOS1_1-5): the nonlinear stage (a = kbar^2 tau / 2) first, then three
 *   line solves from its result with 3r (or 3r/2 on each side), each with tau Q; U^{n+1} is the
 *   mean of the three.
 * The source enters after the explicit half of a Crank-Nicolson solve.  work: 4 states. */
void or_additive_run(int nx, int ny, int nz, double *u, double *work, const double *rho,
                     const double *kappa2_node, const double *ex, const double *ey, const double *ez,
                     double tau, double h, int n_steps, int scheme) {
    const int64_t total = (int64_t)nx * ny * nz;
    const int aos = scheme >= 5 && scheme <= 8;
    const int cn = scheme == 7 || scheme == 8 || scheme == 10;
    const double c = aos ? 4.0 : 3.0;
    const double r = c * tau / (h * h);
    double share[3] = {1.0, 1.0, 1.0};
    if (scheme == 5 || scheme == 7) share[0] = 4.0, share[1] = share[2] = 0.0;
    if (scheme == 6 || scheme == 8) share[0] = share[1] = share[2] = 4.0 / 3.0;
    const double *e[3] = {ex, ey, ez};
    double *w = work, *v[3] = {work + total, work + 2 * total, work + 3 * total};
    for (int s = 0; s < n_steps; ++s) {
        memcpy(w, u, sizeof(double) * (size_t)total);
        or_nonlinear(nx, ny, nz, w, kappa2_node, aos ? 4.0 * tau : tau);
        const double *from = aos ? u : w;
        for (int d = 0; d < 3; ++d) {
            memcpy(v[d], from, sizeof(double) * (size_t)total);
            if (cn) cn_explicit(nx, ny, nz, v[d], e[d], d, 0.5 * r);
            if (share[d] != 0.0) or_source(nx, ny, nz, v[d], rho, share[d] * tau);
            or_sweep(nx, ny, nz, v[d], e[d], d, cn ? 0.5 * r : r);
        }
#pragma omp parallel for collapse(2) schedule(static) num_threads(g_threads)
        for (int k = 1; k < nz - 1; ++k)
            for (int j = 1; j < ny - 1; ++j)
                for (int i = 1; i < nx - 1; ++i) {
                    const int64_t p = idx3(i, j, k, nx, ny);
                    u[p] = aos ? (w[p] + v[0][p] + v[1][p] + v[2][p]) / 4.0
                               : (v[0][p] + v[1][p] + v[2][p]) / 3.0;
                }
    }
}

/* Explicit Euler for Eq. (TimeDepNPB) with the same stencil:
 *   u += tau * (delta_x^2 u + delta_y^2 u + delta_z^2 u - kbar^2 sinh u + rho).
 * Used as an independent check of the steady state (Sec. 5.2 uses it as reference). */
void or_euler_run(int nx, int ny, int nz, double *u, double *work, const double *rho,
                  const double *kappa2_node, const double *ex, const double *ey,
                  const double *ez, double tau, double h, int n_steps) {
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const double ih2 = 1.0 / (h * h);
    const int64_t total = (int64_t)nx * ny * nz;
    for (int s = 0; s < n_steps; ++s) {
        memcpy(work, u, sizeof(double) * (size_t)total);
#pragma omp parallel for collapse(2) schedule(static) num_threads(g_threads)
        for (int k = 1; k < nz - 1; ++k)
            for (int j = 1; j < ny - 1; ++j)
                for (int i = 1; i < nx - 1; ++i) {
                    const int64_t p = idx3(i, j, k, nx, ny);
                    const double w = work[p];
                    double lap = ex[p] * (work[p + sx] - w) + ex[p - sx] * (work[p - sx] - w);
                    lap += ey[p] * (work[p + sy] - w) + ey[p - sy] * (work[p - sy] - w);
                    lap += ez[p] * (work[p + sz] - w) + ez[p - sz] * (work[p - sz] - w);
                    const double nl = kappa2_node[p] > 0.0 ? kappa2_node[p] * sinh(w) : 0.0;
                    u[p] = w + tau * (lap * ih2 - nl + rho[p]);
                }
    }
}
