// fft_vacuum.cu -- phi_0^FFT of Eq. (deltaG2): the vacuum potential as the direct solution of the
// discrete Poisson problem eps_in Delta_h u + rho = 0 with the vacuum Dirichlet faces (Sec. 5.1
// names the FFT fast Poisson solver for it).
//
// The face values move to the right-hand side (each interior node adds its face neighbours / h^2),
// leaving -Delta_h v = f on the N_x x N_y x N_z interior with zero faces.  The products of sine
// vectors sin(pi k n / (N+1)) diagonalise it with eigenvalue sum_d (2 - 2 cos(pi k_d/(N_d+1)))/h^2,
// so v = S^-1 (S f / lambda) with S the 3-D type-1 sine transform, applied one axis at a time.  A
// type-1 sine transform of length N is read off the FFT of the odd extension
// [0, x_1 .. x_N, 0, -x_N .. -x_1] (length M = 2(N+1)): X_k = -Im(Y_k)/2.  The FFTs are batched
// real-to-complex cuFFT plans (a library call); the result, in FP64, is cached on the grid until
// its set-up data change.
#include <cufft.h>

#include <cmath>

#include "runtime.h"

namespace npb {

static int cufft_check(cufftResult r, const char *what) {
    return r == CUFFT_SUCCESS ? 0 : fail(NPB_ECUDA, "%s failed: cufft error %d", what, (int)r);
}

// Right-hand side on the dense interior array a[k][j][i] (sizes nz-2, ny-2, nx-2).
__global__ void k_vac_rhs(GridGeom g, const double *__restrict__ u0, const double *__restrict__ qt_dense,
                          double rho_scale, double inv_eps, double *__restrict__ a) {
    const int Nx = g.nx - 2, Ny = g.ny - 2, Nz = g.nz - 2;
    const int64_t total = (int64_t)Nx * Ny * Nz;
    const double ih2 = 1.0 / (g.h * g.h);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(q % Nx);
        const int64_t r = q / Nx;
        const int j = 1 + (int)(r % Ny), k = 1 + (int)(r / Ny);
        const int64_t p = ((int64_t)k * g.ny + j) * g.pitch + i;
        const int64_t rowp = g.pitch, planep = (int64_t)g.ny * g.pitch;
        const double nb = u0[p - 1] + u0[p + 1] + u0[p - rowp] + u0[p + rowp] + u0[p - planep] + u0[p + planep];
        const double qv = qt_dense[((int64_t)k * g.ny + j) * g.nx + i];
        a[q] = rho_scale * qv * inv_eps + nb * ih2;  // interior neighbours of u0 are zero
    }
}

// Element n of line b of axis d in a[k][j][i]: the flat index.
__device__ __forceinline__ int64_t vac_index(int d, int64_t b, int n, int Nx, int Ny) {
    if (d == 0) return b * Nx + n;                                      // b = k*Ny + j
    if (d == 1) return ((b / Nx) * Ny + n) * (int64_t)Nx + (b % Nx);   // b = k*Nx + i
    return ((int64_t)n * Ny + (b / Nx)) * Nx + (b % Nx);               // b = j*Nx + i
}

__global__ void k_vac_pack(int d, const double *__restrict__ a, double *__restrict__ ext, int64_t lines, int N,
                           int M, int Nx, int Ny) {
    const int64_t total = lines * M;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = q / M;
        const int m = (int)(q - b * M);
        double v = 0.0;
        if (m >= 1 && m <= N) v = a[vac_index(d, b, m - 1, Nx, Ny)];
        else if (m >= N + 2) v = -a[vac_index(d, b, M - m - 1, Nx, Ny)];
        ext[q] = v;
    }
}

__global__ void k_vac_unpack(int d, const cufftDoubleComplex *__restrict__ Y, double *__restrict__ a,
                             int64_t lines, int N, int M, int Nx, int Ny, double scale) {
    const int H = M / 2 + 1;
    const int64_t total = lines * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = q / N;
        const int k = (int)(q - b * N) + 1;
        a[vac_index(d, b, k - 1, Nx, Ny)] = -0.5 * Y[b * H + k].y * scale;
    }
}

__global__ void k_vac_divide(double *__restrict__ a, int Nx, int Ny, int Nz, double h) {
    const int64_t total = (int64_t)Nx * Ny * Nz;
    const double ih2 = 1.0 / (h * h);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % Nx);
        const int64_t r = q / Nx;
        const int j = (int)(r % Ny), k = (int)(r / Ny);
        const double lam = (2.0 - 2.0 * cospi((double)(i + 1) / (Nx + 1))) * ih2 +
                           (2.0 - 2.0 * cospi((double)(j + 1) / (Ny + 1))) * ih2 +
                           (2.0 - 2.0 * cospi((double)(k + 1) / (Nz + 1))) * ih2;
        a[q] /= lam;
    }
}

__global__ void k_vac_store(GridGeom g, const double *__restrict__ a, double *__restrict__ u) {
    const int Nx = g.nx - 2, Ny = g.ny - 2, Nz = g.nz - 2;
    const int64_t total = (int64_t)Nx * Ny * Nz;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(q % Nx);
        const int64_t r = q / Nx;
        const int j = 1 + (int)(r % Ny), k = 1 + (int)(r / Ny);
        u[((int64_t)k * g.ny + j) * g.pitch + i] = a[q];
    }
}

static int blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// phi_0^FFT into g->d_vac_fft (a padded FP64 state with the vacuum faces of the legs' flavour:
// FP64 pair terms for the FP64 path, FP32 pair terms for the FP32 one); computed once per set-up.
int grid_vacuum_fft(Grid *g, int prec, cudaStream_t st) {
    const int kind = prec == NPB_FP64 ? 0 : 1;  // the faces of the legs it is combined with
    if (g->d_vac_fft && g->vac_fft_valid && g->vac_fft_kind == kind) return 0;
    const GridGeom &geo = g->geo;
    int rc;
    const double *bc = nullptr;
    if ((rc = grid_boundary(g, NPB_VACUUM, prec, st, &bc))) return rc;
    int n3[3] = {geo.nx, geo.ny, geo.nz};
    if (!g->d_vac_fft && (rc = galloc(g, &g->d_vac_fft, state_bytes(n3, NPB_FP64) / sizeof(double)))) return rc;
    CU(init_leg(NPB_FP64, geo, bc, g->d_vac_fft, st));  // faces, zero interior and padding
    const int Nx = geo.nx - 2, Ny = geo.ny - 2, Nz = geo.nz - 2;
    const int64_t N3 = (int64_t)Nx * Ny * Nz;
    int64_t work = 0;  // largest odd extension and spectrum over the three axes
    const int Nd[3] = {Nx, Ny, Nz};
    for (int d = 0; d < 3; ++d) {
        const int64_t lines = N3 / Nd[d];
        const int M = 2 * (Nd[d] + 1);
        work = std::max<int64_t>(work, lines * M + lines * (M / 2 + 1) * 2 + 2);
    }
    const size_t dense_bytes = (size_t)geo.nx * geo.ny * geo.nz * sizeof(double);
    const size_t bytes = (size_t)N3 * sizeof(double) + (size_t)work * sizeof(double) + dense_bytes + 512;
    void *mem = nullptr;
    if ((rc = g->ctx->alloc(&mem, bytes))) return rc;
    double *a = static_cast<double *>(mem);
    double *qt = a + N3;
    double *ext = qt + (size_t)geo.nx * geo.ny * geo.nz;
    auto release = [&](int r) {
        cudaStreamSynchronize(st);
        g->ctx->release(mem, bytes);
        return r;
    };
    cudaError_t e = cudaMemsetAsync(qt, 0, dense_bytes, st);
    if (e == cudaSuccess) e = qt_dense(geo, g->d_line_begin, g->d_line_count, g->d_ent_x, g->d_ent_qt, qt, st);
    if (e == cudaSuccess) {
        const double rho_scale = 4.0 * kPi * kBjerrum / (geo.h * geo.h * geo.h);
        k_vac_rhs<<<blocks(N3), 256, 0, st>>>(geo, g->d_vac_fft, qt, rho_scale, 1.0 / g->eps_in, a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return release(fail(NPB_ECUDA, "vacuum FFT set-up: %s", cudaGetErrorString(e)));
    // forward transform, division by the eigenvalues, inverse transform (the same transform,
    // scaled by 2/(N+1) per axis)
    for (int pass = 0; pass < 2; ++pass) {
        for (int d = 0; d < 3; ++d) {
            const int N = Nd[d], M = 2 * (N + 1);
            const int64_t lines = N3 / N;
            double *x = ext;
            cufftDoubleComplex *Y = reinterpret_cast<cufftDoubleComplex *>(
                reinterpret_cast<uintptr_t>(ext + lines * M + 1) & ~(uintptr_t)15);
            k_vac_pack<<<blocks(lines * M), 256, 0, st>>>(d, a, x, lines, N, M, Nx, Ny);
            cufftHandle plan;
            int n = M, inembed = M, onembed = M / 2 + 1;
            if ((rc = cufft_check(cufftPlanMany(&plan, 1, &n, &inembed, 1, M, &onembed, 1, M / 2 + 1, CUFFT_D2Z,
                                                (int)lines),
                                  "cufftPlanMany")))
                return release(rc);
            rc = cufft_check(cufftSetStream(plan, st), "cufftSetStream");
            if (!rc) rc = cufft_check(cufftExecD2Z(plan, x, Y), "cufftExecD2Z");
            cufftDestroy(plan);
            if (rc) return release(rc);
            const double scale = pass == 1 ? 2.0 / (N + 1) : 1.0;
            k_vac_unpack<<<blocks(lines * N), 256, 0, st>>>(d, Y, a, lines, N, M, Nx, Ny, scale);
        }
        if (pass == 0) k_vac_divide<<<blocks(N3), 256, 0, st>>>(a, Nx, Ny, Nz, geo.h);
    }
    k_vac_store<<<blocks(N3), 256, 0, st>>>(geo, a, g->d_vac_fft);
    e = cudaGetLastError();
    if (e != cudaSuccess) return release(fail(NPB_ECUDA, "vacuum FFT: %s", cudaGetErrorString(e)));
    g->vac_fft_valid = true;
    g->vac_fft_kind = kind;
    return release(0);
}

}  // namespace npb
