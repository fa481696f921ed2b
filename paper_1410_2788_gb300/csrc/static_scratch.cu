// static_scratch.cu -- npb_charge_list_static: the charge-list build without any allocation.
//
// Some callers cannot allocate device memory at the moment they need a charge list: host
// applications that own all device memory through their own pool and do not let libraries
// call cudaMalloc, and latency-critical paths that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree.  This entry point builds the same x-line-grouped
// trilinear charge list as npb_grid_create, into device buffers the caller provides, and
// takes every temporary it needs from one fixed array in this file's device memory.
//
// The array lives as long as the library is loaded, on every GPU that loads it.  The first
// call on a device looks up the array's device address with cudaGetSymbolAddress, with that
// device current; host code never hands the array's name itself to a kernel.  All calls
// share the array and each call clears the counters it accumulates into, so calls whose work
// overlaps on the GPU (different streams, or different host threads, on one device) race and
// must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "runtime.h"

using namespace npb;

namespace {

constexpr int kMaxAtoms = NPB_STATIC_MAX_ATOMS;
constexpr int kMaxLines = NPB_STATIC_MAX_LINES;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kXyzBytes = align256(sizeof(double) * 3 * kMaxAtoms);
constexpr size_t kQBytes = align256(sizeof(double) * kMaxAtoms);
constexpr size_t kLineBytes = align256(sizeof(int32_t) * kMaxLines);
constexpr size_t kTotalBytes = align256(16);
constexpr size_t kRawBytes = align256(sizeof(RawEntry) * 8 * kMaxAtoms);
constexpr size_t kScratchBytes = kXyzBytes + kQBytes + 3 * kLineBytes + kTotalBytes + 2 * kRawBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

}  // namespace

extern "C" int npb_charge_list_static(const double *xyz, const double *q, int32_t n_atoms, const int32_t n[3],
                                      double h, const double origin[3], int32_t *d_line_begin,
                                      int32_t *d_line_count, int32_t *d_ent_x, double *d_ent_qt,
                                      int64_t *d_ent_off, int32_t *d_n_entries, void *stream) {
    if (!n || !origin || !d_line_begin || !d_line_count || !d_ent_x || !d_ent_qt || !d_ent_off || !d_n_entries)
        return fail(NPB_EINVAL, "NULL argument");
    if (n_atoms < 0 || (n_atoms > 0 && (!xyz || !q))) return fail(NPB_EINVAL, "bad atom arrays");
    if (n_atoms > kMaxAtoms)
        return fail(NPB_EINVAL, "n_atoms = %d exceeds the static scratch limit of %d atoms", n_atoms, kMaxAtoms);
    for (int d = 0; d < 3; ++d)
        if (n[d] < 3 || n[d] > kMaxLine) return fail(NPB_EINVAL, "n[%d] = %d outside [3, %d]", d, n[d], kMaxLine);
    if ((int64_t)n[1] * n[2] > kMaxLines)
        return fail(NPB_EINVAL, "ny*nz = %lld exceeds the static scratch limit of %d x-lines",
                    (long long)n[1] * n[2], kMaxLines);
    if (!(h > 0)) return fail(NPB_EINVAL, "h must be > 0");
    for (int a = 0; a < n_atoms; ++a)
        for (int d = 0; d < 3; ++d) {
            const double s = (xyz[3 * a + d] - origin[d]) / h;
            if (!std::isfinite(s)) return fail(NPB_EINVAL, "atom %d: non-finite position", a);
            const double i0 = std::floor(s);
            if (i0 < 1 || i0 + 1 > n[d] - 2)
                return fail(NPB_EINVAL, "atom %d: charge stencil leaves the interior along axis %d", a, d);
        }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(NPB_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(NPB_EINVAL, "device %d out of range", dev);
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess)
                return fail(NPB_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                            cudaGetErrorString(e));
            g_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    double *s_xyz = reinterpret_cast<double *>(base);
    double *s_q = reinterpret_cast<double *>(base + kXyzBytes);
    unsigned char *lines = base + kXyzBytes + kQBytes;
    ChargeScratch sc{};
    sc.count = reinterpret_cast<int32_t *>(lines);
    sc.fill = reinterpret_cast<int32_t *>(lines + kLineBytes);
    sc.raw_begin = reinterpret_cast<int32_t *>(lines + 2 * kLineBytes);
    sc.total = reinterpret_cast<int32_t *>(lines + 3 * kLineBytes);
    sc.raw = reinterpret_cast<RawEntry *>(lines + 3 * kLineBytes + kTotalBytes);
    sc.bucket = reinterpret_cast<RawEntry *>(lines + 3 * kLineBytes + kTotalBytes + kRawBytes);

    if (n_atoms > 0) {
        e = cudaMemcpyAsync(s_xyz, xyz, sizeof(double) * 3 * n_atoms, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s_q, q, sizeof(double) * n_atoms, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(NPB_ECUDA, "atom upload failed: %s", cudaGetErrorString(e));
    }
    GridGeom geo{};
    geo.nx = n[0];
    geo.ny = n[1];
    geo.nz = n[2];
    geo.pitch = (n[0] + 31) / 32 * 32;
    geo.h = h;
    geo.ox = origin[0];
    geo.oy = origin[1];
    geo.oz = origin[2];
    // setup_charges clears the per-line counters it accumulates into before using them
    e = setup_charges(geo, s_xyz, s_q, n_atoms, sc, d_line_begin, d_line_count, d_ent_x, d_ent_qt, d_ent_off, nullptr, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_n_entries, sc.total, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(NPB_ECUDA, "static charge-list build failed: %s", cudaGetErrorString(e));
    return NPB_OK;
}
