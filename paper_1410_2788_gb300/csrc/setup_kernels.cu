// setup_kernels.cu -- per-grid set-up on the device (run once per molecule).
//
//   mask        node bits of Omega_m: a node is inside iff it lies on or inside some
//               atom's ball (Sec. 3.1: eps_m "on/inside" the surface).  For the midpoint
//               eps reading, the same test on the half points p + e_d/2.
//   charges     the trilinear spread of the point charges (Sec. 3.1, Eq. RhoEq) as a
//               list of (node, qtilde) entries grouped by x-line.  Built without
//               order-dependent floating-point atomics: entries are bucketed by line,
//               sorted by (x, atom, corner) and summed in that fixed order.
//   boundary    Eq. (BoundaryCond) on the 6 faces: solvent uses eps_out and kbar,
//               vacuum eps_in and kbar = 0, both in one pass.  FP64 pair terms, or FP32 pair
//               terms with per-chunk FP64 accumulation for the mixed-precision path.
//
// The distance tests and weights use explicitly rounded FP64 operations (no fused
// multiply-add), so that inside/outside decisions and node charges are reproducible.
#include <algorithm>

#include "npb_internal.cuh"
#include "setup_kernels.cuh"
#include "exp_table.cuh"
#include "f32x2.cuh"

namespace npb {

__device__ __forceinline__ double node_coord(double o, int i, double h) {
    return __dadd_rn(o, __dmul_rn((double)i, h));
}

__device__ __forceinline__ double dist2(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// One block per atom.  A thread owns one 32-node word of an x-row (j, k) of the atom's bounding box,
// decides its nodes one by one (the oracle's distance test, in the same FP64 operations), and sets
// them with one atomicOr per array: the node mask and, for the midpoint reading, the three
// half-point arrays.
__global__ void k_mask_atoms(GridGeom g, const double *__restrict__ xyz,
                             const double *__restrict__ radius, int n_atoms,
                             uint32_t *__restrict__ mask, uint32_t *__restrict__ hx,
                             uint32_t *__restrict__ hy, uint32_t *__restrict__ hz) {
    const int a = blockIdx.x;
    if (a >= n_atoms) return;
    const double c[3] = {xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
    const double rho = radius[a];
    const double r2 = __dmul_rn(rho, rho);
    const int n[3] = {g.nx, g.ny, g.nz};
    const double o[3] = {g.ox, g.oy, g.oz};
    // The atom's node box, widened by one node on either side: any superset of the nodes within rho
    // gives the same bits (every node is tested below), so it is estimated in FP32 with the
    // reciprocal of h (an index off by one where the FP64 quotient lies within 1e-5 of an integer is
    // covered by the widening), not with six FP64 divisions per thread.
    const float ihf = 1.0f / (float)g.h;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = (int)floorf((float)(c[d] - rho - o[d]) * ihf) - 1;
        hi[d] = (int)ceilf((float)(c[d] + rho - o[d]) * ihf) + 1;
        lo[d] = max(lo[d], 0);
        hi[d] = min(hi[d], n[d] - 1);
    }
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    if (ex <= 0 || ey <= 0 || ez <= 0) return;
    const int w0 = lo[0] >> 5, nw = (hi[0] >> 5) - w0 + 1;
    const int total = nw * ey * ez;
    const int wpr = mask_words_per_row(g.pitch);
    const double hh = __dmul_rn(0.5, g.h);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int wi = w0 + t % nw;
        const int j = lo[1] + (t / nw) % ey;
        const int k = lo[2] + t / (nw * ey);
        const int ib = max(lo[0], wi * 32), ie = min(hi[0], wi * 32 + 31);
        const double py = node_coord(o[1], j, g.h), pz = node_coord(o[2], k, g.h);
        // An FP32 estimate of the squared distance decides every node outside a relative band of
        // 1e-5 around r^2 (its error is below 1e-6 of d^2); inside the band the FP64 test decides.
        const float dyf = (float)__dsub_rn(py, c[1]), dzf = (float)__dsub_rn(pz, c[2]);
        const float dx0 = (float)__dsub_rn(node_coord(o[0], ib, g.h), c[0]), hf = (float)g.h, hhf = (float)hh;
        const float r2f = (float)r2, lo_band = r2f * (1.f - 1e-5f), hi_band = r2f * (1.f + 1e-5f);
        auto inside = [&](float ex2, int i, int axis) -> bool {  // ex2: FP32 d^2 of the point
            if (ex2 < lo_band) return true;
            if (ex2 > hi_band) return false;
            double px = node_coord(o[0], i, g.h), qy = py, qz = pz;
            if (axis == 0) px = __dadd_rn(px, hh);
            if (axis == 1) qy = __dadd_rn(qy, hh);
            if (axis == 2) qz = __dadd_rn(qz, hh);
            return dist2(__dsub_rn(px, c[0]), __dsub_rn(qy, c[1]), __dsub_rn(qz, c[2])) <= r2;
        };
        const float yz2 = fmaf(dyf, dyf, dzf * dzf);
        uint32_t m = 0, mx = 0, my = 0, mz = 0;
        for (int i = ib; i <= ie; ++i) {
            const float dxf = fmaf((float)(i - ib), hf, dx0);
            const uint32_t bit = 1u << (i & 31);
            if (inside(fmaf(dxf, dxf, yz2), i, -1)) m |= bit;
            if (hx) {
                const float dxh = dxf + hhf, dyh = dyf + hhf, dzh = dzf + hhf;
                if (inside(fmaf(dxh, dxh, yz2), i, 0)) mx |= bit;
                if (inside(fmaf(dxf, dxf, fmaf(dyh, dyh, dzf * dzf)), i, 1)) my |= bit;
                if (inside(fmaf(dxf, dxf, fmaf(dyf, dyf, dzh * dzh)), i, 2)) mz |= bit;
            }
        }
        const int64_t w = ((int64_t)k * g.ny + j) * wpr + wi;
        if (m) atomicOr(mask + w, m);
        if (mx) atomicOr(hx + w, mx);
        if (my) atomicOr(hy + w, my);
        if (mz) atomicOr(hz + w, mz);
    }
}

// The line-major copies of the node mask -- bit y of line (x, z) into my, bit z of line (x, y)
// into mz -- as 32 x 32 bit transposes of the x-row mask, one tile per warp: lane l loads the word
// of row l of the tile, and a ballot over the lanes gathers each column.
__global__ void k_mask_transpose(GridGeom g, const uint32_t *__restrict__ mask, uint32_t *__restrict__ my,
                                 uint32_t *__restrict__ mz) {
    const int lane = threadIdx.x & 31;
    const int wpr = mask_words_per_row(g.pitch);
    const int xw = (g.nx + 31) >> 5, ty = (g.ny + 31) >> 5, tz = (g.nz + 31) >> 5;
    const int64_t n_y = (int64_t)g.nz * ty * xw, n_z = (int64_t)g.ny * tz * xw;
    const int wy = line_words(g.ny), wz = line_words(g.nz);
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < n_y + n_z;
         tile += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const bool to_y = tile < n_y;
        const int64_t q = to_y ? tile : tile - n_y;
        const int x_word = (int)(q % xw);
        const int64_t r = q / xw;
        const int rt = (int)(r % (to_y ? ty : tz));      // tile of the transposed coordinate
        const int plane = (int)(r / (to_y ? ty : tz));    // z for my, y for mz
        const int row = rt * 32 + lane;                   // y (my) or z (mz) of this lane's row
        uint32_t wv = 0;
        if (to_y ? row < g.ny : row < g.nz) {
            const int64_t rr = to_y ? (int64_t)plane * g.ny + row : (int64_t)row * g.ny + plane;
            wv = mask[rr * wpr + x_word];
        }
        uint32_t mine = 0;
#pragma unroll
        for (int cbit = 0; cbit < 32; ++cbit) {
            const uint32_t col = __ballot_sync(0xffffffffu, (wv >> cbit) & 1u);
            if (lane == cbit) mine = col;
        }
        const int x = x_word * 32 + lane;
        if (x < g.nx) {
            if (to_y && my) my[((int64_t)plane * g.nx + x) * wy + rt] = mine;
            if (!to_y && mz) mz[((int64_t)plane * g.nx + x) * wz + rt] = mine;
        }
    }
}

// Raw trilinear entries: thread per (atom, corner).
__global__ void k_charge_raw(GridGeom g, const double *__restrict__ xyz, const double *__restrict__ q,
                             int n_atoms, RawEntry *__restrict__ raw, int32_t *__restrict__ count) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 8 * n_atoms) return;
    const int a = e >> 3, corner = e & 7;
    const double o[3] = {g.ox, g.oy, g.oz};
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
        const double s = __ddiv_rn(__dsub_rn(xyz[3 * a + d], o[d]), g.h);
        i0[d] = (int)floor(s);
        f[d] = __dsub_rn(s, (double)i0[d]);
    }
    const int ox = corner & 1, oy = (corner >> 1) & 1, oz = (corner >> 2) & 1;
    const double wx = ox ? f[0] : __dsub_rn(1.0, f[0]);
    const double wy = oy ? f[1] : __dsub_rn(1.0, f[1]);
    const double wz = oz ? f[2] : __dsub_rn(1.0, f[2]);
    const double w = __dmul_rn(__dmul_rn(wx, wy), wz);
    RawEntry r;
    r.x = i0[0] + ox;
    r.line = (i0[2] + oz) * g.ny + (i0[1] + oy);
    r.key = e;
    r.val = __dmul_rn(q[a], w);
    raw[e] = r;
    atomicAdd(count + r.line, 1);
}

// Exclusive scan of count[0..n) into begin[] (and the sum into *total); one block of 1024 threads.
__global__ void k_scan_lines(const int32_t *__restrict__ count, int32_t *__restrict__ begin, int n,
                             int32_t *__restrict__ total) {
    __shared__ int32_t part[1024];
    const int t = threadIdx.x;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    int32_t s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = t > 0 ? part[t - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        begin[i] = run;
        run += count[i];
    }
    if (total && t == (int)blockDim.x - 1) *total = part[t];
}

__global__ void k_charge_scatter(const RawEntry *__restrict__ raw, int n_raw,
                                 const int32_t *__restrict__ begin, int32_t *__restrict__ fill,
                                 RawEntry *__restrict__ bucket) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_raw) return;
    const RawEntry r = raw[e];
    const int pos = begin[r.line] + atomicAdd(fill + r.line, 1);
    bucket[pos] = r;
}

// Thread per line: sort the line's bucket by (x, key), sum equal x in that order, and
// write the merged entries back to the front of the bucket.
__global__ void k_charge_merge(RawEntry *__restrict__ bucket, const int32_t *__restrict__ begin,
                               const int32_t *__restrict__ count, int32_t *__restrict__ out_count,
                               int n_lines) {
    const int ln = blockIdx.x * blockDim.x + threadIdx.x;
    if (ln >= n_lines) return;
    const int b = begin[ln], c = count[ln];
    RawEntry *v = bucket + b;
    for (int i = 1; i < c; ++i) {  // insertion sort; buckets hold a few dozen entries
        const RawEntry t = v[i];
        int j = i - 1;
        while (j >= 0 && (v[j].x > t.x || (v[j].x == t.x && v[j].key > t.key))) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = t;
    }
    int m = 0;
    for (int i = 0; i < c;) {
        const int x = v[i].x;
        double s = 0.0;
        while (i < c && v[i].x == x) s = __dadd_rn(s, v[i++].val);
        v[m].x = x;
        v[m].val = s;
        ++m;
    }
    out_count[ln] = m;
}

// Thread per line: copy the merged entries into the final, contiguous charge list.
__global__ void k_charge_compact(GridGeom g, const RawEntry *__restrict__ bucket,
                                 const int32_t *__restrict__ raw_begin, const int32_t *__restrict__ begin,
                                 const int32_t *__restrict__ count, int32_t *__restrict__ ent_x,
                                 double *__restrict__ ent_qt, int64_t *__restrict__ ent_off,
                                 int2 *__restrict__ ent_xq, int n_lines) {
    const int ln = blockIdx.x * blockDim.x + threadIdx.x;
    if (ln >= n_lines) return;
    const int rb = raw_begin[ln], b = begin[ln], c = count[ln];
    const int y = ln % g.ny, z = ln / g.ny;
    for (int i = 0; i < c; ++i) {
        const RawEntry r = bucket[rb + i];
        ent_x[b + i] = r.x;
        ent_qt[b + i] = r.val;
        ent_off[b + i] = ((int64_t)z * g.ny + y) * g.pitch + r.x;
        if (ent_xq) ent_xq[b + i] = make_int2(r.x | (y << 16), __float_as_int((float)r.val));
    }
}

// Face enumeration: f0 z=0 (nx*ny), f1 z=nz-1, f2 y=0 (nx*(nz-2)), f3 y=ny-1,
// f4 x=0 ((ny-2)*(nz-2)), f5 x=nx-1.
__host__ __device__ int64_t face_count(int nx, int ny, int nz) {
    return 2LL * nx * ny + 2LL * nx * (nz - 2) + 2LL * (ny - 2) * (nz - 2);
}

__device__ __forceinline__ void face_node(int64_t f, int nx, int ny, int nz, int &i, int &j, int &k) {
    const int64_t A = (int64_t)nx * ny, B = (int64_t)nx * (nz - 2), Cc = (int64_t)(ny - 2) * (nz - 2);
    if (f < 2 * A) {
        k = f < A ? 0 : nz - 1;
        const int64_t r = f % A;
        i = (int)(r % nx);
        j = (int)(r / nx);
    } else if (f < 2 * A + 2 * B) {
        const int64_t ff = f - 2 * A;
        j = ff < B ? 0 : ny - 1;
        const int64_t r = ff % B;
        i = (int)(r % nx);
        k = 1 + (int)(r / nx);
    } else {
        const int64_t ff = f - 2 * A - 2 * B;
        i = ff < Cc ? 0 : nx - 1;
        const int64_t r = ff % Cc;
        j = 1 + (int)(r % (ny - 2));
        k = 1 + (int)(r / (ny - 2));
    }
}

constexpr int kAtomChunk = 256;

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Face rows: each thread takes kRowBlock adjacent nodes of one face row, all six faces in one
// launch.  A block serves one face type (ft 0: the z faces, rows along x at fixed y; 1: the y
// faces, rows along x at fixed z; 2: the x faces, rows along y at fixed z), blocks [0, b0) type 0,
// [b0, b0 + b1) type 1, the rest type 2.  Per atom the two fixed-coordinate differences and the
// sum of their squares serve the row's nodes, so a pair term costs one subtraction and one fused
// multiply-add for its squared distance instead of six operations.  Two nodes per thread keep
// about 40 warps on each SM at 257^3, enough to feed the special-function unit (rsqrt and exp2
// per pair term), which bounds the kernel; four nodes (20 warps) ran 9% slower.
constexpr int kRowBlock = 2;

struct FaceRow {
    int ft;          // face type
    int64_t f0;      // compact face index of the first node; the next nodes follow at +1
    int n_here;      // nodes of the row this thread owns (0: none)
    int i0, j0, k0;  // grid indices of the first node
};

__device__ __forceinline__ FaceRow face_row(int nx, int ny, int nz, int b0, int b1) {
    FaceRow R{};
    const int64_t A = (int64_t)nx * ny, B = (int64_t)nx * (nz - 2), Cc = (int64_t)(ny - 2) * (nz - 2);
    R.ft = (int)blockIdx.x < b0 ? 0 : ((int)blockIdx.x < b0 + b1 ? 1 : 2);
    const int blk = (int)blockIdx.x - (R.ft == 0 ? 0 : (R.ft == 1 ? b0 : b0 + b1));
    const int len = R.ft == 2 ? ny - 2 : nx;  // nodes per row
    const int rows = R.ft == 0 ? ny : nz - 2;  // rows per face
    const int chunks = (len + kRowBlock - 1) / kRowBlock;
    const int64_t items = 2LL * rows * chunks;
    const int64_t it = (int64_t)blk * blockDim.x + threadIdx.x;
    const bool live = it < items;
    const int side = live ? (int)(it / ((int64_t)rows * chunks)) : 0;
    const int64_t rr = live ? it % ((int64_t)rows * chunks) : 0;
    const int row = (int)(rr / chunks), ch = (int)(rr % chunks);
    if (R.ft == 0) {
        R.k0 = side ? nz - 1 : 0;
        R.j0 = row;
        R.i0 = ch * kRowBlock;
        R.f0 = (side ? A : 0) + (int64_t)R.j0 * nx + R.i0;
    } else if (R.ft == 1) {
        R.j0 = side ? ny - 1 : 0;
        R.k0 = 1 + row;
        R.i0 = ch * kRowBlock;
        R.f0 = 2 * A + (side ? B : 0) + (int64_t)row * nx + R.i0;
    } else {
        R.i0 = side ? nx - 1 : 0;
        R.k0 = 1 + row;
        R.j0 = 1 + ch * kRowBlock;
        R.f0 = 2 * A + 2 * B + (side ? Cc : 0) + (int64_t)row * (ny - 2) + (R.j0 - 1);
    }
    R.n_here = live ? min(kRowBlock, len - ch * kRowBlock) : 0;
    return R;
}

// Blocks of each face type for the row kernels (t threads per block).
static void face_row_blocks(const GridGeom &g, int t, int &b0, int &b1, int &b2) {
    const int64_t cz = (g.nx + kRowBlock - 1) / kRowBlock, cx = (g.ny - 2 + kRowBlock - 1) / kRowBlock;
    const int64_t n0 = 2LL * g.ny * cz, n1 = 2LL * (g.nz - 2) * cz, n2 = 2LL * (g.nz - 2) * cx;
    b0 = (int)((n0 + t - 1) / t);
    b1 = (int)((n1 + t - 1) / t);
    b2 = (int)((n2 + t - 1) / t);
}

// The hardware reciprocal square root, flushing subnormals (d^2 at a face node is at least the
// squared distance from the face to the molecule, far above them).
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32 pair terms of one atom chunk for a row along x (ALONG_Y false) or y; COULOMB: no screening
// (kbar = 0), the solvent sum is the vacuum one.  The row's two nodes go as packed pairs (one
// instruction for both nodes' subtraction, squared distance, charge over distance, sums and
// exponent), each lane rounded as the scalar operation; the rsqrt and exp2 stay per node.
static_assert(kRowBlock == 2, "the packed face terms take two nodes per thread");
template <bool ALONG_Y, bool COULOMB>
__device__ __forceinline__ void face_row_sums(const float4 *sa, int na, const float *w, float fu, float fv, float c,
                                              float *ps, float *pv) {
    const unsigned long long W = f2_pack(w[0], w[1]), kNeg1 = f2_pack(-1.0f, -1.0f), C = f2_pack(c, c);
    unsigned long long PS = f2_pack(ps[0], ps[1]), PV = f2_pack(pv[0], pv[1]);
#pragma unroll 4
    for (int t = 0; t < na; ++t) {
        const float4 P = sa[t];
        const float pw = ALONG_Y ? P.y : P.x, pu = ALONG_Y ? P.x : P.y;
        const float du = fu - pu, dv = fv - P.z;
        const float uv2 = fmaf(du, du, dv * dv);
        const unsigned long long DW = f2_fma(f2_pack(pw, pw), kNeg1, W);  // w - pw, exactly rounded
        const unsigned long long D2 = f2_fma(DW, DW, f2_pack(uv2, uv2));
        float d0, d1;
        f2_unpack(D2, d0, d1);
        const unsigned long long ID = f2_pack(rsqrt_approx(d0), rsqrt_approx(d1));
        const unsigned long long QI = f2_mul(f2_pack(P.w, P.w), ID);
        PV = f2_add(PV, QI);
        if (!COULOMB) {
            float a0, a1;
            f2_unpack(f2_mul(C, f2_mul(D2, ID)), a0, a1);
            PS = f2_fma(QI, f2_pack(ex2_approx(a0), ex2_approx(a1)), PS);
        }
    }
    f2_unpack(PS, ps[0], ps[1]);
    f2_unpack(PV, pv[0], pv[1]);
}

// Both media's faces, FP32 pair terms (chunk sums in FP32, chunks accumulated in FP64):
// solvent C sum q exp(-kbar d / sqrt(eps_out)) / (eps_out d), vacuum C sum q / (eps_in d).
__global__ void k_boundary_rows_f32(GridGeom g, const double *__restrict__ xyz, const double *__restrict__ q,
                                    int n_atoms, double eps_s, double kbar, double eps_v, int b0, int b1,
                                    double *__restrict__ out_s, double *__restrict__ out_v) {
    __shared__ float4 sa[kAtomChunk];
    const FaceRow R = face_row(g.nx, g.ny, g.nz, b0, b1);
    // positions relative to the grid origin keep FP32 resolution near 1e-5 A
    float w[kRowBlock];  // the row's coordinate of each node
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r) w[r] = R.ft == 2 ? (float)((R.j0 + r) * g.h) : (float)((R.i0 + r) * g.h);
    const float fu = R.ft == 2 ? (float)(R.i0 * g.h) : (float)(R.j0 * g.h);  // fixed: x (type 2) or y
    const float fv = (float)(R.k0 * g.h);                                     // fixed: z
    const float c = (float)(-kbar / sqrt(eps_s) * 1.4426950408889634);  // -kbar/sqrt(eps) * log2(e)
    const bool coulomb = kbar == 0.0;
    double ss[kRowBlock], sv[kRowBlock];
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r) ss[r] = sv[r] = 0.0;
    for (int a0 = 0; a0 < n_atoms; a0 += kAtomChunk) {
        __syncthreads();
        for (int t = threadIdx.x; t < kAtomChunk && a0 + t < n_atoms; t += blockDim.x)
            sa[t] = make_float4((float)(xyz[3 * (a0 + t)] - g.ox), (float)(xyz[3 * (a0 + t) + 1] - g.oy),
                                (float)(xyz[3 * (a0 + t) + 2] - g.oz), (float)q[a0 + t]);
        __syncthreads();
        const int na = min(kAtomChunk, n_atoms - a0);
        float ps[kRowBlock], pv[kRowBlock];
#pragma unroll
        for (int r = 0; r < kRowBlock; ++r) ps[r] = pv[r] = 0.f;
        if (coulomb) {
            if (R.ft == 2) face_row_sums<true, true>(sa, na, w, fu, fv, c, ps, pv);
            else face_row_sums<false, true>(sa, na, w, fu, fv, c, ps, pv);
        } else {
            if (R.ft == 2) face_row_sums<true, false>(sa, na, w, fu, fv, c, ps, pv);
            else face_row_sums<false, false>(sa, na, w, fu, fv, c, ps, pv);
        }
#pragma unroll
        for (int r = 0; r < kRowBlock; ++r) {
            ss[r] += (double)(coulomb ? pv[r] : ps[r]);
            sv[r] += (double)pv[r];
        }
    }
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r)
        if (r < R.n_here) {
            out_s[R.f0 + r] = kBjerrum / eps_s * ss[r];
            out_v[R.f0 + r] = kBjerrum / eps_v * sv[r];
        }
}

// FP64 pair terms of one atom chunk for a row along x (ALONG_Y false) or y, atoms in index order.
template <bool ALONG_Y>
__device__ __forceinline__ void face_row_sums64(const double4_32a *sa, int na, const double *w, double fu, double fv,
                                                double ks, const double *T, double *ss, double *sv) {
    for (int t = 0; t < na; ++t) {
        const double4_32a P = sa[t];
        const double pw = ALONG_Y ? P.y : P.x, pu = ALONG_Y ? P.x : P.y;
        const double du = fu - pu, dv = fv - P.z;
        const double uv2 = du * du + dv * dv;
#pragma unroll
        for (int r = 0; r < kRowBlock; ++r) {
            const double dw = w[r] - pw;
            const double d2 = dw * dw + uv2;
            const double id = rsqrt(d2);
            const double qi = P.w * id;
            sv[r] += qi;
            ss[r] += ks == 0.0 ? qi : qi * exp_nonpos(-ks * (d2 * id), T);
        }
    }
}

// Both media's faces, FP64 pair terms (the parity path): the two sums share the distance, taken
// as d^2 * rsqrt(d^2), and 1/d = rsqrt(d^2); only the solvent's screening needs its exponential.
__global__ void k_boundary_rows_f64(GridGeom g, const double *__restrict__ xyz, const double *__restrict__ q,
                                    int n_atoms, double eps_s, double kbar, double eps_v, int b0, int b1,
                                    double *__restrict__ out_s, double *__restrict__ out_v) {
    __shared__ double4_32a sa[kAtomChunk];
    __shared__ double T[32];  // 2^(j/32) for exp_nonpos
    exp_table_init(T);
    const FaceRow R = face_row(g.nx, g.ny, g.nz, b0, b1);
    double w[kRowBlock];
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r)
        w[r] = R.ft == 2 ? node_coord(g.oy, R.j0 + r, g.h) : node_coord(g.ox, R.i0 + r, g.h);
    const double fu = R.ft == 2 ? node_coord(g.ox, R.i0, g.h) : node_coord(g.oy, R.j0, g.h);
    const double fv = node_coord(g.oz, R.k0, g.h);
    const double ks = kbar / sqrt(eps_s);
    double ss[kRowBlock], sv[kRowBlock];
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r) ss[r] = sv[r] = 0.0;
    for (int a0 = 0; a0 < n_atoms; a0 += kAtomChunk) {
        __syncthreads();
        for (int t = threadIdx.x; t < kAtomChunk && a0 + t < n_atoms; t += blockDim.x)
            sa[t] = make_double4_32a(xyz[3 * (a0 + t)], xyz[3 * (a0 + t) + 1], xyz[3 * (a0 + t) + 2], q[a0 + t]);
        __syncthreads();
        const int na = min(kAtomChunk, n_atoms - a0);
        if (R.ft == 2) face_row_sums64<true>(sa, na, w, fu, fv, ks, T, ss, sv);
        else face_row_sums64<false>(sa, na, w, fu, fv, ks, T, ss, sv);
    }
#pragma unroll
    for (int r = 0; r < kRowBlock; ++r)
        if (r < R.n_here) {
            out_s[R.f0 + r] = kBjerrum / eps_s * ss[r];
            out_v[R.f0 + r] = kBjerrum / eps_v * sv[r];
        }
}

// Zero interior, Dirichlet faces, zero padding: the initial state of a leg (Sec. 2.2).
template <typename T>
struct InitVec;
template <>
struct InitVec<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct InitVec<double> {
    using type = double2;
    static constexpr int n = 2;
};

// A thread per 16-byte vector of the padded state (rows of pitch elements, pitch a multiple of 32).
template <typename T>
__global__ void k_init_leg(GridGeom g, const double *__restrict__ bc, T *__restrict__ u) {
    using V = typename InitVec<T>::type;
    constexpr int NV = InitVec<T>::n;
    const int vpr = g.pitch / NV;
    const int total = g.nz * g.ny * vpr;  // below 2^31 for every admitted grid
    const int64_t A = (int64_t)g.nx * g.ny, B = (int64_t)g.nx * (g.nz - 2), Cc = (int64_t)(g.ny - 2) * (g.nz - 2);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int row = q / vpr, c = q - row * vpr;
        const int j = row % g.ny, k = row / g.ny;
        const bool zface = k == 0 || k == g.nz - 1, yface = j == 0 || j == g.ny - 1;
        alignas(16) T v[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            const int i = c * NV + e;
            v[e] = T(0);
            if (i < g.nx) {
                if (zface) v[e] = (T)bc[(k == 0 ? 0 : A) + (int64_t)j * g.nx + i];
                else if (yface) v[e] = (T)bc[2 * A + (j == 0 ? 0 : B) + (int64_t)(k - 1) * g.nx + i];
                else if (i == 0 || i == g.nx - 1)
                    v[e] = (T)bc[2 * A + 2 * B + (i == 0 ? 0 : Cc) + (int64_t)(k - 1) * (g.ny - 2) + (j - 1)];
            }
        }
        reinterpret_cast<V *>(u)[(int64_t)row * vpr + c] = *reinterpret_cast<const V *>(v);
    }
}

// Dense FP64 copy of a padded state (for export / potential read-back).
template <typename T>
__global__ void k_unpad(GridGeom g, const T *__restrict__ u, double *__restrict__ out) {
    const int64_t total = (int64_t)g.nz * g.ny * g.nx;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nx);
        const int64_t r = p / g.nx;
        out[p] = (double)u[r * g.pitch + i];
    }
}

template <typename T>
__global__ void k_pad(GridGeom g, const double *__restrict__ in, T *__restrict__ u) {
    const int64_t total = (int64_t)g.nz * g.ny * g.nx;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nx);
        const int64_t r = p / g.nx;
        u[r * g.pitch + i] = (T)in[p];
    }
}

__global__ void k_mask_dense(GridGeom g, const uint32_t *__restrict__ mask, uint8_t *__restrict__ out) {
    const int64_t total = (int64_t)g.nz * g.ny * g.nx;
    const int wpr = mask_words_per_row(g.pitch);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nx);
        const int64_t r = p / g.nx;
        out[p] = (uint8_t)((mask[r * wpr + (i >> 5)] >> (i & 31)) & 1u);
    }
}

__global__ void k_qt_dense(GridGeom g, const int32_t *__restrict__ line_begin,
                           const int32_t *__restrict__ line_count, const int32_t *__restrict__ ent_x,
                           const double *__restrict__ ent_qt, double *__restrict__ out) {
    const int ln = blockIdx.x * blockDim.x + threadIdx.x;
    if (ln >= g.ny * g.nz) return;
    const int b = line_begin[ln], c = line_count[ln];
    for (int e = b; e < b + c; ++e) out[(int64_t)ln * g.nx + ent_x[e]] = ent_qt[e];
}

// ---------------------------------------------------------------- host launchers
static inline int blocks_for(int64_t n, int t) { return (int)std::min<int64_t>((n + t - 1) / t, 1 << 20); }

cudaError_t setup_mask(const GridGeom &g, const double *xyz, const double *radius, int n_atoms,
                       uint32_t *mask, uint32_t *hx, uint32_t *hy, uint32_t *hz, uint32_t *my, uint32_t *mz,
                       cudaStream_t st) {
    if (n_atoms > 0) k_mask_atoms<<<n_atoms, 128, 0, st>>>(g, xyz, radius, n_atoms, mask, hx, hy, hz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || (!my && !mz)) return e;
    const int64_t tiles = (int64_t)(((g.nx + 31) >> 5)) * ((int64_t)g.nz * ((g.ny + 31) >> 5) + (int64_t)g.ny * ((g.nz + 31) >> 5));
    const int blocks = (int)std::min<int64_t>((tiles + 7) / 8, 152 * 16);
    k_mask_transpose<<<blocks, 256, 0, st>>>(g, mask, my, mz);
    return cudaGetLastError();
}

cudaError_t setup_charges(const GridGeom &g, const double *xyz, const double *q, int n_atoms,
                          ChargeScratch &s, int32_t *line_begin, int32_t *line_count, int32_t *ent_x,
                          double *ent_qt, int64_t *ent_off, int2 *ent_xq, cudaStream_t st) {
    const int n_lines = g.ny * g.nz;
    const int n_raw = 8 * n_atoms;
    // the per-line counters are accumulated into: a refused clear must not leave stale counts
    cudaError_t e = cudaMemsetAsync(s.count, 0, sizeof(int32_t) * n_lines, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.fill, 0, sizeof(int32_t) * n_lines, st);
    if (e != cudaSuccess) return e;
    if (n_raw > 0) k_charge_raw<<<blocks_for(n_raw, 256), 256, 0, st>>>(g, xyz, q, n_atoms, s.raw, s.count);
    k_scan_lines<<<1, 1024, 0, st>>>(s.count, s.raw_begin, n_lines, nullptr);
    if (n_raw > 0)
        k_charge_scatter<<<blocks_for(n_raw, 256), 256, 0, st>>>(s.raw, n_raw, s.raw_begin, s.fill, s.bucket);
    k_charge_merge<<<blocks_for(n_lines, 128), 128, 0, st>>>(s.bucket, s.raw_begin, s.count, line_count,
                                                             n_lines);
    k_scan_lines<<<1, 1024, 0, st>>>(line_count, line_begin, n_lines, s.total);
    k_charge_compact<<<blocks_for(n_lines, 128), 128, 0, st>>>(g, s.bucket, s.raw_begin, line_begin, line_count,
                                                               ent_x, ent_qt, ent_off, ent_xq, n_lines);
    return cudaGetLastError();
}

cudaError_t setup_boundary_pair(const GridGeom &g, const double *xyz, const double *q, int n_atoms, double eps_out,
                                double kbar, double eps_in, double *out_s, double *out_v, cudaStream_t st,
                                bool fp64) {
    // one launch over the rows of all six faces, kRowBlock adjacent nodes per thread
    const int t = 128;
    int b0, b1, b2;
    face_row_blocks(g, t, b0, b1, b2);
    if (fp64)
        k_boundary_rows_f64<<<b0 + b1 + b2, t, 0, st>>>(g, xyz, q, n_atoms, eps_out, kbar, eps_in, b0, b1, out_s,
                                                         out_v);
    else
        k_boundary_rows_f32<<<b0 + b1 + b2, t, 0, st>>>(g, xyz, q, n_atoms, eps_out, kbar, eps_in, b0, b1, out_s,
                                                         out_v);
    return cudaGetLastError();
}

cudaError_t init_leg(int prec, const GridGeom &g, const double *bc, void *u, cudaStream_t st) {
    const int t = 256;
    const int64_t vecs = (int64_t)g.nz * g.ny * g.pitch / (prec == 0 ? 2 : 4);
    const int b = (int)std::min<int64_t>((vecs + t - 1) / t, 152 * 16);
    if (prec == 0) k_init_leg<double><<<b, t, 0, st>>>(g, bc, (double *)u);
    else k_init_leg<float><<<b, t, 0, st>>>(g, bc, (float *)u);
    return cudaGetLastError();
}

cudaError_t unpad_state(int prec, const GridGeom &g, const void *u, double *out, cudaStream_t st) {
    const int t = 256, b = 152 * 8;
    if (prec == 0) k_unpad<double><<<b, t, 0, st>>>(g, (const double *)u, out);
    else k_unpad<float><<<b, t, 0, st>>>(g, (const float *)u, out);
    return cudaGetLastError();
}

cudaError_t pad_state(int prec, const GridGeom &g, const double *in, void *u, cudaStream_t st) {
    const int t = 256, b = 152 * 8;
    if (prec == 0) k_pad<double><<<b, t, 0, st>>>(g, in, (double *)u);
    else k_pad<float><<<b, t, 0, st>>>(g, in, (float *)u);
    return cudaGetLastError();
}

cudaError_t mask_dense(const GridGeom &g, const uint32_t *mask, uint8_t *out, cudaStream_t st) {
    k_mask_dense<<<152 * 8, 256, 0, st>>>(g, mask, out);
    return cudaGetLastError();
}

cudaError_t qt_dense(const GridGeom &g, const int32_t *line_begin, const int32_t *line_count,
                     const int32_t *ent_x, const double *ent_qt, double *out, cudaStream_t st) {
    const int n_lines = g.ny * g.nz;
    k_qt_dense<<<blocks_for(n_lines, 128), 128, 0, st>>>(g, line_begin, line_count, ent_x, ent_qt, out);
    return cudaGetLastError();
}

}  // namespace npb
