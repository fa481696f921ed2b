/* Confined self-avoiding random walk for the synthetic molecules (input generation only).
 *
 * Same random stream as npb_inputs.Xoshiro256ss: xoshiro256** (Blackman & Vigna), doubles
 * from the top 53 bits.  Each step draws cos(theta) ~ U[-1,1) and phi ~ U[0, 2 pi) and moves
 * `step` A from the current atom; a candidate outside [lo, hi]^3 or closer than min_sep to a
 * placed atom is rejected; after max_reject consecutive rejections the walk restarts from a
 * placed atom drawn uniformly.  Clashes are found with a cell list (cell side = min_sep).
 * The generator state is read from and written back to s[4].
 * Returns the number of atoms placed (n_atoms on success, fewer if the budget ran out). */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t next_u64(uint64_t *s) {
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static inline double uniform(uint64_t *s, double lo, double hi) {
    return lo + (hi - lo) * ((double)(next_u64(s) >> 11) * (1.0 / 9007199254740992.0));
}

int rw_place(int n_atoms, double lo, double hi, uint64_t *s, double step, double min_sep, int max_reject,
             long budget, double *pos) {
    if (n_atoms <= 0) return 0;
    const double cell = min_sep;
    int nc = (int)floor((hi - lo) / cell);
    if (nc < 1) nc = 1;
    const long ncell = (long)nc * nc * nc;
    int *head = (int *)malloc(sizeof(int) * ncell);
    int *next = (int *)malloc(sizeof(int) * n_atoms);
    for (long c = 0; c < ncell; ++c) head[c] = -1;
#define KEY(v, d) ((int)fmin(nc - 1, fmax(0, (int)(((v)[d] - lo) / cell))))
    double p[3];
    for (int d = 0; d < 3; ++d) p[d] = uniform(s, lo, hi);
    pos[0] = p[0];
    pos[1] = p[1];
    pos[2] = p[2];
    {
        const long c = ((long)KEY(p, 2) * nc + KEY(p, 1)) * nc + KEY(p, 0);
        next[0] = head[c];
        head[c] = 0;
    }
    int cur = 0, placed = 1, rejects = 0;
    const double ms2 = min_sep * min_sep;
    while (placed < n_atoms) {
        const double cz = uniform(s, -1.0, 1.0);
        const double phi = uniform(s, 0.0, 2.0 * 3.141592653589793);
        const double sz = sqrt(fmax(0.0, 1.0 - cz * cz));
        double c[3] = {pos[3 * cur] + step * (sz * cos(phi)), pos[3 * cur + 1] + step * (sz * sin(phi)),
                       pos[3 * cur + 2] + step * cz};
        int bad = c[0] < lo || c[1] < lo || c[2] < lo || c[0] > hi || c[1] > hi || c[2] > hi;
        if (!bad) {
            const int kx = KEY(c, 0), ky = KEY(c, 1), kz = KEY(c, 2);
            for (int dz = -1; dz <= 1 && !bad; ++dz)
                for (int dy = -1; dy <= 1 && !bad; ++dy)
                    for (int dx = -1; dx <= 1 && !bad; ++dx) {
                        const int x = kx + dx, y = ky + dy, z = kz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= nc || y >= nc || z >= nc) continue;
                        for (int i = head[((long)z * nc + y) * nc + x]; i >= 0; i = next[i]) {
                            const double ex = pos[3 * i] - c[0], ey = pos[3 * i + 1] - c[1],
                                         ez = pos[3 * i + 2] - c[2];
                            if (ex * ex + ey * ey + ez * ez < ms2) {
                                bad = 1;
                                break;
                            }
                        }
                    }
        }
        if (bad) {
            ++rejects;
            if (--budget <= 0) break;
            if (rejects >= max_reject) {
                cur = (int)(uniform(s, 0.0, 1.0) * placed) % placed;
                rejects = 0;
            }
            continue;
        }
        pos[3 * placed] = c[0];
        pos[3 * placed + 1] = c[1];
        pos[3 * placed + 2] = c[2];
        const long k = ((long)KEY(c, 2) * nc + KEY(c, 1)) * nc + KEY(c, 0);
        next[placed] = head[k];
        head[k] = placed;
        cur = placed;
        ++placed;
        rejects = 0;
    }
#undef KEY
    free(head);
    free(next);
    return placed;
}
