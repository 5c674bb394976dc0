/*
 * Oracle geometry: seeded grain packings voxelised with integer arithmetic.
 *
 * THIS IS TEST INFRASTRUCTURE (see lbm_oracle.c).  It is a second,
 * independent statement of the geometry recipe; the product library has its
 * own GPU implementation and the two are compared bit for bit.
 *
 * The paper places grains in 2D (section 3.1.1, with an optional hydrodynamic
 * radius of 0.9 R) and takes a CT-segmented sand in 3D (section 3.3).  The
 * recipe below is the synthetic stand-in for both:
 *
 *  RNG       SplitMix64 (Steele, Lea & Flood 2014):
 *              s += 0x9E3779B97F4A7C15; z = s;
 *              z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
 *              z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
 *              return z ^ (z >> 31);
 *            draw_below(n) = ((next() >> 32) * n) >> 32   (n < 2^32)
 *  Units     positions and radii in Q8 fixed point (1 lu = 256); node
 *            (i, j[, k]) sits at (256 i, 256 j[, 256 k]).
 *  Trial     cx = draw_below(256 nx), cy = draw_below(256 ny),
 *            [cz = draw_below(256 nz)], r = 256 r_min + draw_below(256 (r_max - r_min) + 1),
 *            drawn in that order.
 *  Buffer    a trial is rejected unless cx - r > 256 (buf - 1) and
 *            cx + r < 256 (nx - buf): the first and last buf columns stay fluid.
 *  Disks     (kind 1, D2Q9) random sequential addition: also rejected if
 *            (cx - cx')^2 + (cy - cy')^2 < (r + r' + 256)^2 for any placed disk
 *            (a gap of at least 1 lu between grains).
 *  Spheres   (kind 2, D3Q19) Boolean model: overlaps are allowed.
 *  Voxels    node is solid iff (256 i - cx)^2 + (256 j - cy)^2 [+ (256 k - cz)^2]
 *            <= rv^2, rv = (r * hydro_q8) >> 8 (hydro_q8 = 256: factor 1).
 *  Stop      before each trial, stop once the fluid count is <= fluid_target =
 *            (int64)(target_porosity * N), or after max_rejections
 *            consecutive trials that added no solid node (rejected, or a
 *            sphere already covered by others).
 *  Fill      (fill != 0) fluid nodes not reachable from the inlet plane x = 0
 *            through 4-connected (2D) / 6-connected (3D) fluid paths become solid.
 * Kind 0 is the empty channel/duct (no grains).
 *
 * info[0] = grains placed, info[1] = solid nodes before the fill,
 * info[2] = nodes filled, info[3] = fluid nodes at the end.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

uint64_t orc_splitmix64_next(uint64_t* s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int64_t draw_below(uint64_t* s, int64_t n) { return (int64_t)(((orc_splitmix64_next(s) >> 32) * (uint64_t)n) >> 32); }

static long node(int nx, int ny, int x, int y, int z) { return ((long)z * ny + y) * nx + x; }

/* Marks the voxels of one grain; returns how many became solid. */
static long stamp(uint8_t* mask, int nx, int ny, int nz, int d, int64_t cx, int64_t cy, int64_t cz, int64_t rv)
{
    long added = 0;
    int64_t r2 = rv * rv;
    int x0 = (int)((cx - rv) / 256) - 1, x1 = (int)((cx + rv) / 256) + 1;
    int y0 = (int)((cy - rv) / 256) - 1, y1 = (int)((cy + rv) / 256) + 1;
    int z0 = 0, z1 = 0;
    if (d == 3) {
        z0 = (int)((cz - rv) / 256) - 1;
        z1 = (int)((cz + rv) / 256) + 1;
    }
    for (int z = z0; z <= z1; ++z) {
        if (z < 0 || z >= nz) continue;
        for (int y = y0; y <= y1; ++y) {
            if (y < 0 || y >= ny) continue;
            for (int x = x0; x <= x1; ++x) {
                if (x < 0 || x >= nx) continue;
                int64_t dx = 256 * (int64_t)x - cx, dy = 256 * (int64_t)y - cy;
                int64_t dz = d == 3 ? 256 * (int64_t)z - cz : 0;
                if (dx * dx + dy * dy + dz * dz <= r2) {
                    long n = node(nx, ny, x, y, z);
                    if (!mask[n]) {
                        mask[n] = 1;
                        ++added;
                    }
                }
            }
        }
    }
    return added;
}

/* Breadth-first search from the fluid nodes of the inlet plane. */
static long fill_unreachable(uint8_t* mask, int nx, int ny, int nz)
{
    long N = (long)nx * ny * nz;
    uint8_t* seen = (uint8_t*)calloc((size_t)N, 1);
    long* queue = (long*)malloc(sizeof(long) * (size_t)N);
    if (!seen || !queue) {
        free(seen);
        free(queue);
        return -1;
    }
    long head = 0, tail = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            long n = node(nx, ny, 0, y, z);
            if (!mask[n]) {
                seen[n] = 1;
                queue[tail++] = n;
            }
        }
    static const int nb[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    while (head < tail) {
        long n = queue[head++];
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long)nx * ny));
        for (int k = 0; k < 6; ++k) {
            int xx = x + nb[k][0], yy = y + nb[k][1], zz = z + nb[k][2];
            if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
            long m = node(nx, ny, xx, yy, zz);
            if (!mask[m] && !seen[m]) {
                seen[m] = 1;
                queue[tail++] = m;
            }
        }
    }
    long filled = 0;
    for (long n = 0; n < N; ++n)
        if (!mask[n] && !seen[n]) {
            mask[n] = 1;
            ++filled;
        }
    free(seen);
    free(queue);
    return filled;
}

int orc_geometry(int q, int nx, int ny, int nz, int kind, uint64_t seed, int r_min, int r_max,
                 double target_porosity, int hydro_q8, int buf, long max_rejections, int fill, uint8_t* mask,
                 int64_t* info)
{
    int d = q == 19 ? 3 : 2;
    if (d == 2 && nz != 1) return -1;
    long N = (long)nx * ny * nz;
    memset(mask, 0, (size_t)N);
    long n_solid = 0, n_grains = 0, filled = 0;
    if (kind == 1 || kind == 2) {
        uint64_t s = seed;
        long fluid_target = (long)(target_porosity * (double)N);
        int64_t cap = 4096, count = 0;
        int64_t* placed = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)cap);
        if (!placed) return -2;
        long rejections = 0;
        while (N - n_solid > fluid_target && rejections < max_rejections) {
            int64_t cx = draw_below(&s, 256 * (int64_t)nx);
            int64_t cy = draw_below(&s, 256 * (int64_t)ny);
            int64_t cz = d == 3 ? draw_below(&s, 256 * (int64_t)nz) : 0;
            int64_t r = 256 * (int64_t)r_min + draw_below(&s, 256 * (int64_t)(r_max - r_min) + 1);
            int ok = (cx - r > 256 * (int64_t)(buf - 1)) && (cx + r < 256 * (int64_t)(nx - buf));
            if (ok && kind == 1) {
                for (int64_t k = 0; k < count; ++k) {
                    int64_t dx = cx - placed[3 * k], dy = cy - placed[3 * k + 1], sr = r + placed[3 * k + 2] + 256;
                    if (dx * dx + dy * dy < sr * sr) {
                        ok = 0;
                        break;
                    }
                }
            }
            if (!ok) {
                ++rejections;
                continue;
            }
            if (kind == 1) {
                if (count == cap) {
                    cap *= 2;
                    int64_t* p = (int64_t*)realloc(placed, sizeof(int64_t) * 3 * (size_t)cap);
                    if (!p) {
                        free(placed);
                        return -2;
                    }
                    placed = p;
                }
                placed[3 * count] = cx;
                placed[3 * count + 1] = cy;
                placed[3 * count + 2] = r;
                ++count;
            }
            int64_t rv = (r * hydro_q8) >> 8;
            long added = stamp(mask, nx, ny, nz, d, cx, cy, cz, rv);
            n_solid += added;
            ++n_grains;
            rejections = added > 0 ? 0 : rejections + 1;
        }
        free(placed);
    }
    long solid_before = n_solid;
    if (fill) {
        filled = fill_unreachable(mask, nx, ny, nz);
        if (filled < 0) return -2;
    }
    if (info) {
        info[0] = n_grains;
        info[1] = solid_before;
        info[2] = filled;
        info[3] = N - solid_before - filled;
    }
    return 0;
}
