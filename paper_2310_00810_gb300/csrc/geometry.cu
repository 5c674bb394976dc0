// Seeded grain geometry on the device, voxelised with integer arithmetic so
// that the mask is bit-exact: the synthetic stand-in for the paper's 2D grain
// packings (section 3.1.1, optional hydrodynamic radius 0.9 R) and its CT
// sand (section 3.3).
//
// Recipe (the same statement the header gives):
//   SplitMix64 (Steele, Lea & Flood 2014) from state `seed`;
//   draw_below(n) = ((next() >> 32) * n) >> 32;
//   Q8 fixed point (1 lu = 256), node (x, y, z) at (256 x, 256 y, 256 z);
//   trial: cx = draw_below(256 nx), cy = draw_below(256 ny),
//          [cz = draw_below(256 nz)], r = 256 r_min + draw_below(256 (r_max - r_min) + 1);
//   kept iff cx - r > 256 (buf - 1) and cx + r < 256 (nx - buf), and, for
//   disks, (cx - cx')^2 + (cy - cy')^2 >= (r + r' + 256)^2 for every placed
//   disk (random sequential addition with a 1 lu gap; spheres overlap freely);
//   node solid iff |256 x - c|^2 <= rv^2, rv = (r * hydro_q8) >> 8;
//   stop once fluid nodes <= (int64)(target * N), or after max_rejections
//   trials in a row that added no solid node;
//   then (optionally) fluid not 4-/6-connected to the inlet plane x = 0 is
//   filled, and per-node link words are derived.
//
// Placement is inherently sequential (each trial depends on every earlier
// one), so it runs in ONE thread block: thread 0 draws, all threads test the
// trial against the placed disks and stamp its voxels.  The fill is a
// level-synchronous breadth-first search, also in one block, with the queue
// kept in the caller's link array (overwritten afterwards by the link words).
#include "common.cuh"

namespace lbm {

namespace {

constexpr int kGeoThreads = 1024;

__device__ __forceinline__ uint64_t splitmix64(uint64_t& s)
{
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t draw_below(uint64_t& s, int64_t n)
{
    return (int64_t)(((splitmix64(s) >> 32) * (uint64_t)n) >> 32);
}

struct PlaceArgs {
    int nx, ny, nz, d, kind;
    int r_min, r_max, hydro_q8, buf;
    long long N, fluid_target, max_rej, disk_cap;
    uint64_t seed;
};

__global__ void __launch_bounds__(kGeoThreads) k_place(PlaceArgs a, uint8_t* __restrict__ mask,
                                                       int32_t* __restrict__ disks, int64_t* __restrict__ info)
{
    __shared__ long long s_solid, s_rej, s_count, s_grains;
    __shared__ unsigned long long s_added;
    __shared__ long long s_c[4];
    __shared__ int s_go, s_ok;
    __shared__ uint64_t s_rng;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_rng = a.seed;
        s_solid = 0;
        s_rej = 0;
        s_count = 0;
        s_grains = 0;
        s_added = 0;
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            s_go = (a.N - s_solid > a.fluid_target) && (s_rej < a.max_rej);
            if (s_go) {
                uint64_t st = s_rng;
                const long long cx = draw_below(st, 256LL * a.nx);
                const long long cy = draw_below(st, 256LL * a.ny);
                const long long cz = a.d == 3 ? draw_below(st, 256LL * a.nz) : 0;
                const long long r = 256LL * a.r_min + draw_below(st, 256LL * (a.r_max - a.r_min) + 1);
                s_rng = st;
                s_c[0] = cx;
                s_c[1] = cy;
                s_c[2] = cz;
                s_c[3] = r;
                s_ok = (cx - r > 256LL * (a.buf - 1)) && (cx + r < 256LL * (a.nx - a.buf));
                if (s_ok && a.kind == LBM_GEOM_DISKS && s_count >= a.disk_cap) s_go = 0;
            }
        }
        __syncthreads();
        if (!s_go) break;
        const long long cx = s_c[0], cy = s_c[1], cz = s_c[2], r = s_c[3];
        int conflict = 0;
        if (s_ok && a.kind == LBM_GEOM_DISKS) {
            const long long cnt = s_count;
            for (long long k = tid; k < cnt && !conflict; k += blockDim.x) {
                const long long dx = cx - disks[3 * k], dy = cy - disks[3 * k + 1];
                const long long sr = r + disks[3 * k + 2] + 256;
                if (dx * dx + dy * dy < sr * sr) conflict = 1;
            }
        }
        conflict = __syncthreads_or(conflict);
        if (!s_ok || conflict) {
            if (tid == 0) ++s_rej;
            __syncthreads();
            continue;
        }
        // stamp the grain's voxels (each node of the bounding box has one owner)
        const long long rv = (r * a.hydro_q8) >> 8;
        const long long r2 = rv * rv;
        const int x0 = max(0LL, (cx - rv) >> 8), x1 = min((long long)a.nx - 1, (cx + rv) >> 8);
        const int y0 = max(0LL, (cy - rv) >> 8), y1 = min((long long)a.ny - 1, (cy + rv) >> 8);
        int z0 = 0, z1 = 0;
        if (a.d == 3) {
            z0 = (int)max(0LL, (cz - rv) >> 8);
            z1 = (int)min((long long)a.nz - 1, (cz + rv) >> 8);
        }
        unsigned long long added = 0;
        if (x1 >= x0 && y1 >= y0 && z1 >= z0) {
            const long long bx = x1 - x0 + 1, by = y1 - y0 + 1, bz = z1 - z0 + 1;
            for (long long c = tid; c < bx * by * bz; c += blockDim.x) {
                const int x = x0 + (int)(c % bx), y = y0 + (int)((c / bx) % by), z = z0 + (int)(c / (bx * by));
                const long long dx = 256LL * x - cx, dy = 256LL * y - cy, dz = a.d == 3 ? 256LL * z - cz : 0;
                if (dx * dx + dy * dy + dz * dz <= r2) {
                    const long long n = ((long long)z * a.ny + y) * a.nx + x;
                    if (!mask[n]) {
                        mask[n] = 1;
                        ++added;
                    }
                }
            }
        }
        if (added) atomicAdd(&s_added, added);
        __syncthreads();
        if (tid == 0) {
            if (a.kind == LBM_GEOM_DISKS) {
                disks[3 * s_count] = (int32_t)cx;
                disks[3 * s_count + 1] = (int32_t)cy;
                disks[3 * s_count + 2] = (int32_t)r;
                ++s_count;
            }
            ++s_grains;
            s_solid += (long long)s_added;
            s_rej = s_added > 0 ? 0 : s_rej + 1;
            s_added = 0;
        }
        __syncthreads();
    }
    if (tid == 0) {
        info[0] = s_grains;
        info[1] = s_solid;
    }
}

// User mask: normalise to 0/1 and count solids.
__global__ void k_normalise_mask(uint8_t* __restrict__ mask, long long N, unsigned long long* __restrict__ solid)
{
    unsigned long long c = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        if (mask[n]) {
            mask[n] = 1;
            ++c;
        }
    if (c) atomicAdd(solid, c);
}

// Level-synchronous BFS from the inlet plane; visited fluid is marked 2.
__global__ void __launch_bounds__(kGeoThreads) k_bfs(uint8_t* __restrict__ mask, uint32_t* __restrict__ queue, int nx,
                                                     int ny, int nz, int d)
{
    __shared__ unsigned long long s_tail, s_end;
    const int tid = threadIdx.x;
    if (tid == 0) s_tail = 0;
    __syncthreads();
    for (long long c = tid; c < (long long)ny * nz; c += blockDim.x) {
        const long long n = c * nx;  // x = 0
        if (mask[n] == 0) {
            mask[n] = 2;
            queue[atomicAdd(&s_tail, 1ull)] = (uint32_t)n;
        }
    }
    __syncthreads();
    unsigned long long head = 0;
    for (;;) {
        if (tid == 0) s_end = s_tail;
        __syncthreads();
        const unsigned long long end = s_end;
        if (head == end) break;
        for (unsigned long long i = head + tid; i < end; i += blockDim.x) {
            const long long n = queue[i];
            const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
            for (int k = 0; k < 2 * d; ++k) {
                int xx = x, yy = y, zz = z;
                if (k == 0) ++xx;
                else if (k == 1) --xx;
                else if (k == 2) ++yy;
                else if (k == 3) --yy;
                else if (k == 4) ++zz;
                else --zz;
                if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                const long long m = ((long long)zz * ny + yy) * nx + xx;
                if (mask[m] != 0) continue;  // solid (never changes) or already visited
                unsigned int* word = reinterpret_cast<unsigned int*>(mask + (m & ~3LL));
                const unsigned int shift = 8u * (unsigned int)(m & 3);
                const unsigned int old = atomicOr(word, 2u << shift);
                if (((old >> shift) & 0xFFu) == 0u) queue[atomicAdd(&s_tail, 1ull)] = (uint32_t)m;
            }
        }
        head = end;
        __syncthreads();
    }
}

// 0 (unreached fluid) -> 1 (filled), 2 (reached) -> 0.
__global__ void k_fill_finalise(uint8_t* __restrict__ mask, long long N, unsigned long long* __restrict__ filled)
{
    unsigned long long c = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const uint8_t b = mask[n];
        if (b == 0) {
            mask[n] = 1;
            ++c;
        } else if (b == 2) {
            mask[n] = 0;
        }
    }
    if (c) atomicAdd(filled, c);
}

template <int Q>
__global__ void k_links(const uint8_t* __restrict__ mask, uint32_t* __restrict__ link, int nx, int ny, int nz,
                        int periodic_y, unsigned long long* __restrict__ fluid)
{
    using L = Lattice<Q>;
    const long long N = (long long)nx * ny * nz;
    unsigned long long c = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        if (mask[n]) {
            link[n] = kLinkSolid;
            continue;
        }
        ++c;
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
        uint32_t w = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sx = x - L::c(i, 0), sz = z - L::c(i, 2);
            int sy = y - L::c(i, 1);
            if (periodic_y) sy = (sy + ny) % ny;  // sy is in -1..ny
            if (sy < 0 || sy >= ny || sz < 0 || sz >= nz)
                w |= 1u << i;
            else if (sx >= 0 && sx < nx && mask[((long long)sz * ny + sy) * nx + sx])
                w |= 1u << i;
        }
        link[n] = w;
    }
    if (c) atomicAdd(fluid, c);
}

__global__ void k_geometry_info(int64_t* __restrict__ info, long long N, double* __restrict__ porosity)
{
    if (porosity) *porosity = (double)info[3] / (double)N;
}

}  // namespace

lbm_status geometry_launch(const PlanInfo& p, const lbm_geom_desc& g, uint8_t* mask, uint32_t* link,
                           double* porosity, int64_t* info, cudaStream_t s)
{
    const long long N = p.geo.N;
    const int nx = p.geo.nx, ny = p.geo.ny, nz = p.geo.nz;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(info);
    cudaError_t e = cudaMemsetAsync(info, 0, 4 * sizeof(int64_t), s);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
    if (g.kind == LBM_GEOM_MASK) {
        k_normalise_mask<<<blocks, 256, 0, s>>>(mask, N, cnt + 1);
    } else {
        if ((e = cudaMemsetAsync(mask, 0, (size_t)N, s)) != cudaSuccess) return LBM_ERR_CUDA;
        if (g.kind == LBM_GEOM_DISKS || g.kind == LBM_GEOM_SPHERES) {
            PlaceArgs a;
            a.nx = nx;
            a.ny = ny;
            a.nz = nz;
            a.d = p.d;
            a.kind = g.kind;
            a.r_min = g.r_min;
            a.r_max = g.r_max;
            a.hydro_q8 = g.hydro_q8;
            a.buf = g.inlet_buffer;
            a.N = N;
            a.fluid_target = (long long)(g.target_porosity * (double)N);
            a.max_rej = g.max_rejections;
            a.disk_cap = N / 3;
            a.seed = g.seed;
            k_place<<<1, kGeoThreads, 0, s>>>(a, mask, reinterpret_cast<int32_t*>(link), info);
        }
    }
    if (g.fill_isolated) {
        k_bfs<<<1, kGeoThreads, 0, s>>>(mask, link, nx, ny, nz, p.d);
        k_fill_finalise<<<blocks, 256, 0, s>>>(mask, N, cnt + 2);
    }
    if (p.q == 9)
        k_links<9><<<blocks, 256, 0, s>>>(mask, link, nx, ny, nz, p.geo.periodic_y, cnt + 3);
    else
        k_links<19><<<blocks, 256, 0, s>>>(mask, link, nx, ny, nz, p.geo.periodic_y, cnt + 3);
    k_geometry_info<<<1, 1, 0, s>>>(info, N, porosity);
    return cuda_status(cudaGetLastError());
}

}  // namespace lbm
