// TMA-staged stream-collide and adjoint kernels (FP32, D2Q9 and D3Q19).
//
// Same arithmetic as the register kernels (Eq. 1-6 of arXiv 2310.00810 and
// their transpose, through nodes.cuh); what changes is how populations reach
// the SM.  A persistent CTA walks its share of the lattice tile by tile.  One
// producer thread issues, per tile and per direction i, one tensor-memory-
// accelerator copy (cp.async.bulk.tensor) of the box of post-collision
// populations that the tile pulls from (rows shifted by -c_i, four columns of
// halo each side so the box starts 16-byte aligned), into a ring of shared-
// memory stages guarded by mbarriers.  256 consumer threads (4 nodes each)
// read their shifted values from shared memory, apply the boundary rules,
// collide and store straight to global memory.  The bytes in flight are held
// by the copy engine instead of registers, several tiles ahead, which is what
// keeps HBM busy.  Copies that fall outside the lattice are zero-filled by
// the hardware; those links are bounce-back or Eq. 6 links and are replaced.
//
// Every mbarrier wait is bounded in time (%globaltimer; Bc::wait_us): on
// timeout the kernel latches LBM_ERR_TIMEOUT in the status word, raises the
// CTA's abort flag and returns, after the producer has waited for the copies
// it already issued to land (a CTA never exits with a bulk copy still
// writing into its shared memory).  A kernel that starts with
// LBM_ERR_TIMEOUT already latched returns at once, so one wait that gave up
// costs a sweep one wait limit, not one per launch.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "nodes.cuh"

namespace lbm {

namespace {

constexpr uint32_t kPollCap = 1u << 30;            // backstop on the polls of one wait
constexpr uint64_t kDrainNs = 1000000000ull;       // bound of the wait for issued copies before exit (1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on one mbarrier phase: false once limit_ns has elapsed (then
// LBM_ERR_TIMEOUT is latched and the CTA's abort flag raised) or when another
// thread of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status, volatile int* abort,
                                          uint64_t limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < kPollCap; it += 32) {
#pragma unroll 1
        for (int j = 0; j < 32; ++j)
            if (mbar_test(bar, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > limit_ns) break;
    }
    atomicOr(status, 1u << LBM_ERR_TIMEOUT);
    *abort = 1;
    return false;
}

// Producer epilogue: waits until the copies of the last issued tiles (tile j
// completes phase j / stages of full[j % stages]) have landed, so that no
// bulk copy is still writing into this CTA's shared memory when it exits.
// Copies complete in microseconds; the bound only guards a broken memory
// system.
__device__ __forceinline__ void drain_copies(uint64_t* full, int stages, int issued)
{
    for (int j = issued > stages ? issued - stages : 0; j < issued; ++j) {
        const uint64_t t0 = global_ns();
        while (!mbar_test(&full[j % stages], (uint32_t)(j / stages) & 1u))
            if (global_ns() - t0 > kDrainNs) break;
    }
}

// 1 when a bounded wait of an earlier launch gave up (LBM_ERR_TIMEOUT latched
// and not yet read by lbm_get_status): the launch then does nothing.
__device__ __forceinline__ int timeout_latched(const uint32_t* status)
{
    return (int)((*reinterpret_cast<const volatile uint32_t*>(status) >> LBM_ERR_TIMEOUT) & 1u);
}

__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                          int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Tile shapes (nodes) and pipeline depth.  The forward kernel stages Q boxes
// per tile, the adjoint 2Q (post-collision state and lambda).
template <int Q>
struct FwdTile;
template <>
struct FwdTile<9> {
    static constexpr int TX = 128, TY = 8, TZ = 1, STAGES = 4, ARRAYS = 1;
};
template <>
struct FwdTile<19> {
    static constexpr int TX = 64, TY = 4, TZ = 4, STAGES = 2, ARRAYS = 1;
};
template <int Q>
struct AdjTile;
template <>
struct AdjTile<9> {
    static constexpr int TX = 128, TY = 4, TZ = 1, STAGES = 3, ARRAYS = 2;
};
template <>
struct AdjTile<19> {
    static constexpr int TX = 32, TY = 4, TZ = 4, STAGES = 2, ARRAYS = 2;
};

template <int Q, class C>
struct Shape {
    static constexpr int BW = C::TX + 8;            // box row length (floats): 4 halo columns each side
    static constexpr int BOX = BW * C::TY * C::TZ;  // floats per box
    static constexpr int GX = C::TX / 4;            // 4-node groups per row
    static constexpr int NCONS = GX * C::TY * C::TZ;
    static constexpr size_t STAGE_FLOATS = (size_t)C::ARRAYS * Q * BOX;
    static constexpr size_t SMEM = C::STAGES * STAGE_FLOATS * 4 + 2 * C::STAGES * sizeof(uint64_t);
};

static_assert((Shape<9, FwdTile<9>>::BOX * 4) % 128 == 0 && (Shape<19, FwdTile<19>>::BOX * 4) % 128 == 0 &&
                  (Shape<9, AdjTile<9>>::BOX * 4) % 128 == 0 && (Shape<19, AdjTile<19>>::BOX * 4) % 128 == 0,
              "TMA shared-memory destinations must be 128-byte aligned");
static_assert(Shape<9, FwdTile<9>>::SMEM <= 227 * 1024 && Shape<19, FwdTile<19>>::SMEM <= 227 * 1024 &&
                  Shape<9, AdjTile<9>>::SMEM <= 227 * 1024 && Shape<19, AdjTile<19>>::SMEM <= 227 * 1024,
              "shared memory per CTA");

// The 4 values a group receives from a box row: columns shifted by -sx.
template <int BW>
__device__ __forceinline__ void read_box(float (&o)[4], const float* box, int r, int gx, int sx)
{
    const float* p = box + r * BW + 4 + 4 * gx;
    if (sx == 0) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w;
    } else if (sx == 1) {  // from x - 1
        const float4 a = *reinterpret_cast<const float4*>(p - 4), b = *reinterpret_cast<const float4*>(p);
        o[0] = a.w, o[1] = b.x, o[2] = b.y, o[3] = b.z;
    } else {  // from x + 1
        const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
        o[0] = a.y, o[1] = a.z, o[2] = a.w, o[3] = b.x;
    }
}

// True when the lane's 4 nodes and those of the lane beside it (the other
// half of the same 32-byte sector, rows of a multiple of 8 nodes) are all
// solid: the pair then skips its stores.  Solid nodes carry no populations;
// skipping whole sectors never leaves one partly written, which DRAM would
// have to read back and merge.
__device__ __forceinline__ bool sector_solid(const uint32_t (&lw)[4], bool live)
{
    const bool mine = !live || ((lw[0] & lw[1] & lw[2] & lw[3]) & kLinkSolid);
    const bool other = __shfl_xor_sync(0xffffffffu, mine, 1);
    return mine && other;
}

struct TileGrid {
    int ntx, nty, ntz, total;
};

__device__ __forceinline__ TileGrid tile_grid(const Geo& g, int tx, int ty, int tz)
{
    TileGrid t;
    t.ntx = (g.nx + tx - 1) / tx;
    t.nty = (g.ny + ty - 1) / ty;
    t.ntz = (g.nz + tz - 1) / tz;
    t.total = t.ntx * t.nty * t.ntz;
    return t;
}

template <int Q, int MODE>
__global__ void __launch_bounds__(Shape<Q, FwdTile<Q>>::NCONS + 32, 1)
    k_step_tma(const __grid_constant__ CUtensorMap map, const float* __restrict__ src, float* __restrict__ dst,
               Geo g, Bc bc, const double* __restrict__ tau)
{
    pdl_enter();
    using C = FwdTile<Q>;
    using S = Shape<Q, C>;
    using L = Lattice<Q>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* boxes = reinterpret_cast<float*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * S::STAGE_FLOATS * 4);
    uint64_t* empty = full + C::STAGES;
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const TileGrid tg = tile_grid(g, C::TX, C::TY, C::TZ);
    if (tid == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], S::NCONS / 32);
        }
        s_abort = timeout_latched(bc.status);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort = &s_abort;
    if (*abort) return;  // uniform: every thread read the same flag after the barrier
    const uint64_t wait_ns = (uint64_t)bc.wait_us * 1000ull;

    if (tid >= S::NCONS) {  // producer warp: one thread issues the copies
        if (tid == S::NCONS) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
            int k = 0;
            const int n_tiles = bc.test_stall ? 0 : tg.total;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
                const int s = k % C::STAGES;
                if (k >= C::STAGES && !mbar_wait(&empty[s], ((k / C::STAGES) - 1) & 1, bc.status, abort, wait_ns)) break;
                const int x0 = (t % tg.ntx) * C::TX, y0 = ((t / tg.ntx) % tg.nty) * C::TY,
                          z0 = (t / (tg.ntx * tg.nty)) * C::TZ;
                mbar_expect_tx(&full[s], (uint32_t)(Q * S::BOX * 4));
                float* st = boxes + s * S::STAGE_FLOATS;
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    tma_load4(st + i * S::BOX, &map, &full[s], x0 - 4, y0 - L::c(i, 1), z0 - L::c(i, 2), i);
            }
            drain_copies(full, C::STAGES, k);
        }
        return;
    }

    const float omega = 1.0f / (float)*tau;
    const int gx = tid % S::GX, gy = (tid / S::GX) % C::TY, gz = tid / (S::GX * C::TY);
    const int r = gz * C::TY + gy;
    int k = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, ++k) {
        const int s = k % C::STAGES;
        const bool ok = mbar_wait(&full[s], (k / C::STAGES) & 1, bc.status, abort, wait_ns);
        if (!__all_sync(0xffffffffu, ok)) break;
        const int x = (t % tg.ntx) * C::TX + 4 * gx, y = ((t / tg.ntx) % tg.nty) * C::TY + gy,
                  z = (t / (tg.ntx * tg.nty)) * C::TZ + gz;
        const float* st = boxes + s * S::STAGE_FLOATS;
        float v[Q][4];
#pragma unroll
        for (int i = 0; i < Q; ++i) read_box<S::BW>(v[i], st + i * S::BOX, r, gx, L::c(i, 0));
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        if (x < g.nx && y < g.ny && z < g.nz) {
            const long long n0 = ((long long)z * g.ny + y) * g.nx + x;
            uint32_t lw[4];
            load_links<4>(lw, g.link, n0, true);
            pull_fixup<Q, float, 4>(v, src, n0, x, y, z, lw, g, bc);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (lw[j] & kLinkSolid) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) v[i][j] = 0.0f;
                } else if (MODE != kStreamOnly) {
                    float a[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) a[i] = v[i][j];
                    collide<Q, float>(a, omega);
#pragma unroll
                    for (int i = 0; i < Q; ++i) v[i][j] = a[i];
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) Vec<float, 4>::store(dst + (long long)i * g.N + n0, v[i]);
        }
    }
}

// D2Q9 stream-collide, second form: every direction's box covers the tile
// rows plus one halo row above and below (same origin for all nine), so a
// node's pulled values AND its own values (bounce-back, Eq. 6) are all in
// shared memory; the link words arrive by TMA as well.  Consumer threads
// then touch global memory only to store their results.
template <int TY_, int STAGES_>
struct Halo2DT {
    static constexpr int TX = 128, TY = TY_, STAGES = STAGES_;
    static constexpr int BW = TX + 8, BH = TY + 2;
    static constexpr int BOX = ((BW * BH + 31) / 32) * 32;  // floats per direction box, padded to 128 B
    static constexpr int LINKS = TX * TY;                    // link words per tile
    static constexpr int GX = TX / 4;
    static constexpr int NCONS = GX * TY;    // 256 consumer threads, 4 nodes each
    static constexpr size_t STAGE_BYTES = (size_t)9 * BOX * 4 + (size_t)LINKS * 4;
    static constexpr uint32_t TX_BYTES = 9 * BW * BH * 4 + LINKS * 4;  // bytes the copies deliver (no padding)
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + 2 * STAGES * sizeof(uint64_t);
};
using Halo2D8 = Halo2DT<8, 4>;
using Halo2D4 = Halo2DT<4, 6>;
// One stage for lattices of at most one tile per SM (nothing to pipeline):
// a quarter of the shared memory, so the next kernel's CTAs can become
// resident beside these ones and wait at griddepcontrol.wait instead of
// being scheduled after them.
using Halo2D8x1 = Halo2DT<8, 1>;
using Halo2D4x1 = Halo2DT<4, 1>;
// every TMA destination (each box, the link box, each stage) starts on 128 bytes
static_assert((Halo2D8::BOX * 4) % 128 == 0 && (Halo2D8::LINKS * 4) % 128 == 0 && Halo2D8::STAGE_BYTES % 128 == 0,
              "TMA shared-memory destinations must be 128-byte aligned");
static_assert((Halo2D4::BOX * 4) % 128 == 0 && (Halo2D4::LINKS * 4) % 128 == 0 && Halo2D4::STAGE_BYTES % 128 == 0,
              "TMA shared-memory destinations must be 128-byte aligned");
static_assert(Halo2D8::SMEM <= 227 * 1024 && Halo2D4::SMEM <= 227 * 1024, "shared memory per CTA");

template <class H, int MODE>
__global__ void __launch_bounds__(H::NCONS + 32, 1)
    k_step_tma_halo(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map_link,
                    float* __restrict__ dst, Geo g, Bc bc, const double* __restrict__ tau)
{
    pdl_enter();
    using L = Lattice<9>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + H::STAGES * H::STAGE_BYTES);
    uint64_t* empty = full + H::STAGES;
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const TileGrid tg = tile_grid(g, H::TX, H::TY, 1);
    if (tid == 0) {
        for (int s = 0; s < H::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], H::NCONS / 32);
        }
        s_abort = timeout_latched(bc.status);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort = &s_abort;
    if (*abort) return;  // uniform: every thread read the same flag after the barrier
    const uint64_t wait_ns = (uint64_t)bc.wait_us * 1000ull;

    if (tid >= H::NCONS) {
        if (tid == H::NCONS) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_link)) : "memory");
            int k = 0;
            const int n_tiles = bc.test_stall ? 0 : tg.total;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
                const int s = k % H::STAGES;
                if (k >= H::STAGES && !mbar_wait(&empty[s], ((k / H::STAGES) - 1) & 1, bc.status, abort, wait_ns)) break;
                const int x0 = (t % tg.ntx) * H::TX, y0 = (t / tg.ntx) * H::TY;
                unsigned char* st = smem + s * H::STAGE_BYTES;
                mbar_expect_tx(&full[s], H::TX_BYTES);
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    tma_load4(st + (size_t)i * H::BOX * 4, &map, &full[s], x0 - 4, y0 - 1, 0, i);
                tma_load3(st + (size_t)9 * H::BOX * 4, &map_link, &full[s], x0, y0, 0);
            }
            drain_copies(full, H::STAGES, k);
        }
        return;
    }

    const float omega = 1.0f / (float)*tau;
    const int gx = tid % H::GX, gy = tid / H::GX;
    int k = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, ++k) {
        const int s = k % H::STAGES;
        const bool ok = mbar_wait(&full[s], (k / H::STAGES) & 1, bc.status, abort, wait_ns);
        if (!__all_sync(0xffffffffu, ok)) break;
        const int x = (t % tg.ntx) * H::TX + 4 * gx, y = (t / tg.ntx) * H::TY + gy;
        const unsigned char* st = smem + s * H::STAGE_BYTES;
        const float* bx = reinterpret_cast<const float*>(st);
        float v[9][4], own[9][4];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            read_box<H::BW>(v[i], bx + i * H::BOX, gy + 1 - L::c(i, 1), gx, L::c(i, 0));
            read_box<H::BW>(own[i], bx + i * H::BOX, gy + 1, gx, 0);
        }
        const uint4 lq = *reinterpret_cast<const uint4*>(st + (size_t)9 * H::BOX * 4 + (size_t)(gy * H::TX + 4 * gx) * 4);
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        const uint32_t lw[4] = {lq.x, lq.y, lq.z, lq.w};
        const bool live = x < g.nx && y < g.ny;
        const bool skip = g.skip_sectors && sector_solid(lw, live);
        if (live && !skip) {
            pull_fixup_own<9, float, 4>(v, own, x, y, 0, lw, g, bc);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (lw[j] & kLinkSolid) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) v[i][j] = 0.0f;
                } else if (MODE != kStreamOnly) {
                    float a[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) a[i] = v[i][j];
                    collide<9, float>(a, omega);
#pragma unroll
                    for (int i = 0; i < 9; ++i) v[i][j] = a[i];
                }
            }
            const long long n0 = (long long)y * g.nx + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) Vec<float, 4>::store(dst + (long long)i * g.N + n0, v[i]);
        }
    }
}

// D2Q9 stream-collide, two time steps per launch (temporal blocking, for
// lattices whose state stays in L2, where a launch costs more than the bytes
// it moves).  Per tile: TMA brings g^{t-1} over the tile plus two halo rows
// and four halo columns on each side (x from x0 - 4 keeps the copy 16-byte
// aligned) and the link words over the same box.  Step 1 computes g^t node by
// node over the tile plus one halo node on each side into shared memory;
// step 2 computes g^{t+1} on the tile with the 4-wide code of the one-step
// kernel, reading g^t from shared memory.  mid (nullable) also receives g^t
// on the tile (a checkpoint or a segment state).  The halo nodes of step 1
// are computed again by the neighbouring tiles: each step is the one-step
// kernel's arithmetic, so the result is the one-step sweep's.
template <int TY_>
struct Halo2x {
    static constexpr int TX = 128, TY = TY_;
    static constexpr int BW = TX + 8, BH = TY + 4;            // input box: x0 - 4 .. x0 + TX + 4, y0 - 2 .. y0 + TY + 2
    static constexpr int BOX = ((BW * BH + 31) / 32) * 32;    // floats per direction, padded to 128 B
    static constexpr int MH = TY + 2;                         // g^t rows: y0 - 1 .. y0 + TY
    static constexpr int MBOX = ((BW * MH + 31) / 32) * 32;   // floats per direction of g^t (same columns)
    static constexpr int LINKS = BW * BH;                     // link words of the box
    static constexpr int GX = TX / 4;
    static constexpr int NCONS = GX * TY;                     // threads: 4 nodes each in step 2
    static constexpr int MID_NODES = (TX + 2) * MH;           // step-1 nodes: x0 - 1 .. x0 + TX, MH rows
    static constexpr size_t IN_BYTES = (size_t)9 * BOX * 4;
    static constexpr size_t LINK_BYTES = (((size_t)LINKS * 4 + 127) / 128) * 128;
    static constexpr size_t MID_BYTES = (size_t)9 * MBOX * 4;
    static constexpr uint32_t TX_BYTES = 9 * BW * BH * 4 + LINKS * 4;  // bytes the copies deliver
    static constexpr size_t SMEM = IN_BYTES + LINK_BYTES + MID_BYTES + 16;
};
using Halo2x8 = Halo2x<8>;
using Halo2x4 = Halo2x<4>;
static_assert((Halo2x8::BOX * 4) % 128 == 0 && Halo2x8::IN_BYTES % 128 == 0 && Halo2x8::LINK_BYTES % 128 == 0 &&
                  (Halo2x8::MBOX * 4) % 16 == 0 && (Halo2x8::BW * 4) % 16 == 0,
              "TMA destinations 128-byte aligned, float4 rows");
static_assert(Halo2x8::SMEM <= 227 * 1024 && Halo2x4::SMEM <= 227 * 1024, "shared memory per CTA");

template <class H>
__global__ void __launch_bounds__(H::NCONS, 1)
    k_step2_tma_halo(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map_link,
                     float* __restrict__ dst, float* __restrict__ mid, Geo g, Bc bc, const double* __restrict__ tau)
{
    pdl_enter();
    using L = Lattice<9>;
    extern __shared__ __align__(128) unsigned char smem[];
    const float* box = reinterpret_cast<const float*>(smem);                                 // g^{t-1}, [9][BH][BW]
    const uint32_t* lnk = reinterpret_cast<const uint32_t*>(smem + H::IN_BYTES);            // [BH][BW]
    float* M = reinterpret_cast<float*>(smem + H::IN_BYTES + H::LINK_BYTES);                // g^t, [9][MH][BW]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + H::IN_BYTES + H::LINK_BYTES + H::MID_BYTES);
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const TileGrid tg = tile_grid(g, H::TX, H::TY, 1);
    if (tid == 0) {
        mbar_init(bar, 1);
        s_abort = timeout_latched(bc.status);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort = &s_abort;
    if (*abort) return;  // uniform: every thread read the same flag after the barrier
    const uint64_t wait_ns = (uint64_t)bc.wait_us * 1000ull;
    if (tid == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_link)) : "memory");
    }
    const float omega = 1.0f / (float)*tau;
    int issued = 0;
    int k = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, ++k) {
        const int x0 = (t % tg.ntx) * H::TX, y0 = (t / tg.ntx) * H::TY;
        if (tid == 0 && !bc.test_stall) {
            mbar_expect_tx(bar, H::TX_BYTES);
#pragma unroll
            for (int i = 0; i < 9; ++i)
                tma_load4(smem + (size_t)i * H::BOX * 4, &map, bar, x0 - 4, y0 - 2, 0, i);
            tma_load3(smem + H::IN_BYTES, &map_link, bar, x0 - 4, y0 - 2, 0);
            issued = k + 1;
        }
        const bool ok = mbar_wait(bar, (uint32_t)k & 1u, bc.status, abort, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain_copies(bar, 1, issued);
            return;
        }
        // step 1: g^t at x0 - 1 .. x0 + TX, y0 - 1 .. y0 + TY (box column bx = x - x0 + 4, box row by = y - y0 + 2)
        for (int m = tid; m < H::MID_NODES; m += H::NCONS) {
            const int mr = m / (H::TX + 2), mc = m % (H::TX + 2);
            const int x = x0 - 1 + mc, y = y0 - 1 + mr;
            const int bx = mc + 3, by = mr + 1;
            float* mo = M + (size_t)mr * H::BW + bx;
            if (x < 0 || x >= g.nx || y < 0 || y >= g.ny) continue;  // outside the lattice: never pulled
            const uint32_t lw1[1] = {lnk[by * H::BW + bx]};
            if (lw1[0] & kLinkSolid) {
#pragma unroll
                for (int i = 0; i < 9; ++i) mo[(size_t)i * H::MBOX] = 0.0f;
                continue;
            }
            float v[9][1], own[9][1];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float* bi = box + (size_t)i * H::BOX;
                v[i][0] = bi[(by - L::c(i, 1)) * H::BW + bx - L::c(i, 0)];
                own[i][0] = bi[by * H::BW + bx];
            }
            pull_fixup_own<9, float, 1>(v, own, x, y, 0, lw1, g, bc);
            float a[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i] = v[i][0];
            collide<9, float>(a, omega);
#pragma unroll
            for (int i = 0; i < 9; ++i) mo[(size_t)i * H::MBOX] = a[i];
        }
        __syncthreads();
        // step 2: g^{t+1} on the tile from g^t (rows of M start at y0 - 1, columns at x0 - 4)
        {
            const int gx = tid % H::GX, gy = tid / H::GX;
            const int x = x0 + 4 * gx, y = y0 + gy;
            float v[9][4], own[9][4];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                read_box<H::BW>(v[i], M + (size_t)i * H::MBOX, gy + 1 - L::c(i, 1), gx, L::c(i, 0));
                read_box<H::BW>(own[i], M + (size_t)i * H::MBOX, gy + 1, gx, 0);
            }
            const uint4 lq = *reinterpret_cast<const uint4*>(lnk + (gy + 2) * H::BW + 4 + 4 * gx);
            const uint32_t lw[4] = {lq.x, lq.y, lq.z, lq.w};
            const bool live = x < g.nx && y < g.ny;
            const bool skip = g.skip_sectors && sector_solid(lw, live);
            if (live && !skip) {
                const long long n0 = (long long)y * g.nx + x;
                if (mid) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) Vec<float, 4>::store(mid + (long long)i * g.N + n0, own[i]);
                }
                pull_fixup_own<9, float, 4>(v, own, x, y, 0, lw, g, bc);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (lw[j] & kLinkSolid) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) v[i][j] = 0.0f;
                    } else {
                        float a[9];
#pragma unroll
                        for (int i = 0; i < 9; ++i) a[i] = v[i][j];
                        collide<9, float>(a, omega);
#pragma unroll
                        for (int i = 0; i < 9; ++i) v[i][j] = a[i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) Vec<float, 4>::store(dst + (long long)i * g.N + n0, v[i]);
            }
        }
        __syncthreads();  // the next tile's copies overwrite the box and the link words
    }
}

// D2Q9 adjoint, halo form: per tile the nine boxes of g^{t-1} and the nine
// of lambda^{t+1}, each over the tile rows plus one halo row on each side, and
// the link words, so the pulls in both directions and every own value
// (bounce-back, Eq. 6) come from shared memory.
template <int TY_, int STAGES_>
struct HaloAdj2DT {
    static constexpr int TX = 128, TY = TY_, STAGES = STAGES_;
    static constexpr int BW = TX + 8, BH = TY + 2;
    static constexpr int BOX = ((BW * BH + 31) / 32) * 32;
    static constexpr int LINKS = TX * TY;
    static constexpr int GX = TX / 4;
    static constexpr int NCONS = GX * TY;
    static constexpr size_t STAGE_BYTES = (size_t)18 * BOX * 4 + (size_t)LINKS * 4;
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + 2 * STAGES * sizeof(uint64_t);
};
using HaloAdj2D8 = HaloAdj2DT<8, 2>;
using HaloAdj2D4 = HaloAdj2DT<4, 3>;
using HaloAdj2D8x1 = HaloAdj2DT<8, 1>;
using HaloAdj2D4x1 = HaloAdj2DT<4, 1>;
static_assert((HaloAdj2D8::BOX * 4) % 128 == 0 && HaloAdj2D8::STAGE_BYTES % 128 == 0 &&
                  (HaloAdj2D4::BOX * 4) % 128 == 0 && HaloAdj2D4::STAGE_BYTES % 128 == 0,
              "TMA shared-memory destinations must be 128-byte aligned");
static_assert(HaloAdj2D8::SMEM <= 227 * 1024 && HaloAdj2D4::SMEM <= 227 * 1024, "shared memory per CTA");

template <class H, bool T0>
__global__ void __launch_bounds__(H::NCONS + 32, 1)
    k_adjoint_tma_halo(const __grid_constant__ CUtensorMap map_g, const __grid_constant__ CUtensorMap map_l,
                       const __grid_constant__ CUtensorMap map_link, float* __restrict__ lam_out, Geo g, Bc bc,
                       const double* __restrict__ tau, double* __restrict__ grad_acc, double* __restrict__ partial)
{
    pdl_enter();
    using L = Lattice<9>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + H::STAGES * H::STAGE_BYTES);
    uint64_t* empty = full + H::STAGES;
    __shared__ int s_abort;
    __shared__ double s_part[H::NCONS / 32];
    const int tid = threadIdx.x;
    const TileGrid tg = tile_grid(g, H::TX, H::TY, 1);
    if (tid == 0) {
        for (int s = 0; s < H::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], H::NCONS / 32);
        }
        s_abort = timeout_latched(bc.status);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort = &s_abort;
    if (*abort) return;  // uniform: every thread read the same flag after the barrier
    const uint64_t wait_ns = (uint64_t)bc.wait_us * 1000ull;

    if (tid >= H::NCONS) {
        if (tid == H::NCONS) {
            if (!T0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_g)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_l)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_link)) : "memory");
            const uint32_t tx_bytes = (uint32_t)((T0 ? 9 : 18) * H::BW * H::BH * 4 + H::LINKS * 4);
            int k = 0;
            const int n_tiles = bc.test_stall ? 0 : tg.total;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
                const int s = k % H::STAGES;
                if (k >= H::STAGES && !mbar_wait(&empty[s], ((k / H::STAGES) - 1) & 1, bc.status, abort, wait_ns)) break;
                const int x0 = (t % tg.ntx) * H::TX, y0 = (t / tg.ntx) * H::TY;
                unsigned char* st = smem + s * H::STAGE_BYTES;
                mbar_expect_tx(&full[s], tx_bytes);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if (!T0) tma_load4(st + (size_t)i * H::BOX * 4, &map_g, &full[s], x0 - 4, y0 - 1, 0, i);
                    tma_load4(st + (size_t)(9 + i) * H::BOX * 4, &map_l, &full[s], x0 - 4, y0 - 1, 0, i);
                }
                tma_load3(st + (size_t)18 * H::BOX * 4, &map_link, &full[s], x0, y0, 0);
            }
            drain_copies(full, H::STAGES, k);
        }
        return;
    }

    const float omega = 1.0f / (float)*tau;
    const int gx = tid % H::GX, gy = tid / H::GX;
    float dom = 0.0f;
    int k = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, ++k) {
        const int s = k % H::STAGES;
        const bool ok = mbar_wait(&full[s], (k / H::STAGES) & 1, bc.status, abort, wait_ns);
        if (!__all_sync(0xffffffffu, ok)) break;
        const int x = (t % tg.ntx) * H::TX + 4 * gx, y = (t / tg.ntx) * H::TY + gy;
        const unsigned char* st = smem + s * H::STAGE_BYTES;
        const float* bg = reinterpret_cast<const float*>(st);
        const float* bl = bg + 9 * H::BOX;
        float f[9][4], own[9][4], mu[9][4], lown[9][4];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (T0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) f[i][j] = own[i][j] = 0.0f;
            } else {
                read_box<H::BW>(f[i], bg + i * H::BOX, gy + 1 - L::c(i, 1), gx, L::c(i, 0));
                read_box<H::BW>(own[i], bg + i * H::BOX, gy + 1, gx, 0);
            }
            read_box<H::BW>(mu[i], bl + i * H::BOX, gy + 1 + L::c(i, 1), gx, -L::c(i, 0));
            read_box<H::BW>(lown[i], bl + i * H::BOX, gy + 1, gx, 0);
        }
        const uint4 lq =
            *reinterpret_cast<const uint4*>(st + (size_t)18 * H::BOX * 4 + (size_t)(gy * H::TX + 4 * gx) * 4);
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        const uint32_t lw[4] = {lq.x, lq.y, lq.z, lq.w};
        const bool live = x < g.nx && y < g.ny;
        const bool skip = g.skip_sectors && sector_solid(lw, live);
        if (live && !skip) {
            if (!T0) pull_fixup_own<9, float, 4>(f, own, x, y, 0, lw, g, bc);
            const long long n0 = (long long)y * g.nx + x;
            dom += adjoint_nodes_own<9, float, 4>(f, mu, lown, n0, x, y, 0, lw, g, bc, omega, grad_acc);
#pragma unroll
            for (int i = 0; i < 9; ++i) Vec<float, 4>::store(lam_out + (long long)i * g.N + n0, mu[i]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dom += __shfl_xor_sync(0xffffffffu, dom, o);
    if ((tid & 31) == 0) s_part[tid >> 5] = (double)dom;
    asm volatile("bar.sync 1, %0;" ::"r"(H::NCONS) : "memory");  // consumers only
    if (tid == 0) {
        double b = 0.0;
#pragma unroll
        for (int w = 0; w < H::NCONS / 32; ++w) b += s_part[w];
        partial[blockIdx.x] += b;
    }
}

template <int Q, bool T0>
__global__ void __launch_bounds__(Shape<Q, AdjTile<Q>>::NCONS + 32, 1)
    k_adjoint_tma(const __grid_constant__ CUtensorMap map_g, const __grid_constant__ CUtensorMap map_l,
                  const float* __restrict__ gprev, const float* __restrict__ lam_in, float* __restrict__ lam_out,
                  Geo g, Bc bc, const double* __restrict__ tau, double* __restrict__ grad_acc,
                  double* __restrict__ partial)
{
    pdl_enter();
    using C = AdjTile<Q>;
    using S = Shape<Q, C>;
    using L = Lattice<Q>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* boxes = reinterpret_cast<float*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * S::STAGE_FLOATS * 4);
    uint64_t* empty = full + C::STAGES;
    __shared__ int s_abort;
    __shared__ double s_part[S::NCONS / 32];
    const int tid = threadIdx.x;
    const TileGrid tg = tile_grid(g, C::TX, C::TY, C::TZ);
    if (tid == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], S::NCONS / 32);
        }
        s_abort = timeout_latched(bc.status);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort = &s_abort;
    if (*abort) return;  // uniform: every thread read the same flag after the barrier
    const uint64_t wait_ns = (uint64_t)bc.wait_us * 1000ull;

    if (tid >= S::NCONS) {
        if (tid == S::NCONS) {
            if (!T0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_g)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_l)) : "memory");
            int k = 0;
            const int n_tiles = bc.test_stall ? 0 : tg.total;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
                const int s = k % C::STAGES;
                if (k >= C::STAGES && !mbar_wait(&empty[s], ((k / C::STAGES) - 1) & 1, bc.status, abort, wait_ns)) break;
                const int x0 = (t % tg.ntx) * C::TX, y0 = ((t / tg.ntx) % tg.nty) * C::TY,
                          z0 = (t / (tg.ntx * tg.nty)) * C::TZ;
                mbar_expect_tx(&full[s], (uint32_t)((T0 ? 1 : 2) * Q * S::BOX * 4));
                float* st = boxes + s * S::STAGE_FLOATS;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (!T0)
                        tma_load4(st + i * S::BOX, &map_g, &full[s], x0 - 4, y0 - L::c(i, 1), z0 - L::c(i, 2), i);
                    tma_load4(st + (Q + i) * S::BOX, &map_l, &full[s], x0 - 4, y0 + L::c(i, 1), z0 + L::c(i, 2), i);
                }
            }
            drain_copies(full, C::STAGES, k);
        }
        return;
    }

    const float omega = 1.0f / (float)*tau;
    const int gx = tid % S::GX, gy = (tid / S::GX) % C::TY, gz = tid / (S::GX * C::TY);
    const int r = gz * C::TY + gy;
    float dom = 0.0f;
    int k = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, ++k) {
        const int s = k % C::STAGES;
        const bool ok = mbar_wait(&full[s], (k / C::STAGES) & 1, bc.status, abort, wait_ns);
        if (!__all_sync(0xffffffffu, ok)) break;
        const int x = (t % tg.ntx) * C::TX + 4 * gx, y = ((t / tg.ntx) % tg.nty) * C::TY + gy,
                  z = (t / (tg.ntx * tg.nty)) * C::TZ + gz;
        const float* st = boxes + s * S::STAGE_FLOATS;
        float f[Q][4], mu[Q][4];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (T0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) f[i][j] = 0.0f;
            } else {
                read_box<S::BW>(f[i], st + i * S::BOX, r, gx, L::c(i, 0));
            }
            read_box<S::BW>(mu[i], st + (Q + i) * S::BOX, r, gx, -L::c(i, 0));
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        if (x < g.nx && y < g.ny && z < g.nz) {
            const long long n0 = ((long long)z * g.ny + y) * g.nx + x;
            uint32_t lw[4];
            load_links<4>(lw, g.link, n0, true);
            if (!T0) pull_fixup<Q, float, 4>(f, gprev, n0, x, y, z, lw, g, bc);
            dom += adjoint_nodes<Q, float, 4>(f, mu, lam_in, n0, x, y, z, lw, g, bc, omega, grad_acc);
#pragma unroll
            for (int i = 0; i < Q; ++i) Vec<float, 4>::store(lam_out + (long long)i * g.N + n0, mu[i]);
        }
    }
    // CTA sum of the dL/domega contributions: warps in FP32, warps combined in FP64
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dom += __shfl_xor_sync(0xffffffffu, dom, o);
    if ((tid & 31) == 0) s_part[tid >> 5] = (double)dom;
    asm volatile("bar.sync 1, %0;" ::"r"(S::NCONS) : "memory");  // consumers only
    if (tid == 0) {
        double b = 0.0;
#pragma unroll
        for (int w = 0; w < S::NCONS / 32; ++w) b += s_part[w];
        partial[blockIdx.x] += b;
    }
}

// ------------------------------------------------------------------- host

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(ptr);
    });
    return fn;
}

// 4D map over a population array [Q][nz][ny][nx] (float), box (bw, ty, tz, 1).
bool make_map(CUtensorMap* m, const void* base, const Geo& g, int q, int bw, int ty, int tz)
{
    EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)q};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4, (cuuint64_t)g.N * 4};
    const cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)ty, (cuuint32_t)tz, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D map over the link words [nz][ny][nx] (uint32), box (tx, ty, tz).
bool make_link_map(CUtensorMap* m, const void* base, const Geo& g, int tx, int ty, int tz)
{
    EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)tx, (cuuint32_t)ty, (cuuint32_t)tz};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

long long halo_tiles(const PlanInfo& p, int ty)
{
    return (long long)((p.geo.nx + 127) / 128) * ((p.geo.ny + ty - 1) / ty);
}

template <class K>
bool allow_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

bool tma_ok(const PlanInfo& p, const void* a, const void* b, const void* c)
{
    auto al = [](const void* ptr) { return ptr == nullptr || (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; };
    return p.use_tma && p.prec == 4 && p.geo.nx % 4 == 0 && al(a) && al(b) && al(c) &&
           (reinterpret_cast<uintptr_t>(p.geo.link) & 15u) == 0;
}

template <class H>
bool step_tma_halo(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                   cudaStream_t s)
{
    const long long tiles = (long long)((p.geo.nx + H::TX - 1) / H::TX) * ((p.geo.ny + H::TY - 1) / H::TY);
    if (tiles < (long long)p.tma_min_tiles) return false;
    CUtensorMap map, ml;
    if (!make_map(&map, src, p.geo, 9, H::BW, H::BH, 1)) return false;
    if (!make_link_map(&ml, p.geo.link, p.geo, H::TX, H::TY, 1)) return false;
    // one-stage kernels take one tile per CTA (several CTAs per SM overlap their load, compute and store
    // phases); multi-stage kernels are persistent, one CTA per SM
    const int grid = (int)(H::STAGES == 1 ? tiles : std::min<long long>(tiles, sm_count()));
    float* b = static_cast<float*>(dst);
    if (mode == kStreamCollide) {
        static bool ok = allow_smem(k_step_tma_halo<H, kStreamCollide>, H::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_step_tma_halo<H, kStreamCollide>, dim3(grid), dim3(H::NCONS + 32), H::SMEM, s, map, ml, b, p.geo, bc, tau);
    } else {
        static bool ok = allow_smem(k_step_tma_halo<H, kStreamOnly>, H::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_step_tma_halo<H, kStreamOnly>, dim3(grid), dim3(H::NCONS + 32), H::SMEM, s, map, ml, b, p.geo, bc, tau);
    }
    return true;
}

template <class H>
bool step2_tma_halo(const PlanInfo& p, const void* src, void* dst, void* mid, const Bc& bc, const double* tau,
                    cudaStream_t s)
{
    const long long tiles = (long long)((p.geo.nx + H::TX - 1) / H::TX) * ((p.geo.ny + H::TY - 1) / H::TY);
    CUtensorMap map, ml;
    if (!make_map(&map, src, p.geo, 9, H::BW, H::BH, 1)) return false;
    if (!make_link_map(&ml, p.geo.link, p.geo, H::BW, H::BH, 1)) return false;
    static bool ok = allow_smem(k_step2_tma_halo<H>, H::SMEM);
    if (!ok) return false;
    const int per_sm = std::max(1, (int)((227 * 1024) / H::SMEM));
    const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * per_sm);
    launch_k(p.pdl, k_step2_tma_halo<H>, dim3(grid), dim3(H::NCONS), H::SMEM, s, map, ml, static_cast<float*>(dst),
             static_cast<float*>(mid), p.geo, bc, tau);
    return true;
}

template <int Q>
bool step_tma(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
              cudaStream_t s)
{
    using C = FwdTile<Q>;
    using S = Shape<Q, C>;
    const long long tiles = (long long)((p.geo.nx + C::TX - 1) / C::TX) * ((p.geo.ny + C::TY - 1) / C::TY) *
                            ((p.geo.nz + C::TZ - 1) / C::TZ);
    if (tiles < (long long)p.tma_min_tiles) return false;
    CUtensorMap map;
    if (!make_map(&map, src, p.geo, Q, S::BW, C::TY, C::TZ)) return false;
    const int grid = (int)std::min<long long>(tiles, sm_count());
    const float* a = static_cast<const float*>(src);
    float* b = static_cast<float*>(dst);
    if (mode == kStreamCollide) {
        static bool ok = allow_smem(k_step_tma<Q, kStreamCollide>, S::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_step_tma<Q, kStreamCollide>, dim3(grid), dim3(S::NCONS + 32), S::SMEM, s, map, a, b, p.geo, bc, tau);
    } else {
        static bool ok = allow_smem(k_step_tma<Q, kStreamOnly>, S::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_step_tma<Q, kStreamOnly>, dim3(grid), dim3(S::NCONS + 32), S::SMEM, s, map, a, b, p.geo, bc, tau);
    }
    return true;
}

template <class H>
bool adjoint_tma_halo(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                      const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    const long long tiles = (long long)((p.geo.nx + H::TX - 1) / H::TX) * ((p.geo.ny + H::TY - 1) / H::TY);
    if (tiles < (long long)p.tma_min_tiles) return false;
    CUtensorMap mg, ml, mk;
    if (!make_map(&ml, lam_in, p.geo, 9, H::BW, H::BH, 1)) return false;
    if (t0) mg = ml;
    else if (!make_map(&mg, gprev, p.geo, 9, H::BW, H::BH, 1)) return false;
    if (!make_link_map(&mk, p.geo.link, p.geo, H::TX, H::TY, 1)) return false;
    const int grid = (int)std::min<long long>(H::STAGES == 1 ? tiles : std::min<long long>(tiles, sm_count()),
                                              p.n_partial);
    float* lo = static_cast<float*>(lam_out);
    if (t0) {
        static bool ok = allow_smem(k_adjoint_tma_halo<H, true>, H::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_adjoint_tma_halo<H, true>, dim3(grid), dim3(H::NCONS + 32), H::SMEM, s, mg, ml, mk, lo, p.geo, bc, tau, grad_acc,
                                                                      partial);
    } else {
        static bool ok = allow_smem(k_adjoint_tma_halo<H, false>, H::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_adjoint_tma_halo<H, false>, dim3(grid), dim3(H::NCONS + 32), H::SMEM, s, mg, ml, mk, lo, p.geo, bc, tau, grad_acc,
                                                                       partial);
    }
    return true;
}

template <int Q>
bool adjoint_tma(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                 const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    using C = AdjTile<Q>;
    using S = Shape<Q, C>;
    const long long tiles = (long long)((p.geo.nx + C::TX - 1) / C::TX) * ((p.geo.ny + C::TY - 1) / C::TY) *
                            ((p.geo.nz + C::TZ - 1) / C::TZ);
    if (tiles < (long long)p.tma_min_tiles) return false;
    CUtensorMap mg, ml;
    if (!make_map(&ml, lam_in, p.geo, Q, S::BW, C::TY, C::TZ)) return false;
    if (t0) mg = ml;
    else if (!make_map(&mg, gprev, p.geo, Q, S::BW, C::TY, C::TZ)) return false;
    const int grid = (int)std::min<long long>(std::min<long long>(tiles, sm_count()), p.n_partial);
    const float* gp = static_cast<const float*>(gprev);
    const float* li = static_cast<const float*>(lam_in);
    float* lo = static_cast<float*>(lam_out);
    if (t0) {
        static bool ok = allow_smem(k_adjoint_tma<Q, true>, S::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_adjoint_tma<Q, true>, dim3(grid), dim3(S::NCONS + 32), S::SMEM, s, mg, ml, gp, li, lo, p.geo, bc, tau, grad_acc,
                                                                     partial);
    } else {
        static bool ok = allow_smem(k_adjoint_tma<Q, false>, S::SMEM);
        if (!ok) return false;
        launch_k(p.pdl, k_adjoint_tma<Q, false>, dim3(grid), dim3(S::NCONS + 32), S::SMEM, s, mg, ml, gp, li, lo, p.geo, bc, tau, grad_acc,
                                                                      partial);
    }
    return true;
}

}  // namespace

bool step_launch_tma(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                     cudaStream_t s)
{
    if (mode == kCollideOnly || !tma_ok(p, src, dst, nullptr)) return false;
    if (p.q == 9 && p.tma_variant == 1) {
        const bool one = halo_tiles(p, p.tma_ty) <= (long long)p.tma_waves * sm_count();
        if (p.tma_ty == 4)
            return one ? step_tma_halo<Halo2D4x1>(p, mode, src, dst, bc, tau, s)
                       : step_tma_halo<Halo2D4>(p, mode, src, dst, bc, tau, s);
        return one ? step_tma_halo<Halo2D8x1>(p, mode, src, dst, bc, tau, s)
                   : step_tma_halo<Halo2D8>(p, mode, src, dst, bc, tau, s);
    }
    return p.q == 9 ? step_tma<9>(p, mode, src, dst, bc, tau, s) : step_tma<19>(p, mode, src, dst, bc, tau, s);
}

bool step2_launch_tma(const PlanInfo& p, const void* src, void* dst, void* mid, const Bc& bc, const double* tau,
                      cudaStream_t s)
{
    if (p.q != 9 || !tma_ok(p, src, dst, mid)) return false;
    return p.tma_ty == 4 ? step2_tma_halo<Halo2x4>(p, src, dst, mid, bc, tau, s)
                         : step2_tma_halo<Halo2x8>(p, src, dst, mid, bc, tau, s);
}

bool adjoint_launch_tma(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                        const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    if (!tma_ok(p, gprev, lam_in, lam_out)) return false;
    if (p.q == 9 && p.tma_variant == 1) {
        const bool one = halo_tiles(p, p.adj_tma_ty) <= (long long)p.tma_waves * sm_count();
        if (p.adj_tma_ty == 4)
            return one ? adjoint_tma_halo<HaloAdj2D4x1>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s)
                       : adjoint_tma_halo<HaloAdj2D4>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
        return one ? adjoint_tma_halo<HaloAdj2D8x1>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s)
                   : adjoint_tma_halo<HaloAdj2D8>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    }
    return p.q == 9 ? adjoint_tma<9>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s)
                    : adjoint_tma<19>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
}

}  // namespace lbm
