// Vectorised forward and adjoint step kernels: each thread owns VEC
// consecutive nodes of one row and moves every population plane with one
// VEC-wide (8- or 16-byte) coalesced load or store.  The +-1 x-shift of the
// pull is done in registers: a lane takes the neighbouring element from the
// lane beside it with a warp shuffle, and only the two lanes at the ends of a
// warp's row segment read one extra element.  Same arithmetic as step.cu /
// adjoint.cu (Eq. 1-6 of arXiv 2310.00810 and their transpose); the scalar
// kernels remain for rows whose length is not a multiple of VEC.
//
// Thread layout: blockDim = (32, kVecRows); a warp covers 32 * VEC nodes of
// one row (y, z), so row validity and shuffles are warp-uniform.
#include <algorithm>

#include "nodes.cuh"

namespace lbm {

// Minimum resident blocks per SM (register budget) for each instantiation,
// chosen from ptxas -v so that none of the hot variants spills.
template <int Q, typename T, int VEC>
constexpr int step_min_blocks()
{
    return Q == 9 ? (sizeof(T) == 8 ? 5 : (VEC == 4 ? 7 : 8)) : (sizeof(T) == 8 ? 3 : (VEC == 4 ? 3 : 4));
}
template <int Q, typename T, int VEC>
constexpr int adjoint_min_blocks()
{
    return Q == 9 ? (sizeof(T) == 8 ? 3 : (VEC == 4 ? 4 : 5)) : (sizeof(T) == 8 ? 2 : 3);
}

// Stream-collide with every load issued up front and independent of the
// link words: the VEC-wide pulled rows, the lane's own rows of all Q planes
// (for bounce-back and Eq. 6, mostly L1 hits: neighbouring warps of the block
// pull the same lines) and the link words.  One memory latency per thread.
template <int Q, typename T, int VEC, int MODE>
__global__ void __launch_bounds__(32 * kVecRows, (Q == 9 ? 4 : 2))
    k_step_own(const T* __restrict__ src, T* __restrict__ dst, Geo g, Bc bc, const double* __restrict__ tau)
{
    pdl_enter();
    using L = Lattice<Q>;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * kVecRows + threadIdx.y, z = blockIdx.z;
    if (y >= g.ny) return;  // warp-uniform
    const int x0w = blockIdx.x * 32 * VEC, x0 = x0w + lane * VEC;
    const bool live = x0 < g.nx;
    const long long N = g.N;
    const long long n0 = ((long long)z * g.ny + y) * g.nx + x0;
    uint32_t lw[VEC];
    load_links<VEC>(lw, g.link, n0, live);
    Need<VEC> all;
    all.sx0 = all.sxp = all.sxm = live;
    all.edge_p = lane == 0 && live;
    all.edge_m = lane == 31 && live;
    T v[Q][VEC], own[Q][VEC];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (live) {
            Vec<T, VEC>::load(src + (long long)i * N + n0, own[i]);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) own[i][j] = T(0);
        }
        if (MODE == kCollideOnly) continue;
        const int sy = y - L::c(i, 1), sz = z - L::c(i, 2);
        if (sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
            const T* rowp = src + (long long)i * N + ((long long)sz * g.ny + sy) * g.nx;
            load_shift<T, VEC>(v[i], L::c(i, 0), rowp, x0, x0w, g.nx, lane, all);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) v[i][j] = T(0);
        }
    }
    if (!live) return;
    if (MODE == kCollideOnly) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
            for (int j = 0; j < VEC; ++j) v[i][j] = own[i][j];
    } else {
        pull_fixup_own<Q, T, VEC>(v, own, x0, y, z, lw, g, bc);
    }
    if (MODE != kStreamOnly) {
        const T omega = T(1) / T(*tau);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            T a[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) a[i] = v[i][j];
            collide<Q, T>(a, omega);
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i][j] = a[i];
        }
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j)
        if (lw[j] & kLinkSolid)
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i][j] = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) Vec<T, VEC>::store(dst + (long long)i * N + n0, v[i]);
}

template <int Q, typename T, int VEC, int MODE>
__global__ void __launch_bounds__(32 * kVecRows, (step_min_blocks<Q, T, VEC>()))
    k_step_vec(const T* __restrict__ src, T* __restrict__ dst, Geo g, Bc bc, const double* __restrict__ tau)
{
    pdl_enter();
    const int lane = threadIdx.x;
    const int y = blockIdx.y * kVecRows + threadIdx.y, z = blockIdx.z;
    if (y >= g.ny) return;  // warp-uniform
    const int x0w = blockIdx.x * 32 * VEC, x0 = x0w + lane * VEC;
    const bool live = x0 < g.nx;
    const long long n0 = ((long long)z * g.ny + y) * g.nx + x0;
    uint32_t lw[VEC];
    load_links<VEC>(lw, g.link, n0, live);
    const unsigned fl = fluid_bits<VEC>(lw);
    T v[Q][VEC];
    if (MODE == kCollideOnly) {
        if (!live) return;
#pragma unroll
        for (int i = 0; i < Q; ++i) Vec<T, VEC>::load(src + (long long)i * g.N + n0, v[i]);
    } else {
        const Need<VEC> need = lane_needs<VEC>(fl, lane);
        pull_vec<Q, T, VEC>(v, src, n0, x0, x0w, y, z, lw, g, bc, lane, live, need);
        if (!live) return;  // all-solid lanes still store (zeros): a skipped store would leave
                            // 32-byte sectors partly written, which DRAM must read back to merge
    }
    if (MODE != kStreamOnly) {
        const T omega = T(1) / T(*tau);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            T a[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) a[i] = v[i][j];
            collide<Q, T>(a, omega);
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i][j] = a[i];
        }
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j)
        if (lw[j] & kLinkSolid)
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i][j] = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) Vec<T, VEC>::store(dst + (long long)i * g.N + n0, v[i]);
}

// Adjoint step, VEC nodes per thread (the algebra of adjoint.cu).
template <int Q, typename T, int VEC, bool T0>
__global__ void __launch_bounds__(32 * kVecRows, (adjoint_min_blocks<Q, T, VEC>()))
    k_adjoint_vec(const T* __restrict__ gprev, const T* __restrict__ lam_in, T* __restrict__ lam_out, Geo g, Bc bc,
                  const double* __restrict__ tau, double* __restrict__ grad_acc, double* __restrict__ partial)
{
    pdl_enter();
    using L = Lattice<Q>;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * kVecRows + threadIdx.y, z = blockIdx.z;
    const bool row = y < g.ny;
    const int x0w = blockIdx.x * 32 * VEC, x0 = x0w + lane * VEC;
    const bool live = row && x0 < g.nx;
    const long long N = g.N;
    const long long n0 = ((long long)z * g.ny + y) * g.nx + x0;
    T dom = T(0);
    if (row) {
        uint32_t lw[VEC];
        load_links<VEC>(lw, g.link, n0, live);
        const unsigned fl = fluid_bits<VEC>(lw);
        const Need<VEC> need = lane_needs<VEC>(fl, lane);
        // 1. f^t for the lane's nodes
        T f[Q][VEC];
        if (T0) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j) f[i][j] = T(0);
        } else {
            pull_vec<Q, T, VEC>(f, gprev, n0, x0, x0w, y, z, lw, g, bc, lane, live, need);
        }
        // 2. adjoint pull: mu_j(x) <- lambda_j(x + c_j), rows y + c_jy, z + c_jz
        T mu[Q][VEC];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sy = y + L::c(i, 1), sz = z + L::c(i, 2);
            if (sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
                const T* rowp = lam_in + (long long)i * N + ((long long)sz * g.ny + sy) * g.nx;
                load_shift<T, VEC>(mu[i], -L::c(i, 0), rowp, x0, x0w, g.nx, lane, need);
            } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j) mu[i][j] = T(0);
            }
        }
        if (live) {
            dom = adjoint_nodes<Q, T, VEC>(f, mu, lam_in, n0, x0, y, z, lw, g, bc, T(1) / T(*tau), grad_acc);
#pragma unroll
            for (int i = 0; i < Q; ++i) Vec<T, VEC>::store(lam_out + (long long)i * N + n0, mu[i]);
        }
    }
    // warp sums in T, the kVecRows warp partials added in FP64 (FP64 is slow on this part)
    __shared__ double s_part[kVecRows];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dom += __shfl_xor_sync(0xffffffffu, dom, o);
    if (lane == 0) s_part[threadIdx.y] = (double)dom;
    __syncthreads();
    if (threadIdx.y == 0 && lane == 0) {
        double bs = 0.0;
#pragma unroll
        for (int w = 0; w < kVecRows; ++w) bs += s_part[w];
        partial[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] += bs;
    }
}

// ------------------------------------------------------------------ dispatch

// Widest VEC (4 for float, 2 for double; else 2; else 0 = scalar kernels)
// for which every row start and every buffer is VEC-element aligned.
template <typename T>
static int vec_width(const PlanInfo& p, const void* a, const void* b, const void* c)
{
    if (p.max_vec < 2) return 0;
    auto al = [](const void* ptr, size_t bytes) { return (reinterpret_cast<uintptr_t>(ptr) % bytes) == 0; };
    const int cands[2] = {sizeof(T) == 4 ? 4 : 2, 2};
    for (int w : cands) {
        if (w > p.max_vec) continue;
        const size_t bytes = (size_t)w * sizeof(T);
        if (p.geo.nx % w == 0 && al(a, bytes) && al(b, bytes) && al(c, bytes) && al(p.geo.link, (size_t)w * 4))
            return w;
    }
    return 0;
}

dim3 vec_grid(const PlanInfo& p, int vec)
{
    return dim3((unsigned)((p.geo.nx + 32 * vec - 1) / (32 * vec)), (unsigned)((p.geo.ny + kVecRows - 1) / kVecRows),
                (unsigned)p.geo.nz);
}

template <int Q, typename T, int VEC>
static void step_vec(const PlanInfo& p, int mode, const T* a, T* b, const Bc& bc, const double* tau, cudaStream_t s)
{
    const dim3 grid = vec_grid(p, VEC), block(32, kVecRows);
    if (p.step_variant == 1) {
        if (mode == kStreamCollide)
            launch_k(p.pdl, k_step_own<Q, T, VEC, kStreamCollide>, dim3(grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
        else if (mode == kCollideOnly)
            launch_k(p.pdl, k_step_own<Q, T, VEC, kCollideOnly>, dim3(grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
        else
            launch_k(p.pdl, k_step_own<Q, T, VEC, kStreamOnly>, dim3(grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
        return;
    }
    if (mode == kStreamCollide)
        launch_k(p.pdl, k_step_vec<Q, T, VEC, kStreamCollide>, dim3(grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
    else if (mode == kCollideOnly)
        launch_k(p.pdl, k_step_vec<Q, T, VEC, kCollideOnly>, dim3(grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
    else
        launch_k(p.pdl, k_step_vec<Q, T, VEC, kStreamOnly>, dim3(grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
}

template <int Q, typename T>
static bool try_step(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                     cudaStream_t s)
{
    const int w = vec_width<T>(p, src, dst, dst);
    const T* a = static_cast<const T*>(src);
    T* b = static_cast<T*>(dst);
    if (w == 4) step_vec<Q, T, (sizeof(T) == 4 ? 4 : 2)>(p, mode, a, b, bc, tau, s);
    else if (w == 2) step_vec<Q, T, 2>(p, mode, a, b, bc, tau, s);
    else return false;
    return true;
}

bool step_launch_vec(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                     cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4) return try_step<9, float>(p, mode, src, dst, bc, tau, s);
    if (p.q == 9 && p.prec == 8) return try_step<9, double>(p, mode, src, dst, bc, tau, s);
    if (p.q == 19 && p.prec == 4) return try_step<19, float>(p, mode, src, dst, bc, tau, s);
    if (p.q == 19 && p.prec == 8) return try_step<19, double>(p, mode, src, dst, bc, tau, s);
    return false;
}

template <int Q, typename T, int VEC>
static void adj_vec(const PlanInfo& p, int t0, const T* gp, const T* li, T* lo, const Bc& bc, const double* tau,
                    double* grad_acc, double* partial, cudaStream_t s)
{
    const dim3 grid = vec_grid(p, VEC), block(32, kVecRows);
    if (t0)
        launch_k(p.pdl, k_adjoint_vec<Q, T, VEC, true>, dim3(grid), dim3(block), 0, s, gp, li, lo, p.geo, bc, tau, grad_acc, partial);
    else
        launch_k(p.pdl, k_adjoint_vec<Q, T, VEC, false>, dim3(grid), dim3(block), 0, s, gp, li, lo, p.geo, bc, tau, grad_acc, partial);
}

template <int Q, typename T, int VECMAX>
static bool try_adj(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                    const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    const void* gp_chk = gprev ? gprev : lam_in;
    int w = vec_width<T>(p, gp_chk, lam_in, lam_out);
    if (w > VECMAX) w = VECMAX;
    const T* gp = static_cast<const T*>(gprev);
    const T* li = static_cast<const T*>(lam_in);
    T* lo = static_cast<T*>(lam_out);
    if (w == 4) adj_vec<Q, T, (VECMAX >= 4 ? 4 : 2)>(p, t0, gp, li, lo, bc, tau, grad_acc, partial, s);
    else if (w == 2) adj_vec<Q, T, 2>(p, t0, gp, li, lo, bc, tau, grad_acc, partial, s);
    else return false;
    return true;
}

bool adjoint_launch_vec(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                        const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4) return try_adj<9, float, 4>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    if (p.q == 9 && p.prec == 8) return try_adj<9, double, 2>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    if (p.q == 19 && p.prec == 4)
        return try_adj<19, float, 2>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    if (p.q == 19 && p.prec == 8)
        return try_adj<19, double, 2>(p, t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    return false;
}

int vec_blocks_max(const PlanInfo& p)
{
    const dim3 a = vec_grid(p, 2), b = vec_grid(p, 4);
    return (int)std::max(a.x * a.y * a.z, b.x * b.y * b.z);
}

}  // namespace lbm
