// Persistent sweeps for lattices that fit in L2: the whole forward sweep is
// one cooperative launch, and so is the whole reverse sweep (segment
// recompute + adjoint steps), with a bounded grid barrier between time
// steps instead of a kernel boundary.  Opt-in (LBM_PERSIST=1): on GB300 a
// grid-wide barrier across both dies measured about 5.9 us per 512x256 step,
// more than a kernel boundary inside a replayed CUDA graph with programmatic
// dependent launch (about 4.4 us), so the per-step launches stay the default.
//
// The arithmetic is the one of step.cu / adjoint.cu (Eq. 1-6 of
// arXiv 2310.00810 and their transpose) through the register helpers of
// nodes.cuh.  Buffers written inside the kernel are read with ld.global.cg
// (L2, never a stale L1 line), and each warp handles one row segment of
// 32 * VEC nodes at a time so the +-1 x-shifts stay warp shuffles.
//
// Grid barrier: sense reversal on a counter and a generation word in the
// workspace, spinning at most spin_limit times; a CTA that gives up latches
// LBM_ERR_TIMEOUT and raises an abort word that makes every other CTA leave
// at its next barrier.
#include <algorithm>

#include "nodes.cuh"

namespace lbm {

namespace {

constexpr int kPersistThreads = 256;

__device__ __forceinline__ bool grid_sync(PersistBar* b, unsigned nblocks, uint32_t* status, unsigned spin_limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = &b->gen;
        volatile int* vabort = &b->abort;
        const unsigned g0 = *vgen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == g0) {
                if (*vabort || ++it > spin_limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        if (!ok || *vabort) {
            ok = 0;
            atomicOr(status, 1u << LBM_ERR_TIMEOUT);
            atomicExch(&b->abort, 1);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T, int VEC>
struct VecCg;
template <>
struct VecCg<float, 4> {
    __device__ static void load(const float* p, float (&o)[4])
    {
        const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
    }
};
template <>
struct VecCg<float, 2> {
    __device__ static void load(const float* p, float (&o)[2])
    {
        const float2 t = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = t.x, o[1] = t.y;
    }
};
template <>
struct VecCg<float, 1> {
    __device__ static void load(const float* p, float (&o)[1]) { o[0] = __ldcg(p); }
};
template <>
struct VecCg<double, 2> {
    __device__ static void load(const double* p, double (&o)[2])
    {
        const double2 t = __ldcg(reinterpret_cast<const double2*>(p));
        o[0] = t.x, o[1] = t.y;
    }
};
template <>
struct VecCg<double, 1> {
    __device__ static void load(const double* p, double (&o)[1]) { o[0] = __ldcg(p); }
};

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T* p, const T (&v)[VEC])
{
    if constexpr (VEC == 1) {
        p[0] = v[0];
    } else {
        Vec<T, VEC>::store(p, v);
    }
}

// Row segment values shifted by -sx (sx in {-1, 0, 1}), through L2.
template <typename T, int VEC>
__device__ __forceinline__ void load_row(T (&o)[VEC], const T* rowp, int sx, int x0, int x0w, int nx, int lane,
                                         bool live)
{
    T V[VEC];
    if (live) {
        VecCg<T, VEC>::load(rowp + x0, V);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) V[j] = T(0);
    }
    if (sx == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) o[j] = V[j];
    } else if (sx == 1) {
        T prev = __shfl_up_sync(0xffffffffu, V[VEC - 1], 1);
        if (lane == 0) prev = (x0w > 0 && live) ? __ldcg(rowp + x0w - 1) : T(0);
        o[0] = prev;
#pragma unroll
        for (int j = 1; j < VEC; ++j) o[j] = V[j - 1];
    } else {
        T next = __shfl_down_sync(0xffffffffu, V[0], 1);
        if (lane == 31) next = (x0w + 32 * VEC < nx && live) ? __ldcg(rowp + x0w + 32 * VEC) : T(0);
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) o[j] = V[j + 1];
        o[VEC - 1] = next;
    }
}

template <int VEC>
__device__ __forceinline__ void links_of(uint32_t (&lw)[VEC], const uint32_t* link, long long n0, bool live)
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) lw[j] = live ? link[n0 + j] : kLinkSolid;
}

struct Unit {
    int y, z, x0w, x0;
    long long n0;
    bool live;
};

__device__ __forceinline__ Unit unit_of(const Geo& g, int u, int vec, int lane)
{
    const int per_row = (g.nx + 32 * vec - 1) / (32 * vec);
    Unit r;
    const int seg = u % per_row, row = u / per_row;
    r.y = row % g.ny;
    r.z = row / g.ny;
    r.x0w = seg * 32 * vec;
    r.x0 = r.x0w + lane * vec;
    r.live = r.x0 < g.nx;
    r.n0 = ((long long)r.z * g.ny + r.y) * g.nx + r.x0;
    return r;
}

// Pulled values (from x - c_i) and own values of the unit's nodes.
template <int Q, typename T, int VEC>
__device__ __forceinline__ void gather(T (&v)[Q][VEC], T (&own)[Q][VEC], const T* src, const Unit& U, const Geo& g,
                                       int lane, int dir)
{
    using L = Lattice<Q>;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T* plane = src + (long long)i * g.N;
        if (U.live) {
            VecCg<T, VEC>::load(plane + U.n0, own[i]);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) own[i][j] = T(0);
        }
        const int sy = U.y - dir * L::c(i, 1), sz = U.z - dir * L::c(i, 2);
        if (sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz)
            load_row<T, VEC>(v[i], plane + ((long long)sz * g.ny + sy) * g.nx, dir * L::c(i, 0), U.x0, U.x0w, g.nx,
                             lane, U.live);
        else
#pragma unroll
            for (int j = 0; j < VEC; ++j) v[i][j] = T(0);
    }
}

// One stream-collide (or stream-only) step over all units of the lattice.
template <int Q, typename T, int VEC>
__device__ void step_all(const T* src, T* dst, const Geo& g, const Bc& bc, T omega, bool stream_only, int units,
                         int warp, int nwarps, int lane)
{
    for (int u = warp; u < units; u += nwarps) {
        const Unit U = unit_of(g, u, VEC, lane);
        uint32_t lw[VEC];
        links_of<VEC>(lw, g.link, U.n0, U.live);
        T v[Q][VEC], own[Q][VEC];
        gather<Q, T, VEC>(v, own, src, U, g, lane, 1);
        if (!U.live) continue;
        pull_fixup_own<Q, T, VEC>(v, own, U.x0, U.y, U.z, lw, g, bc);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            if (lw[j] & kLinkSolid) {
#pragma unroll
                for (int i = 0; i < Q; ++i) v[i][j] = T(0);
            } else if (!stream_only) {
                T a[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) a[i] = v[i][j];
                collide<Q, T>(a, omega);
#pragma unroll
                for (int i = 0; i < Q; ++i) v[i][j] = a[i];
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) store_vec<T, VEC>(dst + (long long)i * g.N + U.n0, v[i]);
    }
}

template <typename T>
__device__ void zero_all(T* dst, long long n, int tid, int nthreads)
{
    for (long long i = tid; i < n; i += nthreads) dst[i] = T(0);
}

// Where the sweep keeps g^t: checkpoint slot s for t = s k - 1 (s = 1..S-1),
// otherwise ping-pong buffer t & 1.
template <typename T>
__device__ __forceinline__ T* state_at(const PersistArgs& a, int t)
{
    const int s1 = t + 1;
    if (s1 % a.k == 0 && s1 / a.k >= 1 && s1 / a.k <= a.S - 1)
        return reinterpret_cast<T*>(a.ckpt + a.state_stride * (size_t)(s1 / a.k - 1));
    return reinterpret_cast<T*>(a.ping[t & 1]);
}

template <int Q, typename T, int VEC>
__global__ void __launch_bounds__(kPersistThreads, 1) k_forward_persist(PersistArgs a, Geo g, Bc bc,
                                                                        const double* __restrict__ tau)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * kPersistThreads + threadIdx.x) >> 5, nwarps = gridDim.x * kPersistThreads / 32;
    const int per_row = (g.nx + 32 * VEC - 1) / (32 * VEC);
    const int units = per_row * g.ny * g.nz;
    const T omega = T(1) / T(*tau);
    for (int t = 1; t <= a.T - 1; ++t) {
        step_all<Q, T, VEC>(state_at<T>(a, t - 1), state_at<T>(a, t), g, bc, omega, false, units, warp, nwarps, lane);
        if (!grid_sync(a.bar, gridDim.x, bc.status, a.spin_limit)) return;
    }
    step_all<Q, T, VEC>(state_at<T>(a, a.T - 1), reinterpret_cast<T*>(a.out), g, bc, omega, true, units, warp, nwarps,
                        lane);
}

// One adjoint step over all units: lambda_out from lambda_in and g^{t-1}
// (rest state when gprev == nullptr).  Returns this thread's dL/domega sum.
template <int Q, typename T, int VEC>
__device__ double adjoint_all(const T* gprev, const T* lam_in, T* lam_out, const Geo& g, const Bc& bc, T omega,
                              double* grad_acc, int units, int warp, int nwarps, int lane)
{
    double dom = 0.0;
    for (int u = warp; u < units; u += nwarps) {
        const Unit U = unit_of(g, u, VEC, lane);
        uint32_t lw[VEC];
        links_of<VEC>(lw, g.link, U.n0, U.live);
        T f[Q][VEC], mu[Q][VEC], lown[Q][VEC];
        if (gprev) {
            T own[Q][VEC];
            gather<Q, T, VEC>(f, own, gprev, U, g, lane, 1);
            if (U.live) pull_fixup_own<Q, T, VEC>(f, own, U.x0, U.y, U.z, lw, g, bc);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j) f[i][j] = T(0);
        }
        gather<Q, T, VEC>(mu, lown, lam_in, U, g, lane, -1);
        if (!U.live) continue;
        dom += (double)adjoint_nodes_own<Q, T, VEC>(f, mu, lown, U.n0, U.x0, U.y, U.z, lw, g, bc, omega, grad_acc);
#pragma unroll
        for (int i = 0; i < Q; ++i) store_vec<T, VEC>(lam_out + (long long)i * g.N + U.n0, mu[i]);
    }
    return dom;
}

template <int Q, typename T, int VEC>
__global__ void __launch_bounds__(kPersistThreads, 1) k_reverse_persist(PersistArgs a, Geo g, Bc bc,
                                                                        const double* __restrict__ tau,
                                                                        double* __restrict__ grad_acc,
                                                                        double* __restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int gtid = blockIdx.x * kPersistThreads + threadIdx.x, gthreads = gridDim.x * kPersistThreads;
    const int warp = gtid >> 5, nwarps = gthreads / 32;
    const int per_row = (g.nx + 32 * VEC - 1) / (32 * VEC);
    const int units = per_row * g.ny * g.nz;
    const T omega = T(1) / T(*tau);
    const long long qn = (long long)Q * g.N;
    double dom = 0.0;
    const T* lam_cur = reinterpret_cast<const T*>(a.lam_in);
    int lam_next = 0;
    bool ok = true;
    for (int sg = a.S - 1; sg >= 0 && ok; --sg) {
        const int t0 = sg * a.k, len = min(a.k, a.T - t0);
        auto seg = [&](int j) { return reinterpret_cast<T*>(a.seg + a.state_stride * (size_t)j); };
        const T* base = sg >= 1 ? reinterpret_cast<const T*>(a.ckpt + a.state_stride * (size_t)(sg - 1)) : nullptr;
        const T* prev = base;
        for (int j = 1; j < len && ok; ++j) {
            if (sg == 0 && j == 1)
                zero_all<T>(seg(1), qn, gtid, gthreads);
            else
                step_all<Q, T, VEC>(prev, seg(j), g, bc, omega, false, units, warp, nwarps, lane);
            prev = seg(j);
            ok = grid_sync(a.bar, gridDim.x, bc.status, a.spin_limit);
        }
        for (int j = len - 1; j >= 0 && ok; --j) {
            const T* src = j == 0 ? base : seg(j);  // nullptr: the rest state (sg = 0, j = 0)
            T* lo = reinterpret_cast<T*>(a.lam[lam_next]);
            dom += adjoint_all<Q, T, VEC>(src, lam_cur, lo, g, bc, omega, grad_acc, units, warp, nwarps, lane);
            lam_cur = lo;
            lam_next ^= 1;
            ok = grid_sync(a.bar, gridDim.x, bc.status, a.spin_limit);
        }
    }
    // CTA sum of the dL/domega contributions (FP64; fixed order)
    __shared__ double s_part[kPersistThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dom += __shfl_xor_sync(0xffffffffu, dom, o);
    if (lane == 0) s_part[threadIdx.x >> 5] = dom;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kPersistThreads / 32; ++w) b += s_part[w];
        partial[blockIdx.x] += b;
    }
}

int device_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <class K, class... Args>
lbm_status launch_coop(K kernel, int grid, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_status(cudaLaunchKernelEx(&cfg, kernel, args...));
}

template <class K>
int coop_grid(K kernel, const PlanInfo& p)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPersistThreads, 0) != cudaSuccess) return 0;
    const int sms = device_sms();
    const int cap = std::min(per_sm, 1) * sms;
    return std::min(cap, p.n_partial);
}

template <int Q, typename T, int VF, int VA>
lbm_status forward_impl(const PlanInfo& p, const PersistArgs& a, const Bc& bc, const double* tau, cudaStream_t s)
{
    auto k = k_forward_persist<Q, T, VF>;
    const int grid = coop_grid(k, p);
    if (grid <= 0) return LBM_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(a.bar, 0, sizeof(PersistBar), s) != cudaSuccess) return LBM_ERR_CUDA;
    return launch_coop(k, grid, s, a, p.geo, bc, tau);
}

template <int Q, typename T, int VF, int VA>
lbm_status reverse_impl(const PlanInfo& p, const PersistArgs& a, const Bc& bc, const double* tau, double* grad_acc,
                        double* partial, cudaStream_t s)
{
    auto k = k_reverse_persist<Q, T, VA>;
    const int grid = coop_grid(k, p);
    if (grid <= 0) return LBM_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(a.bar, 0, sizeof(PersistBar), s) != cudaSuccess) return LBM_ERR_CUDA;
    return launch_coop(k, grid, s, a, p.geo, bc, tau, grad_acc, partial);
}

}  // namespace

// Widest row vector every persistent kernel variant of this plan can use.
bool persist_ok(const PlanInfo& p)
{
    return p.use_persist && p.cmp.nf == 0 && !p.uw_extrap && !p.mrt && p.geo.nx % 4 == 0 && p.state_bytes <= p.persist_max_bytes;
}

lbm_status forward_persist(const PlanInfo& p, const PersistArgs& a, const Bc& bc, const double* tau, cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4) return forward_impl<9, float, 4, 2>(p, a, bc, tau, s);
    if (p.q == 9 && p.prec == 8) return forward_impl<9, double, 2, 1>(p, a, bc, tau, s);
    if (p.q == 19 && p.prec == 4) return forward_impl<19, float, 2, 1>(p, a, bc, tau, s);
    if (p.q == 19 && p.prec == 8) return forward_impl<19, double, 1, 1>(p, a, bc, tau, s);
    return LBM_ERR_UNSUPPORTED;
}

lbm_status reverse_persist(const PlanInfo& p, const PersistArgs& a, const Bc& bc, const double* tau,
                           double* grad_acc, double* partial, cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4) return reverse_impl<9, float, 4, 2>(p, a, bc, tau, grad_acc, partial, s);
    if (p.q == 9 && p.prec == 8) return reverse_impl<9, double, 2, 1>(p, a, bc, tau, grad_acc, partial, s);
    if (p.q == 19 && p.prec == 4) return reverse_impl<19, float, 2, 1>(p, a, bc, tau, grad_acc, partial, s);
    if (p.q == 19 && p.prec == 8) return reverse_impl<19, double, 1, 1>(p, a, bc, tau, grad_acc, partial, s);
    return LBM_ERR_UNSUPPORTED;
}

}  // namespace lbm
