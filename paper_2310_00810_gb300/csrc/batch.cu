// Batches: many independent lattices of different sizes (the batched
// inversions of uneven grain geometries) advanced by shared kernels.
//
// All instances are packed back to back in one set of buffers.  A device
// table of work units, one per (instance, row, segment of 32 * VEC nodes),
// lets a single launch per time step cover every instance: one warp per unit,
// the same row-segment code as the vectorised single-lattice kernels (so the
// per-node arithmetic, Eq. 1-6 of arXiv 2310.00810 and its transpose, is
// identical and a batch reproduces single-instance populations bit for bit).
// With tens of instances a step moves hundreds of MB, so the per-step launch
// cost is negligible; each sweep is replayed as one CUDA graph.
//
// Reductions are deterministic: per-unit FP64 partials (accumulated in place
// across the steps of a sweep by the warp that owns the unit), summed per
// instance in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "nodes.cuh"

using namespace lbm;

namespace {

struct BInst {
    Geo g;                // sizes and this instance's link words (absolute pointer)
    long long f_off;      // populations in a packed state (elements)
    long long vel_off;    // velocity fields (doubles)
    long long node_off;   // node fields (mask, roi)
    long long in_off;     // inlet densities and their gradients
    long long acc_off;    // per-inlet-node accumulators (ny * nz)
    int n_in;
    int unit0, units;
};

struct BUnit {
    int inst, row, x0w, pad;  // row = z * ny + y
};

constexpr int kBatchThreads = 128;

// Nodes per lane: the vector widths of the single-lattice register kernels.
template <int Q, typename T>
constexpr int batch_vec()
{
    return (Q == 9 && sizeof(T) == 4) ? 4 : 2;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
long long al64(long long e) { return (e + 63) & ~63LL; }

// ------------------------------------------------------------------ kernels

template <int Q, typename T, int VEC, int MODE>
__global__ void __launch_bounds__(kBatchThreads) k_batch_step(const BInst* __restrict__ insts,
                                                              const BUnit* __restrict__ units, int n_units,
                                                              const T* __restrict__ src, T* __restrict__ dst,
                                                              const double* __restrict__ rho_in,
                                                              const double* __restrict__ tau, double rho_out,
                                                              uint32_t* status)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * kBatchThreads + threadIdx.x) >> 5;
    if (w >= n_units) return;  // warp-uniform
    const BUnit un = units[w];
    const BInst I = insts[un.inst];
    const Geo& g = I.g;
    const int y = un.row % g.ny, z = un.row / g.ny;
    const int x0w = un.x0w, x0 = x0w + lane * VEC;
    const bool live = x0 < g.nx;
    const long long n0 = (long long)un.row * g.nx + x0;
    const T* s = src + I.f_off;
    T* d = dst + I.f_off;
    Bc bc;
    bc.rho_in = rho_in + I.in_off;
    bc.profile = I.n_in > 1 ? 1 : 0;
    bc.rho_out = rho_out;
    bc.status = status;
    uint32_t lw[VEC];
    load_links<VEC>(lw, g.link, n0, live);
    const unsigned fl = fluid_bits<VEC>(lw);
    T v[Q][VEC];
    if (MODE == kCollideOnly) {
        if (!live) return;
#pragma unroll
        for (int i = 0; i < Q; ++i) Vec<T, VEC>::load(s + (long long)i * g.N + n0, v[i]);
    } else {
        const Need<VEC> need = lane_needs<VEC>(fl, lane);
        pull_vec<Q, T, VEC>(v, s, n0, x0, x0w, y, z, lw, g, bc, lane, live, need);
        if (!live) return;
    }
    if (MODE != kStreamOnly) {
        const T omega = T(1) / T(tau[un.inst]);
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
    for (int i = 0; i < Q; ++i) Vec<T, VEC>::store(d + (long long)i * g.N + n0, v[i]);
}

template <int Q, typename T, int VEC, bool T0>
__global__ void __launch_bounds__(kBatchThreads) k_batch_adjoint(const BInst* __restrict__ insts,
                                                                 const BUnit* __restrict__ units, int n_units,
                                                                 const T* __restrict__ gprev,
                                                                 const T* __restrict__ lam_in, T* __restrict__ lam_out,
                                                                 const double* __restrict__ rho_in,
                                                                 const double* __restrict__ tau, double rho_out,
                                                                 double* __restrict__ grad_acc,
                                                                 double* __restrict__ partial, uint32_t* status)
{
    using L = Lattice<Q>;
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * kBatchThreads + threadIdx.x) >> 5;
    if (w >= n_units) return;  // warp-uniform
    const BUnit un = units[w];
    const BInst I = insts[un.inst];
    const Geo& g = I.g;
    const long long N = g.N;
    const int y = un.row % g.ny, z = un.row / g.ny;
    const int x0w = un.x0w, x0 = x0w + lane * VEC;
    const bool live = x0 < g.nx;
    const long long n0 = (long long)un.row * g.nx + x0;
    const T* li = lam_in + I.f_off;
    Bc bc;
    bc.rho_in = rho_in + I.in_off;
    bc.profile = I.n_in > 1 ? 1 : 0;
    bc.rho_out = rho_out;
    bc.status = status;
    uint32_t lw[VEC];
    load_links<VEC>(lw, g.link, n0, live);
    const unsigned fl = fluid_bits<VEC>(lw);
    const Need<VEC> need = lane_needs<VEC>(fl, lane);
    T f[Q][VEC];
    if (T0) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
            for (int j = 0; j < VEC; ++j) f[i][j] = T(0);
    } else {
        pull_vec<Q, T, VEC>(f, gprev + I.f_off, n0, x0, x0w, y, z, lw, g, bc, lane, live, need);
    }
    T mu[Q][VEC];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sy = y + L::c(i, 1), sz = z + L::c(i, 2);
        if (sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
            const T* rowp = li + (long long)i * N + ((long long)sz * g.ny + sy) * g.nx;
            load_shift<T, VEC>(mu[i], -L::c(i, 0), rowp, x0, x0w, g.nx, lane, need);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) mu[i][j] = T(0);
        }
    }
    T dom = T(0);
    if (live) {
        dom = adjoint_nodes<Q, T, VEC>(f, mu, li, n0, x0, y, z, lw, g, bc, T(1) / T(tau[un.inst]),
                                       grad_acc + I.acc_off);
#pragma unroll
        for (int i = 0; i < Q; ++i) Vec<T, VEC>::store(lam_out + I.f_off + (long long)i * N + n0, mu[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dom += __shfl_xor_sync(0xffffffffu, dom, o);
    if (lane == 0) partial[w] += (double)dom;
}

// Loss terms and the seed lambda^T per unit (one node per lane, 32 * VEC
// nodes per unit); count = 1 computes the ROI fluid-node counts instead.
template <int Q, typename T, int VEC>
__global__ void __launch_bounds__(kBatchThreads) k_batch_loss(const BInst* __restrict__ insts,
                                                              const BUnit* __restrict__ units, int n_units,
                                                              const T* __restrict__ f, const double* __restrict__ ut,
                                                              const uint8_t* __restrict__ roi, int kind,
                                                              const double* __restrict__ weight, T* __restrict__ lam,
                                                              double* __restrict__ partial, int count)
{
    using L = Lattice<Q>;
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * kBatchThreads + threadIdx.x) >> 5;
    if (w >= n_units) return;
    const BUnit un = units[w];
    const BInst I = insts[un.inst];
    const Geo& g = I.g;
    const long long N = g.N;
    double term = 0.0;
    for (int j = 0; j < VEC; ++j) {
        const int x = un.x0w + j * 32 + lane;
        if (x >= g.nx) continue;
        const long long n = (long long)un.row * g.nx + x;
        const bool in = !(g.link[n] & kLinkSolid) && (!roi || roi[I.node_off + n]);
        if (count) {
            term += in ? 1.0 : 0.0;
            continue;
        }
        T out[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i] = T(0);
        if (in) {
            T v[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = f[I.f_off + (long long)i * N + n];
            T drho, rho, u[3];
            moments<Q, T>(v, drho, rho, u);
            const double wgt = weight[un.inst];
            double du[3] = {0.0, 0.0, 0.0};
            if (kind == LBM_LOSS_VEC) {
#pragma unroll
                for (int a = 0; a < L::D; ++a) {
                    const double e = (double)u[a] - ut[I.vel_off + (long long)a * N + n];
                    term += wgt * e * e;
                    du[a] = 2.0 * wgt * e;
                }
            } else {
                double uu = 0.0, tt = 0.0;
#pragma unroll
                for (int a = 0; a < L::D; ++a) {
                    uu += (double)u[a] * (double)u[a];
                    const double t = ut[I.vel_off + (long long)a * N + n];
                    tt += t * t;
                }
                const double un_ = sqrt(uu), e = un_ - sqrt(tt);
                term += wgt * e * e;
                if (uu != 0.0)
#pragma unroll
                    for (int a = 0; a < L::D; ++a) du[a] = 2.0 * wgt * e * (double)u[a] / un_;
            }
            const T inv = T(1) / rho;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                T sacc = 0;
#pragma unroll
                for (int a = 0; a < L::D; ++a) sacc += T(du[a]) * (T(L::c(k, a)) - u[a]);
                out[k] = sacc * inv;
            }
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) lam[I.f_off + (long long)k * N + n] = out[k];
    }
    term = warp_sum(term);
    if (lane == 0) partial[w] = term;
}

// Per instance (one block each): out[i] = sum of its units' partials; with
// mode 1 the weights (1 or 1 / count) are written instead.
__global__ void k_batch_reduce(const BInst* __restrict__ insts, const double* __restrict__ partial, int mode,
                               int mean, double* __restrict__ out, uint32_t* status)
{
    const BInst I = insts[blockIdx.x];
    double v = 0.0;
    for (int u = threadIdx.x; u < I.units; u += blockDim.x) v += partial[I.unit0 + u];
    v = block_sum(v, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        if (mode == 1) {
            out[blockIdx.x] = mean ? (v > 0.0 ? 1.0 / v : 0.0) : 1.0;
        } else {
            out[blockIdx.x] = v;
            if (!isfinite(v)) atomicOr(status, 1u << LBM_ERR_NONFINITE);
        }
    }
}

// Per instance: dL/dtau and dL/drho_in from the unit partials and inlet accumulators.
__global__ void k_batch_finish(const BInst* __restrict__ insts, const double* __restrict__ partial,
                               const double* __restrict__ grad_acc, const double* __restrict__ tau,
                               double* __restrict__ g_in, double* __restrict__ g_tau, uint32_t* status)
{
    const BInst I = insts[blockIdx.x];
    double v = 0.0;
    for (int u = threadIdx.x; u < I.units; u += blockDim.x) v += partial[I.unit0 + u];
    v = block_sum(v, threadIdx.x, blockDim.x);
    const int n_acc = I.g.ny * I.g.nz;
    double gs = 0.0;
    if (I.n_in == 1) {
        for (int a = threadIdx.x; a < n_acc; a += blockDim.x) gs += grad_acc[I.acc_off + a];
        gs = block_sum(gs, threadIdx.x, blockDim.x);
    } else {
        for (int a = threadIdx.x; a < n_acc; a += blockDim.x) g_in[I.in_off + a] = grad_acc[I.acc_off + a];
    }
    if (threadIdx.x == 0) {
        const double t = tau[blockIdx.x];
        g_tau[blockIdx.x] = -v / (t * t);
        if (I.n_in == 1) g_in[I.in_off] = gs;
        if (!isfinite(v) || !isfinite(gs)) atomicOr(status, 1u << LBM_ERR_NONFINITE);
    }
}

// The same in the fluid-only layout: instance i's dL/domega partials are the
// warp slots [k0 / 32, (k0 + nf + 31) / 32) of the packed compact kernels,
// summed in the order a single compact plan sums its own.
__global__ void k_batch_finish_cmp(const BCmpInst* __restrict__ insts, const double* __restrict__ partial,
                                   const double* __restrict__ grad_acc, const double* __restrict__ tau,
                                   double* __restrict__ g_in, double* __restrict__ g_tau, uint32_t* status)
{
    const BCmpInst I = insts[blockIdx.x];
    const long long w0 = I.k0 >> 5, nw = (I.nf + 31) >> 5;
    double v = 0.0;
    for (long long u = threadIdx.x; u < nw; u += blockDim.x) v += partial[w0 + u];
    v = block_sum(v, threadIdx.x, blockDim.x);
    const int n_acc = I.g.ny * I.g.nz;
    double gs = 0.0;
    if (I.n_in == 1) {
        for (int a = threadIdx.x; a < n_acc; a += blockDim.x) gs += grad_acc[I.acc_off + a];
        gs = block_sum(gs, threadIdx.x, blockDim.x);
    } else {
        for (int a = threadIdx.x; a < n_acc; a += blockDim.x) g_in[I.in_off + a] = grad_acc[I.acc_off + a];
    }
    if (threadIdx.x == 0) {
        const double t = tau[blockIdx.x];
        g_tau[blockIdx.x] = -v / (t * t);
        if (I.n_in == 1) g_in[I.in_off] = gs;
        if (!isfinite(v) || !isfinite(gs)) atomicOr(status, 1u << LBM_ERR_NONFINITE);
    }
}

}  // namespace

// -------------------------------------------------------------------- host

struct lbm_batch {
    lbm_desc desc;
    int n, q, d, prec, k, S;
    std::vector<PlanInfo> info;  // per instance (geometry launches)
    std::vector<long long> state_off, node_off, vel_off, in_off, acc_off;
    std::vector<BInst> insts;
    std::vector<BUnit> units;
    size_t state_elems = 0, state_bytes = 0;
    // workspace layout (bytes)
    size_t o_status = 0, o_insts = 0, o_units = 0, o_acc = 0, o_part = 0, o_part2 = 0, o_scal = 0, o_ping[2] = {},
           o_lam[2] = {}, o_ckpt = 0, o_seg = 0, total = 0;
    bool tables_ready = false;
    void* tables_ws = nullptr;
    bool pdl = true;
    size_t n_part = 0;  // FP64 dL/domega slots: one per unit (dense) or per warp (fluid-only)
    // fluid-only layout (lbm_batch_compact_bind)
    bool cmp = false;
    long long nfp = 0;                 // packed compact nodes (every instance padded to kBatchCmpAlign)
    std::vector<BCmpInst> cinsts;
    std::vector<int> blk_inst;
    BCmpArgs ca = {};
    size_t cmp_state_bytes = 0;
    struct G {
        int op;
        const void* ptr[6];
        double scalar;
        cudaGraphExec_t exec;
    };
    std::vector<G> graphs;
    ~lbm_batch()
    {
        for (auto& g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    }
};

namespace {

template <int Q, typename T>
void launch_step(const lbm_batch* b, int mode, const void* src, void* dst, const double* rho_in, const double* tau,
                 double rho_out, unsigned char* ws, cudaStream_t s)
{
    constexpr int VEC = batch_vec<Q, T>();
    const int nu = (int)b->units.size();
    const dim3 grid((unsigned)((nu * 32 + kBatchThreads - 1) / kBatchThreads)), block(kBatchThreads);
    const BInst* I = reinterpret_cast<const BInst*>(ws + b->o_insts);
    const BUnit* U = reinterpret_cast<const BUnit*>(ws + b->o_units);
    uint32_t* st = reinterpret_cast<uint32_t*>(ws + b->o_status);
    const T* a = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
    if (mode == kStreamCollide)
        launch_k(b->pdl, k_batch_step<Q, T, VEC, kStreamCollide>, grid, block, 0, s, I, U, nu, a, d, rho_in, tau,
                 rho_out, st);
    else if (mode == kCollideOnly)
        launch_k(b->pdl, k_batch_step<Q, T, VEC, kCollideOnly>, grid, block, 0, s, I, U, nu, a, d, rho_in, tau,
                 rho_out, st);
    else
        launch_k(b->pdl, k_batch_step<Q, T, VEC, kStreamOnly>, grid, block, 0, s, I, U, nu, a, d, rho_in, tau,
                 rho_out, st);
}

lbm_status step(const lbm_batch* b, int mode, const void* src, void* dst, const double* rho_in, const double* tau,
                double rho_out, unsigned char* ws, cudaStream_t s)
{
    if (b->q == 9 && b->prec == 4) launch_step<9, float>(b, mode, src, dst, rho_in, tau, rho_out, ws, s);
    else if (b->q == 9 && b->prec == 8) launch_step<9, double>(b, mode, src, dst, rho_in, tau, rho_out, ws, s);
    else if (b->q == 19 && b->prec == 4) launch_step<19, float>(b, mode, src, dst, rho_in, tau, rho_out, ws, s);
    else launch_step<19, double>(b, mode, src, dst, rho_in, tau, rho_out, ws, s);
    return cuda_status(cudaGetLastError());
}

template <int Q, typename T>
void launch_adj(const lbm_batch* b, bool t0, const void* gprev, const void* lam_in, void* lam_out,
                const double* rho_in, const double* tau, double rho_out, unsigned char* ws, cudaStream_t s)
{
    constexpr int VEC = batch_vec<Q, T>();
    const int nu = (int)b->units.size();
    const dim3 grid((unsigned)((nu * 32 + kBatchThreads - 1) / kBatchThreads)), block(kBatchThreads);
    const BInst* I = reinterpret_cast<const BInst*>(ws + b->o_insts);
    const BUnit* U = reinterpret_cast<const BUnit*>(ws + b->o_units);
    uint32_t* st = reinterpret_cast<uint32_t*>(ws + b->o_status);
    double* acc = reinterpret_cast<double*>(ws + b->o_acc);
    double* part = reinterpret_cast<double*>(ws + b->o_part);
    const T* gp = static_cast<const T*>(gprev);
    const T* li = static_cast<const T*>(lam_in);
    T* lo = static_cast<T*>(lam_out);
    if (t0)
        launch_k(b->pdl, k_batch_adjoint<Q, T, VEC, true>, grid, block, 0, s, I, U, nu, gp, li, lo, rho_in, tau,
                 rho_out, acc, part, st);
    else
        launch_k(b->pdl, k_batch_adjoint<Q, T, VEC, false>, grid, block, 0, s, I, U, nu, gp, li, lo, rho_in, tau,
                 rho_out, acc, part, st);
}

lbm_status adjoint(const lbm_batch* b, bool t0, const void* gprev, const void* lam_in, void* lam_out,
                   const double* rho_in, const double* tau, double rho_out, unsigned char* ws, cudaStream_t s)
{
    if (b->q == 9 && b->prec == 4) launch_adj<9, float>(b, t0, gprev, lam_in, lam_out, rho_in, tau, rho_out, ws, s);
    else if (b->q == 9 && b->prec == 8)
        launch_adj<9, double>(b, t0, gprev, lam_in, lam_out, rho_in, tau, rho_out, ws, s);
    else if (b->q == 19 && b->prec == 4)
        launch_adj<19, float>(b, t0, gprev, lam_in, lam_out, rho_in, tau, rho_out, ws, s);
    else launch_adj<19, double>(b, t0, gprev, lam_in, lam_out, rho_in, tau, rho_out, ws, s);
    return cuda_status(cudaGetLastError());
}

lbm_status run_graph(lbm_batch* b, int op, std::initializer_list<const void*> ptrs, double scalar, cudaStream_t s,
                     const std::function<lbm_status(cudaStream_t)>& issue)
{
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return issue(s);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return LBM_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return issue(s);
    lbm_batch::G key = {};
    key.op = op;
    int i = 0;
    for (const void* p : ptrs) key.ptr[i++] = p;
    key.scalar = scalar;
    for (auto& g : b->graphs)
        if (g.op == key.op && g.scalar == key.scalar && std::memcmp(g.ptr, key.ptr, sizeof(key.ptr)) == 0)
            return cuda_status(cudaGraphLaunch(g.exec, s));
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
    lbm_status st = issue(s);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != LBM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != LBM_OK ? st : LBM_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&key.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (b->graphs.size() >= 8) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back(key);
    return cuda_status(cudaGraphLaunch(key.exec, s));
}

lbm_status check(const lbm_batch* b, const void* ws)
{
    if (!b || !ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return LBM_ERR_INVALID_ARG;
    if (!b->tables_ready || b->tables_ws != ws) return LBM_ERR_INVALID_ARG;  // geometry not initialised on this ws
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_desc* c, int32_t n, const int32_t* nx, const int32_t* ny, const int32_t* nz,
                            lbm_batch** out)
{
    if (!c || !out || n < 1 || !nx || !ny || !nz) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if ((c->q != 9 && c->q != 19) || (c->precision != 4 && c->precision != 8) || c->n_steps < 1 ||
        c->ckpt_stride < 0)
        return LBM_ERR_INVALID_ARG;
    if (c->loss_kind != LBM_LOSS_VEC && c->loss_kind != LBM_LOSS_NORM) return LBM_ERR_INVALID_ARG;
    if (c->loss_norm != LBM_NORM_SUM && c->loss_norm != LBM_NORM_MEAN_FLUID) return LBM_ERR_INVALID_ARG;
    if (c->inlet_kind != LBM_INLET_CONST && c->inlet_kind != LBM_INLET_PROFILE) return LBM_ERR_INVALID_ARG;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->desc = *c;
    b->n = n;
    b->q = c->q;
    b->d = c->q == 9 ? 2 : 3;
    b->prec = c->precision;
    const int T = c->n_steps;
    b->k = c->ckpt_stride > 0 ? std::min(c->ckpt_stride, T) : std::max(1, (int)std::ceil(std::sqrt((double)T)));
    b->S = (T + b->k - 1) / b->k;
    const char* pd = std::getenv("LBM_PDL");
    b->pdl = !(pd && pd[0] == '0');
    const int vec = (c->q == 9 && c->precision == 4) ? 4 : 2;
    long long so = 0, no = 0, vo = 0, io = 0, ao = 0;
    for (int i = 0; i < n; ++i) {
        if (nx[i] < 2 || ny[i] < 1 || nz[i] < 1 || ny[i] > 65535 || nz[i] > 65535 || (c->q == 9 && nz[i] != 1) ||
            nx[i] % vec != 0) {
            delete b;
            return LBM_ERR_INVALID_ARG;
        }
        const long long N = (long long)nx[i] * ny[i] * nz[i];
        PlanInfo I = {};
        I.q = c->q;
        I.d = b->d;
        I.prec = c->precision;
        I.geo.nx = nx[i];
        I.geo.ny = ny[i];
        I.geo.nz = nz[i];
        I.geo.N = N;
        I.geo.skip_sectors = 0;
        I.grid = dim3((unsigned)((nx[i] + kStepThreads - 1) / kStepThreads), (unsigned)ny[i], (unsigned)nz[i]);
        I.n_blocks = (int)(I.grid.x * I.grid.y * I.grid.z);
        I.n_in = c->inlet_kind == LBM_INLET_PROFILE ? ny[i] * nz[i] : 1;
        I.n_acc = ny[i] * nz[i];
        b->info.push_back(I);
        b->state_off.push_back(so);
        b->node_off.push_back(no);
        b->vel_off.push_back(vo);
        b->in_off.push_back(io);
        b->acc_off.push_back(ao);
        so += al64((long long)c->q * N);
        no += al64(N);
        vo += al64((long long)b->d * N);
        io += al64(I.n_in);
        ao += al64(I.n_acc);
        BInst bi = {};
        bi.g = I.geo;
        bi.f_off = b->state_off.back();
        bi.vel_off = b->vel_off.back();
        bi.node_off = b->node_off.back();
        bi.in_off = b->in_off.back();
        bi.acc_off = b->acc_off.back();
        bi.n_in = I.n_in;
        bi.unit0 = (int)b->units.size();
        const int per_row = (nx[i] + 32 * vec - 1) / (32 * vec);
        for (int row = 0; row < ny[i] * nz[i]; ++row)
            for (int sgm = 0; sgm < per_row; ++sgm) b->units.push_back(BUnit{i, row, sgm * 32 * vec, 0});
        bi.units = (int)b->units.size() - bi.unit0;
        b->insts.push_back(bi);
    }
    b->state_off.push_back(so);
    b->node_off.push_back(no);
    b->vel_off.push_back(vo);
    b->in_off.push_back(io);
    b->acc_off.push_back(ao);
    b->state_elems = (size_t)so;
    // a workspace state slot holds a packed dense state or a packed fluid-only one (every instance's fluid
    // nodes rounded up to kBatchCmpAlign, which can exceed its dense size when nearly all nodes are fluid)
    long long cmp_bound = 0;
    for (int i = 0; i < n; ++i)
        cmp_bound += (b->info[i].geo.N + kBatchCmpAlign - 1) / kBatchCmpAlign * kBatchCmpAlign;
    b->state_bytes = al256((size_t)std::max(so, (long long)c->q * cmp_bound) * (size_t)c->precision);
    size_t o = 0;
    b->o_status = o;
    o += 256;
    b->o_insts = o;
    o += al256(sizeof(BInst) * (size_t)n);
    b->o_units = o;
    o += al256(sizeof(BUnit) * b->units.size());
    b->o_acc = o;
    o += al256(sizeof(double) * (size_t)ao);
    // dL/domega slots: one per unit in the dense layout, one per warp of the packed fluid-only
    // layout (at most ceil(N_i / 256) blocks of 8 warps per instance)
    long long warps = 0;
    for (int i = 0; i < n; ++i) warps += (b->info[i].geo.N + kBatchCmpAlign - 1) / kBatchCmpAlign * (kBatchCmpAlign / 32);
    b->n_part = std::max(b->units.size(), (size_t)warps);
    b->o_part = o;
    o += al256(sizeof(double) * b->n_part);
    b->o_part2 = o;
    o += al256(sizeof(double) * b->units.size());
    b->o_scal = o;
    o += al256(sizeof(double) * (size_t)n);
    for (int i = 0; i < 2; ++i) {
        b->o_ping[i] = o;
        o += b->state_bytes;
    }
    for (int i = 0; i < 2; ++i) {
        b->o_lam[i] = o;
        o += b->state_bytes;
    }
    b->o_ckpt = o;
    o += b->state_bytes * (size_t)(b->S - 1);
    b->o_seg = o;
    o += b->state_bytes * (size_t)b->k;
    b->total = o;
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b)
{
    delete b;
    return LBM_OK;
}

lbm_status lbm_batch_layout(const lbm_batch* b, int64_t* state_off, int64_t* node_off, int64_t* vel_off,
                            int64_t* inlet_off, size_t* ws_bytes)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i <= b->n; ++i) {
        if (state_off) state_off[i] = b->state_off[i];
        if (node_off) node_off[i] = b->node_off[i];
        if (vel_off) vel_off[i] = b->vel_off[i];
        if (inlet_off) inlet_off[i] = b->in_off[i];
    }
    if (ws_bytes) *ws_bytes = b->total;
    return LBM_OK;
}

lbm_status lbm_batch_init_geometry(lbm_batch* b, const lbm_geom_desc* g, uint8_t* d_mask, uint32_t* d_link,
                                   double* d_porosity, int64_t* d_info, void* d_ws, void* stream)
{
    if (!b || !g || !d_mask || !d_link || !d_info || !d_ws) return LBM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255u) || (reinterpret_cast<uintptr_t>(d_mask) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_link) & 15u))
        return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < b->n; ++i) {
        const lbm_geom_desc& gi = g[i];
        if (gi.kind == LBM_GEOM_DISKS && b->q != 9) return LBM_ERR_INVALID_ARG;
        if (gi.kind == LBM_GEOM_SPHERES && b->q != 19) return LBM_ERR_INVALID_ARG;
        if (gi.kind < LBM_GEOM_CHANNEL || gi.kind > LBM_GEOM_MASK) return LBM_ERR_INVALID_ARG;
        if (gi.kind == LBM_GEOM_DISKS || gi.kind == LBM_GEOM_SPHERES) {
            if (gi.r_min < 0 || gi.r_max < gi.r_min || gi.r_max > 4096 || gi.hydro_q8 < 0 || gi.hydro_q8 > 256 ||
                gi.inlet_buffer < 1 || gi.max_rejections < 1 ||
                !(gi.target_porosity >= 0.0 && gi.target_porosity <= 1.0))
                return LBM_ERR_INVALID_ARG;
        }
        lbm_status st = geometry_launch(b->info[i], gi, d_mask + b->node_off[i], d_link + b->node_off[i],
                                        d_porosity ? d_porosity + i : nullptr, d_info + 4 * i, s);
        if (st != LBM_OK) return st;
        b->insts[i].g.link = d_link + b->node_off[i];
    }
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    b->cmp = false;  // a new geometry invalidates fluid-only tables
    for (auto& gr : b->graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    b->graphs.clear();
    if (cudaMemsetAsync(ws + b->o_status, 0, 256, s) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(ws + b->o_insts, b->insts.data(), sizeof(BInst) * b->insts.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(ws + b->o_units, b->units.data(), sizeof(BUnit) * b->units.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;  // host tables must outlive the copies
    b->tables_ready = true;
    b->tables_ws = d_ws;
    return LBM_OK;
}

lbm_status lbm_batch_forward(lbm_batch* b, const double* d_rho_in, const double* d_tau, double rho_out, void* d_f,
                             void* d_ws, void* stream)
{
    lbm_status chk = check(b, d_ws);
    if (chk != LBM_OK) return chk;
    if (!d_rho_in || !d_tau || !d_f) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    const int T = b->desc.n_steps, k = b->k, S = b->S;
    auto slot = [&](int t) -> unsigned char* {
        const int s1 = t + 1;
        if (s1 % k == 0 && s1 / k >= 1 && s1 / k <= S - 1) return ws + b->o_ckpt + b->state_bytes * (size_t)(s1 / k - 1);
        return nullptr;
    };
    BCmpArgs ca = b->ca;
    ca.status = reinterpret_cast<uint32_t*>(ws + b->o_status);
    auto issue = [&](cudaStream_t st_) -> lbm_status {
        unsigned char* cur = slot(0) ? slot(0) : ws + b->o_ping[0];
        if (cudaMemsetAsync(cur, 0, b->cmp ? b->cmp_state_bytes : b->state_bytes, st_) != cudaSuccess)
            return LBM_ERR_CUDA;
        for (int t = 1; t <= T - 1; ++t) {
            unsigned char* dst = slot(t);
            if (!dst) dst = ws + b->o_ping[t & 1];
            lbm_status st = b->cmp ? bstep_launch_cmp(ca, kStreamCollide, cur, dst, false, d_rho_in, d_tau, rho_out, st_)
                                   : step(b, kStreamCollide, cur, dst, d_rho_in, d_tau, rho_out, ws, st_);
            if (st != LBM_OK) return st;
            cur = dst;
        }
        if (!b->cmp) return step(b, kStreamOnly, cur, d_f, d_rho_in, d_tau, rho_out, ws, st_);
        // fluid nodes only: the solid entries of the caller's packed array are zeroed first
        if (cudaMemsetAsync(d_f, 0, (size_t)b->state_elems * (size_t)b->prec, st_) != cudaSuccess) return LBM_ERR_CUDA;
        return bstep_launch_cmp(ca, kStreamOnly, cur, d_f, true, d_rho_in, d_tau, rho_out, st_);
    };
    return run_graph(b, b->cmp ? 11 : 1, {d_rho_in, d_tau, d_f, d_ws}, rho_out, s, issue);
}

lbm_status lbm_batch_loss_grad(lbm_batch* b, const void* d_f, const double* d_u_target, const uint8_t* d_roi,
                               double* d_loss, void* d_lambda, void* d_ws, void* stream)
{
    lbm_status chk = check(b, d_ws);
    if (chk != LBM_OK) return chk;
    if (!d_f || !d_u_target || !d_loss || !d_lambda) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    const int nu = (int)b->units.size();
    const dim3 grid((unsigned)((nu * 32 + kBatchThreads - 1) / kBatchThreads)), block(kBatchThreads);
    const BInst* I = reinterpret_cast<const BInst*>(ws + b->o_insts);
    const BUnit* U = reinterpret_cast<const BUnit*>(ws + b->o_units);
    uint32_t* st = reinterpret_cast<uint32_t*>(ws + b->o_status);
    double* part = reinterpret_cast<double*>(ws + b->o_part2);
    double* wgt = reinterpret_cast<double*>(ws + b->o_scal);
    const int kind = b->desc.loss_kind, mean = b->desc.loss_norm == LBM_NORM_MEAN_FLUID;
#define LBM_BATCH_LOSS(Q, T)                                                                                        \
    do {                                                                                                            \
        constexpr int V = batch_vec<Q, T>();                                                                           \
        k_batch_loss<Q, T, V><<<grid, block, 0, s>>>(I, U, nu, static_cast<const T*>(d_f), d_u_target, d_roi, kind, \
                                                     wgt, static_cast<T*>(d_lambda), part, 1);                      \
        k_batch_reduce<<<b->n, kReduceThreads, 0, s>>>(I, part, 1, mean, wgt, st);                                 \
        k_batch_loss<Q, T, V><<<grid, block, 0, s>>>(I, U, nu, static_cast<const T*>(d_f), d_u_target, d_roi, kind, \
                                                     wgt, static_cast<T*>(d_lambda), part, 0);                      \
        k_batch_reduce<<<b->n, kReduceThreads, 0, s>>>(I, part, 0, mean, d_loss, st);                              \
    } while (0)
    if (b->q == 9 && b->prec == 4) LBM_BATCH_LOSS(9, float);
    else if (b->q == 9 && b->prec == 8) LBM_BATCH_LOSS(9, double);
    else if (b->q == 19 && b->prec == 4) LBM_BATCH_LOSS(19, float);
    else LBM_BATCH_LOSS(19, double);
#undef LBM_BATCH_LOSS
    return cuda_status(cudaGetLastError());
}

lbm_status lbm_batch_adjoint(lbm_batch* b, const double* d_rho_in, const double* d_tau, double rho_out,
                             const void* d_lambda, double* d_grad_rho_in, double* d_grad_tau, void* d_ws,
                             void* stream)
{
    lbm_status chk = check(b, d_ws);
    if (chk != LBM_OK) return chk;
    if (!d_rho_in || !d_tau || !d_lambda || !d_grad_rho_in || !d_grad_tau) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    const int T = b->desc.n_steps, k = b->k, S = b->S;
    BCmpArgs ca = b->ca;
    ca.status = reinterpret_cast<uint32_t*>(ws + b->o_status);
    const size_t sb = b->cmp ? b->cmp_state_bytes : b->state_bytes;
    auto issue = [&](cudaStream_t st_) -> lbm_status {
        if (cudaMemsetAsync(ws + b->o_acc, 0, sizeof(double) * (size_t)b->acc_off.back(), st_) != cudaSuccess)
            return LBM_ERR_CUDA;
        if (cudaMemsetAsync(ws + b->o_part, 0, sizeof(double) * b->n_part, st_) != cudaSuccess) return LBM_ERR_CUDA;
        const void* lam_cur = d_lambda;
        int lam_next = 0;
        if (b->cmp) {  // lambda^T into the packed compact layout; its padding slots must start at zero
            if (cudaMemsetAsync(ws + b->o_lam[1], 0, b->cmp_state_bytes, st_) != cudaSuccess) return LBM_ERR_CUDA;
            lbm_status st = bgather_launch_cmp(ca, d_lambda, ws + b->o_lam[1], st_);
            if (st != LBM_OK) return st;
            lam_cur = ws + b->o_lam[1];
        }
        double* acc = reinterpret_cast<double*>(ws + b->o_acc);
        double* part = reinterpret_cast<double*>(ws + b->o_part);
        for (int sg = S - 1; sg >= 0; --sg) {
            const int t0 = sg * k, len = std::min(k, T - t0);
            auto seg = [&](int j) -> unsigned char* { return ws + b->o_seg + b->state_bytes * (size_t)j; };
            const unsigned char* base = sg >= 1 ? ws + b->o_ckpt + b->state_bytes * (size_t)(sg - 1) : nullptr;
            const unsigned char* prev = base;
            for (int j = 1; j < len; ++j) {
                if (sg == 0 && j == 1) {
                    if (cudaMemsetAsync(seg(1), 0, sb, st_) != cudaSuccess) return LBM_ERR_CUDA;
                } else {
                    lbm_status st =
                        b->cmp ? bstep_launch_cmp(ca, kStreamCollide, prev, seg(j), false, d_rho_in, d_tau, rho_out, st_)
                               : step(b, kStreamCollide, prev, seg(j), d_rho_in, d_tau, rho_out, ws, st_);
                    if (st != LBM_OK) return st;
                }
                prev = seg(j);
            }
            for (int j = len - 1; j >= 0; --j) {
                const unsigned char* src = j == 0 ? base : seg(j);
                void* lam_out = ws + b->o_lam[lam_next];
                const bool at0 = sg == 0 && j == 0;
                lbm_status st = b->cmp ? badjoint_launch_cmp(ca, at0 ? 1 : 0, src, lam_cur, lam_out, d_rho_in, d_tau,
                                                             rho_out, acc, part, st_)
                                       : adjoint(b, at0, src, lam_cur, lam_out, d_rho_in, d_tau, rho_out, ws, st_);
                if (st != LBM_OK) return st;
                lam_cur = lam_out;
                lam_next ^= 1;
            }
        }
        if (b->cmp)
            k_batch_finish_cmp<<<b->n, kReduceThreads, 0, st_>>>(ca.insts, part, acc, d_tau, d_grad_rho_in, d_grad_tau,
                                                                ca.status);
        else
            k_batch_finish<<<b->n, kReduceThreads, 0, st_>>>(
                reinterpret_cast<const BInst*>(ws + b->o_insts), part, acc, d_tau, d_grad_rho_in, d_grad_tau,
                ca.status);
        return cuda_status(cudaGetLastError());
    };
    return run_graph(b, b->cmp ? 13 : 3, {d_rho_in, d_tau, d_lambda, d_grad_rho_in, d_grad_tau, d_ws}, rho_out, s,
                     issue);
}

lbm_status lbm_batch_compact_size(const lbm_batch* b, const int64_t* n_fluid, size_t* bytes)
{
    if (!b || !n_fluid || !bytes) return LBM_ERR_INVALID_ARG;
    long long nfp = 0;
    for (int i = 0; i < b->n; ++i) {
        if (n_fluid[i] < 0 || n_fluid[i] > b->info[i].geo.N) return LBM_ERR_INVALID_ARG;
        nfp += (n_fluid[i] + kBatchCmpAlign - 1) / kBatchCmpAlign * kBatchCmpAlign;
    }
    *bytes = al256(sizeof(BCmpInst) * (size_t)b->n) + al256(sizeof(int) * (size_t)(nfp / kBatchCmpAlign)) +
             al256(sizeof(int32_t) * (size_t)nfp) + al256(sizeof(int32_t) * (size_t)(b->q - 1) * (size_t)nfp) +
             al256(sizeof(uint32_t) * (size_t)(nfp / 32));
    return LBM_OK;
}

lbm_status lbm_batch_compact_bind(lbm_batch* b, const int64_t* n_fluid, void* d_tables, void* d_ws, void* stream)
{
    if (!b || !b->tables_ready || d_ws != b->tables_ws) return LBM_ERR_INVALID_ARG;
    for (auto& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    if (!n_fluid) {  // back to the dense layout
        b->cmp = false;
        return LBM_OK;
    }
    if (!d_tables || (reinterpret_cast<uintptr_t>(d_tables) & 255u)) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    std::vector<BCmpInst> ci((size_t)b->n);
    long long nfp = 0;
    for (int i = 0; i < b->n; ++i) {
        if (n_fluid[i] < 0 || n_fluid[i] > b->info[i].geo.N) return LBM_ERR_INVALID_ARG;
        BCmpInst& c = ci[(size_t)i];
        c.g = b->insts[(size_t)i].g;
        c.k0 = nfp;
        c.nf = n_fluid[i];
        c.f_off = b->state_off[(size_t)i];
        c.in_off = b->in_off[(size_t)i];
        c.acc_off = b->acc_off[(size_t)i];
        c.n_in = b->info[(size_t)i].n_in;
        nfp += (c.nf + kBatchCmpAlign - 1) / kBatchCmpAlign * kBatchCmpAlign;
    }
    if (nfp >= (1LL << 31)) return LBM_ERR_INVALID_ARG;  // neighbour codes are int32
    unsigned char* tb = static_cast<unsigned char*>(d_tables);
    const size_t t_insts = 0, t_blk = al256(sizeof(BCmpInst) * (size_t)b->n);
    const size_t t_idx = t_blk + al256(sizeof(int) * (size_t)(nfp / kBatchCmpAlign));
    const size_t t_nbr = t_idx + al256(sizeof(int32_t) * (size_t)nfp);
    int32_t* idx = reinterpret_cast<int32_t*>(tb + t_idx);
    int32_t* nbr = reinterpret_cast<int32_t*>(tb + t_nbr);
    const size_t t_eq6 = t_nbr + al256(sizeof(int32_t) * (size_t)(b->q - 1) * (size_t)nfp);
    uint32_t* eq6 = reinterpret_cast<uint32_t*>(tb + t_eq6);
    std::vector<int> blk((size_t)(nfp / kBatchCmpAlign));
    // each instance's tables are built in the workspace's state buffers (free at this point), then
    // packed; compact_build checks the fluid count against the link words (and synchronises)
    // padding nodes: bounce-back in every direction (their loads stay at their own index)
    static_assert(kCmpBB == -1, "padding codes are written as all-ones bytes");
    if (nfp > 0 && cudaMemsetAsync(nbr, 0xFF, sizeof(int32_t) * (size_t)(b->q - 1) * (size_t)nfp, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    unsigned char* scratch = ws + b->o_ping[0];
    const size_t cap = b->o_ckpt - b->o_ping[0];
    for (int i = 0; i < b->n; ++i) {
        const BCmpInst& c = ci[(size_t)i];
        PlanInfo I = b->info[(size_t)i];
        I.geo.link = b->insts[(size_t)i].g.link;
        if (compact_table_bytes(I, c.nf) > cap) return LBM_ERR_INVALID_ARG;
        Cmp local{0, nullptr, nullptr};
        const int32_t* cmap = nullptr;
        lbm_status st = compact_build(I, c.nf, scratch, &local, &cmap, nullptr, s);
        if (st != LBM_OK) return st;
        st = bpack_launch_cmp(local, b->q, c.k0, nfp, idx, nbr, s);
        if (st != LBM_OK) return st;
        for (long long bl = c.k0 / kBatchCmpAlign; bl < (c.k0 + c.nf + kBatchCmpAlign - 1) / kBatchCmpAlign; ++bl)
            blk[(size_t)bl] = i;
    }
    {
        const lbm_status st = eq6_bits_launch_cmp(b->q, nbr, nfp, eq6, s);  // padding nodes: bounce-back, bit 0
        if (st != LBM_OK) return st;
    }
    if (cudaMemcpyAsync(tb + t_insts, ci.data(), sizeof(BCmpInst) * ci.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        (!blk.empty() &&
         cudaMemcpyAsync(tb + t_blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice, s) != cudaSuccess))
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;  // host vectors outlive the copies
    b->cinsts = ci;
    b->blk_inst = blk;
    b->nfp = nfp;
    b->cmp_state_bytes = (size_t)b->q * (size_t)nfp * (size_t)b->prec;
    BCmpArgs& a = b->ca;
    a.c = Cmp{nfp, idx, nbr, eq6};
    a.insts = reinterpret_cast<const BCmpInst*>(tb + t_insts);
    a.blk_inst = reinterpret_cast<const int*>(tb + t_blk);
    a.n_blocks = (unsigned)(nfp / kBatchCmpAlign);
    a.q = b->q;
    a.prec = b->prec;
    a.pdl = b->pdl ? 1 : 0;
    a.status = nullptr;  // set per call from the workspace
    b->cmp = true;
    return LBM_OK;
}

lbm_status lbm_batch_get_status(lbm_batch* b, void* d_ws, lbm_status* status)
{
    if (!b || !d_ws || !status || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return LBM_ERR_INVALID_ARG;
    *status = LBM_OK;
    uint32_t word = 0;
    uint32_t* dev = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(d_ws) + b->o_status);
    if (cudaMemcpy(&word, dev, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemset(dev, 0, sizeof(word)) != cudaSuccess) return LBM_ERR_CUDA;
    for (int bit = 1; bit < 32; ++bit)
        if (word & (1u << bit)) {
            *status = static_cast<lbm_status>(bit);
            break;
        }
    return LBM_OK;
}

}  // extern "C"
