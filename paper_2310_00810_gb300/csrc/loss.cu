// Loss at the final step and its seed, gradient finalisation, macroscopic
// fields, Darcy permeability and the Adam update (arXiv 2310.00810:
// compute_loss of section 2.2, Eq. 7, Eq. 15, Eq. 12, Eq. 9, section 3.4).
//
// All sums over nodes are FP64: per-block partials (warp shuffles, then
// shared memory) followed by one fixed-order pass, so results are
// deterministic run to run.
#include <cuda.h>

#include <algorithm>

#include <mutex>

#include "device.cuh"

namespace lbm {

// Fixed-order sum of a[0..n) by one block of kReduceThreads threads.
__device__ double block_reduce_array(const double* __restrict__ a, long long n)
{
    double v = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) v += a[i];
    return block_sum(v, threadIdx.x, blockDim.x);
}

// -------------------------------------------------------------- loss

__global__ void __launch_bounds__(kStepThreads) k_count_roi(Geo g, const uint8_t* __restrict__ roi,
                                                            double* __restrict__ partial)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    const long long n = ((long long)z * g.ny + y) * g.nx + x;
    double c = 0.0;
    if (x < g.nx && !(g.link[n] & kLinkSolid) && (!roi || roi[n])) c = 1.0;
    const double bs = block_sum(c, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) partial[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = bs;
}

// weight = 1 (sum) or 1 / count (mean over ROI fluid nodes)
__global__ void k_loss_weight(const double* __restrict__ partial, int nb, int mean, double* __restrict__ scalars)
{
    const double c = block_reduce_array(partial, nb);
    if (threadIdx.x == 0) {
        scalars[0] = c;
        scalars[1] = mean ? (c > 0.0 ? 1.0 / c : 0.0) : 1.0;
    }
}

// Per node: u from shifted f^T; loss term; lambda^T_k = sum_a dL/du_a (c_ka - u_a) / rho.
template <int Q, typename T, int KIND>
__global__ void __launch_bounds__(kStepThreads)
    k_loss(const T* __restrict__ f, const double* __restrict__ ut, const uint8_t* __restrict__ roi, Geo g,
           const double* __restrict__ weight, T* __restrict__ lam, double* __restrict__ partial)
{
    using L = Lattice<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    const long long N = g.N;
    const long long n = ((long long)z * g.ny + y) * g.nx + x;
    double term = 0.0;
    if (x < g.nx) {
        const uint32_t lw = g.link[n];
        T out[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i] = T(0);
        if (!(lw & kLinkSolid) && (!roi || roi[n])) {
            T v[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = f[(long long)i * N + n];
            T drho, rho, u[3];
            moments<Q, T>(v, drho, rho, u);
            const double wgt = *weight;
            double du[3] = {0.0, 0.0, 0.0};
            if (KIND == LBM_LOSS_VEC) {
#pragma unroll
                for (int a = 0; a < L::D; ++a) {
                    const double e = (double)u[a] - ut[(long long)a * N + n];
                    term += wgt * e * e;
                    du[a] = 2.0 * wgt * e;
                }
            } else {
                double uu = 0.0, tt = 0.0;
#pragma unroll
                for (int a = 0; a < L::D; ++a) {
                    uu += (double)u[a] * (double)u[a];
                    const double t = ut[(long long)a * N + n];
                    tt += t * t;
                }
                const double un = sqrt(uu);
                const double e = un - sqrt(tt);
                term += wgt * e * e;
                if (uu != 0.0)
#pragma unroll
                    for (int a = 0; a < L::D; ++a) du[a] = 2.0 * wgt * e * (double)u[a] / un;
            }
            const T inv = T(1) / rho;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                T s = 0;
#pragma unroll
                for (int a = 0; a < L::D; ++a) s += T(du[a]) * (T(L::c(k, a)) - u[a]);
                out[k] = s * inv;
            }
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) lam[(long long)k * N + n] = out[k];
    }
    const double bs = block_sum(term, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) partial[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = bs;
}

// Density probes, a second loss term (w sum_p (rho(x_p) - rho_p)^2) for the
// joint inversion of the head and tau, whose velocity field alone fixes only
// their ratio in the Stokes regime.  Adds the term to *d_loss and its seed
// 2 w (rho(x_p) - rho_p) to every direction of lambda^T at x_p (drho/df_k = 1,
// Eq. 1).  One block: the loss is summed in a fixed order; a node listed twice
// gets both seeds through atomics (their order, so the last bit, may vary).
// An out-of-range node latches LBM_ERR_INVALID_ARG and is skipped; a solid
// node contributes nothing.
template <int Q, typename T>
__global__ void __launch_bounds__(kReduceThreads)
    k_probe_loss(const T* __restrict__ f, Geo g, long long n_probe, const int64_t* __restrict__ node,
                 const double* __restrict__ rho_t, double w, double* __restrict__ d_loss, T* __restrict__ lam,
                 uint32_t* __restrict__ status)
{
    const long long N = g.N;
    double term = 0.0;
    for (long long p = threadIdx.x; p < n_probe; p += blockDim.x) {
        const long long n = node[p];
        if (n < 0 || n >= N) {
            atomicOr(status, 1u << LBM_ERR_INVALID_ARG);
            continue;
        }
        if (g.link[n] & kLinkSolid) continue;
        T s = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) s += f[(long long)i * N + n];
        const double e = (1.0 + (double)s) - rho_t[p];
        term += w * e * e;
        const T seed = T(2.0 * w * e);
#pragma unroll
        for (int k = 0; k < Q; ++k) atomicAdd(lam + (long long)k * N + n, seed);
    }
    const double bs = block_sum(term, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        *d_loss += bs;
        if (!isfinite(*d_loss)) atomicOr(status, 1u << LBM_ERR_NONFINITE);
    }
}

lbm_status probe_launch(const PlanInfo& p, const void* f, long long n_probe, const int64_t* node,
                        const double* rho_target, double weight, double* d_loss, void* lambda, uint32_t* status,
                        cudaStream_t s)
{
    const dim3 grid(1), block(kReduceThreads);
    if (p.q == 9 && p.prec == 4)
        k_probe_loss<9, float><<<grid, block, 0, s>>>(static_cast<const float*>(f), p.geo, n_probe, node, rho_target,
                                                      weight, d_loss, static_cast<float*>(lambda), status);
    else if (p.q == 9)
        k_probe_loss<9, double><<<grid, block, 0, s>>>(static_cast<const double*>(f), p.geo, n_probe, node,
                                                       rho_target, weight, d_loss, static_cast<double*>(lambda),
                                                       status);
    else if (p.prec == 4)
        k_probe_loss<19, float><<<grid, block, 0, s>>>(static_cast<const float*>(f), p.geo, n_probe, node, rho_target,
                                                       weight, d_loss, static_cast<float*>(lambda), status);
    else
        k_probe_loss<19, double><<<grid, block, 0, s>>>(static_cast<const double*>(f), p.geo, n_probe, node,
                                                        rho_target, weight, d_loss, static_cast<double*>(lambda),
                                                        status);
    return cuda_status(cudaGetLastError());
}

__global__ void k_loss_final(const double* __restrict__ partial, int nb, double* __restrict__ d_loss,
                             uint32_t* __restrict__ status)
{
    const double L = block_reduce_array(partial, nb);
    if (threadIdx.x == 0) {
        *d_loss = L;
        if (status && !isfinite(L)) atomicOr(status, 1u << LBM_ERR_NONFINITE);
    }
}

template <int Q, typename T>
static void loss_impl(const PlanInfo& p, const void* f, const double* ut, const uint8_t* roi, int kind, int norm,
                      double* d_loss, void* lambda, unsigned char* ws, const Workspace& w, cudaStream_t s)
{
    double* partial = reinterpret_cast<double*>(ws + w.partial2);
    double* scalars = reinterpret_cast<double*>(ws + w.status + kScalarCount);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + w.status);
    k_count_roi<<<p.grid, kStepThreads, 0, s>>>(p.geo, roi, partial);
    k_loss_weight<<<1, kReduceThreads, 0, s>>>(partial, p.n_blocks, norm == LBM_NORM_MEAN_FLUID, scalars);
    const T* fp = static_cast<const T*>(f);
    T* lp = static_cast<T*>(lambda);
    if (kind == LBM_LOSS_VEC)
        k_loss<Q, T, LBM_LOSS_VEC><<<p.grid, kStepThreads, 0, s>>>(fp, ut, roi, p.geo, scalars + 1, lp, partial);
    else
        k_loss<Q, T, LBM_LOSS_NORM><<<p.grid, kStepThreads, 0, s>>>(fp, ut, roi, p.geo, scalars + 1, lp, partial);
    k_loss_final<<<1, kReduceThreads, 0, s>>>(partial, p.n_blocks, d_loss, status);
}

lbm_status loss_launch(const PlanInfo& p, const void* f, const double* u_target, const uint8_t* roi, int kind,
                       int norm, double* d_loss, void* lambda, unsigned char* ws, const Workspace& w,
                       cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4) loss_impl<9, float>(p, f, u_target, roi, kind, norm, d_loss, lambda, ws, w, s);
    else if (p.q == 9 && p.prec == 8) loss_impl<9, double>(p, f, u_target, roi, kind, norm, d_loss, lambda, ws, w, s);
    else if (p.q == 19 && p.prec == 4) loss_impl<19, float>(p, f, u_target, roi, kind, norm, d_loss, lambda, ws, w, s);
    else if (p.q == 19 && p.prec == 8)
        loss_impl<19, double>(p, f, u_target, roi, kind, norm, d_loss, lambda, ws, w, s);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------- loss without a workspace

// Scratch of lbm_loss_grad_noalloc: two scalars, then one FP64 partial per
// thread block of the loss grid.  Every GPU that loads the library holds this
// array until the process exits.
constexpr int kNoallocHead = 32;  // doubles before the partials (count, weight, padding)
static __device__ __align__(256) double g_noalloc_scratch[kNoallocHead + LBM_NOALLOC_MAX_BLOCKS];

namespace {
constexpr int kMaxDevices = 64;

// The array's device address is looked up once per device and context: a
// device reset (cudaDeviceReset) or a new primary context loads the module
// again, possibly at another address, so the cached address is kept with the
// id of the context it was taken in and looked up again when that id changes.
struct NoallocAddr {
    unsigned long long ctx_id = 0;
    double* addr = nullptr;
};
NoallocAddr g_noalloc_addr[kMaxDevices];
std::mutex g_noalloc_mu;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context (driver entry points fetched
// through the runtime, so the library does not link the driver library).
bool current_context_id(unsigned long long* id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess || !a)
            return false;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qb != cudaDriverEntryPointSuccess || !b)
            return false;
        get_current = reinterpret_cast<PfnCtxGetCurrent>(a);
        get_id = reinterpret_cast<PfnCtxGetId>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

lbm_status loss_launch_noalloc(const PlanInfo& p, const void* f, const double* u_target, const uint8_t* roi, int kind,
                               int norm, double* d_loss, void* lambda, cudaStream_t s)
{
    if (p.n_blocks > LBM_NOALLOC_MAX_BLOCKS) return LBM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
    // makes the device's primary context current on this thread (the runtime
    // initialises it here), so that its id can be read; allocates nothing
    if (cudaSetDevice(dev) != cudaSuccess) return LBM_ERR_CUDA;
    unsigned long long ctx_id = 0;
    if (!current_context_id(&ctx_id)) return LBM_ERR_CUDA;
    double* base = nullptr;
    {
        // set-up per device and context (with that device current): the
        // host-side name of the array is not a device address, so ask the
        // runtime for it
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoallocAddr& a = g_noalloc_addr[dev];
        if (!a.addr || a.ctx_id != ctx_id) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LBM_ERR_CUDA;
            a.addr = static_cast<double*>(ptr);
            a.ctx_id = ctx_id;
        }
        base = a.addr;
    }
    double* scalars = base;  // [0] ROI fluid count, [1] loss weight
    double* partial = base + kNoallocHead;
    // the scalars and the partials are fully overwritten before they are read
    k_count_roi<<<p.grid, kStepThreads, 0, s>>>(p.geo, roi, partial);
    k_loss_weight<<<1, kReduceThreads, 0, s>>>(partial, p.n_blocks, norm == LBM_NORM_MEAN_FLUID, scalars);
#define LBM_NOALLOC_LOSS(Q, T)                                                                                     \
    do {                                                                                                           \
        const T* fp = static_cast<const T*>(f);                                                                    \
        T* lp = static_cast<T*>(lambda);                                                                           \
        if (kind == LBM_LOSS_VEC)                                                                                  \
            k_loss<Q, T, LBM_LOSS_VEC><<<p.grid, kStepThreads, 0, s>>>(fp, u_target, roi, p.geo, scalars + 1, lp,    \
                                                                       partial);                                   \
        else                                                                                                       \
            k_loss<Q, T, LBM_LOSS_NORM><<<p.grid, kStepThreads, 0, s>>>(fp, u_target, roi, p.geo, scalars + 1, lp,   \
                                                                        partial);                                  \
    } while (0)
    if (p.q == 9 && p.prec == 4) LBM_NOALLOC_LOSS(9, float);
    else if (p.q == 9 && p.prec == 8) LBM_NOALLOC_LOSS(9, double);
    else if (p.q == 19 && p.prec == 4) LBM_NOALLOC_LOSS(19, float);
    else if (p.q == 19 && p.prec == 8) LBM_NOALLOC_LOSS(19, double);
    else return LBM_ERR_UNSUPPORTED;
#undef LBM_NOALLOC_LOSS
    // no status word on this path: a non-finite loss shows as NaN/Inf in d_loss
    k_loss_final<<<1, kReduceThreads, 0, s>>>(partial, p.n_blocks, d_loss, nullptr);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------- sums of a time-window loss

__global__ void k_accumulate(double* __restrict__ dst, const double* __restrict__ src) { *dst += *src; }

template <typename T>
__global__ void k_add_state(T* __restrict__ dst, const T* __restrict__ src, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

lbm_status accumulate_launch(double* dst, const double* src, cudaStream_t s)
{
    k_accumulate<<<1, 1, 0, s>>>(dst, src);
    return cuda_status(cudaGetLastError());
}

// dst += src over a dense state (Q N values of the plan's precision).
lbm_status add_state_launch(const PlanInfo& p, void* dst, const void* src, cudaStream_t s)
{
    const long long n = (long long)p.q * p.geo.N;
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 4096);
    if (p.prec == 4) k_add_state<float><<<grid, 256, 0, s>>>(static_cast<float*>(dst), static_cast<const float*>(src), n);
    else k_add_state<double><<<grid, 256, 0, s>>>(static_cast<double*>(dst), static_cast<const double*>(src), n);
    return cuda_status(cudaGetLastError());
}

// ----------------------------------------------------- gradient finalise

// dL/dtau = -(sum of dL/domega partials) / tau^2 ; dL/drho_in from the
// per-inlet-node accumulators (summed for a constant head).
__global__ void k_finish_gradients(const double* __restrict__ grad_acc, int n_acc, int profile,
                                   const double* __restrict__ partial, int nb, const double* __restrict__ tau,
                                   double* __restrict__ g_rho_in, double* __restrict__ g_tau,
                                   uint32_t* __restrict__ status)
{
    const double gw = block_reduce_array(partial, nb);
    double gsum = 0.0;
    if (!profile) gsum = block_reduce_array(grad_acc, n_acc);
    bool bad = false;
    if (profile)
        for (int i = threadIdx.x; i < n_acc; i += blockDim.x) {
            g_rho_in[i] = grad_acc[i];
            bad |= !isfinite(grad_acc[i]);
        }
    if (threadIdx.x == 0) {
        const double t = *tau;
        *g_tau = -gw / (t * t);
        if (!profile) g_rho_in[0] = gsum;
        bad |= !isfinite(gw) || !isfinite(gsum);
    }
    if (bad) atomicOr(status, 1u << LBM_ERR_NONFINITE);
}

lbm_status finish_gradients_launch(const PlanInfo& p, const double* grad_acc, const double* partial,
                                   const double* tau, double* d_grad_rho_in, double* d_grad_tau, uint32_t* status,
                                   cudaStream_t s)
{
    k_finish_gradients<<<1, kReduceThreads, 0, s>>>(grad_acc, p.n_acc, p.n_in > 1 ? 1 : 0, partial, p.n_partial, tau,
                                                    d_grad_rho_in, d_grad_tau, status);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------- macroscopic

template <int Q, typename T>
__global__ void __launch_bounds__(kStepThreads)
    k_macroscopic(const T* __restrict__ f, Geo g, double* __restrict__ rho_out, double* __restrict__ u_out)
{
    using L = Lattice<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const long long N = g.N, n = ((long long)z * g.ny + y) * g.nx + x;
    double r = 0.0, u[3] = {0.0, 0.0, 0.0};
    if (!(g.link[n] & kLinkSolid)) {
        double s = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = (double)f[(long long)i * N + n];
            s += v;
#pragma unroll
            for (int a = 0; a < L::D; ++a) j[a] += L::c(i, a) * v;
        }
        r = 1.0 + s;
#pragma unroll
        for (int a = 0; a < L::D; ++a) u[a] = j[a] / r;
    }
    if (rho_out) rho_out[n] = r;
#pragma unroll
    for (int a = 0; a < L::D; ++a) u_out[(long long)a * N + n] = u[a];
}

lbm_status macroscopic_launch(const PlanInfo& p, const void* f, double* rho, double* u, cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4)
        k_macroscopic<9, float><<<p.grid, kStepThreads, 0, s>>>(static_cast<const float*>(f), p.geo, rho, u);
    else if (p.q == 9 && p.prec == 8)
        k_macroscopic<9, double><<<p.grid, kStepThreads, 0, s>>>(static_cast<const double*>(f), p.geo, rho, u);
    else if (p.q == 19 && p.prec == 4)
        k_macroscopic<19, float><<<p.grid, kStepThreads, 0, s>>>(static_cast<const float*>(f), p.geo, rho, u);
    else if (p.q == 19 && p.prec == 8)
        k_macroscopic<19, double><<<p.grid, kStepThreads, 0, s>>>(static_cast<const double*>(f), p.geo, rho, u);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------- Darcy

// k = nu J / (dp/dx), J = section mean of rho u_x, nu = (tau - 1/2)/3 (Eq. 9),
// dp/dx = (mean rho_in - rho_out) / (3 nx)  (Eq. 12).
template <int Q, typename T>
__global__ void k_darcy(const T* __restrict__ f, Geo g, const double* __restrict__ rho_in, int n_in,
                        const double* __restrict__ tau, double rho_out, int xs, double* __restrict__ k,
                        double* __restrict__ flux)
{
    using L = Lattice<Q>;
    const long long N = g.N;
    const long long cells = (long long)g.ny * g.nz;
    double J = 0.0;
    for (long long c = threadIdx.x; c < cells; c += blockDim.x) {
        const long long n = c * g.nx + xs;  // c = z * ny + y
        if (g.link[n] & kLinkSolid) continue;
        double jx = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (L::c(i, 0) != 0) jx += L::c(i, 0) * (double)f[(long long)i * N + n];
        J += jx;  // rho u_x = sum_i c_ix f_i (the rest shift has zero momentum)
    }
    J = block_sum(J, threadIdx.x, blockDim.x);
    const double rin = block_reduce_array(rho_in, n_in);
    if (threadIdx.x == 0) {
        J /= (double)cells;
        const double nu = (*tau - 0.5) / 3.0;
        const double dpdx = (rin / n_in - rho_out) / (3.0 * g.nx);
        *k = nu * J / dpdx;
        if (flux) *flux = J;
    }
}

lbm_status darcy_launch(const PlanInfo& p, const void* f, const double* rho_in, int n_in, const double* tau,
                        double rho_out, int xs, double* k, double* flux, cudaStream_t s)
{
    if (p.q == 9 && p.prec == 4)
        k_darcy<9, float><<<1, kReduceThreads, 0, s>>>(static_cast<const float*>(f), p.geo, rho_in, n_in, tau,
                                                        rho_out, xs, k, flux);
    else if (p.q == 9 && p.prec == 8)
        k_darcy<9, double><<<1, kReduceThreads, 0, s>>>(static_cast<const double*>(f), p.geo, rho_in, n_in, tau,
                                                         rho_out, xs, k, flux);
    else if (p.q == 19 && p.prec == 4)
        k_darcy<19, float><<<1, kReduceThreads, 0, s>>>(static_cast<const float*>(f), p.geo, rho_in, n_in, tau,
                                                         rho_out, xs, k, flux);
    else if (p.q == 19 && p.prec == 8)
        k_darcy<19, double><<<1, kReduceThreads, 0, s>>>(static_cast<const double*>(f), p.geo, rho_in, n_in, tau,
                                                          rho_out, xs, k, flux);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

// -------------------------------------------------------------- Adam

__global__ void k_adam(int n, double* __restrict__ theta, double* __restrict__ m, double* __restrict__ v,
                       const double* __restrict__ grad_p, double* __restrict__ p, double off, double scale, double bc1,
                       double bc2, double lr, double b1, double b2, double eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double g = grad_p[i] * scale;  // dL/dtheta = dL/dp * dp/dtheta
    const double mi = b1 * m[i] + (1.0 - b1) * g;
    const double vi = b2 * v[i] + (1.0 - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const double th = theta[i] - lr * (mi / bc1) / (sqrt(vi / bc2) + eps);
    theta[i] = th;
    p[i] = off + scale * th;
}

lbm_status adam_launch(int n, double* theta, double* m, double* v, const double* grad_p, double* p, double off,
                       double scale, int t, double lr, double b1, double b2, double eps, cudaStream_t s)
{
    const double bc1 = 1.0 - pow(b1, (double)t), bc2 = 1.0 - pow(b2, (double)t);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(n, theta, m, v, grad_p, p, off, scale, bc1, bc2, lr, b1, b2, eps);
    return cuda_status(cudaGetLastError());
}

}  // namespace lbm
