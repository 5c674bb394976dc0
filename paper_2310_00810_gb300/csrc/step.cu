// Forward lattice update: fused pull-streaming, halfway bounce-back,
// anti-bounce-back pressure planes and BGK collision (arXiv 2310.00810,
// section 2.1, Eq. 1-6, and the "Bounce Back" stage of section 2.2).
//
// The library keeps the POST-collision state g^t = f*^t in memory, so one
// launch in stream-collide mode computes g^{t+1} = C(S(g^t)): each node
// pulls what streams into it (from x - c_i), applies the boundary rules on
// its own links, then collides in registers and stores locally.  The paper's
// cycle f^{t+1} = S(C(f^t)) is recovered as
//     f^T = S o (C o S)^{T-1} o C (f^0),
// i.e. one collide-only launch (or the rest state, which collision leaves
// unchanged), T - 1 stream-collide launches and one stream-only launch.
// Populations are stored shifted by the rest state (f - w_i), which keeps
// FP32 from cancelling 1 - 1e-4 size differences.
//
// Link rules for what fluid node x receives in direction i (the link from
// x - c_i):
//   bounce-back bit i set in the link word   ->  g_opp(i)(x)
//   x - c_i beyond the plane x = -1/2 / nx - 1/2 (and not a wall link)
//        -> -g_opp(i)(x) + 2 w_i (rho_w (1 + 4.5 (c_i.u_w)^2 - 1.5 u_w.u_w) - 1)   (Eq. 6,
//           shifted; u_w is the node's own velocity at time t, from its
//           post-collision populations, which collision does not change, or
//           with Bc::uw_extrap that velocity extrapolated to the plane)
//   otherwise                                  ->  g_i(x - c_i)
#include "device.cuh"

namespace lbm {

template <int Q, typename T, int MODE>
__global__ void __launch_bounds__(kStepThreads) k_step(const T* __restrict__ src, T* __restrict__ dst, Geo g, Bc bc,
                                                        const double* __restrict__ tau)
{
    pdl_enter();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const long long n = ((long long)z * g.ny + y) * g.nx + x;
    const uint32_t lw = g.link[n];
    if (lw & kLinkSolid) return;
    T v[Q];
    if (MODE == kCollideOnly) {
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = src[(long long)i * g.N + n];
    } else {
        pull<Q, T>(v, src, n, x, y, z, lw, g, bc);
    }
    if (MODE != kStreamOnly) collide_any<Q, T>(v, T(1.0 / *tau), bc);
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[(long long)i * g.N + n] = v[i];
}

template <int Q, typename T>
static void launch(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                   cudaStream_t s)
{
    const T* a = static_cast<const T*>(src);
    T* b = static_cast<T*>(dst);
    dim3 block(kStepThreads);
    if (mode == kStreamCollide)
        launch_k(p.pdl, k_step<Q, T, kStreamCollide>, dim3(p.grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
    else if (mode == kCollideOnly)
        launch_k(p.pdl, k_step<Q, T, kCollideOnly>, dim3(p.grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
    else
        launch_k(p.pdl, k_step<Q, T, kStreamOnly>, dim3(p.grid), dim3(block), 0, s, a, b, p.geo, bc, tau);
}

lbm_status step_launch(const PlanInfo& plan, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                       cudaStream_t s)
{
    if (plan.cmp.nf) return step_launch_cmp(plan, mode, src, dst, false, false, bc, tau, s);
    // the extrapolated Eq. 6 velocity and the MRT collision are implemented by the one-node-per-thread kernels
    const PlanInfo p = with_family(plan, (bc.uw_extrap || bc.mrt) ? LBM_FAMILY_SCALAR : plan.step_family);
    if (step_launch_tma(p, mode, src, dst, bc, tau, s)) return cuda_status(cudaGetLastError());
    if (step_launch_vec(p, mode, src, dst, bc, tau, s)) return cuda_status(cudaGetLastError());
    if (p.q == 9 && p.prec == 4) launch<9, float>(p, mode, src, dst, bc, tau, s);
    else if (p.q == 9 && p.prec == 8) launch<9, double>(p, mode, src, dst, bc, tau, s);
    else if (p.q == 19 && p.prec == 4) launch<19, float>(p, mode, src, dst, bc, tau, s);
    else if (p.q == 19 && p.prec == 8) launch<19, double>(p, mode, src, dst, bc, tau, s);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

// Two stream-collide steps in one launch, g^{t+1} = C S C S (g^{t-1}), and
// g^t into mid (nullable): the temporally blocked TMA kernel of the dense
// D2Q9 FP32 layout (node-velocity Eq. 6, BGK).  step2_possible says whether
// it applies; step2_launch otherwise runs the two steps as two launches
// (through mid, which must then be a state buffer).
bool step2_possible(const PlanInfo& p, const Bc& bc)
{
    const PlanInfo q = with_family(p, p.step_family);
    return p.steps2 && !p.cmp.nf && p.q == 9 && p.prec == 4 && p.geo.nx % 4 == 0 && q.use_tma && p.tma_variant == 1 &&
           !bc.uw_extrap && !bc.mrt && (reinterpret_cast<uintptr_t>(p.geo.link) & 15u) == 0;
}

lbm_status step2_launch(const PlanInfo& p, const void* src, void* mid, void* dst, const Bc& bc, const double* tau,
                        cudaStream_t s)
{
    if (step2_possible(p, bc) && step2_launch_tma(with_family(p, p.step_family), src, dst, mid, bc, tau, s))
        return cuda_status(cudaGetLastError());
    if (!mid) return LBM_ERR_INVALID_ARG;
    lbm_status st = step_launch(p, kStreamCollide, src, mid, bc, tau, s);
    if (st != LBM_OK) return st;
    return step_launch(p, kStreamCollide, mid, dst, bc, tau, s);
}

}  // namespace lbm
