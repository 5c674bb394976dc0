// Reverse (adjoint) lattice step: the exact transpose of one forward step
// f^{t+1} = S(C(f^t)) (Eq. 3-6 of arXiv 2310.00810), written by hand in
// gather form.  It replaces the paper's Taichi tape (section 2.2).
//
// With lambda^t = dL/df^t and mu^t = dL/df*^t (adjoint of the
// post-collision state), one launch computes at every fluid node x:
//   1. f^t(x) by pulling the stored post-collision state g^{t-1} (the same
//      pull as the forward kernel; f^0 is the rest state);
//   2. mu_j(x) = transpose of streaming: the forward copies f*_j(x) to
//        lambda_j(x + c_j)          (x + c_j fluid)
//        lambda_opp(j)(x)           (bounce-back link)
//       -lambda_opp(j)(x)           (anti-bounce-back link, Eq. 6)
//      so mu_j gathers from x + c_j: the adjoint pull runs the other way;
//   3. transpose of BGK, f*_j = (1 - w) f_j + w f^eq_j(rho(f), u(f)):
//        lambda_k = (1 - w) mu_k + w A + sum_a (w B_a + G_a) (c_ka - u_a) / rho,
//        A   = sum_j mu_j w_j P_j,  P_j = 1 + 3 c_j.u + 4.5 (c_j.u)^2 - 1.5 u.u,
//        B_a = sum_j mu_j w_j rho (3 c_ja + 9 (c_j.u) c_ja - 3 u_a),
//        G_a = sum over this node's Eq. 6 links i of lambda_i 2 w_i rho_w (9 (c_i.u) c_ia - 3 u_a)
//      (Eq. 6 uses the node's own u at time t);
//   4. dL/domega += sum_j mu_j (f^eq_j - f_j)  (one FP64 partial per block,
//      accumulated in place across steps: fixed order, no atomics);
//      dL/drho_w(y, z) += sum over Eq. 6 inlet links of lambda_i 2 w_i (1 + 4.5 (c_i.u)^2 - 1.5 u.u)
//      (one owner thread per inlet node, accumulated in place across steps).
// With the extrapolated Eq. 6 velocity a second, per-row pass adds what the
// extrapolation changes (k_adjoint_uw).
#include "device.cuh"

namespace lbm {

template <int Q, typename T, bool T0>
__global__ void __launch_bounds__(kStepThreads)
    k_adjoint(const T* __restrict__ gprev, const T* __restrict__ lam_in, T* __restrict__ lam_out, Geo g, Bc bc,
              const double* __restrict__ tau, double* __restrict__ grad_acc, double* __restrict__ partial)
{
    pdl_enter();
    using L = Lattice<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    const long long N = g.N, plane = (long long)g.nx * g.ny;
    const long long n = ((long long)z * g.ny + y) * g.nx + x;
    uint32_t lw = kLinkSolid;
    if (x < g.nx) lw = g.link[n];
    double dom = 0.0;
    if (!(lw & kLinkSolid)) {
        // 1. f^t(x)
        T f[Q];
        if (T0) {
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = T(0);
        } else {
            pull<Q, T>(f, gprev, n, x, y, z, lw, g, bc);
        }
        T drho, rho, u[3];
        moments<Q, T>(f, drho, rho, u);
        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const T omega = T(1.0 / *tau);

        // 2. transpose of streaming and boundaries
        const bool xin = x == 0, xout = x == g.nx - 1;
        T mu[Q];
        T G[3] = {T(0), T(0), T(0)};
        double grw = 0.0;
        T rwT = T(0);
        if (xin || xout) rwT = T(xin ? (bc.profile ? bc.rho_in[(long long)z * g.ny + y] : bc.rho_in[0]) : bc.rho_out);
        if (!(xin || xout)) {
            // interior node: select the address, then load (all Q loads in flight together)
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int o = L::opp(j);
                const bool bb = (lw >> o) & 1u;
                mu[j] = lam_in[bb ? (long long)o * N + n : (long long)j * N + n + link_offset<Q>(j, g.nx, plane)];
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int o = L::opp(j), cx = L::c(j, 0);
                if ((lw >> o) & 1u) {
                    mu[j] = lam_in[(long long)o * N + n];
                } else if ((cx == -1 && xin) || (cx == 1 && xout)) {
                    const T li = lam_in[(long long)o * N + n];
                    mu[j] = -li;
                    const T cu = cdot<Q, T>(o, u);
                    const T two_w = T(2.0 * L::w(o));
                    if (xin) grw += (double)(li * two_w * (T(1) + T(4.5) * cu * cu - T(1.5) * uu));
#pragma unroll
                    for (int a = 0; a < L::D; ++a)
                        G[a] += li * two_w * rwT * (T(9) * cu * T(L::c(o, a)) - T(3) * u[a]);
                } else {
                    mu[j] = lam_in[(long long)j * N + n + link_offset<Q>(j, g.nx, plane)];
                }
            }
        }

        // 3. transpose of the collision (BGK here, MRT in adjoint_collision_mrt)
        T lamv[Q], domT = 0;
        bool mrt_done = false;
        if constexpr (Q == 9) {
            if (bc.mrt) {
                domT = adjoint_collision_mrt<T>(f, mu, drho, rho, u, G, omega, mrt_rates(bc.status), lamv);
                mrt_done = true;
            }
        }
        if (!mrt_done) {
            T A = 0, B[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const T cu = cdot<Q, T>(j, u);
                const T wj = T(L::w(j));
                const T P = T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
                const T feq = wj * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
                domT += mu[j] * (feq - f[j]);
                A += mu[j] * wj * P;
#pragma unroll
                for (int a = 0; a < L::D; ++a)
                    B[a] += mu[j] * wj * rho * (T(3 * L::c(j, a)) + T(9) * cu * T(L::c(j, a)) - T(3) * u[a]);
            }
            const T inv = T(1) / rho;
            T Bt[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) Bt[a] = (omega * B[a] + G[a]) * inv;
            const T base = omega * A;
            const T keep = T(1) - omega;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                T sk = keep * mu[k] + base;
#pragma unroll
                for (int a = 0; a < L::D; ++a) sk += Bt[a] * (T(L::c(k, a)) - u[a]);
                lamv[k] = sk;
            }
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) lam_out[(long long)k * N + n] = lamv[k];

        // 4. parameter gradients
        dom = (double)domT;
        if (xin) grad_acc[(long long)z * g.ny + y] += grw;
    }
    const int tid = threadIdx.x;
    const double bs = block_sum(dom, tid, blockDim.x);
    if (tid == 0) partial[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] += bs;
}

// Reverse of the extrapolated Eq. 6 velocity (Bc::uw_extrap), run after the
// adjoint step: one thread per row adds adjoint_uw_delta at the row's inlet
// node and its inward neighbour, then at the outlet node and its neighbour
// (one thread for both sides, so the two never race on a short row).  A side
// whose boundary node or inward neighbour is solid keeps the node velocity
// and needs nothing.  Not used at t = 0: at rest u = u_w = 0 and every delta
// vanishes.
template <int Q, typename T>
__global__ void __launch_bounds__(kStepThreads)
    k_adjoint_uw(const T* __restrict__ gprev, const T* __restrict__ lam_in, T* __restrict__ lam_out, Geo g, Bc bc,
                 double* __restrict__ grad_acc)
{
    pdl_enter();
    using L = Lattice<Q>;
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (long long)g.ny * g.nz) return;
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const long long N = g.N;
    for (int side = 0; side < 2; ++side) {
        const bool xin = side == 0;
        const int xb = xin ? 0 : g.nx - 1, xe = xin ? 1 : g.nx - 2;
        const long long nb = row * g.nx + xb, ne = row * g.nx + xe;
        const uint32_t lb = g.link[nb];
        if ((lb & kLinkSolid) || ((lb >> inward_dir<Q>(xin)) & 1u)) continue;
        T fb[Q], fe[Q], li[Q];
        pull<Q, T>(fb, gprev, nb, xb, y, z, lb, g, bc);
        pull<Q, T>(fe, gprev, ne, xe, y, z, g.link[ne], g, bc);
        uint32_t eq6 = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0);
            const bool on = ((cx == 1 && xin) || (cx == -1 && !xin)) && !((lb >> i) & 1u);
            eq6 |= on ? (1u << i) : 0u;
            li[i] = on ? lam_in[(long long)i * N + nb] : T(0);
        }
        const T rw = T(xin ? (bc.profile ? bc.rho_in[row] : bc.rho_in[0]) : bc.rho_out);
        T db[Q], de[Q];
        const double dg = adjoint_uw_delta<Q, T>(fb, fe, li, eq6, rw, db, de);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            lam_out[(long long)k * N + nb] += db[k];
            lam_out[(long long)k * N + ne] += de[k];
        }
        if (xin) grad_acc[row] += dg;
    }
}

template <int Q, typename T>
static void launch_uw(const PlanInfo& p, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                      double* grad_acc, cudaStream_t s)
{
    const long long rows = (long long)p.geo.ny * p.geo.nz;
    launch_k(p.pdl, k_adjoint_uw<Q, T>, dim3((unsigned)((rows + kStepThreads - 1) / kStepThreads)), dim3(kStepThreads),
             0, s, static_cast<const T*>(gprev), static_cast<const T*>(lam_in), static_cast<T*>(lam_out), p.geo, bc,
             grad_acc);
}

template <int Q, typename T>
static void launch(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                   const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    const T* gp = static_cast<const T*>(gprev);
    const T* li = static_cast<const T*>(lam_in);
    T* lo = static_cast<T*>(lam_out);
    if (t0)
        launch_k(p.pdl, k_adjoint<Q, T, true>, dim3(p.grid), dim3(kStepThreads), 0, s, gp, li, lo, p.geo, bc, tau, grad_acc, partial);
    else
        launch_k(p.pdl, k_adjoint<Q, T, false>, dim3(p.grid), dim3(kStepThreads), 0, s, gp, li, lo, p.geo, bc, tau, grad_acc, partial);
}

lbm_status adjoint_launch(const PlanInfo& plan, int t_is_zero, const void* gprev, const void* lam_in, void* lam_out,
                          const Bc& bc, const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    if (plan.cmp.nf) return adjoint_launch_cmp(plan, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    if (bc.uw_extrap || bc.mrt) {
        // the extrapolated u_w and the MRT collision run on the one-node-per-thread kernels
        // (plus, for u_w, its reverse pass)
        const PlanInfo p = with_family(plan, LBM_FAMILY_SCALAR);
        if (p.q == 9 && p.prec == 4) launch<9, float>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
        else if (p.q == 9 && p.prec == 8)
            launch<9, double>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
        else if (p.q == 19 && p.prec == 4)
            launch<19, float>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
        else if (p.q == 19 && p.prec == 8)
            launch<19, double>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
        else return LBM_ERR_UNSUPPORTED;
        if (bc.uw_extrap && !t_is_zero) {
            if (p.q == 9 && p.prec == 4) launch_uw<9, float>(p, gprev, lam_in, lam_out, bc, grad_acc, s);
            else if (p.q == 9) launch_uw<9, double>(p, gprev, lam_in, lam_out, bc, grad_acc, s);
            else if (p.prec == 4) launch_uw<19, float>(p, gprev, lam_in, lam_out, bc, grad_acc, s);
            else launch_uw<19, double>(p, gprev, lam_in, lam_out, bc, grad_acc, s);
        }
        return cuda_status(cudaGetLastError());
    }
    const PlanInfo p = with_family(plan, plan.adj_family);
    if (adjoint_launch_tma(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s))
        return cuda_status(cudaGetLastError());
    if (adjoint_launch_vec(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s))
        return cuda_status(cudaGetLastError());
    if (p.q == 9 && p.prec == 4) launch<9, float>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    else if (p.q == 9 && p.prec == 8)
        launch<9, double>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    else if (p.q == 19 && p.prec == 4)
        launch<19, float>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    else if (p.q == 19 && p.prec == 8)
        launch<19, double>(p, t_is_zero, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

}  // namespace lbm
