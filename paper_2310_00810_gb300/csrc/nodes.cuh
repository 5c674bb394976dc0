// Per-node pieces shared by the vectorised register kernels (vstep.cu) and
// the TMA-staged kernels (tma.cu): vector loads/stores, the boundary rules
// of the pull (Eq. 3, Eq. 6, halfway bounce-back) and the adjoint of one
// step at a group of VEC consecutive nodes of a row.
#pragma once

#include "device.cuh"

namespace lbm {

template <typename T, int VEC>
struct Vec;
template <>
struct Vec<float, 4> {
    using type = float4;
    __device__ static void load(const float* p, float (&o)[4])
    {
        const float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
    }
    __device__ static void store(float* p, const float (&o)[4])
    {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <>
struct Vec<float, 2> {
    __device__ static void load(const float* p, float (&o)[2])
    {
        const float2 t = *reinterpret_cast<const float2*>(p);
        o[0] = t.x, o[1] = t.y;
    }
    __device__ static void store(float* p, const float (&o)[2]) { *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]); }
};
template <>
struct Vec<double, 2> {
    __device__ static void load(const double* p, double (&o)[2])
    {
        const double2 t = *reinterpret_cast<const double2*>(p);
        o[0] = t.x, o[1] = t.y;
    }
    __device__ static void store(double* p, const double (&o)[2])
    {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};

// Boundary rules of the pull (halfway bounce-back, Eq. 6) applied to the
// values a lane's VEC nodes received from their neighbours: bounce-back links
// take the node's own post-collision population of the opposite direction,
// anti-bounce-back links at x = 0 / nx - 1 the Eq. 6 value built from the
// node's own velocity at time t.  Reads the node's own state from `src`.
template <int Q, typename T, int VEC>
__device__ __forceinline__ void pull_fixup(T (&v)[Q][VEC], const T* __restrict__ src, long long n0, int x0, int y,
                                           int z, const uint32_t (&lw)[VEC], const Geo& g, const Bc& bc)
{
    using L = Lattice<Q>;
    const long long N = g.N;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const uint32_t w = lw[j];
        if (w & kLinkSolid) continue;
        const long long n = n0 + j;
        const int x = x0 + j;
        if (x == 0 || x == g.nx - 1) {
            const bool xin = x == 0;
            T loc[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) loc[i] = src[(long long)i * N + n];
            T drho, rho, u[3];
            moments<Q, T>(loc, drho, rho, u);
            const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const double rw = xin ? (bc.profile ? bc.rho_in[(long long)z * g.ny + y] : bc.rho_in[0]) : bc.rho_out;
            const T drw = T(rw - 1.0), rwT = T(rw);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = L::c(i, 0);
                if ((w >> i) & 1u) {
                    v[i][j] = loc[L::opp(i)];
                } else if ((cx == 1 && xin) || (cx == -1 && !xin)) {
                    const T cu = cdot<Q, T>(i, u);
                    v[i][j] = -loc[L::opp(i)] + T(2.0 * L::w(i)) * (drw + rwT * (T(4.5) * cu * cu - T(1.5) * uu));
                }
            }
        } else if (w) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((w >> i) & 1u) v[i][j] = src[(long long)L::opp(i) * N + n];
        }
    }
}


// The adjoint of one step at a lane's VEC nodes (the algebra of adjoint.cu):
// on entry f holds f^t (pulled and fixed up) and mu the values gathered from
// lambda^{t+1} at x + c_j; the bounce-back / Eq. 6 links are fixed up here
// from the node's own lambda^{t+1}, then mu is overwritten with lambda^t.
// Returns this lane's sum of dL/domega contributions; adds the inlet nodes'
// dL/drho_w to grad_acc (one owner per inlet node).
template <int Q, typename T, int VEC>
__device__ __forceinline__ T adjoint_nodes(const T (&f)[Q][VEC], T (&mu)[Q][VEC], const T* __restrict__ lam_in,
                                           long long n0, int x0, int y, int z, const uint32_t (&lw)[VEC],
                                           const Geo& g, const Bc& bc, const T omega, double* __restrict__ grad_acc)
{
    using L = Lattice<Q>;
    const long long N = g.N;
    T dom = T(0);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const uint32_t w = lw[j];
        if (w & kLinkSolid) {
#pragma unroll
            for (int i = 0; i < Q; ++i) mu[i][j] = T(0);
            continue;
        }
        const long long n = n0 + j;
        const int x = x0 + j;
        const bool xin = x == 0, xout = x == g.nx - 1;
        T fl[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fl[i] = f[i][j];
        T drho, rho, u[3];
        moments<Q, T>(fl, drho, rho, u);
        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        T G[3] = {T(0), T(0), T(0)};
        double grw = 0.0;
        T m[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) m[i] = mu[i][j];
        if (w & ((1u << Q) - 1u)) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((w >> L::opp(i)) & 1u) m[i] = lam_in[(long long)L::opp(i) * N + n];
        }
        if (xin || xout) {
            const T rwT =
                T(xin ? (bc.profile ? bc.rho_in[(long long)z * g.ny + y] : bc.rho_in[0]) : bc.rho_out);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int o = L::opp(i), cx = L::c(i, 0);
                if (((w >> o) & 1u) == 0u && ((cx == -1 && xin) || (cx == 1 && xout))) {
                    const T li = lam_in[(long long)o * N + n];
                    m[i] = -li;
                    const T cu = cdot<Q, T>(o, u);
                    const T two_w = T(2.0 * L::w(o));
                    if (xin) grw += (double)(li * two_w * (T(1) + T(4.5) * cu * cu - T(1.5) * uu));
#pragma unroll
                    for (int a = 0; a < L::D; ++a)
                        G[a] += li * two_w * rwT * (T(9) * cu * T(L::c(o, a)) - T(3) * u[a]);
                }
            }
        }
        T A = 0, B[3] = {T(0), T(0), T(0)}, domT = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T cu = cdot<Q, T>(i, u);
            const T wi = T(L::w(i));
            const T P = T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
            const T feq = wi * (drho + rho * (P - T(1)));
            domT += m[i] * (feq - fl[i]);
            A += m[i] * wi * P;
#pragma unroll
            for (int a = 0; a < L::D; ++a)
                B[a] += m[i] * wi * rho * (T(3 * L::c(i, a)) + T(9) * cu * T(L::c(i, a)) - T(3) * u[a]);
        }
        const T inv = T(1) / rho;
        T Bt[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Bt[a] = (omega * B[a] + G[a]) * inv;
        const T base = omega * A, keep = T(1) - omega;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            T s = keep * m[k] + base;
#pragma unroll
            for (int a = 0; a < L::D; ++a) s += Bt[a] * (T(L::c(k, a)) - u[a]);
            mu[k][j] = s;  // mu now holds lambda^t
        }
        dom += domT;
        if (xin) grad_acc[(long long)z * g.ny + y] += grw;
    }
    return dom;
}

// adjoint_nodes with the node's own lambda^{t+1} already in registers
// (lam_own[k][j] = lambda^{t+1}_k at the lane's node j).
// The adjoint of one step at a lane's VEC nodes (the algebra of adjoint.cu):
// on entry f holds f^t (pulled and fixed up) and mu the values gathered from
// lambda^{t+1} at x + c_j; the bounce-back / Eq. 6 links are fixed up here
// from the node's own lambda^{t+1}, then mu is overwritten with lambda^t.
// Returns this lane's sum of dL/domega contributions; adds the inlet nodes'
// dL/drho_w to grad_acc (one owner per inlet node).
template <int Q, typename T, int VEC>
__device__ __forceinline__ T adjoint_nodes_own(const T (&f)[Q][VEC], T (&mu)[Q][VEC], const T (&lam_own)[Q][VEC],
                                           long long n0, int x0, int y, int z, const uint32_t (&lw)[VEC],
                                           const Geo& g, const Bc& bc, const T omega, double* __restrict__ grad_acc)
{
    using L = Lattice<Q>;
    T dom = T(0);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const uint32_t w = lw[j];
        if (w & kLinkSolid) {
#pragma unroll
            for (int i = 0; i < Q; ++i) mu[i][j] = T(0);
            continue;
        }
        const int x = x0 + j;
        const bool xin = x == 0, xout = x == g.nx - 1;
        T fl[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fl[i] = f[i][j];
        T drho, rho, u[3];
        moments<Q, T>(fl, drho, rho, u);
        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        T G[3] = {T(0), T(0), T(0)};
        double grw = 0.0;
        T m[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) m[i] = mu[i][j];
        if (w & ((1u << Q) - 1u)) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((w >> L::opp(i)) & 1u) m[i] = lam_own[L::opp(i)][j];
        }
        if (xin || xout) {
            const T rwT =
                T(xin ? (bc.profile ? bc.rho_in[(long long)z * g.ny + y] : bc.rho_in[0]) : bc.rho_out);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int o = L::opp(i), cx = L::c(i, 0);
                if (((w >> o) & 1u) == 0u && ((cx == -1 && xin) || (cx == 1 && xout))) {
                    const T li = lam_own[o][j];
                    m[i] = -li;
                    const T cu = cdot<Q, T>(o, u);
                    const T two_w = T(2.0 * L::w(o));
                    if (xin) grw += (double)(li * two_w * (T(1) + T(4.5) * cu * cu - T(1.5) * uu));
#pragma unroll
                    for (int a = 0; a < L::D; ++a)
                        G[a] += li * two_w * rwT * (T(9) * cu * T(L::c(o, a)) - T(3) * u[a]);
                }
            }
        }
        T A = 0, B[3] = {T(0), T(0), T(0)}, domT = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T cu = cdot<Q, T>(i, u);
            const T wi = T(L::w(i));
            const T P = T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
            const T feq = wi * (drho + rho * (P - T(1)));
            domT += m[i] * (feq - fl[i]);
            A += m[i] * wi * P;
#pragma unroll
            for (int a = 0; a < L::D; ++a)
                B[a] += m[i] * wi * rho * (T(3 * L::c(i, a)) + T(9) * cu * T(L::c(i, a)) - T(3) * u[a]);
        }
        const T inv = T(1) / rho;
        T Bt[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Bt[a] = (omega * B[a] + G[a]) * inv;
        const T base = omega * A, keep = T(1) - omega;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            T s = keep * m[k] + base;
#pragma unroll
            for (int a = 0; a < L::D; ++a) s += Bt[a] * (T(L::c(k, a)) - u[a]);
            mu[k][j] = s;  // mu now holds lambda^t
        }
        dom += domT;
        if (xin) grad_acc[(long long)z * g.ny + y] += grw;
    }
    return dom;
}

// The same boundary rules as pull_fixup, but with the node's own
// post-collision populations already in registers (own[k][j] = g_k at the
// lane's node j), so no load depends on the link words.
template <int Q, typename T, int VEC>
__device__ __forceinline__ void pull_fixup_own(T (&v)[Q][VEC], const T (&own)[Q][VEC], int x0, int y, int z,
                                               const uint32_t (&lw)[VEC], const Geo& g, const Bc& bc)
{
    using L = Lattice<Q>;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const uint32_t w = lw[j];
        if (w & kLinkSolid) continue;
        const int x = x0 + j;
        if (x == 0 || x == g.nx - 1) {
            const bool xin = x == 0;
            T loc[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) loc[i] = own[i][j];
            T drho, rho, u[3];
            moments<Q, T>(loc, drho, rho, u);
            const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const double rw = xin ? (bc.profile ? bc.rho_in[(long long)z * g.ny + y] : bc.rho_in[0]) : bc.rho_out;
            const T drw = T(rw - 1.0), rwT = T(rw);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = L::c(i, 0);
                if ((w >> i) & 1u) {
                    v[i][j] = loc[L::opp(i)];
                } else if ((cx == 1 && xin) || (cx == -1 && !xin)) {
                    const T cu = cdot<Q, T>(i, u);
                    v[i][j] = -loc[L::opp(i)] + T(2.0 * L::w(i)) * (drw + rwT * (T(4.5) * cu * cu - T(1.5) * uu));
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((w >> i) & 1u) v[i][j] = own[L::opp(i)][j];
        }
    }
}

template <int VEC>
__device__ __forceinline__ unsigned fluid_bits(const uint32_t (&lw)[VEC])
{
    unsigned fl = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j)
        if (!(lw[j] & kLinkSolid)) fl |= 1u << j;
    return fl;
}

template <int VEC>
__device__ __forceinline__ void load_links(uint32_t (&lw)[VEC], const uint32_t* __restrict__ link, long long n0,
                                           bool live)
{
    if (!live) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) lw[j] = kLinkSolid;
        return;
    }
    if constexpr (VEC == 4) {
        const uint4 t = *reinterpret_cast<const uint4*>(link + n0);
        lw[0] = t.x, lw[1] = t.y, lw[2] = t.z, lw[3] = t.w;
    } else {
        const uint2 t = *reinterpret_cast<const uint2*>(link + n0);
        lw[0] = t.x, lw[1] = t.y;
    }
}

// Loads the VEC values of row `rowp` that the lane's nodes x0 .. x0+VEC-1
// receive from columns x0 - SX .. x0 + VEC - 1 - SX (SX in {-1, 0, 1}).
// `live` is false for lanes past the end of the row (they still shuffle).
// Which of a lane's loads some fluid node needs.  `fl` has bit j set when
// the lane's node j is fluid; nodes of other lanes are seen through shuffles.
// A lane whose nodes are all solid, and whose edge element no neighbouring
// fluid node takes, skips its loads and its stores (solid nodes carry no
// populations), which removes most of the traffic of grain interiors.
template <int VEC>
struct Need {
    bool sx0, sxp, sxm;   // need the own vector for shift 0, +1 (from x - 1), -1 (from x + 1)
    bool edge_p, edge_m;  // lane 0 / lane 31 need the element beyond the warp's segment
};

template <int VEC>
__device__ __forceinline__ Need<VEC> lane_needs(unsigned fl, int lane)
{
    const unsigned first = fl & 1u, last = (fl >> (VEC - 1)) & 1u;
    const unsigned next_first = __shfl_down_sync(0xffffffffu, first, 1);
    const unsigned prev_last = __shfl_up_sync(0xffffffffu, last, 1);
    Need<VEC> n;
    n.sx0 = fl != 0u;
    n.sxp = (fl & ~1u) != 0u || (lane < 31 && next_first);
    n.sxm = (fl & ~(1u << (VEC - 1))) != 0u || (lane > 0 && prev_last);
    n.edge_p = lane == 0 && first;
    n.edge_m = lane == 31 && last;
    return n;
}

template <typename T, int VEC, int SX>
__device__ __forceinline__ void load_shifted(T (&o)[VEC], const T* __restrict__ rowp, int x0, int x0w, int nx,
                                             int lane, const Need<VEC>& need)
{
    T V[VEC];
    const bool ld = SX == 0 ? need.sx0 : (SX == 1 ? need.sxp : need.sxm);
    if (ld) {
        Vec<T, VEC>::load(rowp + x0, V);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) V[j] = T(0);
    }
    if (SX == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) o[j] = V[j];
    } else if (SX == 1) {  // from x - 1
        T prev = __shfl_up_sync(0xffffffffu, V[VEC - 1], 1);
        if (lane == 0) prev = (x0w > 0 && need.edge_p) ? rowp[x0w - 1] : T(0);
        o[0] = prev;
#pragma unroll
        for (int j = 1; j < VEC; ++j) o[j] = V[j - 1];
    } else {  // from x + 1
        T next = __shfl_down_sync(0xffffffffu, V[0], 1);
        if (lane == 31) next = (x0w + 32 * VEC < nx && need.edge_m) ? rowp[x0w + 32 * VEC] : T(0);
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) o[j] = V[j + 1];
        o[VEC - 1] = next;
    }
}

// load_shifted with the shift chosen at run time (folded after unrolling).
template <typename T, int VEC>
__device__ __forceinline__ void load_shift(T (&o)[VEC], int sx, const T* __restrict__ rowp, int x0, int x0w, int nx,
                                           int lane, const Need<VEC>& need)
{
    if (sx == 0) load_shifted<T, VEC, 0>(o, rowp, x0, x0w, nx, lane, need);
    else if (sx == 1) load_shifted<T, VEC, 1>(o, rowp, x0, x0w, nx, lane, need);
    else load_shifted<T, VEC, -1>(o, rowp, x0, x0w, nx, lane, need);
}

// What each of the lane's VEC nodes receives (the pull of step.cu, Eq. 3 and 6).
template <int Q, typename T, int VEC>
__device__ __forceinline__ void pull_vec(T (&v)[Q][VEC], const T* __restrict__ src, long long n0, int x0, int x0w,
                                         int y, int z, const uint32_t (&lw)[VEC], const Geo& g, const Bc& bc,
                                         int lane, bool live, const Need<VEC>& need)
{
    using L = Lattice<Q>;
    const long long N = g.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sy = y - L::c(i, 1), sz = z - L::c(i, 2);
        if (sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
            const T* rowp = src + (long long)i * N + ((long long)sz * g.ny + sy) * g.nx;
            load_shift<T, VEC>(v[i], L::c(i, 0), rowp, x0, x0w, g.nx, lane, need);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) v[i][j] = T(0);
        }
    }
    if (live) pull_fixup<Q, T, VEC>(v, src, n0, x0, y, z, lw, g, bc);
}

}  // namespace lbm
