// Device helpers shared by the forward and adjoint kernels: moments of
// shifted populations (Eq. 1-2), BGK collision (Eq. 4-5) and the pull with
// halfway bounce-back and anti-bounce-back (Eq. 3, Eq. 6).
#pragma once

#include "common.cuh"

namespace lbm {

template <int Q>
__host__ __device__ constexpr long long link_offset(int i, int nx, long long plane)
{
    return (long long)Lattice<Q>::c(i, 0) + (long long)Lattice<Q>::c(i, 1) * nx +
           (long long)Lattice<Q>::c(i, 2) * plane;
}

// Moments of shifted populations: rho = 1 + sum v, rho u = sum c v.
template <int Q, typename T>
__device__ __forceinline__ void moments(const T (&v)[Q], T& drho, T& rho, T (&u)[3])
{
    using L = Lattice<Q>;
    T s = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s += v[i];
#pragma unroll
        for (int a = 0; a < L::D; ++a)
            if (L::c(i, a) != 0) j[a] += L::c(i, a) > 0 ? v[i] : -v[i];
    }
    drho = s;
    rho = T(1) + s;
    T inv = T(1) / rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = a < L::D ? j[a] * inv : T(0);
}

template <int Q, typename T>
__device__ __forceinline__ T cdot(int i, const T (&u)[3])
{
    using L = Lattice<Q>;
    T s = 0;
#pragma unroll
    for (int a = 0; a < L::D; ++a)
        if (L::c(i, a) != 0) s += L::c(i, a) > 0 ? u[a] : -u[a];
    return s;
}

// BGK collision (Eq. 4-5) in place on shifted populations.
template <int Q, typename T>
__device__ __forceinline__ void collide(T (&v)[Q], T omega)
{
    using L = Lattice<Q>;
    T drho, rho, u[3];
    moments<Q, T>(v, drho, rho, u);
    T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T cu = cdot<Q, T>(i, u);
        T feq = T(L::w(i)) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
        v[i] = v[i] - omega * (v[i] - feq);
    }
}

// ------------------------------------------------------------- MRT (D2Q9)
// The moment matrix of the MRT operator (section 3.4, Eq. 18) in this
// lattice's direction order; rows rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx,
// p_xy (the printed p_xy row |c_x c_y| read as the orthogonal c_x c_y), and
// 1 / |row|^2 (the rows are orthogonal: M^{-1} = M^T diag(1 / |row|^2)).
__host__ __device__ constexpr int mrt_m(int r, int j)
{
    constexpr int t[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                             {4, -2, -2, -2, -2, 1, 1, 1, 1},  {0, 1, 0, -1, 0, 1, -1, -1, 1},
                             {0, -2, 0, 2, 0, 1, -1, -1, 1},   {0, 0, 1, 0, -1, 1, 1, -1, -1},
                             {0, 0, -2, 0, 2, 1, 1, -1, -1},   {0, 1, -1, 1, -1, 0, 0, 0, 0},
                             {0, 0, 0, 0, 0, 1, -1, 1, -1}};
    return t[r][j];
}

__host__ __device__ constexpr double mrt_inv_norm2(int r)
{
    constexpr double t[9] = {1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 6, 1.0 / 12, 1.0 / 6, 1.0 / 12, 1.0 / 4, 1.0 / 4};
    return t[r];
}

// Relaxation rate of moment row r: 0 for the conserved rho, j_x, j_y (their
// m - m^eq vanishes), s_e, s_eps, s_q for the free rows, omega = 1/tau for the
// stress rows p_xx, p_xy.
template <typename T>
__device__ __forceinline__ T mrt_rate(int r, T omega, const T (&s)[3])
{
    return r == 1 ? s[0] : r == 2 ? s[1] : (r == 4 || r == 6) ? s[2] : (r >= 7 ? omega : T(0));
}

// MRT collision (Eq. 16) in place on shifted populations:
// f* = f - M^{-1} S M (f - f^eq), m^eq = M f^eq with f^eq of Eq. 5.
template <typename T>
__device__ __forceinline__ void collide_mrt(T (&v)[9], T omega, const double* __restrict__ rates)
{
    using L = Lattice<9>;
    const T s[3] = {T(rates[0]), T(rates[1]), T(rates[2])};
    T drho, rho, u[3];
    moments<9, T>(v, drho, rho, u);
    const T uu = u[0] * u[0] + u[1] * u[1];
    T d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T cu = cdot<9, T>(i, u);
        d[i] = v[i] - T(L::w(i)) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
    }
    T dm[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        T m = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j)
            if (mrt_m(r, j) != 0) m += T(mrt_m(r, j)) * d[j];
        dm[r] = mrt_rate<T>(r, omega, s) * m * T(mrt_inv_norm2(r));
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        T c = 0;
#pragma unroll
        for (int r = 0; r < 9; ++r)
            if (mrt_m(r, j) != 0 && r != 0 && r != 3 && r != 5) c += T(mrt_m(r, j)) * dm[r];
        v[j] -= c;
    }
}

// BGK (Eq. 4-5) or, on D2Q9 plans with Bc::mrt, MRT.
template <int Q, typename T>
__device__ __forceinline__ void collide_any(T (&v)[Q], T omega, const Bc& bc)
{
    if constexpr (Q == 9) {
        if (bc.mrt) {
            collide_mrt<T>(v, omega, mrt_rates(bc.status));
            return;
        }
    }
    collide<Q, T>(v, omega);
}

// Transpose of the MRT collision at one node, from f^t (moments drho, rho, u)
// and mu = dL/df*: with nu = M^T S diag(1/|row|^2) M mu (nu = omega mu for
// BGK), lambda_k = mu_k - nu_k + A + sum_a (B_a + G_a) (c_ka - u_a) / rho,
// A = sum_j nu_j w_j P_j, B_a = sum_j nu_j w_j rho (3 c_ja + 9 (c_j.u) c_ja - 3 u_a),
// G the Eq. 6 velocity terms.  Returns the node's dL/domega term: only the
// stress rows depend on omega, -sum_{p_xx, p_xy} (M mu)_r (M (f - f^eq))_r / |row_r|^2.
template <typename T>
__device__ __forceinline__ T adjoint_collision_mrt(const T (&f)[9], const T (&mu)[9], T drho, T rho,
                                                   const T (&u)[3], const T (&G)[3], T omega,
                                                   const double* __restrict__ rates, T (&lam)[9])
{
    using L = Lattice<9>;
    const T s[3] = {T(rates[0]), T(rates[1]), T(rates[2])};
    const T uu = u[0] * u[0] + u[1] * u[1];
    T d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T cu = cdot<9, T>(i, u);
        d[i] = f[i] - T(L::w(i)) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
    }
    T sm[9], dom = T(0);
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        T mm = 0, md = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j)
            if (mrt_m(r, j) != 0) {
                mm += T(mrt_m(r, j)) * mu[j];
                md += T(mrt_m(r, j)) * d[j];
            }
        if (r >= 7) dom -= mm * md * T(mrt_inv_norm2(r));
        sm[r] = mrt_rate<T>(r, omega, s) * mm * T(mrt_inv_norm2(r));
    }
    T nu[9], A = 0, B[2] = {T(0), T(0)};
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        T c = 0;
#pragma unroll
        for (int r = 0; r < 9; ++r)
            if (mrt_m(r, j) != 0 && r != 0 && r != 3 && r != 5) c += T(mrt_m(r, j)) * sm[r];
        nu[j] = c;
        const T cu = cdot<9, T>(j, u);
        const T wj = T(L::w(j));
        A += c * wj * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
#pragma unroll
        for (int a = 0; a < 2; ++a)
            B[a] += c * wj * rho * (T(3 * L::c(j, a)) + T(9) * cu * T(L::c(j, a)) - T(3) * u[a]);
    }
    const T inv = T(1) / rho;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        T sk = mu[k] - nu[k] + A;
#pragma unroll
        for (int a = 0; a < 2; ++a) sk += (B[a] + G[a]) * inv * (T(L::c(k, a)) - u[a]);
        lam[k] = sk;
    }
    return dom;
}

// Eq. 6 with the wall velocity extrapolated to the pressure plane half a
// link outside the boundary node (Bc::uw_extrap): u_w = u(x_b) + (u(x_b) -
// u(x_b + e)) / 2, with x_b + e the inward neighbour, whose velocity comes from
// its post-collision populations (collision keeps u).  `nb` indexes the
// neighbour in a state of `stride` nodes per direction.
template <int Q, typename T>
__device__ __forceinline__ void extrapolate_wall_velocity(T (&u)[3], const T* __restrict__ src, long long stride,
                                                          long long nb)
{
    T v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = src[(long long)i * stride + nb];
    T drho, rho, ue[3];
    moments<Q, T>(v, drho, rho, ue);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = T(1.5) * u[a] - T(0.5) * ue[a];
}

// The direction whose link starts at the inward neighbour of a boundary node:
// c = (-1, 0, 0) at the inlet (x - c = x + 1), (+1, 0, 0) at the outlet.
template <int Q>
__host__ __device__ constexpr int inward_dir(bool xin)
{
    return xin ? Lattice<Q>::opp(1) : 1;
}

// Reverse of the extrapolated u_w at one boundary node x_b with inward
// neighbour x_e.  The adjoint kernels take u_w as the node's own velocity u;
// this returns what the extrapolation changes: the velocity terms of x_b
// become 1.5 G(u_w) instead of G(u), x_e gains -0.5 G(u_w), and the inlet
// gradient changes by the difference of d(Eq. 6)/drho_w.  With
// G_a(v) = sum over the node's Eq. 6 links i of lambda_i 2 w_i rho_w (9 (c_i.v) c_ia - 3 v_a),
// the deltas are  d_b[k] = sum_a (1.5 G_a(u_w) - G_a(u)) (c_ka - u_a) / rho(x_b)
// and d_e[k] = sum_a (-0.5 G_a(u_w)) (c_ka - u_e,a) / rho(x_e).
// fb, fe: f^t at x_b and x_e; li[i]: lambda^{t+1}_i(x_b) for the Eq. 6 links
// (bit i of eq6); returns the change of dL/drho_w.
template <int Q, typename T>
__device__ __forceinline__ double adjoint_uw_delta(const T (&fb)[Q], const T (&fe)[Q], const T (&li)[Q],
                                                   uint32_t eq6, T rw, T (&db)[Q], T (&de)[Q])
{
    using L = Lattice<Q>;
    T drb, rhob, ub[3], dre, rhoe, ue[3];
    moments<Q, T>(fb, drb, rhob, ub);
    moments<Q, T>(fe, dre, rhoe, ue);
    T uw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) uw[a] = T(1.5) * ub[a] - T(0.5) * ue[a];
    const T uub = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
    const T uuw = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
    T Gw[3] = {T(0), T(0), T(0)}, Gu[3] = {T(0), T(0), T(0)};
    double dgrw = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (!((eq6 >> i) & 1u)) continue;
        const T two_w = T(2.0 * L::w(i));
        const T cw = cdot<Q, T>(i, uw), cb = cdot<Q, T>(i, ub);
        dgrw += (double)(li[i] * two_w * (T(4.5) * (cw * cw - cb * cb) - T(1.5) * (uuw - uub)));
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            Gw[a] += li[i] * two_w * rw * (T(9) * cw * T(L::c(i, a)) - T(3) * uw[a]);
            Gu[a] += li[i] * two_w * rw * (T(9) * cb * T(L::c(i, a)) - T(3) * ub[a]);
        }
    }
    const T invb = T(1) / rhob, inve = T(1) / rhoe;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        T sb = 0, se = 0;
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            sb += (T(1.5) * Gw[a] - Gu[a]) * (T(L::c(k, a)) - ub[a]);
            se += T(-0.5) * Gw[a] * (T(L::c(k, a)) - ue[a]);
        }
        db[k] = sb * invb;
        de[k] = se * inve;
    }
    return dgrw;
}

// Pull with boundaries: fills v with what node n (at x, y, z) receives.
template <int Q, typename T>
__device__ __forceinline__ void pull(T (&v)[Q], const T* __restrict__ src, long long n, int x, int y, int z,
                                     uint32_t lw, const Geo& g, const Bc& bc)
{
    using L = Lattice<Q>;
    const long long N = g.N, plane = (long long)g.nx * g.ny;
    const bool xin = x == 0, xout = x == g.nx - 1;
    if (xin || xout) {
        // the node's own velocity u(x, t) for Eq. 6, from its local state
        T loc[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) loc[i] = src[(long long)i * N + n];
        T drho, rho, u[3];
        moments<Q, T>(loc, drho, rho, u);
        if (bc.uw_extrap && !((lw >> inward_dir<Q>(xin)) & 1u))
            extrapolate_wall_velocity<Q, T>(u, src, N, xin ? n + 1 : n - 1);
        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double rw = xin ? (bc.profile ? bc.rho_in[(long long)z * g.ny + y] : bc.rho_in[0]) : bc.rho_out;
        const T drw = T(rw - 1.0), rwT = T(rw);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::c(i, 0);
            if ((lw >> i) & 1u) {
                v[i] = loc[L::opp(i)];
            } else if ((cx == 1 && xin) || (cx == -1 && xout)) {
                const T cu = cdot<Q, T>(i, u);
                v[i] = -loc[L::opp(i)] + T(2.0 * L::w(i)) * (drw + rwT * (T(4.5) * cu * cu - T(1.5) * uu));
            } else {
                v[i] = src[(long long)i * N + n - link_offset<Q>(i, g.nx, plane)];
            }
        }
    } else {
        // the address is selected, then loaded unconditionally: the Q loads
        // then issue together instead of one branch (and one wait) at a time
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = (lw >> i) & 1u;
            const long long a = bb ? (long long)L::opp(i) * N + n : (long long)i * N + n - link_offset<Q>(i, g.nx, plane);
            v[i] = src[a];
        }
    }
}

}  // namespace lbm
