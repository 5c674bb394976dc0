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
