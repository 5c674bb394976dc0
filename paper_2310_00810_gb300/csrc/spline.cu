// Cubic-spline inlet profiles (arXiv 2310.00810, section 3.1.2: the
// multi-parameter inversion imposes the inlet pressure as a cubic spline
// through a few inlet densities).  Knot values c[Kz][Ky] map linearly to the
// inlet density,
//     rho_in[z ny + y] = rho_out + sum_{b,a} Bz[z][b] By[y][a] c[b][a],
// with By (Bz) the natural cubic spline basis over the rows (layers): column a
// holds the spline through the a-th unit knot vector, knots evenly spaced at
// t_a = a (n - 1) / (K - 1), zero second derivative at both ends (K = 1: a
// constant).  The basis is built on the host (one tridiagonal solve per
// column); the profile and the gradient dL/dc = Bz^T G By, G = dL/drho_in
// as [nz][ny], are small device kernels.
#include <vector>

#include "common.cuh"

namespace lbm {

// Natural cubic spline through (t_j, v_j), t_j = j h, evaluated at x = 0..n-1.
static void spline_column(int K, int n, int a, double* out, int stride)
{
    if (K == 1) {
        for (int x = 0; x < n; ++x) out[(size_t)x * stride] = 1.0;
        return;
    }
    const double h = (double)(n - 1) / (double)(K - 1);
    std::vector<double> v(K, 0.0), M(K, 0.0);
    v[a] = 1.0;
    if (K > 2) {
        // interior equations j = 1..K-2: h M_{j-1} + 4 h M_j + h M_{j+1} = 6 (v_{j+1} - 2 v_j + v_{j-1}) / h,
        // solved by forward elimination and back substitution (diagonally dominant)
        const int m = K - 2;
        std::vector<double> diag(m, 4.0 * h), rhs(m), cp(m);
        for (int j = 0; j < m; ++j) rhs[j] = 6.0 * (v[j + 2] - 2.0 * v[j + 1] + v[j]) / h;
        cp[0] = h / diag[0];
        rhs[0] = rhs[0] / diag[0];
        for (int j = 1; j < m; ++j) {
            const double den = diag[j] - h * cp[j - 1];
            cp[j] = h / den;
            rhs[j] = (rhs[j] - h * rhs[j - 1]) / den;
        }
        M[m] = rhs[m - 1];
        for (int j = m - 2; j >= 0; --j) M[j + 1] = rhs[j] - cp[j] * M[j + 2];
    }
    for (int x = 0; x < n; ++x) {
        int k = (int)((double)x / h);
        if (k > K - 2) k = K - 2;
        const double tl = k * h, tr = (k + 1) * h;
        const double p = tr - x, q = x - tl;
        out[(size_t)x * stride] = M[k] * p * p * p / (6.0 * h) + M[k + 1] * q * q * q / (6.0 * h) +
                                  (v[k] / h - M[k] * h / 6.0) * p + (v[k + 1] / h - M[k + 1] * h / 6.0) * q;
    }
}

void spline_basis_host(int K, int n, double* basis)
{
    for (int a = 0; a < K; ++a) spline_column(K, n, a, basis + a, K);
}

__global__ void __launch_bounds__(256) k_spline_profile(int ky, int kz, int ny, int nz, const double* __restrict__ by,
                                                       const double* __restrict__ bz, const double* __restrict__ c,
                                                       double rho_out, double* __restrict__ rho_in)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ny * nz) return;
    const int y = i % ny, z = i / ny;
    double s = 0.0;
    for (int b = 0; b < kz; ++b) {
        double r = 0.0;
        for (int a = 0; a < ky; ++a) r += by[(size_t)y * ky + a] * c[(size_t)b * ky + a];
        s += bz[(size_t)z * kz + b] * r;
    }
    rho_in[i] = rho_out + s;
}

// One block per knot (b, a): dL/dc[b][a] = sum_{z,y} Bz[z][b] By[y][a] G[z][y], in a fixed order.
__global__ void __launch_bounds__(256) k_spline_grad(int ky, int kz, int ny, int nz, const double* __restrict__ by,
                                                    const double* __restrict__ bz, const double* __restrict__ g,
                                                    double* __restrict__ gc)
{
    const int a = blockIdx.x % ky, b = blockIdx.x / ky;
    double s = 0.0;
    for (int i = threadIdx.x; i < ny * nz; i += blockDim.x) {
        const int y = i % ny, z = i / ny;
        s += bz[(size_t)z * kz + b] * by[(size_t)y * ky + a] * g[i];
    }
    const double t = block_sum(s, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) gc[blockIdx.x] = t;
}

lbm_status spline_profile_launch(const PlanInfo& p, int ky, int kz, const double* by, const double* bz,
                                 const double* c, double rho_out, double* rho_in, cudaStream_t s)
{
    const int n = p.geo.ny * p.geo.nz;
    k_spline_profile<<<(n + 255) / 256, 256, 0, s>>>(ky, kz, p.geo.ny, p.geo.nz, by, bz, c, rho_out, rho_in);
    return cuda_status(cudaGetLastError());
}

lbm_status spline_grad_launch(const PlanInfo& p, int ky, int kz, const double* by, const double* bz,
                              const double* g, double* gc, cudaStream_t s)
{
    k_spline_grad<<<ky * kz, 256, 0, s>>>(ky, kz, p.geo.ny, p.geo.nz, by, bz, g, gc);
    return cuda_status(cudaGetLastError());
}

}  // namespace lbm
