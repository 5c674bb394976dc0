// Internal declarations shared by the library's translation units: the plan,
// the workspace layout, launch helpers and block-level FP64 reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/lbm.h"
#include "lattice.cuh"

namespace lbm {

constexpr int kStepThreads = 128;   // threads per block along x for the step kernels
constexpr int kReduceThreads = 1024;

enum StepMode : int { kStreamCollide = 0, kCollideOnly = 1, kStreamOnly = 2 };

// Workspace sections (byte offsets into the caller's d_ws, 256-byte aligned).
struct Workspace {
    size_t status;      // uint32 status word + FP64 scalars (count, weight)
    size_t grad_acc;    // double[n_acc]   per-inlet-node dL/drho_w accumulators
    size_t partial;     // double[n_blocks] per-block dL/domega accumulators
    size_t partial2;    // double[n_blocks] per-block loss / count partials
    size_t ping[2];     // forward ping-pong states
    size_t lam[2];      // adjoint ping-pong states
    size_t ckpt;        // (S - 1) checkpoint states, slot s (1..S-1) at index s - 1
    size_t seg;         // k segment states
    size_t total;
};

struct Geo {
    int nx, ny, nz;
    long long N;
    const uint32_t* link;
};

struct Bc {
    const double* rho_in;  // device: 1 or ny*nz entries
    int profile;           // 1: rho_in[z*ny + y], 0: rho_in[0]
    double rho_out;
};

// Everything a launch needs to know about the lattice and its precision.
struct PlanInfo {
    int q, d, prec;
    Geo geo;
    dim3 grid;        // step grid: (ceil(nx/kStepThreads), ny, nz)
    int n_blocks;     // grid.x * grid.y * grid.z
    int n_in;         // inlet entries (1 or ny*nz)
    int n_acc;        // per-inlet-node accumulators (always ny*nz)
    size_t state_bytes;
};

// Slots of the FP64 scalars inside the status section.
constexpr size_t kScalarCount = 8;    // double: ROI fluid-node count
constexpr size_t kScalarWeight = 16;  // double: loss weight
constexpr size_t kScalarTmp = 24;     // double: scratch

// --------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block with a linear thread index tid in [0, nthreads); result
// valid in tid 0.  All threads of the block must call it.  Fixed order.
__device__ __forceinline__ double block_sum(double v, int tid, int nthreads)
{
    __shared__ double s[32];
    v = warp_sum(v);
    if ((tid & 31) == 0) s[tid >> 5] = v;
    __syncthreads();
    int nw = (nthreads + 31) >> 5;
    v = tid < nw ? s[tid] : 0.0;
    if (tid < 32) v = warp_sum(v);
    __syncthreads();
    return v;
}

// ------------------------------------------------------------ launchers

lbm_status step_launch(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                       cudaStream_t s);
lbm_status adjoint_launch(const PlanInfo& p, int t_is_zero, const void* gprev, const void* lam_in, void* lam_out,
                          const Bc& bc, const double* tau, double* grad_acc, double* partial, cudaStream_t s);
lbm_status loss_launch(const PlanInfo& p, const void* f, const double* u_target, const uint8_t* roi, int kind,
                       int norm, double* d_loss, void* lambda, unsigned char* ws, const Workspace& w,
                       cudaStream_t s);
lbm_status loss_launch_noalloc(const PlanInfo& p, const void* f, const double* u_target, const uint8_t* roi, int kind,
                               int norm, double* d_loss, void* lambda, cudaStream_t s);
lbm_status finish_gradients_launch(const PlanInfo& p, const double* grad_acc, const double* partial,
                                   const double* tau, double* d_grad_rho_in, double* d_grad_tau,
                                   uint32_t* status, cudaStream_t s);
lbm_status macroscopic_launch(const PlanInfo& p, const void* f, double* rho, double* u, cudaStream_t s);
lbm_status darcy_launch(const PlanInfo& p, const void* f, const double* rho_in, int n_in, const double* tau,
                        double rho_out, int xs, double* k, double* flux, cudaStream_t s);
lbm_status adam_launch(int n, double* theta, double* m, double* v, const double* grad_p, double* p, double off,
                       double scale, int t, double lr, double b1, double b2, double eps, cudaStream_t s);
lbm_status geometry_launch(const PlanInfo& p, const lbm_geom_desc& g, uint8_t* mask, uint32_t* link,
                           double* porosity, int64_t* info, cudaStream_t s);

inline lbm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

}  // namespace lbm
