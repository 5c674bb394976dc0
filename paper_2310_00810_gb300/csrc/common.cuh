// Internal declarations shared by the library's translation units: the plan,
// the workspace layout, launch helpers and block-level FP64 reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/lbm.h"
#include "lattice.cuh"

namespace lbm {

constexpr int kStepThreads = 128;   // threads per block along x for the scalar step kernels
constexpr int kVecRows = 4;         // rows per block (one warp per row) for the vectorised kernels
constexpr int kReduceThreads = 1024;

enum StepMode : int { kStreamCollide = 0, kCollideOnly = 1, kStreamOnly = 2 };

// Workspace sections (byte offsets into the caller's d_ws, 256-byte aligned).
struct Workspace {
    size_t status;      // uint32 status word + FP64 scalars (count, weight)
    size_t call;        // double[n_in + 1]: this call's rho_in and tau, copied from the caller's arrays
    size_t grad_acc;    // double[n_acc]   per-inlet-node dL/drho_w accumulators
    size_t partial;     // double[n_blocks] per-block dL/domega accumulators
    size_t partial2;    // double[n_blocks] per-block loss / count partials
    size_t side;        // in-place schedule: velocity of each Eq. 6 node's last output (2 ny nz x 3, plan precision)
    size_t ping[2];     // forward ping-pong states (the in-place schedule uses ping[0] only)
    size_t lam[2];      // adjoint ping-pong states (the in-place schedule uses lam[1] only)
    size_t ckpt;        // (S - 1) checkpoint states, slot s (1..S-1) at index s - 1
    size_t seg;         // two buffers of k segment states
    size_t total;
};

struct Geo {
    int nx, ny, nz;
    long long N;
    const uint32_t* link;
    int skip_sectors;  // 1: kernels may skip stores of 32-byte sectors holding only solid nodes (nx % 8 == 0)
    int periodic_y = 0;  // 1: links leaving the y range re-enter on the other side (fluid-only layout only)
};

struct Bc {
    const double* rho_in;  // device: 1 or ny*nz entries
    short profile;         // 1: rho_in[z*ny + y], 0: rho_in[0]
    char uw_extrap = 0;    // 1: Eq. 6 takes u_w extrapolated to the pressure plane (LBM_ABB_U_EXTRAP)
    char mrt = 0;          // 1: D2Q9 MRT collision (Eq. 16-18); its free rates are in the status section
    char vel_inlet = 0;    // 1: velocity inlet through x = -1/2 (moving-wall bounce-back); u_in in the status section
    double rho_out;
    uint32_t* status;      // device status word (bounded waits latch LBM_ERR_TIMEOUT here)
    uint32_t wait_us = 2000000u;  // time bound of each mbarrier wait of the TMA kernels, in microseconds
    char test_stall = 0;   // 1: TMA producers issue no copies, so every consumer wait runs out (tests only)
    int t_level = 0;       // the time level this launch's streaming produces (f^t_level)
    int ramp_steps = 0;    // the velocity inlet starts gradually: u_in r(t_level), r = 1 from ramp_steps on
    void* side_u = nullptr;  // in-place forward steps: the Eq. 6 nodes' velocities (read, then rewritten)
};

// The gradual start of the velocity inlet: r(t) = sin^2(pi t / (2 R)) for
// 0 < t < R, 0 at t <= 0 and 1 from R on (R <= 0: no ramp).
__device__ __forceinline__ double inlet_ramp(const Bc& bc)
{
    if (bc.ramp_steps <= 0 || bc.t_level >= bc.ramp_steps) return 1.0;
    if (bc.t_level <= 0) return 0.0;
    const double s = sin(3.14159265358979323846 * (double)bc.t_level / (2.0 * (double)bc.ramp_steps));
    return s * s;
}

// The boundary data of a launch whose streaming produces time level t.
inline Bc at_time(const Bc& bc, int t)
{
    Bc b = bc;
    b.t_level = t;
    return b;
}

// Fluid-only ("compact") layout tables (compact.cu).  nf = 0: dense layout.
constexpr int32_t kCmpBB = -1;   // neighbour code: halfway bounce-back link
constexpr int32_t kCmpABB = -2;  // neighbour code: Eq. 6 link through x = -1/2 or nx - 1/2
struct Cmp {
    long long nf;          // fluid nodes stored
    const int32_t* idx;    // idx[k]: dense node index of compact node k (interior nodes, then x = 0 / nx - 1)
    const int32_t* nbr;    // nbr[(i - 1) * nf + k], i = 1..Q-1: compact index of x - c_i, or kCmpBB / kCmpABB
    const uint32_t* eq6;   // bit k & 31 of eq6[k >> 5]: node k has an Eq. 6 / velocity-inlet link
};

struct BCmpInst;

// Everything a launch needs to know about the lattice and its precision.
struct PlanInfo {
    int q, d, prec;
    Geo geo;
    dim3 grid;        // step grid: (ceil(nx/kStepThreads), ny, nz)
    int n_blocks;     // grid.x * grid.y * grid.z
    int n_in;         // inlet entries (1 or ny*nz)
    int n_acc;        // per-inlet-node accumulators (always ny*nz)
    int n_partial;    // per-block FP64 partial slots (covers every step-kernel grid)
    int max_vec;      // widest nodes-per-thread of the step/adjoint kernels (0/1: scalar kernels only)
    int use_tma;      // 1: TMA-staged FP32 step/adjoint kernels where alignment allows
    int step_variant; // register stream-collide kernel: 0 link-dependent loads, 1 all loads up front
    int tma_variant;  // D2Q9 TMA stream-collide: 0 per-direction shifted boxes, 1 halo boxes + TMA link words
    int tma_ty;       // D2Q9 halo TMA tile height of the stream-collide kernels: 8 or 4 rows
    int tma_waves;    // D2Q9 halo TMA: one-stage kernels (one tile per CTA) up to tma_waves x SMs tiles
    int adj_tma_ty;   // the same for the adjoint kernels
    int step_family;  // LBM_FAMILY_* of the stream-collide kernels
    int adj_family;   // LBM_FAMILY_* of the adjoint kernels
    int rec_family;   // LBM_FAMILY_* of the reverse sweep's segment recompute (AUTO: as step_family)
    int pdl;          // 1: launch the sweep kernels with programmatic dependent launch
    int steps2;       // 1: two stream-collide steps per launch where the two-step kernel applies
    int use_persist;  // 1: one cooperative launch per sweep for lattices of at most persist_max_bytes
    int overlap;      // 1: reverse sweep recomputes the next segment on a second stream during the adjoint steps
    int aa;           // 1: in-place (AA-pattern) streaming in the fluid-only layout
    int uw_extrap;    // 1: Eq. 6 with the extrapolated wall velocity (one-node-per-thread or fluid-only kernels)
    int mrt;          // 1: D2Q9 MRT collision (one-node-per-thread or fluid-only kernels)
    int vel_inlet;    // 1: velocity inlet instead of Eq. 6 at x = -1/2 (fluid-only kernels)
    double u_in[3];   // its velocity
    int ramp_steps;   // its gradual start (0: none)
    double mrt_rates[3];  // s_e, s_eps, s_q of the MRT collision
    unsigned spin_limit;  // grid-barrier spin limit of the persistent sweeps
    unsigned wait_us;     // time bound of each mbarrier wait of the TMA kernels (microseconds)
    int test_stall;       // LBM_TEST_STALL_TMA=1: the TMA producers issue nothing (failure-path tests)
    size_t persist_max_bytes;
    int tma_min_tiles;  // smallest tile count for which the TMA kernels are used
    size_t state_bytes;   // bytes of one internal state (Q N, or Q nf in the compact layout)
    Cmp cmp;
    const int32_t* cmp_map;  // cmap[n]: compact index of dense node n, or -1 for a solid node (compact layout)
    const BCmpInst* cmp_inst;  // the lattice as a one-instance pack (compact layout; device)
};

// Grid barrier words of the persistent sweeps (in the status section).
struct PersistBar {
    unsigned count;
    unsigned gen;
    int abort;
    int pad;
};

// Buffers and schedule of a persistent sweep (see persist.cu).
struct PersistArgs {
    unsigned char* ping[2];  // forward ping-pong states
    unsigned char* ckpt;     // checkpoint slot s (1..S-1) at (s - 1) * state_stride
    unsigned char* seg;      // segment state j at j * state_stride
    unsigned char* lam[2];   // adjoint ping-pong states
    const void* lam_in;      // lambda^T (reverse sweep input)
    void* out;               // f^T (forward sweep output)
    size_t state_stride;
    int T, k, S;
    unsigned spin_limit;     // grid-barrier spins before a CTA gives up (LBM_ERR_TIMEOUT)
    PersistBar* bar;
};
constexpr size_t kBarOffset = 64;  // byte offset of the PersistBar in the status section

// Slots of the FP64 scalars inside the status section.
constexpr size_t kScalarCount = 8;    // double: ROI fluid-node count
constexpr size_t kScalarWeight = 16;  // double: loss weight
constexpr size_t kScalarTmp = 24;     // double: scratch
constexpr size_t kMrtRates = 128;     // double[3]: s_e, s_eps, s_q of the MRT collision (written per call)
constexpr size_t kInletVelocity = 160;  // double[3]: the velocity inlet's u_in (written per call)

// The velocity inlet's u_in a kernel reads (Bc::vel_inlet).
__device__ __forceinline__ const double* inlet_velocity(const uint32_t* status)
{
    return reinterpret_cast<const double*>(reinterpret_cast<const unsigned char*>(status) + kInletVelocity);
}

// The MRT rates a kernel reads (Bc::mrt): s_e, s_eps, s_q.
__device__ __forceinline__ const double* mrt_rates(const uint32_t* status)
{
    return reinterpret_cast<const double*>(reinterpret_cast<const unsigned char*>(status) + kMrtRates);
}

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

// ------------------------------------------- programmatic dependent launch

// The sweep kernels are launched with programmatic stream serialization: the
// next kernel of the stream may be scheduled while this one is still running,
// and each kernel first waits (griddepcontrol.wait) until its predecessor has
// completed and its writes are visible.  Launched without the attribute,
// both instructions are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class K, class... Args>
inline void launch_k(bool pdl, K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------ launchers

lbm_status step_launch(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                       cudaStream_t s);
bool step_launch_vec(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                     cudaStream_t s);
bool adjoint_launch_vec(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                        const double* tau, double* grad_acc, double* partial, cudaStream_t s);
int vec_blocks_max(const PlanInfo& p);
bool step_launch_tma(const PlanInfo& p, int mode, const void* src, void* dst, const Bc& bc, const double* tau,
                     cudaStream_t s);
bool step2_launch_tma(const PlanInfo& p, const void* src, void* dst, void* mid, const Bc& bc, const double* tau,
                      cudaStream_t s);
bool step2_possible(const PlanInfo& p, const Bc& bc);
lbm_status step2_launch(const PlanInfo& p, const void* src, void* mid, void* dst, const Bc& bc, const double* tau,
                        cudaStream_t s);
bool adjoint_launch_tma(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out, const Bc& bc,
                        const double* tau, double* grad_acc, double* partial, cudaStream_t s);
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

// The plan as seen by a launcher of the given kernel family.
inline PlanInfo with_family(const PlanInfo& p, int family)
{
    PlanInfo q = p;
    if (family == LBM_FAMILY_SCALAR) {
        q.max_vec = 0;
        q.use_tma = 0;
    } else if (family == LBM_FAMILY_VEC) {
        q.use_tma = 0;
        if (q.max_vec < 2) q.max_vec = 4;
    } else if (family == LBM_FAMILY_TMA) {
        q.use_tma = 1;
        q.tma_min_tiles = 1;
        if (q.max_vec < 2) q.max_vec = 4;
    }
    return q;
}

size_t compact_table_bytes(const PlanInfo& p, long long nf);

// Batches in the fluid-only layout: the fluid nodes of every instance packed
// into one compact state [Q][nfp], instance i at compact indices
// [k0, k0 + nf), k0 a multiple of kBatchCmpAlign, so that every thread block
// of the compact kernels belongs to one instance (blk_inst[block]).
constexpr int kBatchCmpAlign = 256;
struct BCmpInst {
    Geo g;              // the instance's sizes (the compact kernels use no link words)
    long long k0, nf;   // first compact index and fluid nodes
    long long f_off;    // its dense [Q][N] arrays in a packed dense state (elements)
    long long in_off;   // inlet densities and their gradients
    long long acc_off;  // per-inlet-node accumulators (ny * nz)
    int n_in, pad;
};
struct BCmpArgs {
    Cmp c;                   // c.nf = nfp (the packed stride), c.idx local dense indices, c.nbr packed codes
    const BCmpInst* insts;   // device
    const int* blk_inst;     // device: instance of each kBatchCmpAlign-node block
    unsigned n_blocks;       // nfp / kBatchCmpAlign
    int q, prec, pdl;
    uint32_t* status;
};
lbm_status bstep_launch_cmp(const BCmpArgs& a, int mode, const void* src, void* dst, bool dense_out,
                            const double* rho_in, const double* tau, double rho_out, cudaStream_t s);
lbm_status badjoint_launch_cmp(const BCmpArgs& a, int t0, const void* gprev, const void* lam_in, void* lam_out,
                               const double* rho_in, const double* tau, double rho_out, double* grad_acc,
                               double* partial, cudaStream_t s);
lbm_status bgather_launch_cmp(const BCmpArgs& a, const void* dense, void* compact, cudaStream_t s);
lbm_status bpack_launch_cmp(const Cmp& local, int q, long long k0, long long nfp, int32_t* idx, int32_t* nbr,
                            cudaStream_t s);
// the per-node Eq. 6 bit array of a (packed) table: bit k & 31 of bits[k >> 5]
lbm_status eq6_bits_launch_cmp(int q, const int32_t* nbr, long long nf, uint32_t* bits, cudaStream_t s);
lbm_status compact_build(const PlanInfo& p, long long nf, void* tables, Cmp* out, const int32_t** cmap_out,
                         const BCmpInst** inst_out, cudaStream_t s);
// Layouts of a fluid-only state (compact.cu): natural, or swapped (the
// in-place schedule's layout of g^t and lambda^t at odd t).
constexpr int kLayoutNatural = 0;
constexpr int kLayoutSwapped = 1;
// The layout of g^t (and lambda^t) in a sweep of the in-place schedule.
inline int layout_at(bool aa, long long t) { return aa && (t & 1) ? kLayoutSwapped : kLayoutNatural; }
// lin / lout: layouts of the input and output states (stream-collide: natural -> natural is the two-buffer pull,
// natural -> swapped and swapped -> natural the in-place pair; stream-only into the caller's array: any lin)
lbm_status step_launch_cmp(const PlanInfo& p, int mode, const void* src, void* dst, bool dense_in, bool dense_out,
                           const Bc& bc, const double* tau, cudaStream_t s, int lin = kLayoutNatural,
                           int lout = kLayoutNatural);
// lin: layout of g^{t-1} and lambda^{t+1}; lout: of lambda^t (as for the step)
lbm_status adjoint_launch_cmp(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out,
                              const Bc& bc, const double* tau, double* grad_acc, double* partial, cudaStream_t s,
                              int lin = kLayoutNatural, int lout = kLayoutNatural);
// the caller's dense array into a compact state (lambda's layouts: swapped puts lambda_d(x) at (x - c_d, opp(d)))
lbm_status compact_gather_launch(const PlanInfo& p, const void* dense, void* compact, cudaStream_t s,
                                 int layout = kLayoutNatural);
lbm_status compact_gather_add_launch(const PlanInfo& p, const void* dense, void* compact, cudaStream_t s,
                                     int layout = kLayoutNatural);
lbm_status add_state_launch(const PlanInfo& p, void* dst, const void* src, cudaStream_t s);
lbm_status accumulate_launch(double* dst, const double* src, cudaStream_t s);

lbm_status probe_launch(const PlanInfo& p, const void* f, long long n_probe, const int64_t* node,
                        const double* rho_target, double weight, double* d_loss, void* lambda, uint32_t* status,
                        cudaStream_t s);

void spline_basis_host(int K, int n, double* basis);
lbm_status spline_profile_launch(const PlanInfo& p, int ky, int kz, const double* by, const double* bz,
                                 const double* c, double rho_out, double* rho_in, cudaStream_t s);
lbm_status spline_grad_launch(const PlanInfo& p, int ky, int kz, const double* by, const double* bz,
                              const double* g, double* gc, cudaStream_t s);

bool persist_ok(const PlanInfo& p);
lbm_status forward_persist(const PlanInfo& p, const PersistArgs& a, const Bc& bc, const double* tau, cudaStream_t s);
lbm_status reverse_persist(const PlanInfo& p, const PersistArgs& a, const Bc& bc, const double* tau,
                           double* grad_acc, double* partial, cudaStream_t s);

inline lbm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

}  // namespace lbm
