// Fluid-only ("compact") layout: the forward and adjoint steps over the
// fluid nodes alone.
//
// The step of Eq. 1-6 of arXiv 2310.00810 (and, in the adjoint, its exact
// transpose) moves Q populations in and Q out per node, so its time is set
// by the bytes it moves.  A dense layout moves solid nodes as well: in a
// Boolean sphere packing at porosity 0.45 with r = 6 the solid runs along x
// are short, nearly every 32-byte sector holds some fluid node, and skipping
// solid nodes saves almost nothing.  Here the state holds only the nf fluid
// nodes (compact index k: the interior in node order, then the columns
// x = 0 and nx - 1 in node order), and a neighbour table gives, per
// direction i >= 1, where node k pulls from:
//   nbr[(i - 1) nf + k] = compact index of x - c_i    (a fluid node)
//                       = kCmpBB                     (halfway bounce-back link)
//                       = kCmpABB                    (Eq. 6 link through x = -1/2 or nx - 1/2)
// built once from the link words.  Per fluid-node update the forward moves
// 2 Q populations plus 4 (Q - 1) table bytes and nothing for solid nodes.
// Consecutive fluid nodes of a row have mostly consecutive neighbours, so
// the table-driven loads of a warp stay nearly coalesced.
//
// Boundary rules, collision and the adjoint algebra are the ones of step.cu
// and adjoint.cu (same helpers); only the addressing differs.  The dense
// index idx[k] recovers (x, y, z) where the rules need it: the Eq. 6 nodes
// (density and inlet-gradient slot of the row) and the conversions between
// the caller's dense arrays and the internal compact states.
//
// In-place (AA-pattern) streaming.  Slot (x, i) of a state is entry
// [i][x].  A state is stored in one of two layouts:
//   natural (N): slot (x, i) holds g_i(x);
//   swapped (W): g_i(x) sits at (x + c_i, opp(i)) where x + c_i is a fluid
//                node, else at (x, i) (the population comes back to x:
//                bounce-back, Eq. 6, the velocity inlet),
// so that in W everything node x receives sits in its own slots: direction
// i at (x, opp(i)).  A step from N gathers through the table and scatters
// its output into W (the gather step); a step from W reads and writes node
// x's own slots (the local step, no table).  In both, the slots a node
// writes are exactly the slots it reads, so each step can run in place on
// one buffer.  The adjoint (gather form) streams the other way: for lambda,
// W puts lambda_m(x) at (x - c_m, opp(m)) where x - c_m is a fluid node,
// else at (x, m), and the same two steps alternate.  A sweep stores g^t in N
// for even t and in W for odd t (lambda^t likewise), so that every other
// step of the forward and of the adjoint reads no table.  The Eq. 6 nodes
// need the velocity of their own g^{t-1}, which in place may already be
// overwritten by a neighbour: each in-place forward step keeps it per
// boundary node in a small side array (the node writes the velocity of its
// output, and reads it back at the next step).
#include <algorithm>
#include <type_traits>

#include "device.cuh"

namespace lbm {

#define LBM_CMP_TRY(expr)                 \
    do {                                  \
        lbm_status st__ = (expr);         \
        if (st__ != LBM_OK) return st__;  \
    } while (0)

namespace {

constexpr int kCmpThreads = 256;
constexpr int kScanNodes = 1024;  // nodes per block of the table-building scan (256 threads x 4)

// How a step finds what node x receives, and where it writes what x sends.
constexpr int kInGather = 0;    // from a natural state through the table (also the two-buffer pull)
constexpr int kInLocal = 1;     // from a swapped state, in x's own slots
constexpr int kOutOwn = 0;      // into x's own slots: natural layout
constexpr int kOutScatter = 1;  // through the table: swapped layout
constexpr int kOutDense = 2;    // into the caller's dense [Q][N] array

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct TableLayout {
    size_t inst, idx, nbr, eq6, cmap, blk, total_slot, bytes;
};

TableLayout table_layout(const PlanInfo& p, long long nf)
{
    TableLayout t;
    const long long nblk = (p.geo.N + kScanNodes - 1) / kScanNodes;
    size_t o = 0;
    t.inst = o;  // the lattice as a pack of one (BCmpInst)
    o += a256(sizeof(BCmpInst));
    t.idx = o;
    o += a256(sizeof(int32_t) * (size_t)nf);
    t.nbr = o;
    o += a256(sizeof(int32_t) * (size_t)(p.q - 1) * (size_t)nf);
    t.eq6 = o;
    o += a256(sizeof(uint32_t) * (size_t)((nf + 31) / 32));
    t.cmap = o;
    o += a256(sizeof(int32_t) * (size_t)p.geo.N);
    t.blk = o;
    o += a256(sizeof(int32_t) * (size_t)nblk);
    t.total_slot = o;
    o += 256;
    t.bytes = o;
    return t;
}

// --------------------------------------------------------------- the tables

__device__ __forceinline__ int block_sum_int(int v)
{
    __shared__ int s[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (int)threadIdx.x < nw ? s[threadIdx.x] : 0;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

// Exclusive scan of one int per thread over the block (blockDim.x a multiple
// of 32, at most 1024); *total gets the block sum.
__device__ __forceinline__ int block_excl_scan(int v, int* total)
{
    __shared__ int s[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = lane < nw ? s[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane < nw) s[lane] = x;  // inclusive warp totals
    }
    __syncthreads();
    const int before = w > 0 ? s[w - 1] : 0;
    *total = s[nw - 1];
    __syncthreads();
    return before + inc - v;
}

// The compact order: the interior fluid nodes first, in node order, then the
// fluid nodes of the columns x = 0 and x = nx - 1 (the only ones that can
// have an Eq. 6 or velocity-inlet link), in node order.  The boundary nodes
// take a longer branch of the step and adjoint kernels; grouped, they do not
// split the warps of the interior.
__device__ __forceinline__ bool cmp_member(const uint32_t* __restrict__ link, long long n, long long N, int nx, int cls)
{
    if (n >= N || (link[n] & kLinkSolid)) return false;
    const int x = (int)(n % nx);
    return ((x == 0 || x == nx - 1) ? 1 : 0) == cls;
}

// Fluid nodes of class cls (0 interior, 1 boundary columns) per 1024-node block.
__global__ void __launch_bounds__(256) k_cmp_count(const uint32_t* __restrict__ link, long long N, int nx, int cls,
                                                   int* __restrict__ blk)
{
    const long long base = (long long)blockIdx.x * kScanNodes;
    int c = 0;
    for (int j = threadIdx.x; j < kScanNodes; j += blockDim.x)
        if (cmp_member(link, base + j, N, nx, cls)) ++c;
    c = block_sum_int(c);
    if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

// In-place exclusive scan of the block counts (one block); total fluid count out.
__global__ void __launch_bounds__(1024) k_cmp_scan(int* __restrict__ blk, long long nblk, long long* __restrict__ total)
{
    long long carry = 0;
    for (long long b0 = 0; b0 < nblk; b0 += blockDim.x) {
        const long long b = b0 + threadIdx.x;
        const int v = b < nblk ? blk[b] : 0;
        int sum;
        const int ex = block_excl_scan(v, &sum);
        if (b < nblk) blk[b] = (int)(carry + ex);
        carry += sum;
    }
    if (threadIdx.x == 0) *total = carry;
}

// Dense -> compact map and the compact -> dense index of the class-cls
// nodes, in node order from compact index *base (0 for the interior, the
// interior count for the boundary columns).  The interior pass marks every
// other node -1; the boundary pass then fills its own entries.
__global__ void __launch_bounds__(256) k_cmp_index(const uint32_t* __restrict__ link, long long N, int nx, int cls,
                                                   const long long* __restrict__ base, const int* __restrict__ blk,
                                                   int32_t* __restrict__ cmap, int32_t* __restrict__ idx, long long nf)
{
    const long long n0 = (long long)blockIdx.x * kScanNodes + 4LL * threadIdx.x;
    bool fl[4];
    int c = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        fl[j] = cmp_member(link, n0 + j, N, nx, cls);
        c += fl[j] ? 1 : 0;
    }
    int sum;
    long long k = (cls ? *base : 0) + (long long)blk[blockIdx.x] + block_excl_scan(c, &sum);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long long n = n0 + j;
        if (n >= N) break;
        if (fl[j] && k >= 0 && k < nf) {
            cmap[n] = (int32_t)k;
            idx[k] = (int32_t)n;
            ++k;
        } else if (!cls) {
            cmap[n] = -1;
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(256) k_cmp_nbr(const uint32_t* __restrict__ link, const int32_t* __restrict__ cmap,
                                                 const int32_t* __restrict__ idx, int32_t* __restrict__ nbr,
                                                 long long nf, Geo g)
{
    using L = Lattice<Q>;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const long long n = idx[k];
    const int x = (int)(n % g.nx), y = (int)((n / g.nx) % g.ny), z = (int)(n / ((long long)g.nx * g.ny));
    const uint32_t lw = link[n];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        int32_t code;
        const int xs = x - L::c(i, 0), zs = z - L::c(i, 2);
        int ys = y - L::c(i, 1);
        if (g.periodic_y) ys = (ys + g.ny) % g.ny;  // ys is in -1..ny
        if ((lw >> i) & 1u) {
            code = kCmpBB;
        } else if (xs < 0 || xs >= g.nx) {
            code = kCmpABB;
        } else {
            // a link that is neither bounce-back nor Eq. 6 starts at a fluid node inside the lattice;
            // anything else (an inconsistent link array) is treated as bounce-back
            const bool inside = ys >= 0 && ys < g.ny && zs >= 0 && zs < g.nz;
            const long long m = ((long long)zs * g.ny + ys) * g.nx + xs;
            code = inside ? cmap[m] : kCmpBB;
            if (code < 0) code = kCmpBB;
        }
        nbr[(long long)(i - 1) * nf + k] = code;
    }
}

// One bit per compact node: set where the node has an Eq. 6 (or velocity
// inlet) link, the nodes the local step of the in-place schedule sends to
// the table path.  Bit k & 31 of word k >> 5.
template <int Q>
__global__ void __launch_bounds__(256) k_cmp_eq6_bits(const int32_t* __restrict__ nbr, long long nf,
                                                      uint32_t* __restrict__ bits)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool b = false;
    if (k < nf)
        for (int i = 1; i < Q; ++i) b |= nbr[(long long)(i - 1) * nf + k] == kCmpABB;
    const unsigned w = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && k < nf) bits[k >> 5] = w;
}

// ----------------------------------------------------------- the step kernels

// The node's own inlet/outlet data for Eq. 6 (only nodes with an Eq. 6 link).
struct Side {
    bool xin;
    long long row;  // z * ny + y
};

__device__ __forceinline__ Side side_of(const int32_t* __restrict__ idx, long long k, const Geo& g)
{
    const long long n = idx[k];
    Side s;
    s.xin = (n % g.nx) == 0;
    s.row = n / g.nx;
    return s;
}

// The side-array entry of an Eq. 6 node (three values): inlet rows first,
// then outlet rows; acc_off counts the rows of the instances before it.
template <typename T>
__device__ __forceinline__ T* side_entry(const Bc& bc, const Geo& g, long long acc_off, const Side& sd)
{
    const long long rows = (long long)g.ny * g.nz;
    return static_cast<T*>(bc.side_u) + 3 * (2 * acc_off + (sd.xin ? 0 : rows) + sd.row);
}

__device__ __forceinline__ bool eq6_bit(const Cmp& c, long long k)
{
    return (__ldg(c.eq6 + (k >> 5)) >> (k & 31)) & 1u;
}

// The velocity of node k's own post-collision populations g(x), from a
// state in layout IN (natural: own slots; swapped: where x sent them).
template <int Q, typename T, int IN>
__device__ __forceinline__ void own_velocity(T (&u)[3], const T* __restrict__ src, long long k, long long NF,
                                             const int32_t (&code)[Q])
{
    using L = Lattice<Q>;
    T loc[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int32_t co = i > 0 ? code[L::opp(i)] : -1;
        loc[i] = (IN == kInLocal && co >= 0) ? src[(size_t)L::opp(i) * NF + co] : src[(size_t)i * NF + k];
    }
    T drho, rho;
    moments<Q, T>(loc, drho, rho, u);
}

// What an Eq. 6 node receives.  Its velocity comes from the side array in
// the in-place forward steps (bc.side_u), else from src.  A population that
// comes back to x (bounce-back, Eq. 6, velocity inlet) starts from x's own
// g_opp(i), at slot (x, opp(i)) in both layouts.
template <int Q, typename T, int IN>
__device__ __forceinline__ void pull_eq6(T (&v)[Q], const T* __restrict__ src, long long k, long long NF,
                                         const int32_t (&code)[Q], const Cmp& c, const Geo& g, const Bc& bc,
                                         long long acc_off)
{
    using L = Lattice<Q>;
    const Side sd = side_of(c.idx, k, g);
    T u[3];
    if (bc.side_u) {
        const T* e = side_entry<T>(bc, g, acc_off, sd);
        u[0] = e[0];
        u[1] = e[1];
        u[2] = e[2];
    } else {
        own_velocity<Q, T, IN>(u, src, k, NF, code);
        if constexpr (IN == kInGather) {
            if (bc.uw_extrap) {
                const int32_t ke = code[inward_dir<Q>(sd.xin)];
                if (ke >= 0) extrapolate_wall_velocity<Q, T>(u, src, NF, ke);
            }
        }
    }
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double rw = sd.xin ? (bc.profile ? bc.rho_in[sd.row] : bc.rho_in[0]) : bc.rho_out;
    const T drw = T(rw - 1.0), rwT = T(rw);
    v[0] = src[k];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (code[i] >= 0) {
            v[i] = IN == kInGather ? src[(size_t)i * NF + code[i]] : src[(size_t)L::opp(i) * NF + k];
            continue;
        }
        const T back = src[(size_t)L::opp(i) * NF + k];
        if (code[i] == kCmpBB) {
            v[i] = back;
        } else if (sd.xin && bc.vel_inlet) {
            // velocity inlet: moving-wall bounce-back, f_i = f*_opp(i) + 6 w_i (c_i . u_in) (rho_0 = 1)
            const double* uin = inlet_velocity(bc.status);
            double cu = 0.0;
#pragma unroll
            for (int a = 0; a < L::D; ++a) cu += (double)L::c(i, a) * uin[a];
            v[i] = back + T(6.0 * L::w(i) * cu * inlet_ramp(bc));
        } else {
            const T cu = cdot<Q, T>(i, u);
            v[i] = -back + T(2.0 * L::w(i)) * (drw + rwT * (T(4.5) * cu * cu - T(1.5) * uu));
        }
    }
}

// What an interior node receives (no Eq. 6 link): through the table from a
// natural state, or its own slots of a swapped state.  Per-direction base
// pointers are uniform across the block; the per-thread part of each address
// is a 32-bit index.
template <int Q, typename T, int IN>
__device__ __forceinline__ void pull_interior(T (&v)[Q], const T* __restrict__ src, int32_t k32, size_t NF,
                                              const int32_t (&code)[Q])
{
    using L = Lattice<Q>;
    v[0] = src[k32];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (IN == kInLocal) {
            v[i] = src[(size_t)L::opp(i) * NF + k32];
        } else {
            const bool fl = code[i] >= 0;
            const T* __restrict__ base = src + (size_t)(fl ? i : L::opp(i)) * NF;
            v[i] = base[fl ? code[i] : k32];
        }
    }
}

// The two-buffer pull of node k (natural state in), for the per-row pass
// of the extrapolated-velocity adjoint.
template <int Q, typename T>
__device__ __forceinline__ void pull_cmp(T (&v)[Q], const T* __restrict__ src, long long k, long long NF,
                                         const int32_t (&code)[Q], bool bnd, const Cmp& c, const Geo& g,
                                         const Bc& bc)
{
    if (bnd) pull_eq6<Q, T, kInGather>(v, src, k, NF, code, c, g, bc, 0);
    else pull_interior<Q, T, kInGather>(v, src, (int32_t)k, (size_t)NF, code);
}

template <int Q>
__device__ __forceinline__ bool load_codes(int32_t (&code)[Q], const Cmp& c, long long k)
{
    code[0] = 0;
    bool bnd = false;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        code[i] = __ldg(c.nbr + (size_t)(i - 1) * (size_t)c.nf + (int32_t)k);
        bnd |= code[i] == kCmpABB;
    }
    return bnd;
}

// A table entry loaded again where it is needed (an L1 hit: the node loaded
// it at the start of its update).  The scattered stores of the in-place
// steps need the whole table of a node after its collision; on D3Q19,
// keeping it in registers through the collision spills.  `after` is a zero
// computed from the collision's output, so the reload cannot be scheduled
// before the collision; the asm is volatile so that it is not merged with
// the first load.
__device__ __forceinline__ int32_t reload_code(const Cmp& c, int i, int32_t k32, int32_t after)
{
    int32_t v;
    const int32_t* p = c.nbr + (size_t)(i - 1) * (size_t)c.nf + (k32 + after);
    asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// An opaque zero that depends on x.
template <typename T>
__device__ __forceinline__ int32_t zero_after(T x)
{
    int32_t z;
    const float f = (float)x;
    asm volatile("and.b32 %0, %1, 0;" : "=r"(z) : "r"(__float_as_int(f)));
    return z;
}

// D3Q19 reloads its table for the scattered stores; D2Q9 keeps it in registers.
template <int Q>
constexpr bool kReloadCodes = Q == 19;

// Stores what node k sends: into its own slots (natural), through the table
// (swapped: g_i(x) to (x + c_i, opp(i)) where that node is fluid), or into
// the caller's dense array.
template <int Q, typename T, int OUT>
__device__ __forceinline__ void store_node(T* __restrict__ dst, const T (&v)[Q], long long k, const Cmp& c,
                                           const Geo& g, const int32_t (&code)[Q])
{
    using L = Lattice<Q>;
    if (OUT == kOutScatter) {
        const size_t NF = (size_t)c.nf;
        const int32_t k32 = (int32_t)k;
        const int32_t after = kReloadCodes<Q> ? zero_after(v[Q - 1]) : 0;
        dst[k32] = v[0];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int32_t co = kReloadCodes<Q> ? reload_code(c, L::opp(i), k32, after) : code[L::opp(i)];
            const bool fl = co >= 0;
            (dst + (size_t)(fl ? L::opp(i) : i) * NF)[fl ? co : k32] = v[i];
        }
        return;
    }
    const long long n = OUT == kOutDense ? (long long)c.idx[k] : k;
    const size_t S = OUT == kOutDense ? (size_t)g.N : (size_t)c.nf;
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[(size_t)i * S + n] = v[i];
}

// The velocity of an Eq. 6 node's output, for the next in-place step.
template <int Q, typename T>
__device__ __forceinline__ void keep_velocity(const T (&v)[Q], long long k, const Cmp& c, const Geo& g, const Bc& bc,
                                              long long acc_off)
{
    T drho, rho, u[3];
    moments<Q, T>(v, drho, rho, u);
    T* e = side_entry<T>(bc, g, acc_off, side_of(c.idx, k, g));
    e[0] = u[0];
    e[1] = u[1];
    e[2] = u[2];
}

__device__ __forceinline__ int block_instance(const int* __restrict__ blk_inst, long long k)
{
    return blk_inst ? blk_inst[k / kCmpThreads] : 0;
}

// The instance's boundary data: its inlet densities, on top of the call's
// options and status word (tmpl.rho_in is the base of the inlet array).
__device__ __forceinline__ Bc instance_bc(const Bc& tmpl, const BCmpInst& I)
{
    Bc bc = tmpl;
    bc.rho_in = tmpl.rho_in + I.in_off;
    bc.profile = I.n_in > 1 ? 1 : 0;
    return bc;
}

// Update of a node with an Eq. 6 link (x = 0 or nx - 1), out of line so that
// its extra live values (the node's own populations and velocity) do not
// raise the register count, and lower the occupancy, of the interior path.
template <int Q, typename T, int MODE, int IN, int OUT>
__device__ __noinline__ void step_node_eq6(const T* __restrict__ src, T* __restrict__ dst, long long k, const Cmp& c,
                                           const BCmpInst* __restrict__ Ip, const Bc& tmpl, T omega)
{
    const Geo g = Ip->g;
    const Bc bc = instance_bc(tmpl, *Ip);
    int32_t code[Q];
    load_codes<Q>(code, c, k);
    T v[Q];
    pull_eq6<Q, T, IN>(v, src, k, c.nf, code, c, g, bc, Ip->acc_off);
    if (MODE != kStreamOnly) collide_any<Q, T>(v, omega, bc);
    store_node<Q, T, OUT>(OUT == kOutDense ? dst + Ip->f_off : dst, v, k, c, g, code);
    if (MODE != kStreamOnly && bc.side_u) keep_velocity<Q, T>(v, k, c, g, bc, Ip->acc_off);
}

// The same update inlined into the main stream-collide kernels: the Eq. 6
// nodes take their own branch of the kernel (their extra live values may
// spill there, on the few boundary threads, while the interior path keeps
// its registers), and share the sectors their interior neighbours load in
// the same launch.
template <int Q, typename T, int MODE, int IN, int OUT>
__device__ __forceinline__ void step_node_eq6_inline(const T* __restrict__ src, T* __restrict__ dst, long long k,
                                                     const Cmp& c, const BCmpInst* __restrict__ Ip, const Bc& tmpl,
                                                     T omega)
{
    const Geo g = Ip->g;
    const Bc bc = instance_bc(tmpl, *Ip);
    int32_t code[Q];
    load_codes<Q>(code, c, k);
    T v[Q];
    pull_eq6<Q, T, IN>(v, src, k, c.nf, code, c, g, bc, Ip->acc_off);
    if (MODE != kStreamOnly) collide_any<Q, T>(v, omega, bc);
    store_node<Q, T, OUT>(OUT == kOutDense ? dst + Ip->f_off : dst, v, k, c, g, code);
    if (MODE != kStreamOnly && bc.side_u) keep_velocity<Q, T>(v, k, c, g, bc, Ip->acc_off);
}

// One node of a step (MODE: stream-collide, collide-only or stream-only,
// step.cu) of instance *Ip.  DIN: the collide-only input is the instance's
// dense [Q][N] array.  IN / OUT: the addressing of the input and output
// states (two-buffer pull: gather / own; in place: gather / scatter, then
// local / own; OUT dense: the caller's array, solid entries left to the
// caller).  Interior nodes need only the call's options (tmpl); the
// instance's sizes and inlet data are read on the Eq. 6 path alone.
template <int Q, typename T, int MODE, bool DIN, int IN, int OUT, bool INL = false>
__device__ __forceinline__ void step_cmp_node(const T* __restrict__ src, T* __restrict__ dst, long long k, const Cmp& c,
                                              const BCmpInst* __restrict__ Ip, const Bc& tmpl, T omega)
{
    T v[Q];
    int32_t code[Q];
    if (MODE == kCollideOnly) {
        if (DIN) {
            const long long n = c.idx[k], N = Ip->g.N;
            const T* s = src + Ip->f_off;
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = s[(size_t)i * (size_t)N + n];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = src[(size_t)i * (size_t)c.nf + k];
        }
        collide_any<Q, T>(v, omega, tmpl);
        store_node<Q, T, kOutOwn>(dst, v, k, c, Ip->g, code);
        if (tmpl.side_u && eq6_bit(c, k)) keep_velocity<Q, T>(v, k, c, Ip->g, tmpl, Ip->acc_off);
        return;
    }
    // INL: the Eq. 6 update inlined (the main stream-collide kernels), else out of line
    if (IN == kInLocal ? eq6_bit(c, k) : load_codes<Q>(code, c, k)) {
        if (INL) step_node_eq6_inline<Q, T, MODE, IN, OUT>(src, dst, k, c, Ip, tmpl, omega);
        else step_node_eq6<Q, T, MODE, IN, OUT>(src, dst, k, c, Ip, tmpl, omega);
        return;
    }
    pull_interior<Q, T, IN>(v, src, (int32_t)k, (size_t)c.nf, code);  // interior: no sizes or inlet data used
    if (MODE != kStreamOnly) collide_any<Q, T>(v, omega, tmpl);
    store_node<Q, T, OUT>(OUT == kOutDense ? dst + Ip->f_off : dst, v, k, c, Ip->g, code);
}

// Transpose of the collision (adjoint.cu, step 3) at one node, from f^t (its
// moments drho, rho, u) and mu = dL/df*: gives lambda^t and returns the
// node's dL/domega term.  G holds the Eq. 6 velocity terms (zero inside).
template <int Q, typename T>
__device__ __forceinline__ T adjoint_collision(const T (&f)[Q], const T (&mu)[Q], T drho, T rho, const T (&u)[3],
                                               const T (&G)[3], T omega, T (&lam)[Q], const Bc& bc)
{
    using L = Lattice<Q>;
    if constexpr (Q == 9) {
        if (bc.mrt) return adjoint_collision_mrt<T>(f, mu, drho, rho, u, G, omega, mrt_rates(bc.status), lam);
    }
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T A = 0, B[3] = {T(0), T(0), T(0)}, domT = 0;
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
    for (int kk = 0; kk < Q; ++kk) {
        T s = keep * mu[kk] + base;
#pragma unroll
        for (int a = 0; a < L::D; ++a) s += Bt[a] * (T(L::c(kk, a)) - u[a]);
        lam[kk] = s;
    }
    return domT;
}

// Stores lambda^t(x): into x's own slots (natural), or through the table
// (swapped: lambda_m(x) to (x - c_m, opp(m)) where that node is fluid).
template <int Q, typename T, int OUT>
__device__ __forceinline__ void store_lambda(T* __restrict__ lam_out, const T (&lam)[Q], long long k, const Cmp& c,
                                             const int32_t (&code)[Q])
{
    using L = Lattice<Q>;
    const size_t NF = (size_t)c.nf;
    const int32_t k32 = (int32_t)k;
    const int32_t after = OUT == kOutScatter && kReloadCodes<Q> ? zero_after(lam[Q - 1]) : 0;
    lam_out[k32] = lam[0];
#pragma unroll
    for (int m = 1; m < Q; ++m) {
        const int32_t co = OUT != kOutScatter ? -1 : (kReloadCodes<Q> ? reload_code(c, m, k32, after) : code[m]);
        const bool fl = co >= 0;
        (lam_out + (size_t)(fl ? L::opp(m) : m) * NF)[fl ? co : k32] = lam[m];
    }
}

// Adjoint update of a node with an Eq. 6 link, out of line (see
// step_node_eq6).  Adds the node's inlet gradient term (one owner per inlet
// node) and returns its dL/domega term.  mu_j(x) is lambda^{t+1}_j(x + c_j)
// where that node is fluid, else lambda^{t+1}_opp(j)(x), at slot
// (x, opp(j)) in both layouts.
template <int Q, typename T, bool T0, int IN, int OUT>
__device__ __noinline__ T adjoint_node_eq6(const T* __restrict__ gprev, const T* __restrict__ lam_in,
                                           T* __restrict__ lam_out, long long k,
                                           Cmp c, const BCmpInst* __restrict__ Ip, Bc tmpl, T omega,
                                           double* __restrict__ grad_acc_base)
{
    using L = Lattice<Q>;
    const Geo g = Ip->g;
    Bc bc = instance_bc(tmpl, *Ip);
    bc.side_u = nullptr;  // the segment states are read-only here: the velocity comes from gprev
    double* __restrict__ grad_acc = grad_acc_base + Ip->acc_off;
    const size_t NF = (size_t)c.nf;
    int32_t code[Q];
    load_codes<Q>(code, c, k);
    // 1. f^t(x)
    T f[Q];
    if (T0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = T(0);
    } else {
        pull_eq6<Q, T, IN>(f, gprev, k, c.nf, code, c, g, bc, Ip->acc_off);
    }
    T drho, rho, u[3];
    moments<Q, T>(f, drho, rho, u);
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    // 2. transpose of streaming and boundaries
    const Side sd = side_of(c.idx, k, g);
    const T rwT = T(sd.xin ? (bc.profile ? bc.rho_in[sd.row] : bc.rho_in[0]) : bc.rho_out);
    T mu[Q];
    T G[3] = {T(0), T(0), T(0)};
    double grw = 0.0;
    mu[0] = lam_in[k];
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        const int o = L::opp(j);
        const int32_t co = code[o];
        if (co >= 0) {
            mu[j] = IN == kInGather ? lam_in[(size_t)j * NF + co] : lam_in[(size_t)o * NF + k];
        } else if (co == kCmpBB || (sd.xin && bc.vel_inlet)) {
            mu[j] = lam_in[(size_t)o * NF + k];  // the velocity inlet's source is constant
        } else {
            const T li = lam_in[(size_t)o * NF + k];
            mu[j] = -li;
            const T cu = cdot<Q, T>(o, u);
            const T two_w = T(2.0 * L::w(o));
            if (sd.xin) grw += (double)(li * two_w * (T(1) + T(4.5) * cu * cu - T(1.5) * uu));
#pragma unroll
            for (int a = 0; a < L::D; ++a) G[a] += li * two_w * rwT * (T(9) * cu * T(L::c(o, a)) - T(3) * u[a]);
        }
    }
    T lam[Q];
    const T domT = adjoint_collision<Q, T>(f, mu, drho, rho, u, G, omega, lam, bc);
    store_lambda<Q, T, OUT>(lam_out, lam, k, c, code);
    // 4. inlet gradient (one owner per inlet node)
    if (sd.xin) grad_acc[sd.row] += grw;
    return domT;
}

// Adjoint step in the compact layout: the gather form of adjoint.cu.  The
// forward copies f*_j(x) to x + c_j, the node that pulls direction j from x;
// its compact index is nbr of direction opp(j) at k (x + c_j = x - c_opp(j)).
// IN gather: f^t and mu through the table, lambda^t to OUT (own: the
// two-buffer pull; scatter: the gather step in place); IN local: both from
// x's own slots, lambda^t to its own slots.  lam_in and lam_out may be the
// same buffer (in place: each node reads all it needs before it writes the
// same slots).  One node of instance *Ip; returns its dL/domega term.  As in
// step_cmp_node, interior nodes use the call's options only.
template <int Q, typename T, bool T0, int IN, int OUT>
__device__ __forceinline__ T adjoint_cmp_node(const T* __restrict__ gprev, const T* __restrict__ lam_in,
                                              T* __restrict__ lam_out, long long k,
                                              const Cmp& c, const BCmpInst* __restrict__ Ip, const Bc& tmpl, T omega,
                                              double* __restrict__ grad_acc)
{
    using L = Lattice<Q>;
    int32_t code[Q];
    if (IN == kInLocal) {
        if (eq6_bit(c, k))
            return adjoint_node_eq6<Q, T, T0, IN, OUT>(gprev, lam_in, lam_out, k, c, Ip, tmpl, omega, grad_acc);
    } else if (load_codes<Q>(code, c, k)) {
        return adjoint_node_eq6<Q, T, T0, IN, OUT>(gprev, lam_in, lam_out, k, c, Ip, tmpl, omega, grad_acc);
    }
    // Interior node: every load of f^t and of the gathered lambda depends
    // only on the table (or on k alone), so all 2 Q are in flight together.
    const size_t NF = (size_t)c.nf;
    const int32_t k32 = (int32_t)k;
    T f[Q], mu[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int o = L::opp(i);
        if (IN == kInLocal) {
            f[i] = T0 ? T(0) : gprev[(size_t)o * NF + k32];
            mu[i] = lam_in[(size_t)o * NF + k32];
            continue;
        }
        if (T0) {
            f[i] = T(0);
        } else {
            const bool fl = i > 0 && code[i] >= 0;
            f[i] = (gprev + (size_t)(fl ? i : o) * NF)[fl ? code[i] : k32];
        }
        const bool ml = i > 0 && code[o] >= 0;
        mu[i] = (lam_in + (size_t)(ml ? i : o) * NF)[ml ? code[o] : k32];
    }
    T drho, rho, u[3];
    moments<Q, T>(f, drho, rho, u);
    const T G[3] = {T(0), T(0), T(0)};
    T lam[Q];
    const T dom = adjoint_collision<Q, T>(f, mu, drho, rho, u, G, omega, lam, tmpl);
    store_lambda<Q, T, OUT>(lam_out, lam, k, c, code);
    return dom;
}

// One FP64 partial per warp (its sum in T), accumulated in place across time
// steps: no block barrier, so a warp that finishes early frees its slot at
// once instead of waiting for the slowest warp of the block.  The warp of
// compact node k owns slot k >> 5 (lane 0 holds the warp's first node).
template <typename T>
__device__ __forceinline__ void add_warp_partial(T dom, bool live, long long k, double* __restrict__ partial)
{
    T dw = dom;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dw += __shfl_xor_sync(0xffffffffu, dw, o);
    if ((threadIdx.x & 31) == 0 && live) partial[k >> 5] += (double)dw;
}

// Reverse of the extrapolated Eq. 6 velocity in the compact layout: the
// per-row pass of adjoint.cu (k_adjoint_uw), with the boundary node found
// through cmap and its inward neighbour through its own table entry.
template <int Q, typename T>
__global__ void __launch_bounds__(kCmpThreads)
    k_adjoint_uw_cmp(const T* __restrict__ gprev, const T* __restrict__ lam_in, T* __restrict__ lam_out, Cmp c,
                     const int32_t* __restrict__ cmap, Geo g, Bc bc, double* __restrict__ grad_acc)
{
    pdl_enter();
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (long long)g.ny * g.nz) return;
    const size_t NF = (size_t)c.nf;
    for (int side = 0; side < 2; ++side) {
        const bool xin = side == 0;
        if (xin && bc.vel_inlet) continue;  // the velocity inlet does not use u_w
        const int32_t kb = cmap[row * g.nx + (xin ? 0 : g.nx - 1)];
        if (kb < 0) continue;
        int32_t cb[Q], ce[Q];
        const bool bb = load_codes<Q>(cb, c, kb);
        const int32_t ke = cb[inward_dir<Q>(xin)];
        if (ke < 0) continue;  // inward neighbour solid: u_w is the node's own velocity
        const bool be = load_codes<Q>(ce, c, ke);
        T fb[Q], fe[Q], li[Q];
        pull_cmp<Q, T>(fb, gprev, kb, c.nf, cb, bb, c, g, bc);
        pull_cmp<Q, T>(fe, gprev, ke, c.nf, ce, be, c, g, bc);
        uint32_t eq6 = 0;
        li[0] = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool on = cb[i] == kCmpABB;
            eq6 |= on ? (1u << i) : 0u;
            li[i] = on ? lam_in[(size_t)i * NF + kb] : T(0);
        }
        const T rw = T(xin ? (bc.profile ? bc.rho_in[row] : bc.rho_in[0]) : bc.rho_out);
        T db[Q], de[Q];
        const double dg = adjoint_uw_delta<Q, T>(fb, fe, li, eq6, rw, db, de);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            lam_out[(size_t)k * NF + kb] += db[k];
            lam_out[(size_t)k * NF + ke] += de[k];
        }
        if (xin) grad_acc[row] += dg;
    }
}

// CTAs of `kernel` that fit on the GPU at once (the grid of a grid-stride launch).
template <class K>
unsigned resident_ctas(K kernel)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kCmpThreads, 0);
    return (unsigned)(std::max(per_sm, 1) * std::max(sms, 1));
}

// --------------------------------------------- the kernels, lattices and batches
//
// The kernels below serve a single lattice and a packed batch alike.  A
// block's nodes belong to one instance (blk_inst[block]; a single lattice
// passes no block table and is instance 0), whose entry gives its sizes, the
// offsets of its inlet data and dense arrays, and its tau.  A single lattice
// is a pack of one, so a batch instance gets bit for bit what a single plan
// computes: the same kernels run the same per-node code.

static_assert(kBatchCmpAlign == kCmpThreads, "one thread block per aligned node range of a batch instance");

// One step.  MODE: stream-collide, collide-only or stream-only (step.cu);
// DIN: the input is the instance's dense [Q][N] array; IN / OUT: see
// step_cmp_node.  src == dst is allowed for the in-place pairs (gather in,
// scatter out; local in, own out): the slot sets of different nodes are
// disjoint, and a node loads every slot it owns before it stores any (each
// stored value depends on all loaded ones through the moments), so no load
// can see a store of the same launch and the pointers stay __restrict__.
// Padding nodes of a batch carry
// bounce-back codes in every direction and start at zero (the rest state),
// so they stay exactly zero: they run through the interior path like any
// node, and only a dense read or write needs them skipped.
// INL: the Eq. 6 update inlined (see step_node_eq6_inline).
template <int Q, typename T, int MODE, bool DIN, int IN, int OUT, bool INL = false>
__global__ void __launch_bounds__(kCmpThreads, 4)
    k_step_cmp(const T* __restrict__ src, T* __restrict__ dst, Cmp c, const BCmpInst* __restrict__ insts,
               const int* __restrict__ blk_inst, Bc tmpl, const double* __restrict__ tau)
{
    pdl_enter();
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= c.nf) return;
    const int i = block_instance(blk_inst, k);
    const BCmpInst* Ip = insts + i;
    if ((DIN || OUT == kOutDense) && k >= Ip->k0 + Ip->nf) return;
    const T omega = T(1) / T(tau[i]);  // in T: FP64 arithmetic is slow on this part
    step_cmp_node<Q, T, MODE, DIN, IN, OUT, INL>(src, dst, k, c, Ip, tmpl, omega);
}

// Grid-stride form of the stream-collide step from a natural state (the
// two-buffer pull, OUT own, or the in-place gather step, OUT scatter): a
// thread walks the nodes k, k + stride, ... and loads the table entries of
// its next node before the populations of the current one, so the table
// latency of node k + stride overlaps the population loads of node k.  The
// nodes of a block stay in one kCmpThreads-aligned range per iteration, so
// its instance is uniform across the block (padding nodes of a batch run
// like any node, see k_step_cmp).  The Eq. 6 update is inlined (an
// out-of-line call inside the loop makes the register allocator spill the
// loop's state).  Compact indices fit in 32 bits (checked when the tables
// are built).
template <int Q, typename T, int MINB, int OUT>
__global__ void __launch_bounds__(kCmpThreads, MINB)
    k_step_cmp_gs(const T* __restrict__ src, T* __restrict__ dst, Cmp c, const BCmpInst* __restrict__ insts,
                  const int* __restrict__ blk_inst, Bc tmpl, const double* __restrict__ tau)
{
    pdl_enter();
    const int nf = (int)c.nf, stride = (int)(gridDim.x * blockDim.x);
    int k = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    int32_t nxt[Q];
    bool bnd_next = k < nf ? load_codes<Q>(nxt, c, k) : false;
    int cur = -1;
    T omega = T(0);
    for (; k < nf; k += stride) {
        const bool bnd = bnd_next;
        T v[Q];
        int32_t code[Q];
        if (!bnd) pull_interior<Q, T, kInGather>(v, src, k, (size_t)c.nf, nxt);  // population loads first
        if (OUT == kOutScatter) {
#pragma unroll
            for (int d = 0; d < Q; ++d) code[d] = nxt[d];
        }
        if (k + stride < nf) bnd_next = load_codes<Q>(nxt, c, k + stride);  // then the next node's table
        const int i = block_instance(blk_inst, k);
        if (i != cur) {
            cur = i;
            omega = T(1) / T(tau[i]);
        }
        if (bnd) {
            step_node_eq6_inline<Q, T, kStreamCollide, kInGather, OUT>(src, dst, k, c, insts + i, tmpl, omega);
            continue;
        }
        collide_any<Q, T>(v, omega, tmpl);
        store_node<Q, T, OUT>(dst, v, k, c, insts->g, code);
    }
}

// One adjoint step; the warp partials of an instance occupy slots
// [k0 / 32, (k0 + nf + 31) / 32).  Padding nodes of a batch (see k_step_cmp;
// lambda's padding starts at zero too) stay zero and add exactly 0 to the
// dL/domega sum.  lam_in == lam_out is allowed for the in-place pairs (as
// for k_step_cmp: disjoint slot sets, all loads of a node before its stores).
template <int Q, typename T, bool T0, int IN, int OUT>
__global__ void __launch_bounds__(kCmpThreads, 4)
    k_adjoint_cmp(const T* __restrict__ gprev, const T* __restrict__ lam_in, T* __restrict__ lam_out, Cmp c,
                  const BCmpInst* __restrict__ insts,
                  const int* __restrict__ blk_inst, Bc tmpl, const double* __restrict__ tau,
                  double* __restrict__ grad_acc, double* __restrict__ partial)
{
    pdl_enter();
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T dom = T(0);
    if (k < c.nf) {
        const int i = block_instance(blk_inst, k);
        const T omega = T(1) / T(tau[i]);  // in T: FP64 arithmetic is slow on this part
        dom = adjoint_cmp_node<Q, T, T0, IN, OUT>(gprev, lam_in, lam_out, k, c, insts + i, tmpl, omega, grad_acc);
    }
    add_warp_partial<T>(dom, k < c.nf, k, partial);
}

// The caller's dense arrays (packed, for a batch) -> the compact state
// (ADD: added to it).  SWAP: into the swapped lambda layout (lambda_d(x) to
// (x - c_d, opp(d)) where that node is fluid), the layout of lambda^t at odd
// t in the in-place reverse sweep.
template <int Q, typename T, bool ADD, bool SWAP>
__global__ void __launch_bounds__(kCmpThreads)
    k_cmp_gather(const T* __restrict__ dense, T* __restrict__ cmp, Cmp c, const BCmpInst* __restrict__ insts,
                 const int* __restrict__ blk_inst)
{
    using L = Lattice<Q>;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const BCmpInst I = insts[block_instance(blk_inst, k)];
    if (k >= I.k0 + I.nf) return;
    const long long n = c.idx[k];
    for (int d = 0; d < Q; ++d) {
        const T v = dense[I.f_off + (long long)d * I.g.N + n];
        long long slot = (long long)d * c.nf + k;
        if (SWAP && d > 0) {
            const int32_t co = c.nbr[(long long)(d - 1) * c.nf + k];
            if (co >= 0) slot = (long long)L::opp(d) * c.nf + co;
        }
        if (ADD) cmp[slot] += v;
        else cmp[slot] = v;
    }
}

// One instance's tables (built by compact_build) into the packed arrays:
// dense indices as they are, neighbour codes shifted by the instance's k0.
__global__ void __launch_bounds__(256) k_bpack_cmp(const int32_t* __restrict__ idx_l, const int32_t* __restrict__ nbr_l,
                                                   long long nf, int q, long long k0, long long nfp,
                                                   int32_t* __restrict__ idx, int32_t* __restrict__ nbr)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    idx[k0 + k] = idx_l[k];
    for (int d = 0; d < q - 1; ++d) {
        const int32_t code = nbr_l[(long long)d * nf + k];
        nbr[(long long)d * nfp + k0 + k] = code >= 0 ? (int32_t)(code + k0) : code;
    }
}

unsigned cmp_grid(long long nf) { return (unsigned)((nf + kCmpThreads - 1) / kCmpThreads); }

// The launch of a single lattice: a pack of one (no block table).
BCmpArgs single_args(const PlanInfo& p, uint32_t* status)
{
    BCmpArgs a = {};
    a.c = p.cmp;
    a.insts = p.cmp_inst;
    a.blk_inst = nullptr;
    a.n_blocks = cmp_grid(p.cmp.nf);
    a.q = p.q;
    a.prec = p.prec;
    a.pdl = p.pdl;
    a.status = status;
    return a;
}

// The sweeps use: stream-collide compact -> compact (two-buffer pull
// natural -> natural, or the in-place pair natural -> swapped, swapped ->
// natural); collide-only from a dense or compact state into compact;
// stream-only into compact or into the caller's dense array, from either
// layout.
template <int Q, typename T>
void launch_step(const BCmpArgs& a, int mode, const void* src, void* dst, bool din, bool dout, int lin, int lout,
                 const Bc& tmpl, const double* tau, cudaStream_t s)
{
    const T* x = static_cast<const T*>(src);
    T* y = static_cast<T*>(dst);
    const dim3 grid(a.n_blocks), block(kCmpThreads);
    const bool swap_in = lin == kLayoutSwapped, swap_out = lout == kLayoutSwapped;
    if (mode == kStreamCollide) {
        if (swap_in) {  // the local step: no table for interior nodes
            launch_k(a.pdl, k_step_cmp<Q, T, kStreamCollide, false, kInLocal, kOutOwn, true>, grid, block, 0, s, x, y,
                     a.c, a.insts, a.blk_inst, tmpl, tau);
            return;
        }
        // D2Q9 FP32: the grid-stride form with table prefetch (measured faster);
        // D3Q19 and FP64 keep one node per thread (the prefetched table spills)
        if constexpr (Q == 9 && std::is_same<T, float>::value) {
            if (swap_out) {
                static const unsigned resident = resident_ctas(k_step_cmp_gs<Q, T, 3, kOutScatter>);
                launch_k(a.pdl, k_step_cmp_gs<Q, T, 3, kOutScatter>, dim3(std::min<unsigned>(resident, grid.x)), block,
                         0, s, x, y, a.c, a.insts, a.blk_inst, tmpl, tau);
            } else {
                static const unsigned resident = resident_ctas(k_step_cmp_gs<Q, T, 3, kOutOwn>);
                launch_k(a.pdl, k_step_cmp_gs<Q, T, 3, kOutOwn>, dim3(std::min<unsigned>(resident, grid.x)), block, 0,
                         s, x, y, a.c, a.insts, a.blk_inst, tmpl, tau);
            }
            return;
        }
        if (swap_out) {
            launch_k(a.pdl, k_step_cmp<Q, T, kStreamCollide, false, kInGather, kOutScatter, true>, grid, block, 0, s,
                     x, y, a.c, a.insts, a.blk_inst, tmpl, tau);
        } else {
            launch_k(a.pdl, k_step_cmp<Q, T, kStreamCollide, false, kInGather, kOutOwn, true>, grid, block, 0, s, x,
                     y, a.c, a.insts, a.blk_inst, tmpl, tau);
        }
    } else if (mode == kCollideOnly && din) {
        launch_k(a.pdl, k_step_cmp<Q, T, kCollideOnly, true, kInGather, kOutOwn>, grid, block, 0, s, x, y, a.c,
                 a.insts, a.blk_inst, tmpl, tau);
    } else if (mode == kCollideOnly) {
        launch_k(a.pdl, k_step_cmp<Q, T, kCollideOnly, false, kInGather, kOutOwn>, grid, block, 0, s, x, y, a.c,
                 a.insts, a.blk_inst, tmpl, tau);
    } else if (dout && swap_in) {
        launch_k(a.pdl, k_step_cmp<Q, T, kStreamOnly, false, kInLocal, kOutDense>, grid, block, 0, s, x, y, a.c,
                 a.insts, a.blk_inst, tmpl, tau);
    } else if (dout) {
        launch_k(a.pdl, k_step_cmp<Q, T, kStreamOnly, false, kInGather, kOutDense>, grid, block, 0, s, x, y, a.c,
                 a.insts, a.blk_inst, tmpl, tau);
    } else {
        launch_k(a.pdl, k_step_cmp<Q, T, kStreamOnly, false, kInGather, kOutOwn>, grid, block, 0, s, x, y, a.c,
                 a.insts, a.blk_inst, tmpl, tau);
    }
}

template <int Q, typename T, int IN, int OUT>
void launch_adjoint_as(const BCmpArgs& a, int t0, const T* gp, const T* li, T* lo, const Bc& tmpl, const double* tau,
                       double* grad_acc, double* partial, cudaStream_t s)
{
    const dim3 grid(a.n_blocks), block(kCmpThreads);
    if (t0)
        launch_k(a.pdl, k_adjoint_cmp<Q, T, true, IN, OUT>, grid, block, 0, s, gp, li, lo, a.c, a.insts, a.blk_inst,
                 tmpl, tau, grad_acc, partial);
    else
        launch_k(a.pdl, k_adjoint_cmp<Q, T, false, IN, OUT>, grid, block, 0, s, gp, li, lo, a.c, a.insts, a.blk_inst,
                 tmpl, tau, grad_acc, partial);
}

// lin: the layout of g^{t-1} and lambda^{t+1} (the same in every sweep);
// lout: the layout of lambda^t.
template <int Q, typename T>
void launch_adjoint(const BCmpArgs& a, int t0, const void* gprev, const void* lam_in, void* lam_out, int lin,
                    int lout, const Bc& tmpl, const double* tau, double* grad_acc, double* partial, cudaStream_t s)
{
    const T* gp = static_cast<const T*>(gprev);
    const T* li = static_cast<const T*>(lam_in);
    T* lo = static_cast<T*>(lam_out);
    if (lin == kLayoutSwapped)
        launch_adjoint_as<Q, T, kInLocal, kOutOwn>(a, t0, gp, li, lo, tmpl, tau, grad_acc, partial, s);
    else if (lout == kLayoutSwapped)
        launch_adjoint_as<Q, T, kInGather, kOutScatter>(a, t0, gp, li, lo, tmpl, tau, grad_acc, partial, s);
    else
        launch_adjoint_as<Q, T, kInGather, kOutOwn>(a, t0, gp, li, lo, tmpl, tau, grad_acc, partial, s);
}

lbm_status step_any(const BCmpArgs& a, int mode, const void* src, void* dst, bool din, bool dout, const Bc& tmpl,
                    const double* tau, cudaStream_t s, int lin = kLayoutNatural, int lout = kLayoutNatural)
{
    if (a.n_blocks == 0) return LBM_OK;
    if (a.q == 9 && a.prec == 4) launch_step<9, float>(a, mode, src, dst, din, dout, lin, lout, tmpl, tau, s);
    else if (a.q == 9 && a.prec == 8) launch_step<9, double>(a, mode, src, dst, din, dout, lin, lout, tmpl, tau, s);
    else if (a.q == 19 && a.prec == 4) launch_step<19, float>(a, mode, src, dst, din, dout, lin, lout, tmpl, tau, s);
    else if (a.q == 19 && a.prec == 8) launch_step<19, double>(a, mode, src, dst, din, dout, lin, lout, tmpl, tau, s);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

lbm_status adjoint_any(const BCmpArgs& a, int t0, const void* gprev, const void* lam_in, void* lam_out,
                       const Bc& tmpl, const double* tau, double* grad_acc, double* partial, cudaStream_t s,
                       int lin = kLayoutNatural, int lout = kLayoutNatural)
{
    if (a.n_blocks == 0) return LBM_OK;
    if (a.q == 9 && a.prec == 4)
        launch_adjoint<9, float>(a, t0, gprev, lam_in, lam_out, lin, lout, tmpl, tau, grad_acc, partial, s);
    else if (a.q == 9 && a.prec == 8)
        launch_adjoint<9, double>(a, t0, gprev, lam_in, lam_out, lin, lout, tmpl, tau, grad_acc, partial, s);
    else if (a.q == 19 && a.prec == 4)
        launch_adjoint<19, float>(a, t0, gprev, lam_in, lam_out, lin, lout, tmpl, tau, grad_acc, partial, s);
    else if (a.q == 19 && a.prec == 8)
        launch_adjoint<19, double>(a, t0, gprev, lam_in, lam_out, lin, lout, tmpl, tau, grad_acc, partial, s);
    else return LBM_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

template <int Q, typename T>
void launch_gather(const BCmpArgs& a, const void* dense, void* compact, bool add, bool swap, cudaStream_t s)
{
    const dim3 grid(a.n_blocks), block(kCmpThreads);
    const T* d = static_cast<const T*>(dense);
    T* c = static_cast<T*>(compact);
    if (add && swap) k_cmp_gather<Q, T, true, true><<<grid, block, 0, s>>>(d, c, a.c, a.insts, a.blk_inst);
    else if (add) k_cmp_gather<Q, T, true, false><<<grid, block, 0, s>>>(d, c, a.c, a.insts, a.blk_inst);
    else if (swap) k_cmp_gather<Q, T, false, true><<<grid, block, 0, s>>>(d, c, a.c, a.insts, a.blk_inst);
    else k_cmp_gather<Q, T, false, false><<<grid, block, 0, s>>>(d, c, a.c, a.insts, a.blk_inst);
}

lbm_status gather_any(const BCmpArgs& a, const void* dense, void* compact, cudaStream_t s, bool add = false,
                      int layout = kLayoutNatural)
{
    if (a.n_blocks == 0) return LBM_OK;
    const bool swap = layout == kLayoutSwapped;
    if (a.q == 9 && a.prec == 4) launch_gather<9, float>(a, dense, compact, add, swap, s);
    else if (a.q == 9) launch_gather<9, double>(a, dense, compact, add, swap, s);
    else if (a.prec == 4) launch_gather<19, float>(a, dense, compact, add, swap, s);
    else launch_gather<19, double>(a, dense, compact, add, swap, s);
    return cuda_status(cudaGetLastError());
}

// The call's options on a batch: node-velocity Eq. 6 and BGK.
Bc batch_tmpl(const double* rho_in, double rho_out, uint32_t* status)
{
    Bc bc;
    bc.rho_in = rho_in;
    bc.profile = 0;
    bc.rho_out = rho_out;
    bc.status = status;
    return bc;
}

}  // namespace

size_t compact_table_bytes(const PlanInfo& p, long long nf) { return table_layout(p, nf).bytes; }

lbm_status compact_build(const PlanInfo& p, long long nf, void* tables, Cmp* out, const int32_t** cmap_out,
                         const BCmpInst** inst_out, cudaStream_t s)
{
    const TableLayout t = table_layout(p, nf);
    unsigned char* base = static_cast<unsigned char*>(tables);
    BCmpInst* inst = reinterpret_cast<BCmpInst*>(base + t.inst);
    int32_t* idx = reinterpret_cast<int32_t*>(base + t.idx);
    int32_t* nbr = reinterpret_cast<int32_t*>(base + t.nbr);
    uint32_t* eq6 = reinterpret_cast<uint32_t*>(base + t.eq6);
    int32_t* cmap = reinterpret_cast<int32_t*>(base + t.cmap);
    int* blk = reinterpret_cast<int*>(base + t.blk);
    long long* total = reinterpret_cast<long long*>(base + t.total_slot);
    const long long N = p.geo.N;
    const long long nblk = (N + kScanNodes - 1) / kScanNodes;
    BCmpInst one = {};
    one.g = p.geo;
    one.k0 = 0;
    one.nf = nf;
    one.f_off = 0;
    one.in_off = 0;
    one.acc_off = 0;
    one.n_in = p.n_in;
    if (cudaMemcpyAsync(inst, &one, sizeof(one), cudaMemcpyHostToDevice, s) != cudaSuccess) return LBM_ERR_CUDA;
    // interior nodes, then the boundary columns (index kernels guard against counts above nf)
    const int nx = p.geo.nx;
    for (int cls = 0; cls < 2; ++cls) {
        k_cmp_count<<<(unsigned)nblk, 256, 0, s>>>(p.geo.link, N, nx, cls, blk);
        k_cmp_scan<<<1, 1024, 0, s>>>(blk, nblk, total + cls);
        k_cmp_index<<<(unsigned)nblk, 256, 0, s>>>(p.geo.link, N, nx, cls, total, blk, cmap, idx, nf);
    }
    long long got[2] = {-1, -1};
    if (cudaMemcpyAsync(got, total, sizeof(got), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;  // also ends the copy of `one`
    if (got[0] + got[1] != nf) return LBM_ERR_INVALID_ARG;
    if (nf > 0) {
        const unsigned g = cmp_grid(nf);
        if (p.q == 9) k_cmp_nbr<9><<<g, 256, 0, s>>>(p.geo.link, cmap, idx, nbr, nf, p.geo);
        else k_cmp_nbr<19><<<g, 256, 0, s>>>(p.geo.link, cmap, idx, nbr, nf, p.geo);
        if (p.q == 9) k_cmp_eq6_bits<9><<<g, 256, 0, s>>>(nbr, nf, eq6);
        else k_cmp_eq6_bits<19><<<g, 256, 0, s>>>(nbr, nf, eq6);
    }
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    out->nf = nf;
    out->idx = idx;
    out->nbr = nbr;
    out->eq6 = eq6;
    *cmap_out = cmap;
    if (inst_out) *inst_out = inst;
    return LBM_OK;
}

lbm_status step_launch_cmp(const PlanInfo& p, int mode, const void* src, void* dst, bool dense_in, bool dense_out,
                           const Bc& bc, const double* tau, cudaStream_t s, int lin, int lout)
{
    if (p.cmp.nf == 0) return LBM_OK;
    return step_any(single_args(p, bc.status), mode, src, dst, dense_in, dense_out, bc, tau, s, lin, lout);
}

lbm_status adjoint_launch_cmp(const PlanInfo& p, int t0, const void* gprev, const void* lam_in, void* lam_out,
                              const Bc& bc, const double* tau, double* grad_acc, double* partial, cudaStream_t s,
                              int lin, int lout)
{
    if (p.cmp.nf == 0) return LBM_OK;
    LBM_CMP_TRY(adjoint_any(single_args(p, bc.status), t0, gprev, lam_in, lam_out, bc, tau, grad_acc, partial, s,
                            lin, lout));
    if (bc.uw_extrap && !t0) {  // at t = 0 the fluid is at rest and the pass adds nothing
        // (two-buffer pull only: the in-place schedule refuses the extrapolated velocity)
        const long long rows = (long long)p.geo.ny * p.geo.nz;
        const dim3 grid((unsigned)((rows + kCmpThreads - 1) / kCmpThreads)), block(kCmpThreads);
        if (p.q == 9 && p.prec == 4)
            launch_k(p.pdl, k_adjoint_uw_cmp<9, float>, grid, block, 0, s, static_cast<const float*>(gprev),
                     static_cast<const float*>(lam_in), static_cast<float*>(lam_out), p.cmp, p.cmp_map, p.geo, bc,
                     grad_acc);
        else if (p.q == 9)
            launch_k(p.pdl, k_adjoint_uw_cmp<9, double>, grid, block, 0, s, static_cast<const double*>(gprev),
                     static_cast<const double*>(lam_in), static_cast<double*>(lam_out), p.cmp, p.cmp_map, p.geo, bc,
                     grad_acc);
        else if (p.prec == 4)
            launch_k(p.pdl, k_adjoint_uw_cmp<19, float>, grid, block, 0, s, static_cast<const float*>(gprev),
                     static_cast<const float*>(lam_in), static_cast<float*>(lam_out), p.cmp, p.cmp_map, p.geo, bc,
                     grad_acc);
        else
            launch_k(p.pdl, k_adjoint_uw_cmp<19, double>, grid, block, 0, s, static_cast<const double*>(gprev),
                     static_cast<const double*>(lam_in), static_cast<double*>(lam_out), p.cmp, p.cmp_map, p.geo, bc,
                     grad_acc);
    }
    return cuda_status(cudaGetLastError());
}

lbm_status compact_gather_launch(const PlanInfo& p, const void* dense, void* compact, cudaStream_t s, int layout)
{
    if (p.cmp.nf == 0) return LBM_OK;
    return gather_any(single_args(p, nullptr), dense, compact, s, false, layout);
}

lbm_status compact_gather_add_launch(const PlanInfo& p, const void* dense, void* compact, cudaStream_t s, int layout)
{
    if (p.cmp.nf == 0) return LBM_OK;
    return gather_any(single_args(p, nullptr), dense, compact, s, true, layout);
}

lbm_status bstep_launch_cmp(const BCmpArgs& a, int mode, const void* src, void* dst, bool dense_out,
                            const double* rho_in, const double* tau, double rho_out, cudaStream_t s)
{
    return step_any(a, mode, src, dst, false, dense_out, batch_tmpl(rho_in, rho_out, a.status), tau, s);
}

lbm_status badjoint_launch_cmp(const BCmpArgs& a, int t0, const void* gprev, const void* lam_in, void* lam_out,
                               const double* rho_in, const double* tau, double rho_out, double* grad_acc,
                               double* partial, cudaStream_t s)
{
    return adjoint_any(a, t0, gprev, lam_in, lam_out, batch_tmpl(rho_in, rho_out, a.status), tau, grad_acc, partial,
                       s);
}

lbm_status bgather_launch_cmp(const BCmpArgs& a, const void* dense, void* compact, cudaStream_t s)
{
    return gather_any(a, dense, compact, s);
}

lbm_status eq6_bits_launch_cmp(int q, const int32_t* nbr, long long nf, uint32_t* bits, cudaStream_t s)
{
    if (nf == 0) return LBM_OK;
    if (q == 9) k_cmp_eq6_bits<9><<<cmp_grid(nf), 256, 0, s>>>(nbr, nf, bits);
    else k_cmp_eq6_bits<19><<<cmp_grid(nf), 256, 0, s>>>(nbr, nf, bits);
    return cuda_status(cudaGetLastError());
}

lbm_status bpack_launch_cmp(const Cmp& local, int q, long long k0, long long nfp, int32_t* idx, int32_t* nbr,
                            cudaStream_t s)
{
    if (local.nf == 0) return LBM_OK;
    k_bpack_cmp<<<(unsigned)((local.nf + 255) / 256), 256, 0, s>>>(local.idx, local.nbr, local.nf, q, k0, nfp, idx, nbr);
    return cuda_status(cudaGetLastError());
}

}  // namespace lbm
