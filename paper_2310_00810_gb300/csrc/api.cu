// The C ABI (include/lbm.h): plans, workspace layout, and the orchestration
// of the forward sweep, the sqrt(T) checkpointed reverse sweep, the loss and
// the post-processing calls.  Everything that touches lattice data runs in
// this library's CUDA kernels; the host only sequences launches.
//
// Time indexing.  The paper's state f^t (pre-collision) evolves as
// f^{t+1} = S(C(f^t)) from f^0 = rest.  The kernels store g^t = C(f^t), so
//   g^0 = rest (collision leaves the rest state unchanged),
//   g^t = C(S(g^{t-1}))  for t = 1..T-1  (stream-collide launches),
//   f^T = S(g^{T-1})                      (stream-only launch).
// The adjoint step for time t needs f^t = S(g^{t-1}) (or the rest state at
// t = 0).  With stride k and S = ceil(T / k) segments, segment s covers
// t in [s k, min((s+1) k, T)); its base is g^{s k - 1}, which the forward
// sweep writes straight into checkpoint slot s (s = 1..S-1) instead of a
// ping-pong buffer, so checkpointing costs no extra traffic.  The reverse
// sweep recomputes g^{s k} .. g^{s k + len - 2} into the segment buffer and
// then runs the adjoint steps of the segment backwards.
//
// Launch sequences.  A forward or reverse sweep is T to 3T kernel launches;
// on a stream other than the legacy default stream the part of the sequence
// that touches only the workspace and the geometry is captured once into a
// CUDA graph and replayed with one cudaGraphLaunch.  The graph does not
// depend on the caller's arrays: every call first copies its rho_in and tau
// into the workspace (and the reverse sweep its lambda^T), and the launches
// that write the caller's outputs (the final stream-only launch, the gradient
// finalisation) run after the graph, outside it.  So a caller that passes
// fresh tensors on every call still replays the same graph; only a new
// workspace, geometry or rho_out (or a kernel choice) captures a new one.
// When the caller's stream is itself being captured, the launches go
// straight into the caller's graph.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "common.cuh"

using namespace lbm;

namespace {

struct GraphKey {
    int op = 0;
    const void* ptr[8] = {};
    double scalar = 0.0;
    long long n = 0;
    bool operator==(const GraphKey& o) const
    {
        return op == o.op && scalar == o.scalar && n == o.n && std::memcmp(ptr, o.ptr, sizeof(ptr)) == 0;
    }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
};

constexpr size_t kMaxGraphs = 8;

}  // namespace

struct lbm_plan {
    lbm_desc desc;
    PlanInfo info;
    int k;      // checkpoint stride
    int S;      // segments
    Workspace ws;
    uint8_t* mask = nullptr;
    uint32_t* link = nullptr;
    size_t dense_state_bytes = 0;  // Q N precision: the caller's state arrays
    int dense_n_partial = 0;       // FP64 partial slots of the dense kernels
    void* last_ws = nullptr;
    int fwd_aa = -1;               // schedule of the last lbm_forward (1: in place): its checkpoints' layouts
    bool use_graphs = true;
    std::vector<GraphEntry> graphs;  // most recently used last
    // second stream and events of the overlapped reverse sweep (created on first use)
    cudaStream_t helper = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // fork, join, recompute done, adjoint done
    ~lbm_plan()
    {
        for (auto& g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (helper) cudaStreamDestroy(helper);
    }
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The in-place (AA-pattern) schedule runs where it is chosen and the plan
// is in the fluid-only layout.
bool in_place(const lbm_plan* p) { return p->info.aa && p->info.cmp.nf; }

void layout(lbm_plan* p)
{
    const size_t st = align256(p->info.state_bytes);
    Workspace& w = p->ws;
    size_t o = 0;
    w.status = o;
    o += 256;
    w.call = o;
    o += align256(sizeof(double) * (size_t)(p->info.n_in + 1));
    w.grad_acc = o;
    o += align256(sizeof(double) * (size_t)p->info.n_acc);
    w.partial = o;
    o += align256(sizeof(double) * (size_t)p->info.n_partial);
    w.partial2 = o;
    o += align256(sizeof(double) * (size_t)p->info.n_blocks);
    w.side = o;
    o += align256((size_t)p->info.prec * 3 * 2 * (size_t)p->info.n_acc);
    w.ping[0] = o;
    o += st;
    w.lam[1] = o;
    o += st;
    w.ckpt = o;
    o += st * (size_t)(p->S - 1);
    w.seg = o;
    o += st * (size_t)p->k * 2;
    // the second forward and adjoint buffers last: the in-place schedule has none
    const bool one = in_place(p);
    w.ping[1] = o;
    o += one ? 0 : st;
    w.lam[0] = o;
    o += one ? 0 : st;
    w.total = o;
}

bool aligned256(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 255u) == 0; }

unsigned char* bytes(void* ws) { return static_cast<unsigned char*>(ws); }

// The MRT rates and the inlet velocity into the status section, where the
// kernels read them (Bc::mrt, Bc::vel_inlet).
struct CallParams {
    double rates[3], u_in[3];
};

__global__ void k_write_call_params(uint32_t* status, CallParams c)
{
    unsigned char* b = reinterpret_cast<unsigned char*>(status);
    double* r = reinterpret_cast<double*>(b + kMrtRates);
    double* u = reinterpret_cast<double*>(b + kInletVelocity);
    for (int i = 0; i < 3; ++i) {
        r[i] = c.rates[i];
        u[i] = c.u_in[i];
    }
}

lbm_status write_mrt_rates(const lbm_plan* p, const Bc& bc, cudaStream_t s)
{
    if (!p->info.mrt && !p->info.vel_inlet) return LBM_OK;
    CallParams c;
    for (int i = 0; i < 3; ++i) {
        c.rates[i] = p->info.mrt_rates[i];
        c.u_in[i] = p->info.u_in[i];
    }
    k_write_call_params<<<1, 1, 0, s>>>(bc.status, c);
    return cuda_status(cudaGetLastError());
}

// The periodic-y and velocity-inlet options exist in the fluid-only layout
// only; the in-place schedule keeps no neighbour velocity for the
// extrapolated Eq. 6 velocity.
lbm_status check_layout_options(const lbm_plan* p)
{
    if ((p->info.geo.periodic_y || p->info.vel_inlet) && !p->info.cmp.nf) return LBM_ERR_UNSUPPORTED;
    if (in_place(p) && p->info.uw_extrap) return LBM_ERR_UNSUPPORTED;
    return LBM_OK;
}

Bc make_bc(const lbm_plan* p, const double* rho_in, double rho_out, void* ws)
{
    Bc bc;
    bc.rho_in = rho_in;
    bc.profile = p->info.n_in > 1 ? 1 : 0;
    bc.rho_out = rho_out;
    bc.status = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ws) + p->ws.status);
    bc.uw_extrap = p->info.uw_extrap;
    bc.mrt = p->info.mrt;
    bc.vel_inlet = p->info.vel_inlet;
    bc.wait_us = p->info.wait_us;
    bc.test_stall = p->info.test_stall ? 1 : 0;
    bc.ramp_steps = p->info.vel_inlet ? p->info.ramp_steps : 0;
    return bc;
}

// Copies this call's rho_in and tau into the workspace (stream-ordered), where
// the sweep kernels read them; returns the staged pointers.
lbm_status stage_inputs(const lbm_plan* p, void* d_ws, const double* d_rho_in, const double* d_tau,
                        const double** rho_in, const double** tau, cudaStream_t s)
{
    double* r = reinterpret_cast<double*>(static_cast<unsigned char*>(d_ws) + p->ws.call);
    double* t = r + p->info.n_in;
    if (cudaMemcpyAsync(r, d_rho_in, sizeof(double) * (size_t)p->info.n_in, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(t, d_tau, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    *rho_in = r;
    *tau = t;
    return LBM_OK;
}

PersistArgs persist_args(const lbm_plan* p, void* d_ws)
{
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    PersistArgs a;
    a.ping[0] = ws + p->ws.ping[0];
    a.ping[1] = ws + p->ws.ping[1];
    a.ckpt = ws + p->ws.ckpt;
    a.seg = ws + p->ws.seg;
    a.lam[0] = ws + p->ws.lam[0];
    a.lam[1] = ws + p->ws.lam[1];
    a.lam_in = nullptr;
    a.out = nullptr;
    a.state_stride = align256(p->info.state_bytes);
    a.T = p->desc.n_steps;
    a.k = p->k;
    a.S = p->S;
    a.spin_limit = p->info.spin_limit;
    a.bar = reinterpret_cast<PersistBar*>(ws + p->ws.status + kBarOffset);
    return a;
}

lbm_status check_common(const lbm_plan* p, const void* ws)
{
    if (!p) return LBM_ERR_INVALID_ARG;
    if (!p->link) return LBM_ERR_INVALID_ARG;  // no geometry bound yet
    if (ws && !aligned256(ws)) return LBM_ERR_INVALID_ARG;
    return LBM_OK;
}

void drop_graphs(lbm_plan* p)
{
    for (auto& g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
}

// Back to the dense layout (a new geometry invalidates the compact tables).
void set_dense(lbm_plan* p)
{
    p->info.cmp = Cmp{0, nullptr, nullptr};
    p->info.cmp_map = nullptr;
    p->info.cmp_inst = nullptr;
    p->info.state_bytes = p->dense_state_bytes;
    p->info.n_partial = p->dense_n_partial;
    layout(p);
    drop_graphs(p);
}

#define LBM_TRY(expr)                     \
    do {                                  \
        lbm_status st__ = (expr);         \
        if (st__ != LBM_OK) return st__;  \
    } while (0)

// The last launch of a sweep: stream-only from the internal state cur into
// the caller's dense array.  Solid nodes are zeroed first: the compact layout
// writes fluid nodes only, and the dense kernels skip 32-byte sectors that
// hold only solid nodes.
lbm_status final_stream(const lbm_plan* p, const void* cur, void* d_f, const Bc& bc, const double* tau,
                        cudaStream_t s, int lin = kLayoutNatural)
{
    if (cudaMemsetAsync(d_f, 0, p->dense_state_bytes, s) != cudaSuccess) return LBM_ERR_CUDA;
    if (!p->info.cmp.nf) return step_launch(p->info, kStreamOnly, cur, d_f, bc, tau, s);
    return step_launch_cmp(p->info, kStreamOnly, cur, d_f, false, true, bc, tau, s, lin);
}

// One stream-collide launch of a sweep producing g^t from g^{t-1}: the
// plan's kernels (or those of info, the recompute's choice), or the in-place
// pair (src and dst may be one buffer).
lbm_status sweep_step(const lbm_plan* p, const void* src, void* dst, const Bc& bc, int t, const double* tau,
                      cudaStream_t s, const PlanInfo* info = nullptr)
{
    if (!in_place(p)) return step_launch(info ? *info : p->info, kStreamCollide, src, dst, at_time(bc, t), tau, s);
    return step_launch_cmp(p->info, kStreamCollide, src, dst, false, false, at_time(bc, t), tau, s,
                           layout_at(true, t - 1), layout_at(true, t));
}

// Issues `issue(s)` through a cached CUDA graph when that is possible.
lbm_status run_sequence(lbm_plan* p, const GraphKey& key, cudaStream_t s,
                        const std::function<lbm_status(cudaStream_t)>& issue)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!p->use_graphs || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return issue(s);
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return LBM_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return issue(s);
    for (size_t i = 0; i < p->graphs.size(); ++i)
        if (p->graphs[i].key == key) {
            GraphEntry e = p->graphs[i];
            p->graphs.erase(p->graphs.begin() + (long)i);
            p->graphs.push_back(e);
            return cuda_status(cudaGraphLaunch(e.exec, s));
        }
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
    lbm_status st = issue(s);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != LBM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != LBM_OK ? st : LBM_ERR_CUDA;
    }
    GraphEntry ent;
    ent.key = key;
    e = cudaGraphInstantiate(&ent.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (p->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back(ent);
    return cuda_status(cudaGraphLaunch(ent.exec, s));
}

}  // namespace

extern "C" {

lbm_status lbm_plan_create(const lbm_desc* d, lbm_plan** out)
{
    if (!d || !out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (d->q != 9 && d->q != 19) return LBM_ERR_INVALID_ARG;
    if (d->precision != 4 && d->precision != 8) return LBM_ERR_INVALID_ARG;
    if (d->nx < 2 || d->ny < 1 || d->nz < 1) return LBM_ERR_INVALID_ARG;
    if (d->ny > 65535 || d->nz > 65535) return LBM_ERR_INVALID_ARG;  // grid.y = ny, grid.z = nz
    if (d->q == 9 && d->nz != 1) return LBM_ERR_INVALID_ARG;
    if (d->n_steps < 1 || d->ckpt_stride < 0) return LBM_ERR_INVALID_ARG;
    if (d->loss_kind != LBM_LOSS_VEC && d->loss_kind != LBM_LOSS_NORM) return LBM_ERR_INVALID_ARG;
    if (d->loss_norm != LBM_NORM_SUM && d->loss_norm != LBM_NORM_MEAN_FLUID) return LBM_ERR_INVALID_ARG;
    if (d->inlet_kind != LBM_INLET_CONST && d->inlet_kind != LBM_INLET_PROFILE) return LBM_ERR_INVALID_ARG;
    const long long N = (long long)d->nx * d->ny * d->nz;
    if (N > (1LL << 31) - 1) return LBM_ERR_INVALID_ARG;  // queue and disk scratch use 32-bit node ids
    lbm_plan* p = new (std::nothrow) lbm_plan();
    if (!p) return LBM_ERR_OOM;
    p->desc = *d;
    PlanInfo& I = p->info;
    I.q = d->q;
    I.d = d->q == 9 ? 2 : 3;
    I.prec = d->precision;
    I.geo.nx = d->nx;
    I.geo.ny = d->ny;
    I.geo.nz = d->nz;
    I.geo.N = N;
    I.geo.link = nullptr;
    I.grid = dim3((unsigned)((d->nx + kStepThreads - 1) / kStepThreads), (unsigned)d->ny, (unsigned)d->nz);
    I.n_blocks = (int)(I.grid.x * I.grid.y * I.grid.z);
    I.n_in = d->inlet_kind == LBM_INLET_PROFILE ? d->ny * d->nz : 1;
    I.n_acc = d->ny * d->nz;
    I.geo.link = nullptr;
    I.geo.skip_sectors = d->nx % 8 == 0 ? 1 : 0;
    I.n_partial = std::max(std::max(I.n_blocks, vec_blocks_max(I)), 1024);
    I.state_bytes = (size_t)d->q * (size_t)N * (size_t)d->precision;
    I.cmp = Cmp{0, nullptr, nullptr};
    p->dense_state_bytes = I.state_bytes;
    p->dense_n_partial = I.n_partial;
    const int T = d->n_steps;
    p->k = d->ckpt_stride > 0 ? std::min(d->ckpt_stride, T) : std::max(1, (int)std::ceil(std::sqrt((double)T)));
    p->S = (T + p->k - 1) / p->k;
    layout(p);
    const char* env = std::getenv("LBM_NO_GRAPHS");
    p->use_graphs = !(env && env[0] == '1');
    // LBM_KERNEL=scalar forces the one-node-per-thread kernels; LBM_VEC=n caps the nodes per thread
    const char* kern = std::getenv("LBM_KERNEL");
    const char* vec = std::getenv("LBM_VEC");
    I.max_vec = (kern && std::strcmp(kern, "scalar") == 0) ? 0 : (vec ? std::atoi(vec) : 4);
    // LBM_TMA=0 turns the TMA-staged kernels off; LBM_TMA_MIN_TILES sets the size from which they are used
    const char* tma = std::getenv("LBM_TMA");
    const char* tmin = std::getenv("LBM_TMA_MIN_TILES");
    I.use_tma = I.max_vec >= 2 && !(tma && tma[0] == '0');
    I.tma_min_tiles = tmin ? std::atoi(tmin) : 1;
    const char* sv = std::getenv("LBM_STEP_VARIANT");
    I.step_variant = sv ? std::atoi(sv) : 0;
    const char* tv = std::getenv("LBM_TMA_VARIANT");
    I.tma_variant = tv ? std::atoi(tv) : 1;
    // LBM_PERSIST=1 turns on the one-launch sweeps (off by default: on this part a grid barrier costs more than
    // a graph kernel boundary); LBM_PERSIST_MAX_MB sets the largest state they take
    const char* pd = std::getenv("LBM_PDL");
    I.pdl = !(pd && pd[0] == '0');
    const char* pe = std::getenv("LBM_PERSIST");
    const char* pm = std::getenv("LBM_PERSIST_MAX_MB");
    I.use_persist = I.max_vec >= 2 && pe && pe[0] == '1';
    const char* ov = std::getenv("LBM_OVERLAP");
    I.overlap = !(ov && ov[0] == '0');
    I.persist_max_bytes = (size_t)(pm ? std::atof(pm) : 24.0) * (1u << 20);
    // LBM_SPIN_LIMIT bounds each grid-barrier wait of the persistent sweeps (tests set it tiny to make
    // the wait give up on purpose and check that LBM_ERR_TIMEOUT comes back)
    const char* ty = std::getenv("LBM_TMA_ROWS");
    I.tma_ty = ty && std::atoi(ty) == 4 ? 4 : 8;
    const char* tw = std::getenv("LBM_TMA_WAVES");
    I.tma_waves = tw ? std::max(1, std::atoi(tw)) : 1;
    I.adj_tma_ty = I.tma_ty;
    I.step_family = LBM_FAMILY_AUTO;
    I.adj_family = LBM_FAMILY_AUTO;
    I.rec_family = LBM_FAMILY_AUTO;
    const char* sl = std::getenv("LBM_SPIN_LIMIT");
    I.spin_limit = sl ? (unsigned)std::strtoul(sl, nullptr, 10) : (1u << 24);
    // LBM_WAIT_US bounds each mbarrier wait of the TMA kernels in time (default 2 s; tests set it tiny)
    const char* wu = std::getenv("LBM_WAIT_US");
    I.wait_us = wu ? (unsigned)std::strtoul(wu, nullptr, 10) : 2000000u;
    // LBM_TEST_STALL_TMA=1 makes the TMA producers issue no copies: a wait that nothing completes, for the
    // failure-path test of the bounded waits (no fault: the consumers give up after LBM_WAIT_US)
    const char* ts = std::getenv("LBM_TEST_STALL_TMA");
    I.test_stall = ts && ts[0] == '1';
    *out = p;
    return LBM_OK;
}

lbm_status lbm_plan_destroy(lbm_plan* p)
{
    delete p;
    return LBM_OK;
}

lbm_status lbm_plan_set_kernels(lbm_plan* p, const lbm_kernel_choice* k)
{
    if (!p || !k) return LBM_ERR_INVALID_ARG;
    auto fam_ok = [](int f) { return f >= LBM_FAMILY_AUTO && f <= LBM_FAMILY_TMA; };
    if (!fam_ok(k->step_family) || !fam_ok(k->adjoint_family) || (k->vec != 2 && k->vec != 4) ||
        (k->tma_rows != 4 && k->tma_rows != 8) || (k->pdl != 0 && k->pdl != 1) || (k->persist != 0 && k->persist != 1) ||
        (k->overlap != 0 && k->overlap != 1) ||
        (k->adjoint_tma_rows != 0 && k->adjoint_tma_rows != 4 && k->adjoint_tma_rows != 8) ||
        k->steps_per_launch < 0 || k->steps_per_launch > 2 || (k->aa != 0 && k->aa != 1) ||
        !fam_ok(k->recompute_family))
        return LBM_ERR_INVALID_ARG;
    PlanInfo& I = p->info;
    I.step_family = k->step_family;
    I.adj_family = k->adjoint_family;
    I.rec_family = k->recompute_family;
    I.max_vec = k->vec;
    I.use_tma = 1;
    I.tma_min_tiles = 1;
    I.tma_ty = k->tma_rows;
    I.adj_tma_ty = k->adjoint_tma_rows ? k->adjoint_tma_rows : k->tma_rows;
    I.steps2 = k->steps_per_launch == 2 ? 1 : 0;
    I.pdl = k->pdl;
    I.use_persist = k->persist;
    I.overlap = k->overlap;
    I.aa = k->aa;
    layout(p);  // the in-place schedule needs one forward and one adjoint buffer
    drop_graphs(p);
    return LBM_OK;
}

lbm_status lbm_plan_get_kernels(const lbm_plan* p, lbm_kernel_choice* k)
{
    if (!p || !k) return LBM_ERR_INVALID_ARG;
    const PlanInfo& I = p->info;
    k->step_family = I.step_family;
    k->adjoint_family = I.adj_family;
    k->recompute_family = I.rec_family;
    k->vec = I.max_vec >= 4 ? 4 : 2;
    k->tma_rows = I.tma_ty;
    k->adjoint_tma_rows = I.adj_tma_ty;
    k->steps_per_launch = I.steps2 ? 2 : 1;
    k->pdl = I.pdl;
    k->persist = I.use_persist;
    k->overlap = I.overlap;
    k->aa = I.aa;
    return LBM_OK;
}

lbm_status lbm_set_abb_velocity(lbm_plan* p, int32_t mode)
{
    if (!p || (mode != LBM_ABB_U_NODE && mode != LBM_ABB_U_EXTRAP)) return LBM_ERR_INVALID_ARG;
    p->info.uw_extrap = mode == LBM_ABB_U_EXTRAP ? 1 : 0;
    drop_graphs(p);
    return LBM_OK;
}

lbm_status lbm_get_abb_velocity(const lbm_plan* p, int32_t* mode)
{
    if (!p || !mode) return LBM_ERR_INVALID_ARG;
    *mode = p->info.uw_extrap ? LBM_ABB_U_EXTRAP : LBM_ABB_U_NODE;
    return LBM_OK;
}

lbm_status lbm_set_collision(lbm_plan* p, int32_t mode, double s_e, double s_eps, double s_q)
{
    if (!p || (mode != LBM_COLLISION_BGK && mode != LBM_COLLISION_MRT)) return LBM_ERR_INVALID_ARG;
    if (mode == LBM_COLLISION_MRT) {
        if (p->info.q != 9) return LBM_ERR_UNSUPPORTED;
        auto ok = [](double r) { return r > 0.0 && r < 2.0; };
        if (!ok(s_e) || !ok(s_eps) || !ok(s_q)) return LBM_ERR_INVALID_ARG;
        p->info.mrt_rates[0] = s_e;
        p->info.mrt_rates[1] = s_eps;
        p->info.mrt_rates[2] = s_q;
    }
    p->info.mrt = mode == LBM_COLLISION_MRT ? 1 : 0;
    drop_graphs(p);
    return LBM_OK;
}

lbm_status lbm_set_periodic_y(lbm_plan* p, int32_t on)
{
    if (!p || (on != 0 && on != 1) || p->link) return LBM_ERR_INVALID_ARG;
    p->info.geo.periodic_y = on;
    return LBM_OK;
}

lbm_status lbm_set_velocity_inlet(lbm_plan* p, int32_t on, double ux, double uy, double uz)
{
    if (!p || (on != 0 && on != 1) || !std::isfinite(ux) || !std::isfinite(uy) || !std::isfinite(uz))
        return LBM_ERR_INVALID_ARG;
    if (on && p->info.q == 9 && uz != 0.0) return LBM_ERR_INVALID_ARG;
    p->info.vel_inlet = on;
    p->info.u_in[0] = on ? ux : 0.0;
    p->info.u_in[1] = on ? uy : 0.0;
    p->info.u_in[2] = on ? uz : 0.0;
    drop_graphs(p);
    return LBM_OK;
}

lbm_status lbm_set_velocity_ramp(lbm_plan* p, int32_t steps)
{
    if (!p || steps < 0) return LBM_ERR_INVALID_ARG;
    p->info.ramp_steps = steps;
    drop_graphs(p);
    return LBM_OK;
}

lbm_status lbm_get_collision(const lbm_plan* p, int32_t* mode, double* rates)
{
    if (!p || !mode) return LBM_ERR_INVALID_ARG;
    *mode = p->info.mrt ? LBM_COLLISION_MRT : LBM_COLLISION_BGK;
    if (rates)
        for (int i = 0; i < 3; ++i) rates[i] = p->info.mrt ? p->info.mrt_rates[i] : 0.0;
    return LBM_OK;
}

lbm_status lbm_workspace_size(const lbm_plan* p, size_t* bytes_out)
{
    if (!p || !bytes_out) return LBM_ERR_INVALID_ARG;
    *bytes_out = p->ws.total;
    return LBM_OK;
}

lbm_status lbm_init_geometry(lbm_plan* p, const lbm_geom_desc* g, uint8_t* d_mask, uint32_t* d_link,
                             double* d_porosity, int64_t* d_info, void* stream)
{
    if (!p || !g || !d_mask || !d_link || !d_info) return LBM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_mask) & 3u) != 0) return LBM_ERR_INVALID_ARG;
    if (g->kind < LBM_GEOM_CHANNEL || g->kind > LBM_GEOM_MASK) return LBM_ERR_INVALID_ARG;
    if (g->kind == LBM_GEOM_DISKS && p->info.q != 9) return LBM_ERR_INVALID_ARG;
    if (g->kind == LBM_GEOM_SPHERES && p->info.q != 19) return LBM_ERR_INVALID_ARG;
    if (g->kind == LBM_GEOM_DISKS || g->kind == LBM_GEOM_SPHERES) {
        if (g->r_min < 0 || g->r_max < g->r_min || g->r_max > 4096) return LBM_ERR_INVALID_ARG;
        if (g->hydro_q8 < 0 || g->hydro_q8 > 256 || g->inlet_buffer < 1) return LBM_ERR_INVALID_ARG;
        if (g->max_rejections < 1 || !(g->target_porosity >= 0.0 && g->target_porosity <= 1.0))
            return LBM_ERR_INVALID_ARG;
        if ((long long)p->info.geo.nx * 256 > (1LL << 30)) return LBM_ERR_INVALID_ARG;
    }
    LBM_TRY(geometry_launch(p->info, *g, d_mask, d_link, d_porosity, d_info, static_cast<cudaStream_t>(stream)));
    p->mask = d_mask;
    p->link = d_link;
    p->info.geo.link = d_link;
    if (p->info.cmp.nf) set_dense(p);
    return LBM_OK;
}

lbm_status lbm_bind_geometry(lbm_plan* p, const uint32_t* d_link)
{
    if (!p || !d_link) return LBM_ERR_INVALID_ARG;
    p->link = const_cast<uint32_t*>(d_link);
    p->info.geo.link = d_link;
    if (p->info.cmp.nf) set_dense(p);
    return LBM_OK;
}

lbm_status lbm_compact_size(const lbm_plan* p, int64_t n_fluid, size_t* bytes_out)
{
    if (!p || !bytes_out || n_fluid < 0 || n_fluid > p->info.geo.N) return LBM_ERR_INVALID_ARG;
    *bytes_out = compact_table_bytes(p->info, n_fluid);
    return LBM_OK;
}

lbm_status lbm_compact_bind(lbm_plan* p, int64_t n_fluid, void* d_tables, void* stream)
{
    if (!p || !p->link || n_fluid < 0 || n_fluid > p->info.geo.N) return LBM_ERR_INVALID_ARG;
    if (n_fluid == 0) {
        set_dense(p);
        return LBM_OK;
    }
    if (!d_tables || !aligned256(d_tables)) return LBM_ERR_INVALID_ARG;
    Cmp c{0, nullptr, nullptr};
    const int32_t* cmap = nullptr;
    const BCmpInst* inst = nullptr;
    LBM_TRY(compact_build(p->info, n_fluid, d_tables, &c, &cmap, &inst, static_cast<cudaStream_t>(stream)));
    p->info.cmp = c;
    p->info.cmp_map = cmap;
    p->info.cmp_inst = inst;
    p->info.state_bytes = (size_t)p->info.q * (size_t)n_fluid * (size_t)p->info.prec;
    p->info.n_partial = std::max(p->dense_n_partial, (int)((n_fluid + 31) / 32));  // one slot per warp
    layout(p);
    drop_graphs(p);
    return LBM_OK;
}

lbm_status lbm_forward(lbm_plan* p, const double* d_rho_in, const double* d_tau, double rho_out, void* d_f,
                       void* d_ws, void* stream)
{
    LBM_TRY(check_common(p, d_ws));
    LBM_TRY(check_layout_options(p));
    if (!d_rho_in || !d_tau || !d_f || !d_ws) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = bytes(d_ws);
    p->last_ws = d_ws;
    const double* rho_in = nullptr;
    const double* tau = nullptr;
    LBM_TRY(stage_inputs(p, d_ws, d_rho_in, d_tau, &rho_in, &tau, s));
    const Bc bc = make_bc(p, rho_in, rho_out, d_ws);
    const int T = p->desc.n_steps, k = p->k, S = p->S;
    const size_t st = align256(p->info.state_bytes);
    auto slot = [&](int t) -> unsigned char* {  // checkpoint slot of g^t, or nullptr
        const int s1 = t + 1;
        if (s1 % k == 0 && s1 / k >= 1 && s1 / k <= S - 1) return ws + p->ws.ckpt + st * (size_t)(s1 / k - 1);
        return nullptr;
    };
    unsigned char* ping0 = ws + p->ws.ping[0];
    unsigned char* ping1 = ws + p->ws.ping[1];
    if (persist_ok(p->info)) {
        // one cooperative launch for the whole sweep; g^0 = rest where the sweep expects it
        PersistArgs a = persist_args(p, d_ws);
        a.out = d_f;
        unsigned char* g0 = slot(0) ? slot(0) : ping0;
        if (cudaMemsetAsync(g0, 0, p->info.state_bytes, s) != cudaSuccess) return LBM_ERR_CUDA;
        if (T == 1) return step_launch(p->info, kStreamOnly, g0, d_f, bc, tau, s);
        return forward_persist(p->info, a, bc, tau, s);
    }
    // the state chain g^0 .. g^{T-1}: checkpoint slots where the reverse sweep needs them, else ping-pong
    // (in place: ping0 alone, g^t in the layout of its parity); with two steps per launch, g^t of a pair is
    // written only where it is a checkpoint
    const bool one = in_place(p);
    p->fwd_aa = one ? 1 : 0;
    Bc bcs = bc;
    if (one) bcs.side_u = ws + p->ws.side;  // the Eq. 6 nodes' velocities, carried from step to step
    auto next_state = [&](int t, const unsigned char* cur) -> unsigned char* {
        unsigned char* dst = slot(t);
        return dst ? dst : (one ? ping0 : (cur == ping0 ? ping1 : ping0));
    };
    const bool pairs = !one && step2_possible(p->info, bc);
    // walks the chain, calling launch(src, two, mid, dst) once per launch: two steps (mid: g^t where it is a
    // checkpoint, else nullptr) or one
    using Launch = std::function<lbm_status(const unsigned char*, bool, unsigned char*, unsigned char*, int)>;
    auto chain = [&](const Launch& launch, unsigned char* g0, unsigned char** last_out) -> lbm_status {
        unsigned char* cur = g0;
        int t = 1;
        while (t <= T - 1) {
            const bool two = pairs && t + 1 <= T - 1;
            unsigned char* mid = two ? slot(t) : nullptr;
            unsigned char* dst = next_state(two ? t + 1 : t, cur);
            LBM_TRY(launch(cur, two, mid, dst, t));
            cur = dst;
            t += two ? 2 : 1;
        }
        *last_out = cur;
        return LBM_OK;
    };
    unsigned char* g0 = slot(0) ? slot(0) : ping0;
    unsigned char* last = nullptr;
    chain([](const unsigned char*, bool, unsigned char*, unsigned char*, int) { return LBM_OK; }, g0, &last);
    auto issue = [&](cudaStream_t st_) -> lbm_status {
        LBM_TRY(write_mrt_rates(p, bc, st_));
        if (cudaMemsetAsync(g0, 0, p->info.state_bytes, st_) != cudaSuccess) return LBM_ERR_CUDA;  // g^0 = rest
        if (one && cudaMemsetAsync(bcs.side_u, 0, (size_t)p->info.prec * 6 * (size_t)p->info.n_acc, st_) !=
                       cudaSuccess)
            return LBM_ERR_CUDA;  // at rest every velocity is zero
        unsigned char* end = nullptr;
        return chain(
            [&](const unsigned char* src, bool two, unsigned char* mid, unsigned char* dst, int t) -> lbm_status {
                // the launch producing g^t streams into time level t (the velocity inlet's ramp)
                return two ? step2_launch(p->info, src, mid, dst, at_time(bc, t), tau, st_)
                           : sweep_step(p, src, dst, bcs, t, tau, st_);
            },
            g0, &end);
    };
    GraphKey key;
    key.op = 1;
    key.ptr[0] = d_ws;
    key.ptr[1] = p->link;
    key.scalar = rho_out;
    LBM_TRY(run_sequence(p, key, s, issue));
    // f^T = S(g^{T-1}) into the caller's array
    return final_stream(p, last, d_f, at_time(bc, T), tau, s, layout_at(one, T - 1));
}

lbm_status lbm_step(lbm_plan* p, const double* d_rho_in, const double* d_tau, double rho_out, const void* d_f_in,
                    void* d_f_out, int32_t n_steps, void* d_ws, void* stream)
{
    LBM_TRY(check_common(p, d_ws));
    LBM_TRY(check_layout_options(p));
    if (!d_rho_in || !d_tau || !d_f_in || !d_f_out || !d_ws || n_steps < 1) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* ws = bytes(d_ws);
    const double* rho_in = nullptr;
    const double* tau = nullptr;
    LBM_TRY(stage_inputs(p, d_ws, d_rho_in, d_tau, &rho_in, &tau, s));
    const Bc bc = make_bc(p, rho_in, rho_out, d_ws);
    unsigned char* ping0 = ws + p->ws.ping[0];
    unsigned char* ping1 = ws + p->ws.ping[1];
    // collide the caller's state into ping0, n - 1 stream-collide launches between the ping-pong
    // buffers (in place: on ping0 alone) as the cached part, then stream into the caller's output
    const bool one = in_place(p);
    Bc bcs = bc;
    if (one) bcs.side_u = ws + p->ws.side;  // the collide-only launch writes the Eq. 6 nodes' velocities
    LBM_TRY(write_mrt_rates(p, bc, s));
    if (p->info.cmp.nf)
        LBM_TRY(step_launch_cmp(p->info, kCollideOnly, d_f_in, ping0, true, false, bcs, tau, s));
    else
        LBM_TRY(step_launch(p->info, kCollideOnly, d_f_in, ping0, bc, tau, s));
    // n - 1 stream-collide steps, two per launch where the two-step kernel applies
    const bool pairs = !one && step2_possible(p->info, bc);
    const int launches = pairs ? n_steps / 2 : n_steps - 1;  // (n - 1) / 2 pairs and (n - 1) % 2 single steps
    unsigned char* last = one || launches % 2 == 0 ? ping0 : ping1;
    auto issue = [&](cudaStream_t st_) -> lbm_status {
        unsigned char* cur = ping0;
        int t = 1;
        while (t < n_steps) {
            unsigned char* dst = one ? ping0 : (cur == ping0 ? ping1 : ping0);
            if (pairs && t + 1 < n_steps) {
                LBM_TRY(step2_launch(p->info, cur, nullptr, dst, at_time(bc, t), tau, st_));
                t += 2;
            } else {
                LBM_TRY(sweep_step(p, cur, dst, bcs, t, tau, st_));
                t += 1;
            }
            cur = dst;
        }
        return LBM_OK;
    };
    if (n_steps < 8) {
        LBM_TRY(issue(s));
    } else {
        GraphKey key;
        key.op = 2;
        key.ptr[0] = d_ws;
        key.ptr[1] = p->link;
        key.scalar = rho_out;
        key.n = n_steps;
        LBM_TRY(run_sequence(p, key, s, issue));
    }
    return final_stream(p, last, d_f_out, at_time(bc, n_steps), tau, s, layout_at(one, n_steps - 1));
}

lbm_status lbm_loss_grad(lbm_plan* p, const void* d_f, const double* d_u_target, const uint8_t* d_roi,
                         double* d_loss, void* d_lambda, void* d_ws, void* stream)
{
    LBM_TRY(check_common(p, d_ws));
    if (!d_f || !d_u_target || !d_loss || !d_lambda || !d_ws) return LBM_ERR_INVALID_ARG;
    p->last_ws = d_ws;
    return loss_launch(p->info, d_f, d_u_target, d_roi, p->desc.loss_kind, p->desc.loss_norm, d_loss, d_lambda,
                       bytes(d_ws), p->ws, static_cast<cudaStream_t>(stream));
}

lbm_status lbm_loss_grad_noalloc(lbm_plan* p, const void* d_f, const double* d_u_target, const uint8_t* d_roi,
                                 double* d_loss, void* d_lambda, void* stream)
{
    LBM_TRY(check_common(p, nullptr));
    if (!d_f || !d_u_target || !d_loss || !d_lambda) return LBM_ERR_INVALID_ARG;
    return loss_launch_noalloc(p->info, d_f, d_u_target, d_roi, p->desc.loss_kind, p->desc.loss_norm, d_loss,
                               d_lambda, static_cast<cudaStream_t>(stream));
}

lbm_status lbm_probe_loss_grad(lbm_plan* p, const void* d_f, int64_t n_probe, const int64_t* d_probe_node,
                               const double* d_rho_target, double weight, double* d_loss, void* d_lambda, void* d_ws,
                               void* stream)
{
    LBM_TRY(check_common(p, d_ws));
    if (n_probe < 0 || !d_f || !d_loss || !d_lambda || !d_ws || !std::isfinite(weight)) return LBM_ERR_INVALID_ARG;
    if (n_probe > 0 && (!d_probe_node || !d_rho_target)) return LBM_ERR_INVALID_ARG;
    p->last_ws = d_ws;
    return probe_launch(p->info, d_f, n_probe, d_probe_node, d_rho_target, weight, d_loss, d_lambda,
                        reinterpret_cast<uint32_t*>(bytes(d_ws) + p->ws.status), static_cast<cudaStream_t>(stream));
}

lbm_status lbm_spline_basis(int32_t n_knots, int32_t n, double* h_basis)
{
    if (!h_basis || n < 1 || n_knots < 1 || n_knots > n || n > (1 << 20)) return LBM_ERR_INVALID_ARG;
    spline_basis_host(n_knots, n, h_basis);
    return LBM_OK;
}

static bool spline_args_ok(const lbm_plan* p, int32_t ky, int32_t kz)
{
    return p && p->desc.inlet_kind == LBM_INLET_PROFILE && ky >= 1 && kz >= 1 && ky <= p->info.geo.ny &&
           kz <= p->info.geo.nz;
}

lbm_status lbm_spline_profile(const lbm_plan* p, int32_t ky, int32_t kz, const double* d_by, const double* d_bz,
                              const double* d_knots, double rho_out, double* d_rho_in, void* stream)
{
    if (!spline_args_ok(p, ky, kz) || !d_by || !d_bz || !d_knots || !d_rho_in) return LBM_ERR_INVALID_ARG;
    return spline_profile_launch(p->info, ky, kz, d_by, d_bz, d_knots, rho_out, d_rho_in,
                                 static_cast<cudaStream_t>(stream));
}

lbm_status lbm_spline_grad(const lbm_plan* p, int32_t ky, int32_t kz, const double* d_by, const double* d_bz,
                           const double* d_grad_rho_in, double* d_grad_knots, void* stream)
{
    if (!spline_args_ok(p, ky, kz) || !d_by || !d_bz || !d_grad_rho_in || !d_grad_knots) return LBM_ERR_INVALID_ARG;
    return spline_grad_launch(p->info, ky, kz, d_by, d_bz, d_grad_rho_in, d_grad_knots,
                              static_cast<cudaStream_t>(stream));
}

// The reverse sweep of lbm_adjoint and lbm_adjoint_window: lambda^T from
// d_lambda, or (win) from the window's observations at T; with a window, the
// seed of each observation at t < T is added to lambda^t right after the
// adjoint step that produces it, and the observations' losses are summed
// into win->d_loss.
struct Window {
    int n_obs;
    const int32_t* steps;     // host, 1..T
    const double* targets;    // [n_obs][D][N]
    const uint8_t* roi;       // nullable
    const void* f_T;          // f^T of the preceding forward sweep (dense)
    void* scr_f;              // dense scratch state: f^t of an observation
    void* scr_lam;            // dense scratch state: its seed
    double* d_loss;
};

static lbm_status reverse_sweep(lbm_plan* p, const double* d_rho_in, const double* d_tau, double rho_out,
                                const void* d_lambda, const Window* win, double* d_grad_rho_in, double* d_grad_tau,
                                void* d_ws, cudaStream_t s)
{
    unsigned char* ws = bytes(d_ws);
    p->last_ws = d_ws;
    const double* rho_in = nullptr;
    const double* tau = nullptr;
    LBM_TRY(stage_inputs(p, d_ws, d_rho_in, d_tau, &rho_in, &tau, s));
    const Bc bc = make_bc(p, rho_in, rho_out, d_ws);
    const int T = p->desc.n_steps, k = p->k, S = p->S;
    // the checkpoints must come from a forward sweep of the same schedule (their layouts differ)
    if (p->fwd_aa >= 0 && p->fwd_aa != (in_place(p) ? 1 : 0)) return LBM_ERR_INVALID_ARG;
    const size_t st = align256(p->info.state_bytes);
    double* grad_acc = reinterpret_cast<double*>(ws + p->ws.grad_acc);
    double* partial = reinterpret_cast<double*>(ws + p->ws.partial);
    if (persist_ok(p->info) && !win) {
        // one cooperative launch for all segments: recompute, then adjoint steps backwards
        if (cudaMemsetAsync(grad_acc, 0, sizeof(double) * (size_t)p->info.n_acc, s) != cudaSuccess)
            return LBM_ERR_CUDA;
        if (cudaMemsetAsync(partial, 0, sizeof(double) * (size_t)p->info.n_partial, s) != cudaSuccess)
            return LBM_ERR_CUDA;
        PersistArgs a = persist_args(p, d_ws);
        a.lam_in = d_lambda;
        LBM_TRY(reverse_persist(p->info, a, bc, tau, grad_acc, partial, s));
        return finish_gradients_launch(p->info, grad_acc, partial, tau, d_grad_rho_in, d_grad_tau,
                                       reinterpret_cast<uint32_t*>(ws + p->ws.status), s);
    }
    // seg(b, j): state j of segment buffer b; buffer sg & 1 holds segment sg,
    // g^{t0 + j - 1} at j >= 1 (for sg = 0, j = 0 stands for the rest state f^0)
    auto seg = [&](int sg, int j) -> unsigned char* {
        return ws + p->ws.seg + st * ((size_t)(sg & 1) * (size_t)k + (size_t)j);
    };
    auto base_of = [&](int sg) -> const unsigned char* {
        return sg >= 1 ? ws + p->ws.ckpt + st * (size_t)(sg - 1) : nullptr;
    };
    // in place: g^t and lambda^t in the layout of t's parity, lambda updated in place in lam[1]; the
    // recomputed segment states are written out of place, so they read the Eq. 6 velocities from their input
    const bool one = in_place(p);
    // the recompute's kernels: the plan's, or the recompute family when one is chosen
    PlanInfo rec = p->info;
    if (rec.rec_family != LBM_FAMILY_AUTO) rec.step_family = rec.rec_family;
    const bool pairs = !one && step2_possible(rec, bc);
    auto recompute = [&](int sg, cudaStream_t s_) -> lbm_status {
        const int len = std::min(k, T - sg * k);
        const unsigned char* prev = base_of(sg);
        int j = 1;
        while (j < len) {
            if (sg == 0 && j == 1) {
                if (cudaMemsetAsync(seg(0, 1), 0, p->info.state_bytes, s_) != cudaSuccess) return LBM_ERR_CUDA;
                prev = seg(sg, j);
                j += 1;
            } else if (pairs && j + 1 < len) {  // every segment state is needed: g^t goes to mid
                LBM_TRY(step2_launch(rec, prev, seg(sg, j), seg(sg, j + 1), at_time(bc, sg * k + j - 1), tau, s_));
                prev = seg(sg, j + 1);
                j += 2;
            } else {  // seg(sg, j) holds g^{sg k + j - 1}
                LBM_TRY(sweep_step(p, prev, seg(sg, j), bc, sg * k + j - 1, tau, s_, &rec));
                prev = seg(sg, j);
                j += 1;
            }
        }
        return LBM_OK;
    };
    // lambda^T enters through the workspace (lam[1]), so the cached graph does not depend on d_lambda
    void* lam_T = ws + p->ws.lam[1];
    const void* lam_cur = lam_T;
    int lam_next = 0;
    double* loss_tmp = reinterpret_cast<double*>(ws + p->ws.status + kScalarTmp);
    // one observation of the window at time t: its loss into d_loss, its seed dL_t/df^t added to lam (internal
    // layout); f^t = S(g^{t-1}) is streamed from src into the dense scratch first (or is f^T itself)
    auto observe = [&](int o, int t, const unsigned char* src, void* lam, cudaStream_t s_) -> lbm_status {
        const void* ft = win->f_T;
        if (t < T) {
            LBM_TRY(final_stream(p, src, win->scr_f, at_time(bc, t), tau, s_, layout_at(one, t - 1)));
            ft = win->scr_f;
        }
        const size_t dn = (size_t)p->info.d * (size_t)p->info.geo.N;
        LBM_TRY(loss_launch(p->info, ft, win->targets + (size_t)o * dn, win->roi, p->desc.loss_kind,
                            p->desc.loss_norm, loss_tmp, win->scr_lam, ws, p->ws, s_));
        LBM_TRY(accumulate_launch(win->d_loss, loss_tmp, s_));
        return p->info.cmp.nf ? compact_gather_add_launch(p->info, win->scr_lam, lam, s_, layout_at(one, t))
                              : add_state_launch(p->info, lam, win->scr_lam, s_);
    };
    auto adjoint_steps = [&](int sg, cudaStream_t s_) -> lbm_status {
        const int len = std::min(k, T - sg * k);
        for (int j = len - 1; j >= 0; --j) {
            const unsigned char* src = j == 0 ? base_of(sg) : seg(sg, j);
            const int at_rest = (sg == 0 && j == 0) ? 1 : 0;
            const int t = sg * k + j;
            void* lam_out = one ? lam_T : ws + p->ws.lam[lam_next];
            // the adjoint step at t re-forms f^t = S(g^{t-1}) at the inlet nodes: streaming level t
            if (one)
                LBM_TRY(adjoint_launch_cmp(p->info, at_rest, src, lam_cur, lam_out, at_time(bc, t), tau, grad_acc,
                                           partial, s_, layout_at(true, t - 1), layout_at(true, t)));
            else
                LBM_TRY(adjoint_launch(p->info, at_rest, src, lam_cur, lam_out, at_time(bc, t), tau, grad_acc,
                                       partial, s_));
            if (win)  // src holds g^{t-1}, t = sg k + j
                for (int o = 0; o < win->n_obs; ++o)
                    if (win->steps[o] == sg * k + j && !at_rest) LBM_TRY(observe(o, sg * k + j, src, lam_out, s_));
            lam_cur = lam_out;
            lam_next ^= 1;
        }
        return LBM_OK;
    };
    const bool overlap = p->info.overlap && S > 1;
    if (overlap && !p->helper) {
        if (cudaStreamCreateWithFlags(&p->helper, cudaStreamNonBlocking) != cudaSuccess) return LBM_ERR_CUDA;
        for (auto& e : p->ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LBM_ERR_CUDA;
    }
    if (win) {  // lambda^T: the seeds of the observations at T
        if (cudaMemsetAsync(win->d_loss, 0, sizeof(double), s) != cudaSuccess ||
            cudaMemsetAsync(lam_T, 0, p->info.state_bytes, s) != cudaSuccess)
            return LBM_ERR_CUDA;
        LBM_TRY(write_mrt_rates(p, bc, s));
        for (int o = 0; o < win->n_obs; ++o)
            if (win->steps[o] == T) LBM_TRY(observe(o, T, nullptr, lam_T, s));
    } else if (p->info.cmp.nf) {  // lambda^T into the compact layout
        LBM_TRY(compact_gather_launch(p->info, d_lambda, lam_T, s, layout_at(one, T)));
    } else if (cudaMemcpyAsync(lam_T, d_lambda, p->dense_state_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        return LBM_ERR_CUDA;
    }
    auto issue = [&](cudaStream_t st_) -> lbm_status {
        LBM_TRY(write_mrt_rates(p, bc, st_));
        lam_cur = lam_T;
        lam_next = 0;
        if (cudaMemsetAsync(grad_acc, 0, sizeof(double) * (size_t)p->info.n_acc, st_) != cudaSuccess)
            return LBM_ERR_CUDA;
        if (cudaMemsetAsync(partial, 0, sizeof(double) * (size_t)p->info.n_partial, st_) != cudaSuccess)
            return LBM_ERR_CUDA;
        if (!overlap) {
            for (int sg = S - 1; sg >= 0; --sg) {
                LBM_TRY(recompute(sg, st_));
                LBM_TRY(adjoint_steps(sg, st_));
            }
        } else {
            // Segment sg - 1 is recomputed on the helper stream B while the
            // adjoint steps of segment sg run on A; the two segment buffers
            // alternate, so recomputing sg - 1 waits for the adjoint of sg + 1
            // (the last reader of its buffer).
            cudaStream_t A = st_, B = p->helper;
            cudaEvent_t fork = p->ev[0], join = p->ev[1], rec_done = p->ev[2], adj_done = p->ev[3];
            auto ok = [](cudaError_t e) { return e == cudaSuccess; };
            if (!ok(cudaEventRecord(fork, A)) || !ok(cudaStreamWaitEvent(B, fork, 0))) return LBM_ERR_CUDA;
            LBM_TRY(recompute(S - 1, B));
            if (!ok(cudaEventRecord(rec_done, B)) || !ok(cudaStreamWaitEvent(A, rec_done, 0))) return LBM_ERR_CUDA;
            for (int sg = S - 1; sg >= 0; --sg) {
                if (sg >= 1) {
                    if (sg + 1 <= S - 1 && !ok(cudaStreamWaitEvent(B, adj_done, 0))) return LBM_ERR_CUDA;
                    LBM_TRY(recompute(sg - 1, B));
                    if (!ok(cudaEventRecord(rec_done, B))) return LBM_ERR_CUDA;
                }
                LBM_TRY(adjoint_steps(sg, A));
                if (!ok(cudaEventRecord(adj_done, A))) return LBM_ERR_CUDA;
                if (sg >= 1 && !ok(cudaStreamWaitEvent(A, rec_done, 0))) return LBM_ERR_CUDA;
            }
            if (!ok(cudaEventRecord(join, B)) || !ok(cudaStreamWaitEvent(A, join, 0))) return LBM_ERR_CUDA;
        }
        return LBM_OK;
    };
    GraphKey key;
    key.op = win ? 4 : 3;
    key.ptr[0] = d_ws;
    key.ptr[1] = p->link;
    key.scalar = rho_out;
    if (win) {  // the observations' buffers and steps are part of the launch sequence
        key.ptr[2] = win->targets;
        key.ptr[3] = win->roi;
        key.ptr[4] = win->scr_f;
        key.ptr[5] = win->scr_lam;
        key.ptr[6] = win->d_loss;
        unsigned long long h = 1469598103934665603ull;  // FNV-1a over the step list
        for (int o = 0; o < win->n_obs; ++o) {
            h ^= (unsigned long long)(uint32_t)win->steps[o];
            h *= 1099511628211ull;
        }
        key.n = (long long)(h ^ (unsigned long long)win->n_obs);
    }
    LBM_TRY(run_sequence(p, key, s, issue));
    // the gradients into the caller's arrays
    return finish_gradients_launch(p->info, grad_acc, partial, tau, d_grad_rho_in, d_grad_tau,
                                   reinterpret_cast<uint32_t*>(ws + p->ws.status), s);
}

lbm_status lbm_adjoint(lbm_plan* p, const double* d_rho_in, const double* d_tau, double rho_out,
                       const void* d_lambda, double* d_grad_rho_in, double* d_grad_tau, void* d_ws, void* stream)
{
    LBM_TRY(check_common(p, d_ws));
    LBM_TRY(check_layout_options(p));
    if (!d_rho_in || !d_tau || !d_lambda || !d_grad_rho_in || !d_grad_tau || !d_ws) return LBM_ERR_INVALID_ARG;
    return reverse_sweep(p, d_rho_in, d_tau, rho_out, d_lambda, nullptr, d_grad_rho_in, d_grad_tau, d_ws,
                         static_cast<cudaStream_t>(stream));
}

lbm_status lbm_adjoint_window(lbm_plan* p, const double* d_rho_in, const double* d_tau, double rho_out,
                              const void* d_f, int32_t n_obs, const int32_t* h_obs_steps,
                              const double* d_u_targets, const uint8_t* d_roi, void* d_scratch_f,
                              void* d_scratch_lambda, double* d_loss, double* d_grad_rho_in, double* d_grad_tau,
                              void* d_ws, void* stream)
{
    LBM_TRY(check_common(p, d_ws));
    LBM_TRY(check_layout_options(p));
    if (!d_rho_in || !d_tau || !d_f || !h_obs_steps || !d_u_targets || !d_scratch_f || !d_scratch_lambda ||
        !d_loss || !d_grad_rho_in || !d_grad_tau || !d_ws || n_obs < 1 || n_obs > 65536)
        return LBM_ERR_INVALID_ARG;
    for (int o = 0; o < n_obs; ++o)
        if (h_obs_steps[o] < 1 || h_obs_steps[o] > p->desc.n_steps) return LBM_ERR_INVALID_ARG;
    Window w{n_obs, h_obs_steps, d_u_targets, d_roi, d_f, d_scratch_f, d_scratch_lambda, d_loss};
    return reverse_sweep(p, d_rho_in, d_tau, rho_out, nullptr, &w, d_grad_rho_in, d_grad_tau, d_ws,
                         static_cast<cudaStream_t>(stream));
}

lbm_status lbm_macroscopic(lbm_plan* p, const void* d_f, double* d_rho, double* d_u, void* stream)
{
    LBM_TRY(check_common(p, nullptr));
    if (!d_f || !d_u) return LBM_ERR_INVALID_ARG;
    return macroscopic_launch(p->info, d_f, d_rho, d_u, static_cast<cudaStream_t>(stream));
}

lbm_status lbm_darcy(lbm_plan* p, const void* d_f, const double* d_rho_in, const double* d_tau, double rho_out,
                     int32_t xs, double* d_k, double* d_flux, void* stream)
{
    LBM_TRY(check_common(p, nullptr));
    if (!d_f || !d_rho_in || !d_tau || !d_k || xs < 0 || xs >= p->info.geo.nx) return LBM_ERR_INVALID_ARG;
    return darcy_launch(p->info, d_f, d_rho_in, p->info.n_in, d_tau, rho_out, xs, d_k, d_flux,
                        static_cast<cudaStream_t>(stream));
}

lbm_status lbm_adam_step(int32_t n, double* d_theta, double* d_m, double* d_v, const double* d_grad_p, double* d_p,
                         double p_offset, double p_scale, int32_t t, double lr, double beta1, double beta2,
                         double eps, void* stream)
{
    if (n < 1 || n > 65536 || t < 1 || !d_theta || !d_m || !d_v || !d_grad_p || !d_p) return LBM_ERR_INVALID_ARG;
    return adam_launch(n, d_theta, d_m, d_v, d_grad_p, d_p, p_offset, p_scale, t, lr, beta1, beta2, eps,
                       static_cast<cudaStream_t>(stream));
}

lbm_status lbm_get_status(lbm_plan* p, lbm_status* status)
{
    if (!p || !status) return LBM_ERR_INVALID_ARG;
    *status = LBM_OK;
    if (!p->last_ws) return LBM_OK;
    uint32_t word = 0;
    uint32_t* dev = reinterpret_cast<uint32_t*>(bytes(p->last_ws) + p->ws.status);
    if (cudaMemcpy(&word, dev, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemset(dev, 0, sizeof(word)) != cudaSuccess) return LBM_ERR_CUDA;
    for (int b = 1; b < 32; ++b)
        if (word & (1u << b)) {
            *status = static_cast<lbm_status>(b);
            break;
        }
    return LBM_OK;
}

const char* lbm_error_string(lbm_status st)
{
    switch (st) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_UNSUPPORTED: return "unsupported configuration";
    case LBM_ERR_OOM: return "buffer too small";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_NONFINITE: return "non-finite loss or gradient";
    case LBM_ERR_TIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

}  // extern "C"
