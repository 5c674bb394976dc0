/*
 * lbm.h — C ABI of the GB300 (sm_103a) differentiable lattice Boltzmann
 * library: the forward step and the hand-written reverse (adjoint) step of
 * the AD-LBM inversion of arXiv 2310.00810 (Wang & Kumar), in D2Q9 and D3Q19.
 *
 * The method (section 2.1 of the paper):
 *   Eq. 1-2  rho = sum_i f_i,  rho u = sum_i f_i c_i
 *   Eq. 3-5  BGK: f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq(rho, u)) / tau,
 *            f_i^eq = w_i rho (1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u)  (c_s^2 = 1/3)
 *   Eq. 6    anti-bounce-back pressure planes at x = -1/2 (rho_in) and
 *            x = nx - 1/2 (rho_out)
 *   section 2.2 "Bounce Back": halfway bounce-back at grain nodes and at the
 *            walls y = -1/2, ny - 1/2 (and z = -1/2, nz - 1/2)
 *   section 2.2 / Eq. 7 / Eq. 15: velocity-mismatch loss at the final step,
 *            differentiated with respect to the inlet density (a constant
 *            head or a per-node profile) and tau.
 * The paper differentiates with Taichi's tape (section 2.2); this library
 * instead runs an explicit discrete adjoint with sqrt(T) checkpointing.
 *
 * Conventions
 *  - Every call returns an lbm_status.  Calls that take a stream are
 *    asynchronous on that stream (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream) unless stated otherwise.  Errors detected on the
 *    device (a non-finite loss or gradient, a bounded wait that gave up) are
 *    latched in the plan's status word; lbm_get_status reads it.
 *  - Ownership: every device buffer is allocated and owned by the caller.
 *    The plan keeps host-side state only, plus the device pointers it was
 *    given by lbm_init_geometry (which must stay valid while it is used).
 *  - Layout: node index n = (z * ny + y) * nx + x (x fastest), N = nx ny nz.
 *    Populations f[i * N + n], i = 0..Q-1, stored SHIFTED by the rest state
 *    (f_i - w_i), in the plan's precision (float or double).  Velocity
 *    fields u[a * N + n] (a = 0..D-1) and densities are double.
 *  - D2Q9 order: rest, E, N, W, S, NE, NW, SW, SE (the order of the paper's
 *    Fig. 1 and MRT matrix, Eq. 18).  D3Q19 order: rest, +x, -x, +y, -y, +z,
 *    -z, (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
 *    (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 *  - A plan is not thread-safe; separate plans are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
    LBM_ERR_UNSUPPORTED = 2, /* a valid request the library does not implement */
    LBM_ERR_OOM = 3,         /* a caller-provided buffer is too small */
    LBM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    LBM_ERR_NONFINITE = 5,   /* a loss or gradient came out NaN or Inf */
    LBM_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up */
} lbm_status;

enum { LBM_LOSS_VEC = 0, LBM_LOSS_NORM = 1 };          /* |u - u_t|^2  or  (|u| - |u_t|)^2 */
enum { LBM_NORM_SUM = 0, LBM_NORM_MEAN_FLUID = 1 };    /* Eq. 7 (sum) or Eq. 15 (mean over fluid) */
enum { LBM_INLET_CONST = 0, LBM_INLET_PROFILE = 1 };   /* one rho_in, or one per inlet node */
enum { LBM_GEOM_CHANNEL = 0, LBM_GEOM_DISKS = 1, LBM_GEOM_SPHERES = 2, LBM_GEOM_MASK = 3 };

/* Link-word bits (lbm_init_geometry's d_link): bit i (i < Q) set when a
 * fluid node receives direction i by halfway bounce-back (the link from
 * x - c_i crosses a wall plane or starts at a solid node); LBM_LINK_SOLID set
 * (alone) on solid nodes. */
#define LBM_LINK_SOLID 0x80000000u

typedef struct lbm_desc {
    int32_t q;           /* 9 (D2Q9) or 19 (D3Q19) */
    int32_t nx, ny, nz;  /* lattice size; nz = 1 for D2Q9; nx >= 2, ny >= 1 */
    int32_t precision;   /* bytes per population: 4 (float) or 8 (double) */
    int32_t n_steps;     /* T >= 1: time steps of lbm_forward / lbm_adjoint */
    int32_t ckpt_stride; /* k: keep every k-th state (0: ceil(sqrt(T)); 1: every state) */
    int32_t loss_kind;   /* LBM_LOSS_VEC | LBM_LOSS_NORM */
    int32_t loss_norm;   /* LBM_NORM_SUM | LBM_NORM_MEAN_FLUID */
    int32_t inlet_kind;  /* LBM_INLET_CONST | LBM_INLET_PROFILE (ny * nz entries, [z * ny + y]) */
} lbm_desc;

typedef struct lbm_geom_desc {
    int32_t kind;            /* LBM_GEOM_* ; DISKS needs q = 9, SPHERES q = 19 */
    int32_t r_min, r_max;    /* grain radius range in lattice units, 0 <= r_min <= r_max */
    int32_t hydro_q8;        /* voxelised radius = r * hydro_q8 / 256 (256: factor 1; 230: ~0.9 R) */
    int32_t inlet_buffer;    /* columns kept free of grains at each end (>= 1) */
    int32_t fill_isolated;   /* nonzero: pores not connected to x = 0 become solid */
    int64_t max_rejections;  /* stop after this many trials in a row that add no solid node */
    uint64_t seed;           /* SplitMix64 seed */
    double target_porosity;  /* stop once fluid nodes <= (int64)(target * N) */
} lbm_geom_desc;

typedef struct lbm_plan lbm_plan;

/* Creates a plan for one lattice (host memory only; no device allocation).
 * Errors: INVALID_ARG for an unsupported q/precision, non-positive sizes,
 * ny or nz above 65535 (the kernels put rows and layers on the grid's y and
 * z dimensions), nz != 1 with q = 9, T < 1 or a negative stride. */
LBM_API lbm_status lbm_plan_create(const lbm_desc* desc, lbm_plan** out);
LBM_API lbm_status lbm_plan_destroy(lbm_plan* plan);

/* Kernel families for the step and adjoint kernels (performance only: all
 * give the same results to rounding).  AUTO picks TMA-staged kernels where
 * alignment allows (FP32, nx % 4 == 0), else vectorised register kernels,
 * else one node per thread. */
enum { LBM_FAMILY_AUTO = 0, LBM_FAMILY_SCALAR = 1, LBM_FAMILY_VEC = 2, LBM_FAMILY_TMA = 3 };

typedef struct lbm_kernel_choice {
    int32_t step_family;     /* LBM_FAMILY_* for the stream-collide kernels */
    int32_t adjoint_family;  /* LBM_FAMILY_* for the adjoint kernels */
    int32_t vec;             /* nodes per thread of the register kernels: 2 or 4 */
    int32_t tma_rows;        /* tile height of the D2Q9 TMA kernels: 4 or 8 */
    int32_t pdl;             /* 1: programmatic dependent launch between sweep kernels */
    int32_t persist;         /* 1: one cooperative launch per sweep (lattices up to 24 MB of state) */
    int32_t overlap;         /* 1: the reverse sweep recomputes segment s - 1 on a second stream while
                                the adjoint steps of segment s run (two segment buffers) */
    int32_t adjoint_tma_rows; /* tile height of the D2Q9 TMA adjoint kernels: 4 or 8 (0: as tma_rows) */
    int32_t steps_per_launch; /* 1, or 2: two stream-collide steps per launch (temporal blocking: a tile plus a
                                 two-node halo in shared memory) where the dense D2Q9 FP32 TMA kernels apply,
                                 in the forward sweep, the segment recompute and lbm_step; 0 reads as 1 */
    int32_t recompute_family; /* LBM_FAMILY_* of the reverse sweep's segment recompute (the stream-collide
                                 launches that run on the second stream beside the adjoint steps when overlap
                                 is on); LBM_FAMILY_AUTO: as step_family.  A register family here (no shared
                                 memory) lets its CTAs share the SMs with the adjoint's TMA CTAs.  Every family
                                 computes the same step; only the speed differs. */
    int32_t aa;              /* 1: in-place (AA-pattern) streaming in the fluid-only layout (the dense layout
                                ignores it).  The forward sweep and lbm_step advance one state buffer in place
                                and the reverse sweep updates lambda in place: a step from a state stored in
                                its natural layout gathers through the neighbour table and writes the swapped
                                layout, the next step reads and writes each node's own slots (no table), so
                                every other step moves no table bytes.  Checkpoints and segment states keep
                                one buffer each, as before.  The workspace loses one forward and one adjoint
                                state (re-query lbm_workspace_size after a change: it grows back when aa is
                                cleared).  Results equal those of the two-buffer pull.  lbm_adjoint needs the
                                checkpoints of an lbm_forward run with the same setting (else INVALID_ARG).
                                Not with LBM_ABB_U_EXTRAP (the sweeps return UNSUPPORTED). */
} lbm_kernel_choice;

/* Sets / reads the plan's kernel choice (an autotuner's knob).  Cached CUDA
 * graphs of the plan are dropped on a change.  Errors: INVALID_ARG for an
 * out-of-range field. */
LBM_API lbm_status lbm_plan_set_kernels(lbm_plan* plan, const lbm_kernel_choice* choice);
LBM_API lbm_status lbm_plan_get_kernels(const lbm_plan* plan, lbm_kernel_choice* choice);

/* Where Eq. 6 (section 2.1, the anti-bounce-back pressure boundary) takes
 * the velocity of its quadratic term; the paper writes it as a bare u.
 *   LBM_ABB_U_NODE    the boundary node's own velocity at time t (default)
 *   LBM_ABB_U_EXTRAP  that velocity extrapolated linearly to the pressure
 *                     plane half a link outside the node:
 *                     u_w = u(x_b) + (u(x_b) - u(x_b + e)) / 2, x_b + e the
 *                     next node inward; where that node is solid, u_w = u(x_b)
 * lbm_forward, lbm_step and lbm_adjoint follow the setting.  With
 * LBM_ABB_U_EXTRAP the dense layout runs the one-node-per-thread kernels (no
 * TMA, register-vector or persistent kernels) and each adjoint step is
 * followed by one short per-row pass; the fluid-only layout keeps its
 * kernels.  Batches (lbm_batch_*) use the node velocity.  Cached CUDA graphs
 * are dropped on a change.  Errors: INVALID_ARG for an unknown mode. */
enum { LBM_ABB_U_NODE = 0, LBM_ABB_U_EXTRAP = 1 };
LBM_API lbm_status lbm_set_abb_velocity(lbm_plan* plan, int32_t mode);
LBM_API lbm_status lbm_get_abb_velocity(const lbm_plan* plan, int32_t* mode);

/* Collision operator.  LBM_COLLISION_BGK (default): Eq. 4-5.
 * LBM_COLLISION_MRT (section 3.4, Eq. 16-18; D2Q9 plans only): f* = f -
 * M^{-1} S M (f - f^eq), M the moment matrix of Eq. 18 (rows rho, e,
 * epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy; the printed p_xy row |c_x c_y| is
 * read as the orthogonal c_x c_y), m^eq = M f^eq with f^eq of Eq. 5, and
 * S = diag(-, s_e, s_eps, -, s_q, -, s_q, 1/tau, 1/tau): the stress rates follow
 * tau (so dL/dtau is the derivative through them alone), the free rates s_e,
 * s_eps, s_q are fixed here (each in (0, 2); the conserved moments need no
 * rate).  The dense layout runs the one-node-per-thread kernels while MRT is
 * set; the fluid-only layout keeps its kernels.  Batches use BGK.  Cached
 * CUDA graphs are dropped on a change.  Errors: INVALID_ARG for an unknown
 * mode or a rate outside (0, 2); UNSUPPORTED for MRT on a D3Q19 plan.
 * lbm_get_collision writes the mode and, if rates != NULL, the three rates
 * (zeros under BGK). */
enum { LBM_COLLISION_BGK = 0, LBM_COLLISION_MRT = 1 };
LBM_API lbm_status lbm_set_collision(lbm_plan* plan, int32_t mode, double s_e, double s_eps, double s_q);
LBM_API lbm_status lbm_get_collision(const lbm_plan* plan, int32_t* mode, double* rates);

/* Cylinder-wake options (section 3.4: the flow past a cylinder has a
 * free-stream velocity inlet and periodic top and bottom boundaries).
 * lbm_set_periodic_y: links leaving y = -1/2 or ny - 1/2 re-enter on the
 *   other side instead of bouncing back.  It shapes the link words and the
 *   fluid-only tables, so it must be set before lbm_init_geometry /
 *   lbm_bind_geometry (INVALID_ARG afterwards).  The flood fill of isolated
 *   pores does not wrap.
 * lbm_set_velocity_inlet: the links through x = -1/2 take the moving-wall
 *   bounce-back f_i = f*_opp(i) + 6 w_i rho_0 (c_i . u_in), rho_0 = 1, instead
 *   of Eq. 6 (the outlet keeps Eq. 6; d_rho_in is not used and its gradient
 *   is zero).  u_in finite; uz = 0 on D2Q9 plans.
 * Both run in the fluid-only layout only: lbm_forward, lbm_step and
 * lbm_adjoint return UNSUPPORTED on a dense plan with either option set. */
LBM_API lbm_status lbm_set_periodic_y(lbm_plan* plan, int32_t on);
LBM_API lbm_status lbm_set_velocity_inlet(lbm_plan* plan, int32_t on, double ux, double uy, double uz);

/* A gradual start of the velocity inlet (the flow of section 3.4 started
 * from rest without the impulse that makes it diverge at u_in = 0.2): the
 * step producing f^t uses u_in r(t), r(t) = sin^2(pi t / (2 steps)) for
 * 0 < t < steps and 1 from steps on (steps = 0: none, the default).  Time
 * counts from the rest state of lbm_forward (lbm_step counts from its input
 * state).  The inlet's source does not depend on the state, so no gradient
 * flows through it; the reverse sweep re-forms f^t at inlet nodes with the
 * same r(t) (each adjoint launch carries its step's time level).
 * Errors: INVALID_ARG for steps < 0. */
LBM_API lbm_status lbm_set_velocity_ramp(lbm_plan* plan, int32_t steps);

/* Bytes of device workspace lbm_forward / lbm_adjoint / lbm_step /
 * lbm_loss_grad need: ping-pong states, the sqrt(T) checkpoints and two
 * segment buffers, adjoint ping-pong states and FP64 reduction slots. */
LBM_API lbm_status lbm_workspace_size(const lbm_plan* plan, size_t* bytes);

/* Builds the geometry of section 3.1.1 / 3.3 stand-ins on the device
 * (seeded grains voxelised with integer arithmetic, then isolated pores
 * filled, then link words), bit-identical to the recipe:
 *   SplitMix64 draws, Q8 fixed point, cx = draw_below(256 nx),
 *   cy = draw_below(256 ny), [cz = draw_below(256 nz)],
 *   r = 256 r_min + draw_below(256 (r_max - r_min) + 1); a trial is kept if
 *   it clears the inlet/outlet buffers and (disks) lies 1 lu from every
 *   placed disk; node solid iff |256 x - c|^2 <= (r hydro_q8 / 256)^2.
 * kind = LBM_GEOM_MASK takes d_mask as input (nonzero = solid) and only
 * fills and derives link words.
 *  d_mask      uint8[N]   out (in for MASK): 0 fluid, 1 solid; 4-byte aligned
 *                          and allocated to N rounded up to a multiple of 4
 *  d_link      uint32[N]  out: link words (LBM_LINK_SOLID / bounce-back bits);
 *                          the plan keeps this pointer for later calls
 *  d_porosity  double[1]  out (nullable): fluid fraction after the fill
 *  d_info      int64[4]   out (required): grains placed, solid before fill,
 *                          nodes filled, fluid nodes
 * Errors: INVALID_ARG (bad kind for q, radii, buffer), CUDA. */
LBM_API lbm_status lbm_init_geometry(lbm_plan* plan, const lbm_geom_desc* g, uint8_t* d_mask, uint32_t* d_link,
                             double* d_porosity, int64_t* d_info, void* stream);

/* Binds an existing link array (from lbm_init_geometry of a plan of the
 * same lattice size and Q) to this plan, so plans of different precision or
 * step count can share one geometry.  The pointer must stay valid.  The
 * array must come from a plan with the same lbm_set_periodic_y setting: the
 * dense kernels trust the wall bits at y = 0 and ny - 1 to keep every pull
 * inside the lattice. */
LBM_API lbm_status lbm_bind_geometry(lbm_plan* plan, const uint32_t* d_link);

/* Fluid-only ("compact") internal state layout.  The population traffic of
 * the streaming step (section 2.2: streaming and boundaries are most of the
 * time) is proportional to the nodes stored; a dense layout stores and moves
 * solid nodes too, while the compact layout keeps only the n_fluid fluid
 * nodes (the interior in node order, then the columns x = 0 and nx - 1,
 * whose boundary rules take a longer code path, in node order), with a
 * neighbour table: for fluid node k and
 * direction i >= 1 the compact index of x - c_i, or a code for a
 * bounce-back (section 2.2) or Eq. 6 link.  The layout is internal: every
 * call still takes and returns dense Q N arrays (f^T, lambda^T, the lbm_step
 * states); only the plan's workspace and the tables change.
 *
 * lbm_compact_size: bytes of the table buffer for n_fluid fluid nodes
 *   (4 n_fluid dense indices, 4 (Q - 1) n_fluid neighbour codes, one bit per
 *   fluid node, 4 N dense-to-compact map, scan scratch).
 * lbm_compact_bind: builds the tables from the bound link array into
 *   d_tables (device, caller-owned, 256-byte aligned, lbm_compact_size
 *   bytes, valid while the plan uses it) and switches the plan to the compact
 *   layout; lbm_workspace_size then reports the (smaller) compact workspace,
 *   which the caller must provide from then on.  n_fluid must equal the
 *   number of fluid nodes of the link array (d_info[3] of lbm_init_geometry);
 *   the call synchronises the stream to check it.  n_fluid = 0 switches back
 *   to the dense layout.  The kernel-family choice (lbm_plan_set_kernels)
 *   applies to the dense layout only; the one-launch persistent sweeps are
 *   not used with the compact layout.
 * Errors: INVALID_ARG (no geometry bound, n_fluid out of range or not the
 *   fluid count of the link array, misaligned d_tables), CUDA. */
LBM_API lbm_status lbm_compact_size(const lbm_plan* plan, int64_t n_fluid, size_t* bytes);
LBM_API lbm_status lbm_compact_bind(lbm_plan* plan, int64_t n_fluid, void* d_tables, void* stream);

/* T steps from rest (f = w_i, rho = 1: init_field of section 2.2), keeping
 * the checkpoints the adjoint needs in d_ws.
 *  d_rho_in  double[1 or ny nz]  inlet density (Eq. 6 rho_w at x = -1/2)
 *  d_tau     double[1]           relaxation time (> 1/2)
 *  rho_out   outlet density (Eq. 6 rho_w at x = nx - 1/2)
 *  d_f       out: f^T, shifted, plan precision, Q N values (every entry is
 *            written; solid nodes get 0)
 *  d_ws      workspace of lbm_workspace_size bytes, 256-byte aligned and
 *            zero-filled before its first use (it holds the status word)
 * Errors: INVALID_ARG (null pointers, no geometry bound), CUDA. */
LBM_API lbm_status lbm_forward(lbm_plan* plan, const double* d_rho_in, const double* d_tau, double rho_out, void* d_f,
                       void* d_ws, void* stream);

/* Advances an arbitrary state by n_steps (>= 1) without checkpoints:
 * d_f_out = (stream o collide)^n (d_f_in).  In-place (d_f_in == d_f_out) is
 * allowed.  Uses d_ws for intermediate states. */
LBM_API lbm_status lbm_step(lbm_plan* plan, const double* d_rho_in, const double* d_tau, double rho_out, const void* d_f_in,
                    void* d_f_out, int32_t n_steps, void* d_ws, void* stream);

/* Loss of the final state (section 3.1.2: sum of squared velocity
 * mismatches over the region of interest; Eq. 15 normalisation optional)
 * and its seed lambda^T = dL/df^T (zero at solid and non-ROI nodes).
 *  d_f        f^T (shifted, plan precision)
 *  d_u_target double[D N] target velocity
 *  d_roi      uint8[N] region of interest (nullable: all fluid nodes)
 *  d_loss     double[1] out
 *  d_lambda   out, plan precision, Q N values
 * A non-finite loss latches LBM_ERR_NONFINITE in the status word. */
LBM_API lbm_status lbm_loss_grad(lbm_plan* plan, const void* d_f, const double* d_u_target, const uint8_t* d_roi,
                         double* d_loss, void* d_lambda, void* d_ws, void* stream);

/* The same loss and seed as lbm_loss_grad, for callers that cannot
 * allocate device memory at all: code that runs under an allocator it does
 * not own (a plugin or extension inside a host application that forbids
 * cudaMalloc), real-time loops where an allocation could stall, or hosts
 * that only pass in the buffers they already have.  The paper has no
 * counterpart; this is an interface convenience only.
 * It takes no workspace: its reduction scratch is a fixed, file-scope
 * device array of LBM_NOALLOC_MAX_BLOCKS + 32 doubles (about 512 KB) that
 * every GPU loading this library holds until the process exits.  The call
 * itself allocates nothing (no cudaMalloc, no cudaFree, no allocating
 * library routine).
 *  - Lattices whose loss grid needs more than LBM_NOALLOC_MAX_BLOCKS thread
 *    blocks (ceil(nx / 128) * ny * nz > 65536) are rejected with
 *    LBM_ERR_INVALID_ARG; use lbm_loss_grad for those.
 *  - The first call on a device looks up the array's device address for
 *    that device (with it current); make that first call before any stream
 *    capture.  The address is kept with the id of the CUDA context it was
 *    taken in: after a device reset (cudaDeviceReset) the next call runs in a
 *    new context and looks the address up again (again: before any capture).
 *    The call makes the current device's primary context current on the
 *    calling thread (cudaSetDevice).
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose kernels may overlap on the GPU (different streams without
 *    ordering between them) race on it and must be serialised by the caller.
 *  - A non-finite loss shows up as a NaN/Inf in d_loss; unlike
 *    lbm_loss_grad, it does not latch the plan's status word. */
#define LBM_NOALLOC_MAX_BLOCKS 65536
LBM_API lbm_status lbm_loss_grad_noalloc(lbm_plan* plan, const void* d_f, const double* d_u_target,
                                         const uint8_t* d_roi, double* d_loss, void* d_lambda, void* stream);

/* Density probes: adds the term w sum_p (rho(x_p) - rho_p)^2 to the loss
 * and its seed 2 w (rho(x_p) - rho_p) to every direction of lambda^T at x_p
 * (drho/df_k = 1, Eq. 1).  A second observation for the joint inversion of
 * the inlet head and tau (section 3.3), which the steady velocity alone
 * fixes only through their ratio in the Stokes regime.  Call it after
 * lbm_loss_grad on the same d_loss / d_lambda.
 *  d_f           f^T (shifted, plan precision), dense
 *  n_probe       number of probes (0: nothing to add)
 *  d_probe_node  int64[n_probe] dense node indices (z ny + y) nx + x
 *  d_rho_target  double[n_probe] observed densities
 *  weight        w (finite)
 *  d_loss        double[1] in/out: the term is added
 *  d_lambda      plan precision, Q N values, in/out: the seeds are added
 * A solid probe node contributes nothing.  A node listed twice gets both
 * seeds, added atomically (their order, so the last bit, may vary between
 * runs); distinct nodes give deterministic results.  An out-of-range node
 * latches LBM_ERR_INVALID_ARG in the status word and is skipped; a non-finite
 * loss latches LBM_ERR_NONFINITE. */
LBM_API lbm_status lbm_probe_loss_grad(lbm_plan* plan, const void* d_f, int64_t n_probe, const int64_t* d_probe_node,
                                       const double* d_rho_target, double weight, double* d_loss, void* d_lambda,
                                       void* d_ws, void* stream);

/* Cubic-spline inlet profiles (section 3.1.2: the multi-parameter inversion
 * imposes the inlet pressure as a cubic spline through a few inlet
 * densities).  Knot values c[Kz][Ky] give
 *   rho_in[z ny + y] = rho_out + sum_{b,a} Bz[z][b] By[y][a] c[b][a],
 * By (Bz) the natural cubic spline basis over the rows (layers): column a is
 * the spline through the a-th unit knot vector, knots evenly spaced at
 * t_a = a (n - 1) / (K - 1), zero second derivative at both ends; K = 1 is a
 * constant.  D2Q9 plans use Kz = 1 and Bz = {1}.
 * lbm_spline_basis: host function, writes h_basis[n][n_knots] (row-major).
 *   Errors: INVALID_ARG unless 1 <= n_knots <= n <= 2^20.
 * lbm_spline_profile: d_by double[ny][ky], d_bz double[nz][kz], d_knots
 *   double[kz][ky] -> d_rho_in double[ny nz].
 * lbm_spline_grad: d_grad_rho_in double[ny nz] (from lbm_adjoint) ->
 *   d_grad_knots double[kz][ky] = Bz^T G By, each entry summed in a fixed
 *   order (deterministic).
 * Both need a plan with LBM_INLET_PROFILE and 1 <= ky <= ny, 1 <= kz <= nz
 * (else INVALID_ARG); asynchronous on the stream. */
LBM_API lbm_status lbm_spline_basis(int32_t n_knots, int32_t n, double* h_basis);
LBM_API lbm_status lbm_spline_profile(const lbm_plan* plan, int32_t ky, int32_t kz, const double* d_by,
                                      const double* d_bz, const double* d_knots, double rho_out, double* d_rho_in,
                                      void* stream);
LBM_API lbm_status lbm_spline_grad(const lbm_plan* plan, int32_t ky, int32_t kz, const double* d_by,
                                   const double* d_bz, const double* d_grad_rho_in, double* d_grad_knots,
                                   void* stream);

/* Reverse sweep from lambda^T to t = 0 through the checkpoints left in d_ws
 * by the last lbm_forward with the same parameters: recompute each segment,
 * then run the adjoint step backwards through it.
 *  d_lambda       lambda^T (plan precision; not modified)
 *  d_grad_rho_in  double[1 or ny nz] out: dL/drho_in
 *  d_grad_tau     double[1] out: dL/dtau
 * Gradient sums are FP64 in a fixed order (deterministic run to run). */
LBM_API lbm_status lbm_adjoint(lbm_plan* plan, const double* d_rho_in, const double* d_tau, double rho_out,
                       const void* d_lambda, double* d_grad_rho_in, double* d_grad_tau, void* d_ws, void* stream);

/* A loss over a time window (the wake of section 3.4 observed over time):
 * L = sum_k L_k(f^{t_k}), each L_k the plan's final-step loss (kind,
 * normalisation, ROI of lbm_loss_grad) of the state at step t_k against the
 * k-th target, and its gradient with respect to rho_in and tau, in ONE
 * reverse sweep: lambda^T is the seed of the observations at T, and the seed
 * of each observation at t_k < T is added to lambda^{t_k} right after the
 * adjoint step that produces it (f^{t_k} comes from the recomputed segment
 * state).  Call after lbm_forward with the same parameters.
 *  d_f             f^T from that lbm_forward (dense, plan precision)
 *  n_obs           number of observations (1 .. 65536)
 *  h_obs_steps     int32[n_obs] HOST array of the steps t_k, 1 <= t_k <= T
 *  d_u_targets     double[n_obs][D][N] the observed velocity fields
 *  d_roi           uint8[N] region of interest (nullable: all fluid nodes)
 *  d_scratch_f, d_scratch_lambda   dense Q N scratch states (plan precision)
 *  d_loss          double[1] out: L
 *  d_grad_rho_in, d_grad_tau       out, as lbm_adjoint
 * Errors: INVALID_ARG (null pointers, n_obs or a step out of range), CUDA. */
LBM_API lbm_status lbm_adjoint_window(lbm_plan* plan, const double* d_rho_in, const double* d_tau, double rho_out,
                                      const void* d_f, int32_t n_obs, const int32_t* h_obs_steps,
                                      const double* d_u_targets, const uint8_t* d_roi, void* d_scratch_f,
                                      void* d_scratch_lambda, double* d_loss, double* d_grad_rho_in,
                                      double* d_grad_tau, void* d_ws, void* stream);

/* Moments (Eq. 1-2) in FP64: d_rho double[N] (nullable), d_u double[D N].
 * Solid nodes report rho = 0 and u = 0. */
LBM_API lbm_status lbm_macroscopic(lbm_plan* plan, const void* d_f, double* d_rho, double* d_u, void* stream);

/* Darcy permeability (Eq. 12) of a steady state: k = nu J / (dp/dx) with
 * J = (1 / (ny nz)) sum over section x = xs of rho u_x (solids give 0),
 * nu = (tau - 1/2) / 3 (Eq. 9) and dp/dx = (mean rho_in - rho_out) / (3 nx).
 *  d_k, d_flux   double[1] out (d_flux nullable). */
LBM_API lbm_status lbm_darcy(lbm_plan* plan, const void* d_f, const double* d_rho_in, const double* d_tau, double rho_out,
                     int32_t xs, double* d_k, double* d_flux, void* stream);

/* One Adam step (the optimiser of section 2.2 / 3.4) on a scaled parameter
 * vector: p = p_offset + p_scale * theta.  Reads dL/dp, updates theta, m, v
 * in place and writes p.  t is the 1-based step count.  n <= 65536. */
LBM_API lbm_status lbm_adam_step(int32_t n, double* d_theta, double* d_m, double* d_v, const double* d_grad_p, double* d_p,
                         double p_offset, double p_scale, int32_t t, double lr, double beta1, double beta2,
                         double eps, void* stream);

/* ---------------------------------------------------------------- batches
 * Many independent lattices (instances) of different sizes advanced together:
 * every time step is one kernel over the row segments of all instances, so
 * a batch of small lattices keeps the whole GPU busy.  All instances share Q,
 * precision, T, the checkpoint stride, the loss kind and normalisation and
 * the inlet kind of the common descriptor (its nx, ny, nz are ignored).
 * Packed layouts (element offsets from lbm_batch_layout, each 256-byte
 * aligned): populations of instance i at state_off[i] ([Q][N_i], shifted,
 * plan precision); node fields (mask, link words) at node_off[i]; velocity
 * fields at vel_off[i] ([D][N_i], double); inlet densities and their
 * gradients at inlet_off[i] (1 or ny_i nz_i entries); tau, loss, dL/dtau,
 * porosity one double per instance (info: four int64 per instance). */
typedef struct lbm_batch lbm_batch;

/* n >= 1 instances with sizes nx[i], ny[i], nz[i] (nz = 1 for D2Q9); every
 * nx[i] must be a multiple of 4 (D2Q9 FP32) or 2 (otherwise).
 * Errors: INVALID_ARG as lbm_plan_create, per instance. */
LBM_API lbm_status lbm_batch_create(const lbm_desc* common, int32_t n, const int32_t* nx, const int32_t* ny,
                                    const int32_t* nz, lbm_batch** out);
LBM_API lbm_status lbm_batch_destroy(lbm_batch* batch);

/* Host arrays of n + 1 element offsets (the last entry is the total) and the
 * workspace bytes.  Any pointer may be NULL. */
LBM_API lbm_status lbm_batch_layout(const lbm_batch* batch, int64_t* state_off, int64_t* node_off, int64_t* vel_off,
                                    int64_t* inlet_off, size_t* ws_bytes);

/* lbm_init_geometry for every instance (g: n descriptors), then the batch's
 * work-unit tables are written into d_ws (which must then stay with the
 * batch).  d_mask, d_link, d_porosity, d_info packed as above. */
LBM_API lbm_status lbm_batch_init_geometry(lbm_batch* batch, const lbm_geom_desc* g, uint8_t* d_mask,
                                           uint32_t* d_link, double* d_porosity, int64_t* d_info, void* d_ws,
                                           void* stream);

/* T steps from rest for every instance (lbm_forward, batched); d_tau: n. */
LBM_API lbm_status lbm_batch_forward(lbm_batch* batch, const double* d_rho_in, const double* d_tau, double rho_out,
                                     void* d_f, void* d_ws, void* stream);

/* Per-instance loss (d_loss: n) and seed lambda^T (packed like d_f). */
LBM_API lbm_status lbm_batch_loss_grad(lbm_batch* batch, const void* d_f, const double* d_u_target,
                                       const uint8_t* d_roi, double* d_loss, void* d_lambda, void* d_ws,
                                       void* stream);

/* Reverse sweep for every instance (lbm_adjoint, batched): dL/drho_in packed
 * by inlet_off, dL/dtau one per instance. */
LBM_API lbm_status lbm_batch_adjoint(lbm_batch* batch, const double* d_rho_in, const double* d_tau, double rho_out,
                                     const void* d_lambda, double* d_grad_rho_in, double* d_grad_tau, void* d_ws,
                                     void* stream);

/* Fluid-only layout for a batch (the single-lattice lbm_compact_* calls,
 * batched): the fluid nodes of every instance packed into one compact state,
 * each instance's range padded to a multiple of 256 nodes so that every
 * thread block of the step and adjoint kernels belongs to one instance; per
 * fluid-node update the kernels move 2 Q populations plus the neighbour
 * table instead of every node of every instance.  Each instance gets bit for
 * bit the populations and gradients a single plan in the compact layout
 * computes.  The layout is internal: the batch calls keep taking and
 * returning the packed dense arrays of lbm_batch_layout, and the workspace
 * size does not change.
 * lbm_batch_compact_size: bytes of the table buffer for n_fluid[i] fluid
 *   nodes per instance (host array of n; d_info[4 i + 3] of
 *   lbm_batch_init_geometry).
 * lbm_batch_compact_bind: builds the tables into d_tables (device,
 *   caller-owned, 256-byte aligned, lbm_batch_compact_size bytes, valid while
 *   the batch uses them) from the link words, using d_ws (the workspace given
 *   to lbm_batch_init_geometry) as scratch, and switches the batch to the
 *   fluid-only layout.  Synchronises the stream (it checks every n_fluid[i]
 *   against the link words).  n_fluid = NULL switches back to the dense
 *   layout.  A new lbm_batch_init_geometry switches back as well.
 * Errors: INVALID_ARG (geometry not initialised on d_ws, a count out of
 *   range or not the instance's fluid count, misaligned d_tables), CUDA. */
LBM_API lbm_status lbm_batch_compact_size(const lbm_batch* batch, const int64_t* n_fluid, size_t* bytes);
LBM_API lbm_status lbm_batch_compact_bind(lbm_batch* batch, const int64_t* n_fluid, void* d_tables, void* d_ws,
                                          void* stream);

/* Reads (synchronously) and clears the batch's device status word in d_ws
 * (a non-finite loss or gradient of any instance latches
 * LBM_ERR_NONFINITE). */
LBM_API lbm_status lbm_batch_get_status(lbm_batch* batch, void* d_ws, lbm_status* status);

/* Reads (synchronously) and clears the plan's device status word. */
LBM_API lbm_status lbm_get_status(lbm_plan* plan, lbm_status* status);

/* Static message for a status code. */
LBM_API const char* lbm_error_string(lbm_status status);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
