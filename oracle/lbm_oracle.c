/*
 * Oracle: a plain, slow, obviously-correct FP64 CPU statement of the
 * lattice Boltzmann method of arXiv 2310.00810 and of its reverse sweep.
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never
 * links, includes or calls anything in this directory, and nothing here
 * includes anything from the product tree.
 *
 * What it computes (the paper's notation; section 2.1):
 *   Eq. 1-2   rho = sum_i f_i ,  rho u = sum_i f_i c_i          (i = 0..Q-1)
 *   Eq. 3-4   f_i(x + c_i, t + 1) = f_i(x, t) - (f_i - f_i^eq) / tau
 *   Eq. 5     f_i^eq = w_i rho (1 + u.c_i/c_s^2 + (u.c_i)^2/(2 c_s^4)
 *                                  - u.u/(2 c_s^2)),      c_s^2 = 1/3
 *   Eq. 6     anti-bounce-back at the inlet/outlet planes:
 *             f_i(x_b, t+1) = -f*_opp(i)(x_b, t)
 *                             + 2 w_i rho_w (1 + (u.c_i)^2/(2 c_s^4) - u.u/(2 c_s^2))
 *   "Bounce Back" stage (section 2.2): halfway, link-wise bounce-back at
 *   grain nodes and at the walls y = -1/2, ny - 1/2 (and z = -1/2, nz - 1/2).
 * Readings of garbled or silent passages (Eq. 1-2, Eq. 4, section 3.2, Eq. 6,
 * and the "Bounce Back" stage of section 2.2): sums run
 * over i = 0..Q-1; the BGK sign is -(f - f^eq)/tau; c_s^2 = 1/3; u_w in
 * Eq. 6 is the boundary node's own velocity at time t (or, as an option,
 * that velocity extrapolated to the pressure plane: set_abb_velocity); a
 * link that crosses a wall plane and a pressure plane at once bounces back;
 * solid nodes carry no populations.
 *
 * Density probes (an optional second loss term): w sum_p (rho(x_p) - rho_p)^2
 * over a list of probe nodes, with its seed dL/df_k = 2 w (rho - rho_p).
 *
 * Options for the cylinder-wake flow of section 3.4: periodic top and bottom
 * (set_periodic_y: links leaving y = -1/2 or ny - 1/2 re-enter on the other
 * side instead of bouncing back) and a velocity inlet (set_velocity_inlet:
 * the links through x = -1/2 take the moving-wall bounce-back
 * f_i = f*_opp(i) + 6 w_i rho_0 (c_i . u_in), rho_0 = 1, in place of Eq. 6;
 * the outlet keeps Eq. 6).
 *
 * MRT collision (section 3.4, Eq. 16-18; D2Q9 only, an option set by
 * set_collision): f* = f - M^{-1} S M (f - f^eq), M the moment matrix of
 * Eq. 18 (rows rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy; the printed
 * p_xy row |c_x c_y| is read as the orthogonal c_x c_y), m^eq = M f^eq with
 * f^eq of Eq. 5, S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, 1/tau, 1/tau) (the
 * conserved moments have m = m^eq, so their rates do not matter).  S = I / tau
 * is BGK.
 *
 * Loss (Eq. 7, Eq. 15, and the compute_loss kernel of section 2.2), taken at
 * the final step only; default is the vector mismatch sum |u - u_t|^2,
 * optional is the paper's (|u| - |u_t|)^2.
 *
 * The reverse sweep is the exact transpose of one step, written as the
 * reverse of the forward operations in scatter form: streaming transposed
 * link by link, then the collision Jacobian through the moments.  It
 * replaces the Taichi tape of section 2.2 and is pinned in the tests by
 * complex-step derivatives of the forward alone (no shared formulas).
 *
 * Compiled twice: REAL = double (liboracle) and, with -DORC_COMPLEX,
 * REAL = double _Complex (liboracle_cs) for complex-step differentiation of
 * the forward and the loss.  Built with -O2 -ffp-contract=off and without
 * -ffast-math so that every operation is a plain IEEE round-to-nearest op.
 *
 * Array layouts (dense, x fastest):
 *   node index n = (z * ny + y) * nx + x,  N = nx * ny * nz
 *   f[i * N + n]      populations, UNshifted (f, not f - w)
 *   u[a * N + n]      velocity components, a = 0..D-1
 *   mask[n]           0 = fluid, nonzero = solid
 *   rho_in[]          inlet density: one value (const) or ny * nz values,
 *                     indexed [z * ny + y] (profile)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef ORC_COMPLEX
#include <complex.h>
typedef double _Complex real_t;
#define RE(v) creal(v)
#define SYM(name) orc_cs_##name
#else
typedef double real_t;
#define RE(v) (v)
#define SYM(name) orc_##name
#endif

/* ---------------------------------------------------------------- lattice */

typedef struct {
    int q, d;
    int c[19][3];
    double w[19];
    int opp[19];
} lattice;

/* D2Q9 in the order of Fig. 1 and of the MRT matrix of Eq. 18 (its j_x and
 * j_y rows): rest, the four axis links E N W S, then NE NW SW SE.
 * D3Q19: rest, six axis links, twelve edge links (the paper gives no order). */
static int lattice_make(int q, lattice* L)
{
    static const int c9[9][3] = {
        {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
        {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    static const int c19[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    memset(L, 0, sizeof(*L));
    if (q == 9) {
        L->q = 9;
        L->d = 2;
        memcpy(L->c, c9, sizeof(c9));
    } else if (q == 19) {
        L->q = 19;
        L->d = 3;
        memcpy(L->c, c19, sizeof(c19));
    } else {
        return -1;
    }
    for (int i = 0; i < L->q; ++i) {
        int len2 = L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2];
        if (q == 9)
            L->w[i] = len2 == 0 ? 4.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else
            L->w[i] = len2 == 0 ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        L->opp[i] = -1;
        for (int j = 0; j < L->q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    return 0;
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the per-node loops of the step and the adjoint step (1 =
 * serial).  Every sum over nodes is taken serially in node order, so results
 * do not depend on the thread count. */
int SYM(set_threads)(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
    return n;
#else
    (void)n;
    return 1;
#endif
}

/* Exported copies of the tables, for the isotropy pins in the tests. */
int SYM(lattice)(int q, int* c_out /* q*3 */, double* w_out, int* opp_out)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    for (int i = 0; i < L.q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = L.c[i][a];
        w_out[i] = L.w[i];
        opp_out[i] = L.opp[i];
    }
    return 0;
}

/* ----------------------------------------------------------------- domain */

typedef struct {
    int nx, ny, nz;
    long n;
    const uint8_t* mask;
} domain;

enum { LINK_FLUID = 0, LINK_BB = 1, LINK_ABB_IN = 2, LINK_ABB_OUT = 3 };

static int g_periodic_y = 0;
static int g_vel_inlet = 0;
static double g_u_in[3] = {0, 0, 0};

int SYM(set_periodic_y)(int on)
{
    g_periodic_y = on ? 1 : 0;
    return 0;
}

int SYM(set_velocity_inlet)(int on, double ux, double uy, double uz)
{
    g_vel_inlet = on ? 1 : 0;
    g_u_in[0] = ux;
    g_u_in[1] = uy;
    g_u_in[2] = uz;
    return 0;
}

/* A gradual start of the velocity inlet (the flow of section 3.4 from rest):
 * the step that produces f^t uses u_in r(t) with r(t) = sin^2(pi t / (2 t_r))
 * for t < t_r and 1 from t_r on (t_r = 0: no ramp).  step() produces the
 * time level g_time_next; forward() and gradient() set it step by step,
 * set_time sets it for a lone step() call. */
static int g_ramp_steps = 0;
static int g_time_next = 1;

int SYM(set_velocity_ramp)(int steps)
{
    if (steps < 0) return -1;
    g_ramp_steps = steps;
    return 0;
}

int SYM(set_time)(int t_next)
{
    g_time_next = t_next;
    return 0;
}

static double ramp_factor(int t)
{
    if (g_ramp_steps <= 0 || t >= g_ramp_steps) return 1.0;
    if (t <= 0) return 0.0;
    const double pi = 3.14159265358979323846;
    const double s = sin(pi * (double)t / (2.0 * (double)g_ramp_steps));
    return s * s;
}

/* What node (x,y,z) receives in direction i: the population streaming along
 * the link from x - c_i.  Wall planes (y, z) win over pressure planes (x);
 * with periodic y a link leaving the y range re-enters on the other side. */
static int classify(const domain* D, const lattice* L, int x, int y, int z, int i, long* src)
{
    int sx = x - L->c[i][0], sy = y - L->c[i][1], sz = z - L->c[i][2];
    if (g_periodic_y) sy = (sy + D->ny) % D->ny;
    if (sy < 0 || sy >= D->ny || sz < 0 || sz >= D->nz) return LINK_BB;
    if (sx < 0) return LINK_ABB_IN;
    if (sx >= D->nx) return LINK_ABB_OUT;
    long s = ((long)sz * D->ny + sy) * D->nx + sx;
    if (D->mask && D->mask[s]) return LINK_BB;
    *src = s;
    return LINK_FLUID;
}

static int is_solid(const domain* D, long n) { return D->mask && D->mask[n]; }

/* 1/c_s^2 = 3, 1/(2 c_s^4) = 4.5, 1/(2 c_s^2) = 1.5 for c_s^2 = 1/3 (Eq. 5, Eq. 9-10). */
#define INV_CS2 3.0
#define INV_2CS4 4.5
#define INV_2CS2 1.5

/* Eq. 1-2 at one node. */
static void moments(const lattice* L, const real_t* f, long N, long n, real_t* rho, real_t u[3])
{
    real_t r = 0, m[3] = {0, 0, 0};
    for (int i = 0; i < L->q; ++i) {
        real_t fi = f[(long)i * N + n];
        r += fi;
        for (int a = 0; a < L->d; ++a) m[a] += fi * (double)L->c[i][a];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = a < L->d ? m[a] / r : 0;
}

static real_t dot_cu(const lattice* L, int i, const real_t u[3])
{
    real_t s = 0;
    for (int a = 0; a < L->d; ++a) s += (double)L->c[i][a] * u[a];
    return s;
}

static real_t dot_uu(const lattice* L, const real_t u[3])
{
    real_t s = 0;
    for (int a = 0; a < L->d; ++a) s += u[a] * u[a];
    return s;
}

/* Eq. 5 */
static real_t feq(const lattice* L, int i, real_t rho, const real_t u[3])
{
    real_t cu = dot_cu(L, i, u), uu = dot_uu(L, u);
    return L->w[i] * rho * (1.0 + cu * INV_CS2 + cu * cu * INV_2CS4 - uu * INV_2CS2);
}

/* Eq. 6: the part added to -f*_opp(i). */
static real_t abb_source(const lattice* L, int i, real_t rho_w, const real_t u[3])
{
    real_t cu = dot_cu(L, i, u), uu = dot_uu(L, u);
    return 2.0 * L->w[i] * rho_w * (1.0 + cu * cu * INV_2CS4 - uu * INV_2CS2);
}

static real_t inlet_rho(const real_t* rho_in, int profile, const domain* D, int y, int z)
{
    return profile ? rho_in[(long)z * D->ny + y] : rho_in[0];
}

/* Where u in Eq. 6 is taken.  The paper writes the boundary term with a bare
 * u.  UW_NODE: the boundary node's own velocity at time t.  UW_EXTRAP: that
 * velocity extrapolated linearly to the pressure plane half a link outside
 * the node, u_w = u(x_b) + (u(x_b) - u(x_b + e)) / 2 with x_b + e the next
 * node inward (x = 1 for the inlet node, nx - 2 for the outlet node); where
 * that node is solid, u_w = u(x_b). */
enum { UW_NODE = 0, UW_EXTRAP = 1 };
static int g_uw_mode = UW_NODE;

int SYM(set_abb_velocity)(int mode)
{
    if (mode != UW_NODE && mode != UW_EXTRAP) return -1;
    g_uw_mode = mode;
    return 0;
}

/* The inward neighbour whose velocity enters u_w at boundary node n (at x),
 * or -1 when u_w is the node's own velocity. */
static long wall_partner(const domain* D, int x, long n)
{
    if (g_uw_mode != UW_EXTRAP) return -1;
    long m = x == 0 ? n + 1 : n - 1;
    return is_solid(D, m) ? -1 : m;
}

/* ------------------------------------------------------------- MRT */

enum { COLL_BGK = 0, COLL_MRT = 1 };
static int g_coll = COLL_BGK;
static double g_s_e = 1.0, g_s_eps = 1.0, g_s_q = 1.0;

int SYM(set_collision)(int mode, double s_e, double s_eps, double s_q)
{
    if (mode != COLL_BGK && mode != COLL_MRT) return -1;
    g_coll = mode;
    g_s_e = s_e;
    g_s_eps = s_eps;
    g_s_q = s_q;
    return 0;
}

/* Row r of the D2Q9 moment matrix at direction j, from its polynomial in c_j
 * (Gram-Schmidt over the lattice, the construction behind Eq. 18). */
static double mrt_row(const lattice* L, int r, int j)
{
    double cx = L->c[j][0], cy = L->c[j][1], c2 = cx * cx + cy * cy;
    switch (r) {
    case 0: return 1.0;
    case 1: return -4.0 + 3.0 * c2;
    case 2: return 4.0 - 10.5 * c2 + 4.5 * c2 * c2;
    case 3: return cx;
    case 4: return (-5.0 + 3.0 * c2) * cx;
    case 5: return cy;
    case 6: return (-5.0 + 3.0 * c2) * cy;
    case 7: return cx * cx - cy * cy;
    default: return cx * cy;
    }
}

/* Relaxation rate of moment r for omega = 1/tau. */
static real_t mrt_rate(int r, real_t omega)
{
    switch (r) {
    case 1: return g_s_e;
    case 2: return g_s_eps;
    case 4:
    case 6: return g_s_q;
    case 7:
    case 8: return omega;
    default: return 0.0;
    }
}

/* |row r|^2 = sum_j M_rj^2 (M M^T is diagonal, so M^{-1} = M^T diag(1/|row|^2)). */
static double mrt_norm2(const lattice* L, int r)
{
    double s = 0;
    for (int j = 0; j < 9; ++j) s += mrt_row(L, r, j) * mrt_row(L, r, j);
    return s;
}

/* --------------------------------------------------------- collision */

/* Post-collision populations of one node (BGK, Eq. 4-5, or MRT, Eq. 16). */
static void collide_node(const lattice* L, const real_t* f, long N, long n, real_t tau, real_t* out, long ostride,
                         long on)
{
    real_t rho, u[3];
    moments(L, f, N, n, &rho, u);
    if (g_coll == COLL_MRT && L->q == 9) {
        real_t d[9], dm[9];
        for (int j = 0; j < 9; ++j) d[j] = f[(long)j * N + n] - feq(L, j, rho, u);
        for (int r = 0; r < 9; ++r) {
            real_t m = 0;
            for (int j = 0; j < 9; ++j) m += mrt_row(L, r, j) * d[j];
            dm[r] = mrt_rate(r, 1.0 / tau) * m / mrt_norm2(L, r);
        }
        for (int j = 0; j < 9; ++j) {
            real_t c = 0;
            for (int r = 0; r < 9; ++r) c += mrt_row(L, r, j) * dm[r];
            out[(long)j * ostride + on] = f[(long)j * N + n] - c;
        }
        return;
    }
    for (int i = 0; i < L->q; ++i) {
        real_t fi = f[(long)i * N + n];
        out[(long)i * ostride + on] = fi - (fi - feq(L, i, rho, u)) / tau;
    }
}

/* The collision alone (BGK, Eq. 4-5: f_out_i = f_i - (f_i - f^eq_i) / tau,
 * or MRT, Eq. 16) at every node of an unstructured array of n nodes. */
int SYM(collide)(int q, long n_nodes, const real_t* f_in, real_t* f_out, const real_t* tau)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    if (g_coll == COLL_MRT && q != 9) return -4;
    for (long n = 0; n < n_nodes; ++n) collide_node(&L, f_in, n_nodes, n, *tau, f_out, n_nodes, n);
    return 0;
}

/* f^eq (Eq. 5) for given rho[n] and u[a * n_nodes + n]. */
int SYM(equilibrium)(int q, long n_nodes, const real_t* rho, const real_t* u, real_t* f_out)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    for (long n = 0; n < n_nodes; ++n) {
        real_t uu[3] = {0, 0, 0};
        for (int a = 0; a < L.d; ++a) uu[a] = u[(long)a * n_nodes + n];
        for (int i = 0; i < q; ++i) f_out[(long)i * n_nodes + n] = feq(&L, i, rho[n], uu);
    }
    return 0;
}

/* ------------------------------------------------------------- one step */

/* f_out = stream(collide(f_in)): collision (Eq. 4-5) at every fluid node,
 * then pull streaming with halfway bounce-back and anti-bounce-back (Eq. 3,
 * Eq. 6).  Solid nodes are copied through unchanged. */
int SYM(step)(int q, int nx, int ny, int nz, const uint8_t* mask, const real_t* f_in, real_t* f_out,
              const real_t* rho_in, int inlet_profile, const real_t* rho_out, const real_t* tau)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    if (g_coll == COLL_MRT && q != 9) return -4;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    long N = D.n;
    real_t* fstar = (real_t*)malloc(sizeof(real_t) * (size_t)q * (size_t)N);
    real_t* uvel = (real_t*)malloc(sizeof(real_t) * 3 * (size_t)N);
    if (!fstar || !uvel) {
        free(fstar);
        free(uvel);
        return -2;
    }

    /* collision (nodes are independent: shared among OpenMP threads) */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (is_solid(&D, n)) continue;
        real_t rho, u[3];
        moments(&L, f_in, N, n, &rho, u);
        for (int a = 0; a < 3; ++a) uvel[a * N + n] = u[a];
        collide_node(&L, f_in, N, n, *tau, fstar, N, n);
    }

    /* streaming with boundaries (each node writes only its own populations) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                if (is_solid(&D, n)) {
                    for (int i = 0; i < q; ++i) f_out[(long)i * N + n] = f_in[(long)i * N + n];
                    continue;
                }
                real_t u[3] = {uvel[n], uvel[N + n], uvel[2 * N + n]};
                if (x == 0 || x == nx - 1) {
                    long m = wall_partner(&D, x, n);
                    if (m >= 0)
                        for (int a = 0; a < 3; ++a) u[a] = 1.5 * u[a] - 0.5 * uvel[(long)a * N + m];
                }
                for (int i = 0; i < q; ++i) {
                    long s = -1;
                    int cls = classify(&D, &L, x, y, z, i, &s);
                    real_t v;
                    if (cls == LINK_FLUID) {
                        v = fstar[(long)i * N + s];
                    } else if (cls == LINK_BB) {
                        v = fstar[(long)L.opp[i] * N + n];
                    } else if (cls == LINK_ABB_IN && g_vel_inlet) {
                        double cu = 0;
                        for (int a = 0; a < L.d; ++a) cu += L.c[i][a] * g_u_in[a];
                        v = fstar[(long)L.opp[i] * N + n] + 6.0 * L.w[i] * cu * ramp_factor(g_time_next);
                    } else {
                        real_t rw = cls == LINK_ABB_IN ? inlet_rho(rho_in, inlet_profile, &D, y, z) : *rho_out;
                        v = -fstar[(long)L.opp[i] * N + n] + abb_source(&L, i, rw, u);
                    }
                    f_out[(long)i * N + n] = v;
                }
            }
    free(fstar);
    free(uvel);
    return 0;
}

/* f^0: the fluid at rest with rho = 1 (init_field of section 2.2, and the
 * initial density of 1 mu/lu^3 of section 3.2): f_i = w_i everywhere. */
static void rest_state(const lattice* L, long N, real_t* f)
{
    for (int i = 0; i < L->q; ++i)
        for (long n = 0; n < N; ++n) f[(long)i * N + n] = L->w[i];
}

/* T steps from f0 (NULL: rest).  If tape != NULL it receives f^0..f^{T-1}
 * (T * Q * N values) for the reverse sweep. */
int SYM(forward)(int q, int nx, int ny, int nz, const uint8_t* mask, const real_t* rho_in, int inlet_profile,
                 const real_t* rho_out, const real_t* tau, int T, const real_t* f0, real_t* fT, real_t* tape)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    long N = (long)nx * ny * nz, QN = (long)q * N;
    real_t* a = (real_t*)malloc(sizeof(real_t) * (size_t)QN);
    real_t* b = (real_t*)malloc(sizeof(real_t) * (size_t)QN);
    if (!a || !b) {
        free(a);
        free(b);
        return -2;
    }
    if (f0)
        memcpy(a, f0, sizeof(real_t) * (size_t)QN);
    else
        rest_state(&L, N, a);
    for (int t = 0; t < T; ++t) {
        if (tape) memcpy(tape + (long)t * QN, a, sizeof(real_t) * (size_t)QN);
        g_time_next = t + 1;
        int rc = SYM(step)(q, nx, ny, nz, mask, a, b, rho_in, inlet_profile, rho_out, tau);
        if (rc) {
            free(a);
            free(b);
            return rc;
        }
        real_t* tmp = a;
        a = b;
        b = tmp;
    }
    memcpy(fT, a, sizeof(real_t) * (size_t)QN);
    free(a);
    free(b);
    return 0;
}

/* Macroscopic fields (Eq. 1-2); solid nodes report rho = 0 and u = 0. */
int SYM(macroscopic)(int q, int nx, int ny, int nz, const uint8_t* mask, const real_t* f, real_t* rho_out,
                     real_t* u_out)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    long N = D.n;
    for (long n = 0; n < N; ++n) {
        real_t rho = 0, u[3] = {0, 0, 0};
        if (!is_solid(&D, n)) moments(&L, f, N, n, &rho, u);
        if (rho_out) rho_out[n] = rho;
        for (int a = 0; a < L.d; ++a) u_out[(long)a * N + n] = u[a];
    }
    return 0;
}

/* ------------------------------------------------------------------ loss */

enum { LOSS_VEC = 0, LOSS_NORM = 1 };
enum { NORM_SUM = 0, NORM_MEAN_FLUID = 1 };

/* Loss on the velocity of state f (the final step, section 3.1.2).
 *   LOSS_VEC : sum over ROI fluid nodes of |u - u_t|^2
 *   LOSS_NORM: sum over ROI fluid nodes of (|u| - |u_t|)^2   (Eq. 7, compute_loss)
 * NORM_MEAN_FLUID divides by the number of ROI fluid nodes (Eq. 15).
 * If lam != NULL it receives dL/df (zero at solid and non-ROI nodes):
 *   dL/df_k = sum_a dL/du_a (c_ka - u_a) / rho. */
int SYM(loss)(int q, int nx, int ny, int nz, const uint8_t* mask, const real_t* f, const double* u_target,
              const uint8_t* roi, int kind, int norm, real_t* loss_out, real_t* lam)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    long N = D.n, count = 0;
    for (long n = 0; n < N; ++n)
        if (!is_solid(&D, n) && (!roi || roi[n])) ++count;
    double weight = (norm == NORM_MEAN_FLUID) ? (count > 0 ? 1.0 / (double)count : 0.0) : 1.0;
    real_t total = 0;
    if (lam)
        for (long k = 0; k < (long)q * N; ++k) lam[k] = 0;
    for (long n = 0; n < N; ++n) {
        if (is_solid(&D, n) || (roi && !roi[n])) continue;
        real_t rho, u[3];
        moments(&L, f, N, n, &rho, u);
        real_t du[3] = {0, 0, 0};
        if (kind == LOSS_VEC) {
            for (int a = 0; a < L.d; ++a) {
                real_t e = u[a] - u_target[(long)a * N + n];
                total += weight * e * e;
                du[a] = 2.0 * weight * e;
            }
        } else {
            real_t uu = dot_uu(&L, u);
            double tt = 0;
            for (int a = 0; a < L.d; ++a) tt += u_target[(long)a * N + n] * u_target[(long)a * N + n];
#ifdef ORC_COMPLEX
            real_t un = csqrt(uu);
#else
            real_t un = sqrt(uu);
#endif
            real_t e = un - sqrt(tt);
            total += weight * e * e;
            /* d|u|/du = u/|u|, taken as 0 at u = 0 exactly */
            if (RE(uu) != 0.0)
                for (int a = 0; a < L.d; ++a) du[a] = 2.0 * weight * e * u[a] / un;
        }
        if (lam)
            for (int k = 0; k < q; ++k) {
                real_t s = 0;
                for (int a = 0; a < L.d; ++a) s += du[a] * ((double)L.c[k][a] - u[a]);
                lam[(long)k * N + n] = s / rho;
            }
    }
    *loss_out = total;
    return 0;
}

/* Density probes, a second loss term for the joint inversion of the head and
 * tau (the Stokes-regime velocity fixes only their ratio):
 *   L_p = w sum_p (rho(x_p) - rho_p)^2     (p = 0..n_probe-1, x_p a dense node index)
 * A solid probe node contributes nothing.  If lam != NULL the seed
 * dL_p/df_k(x_p) = 2 w (rho - rho_p) (Eq. 1: drho/df_k = 1) is ADDED to lam. */
int SYM(probe_loss)(int q, int nx, int ny, int nz, const uint8_t* mask, const real_t* f, long n_probe,
                    const int64_t* node, const double* rho_target, double weight, real_t* loss_out, real_t* lam)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    long N = D.n;
    real_t total = 0;
    for (long p = 0; p < n_probe; ++p) {
        long n = (long)node[p];
        if (n < 0 || n >= N) return -3;
        if (is_solid(&D, n)) continue;
        real_t rho, u[3];
        moments(&L, f, N, n, &rho, u);
        real_t e = rho - rho_target[p];
        total += weight * e * e;
        if (lam)
            for (int k = 0; k < q; ++k) lam[(long)k * N + n] += 2.0 * weight * e;
    }
    *loss_out = total;
    return 0;
}

#ifndef ORC_COMPLEX
/* --------------------------------------------------------- link words */

/* The per-node link word the library reports with its geometry: bit 31 set
 * for a solid node (and nothing else); for a fluid node, bit i (i < Q) set
 * iff what the node receives in direction i comes from halfway bounce-back
 * (the link from x - c_i crosses a wall plane or starts at a solid node). */
int orc_links(int q, int nx, int ny, int nz, const uint8_t* mask, uint32_t* link)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                if (is_solid(&D, n)) {
                    link[n] = 1u << 31;
                    continue;
                }
                uint32_t w = 0;
                for (int i = 0; i < q; ++i) {
                    long s = -1;
                    if (classify(&D, &L, x, y, z, i, &s) == LINK_BB) w |= 1u << i;
                }
                link[n] = w;
            }
    return 0;
}

/* ------------------------------------------------------ reverse sweep */

/* One reverse step: given f^t and lam_next = dL/df^{t+1}, write
 * lam_out = dL/df^t and ADD this step's contributions to dL/drho_in
 * (per inlet entry, or into g_rho_in[0] for a constant head) and dL/domega,
 * omega = 1/tau.  The forward step is undone operation by operation:
 *  1. streaming: each link's transpose scatters lam_next back to the
 *     post-collision population it was copied from (with the sign of Eq. 6
 *     for anti-bounce-back links), and the Eq. 6 source contributes to
 *     rho_w and to the boundary node's u;
 *  2. collision: f*_j = f_j - sum_k A_jk (f_k - f^eq_k(rho(f), u(f))), with
 *     A = omega I (BGK) or A = M^{-1} S M (MRT), so with nu = A^T mu
 *     dL/df_k = mu_k - nu_k + rhobar + sum_a ubar_a (c_ka - u_a)/rho
 *     with rhobar = sum_j nu_j df^eq_j/drho and
 *     ubar_a = (Eq. 6 part) + sum_j nu_j df^eq_j/du_a; dL/domega is
 *     -mu . dA/domega (f - f^eq). */
int orc_adjoint_step(int q, int nx, int ny, int nz, const uint8_t* mask, const double* f_t,
                     const double* lam_next, double* lam_out, const double* rho_in, int inlet_profile,
                     const double* rho_out, const double* tau, double* g_rho_in, double* g_omega)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    long N = D.n, QN = (long)q * N;
    double omega = 1.0 / *tau;
    double* mu = (double*)calloc((size_t)QN, sizeof(double));
    double* ubar = (double*)calloc(3 * (size_t)N, sizeof(double));
    if (!mu || !ubar) {
        free(mu);
        free(ubar);
        return -2;
    }

    /* 1. transpose of streaming + boundaries.  Pull streaming with its
     * boundary links is a permutation of the (direction, node) slots, so each
     * mu slot receives from one node only; a node's ubar receives from itself
     * and, with the extrapolated u_w, from the boundary node of its own row,
     * so rows can be shared among threads.  The inlet terms (several nodes
     * feed the single head) go to gin[n] first and are added in node order
     * afterwards. */
    double* gin = (double*)calloc((size_t)N, sizeof(double));
    if (!gin) {
        free(mu);
        free(ubar);
        return -2;
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                if (is_solid(&D, n)) continue;
                double rho, u[3];
                moments(&L, f_t, N, n, &rho, u);
                /* u_w = k_self u(n) + k_part u(m) (Eq. 6 and set_abb_velocity) */
                long m = (x == 0 || x == nx - 1) ? wall_partner(&D, x, n) : -1;
                double k_self = 1.0, k_part = 0.0;
                if (m >= 0) {
                    double rho_m, u_m[3];
                    moments(&L, f_t, N, m, &rho_m, u_m);
                    for (int a = 0; a < 3; ++a) u[a] = 1.5 * u[a] - 0.5 * u_m[a];
                    k_self = 1.5;
                    k_part = -0.5;
                }
                for (int i = 0; i < q; ++i) {
                    long s = -1;
                    int cls = classify(&D, &L, x, y, z, i, &s);
                    double lam = lam_next[(long)i * N + n];
                    if (cls == LINK_FLUID) {
                        mu[(long)i * N + s] += lam;
                    } else if (cls == LINK_BB || (cls == LINK_ABB_IN && g_vel_inlet)) {
                        mu[(long)L.opp[i] * N + n] += lam;  /* the velocity inlet's source is constant */
                    } else {
                        double rw = cls == LINK_ABB_IN ? inlet_rho(rho_in, inlet_profile, &D, y, z) : *rho_out;
                        mu[(long)L.opp[i] * N + n] -= lam;
                        double cu = dot_cu(&L, i, u), uu = dot_uu(&L, u);
                        if (cls == LINK_ABB_IN) {
                            double d_rw = 2.0 * L.w[i] * (1.0 + cu * cu * INV_2CS4 - uu * INV_2CS2);
                            gin[n] += lam * d_rw;
                        }
                        for (int a = 0; a < L.d; ++a) {
                            double du_w =
                                lam * 2.0 * L.w[i] * rw * (2.0 * INV_2CS4 * cu * L.c[i][a] - 2.0 * INV_2CS2 * u[a]);
                            ubar[(long)a * N + n] += k_self * du_w;
                            if (m >= 0) ubar[(long)a * N + m] += k_part * du_w;
                        }
                    }
                }
            }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                if (gin[n] != 0.0) g_rho_in[inlet_profile ? (long)z * ny + y : 0] += gin[n];
            }
    free(gin);

    /* 2. transpose of collision and of the moments.  Nodes are independent
     * here; each node's term of dL/domega goes to gwn[n] and the terms are
     * summed in node order afterwards, so the thread count changes nothing. */
    double* gwn = (double*)calloc((size_t)N, sizeof(double));
    if (!gwn) {
        free(mu);
        free(ubar);
        return -2;
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (is_solid(&D, n)) {
            for (int k = 0; k < q; ++k) lam_out[(long)k * N + n] = 0;
            continue;
        }
        double gw = 0;
        double rho, u[3];
        moments(&L, f_t, N, n, &rho, u);
        double uu = dot_uu(&L, u);
        double rhobar = 0, ub[3] = {ubar[n], ubar[N + n], ubar[2 * N + n]};
        double nu[19];
        if (g_coll == COLL_MRT && q == 9) {
            /* nu = M^T S D^{-1} M mu; dL/domega from the two stress moments */
            double mm[9], md[9];
            for (int r = 0; r < 9; ++r) {
                mm[r] = md[r] = 0;
                for (int j = 0; j < 9; ++j) {
                    mm[r] += mrt_row(&L, r, j) * mu[(long)j * N + n];
                    md[r] += mrt_row(&L, r, j) * (f_t[(long)j * N + n] - feq(&L, j, rho, u));
                }
            }
            for (int r = 7; r < 9; ++r) gw -= mm[r] * md[r] / mrt_norm2(&L, r);
            for (int j = 0; j < 9; ++j) {
                nu[j] = 0;
                for (int r = 0; r < 9; ++r) nu[j] += mrt_row(&L, r, j) * mrt_rate(r, omega) * mm[r] / mrt_norm2(&L, r);
            }
        } else {
            for (int j = 0; j < q; ++j) {
                double m = mu[(long)j * N + n];
                gw += m * (feq(&L, j, rho, u) - f_t[(long)j * N + n]);
                nu[j] = omega * m;
            }
        }
        for (int j = 0; j < q; ++j) {
            double cu = dot_cu(&L, j, u);
            double P = 1.0 + cu * INV_CS2 + cu * cu * INV_2CS4 - uu * INV_2CS2;
            rhobar += nu[j] * L.w[j] * P;
            for (int a = 0; a < L.d; ++a)
                ub[a] += nu[j] * L.w[j] * rho *
                         (INV_CS2 * L.c[j][a] + 2.0 * INV_2CS4 * cu * L.c[j][a] - 2.0 * INV_2CS2 * u[a]);
        }
        for (int k = 0; k < q; ++k) {
            double s = mu[(long)k * N + n] - nu[k] + rhobar;
            for (int a = 0; a < L.d; ++a) s += ub[a] * ((double)L.c[k][a] - u[a]) / rho;
            lam_out[(long)k * N + n] = s;
        }
        gwn[n] = gw;
    }
    double gw = 0;
    for (long n = 0; n < N; ++n) gw += gwn[n];
    *g_omega += gw;
    free(gwn);
    free(mu);
    free(ubar);
    return 0;
}

/* Full gradient of the final-step loss with respect to rho_in (per entry, or
 * the single head) and tau.  ckpt_stride = 0 keeps every f^t (a full tape);
 * k > 0 keeps every k-th state and recomputes each segment before reversing
 * it.  The two give identical values (recompute repeats the same
 * operations).  f0 = NULL starts from rest.  fT_out (optional) gets f^T. */
int orc_gradient(int q, int nx, int ny, int nz, const uint8_t* mask, const double* rho_in, int inlet_profile,
                 const double* rho_out, const double* tau, int T, const double* f0, const double* u_target,
                 const uint8_t* roi, int loss_kind, int loss_norm, long n_probe, const int64_t* probe_node,
                 const double* probe_rho, double probe_weight, int ckpt_stride, double* loss_out,
                 double* g_rho_in, double* g_tau, double* fT_out)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    long N = (long)nx * ny * nz, QN = (long)q * N;
    int n_in = inlet_profile ? ny * nz : 1;
    int k = ckpt_stride > 0 ? ckpt_stride : (T > 0 ? T : 1);
    int n_seg = T > 0 ? (T + k - 1) / k : 0;
    int rc = 0;

    double* ckpt = (double*)malloc(sizeof(double) * (size_t)QN * (size_t)(n_seg > 0 ? n_seg : 1));
    double* seg = (double*)malloc(sizeof(double) * (size_t)QN * (size_t)k);
    double* a = (double*)malloc(sizeof(double) * (size_t)QN);
    double* b = (double*)malloc(sizeof(double) * (size_t)QN);
    double* lam = (double*)malloc(sizeof(double) * (size_t)QN);
    double* lam2 = (double*)malloc(sizeof(double) * (size_t)QN);
    if (!ckpt || !seg || !a || !b || !lam || !lam2) {
        rc = -2;
        goto done;
    }

    /* forward, keeping f^{s k} for every segment s */
    if (f0)
        memcpy(a, f0, sizeof(double) * (size_t)QN);
    else
        rest_state(&L, N, a);
    for (int t = 0; t < T; ++t) {
        if (t % k == 0) memcpy(ckpt + (long)(t / k) * QN, a, sizeof(double) * (size_t)QN);
        g_time_next = t + 1;
        if ((rc = orc_step(q, nx, ny, nz, mask, a, b, rho_in, inlet_profile, rho_out, tau))) goto done;
        double* tmp = a;
        a = b;
        b = tmp;
    }
    if (fT_out) memcpy(fT_out, a, sizeof(double) * (size_t)QN);

    /* loss and its seed lam^T = dL/df^T */
    if ((rc = orc_loss(q, nx, ny, nz, mask, a, u_target, roi, loss_kind, loss_norm, loss_out, lam))) goto done;
    if (n_probe > 0) {
        double lp = 0;
        if ((rc = orc_probe_loss(q, nx, ny, nz, mask, a, n_probe, probe_node, probe_rho, probe_weight, &lp, lam)))
            goto done;
        *loss_out += lp;
    }

    /* reverse sweep, one segment at a time, last segment first */
    for (int i = 0; i < n_in; ++i) g_rho_in[i] = 0;
    double g_omega = 0;
    for (int s = n_seg - 1; s >= 0; --s) {
        int t0 = s * k, len = (t0 + k <= T) ? k : T - t0;
        memcpy(seg, ckpt + (long)s * QN, sizeof(double) * (size_t)QN);
        for (int j = 1; j < len; ++j) {
            g_time_next = t0 + j;
            if ((rc = orc_step(q, nx, ny, nz, mask, seg + (long)(j - 1) * QN, seg + (long)j * QN, rho_in,
                               inlet_profile, rho_out, tau)))
                goto done;
        }
        for (int j = len - 1; j >= 0; --j) {
            if ((rc = orc_adjoint_step(q, nx, ny, nz, mask, seg + (long)j * QN, lam, lam2, rho_in, inlet_profile,
                                       rho_out, tau, g_rho_in, &g_omega)))
                goto done;
            double* tmp = lam;
            lam = lam2;
            lam2 = tmp;
        }
    }
    /* omega = 1/tau  =>  dL/dtau = -dL/domega / tau^2 */
    *g_tau = -g_omega / ((*tau) * (*tau));

done:
    free(ckpt);
    free(seg);
    free(a);
    free(b);
    free(lam);
    free(lam2);
    return rc;
}

/* A loss over a time window: L = sum_k L_k(f^{t_k}), L_k the final-step
 * loss (loss(): kind, normalisation, ROI) of state f^{t_k} against the k-th
 * target u_targets[k][D N], observation steps 0 <= t_k <= T (the wake of
 * section 3.4 observed over time).  Its gradient with respect to rho_in and
 * tau by one reverse sweep: lam^T = dL/df^T (nonzero if T is observed), and
 * for t = T - 1 .. 0, lam^t = J_t^T lam^{t+1} (adjoint_step), plus dL_k/df^t
 * when t = t_k.  Same checkpoint schedule as orc_gradient. */
int orc_gradient_window(int q, int nx, int ny, int nz, const uint8_t* mask, const double* rho_in, int inlet_profile,
                        const double* rho_out, const double* tau, int T, int n_obs, const int* obs_t,
                        const double* u_targets, const uint8_t* roi, int loss_kind, int loss_norm, int ckpt_stride,
                        double* loss_out, double* g_rho_in, double* g_tau)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    if (T < 1 || n_obs < 1) return -1;
    for (int o = 0; o < n_obs; ++o)
        if (obs_t[o] < 0 || obs_t[o] > T) return -1;
    long N = (long)nx * ny * nz, QN = (long)q * N, DN = (long)L.d * N;
    int n_in = inlet_profile ? ny * nz : 1;
    int k = ckpt_stride > 0 ? ckpt_stride : T;
    int n_seg = (T + k - 1) / k;
    int rc = 0;
    double* ckpt = (double*)malloc(sizeof(double) * (size_t)QN * (size_t)n_seg);
    double* seg = (double*)malloc(sizeof(double) * (size_t)QN * (size_t)k);
    double* a = (double*)malloc(sizeof(double) * (size_t)QN);
    double* b = (double*)malloc(sizeof(double) * (size_t)QN);
    double* lam = (double*)malloc(sizeof(double) * (size_t)QN);
    double* lam2 = (double*)malloc(sizeof(double) * (size_t)QN);
    double* seed = (double*)malloc(sizeof(double) * (size_t)QN);
    if (!ckpt || !seg || !a || !b || !lam || !lam2 || !seed) {
        rc = -2;
        goto done;
    }
    *loss_out = 0.0;
    rest_state(&L, N, a);
    /* forward: checkpoints, and the loss terms of the observed states */
    for (int t = 0; t <= T; ++t) {
        for (int o = 0; o < n_obs; ++o)
            if (obs_t[o] == t) {
                double lk = 0.0;
                if ((rc = orc_loss(q, nx, ny, nz, mask, a, u_targets + (long)o * DN, roi, loss_kind, loss_norm, &lk,
                                   NULL)))
                    goto done;
                *loss_out += lk;
            }
        if (t == T) break;
        if (t % k == 0) memcpy(ckpt + (long)(t / k) * QN, a, sizeof(double) * (size_t)QN);
        g_time_next = t + 1;
        if ((rc = orc_step(q, nx, ny, nz, mask, a, b, rho_in, inlet_profile, rho_out, tau))) goto done;
        double* tmp = a;
        a = b;
        b = tmp;
    }
    /* lam^T: the seeds of the observations at T (a holds f^T) */
    for (long i = 0; i < QN; ++i) lam[i] = 0.0;
    for (int o = 0; o < n_obs; ++o)
        if (obs_t[o] == T) {
            double lk = 0.0;
            if ((rc = orc_loss(q, nx, ny, nz, mask, a, u_targets + (long)o * DN, roi, loss_kind, loss_norm, &lk, seed)))
                goto done;
            for (long i = 0; i < QN; ++i) lam[i] += seed[i];
        }
    /* reverse sweep, one segment at a time, last segment first */
    for (int i = 0; i < n_in; ++i) g_rho_in[i] = 0;
    double g_omega = 0;
    for (int s = n_seg - 1; s >= 0; --s) {
        int t0 = s * k, len = (t0 + k <= T) ? k : T - t0;
        memcpy(seg, ckpt + (long)s * QN, sizeof(double) * (size_t)QN);
        for (int j = 1; j < len; ++j) {
            g_time_next = t0 + j;
            if ((rc = orc_step(q, nx, ny, nz, mask, seg + (long)(j - 1) * QN, seg + (long)j * QN, rho_in,
                               inlet_profile, rho_out, tau)))
                goto done;
        }
        for (int j = len - 1; j >= 0; --j) {
            const double* ft = seg + (long)j * QN; /* f^t, t = t0 + j */
            if ((rc = orc_adjoint_step(q, nx, ny, nz, mask, ft, lam, lam2, rho_in, inlet_profile, rho_out, tau,
                                       g_rho_in, &g_omega)))
                goto done;
            double* tmp = lam;
            lam = lam2;
            lam2 = tmp;
            for (int o = 0; o < n_obs; ++o)
                if (obs_t[o] == t0 + j) {
                    double lk = 0.0;
                    if ((rc = orc_loss(q, nx, ny, nz, mask, ft, u_targets + (long)o * DN, roi, loss_kind, loss_norm,
                                       &lk, seed)))
                        goto done;
                    for (long i = 0; i < QN; ++i) lam[i] += seed[i];
                }
        }
    }
    *g_tau = -g_omega / ((*tau) * (*tau));

done:
    free(ckpt);
    free(seg);
    free(a);
    free(b);
    free(lam);
    free(lam2);
    free(seed);
    return rc;
}

/* --------------------------------------------------------------- Adam */

/* One Adam step (Kingma & Ba), the optimiser the paper uses (section 2.2,
 * section 3.4).  t is the 1-based step count. */
void orc_adam(int n, double* theta, const double* grad, double* m, double* v, int t, double lr, double beta1,
              double beta2, double eps)
{
    double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
    for (int i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        theta[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ---------------------------------------------------------- permeability */

/* Darcy permeability (Eq. 12) from a steady state f: k = rho nu U / (dp/dx)
 * with the superficial mass flux J = sum over the cross-section x = xs of
 * rho u_x (solid nodes count as zero flux) divided by the section area
 * standing for rho_fluid U, nu = c_s^2 (tau - 1/2) (Eq. 9), and
 * dp/dx = c_s^2 (mean(rho_in) - rho_out) / nx (pressure planes at x = -1/2
 * and nx - 1/2).  Also returns the porosity of the mask. */
int orc_darcy(int q, int nx, int ny, int nz, const uint8_t* mask, const double* f, const double* rho_in,
              int inlet_profile, double rho_out, double tau, int xs, double* k_out, double* flux_out)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    domain D = {nx, ny, nz, (long)nx * ny * nz, mask};
    long N = D.n;
    double J = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            long n = ((long)z * ny + y) * nx + xs;
            if (is_solid(&D, n)) continue;
            double rho, u[3];
            moments(&L, f, N, n, &rho, u);
            J += rho * u[0];
        }
    J /= (double)ny * (double)nz;
    int n_in = inlet_profile ? ny * nz : 1;
    double rin = 0;
    for (int i = 0; i < n_in; ++i) rin += rho_in[i];
    rin /= (double)n_in;
    double cs2 = 1.0 / INV_CS2;
    double nu = cs2 * (tau - 0.5);
    double dpdx = cs2 * (rin - rho_out) / (double)nx;
    *k_out = nu * J / dpdx;
    if (flux_out) *flux_out = J;
    return 0;
}
#endif /* !ORC_COMPLEX */
